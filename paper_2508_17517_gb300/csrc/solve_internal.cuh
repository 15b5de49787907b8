// Solve-phase data structures shared by solve.cu (single right-hand side)
// and batch.cu (many right-hand sides in lockstep): SELL-32 operators, the
// per-level operators of the nested F/C layout, work buffers, the launch
// counter / profiler and the captured V-cycle graphs.
#pragma once

#include <cuda_runtime.h>

#include <cstdlib>
#include <memory>
#include <string>
#include <vector>

#include "dev_util.cuh"
#include "handle.h"

namespace airg {

struct BatchData;   // batch.cu

enum { PK_RESTRICT = 0, PK_FRESID = 1, PK_HORNER = 2, PK_NEWTON = 3, PK_TOPSPMV = 4, PK_KRYLOV = 5,
       PK_LAYOUT = 6, PROF_KINDS = 7 };

// A solve-phase operator in SELL-32: slices of 32 consecutive rows, entries
// column-major inside a slice (entry k of the slice's 32 rows are adjacent),
// each slice padded to its longest row (padding: value 0, column repeated).
// Lane l of a warp always owns row 32s+l, so at a given entry index the 32
// lanes read adjacent values and columns, and -- rows of these operators
// having similar stencils -- gather nearby entries of x.  k = number of
// warps sharing a slice: for long rows the entries of a slice are split
// among k warps of a block (entry indices interleaved) whose partial sums
// meet in shared memory.  For short rows (k = 1) a warp instead handles r
// consecutive slices (r = 1, 2 or 4, picked per operator by timing in the
// setup) so that each lane keeps r rows' loads in flight.
//
// Square operators keep their diagonal as a dense vector `diag` (read and
// multiplied with coalesced loads, no column index) and only the
// off-diagonal entries in the slices; ndiag counts the diagonal entries
// split out this way (0 when there is no split).
// FP32 V-cycle (with FP32 or bfloat16 restrictor values)
inline bool mixed_precision(const airg_options& o)
{
    return o.precision == AIRG_MIXED_FP32 || o.precision == AIRG_MIXED_FP32_BF16R;
}

// Stored values may be narrower than the arithmetic type T: V = bf16s keeps
// bfloat16 values (the upper 16 bits of an FP32 number), widened exactly to
// FP32 when loaded.
struct bf16s {
    unsigned short bits;
};

//
// col16: the same column indices in 16 bits, read by the single-vector row
// kernels (2 instead of 4 bytes of index per entry): with at most 65536
// columns the index itself (cbase empty), else its offset from the
// slice's smallest column, cbase[s], where every slice of the operator
// spans at most 65536 columns.  `col` stays for the kernels that do not
// read col16 (batched, many-grid work list, staged coarse forms).
template <class T, class V = T>
struct Sell {
    int n_rows = 0, n_cols = 0, n_slices = 0, k = 1, r = 1;
    int persist = 0;   // 1: row kernels run on a grid of resident blocks that stride over the slices
    int stream = 0;    // coarsest operator only: 1 = its steps stream it through shared memory (coarse_stream.cu)
    int xs = 0;   // coarsest operator only: > 0 = its SpMVs stage x in shared memory, on xs blocks (solve.cu)
    long long nnz = 0, padded = 0, ndiag = 0;
    DBuf<int> sptr;
    DBuf<int> col;
    DBuf<unsigned short> col16;
    DBuf<int> cbase;
    DBuf<V> val;
    DBuf<T> diag;
};

template <class T, class V = T>
struct SellView {
    int n_rows, n_slices;
    const int* __restrict__ sptr;
    const int* __restrict__ col;
    const V* __restrict__ val;
    const T* __restrict__ diag;   // nullptr: no diagonal split
    const unsigned short* __restrict__ col16;   // nullptr: none
    const int* __restrict__ cbase;              // nullptr: col16 holds the columns themselves
};

template <class T, class V>
SellView<T, V> view(const Sell<T, V>& s)
{
    return SellView<T, V>{s.n_rows, s.n_slices, s.sptr.p, s.col.p, s.val.p, s.ndiag ? s.diag.p : nullptr,
                          s.col16.n ? s.col16.p : nullptr, s.cbase.n ? s.cbase.p : nullptr};
}

// stored value -> arithmetic type
template <class T, class V>
__device__ __forceinline__ T ldval(const V* p)
{
    return T(__ldg(p));
}
template <>
__device__ __forceinline__ float ldval<float, bf16s>(const bf16s* p)
{
    return __uint_as_float(unsigned(__ldg(reinterpret_cast<const unsigned short*>(p))) << 16);
}
template <>
__device__ __forceinline__ double ldval<double, bf16s>(const bf16s* p)
{
    return double(ldval<float, bf16s>(p));
}

// algorithmic bytes of the stored entries: value + column index per entry
// (2 bytes when the row kernels read col16, else 4), value only for a
// diagonal held densely; plus the slice bases the row kernels then read
template <class T, class V>
long long mat_bytes(const Sell<T, V>& s)
{
    return (s.nnz - s.ndiag) * (long long)(sizeof(V) + (s.col16.n ? 2 : 4)) + s.ndiag * (long long)sizeof(T) +
           4LL * (long long)s.cbase.n;
}
// the same for kernels that read the 32-bit columns (batched, work list)
template <class T, class V>
long long mat_bytes32(const Sell<T, V>& s)
{
    return (s.nnz - s.ndiag) * (long long)(sizeof(V) + 4) + s.ndiag * (long long)sizeof(T);
}

// Warps per slice from the mean row length: the smallest power of two that
// leaves at most `per_lane` entries per lane (default 12), capped at
// `max_parts` (default 8).  Both can be overridden for tuning with
// AIRG_PER_LANE / AIRG_MAX_PARTS.
inline int choose_parts(long long nnz, int n_rows)
{
    static int max_parts = 0, per_lane = 0;
    if (!max_parts) {
        const char* e = getenv("AIRG_MAX_PARTS");
        max_parts = e ? std::max(1, std::min(32, atoi(e))) : 8;
        const char* q = getenv("AIRG_PER_LANE");
        per_lane = q ? std::max(1, atoi(q)) : 12;
    }
    double avg = n_rows ? double(nnz) / n_rows : 0.0;
    int p = 1;
    while (p < max_parts && avg > double(per_lane) * p) p *= 2;
    return p;
}

// Direction of the i-th of a chain of SpMVs with one operator: even steps
// forward, odd steps reversed (serpentine order), so that each step starts
// on the end of the operator that the previous step read last and that is
// most likely still in L2.  Each row is computed the same way in either
// direction.  AIRG_SERPENTINE=0 keeps every step forward.
inline int serpentine(int i)
{
    const char* e = getenv("AIRG_SERPENTINE");
    return (e && e[0] == '0') ? 0 : (i & 1);
}

// warps per block for P warps per slice (blocks of at least 8 warps)
__host__ __device__ constexpr int wpb_for(int P) { return P > 8 ? P : 8; }

template <class T>
struct SolveLevelT {
    Sell<T> Z, M, Aff;
    Sell<T, bf16s> Zb;   // Z with bfloat16 values (precision AIRG_MIXED_FP32_BF16R)
    Sell<T> Ainv;        // assembled Ahat_ff^-1 (smoother AIRG_SMOOTH_ASSEMBLED)
    // C-point smoothing: the C rows [A_cf A_cc] and (FCF) the F rows
    // [A_ff A_fc] of A_l over the level's nested positions, and A_cc over
    // the next level's
    Sell<T> Mc, Acc, Mf;
    Sell<T> Ainvc;       // assembled Ahat_cc^-1 (C-point smoothing, AIRG_SMOOTH_ASSEMBLED)
};

struct SolveLevel {
    int off = 0, n_f = 0, n_c = 0;
    long long rc_off = 0;        // start of this level's saved C residual (C-point smoothing)
    DBuf<int> W;                 // nested-relative C position, -1 none
    std::vector<double> alpha;
    std::vector<double> alpha_c;     // C-point smoother polynomial (empty: none)
    SolveLevelT<double> d;
    SolveLevelT<float> f;
};

struct SolveData {
    int n0 = 0, nlev = 0, off_c = 0, n_coarse = 0;
    DBuf<int> pos0;              // natural index -> nested position (top level)
    Sell<double> Atop;
    std::vector<std::unique_ptr<SolveLevel>> lv;
    Sell<double> Ac;
    Sell<float> Ac32;
    std::vector<Root> roots;
    // persistent coarse polynomial: CSR copies, roots on the device, barrier
    DBuf<double> roots_dev;
    DBuf<unsigned> bar;          // [count, generation, error flag]
    DBuf<unsigned> ticket;       // last-block ticket of the dot kernels
    int newton_grid[2] = {0, 0}; // per precision (0: FP64, 1: FP32); 0 = not usable
    int smooth_grid[2] = {0, 0}; // co-resident blocks of the persistent smoother
    int max_nf = 0, max_nc = 0;  // largest F block; largest C block with C-point smoothing
    long long rc_total = 0;      // rows of all saved C residuals (C-point smoothing)
    // V-cycle work (FP64 and FP32 copies)
    DBuf<double> rwork, t, wa, wb, cx, cr0, cr1, ct;
    DBuf<float> rwork32, e32, t32, wa32, wb32, cx32, cr032, cr132, ct32, vin32;
    int smooth_type = 0;         // AIRG_SMOOTH_F, _FC or _FCF
    DBuf<double> rcs;            // C residuals before restriction, one slot per level l >= 1
                                 // (nested C blocks overlap, so they cannot share positions)
    DBuf<float> rcs32;
    // outer FGMRES
    int restart = 0;
    DBuf<double> V, Zs, w, bp, xp, r, part;
    DBuf<double> hdev;
    HBuf<double> hhost;
    long long bytes_vcycle = 0;
    std::shared_ptr<BatchData> batch;   // work space of the many-RHS solve (batch.cu)
    DBuf<double> stage_b, stage_x;      // device copies of host b and x, kept between calls
    // launch count and optional per-kind CUDA-event timing of the solve kernels
    long long launches = 0;
    bool prof = false;
    // Group timing: with prof_kind >= 0 only the launches of kind prof_kind
    // on level prof_level are timed.  Consecutive V-cycle launches of that
    // group (a run, e.g. the whole chain of coarse Newton steps) share one
    // event pair, so the timed step carries two event records per V-cycle
    // instead of two per kernel.
    int prof_kind = -1, prof_level = -1;
    bool run_open = false;
    cudaEvent_t run_a = nullptr;
    int run_level = 0;
    long long run_bytes = 0, run_flops = 0, run_n = 0;
    struct Rec { int kind, level; cudaEvent_t a, b; long long bytes, flops, n; };
    int cur_level = 0;           // level of the kernels being launched (coarsest = nlev)
    std::vector<cudaEvent_t> evpool;
    size_t evnext = 0;
    std::vector<Rec> recs;
    std::vector<cudaGraphExec_t> prof_execs;   // profiled V-cycle graphs awaiting collect()
    static constexpr int PROF_LEVELS = 65;
    double kind_ms[PROF_KINDS] = {};
    long long kind_launches[PROF_KINDS] = {}, kind_bytes[PROF_KINDS] = {};
    double lev_ms[PROF_KINDS][PROF_LEVELS] = {};
    long long lev_launches[PROF_KINDS][PROF_LEVELS] = {}, lev_bytes[PROF_KINDS][PROF_LEVELS] = {};
    long long lev_flops[PROF_KINDS][PROF_LEVELS] = {};
    cudaEvent_t next_event()
    {
        if (evnext == evpool.size()) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            evpool.push_back(e);
        }
        return evpool[evnext++];
    }
    // inside a stream capture an event record becomes a timing node of the
    // graph only with cudaEventRecordExternal
    static void record(cudaEvent_t e, cudaStream_t st)
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CK(cudaStreamIsCapturing(st, &cs));
        if (cs == cudaStreamCaptureStatusActive) CK(cudaEventRecordWithFlags(e, st, cudaEventRecordExternal));
        else CK(cudaEventRecord(e, st));
    }
    int prof_lvl() const { return cur_level < 0 ? 0 : (cur_level >= PROF_LEVELS ? PROF_LEVELS - 1 : cur_level); }
    bool timed(int kind) const { return prof_kind < 0 || (kind == prof_kind && prof_lvl() == prof_level); }
    // V-cycle kinds run back to back inside one V-cycle: their runs merge
    static bool merges(int kind) { return kind <= PK_NEWTON; }
    // ends an open run of the timed group at the current point of the stream
    void close_run(cudaStream_t st)
    {
        if (!run_open) return;
        cudaEvent_t b = next_event();
        record(b, st);
        recs.push_back(Rec{prof_kind, run_level, run_a, b, run_bytes, run_flops, run_n});
        run_open = false;
    }
    void begin(cudaStream_t st, cudaEvent_t& a, int kind)
    {
        ++launches;
        if (!prof) return;
        if (prof_kind >= 0 && !timed(kind)) { close_run(st); return; }
        if (prof_kind >= 0 && merges(kind)) {
            if (!run_open) {
                run_a = next_event();
                record(run_a, st);
                run_open = true;
                run_level = prof_lvl();
                run_bytes = run_flops = run_n = 0;
            }
            return;
        }
        a = next_event();
        record(a, st);
    }
    void end(int kind, long long bytes, long long flops, cudaStream_t st, cudaEvent_t a)
    {
        if (!prof || !timed(kind)) return;
        if (prof_kind >= 0 && merges(kind)) {
            run_bytes += bytes;
            run_flops += flops;
            ++run_n;
            return;
        }
        cudaEvent_t b = next_event();
        record(b, st);
        recs.push_back(Rec{kind, prof_lvl(), a, b, bytes, flops, 1});
    }
    // after the stream has been synchronised
    void collect()
    {
        for (const Rec& r : recs) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, r.a, r.b));
            kind_ms[r.kind] += ms;
            kind_launches[r.kind] += r.n;
            kind_bytes[r.kind] += r.bytes;
            lev_ms[r.kind][r.level] += ms;
            lev_launches[r.kind][r.level] += r.n;
            lev_bytes[r.kind][r.level] += r.bytes;
            lev_flops[r.kind][r.level] += r.flops;
        }
        recs.clear();
        evnext = 0;
        for (cudaGraphExec_t e : prof_execs) cudaGraphExecDestroy(e);
        prof_execs.clear();
    }
    // private stream (capturable, unlike the legacy default stream) and the
    // V-cycle graphs, one per (input, output) pair = FGMRES basis slot
    cudaStream_t sst = nullptr;
    cudaEvent_t ev_in = nullptr;
    bool use_graphs = true;
    struct GEntry { const void* v; void* z; cudaGraphExec_t exec; long long kernels; };
    std::vector<GEntry> graphs;
    ~SolveData()
    {
        for (cudaEvent_t e : evpool) cudaEventDestroy(e);
        for (GEntry& g : graphs) cudaGraphExecDestroy(g.exec);
        for (cudaGraphExec_t e : prof_execs) cudaGraphExecDestroy(e);
        if (ev_in) cudaEventDestroy(ev_in);
        if (sst) cudaStreamDestroy(sst);
    }
};

// Runs the statement with the compile-time constant MM = mv (1..16).
#define WITH_M(mv, ...)                                                         \
    do {                                                                        \
        switch (mv) {                                                           \
            case 1: { constexpr int MM = 1; __VA_ARGS__; } break;               \
            case 2: { constexpr int MM = 2; __VA_ARGS__; } break;               \
            case 3: { constexpr int MM = 3; __VA_ARGS__; } break;               \
            case 4: { constexpr int MM = 4; __VA_ARGS__; } break;               \
            case 5: { constexpr int MM = 5; __VA_ARGS__; } break;               \
            case 6: { constexpr int MM = 6; __VA_ARGS__; } break;               \
            case 7: { constexpr int MM = 7; __VA_ARGS__; } break;               \
            case 8: { constexpr int MM = 8; __VA_ARGS__; } break;               \
            case 9: { constexpr int MM = 9; __VA_ARGS__; } break;               \
            case 10: { constexpr int MM = 10; __VA_ARGS__; } break;             \
            case 11: { constexpr int MM = 11; __VA_ARGS__; } break;             \
            case 12: { constexpr int MM = 12; __VA_ARGS__; } break;             \
            case 13: { constexpr int MM = 13; __VA_ARGS__; } break;             \
            case 14: { constexpr int MM = 14; __VA_ARGS__; } break;             \
            case 15: { constexpr int MM = 15; __VA_ARGS__; } break;             \
            case 16: { constexpr int MM = 16; __VA_ARGS__; } break;             \
            default: fail(AIRG_ERR_STATE, "bad basis chunk");                   \
        }                                                                       \
    } while (0)

// Launch through the counter / profiler:
//   LAUNCH_F(S, kind, algorithmic bytes, floating-point operations, kernel<<<...>>>(...))
// (an FMA counts as two operations); LAUNCH for kernels that only move data.
#define LAUNCH_F(S, KIND, BYTES, FLOPS, ...)         \
    do {                                             \
        cudaEvent_t ev_a_ = nullptr;                 \
        (S).begin(st, ev_a_, (KIND));                \
        __VA_ARGS__;                                 \
        (S).end((KIND), (BYTES), (FLOPS), st, ev_a_); \
    } while (0)
#define LAUNCH(S, KIND, BYTES, ...) LAUNCH_F(S, KIND, BYTES, 0LL, __VA_ARGS__)


// coarse_stream.cu: the coarsest operator's steps with the operator
// streamed through shared memory by bulk asynchronous copies, for a long-row
// operator of 8 warps per slice with 16-bit columns (coarse_stream_ok);
// bit-identical to the K = 8 row kernels.  err: error word set when a
// bounded wait gives up.
enum { CS_SPMV = 0, CS_REAL = 1, CS_PAIR1 = 2, CS_PAIR2 = 3 };
template <class T>
bool coarse_stream_ok(const Sell<T>& A);
template <class T>
void coarse_stream_launch(const Sell<T>& A, int kind, const T* xin, const T* aux, T* out, T* xacc, T sa, T sb,
                          int first, unsigned* err, cudaStream_t st);

// solve.cu: launch helpers of one problem's solve, for the multi-problem
// solver (multi.cu); all launch on `st` and use the problem's own buffers
void mp_vcycle(Hierarchy& H, const double* v, double* z, cudaStream_t st);
void mp_top_spmv(Hierarchy& H, const double* x, double* y, cudaStream_t st);
void mp_multidot(Hierarchy& H, int m, const double* V, const double* w, double* out, int selfdot,
                 cudaStream_t st);
void mp_multiaxpy_norm(Hierarchy& H, int m, const double* V, const double* h, double* w, double* out,
                       cudaStream_t st);
void mp_scale_dev(Hierarchy& H, const double* w, const double* nrm2, const int* active, double* v,
                  cudaStream_t st);
void mp_residual(Hierarchy& H, const double* b, const double* x, double* y, double* r, cudaStream_t st);
void mp_update(Hierarchy& H, int m, const double* Zs, const double* y, double* x, cudaStream_t st);
void mp_permute(Hierarchy& H, const double* a, double* b, bool to_nested, cudaStream_t st);
void mp_add_dev(Hierarchy& H, const double* z, const int* active, double* x, cudaStream_t st);

// batch.cu: k right-hand sides in lockstep (k <= batch_max_width())
void solve_batched(Hierarchy& H, int k, const double* b, double* x, double rtol, double atol,
                   int maxit, airg_solve_info& info, cudaStream_t st);
int batch_max_width();

}  // namespace airg
