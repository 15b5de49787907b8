// The coarsest operator's row kernels with the operator streamed through
// shared memory by bulk asynchronous copies (the Tensor Memory Accelerator's
// 1-D copy, cp.async.bulk, completing on an mbarrier).
//
// The coarse Newton steps (Sec. 2.3) stream the whole coarsest operator once
// per step; it has long rows (~360 entries on the 4096^2 workload) and is
// larger than L2.  In the row kernels of solve.cu each warp issues its own
// loads and waits for them before its gathers of x, so the memory pipeline
// drains at every step of a lane's sequence.  Here one producer warp per
// block streams chunks of a slice (COLS entry columns: the values and the
// 16-bit column indices, both contiguous in SELL order) into a ring of
// STAGES shared-memory stages, and eight consumer warps compute from
// shared memory while the next chunks are in flight.  Blocks are resident
// (as many as fit) and take the slices in a strided loop.
//
// The arithmetic is that of the K = 8 long-row kernels: warp p of a slice
// takes entry columns p, p + 8, ..., a lane's j-th entry goes to partial sum
// j mod 4, the result is (a0 + a1) + (a2 + a3), the parts are added in order
// in part 0, then the dense diagonal.  Results are bit-identical.
//
// Every wait on an mbarrier is bounded (CS_SPIN polls); a wait that gives up
// sets the error word the solve reads after each call (AIRG_ERR_TIMEOUT) and
// the block goes on.  Before a block exits its producer waits, bounded again,
// for the last fill of every stage, so no copy is in flight into the shared
// memory of a finished block.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>

#include "dev_util.cuh"
#include "solve_internal.cuh"

namespace airg {

namespace {

constexpr int CS_PARTS = 8;                       // consumer warps = parts of a slice
constexpr int CS_THREADS = 32 * (CS_PARTS + 1);   // + one producer warp
// chunks of COLS entry columns (a multiple of 32) in a ring of STAGES
// stages: 64 x 4 by default, 32 x 3 with AIRG_COARSE_STREAM_COLS=32 (less
// shared memory per block, more resident blocks)
constexpr long long CS_SPIN = 1LL << 22;          // polls of one bounded wait

template <class T, int COLS>
struct CsStage {
    T val[COLS * 32];
    unsigned short col[COLS * 32];
};

template <class T, int COLS, int STAGES>
struct CsShared {
    CsStage<T, COLS> st[STAGES];
    unsigned long long full[STAGES];
    unsigned long long empty[STAGES];
    T red[CS_PARTS][32];
};

__device__ __forceinline__ unsigned smem_addr(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, unsigned* err)
{
    for (long long i = 0; i < CS_SPIN; ++i) {
        if (mbar_try_wait(b, parity)) return true;
        if (*(volatile unsigned*)err) return false;
    }
    atomicExch(err, 1u);
    return false;
}

// size bytes from global src to shared dst (both 16-byte aligned, size a
// multiple of 16), completing on mbarrier b
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned size, unsigned long long* b)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(size), "r"(smem_addr(b))
        : "memory");
}

__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(32 * CS_PARTS) : "memory"); }

// KIND (solve_internal.cuh): CS_SPMV out = A x;  CS_REAL x_acc += r a,
// out = r - (A r) a;  CS_PAIR1 t = a r - A r (out), x_acc += t b;
// CS_PAIR2 out = aux - (A t) b.
template <class T, int KIND, int COLS, int STAGES>
__global__ void __launch_bounds__(CS_THREADS)
k_coarse_stream(SellView<T> A, const T* __restrict__ xin, const T* __restrict__ aux, T* __restrict__ out,
                T* __restrict__ xacc, T sa, T sb, int first, unsigned* err)
{
    extern __shared__ __align__(128) unsigned char cs_raw[];
    CsShared<T, COLS, STAGES>& sm = *reinterpret_cast<CsShared<T, COLS, STAGES>*>(cs_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], CS_PARTS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == CS_PARTS) {
        // producer: lane 0 streams every chunk of this block's slices
        if (lane != 0) return;
        long long g = 0;
        for (int s = blockIdx.x; s < A.n_slices; s += gridDim.x) {
            const int b = __ldg(A.sptr + s);
            const int w = (__ldg(A.sptr + s + 1) - b) >> 5;
            for (int c0 = 0; c0 < w; c0 += COLS, ++g) {
                const int stg = int(g % STAGES);
                const long long u = g / STAGES;
                if (u > 0) mbar_wait(&sm.empty[stg], unsigned((u - 1) & 1), err);
                const int cols = min(COLS, w - c0);
                const unsigned vb = unsigned(cols) * 32u * unsigned(sizeof(T));
                const unsigned cb = unsigned(cols) * 32u * 2u;
                mbar_expect_tx(&sm.full[stg], vb + cb);
                const long long off = (long long)b + 32LL * c0;
                bulk_copy(sm.st[stg].val, A.val + off, vb, &sm.full[stg]);
                bulk_copy(sm.st[stg].col, A.col16 + off, cb, &sm.full[stg]);
            }
        }
        // drain: the last fill of each stage has completed before the block exits
        for (long long h = g - 1; h >= 0 && h >= g - STAGES; --h)
            mbar_wait(&sm.full[h % STAGES], unsigned((h / STAGES) & 1), err);
        return;
    }
    // consumers: warp = part of the slice, lane = row of the slice
    const int part = warp;
    long long g = 0;
    for (int s = blockIdx.x; s < A.n_slices; s += gridDim.x) {
        const int b = __ldg(A.sptr + s);
        const int w = (__ldg(A.sptr + s + 1) - b) >> 5;
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
        for (int c0 = 0; c0 < w; c0 += COLS, ++g) {
            const int stg = int(g % STAGES);
            mbar_wait(&sm.full[stg], unsigned((g / STAGES) & 1), err);
            const int cols = min(COLS, w - c0);
            const T* sv = sm.st[stg].val;
            const unsigned short* sc = sm.st[stg].col;
            // columns part + 8 q of the chunk; the chunk starts at a multiple
            // of 32 columns, so entry q of the chunk goes to partial q mod 4
            int k = part;
            for (; k + 24 < cols; k += 32) {
                const int e = k * 32 + lane;
                const T v0 = sv[e], v1 = sv[e + 256], v2 = sv[e + 512], v3 = sv[e + 768];
                const int c0i = sc[e], c1i = sc[e + 256], c2i = sc[e + 512], c3i = sc[e + 768];
                a0 = fma(v0, __ldg(xin + c0i), a0);
                a1 = fma(v1, __ldg(xin + c1i), a1);
                a2 = fma(v2, __ldg(xin + c2i), a2);
                a3 = fma(v3, __ldg(xin + c3i), a3);
            }
            if (k < cols) a0 = fma(sv[k * 32 + lane], __ldg(xin + sc[k * 32 + lane]), a0);
            if (k + 8 < cols) a1 = fma(sv[(k + 8) * 32 + lane], __ldg(xin + sc[(k + 8) * 32 + lane]), a1);
            if (k + 16 < cols) a2 = fma(sv[(k + 16) * 32 + lane], __ldg(xin + sc[(k + 16) * 32 + lane]), a2);
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.empty[stg]);
        }
        T acc = (a0 + a1) + (a2 + a3);
        sm.red[part][lane] = acc;
        consumers_sync();
        if (part == 0) {
#pragma unroll
            for (int q = 1; q < CS_PARTS; ++q) acc += sm.red[q][lane];
            const int r = s * 32 + lane;
            if (r < A.n_rows) {
                if (A.diag) acc = fma(__ldg(A.diag + r), __ldg(xin + r), acc);
                if constexpr (KIND == CS_SPMV) {
                    out[r] = acc;
                } else if constexpr (KIND == CS_REAL) {
                    const T ra = __ldg(xin + r), xb = first ? T(0) : xacc[r];
                    xacc[r] = fma(ra, sa, xb);
                    out[r] = ra - acc * sa;
                } else if constexpr (KIND == CS_PAIR1) {
                    const T ra = __ldg(xin + r), xb = first ? T(0) : xacc[r];
                    T tt = sa * ra - acc;
                    out[r] = tt;
                    xacc[r] = fma(tt, sb, xb);
                } else {
                    out[r] = __ldg(aux + r) - acc * sb;
                }
            }
        }
        consumers_sync();
    }
}

template <class T, int KIND, int COLS, int STAGES>
void launch_cfg(const Sell<T>& A, const T* xin, const T* aux, T* out, T* xacc, T sa, T sb, int first,
                unsigned* err, cudaStream_t st)
{
    static int grid = 0;   // resident blocks of this instantiation (set once)
    const size_t smem = sizeof(CsShared<T, COLS, STAGES>);
    if (!grid) {
        CK(cudaFuncSetAttribute(k_coarse_stream<T, KIND, COLS, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(smem)));
        int dev = 0, sms = 0, per = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_coarse_stream<T, KIND, COLS, STAGES>, CS_THREADS,
                                                         smem));
        grid = std::max(1, per * sms);
    }
    const int g = std::max(1, std::min(grid, A.n_slices));
    k_coarse_stream<T, KIND, COLS, STAGES><<<g, CS_THREADS, smem, st>>>(view(A), xin, aux, out, xacc, sa, sb, first,
                                                                        err);
    CK_LAUNCH();
}

template <class T, int KIND>
void launch_kind(const Sell<T>& A, const T* xin, const T* aux, T* out, T* xacc, T sa, T sb, int first,
                 unsigned* err, cudaStream_t st)
{
    static int cols = -1;
    if (cols < 0) {
        const char* e = getenv("AIRG_COARSE_STREAM_COLS");
        cols = e && atoi(e) == 32 ? 32 : 64;
    }
    if (cols == 32) launch_cfg<T, KIND, 32, 3>(A, xin, aux, out, xacc, sa, sb, first, err, st);
    else launch_cfg<T, KIND, 64, 4>(A, xin, aux, out, xacc, sa, sb, first, err, st);
}

}  // namespace

template <class T>
bool coarse_stream_ok(const Sell<T>& A)
{
    // the layout the stream kernel reproduces: 8 parts per slice, 16-bit
    // columns; the copies start at multiples of 32 entries, so every source
    // address is 64-byte aligned (cudaMalloc bases are 256-byte aligned)
    return A.k == CS_PARTS && A.col16.n && !A.cbase.n && A.n_slices > 0 && A.padded % 32 == 0;
}

template <class T>
void coarse_stream_launch(const Sell<T>& A, int kind, const T* xin, const T* aux, T* out, T* xacc, T sa, T sb,
                          int first, unsigned* err, cudaStream_t st)
{
    switch (kind) {
        case CS_SPMV: launch_kind<T, CS_SPMV>(A, xin, aux, out, xacc, sa, sb, first, err, st); break;
        case CS_REAL: launch_kind<T, CS_REAL>(A, xin, aux, out, xacc, sa, sb, first, err, st); break;
        case CS_PAIR1: launch_kind<T, CS_PAIR1>(A, xin, aux, out, xacc, sa, sb, first, err, st); break;
        default: launch_kind<T, CS_PAIR2>(A, xin, aux, out, xacc, sa, sb, first, err, st); break;
    }
}

template bool coarse_stream_ok<double>(const Sell<double>&);
template bool coarse_stream_ok<float>(const Sell<float>&);
template void coarse_stream_launch<double>(const Sell<double>&, int, const double*, const double*, double*,
                                           double*, double, double, int, unsigned*, cudaStream_t);
template void coarse_stream_launch<float>(const Sell<float>&, int, const float*, const float*, float*, float*,
                                          float, float, int, unsigned*, cudaStream_t);

}  // namespace airg
