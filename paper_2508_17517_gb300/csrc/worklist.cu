// Many separate problems in one persistent launch per FGMRES iteration.
//
// Each problem's part of a lockstep iteration is a chain of row-parallel
// operations (scale v_j; the V-cycle: restriction per level, the coarse
// Newton steps, the F-point residual and Horner terms per level; w = A z_j;
// the Gram-Schmidt dots and update, each followed by a one-tile fixed-order
// sum of its partials).  Operations are cut into tiles of consecutive SELL
// slices (or rows).  The tiles of all problems are queued by the share of
// its problem's work that comes before each operation, so that all problems
// advance at the same relative pace, and the blocks of one kernel take them
// in queue order with one atomic counter.  A tile starts
// once every tile of the operation before it in its problem's chain has
// finished (a completion counter per operation).  A block only waits on
// tiles queued before its own, which blocks that are already running hold,
// so the earliest unfinished tile can always proceed: the list cannot
// deadlock, whatever the number of resident blocks.  The wait is bounded
// all the same: after WL_SPIN_LIMIT polls it records an error flag (the
// host reports AIRG_ERR_TIMEOUT) and the block goes on.
//
// Per row the arithmetic is that of the per-operator kernels of solve.cu
// for the same operator layout (warps per slice), so the V-cycle gives the
// same bits as in the graph form; the Gram-Schmidt sums use their own tile
// partition.  Vectors written inside the launch are read with plain loads
// after the acquiring fence (never through the read-only cache); operator
// arrays, which no launch writes, use it.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "dev_util.cuh"
#include "handle.h"
#include "solve_internal.cuh"
#include "worklist.h"

namespace airg {

namespace {

enum WKind : int {
    W_RESTRICT = 0,   // dst = src_c + Z src_f
    W_FRESID,         // t = r_f - M e_c, w = a t
    W_HORNER,         // out = a t + A win
    W_HORNER_LAST,    // e_f = W e_c + (a t + A win)
    W_SMOOTH0,        // e_f = W e_c + a t
    W_NEWTON_REAL,    // x += r a, r' = r - (A r) a
    W_NEWTON_LAST,    // x += r a
    W_PAIR1,          // t = a r - A r, x += t b
    W_PAIR2,          // r' = r - (A t) b
    W_ZERO,           // x = 0
    W_SPMV,           // y = A x
    W_D2F,            // FP64 -> FP32
    W_F2D,            // FP32 -> FP64
    W_SCALE,          // v = w / sqrt(nrm2) if active, else 0
    W_DOT,            // partials of <V_i, w> (i < m) and <w, w>
    W_DOT_FIN,        // their sums, in tile order
    W_AXPY,           // w -= V h (i < m), partials of ||w||^2
    W_AXPY_FIN        // its sum, in tile order
};

struct WOp {
    long long bytes;   // algorithmic bytes (host bookkeeping only)
    int kind;
    int fp32;          // operator values and vectors in FP32
    int K;             // warps per SELL slice
    int n;             // rows (vector length); W_*_FIN: tiles of the summed op
    int n_slices;
    int tiles;
    int unit;          // slices (SELL ops) or rows per tile
    int prev;          // op that must finish first (-1: none)
    int m;             // W_DOT / W_AXPY / W_*_FIN: basis vectors
    int first;         // Newton steps: first root (x starts at 0)
    const int* sptr;
    const int* col;
    const void* val;
    const void* diag;
    const void* in;    // SELL ops: the gathered input
    const void* in2;
    const void* in3;
    void* out;
    void* out2;
    const int* W;
    const int* active; // null: always run; else skip the work when *active == 0
    double a, b;
    double* part;      // partial sums (W_DOT, W_AXPY and their sums)
    long long ld;      // basis vector stride
};

constexpr int WL_THREADS = 256;
constexpr int WL_WARPS = WL_THREADS / 32;
constexpr long long WL_SPIN_LIMIT = 20000000;   // ~1 s of polls
constexpr int WL_GROUPS = 4;                    // block-groups of slices per tile (long rows)
constexpr int WL_SHORT_SLICES = 64;             // slices per tile (short rows: 2 per warp, 4 times)
constexpr int WL_VEC_UNIT = 2048;               // rows per tile of a vector op
constexpr int WL_MAX_DOT_TILES = 1024;          // partial sums per reduction
constexpr int WL_DOT_CHUNK = 8;                 // basis vectors per pass of a dot tile

// Row (32 slice + lane) of the SELL operator times x, computed by the K
// warps of the block sharing the slice (part = this warp's index among
// them), with the arithmetic of solve.cu's row kernels: K = 1 starts from
// diag_r x_r and adds the entries in slice order; K > 1 splits a lane's
// entries over four partial sums (entry j to sum j mod 4), adds the parts in
// order in the part-0 warp and then the diagonal.  Every thread of the block
// calls it (K > 1 synchronises the block).  Valid in the part-0 warp.
template <class T, int K>
__device__ __forceinline__ T wl_row(const WOp& op, int slice, int lane, int part, const T* x,
                                    double (*red)[32])
{
    const T* val = static_cast<const T*>(op.val);
    const T* diag = static_cast<const T*>(op.diag);
    const bool valid = slice < op.n_slices;
    const int r = slice * 32 + lane;
    T acc = T(0);
    if constexpr (K == 1) {
        if (valid) {
            const int b = __ldg(op.sptr + slice) + lane;
            const int w = (__ldg(op.sptr + slice + 1) - __ldg(op.sptr + slice)) >> 5;
            acc = (diag && r < op.n) ? __ldg(diag + r) * x[r] : T(0);
            for (int u = 0; u < w; ++u) acc = fma(__ldg(val + b + 32 * u), x[__ldg(op.col + b + 32 * u)], acc);
        }
        return acc;
    } else {
        if (valid) {
            const int b = __ldg(op.sptr + slice);
            const int w = (__ldg(op.sptr + slice + 1) - b) >> 5;
            const int stride = 32 * K, end = b + lane + 32 * w;
            int idx = b + lane + 32 * part;
            T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
            for (; idx + 3 * stride < end; idx += 4 * stride) {
                const int c0 = __ldg(op.col + idx), c1 = __ldg(op.col + idx + stride);
                const int c2 = __ldg(op.col + idx + 2 * stride), c3 = __ldg(op.col + idx + 3 * stride);
                const T v0 = __ldg(val + idx), v1 = __ldg(val + idx + stride);
                const T v2 = __ldg(val + idx + 2 * stride), v3 = __ldg(val + idx + 3 * stride);
                a0 = fma(v0, x[c0], a0);
                a1 = fma(v1, x[c1], a1);
                a2 = fma(v2, x[c2], a2);
                a3 = fma(v3, x[c3], a3);
            }
            if (idx < end) a0 = fma(__ldg(val + idx), x[__ldg(op.col + idx)], a0);
            if (idx + stride < end) a1 = fma(__ldg(val + idx + stride), x[__ldg(op.col + idx + stride)], a1);
            if (idx + 2 * stride < end)
                a2 = fma(__ldg(val + idx + 2 * stride), x[__ldg(op.col + idx + 2 * stride)], a2);
            acc = (a0 + a1) + (a2 + a3);
        }
        const int warp = threadIdx.x >> 5;
        red[warp][lane] = double(acc);   // exact for T = float as well
        __syncthreads();
        if (part == 0) {
#pragma unroll
            for (int q = 1; q < K; ++q) acc += T(red[warp + q][lane]);
        }
        __syncthreads();
        if (valid && diag && part == 0 && r < op.n) acc = fma(__ldg(diag + r), x[r], acc);
        return acc;
    }
}

// Rows 32 s + lane of slices s = s0 .. s0 + WL_R - 1 (one warp; slices at
// or past s1 give 0), with the arithmetic of solve.cu's short-row kernels:
// start from diag_r x_r, then the stored entries in slice order, one fused
// multiply-add each.  When every slice is at most 4 wide, all loads of the
// rows are issued (predicated) before their gathers, and all gathers before
// the sums.
constexpr int WL_R = 2;
template <class T>
__device__ __forceinline__ void wl_dot4(const WOp& op, int s0, int s1, int lane, const T* x, T (&acc)[WL_R])
{
    const T* val = static_cast<const T*>(op.val);
    const T* diag = static_cast<const T*>(op.diag);
    int b[WL_R], w[WL_R];
    bool fits = true;
#pragma unroll
    for (int q = 0; q < WL_R; ++q) {
        const int sq = s0 + q;
        const bool ok = sq < s1;
        const int p0 = ok ? __ldg(op.sptr + sq) : 0, p1 = ok ? __ldg(op.sptr + sq + 1) : 0;
        b[q] = p0 + lane;
        w[q] = (p1 - p0) >> 5;
        fits = fits && w[q] <= 4;
        const int r = sq * 32 + lane;
        acc[q] = (ok && diag && r < op.n) ? __ldg(diag + r) * x[r] : T(0);
    }
    if (fits) {
        int c[WL_R][4];
        T v[WL_R][4], xv[WL_R][4];
#pragma unroll
        for (int q = 0; q < WL_R; ++q)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = u < w[q];
                c[q][u] = ok ? __ldg(op.col + b[q] + 32 * u) : 0;
                v[q][u] = ok ? __ldg(val + b[q] + 32 * u) : T(0);
            }
#pragma unroll
        for (int q = 0; q < WL_R; ++q)
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[q][u] = u < w[q] ? x[c[q][u]] : T(0);
#pragma unroll
        for (int q = 0; q < WL_R; ++q)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (u < w[q]) acc[q] = fma(v[q][u], xv[q][u], acc[q]);
    } else {
#pragma unroll
        for (int q = 0; q < WL_R; ++q)
            for (int u = 0; u < w[q]; ++u)
                acc[q] = fma(__ldg(val + b[q] + 32 * u), x[__ldg(op.col + b[q] + 32 * u)], acc[q]);
    }
}

// Epilogue of one row r of a SELL operation, d = (S x)_r.
template <class T>
__device__ __forceinline__ void wl_epi(const WOp& op, int r, T d)
{
    const T a = T(op.a), bsc = T(op.b);
    switch (op.kind) {
        case W_RESTRICT:
            static_cast<T*>(op.out)[r] = static_cast<const T*>(op.in2)[r] + d;
            break;
        case W_FRESID: {
            T tt = static_cast<const T*>(op.in2)[r] - d;
            static_cast<T*>(op.out)[r] = tt;
            static_cast<T*>(op.out2)[r] = a * tt;
            break;
        }
        case W_HORNER:
            static_cast<T*>(op.out)[r] = fma(a, static_cast<const T*>(op.in2)[r], d);
            break;
        case W_HORNER_LAST: {
            const int wc = op.W[r];
            const T cb = wc >= 0 ? static_cast<const T*>(op.in3)[wc] : T(0);
            static_cast<T*>(op.out)[r] = cb + fma(a, static_cast<const T*>(op.in2)[r], d);
            break;
        }
        case W_NEWTON_REAL: {
            T* x = static_cast<T*>(op.out2);
            const T ra = static_cast<const T*>(op.in)[r], xb = op.first ? T(0) : x[r];
            x[r] = fma(ra, a, xb);
            static_cast<T*>(op.out)[r] = ra - d * a;
            break;
        }
        case W_PAIR1: {
            T* x = static_cast<T*>(op.out2);
            const T ra = static_cast<const T*>(op.in)[r], xb = op.first ? T(0) : x[r];
            T tt = a * ra - d;
            static_cast<T*>(op.out)[r] = tt;
            x[r] = fma(tt, bsc, xb);
            break;
        }
        case W_PAIR2:
            static_cast<T*>(op.out)[r] = static_cast<const T*>(op.in2)[r] - d * bsc;
            break;
        default:   // W_SPMV
            static_cast<T*>(op.out)[r] = d;
            break;
    }
}

// Short rows: each warp takes WL_R consecutive slices of the tile at a time.
template <class T>
__device__ void wl_sell_tile1(const WOp& op, int s0, int s1)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T* x = static_cast<const T*>(op.in);
    for (int g = s0 + WL_R * warp; g < s1; g += WL_R * WL_WARPS) {
        T acc[WL_R];
        wl_dot4<T>(op, g, s1, lane, x, acc);
#pragma unroll
        for (int q = 0; q < WL_R; ++q) {
            const int r = (g + q) * 32 + lane;
            if (g + q < s1 && r < op.n) wl_epi<T>(op, r, acc[q]);
        }
    }
}

// The SELL operations: slices [s0, s1) in groups of WL_WARPS / K slices.
template <class T, int K>
__device__ void wl_sell_tile(const WOp& op, int s0, int s1, double (*red)[32])
{
    if constexpr (K == 1) {
        wl_sell_tile1<T>(op, s0, s1);
        return;
    }
    constexpr int SPG = WL_WARPS / K;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int part = warp % K;
    const T a = T(op.a), bsc = T(op.b);
    for (int g = s0; g < s1; g += SPG) {   // uniform over the block
        const int slice = g + warp / K;
        const int sl = slice < s1 ? slice : op.n_slices;   // past the tile: no entries
        const int r = slice * 32 + lane;
        const bool lead = part == 0 && slice < s1 && r < op.n;
        switch (op.kind) {
            case W_RESTRICT: {
                const T* sf = static_cast<const T*>(op.in);
                const T* sc = static_cast<const T*>(op.in2);
                T* dst = static_cast<T*>(op.out);
                T d = wl_row<T, K>(op, sl, lane, part, sf, red);
                if (lead) dst[r] = sc[r] + d;
                break;
            }
            case W_FRESID: {
                const T* ec = static_cast<const T*>(op.in);
                const T* rf = static_cast<const T*>(op.in2);
                T d = wl_row<T, K>(op, sl, lane, part, ec, red);
                if (lead) {
                    T tt = rf[r] - d;
                    static_cast<T*>(op.out)[r] = tt;
                    static_cast<T*>(op.out2)[r] = a * tt;
                }
                break;
            }
            case W_HORNER: {
                const T* win = static_cast<const T*>(op.in);
                const T* t = static_cast<const T*>(op.in2);
                T d = wl_row<T, K>(op, sl, lane, part, win, red);
                if (lead) static_cast<T*>(op.out)[r] = fma(a, t[r], d);
                break;
            }
            case W_HORNER_LAST: {
                const T* win = static_cast<const T*>(op.in);
                const T* t = static_cast<const T*>(op.in2);
                const T* ec = static_cast<const T*>(op.in3);
                T d = wl_row<T, K>(op, sl, lane, part, win, red);
                if (lead) {
                    const int wc = op.W[r];
                    const T cb = wc >= 0 ? ec[wc] : T(0);
                    static_cast<T*>(op.out)[r] = cb + fma(a, t[r], d);
                }
                break;
            }
            case W_NEWTON_REAL: {
                const T* rin = static_cast<const T*>(op.in);
                T* x = static_cast<T*>(op.out2);
                T d = wl_row<T, K>(op, sl, lane, part, rin, red);
                if (lead) {
                    const T ra = rin[r], xb = op.first ? T(0) : x[r];
                    x[r] = fma(ra, a, xb);
                    static_cast<T*>(op.out)[r] = ra - d * a;
                }
                break;
            }
            case W_PAIR1: {
                const T* rin = static_cast<const T*>(op.in);
                T* x = static_cast<T*>(op.out2);
                T d = wl_row<T, K>(op, sl, lane, part, rin, red);
                if (lead) {
                    const T ra = rin[r], xb = op.first ? T(0) : x[r];
                    T tt = a * ra - d;
                    static_cast<T*>(op.out)[r] = tt;
                    x[r] = fma(tt, bsc, xb);
                }
                break;
            }
            case W_PAIR2: {
                const T* t = static_cast<const T*>(op.in);
                const T* rin = static_cast<const T*>(op.in2);
                T d = wl_row<T, K>(op, sl, lane, part, t, red);
                if (lead) static_cast<T*>(op.out)[r] = rin[r] - d * bsc;
                break;
            }
            default: {   // W_SPMV
                const T* x = static_cast<const T*>(op.in);
                T d = wl_row<T, K>(op, sl, lane, part, x, red);
                if (lead) static_cast<T*>(op.out)[r] = d;
                break;
            }
        }
    }
}

template <class T>
__device__ void wl_sell(const WOp& op, int tile, double (*red)[32])
{
    const int s0 = tile * op.unit;
    const int s1 = min(op.n_slices, s0 + op.unit);
    switch (op.K) {
        case 1: wl_sell_tile<T, 1>(op, s0, s1, red); break;
        case 2: wl_sell_tile<T, 2>(op, s0, s1, red); break;
        case 4: wl_sell_tile<T, 4>(op, s0, s1, red); break;
        default: wl_sell_tile<T, 8>(op, s0, s1, red); break;
    }
}

// Element-wise operations on rows [r0, r1).
template <class T>
__device__ void wl_vec(const WOp& op, int r0, int r1)
{
    const T a = T(op.a);
    for (int r = r0 + threadIdx.x; r < r1; r += WL_THREADS) {
        switch (op.kind) {
            case W_SMOOTH0: {
                const T* t = static_cast<const T*>(op.in);
                const T* ec = static_cast<const T*>(op.in3);
                const int wc = op.W[r];
                static_cast<T*>(op.out)[r] = (wc >= 0 ? ec[wc] : T(0)) + a * t[r];
                break;
            }
            case W_NEWTON_LAST: {
                const T* rin = static_cast<const T*>(op.in);
                T* x = static_cast<T*>(op.out);
                x[r] = fma(rin[r], a, op.first ? T(0) : x[r]);
                break;
            }
            default:   // W_ZERO
                static_cast<T*>(op.out)[r] = T(0);
                break;
        }
    }
}

// Block sum of one double per thread; valid in thread 0 (fixed order).
__device__ __forceinline__ double wl_block_sum(double v, double (*red)[32])
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[0][threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < WL_WARPS; ++q) s += red[0][q];
    __syncthreads();
    return s;
}

__device__ void wl_outer(const WOp& op, int tile, double (*red)[32])
{
    const int r0 = tile * op.unit, r1 = min(op.n, r0 + op.unit);
    switch (op.kind) {
        case W_D2F: {
            const double* a = static_cast<const double*>(op.in);
            float* b = static_cast<float*>(op.out);
            for (int r = r0 + threadIdx.x; r < r1; r += WL_THREADS) b[r] = float(a[r]);
            break;
        }
        case W_F2D: {
            const float* a = static_cast<const float*>(op.in);
            double* b = static_cast<double*>(op.out);
            for (int r = r0 + threadIdx.x; r < r1; r += WL_THREADS) b[r] = double(a[r]);
            break;
        }
        case W_SCALE: {
            const double q = *static_cast<const double*>(op.in2);
            const double inv = (*op.active && q > 0.0) ? 1.0 / sqrt(q) : 0.0;
            const double* w = static_cast<const double*>(op.in);
            double* v = static_cast<double*>(op.out);
            for (int r = r0 + threadIdx.x; r < r1; r += WL_THREADS) v[r] = w[r] * inv;
            break;
        }
        case W_DOT: {
            // partial <V_i, w> (i < m) and <w, w> of rows [r0, r1), WL_DOT_CHUNK at a time
            const double* V = static_cast<const double*>(op.in);
            const double* w = static_cast<const double*>(op.in2);
            const int mo = op.m + 1;
            for (int c0 = 0; c0 < mo; c0 += WL_DOT_CHUNK) {
                double acc[WL_DOT_CHUNK] = {};
                for (int r = r0 + threadIdx.x; r < r1; r += WL_THREADS) {
                    const double wv = w[r];
#pragma unroll
                    for (int u = 0; u < WL_DOT_CHUNK; ++u) {
                        const int i = c0 + u;
                        if (i < op.m) acc[u] = fma(V[i * op.ld + r], wv, acc[u]);
                        else if (i == op.m) acc[u] = fma(wv, wv, acc[u]);
                    }
                }
#pragma unroll
                for (int u = 0; u < WL_DOT_CHUNK; ++u) {
                    const double s = wl_block_sum(acc[u], red);
                    if (threadIdx.x == 0 && c0 + u < mo) op.part[(long long)tile * mo + c0 + u] = s;
                }
            }
            break;
        }
        case W_AXPY: {
            // w += sum_i (-h_i) V_i in order i = 0, 1, ...; partial ||w||^2
            const double* V = static_cast<const double*>(op.in);
            const double* h = static_cast<const double*>(op.in2);
            double* w = static_cast<double*>(op.out);
            double ss = 0.0;
            for (int r = r0 + threadIdx.x; r < r1; r += WL_THREADS) {
                double s = w[r];
                for (int i = 0; i < op.m; ++i) s = fma(-h[i], V[i * op.ld + r], s);
                w[r] = s;
                ss = fma(s, s, ss);
            }
            const double t = wl_block_sum(ss, red);
            if (threadIdx.x == 0) op.part[tile] = t;
            break;
        }
        case W_DOT_FIN:
        case W_AXPY_FIN: {
            // out[i] = sum over the summed op's tiles of its partials, in
            // a fixed order (lanes stride the tiles, then a shuffle tree)
            const int mo = op.kind == W_DOT_FIN ? op.m + 1 : 1;
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            double* out = static_cast<double*>(op.out);
            for (int i = warp; i < mo; i += WL_WARPS) {
                double v = 0.0;
                for (int q = lane; q < op.n; q += 32) v += op.part[(long long)q * mo + i];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane == 0) out[i] = v;
            }
            break;
        }
        default:
            break;
    }
}

__device__ void wl_run(const WOp& op, int tile, double (*red)[32])
{
    if (op.active && *(volatile const int*)op.active == 0) return;   // a converged problem
    switch (op.kind) {
        case W_SMOOTH0:
        case W_NEWTON_LAST:
        case W_ZERO: {
            const int r0 = tile * op.unit, r1 = min(op.n, r0 + op.unit);
            if (op.fp32) wl_vec<float>(op, r0, r1);
            else wl_vec<double>(op, r0, r1);
            break;
        }
        case W_D2F:
        case W_F2D:
        case W_SCALE:
        case W_DOT:
        case W_DOT_FIN:
        case W_AXPY:
        case W_AXPY_FIN:
            wl_outer(op, tile, red);
            break;
        default:
            if (op.fp32) wl_sell<float>(op, tile, red);
            else wl_sell<double>(op, tile, red);
            break;
    }
}

// Thread 0 claims the block's next tile while the block works on the
// current one (one tile of look-ahead).  The earliest unfinished tile is
// then always some block's current tile, never a claimed one waiting behind
// it, so the argument above still holds.
__global__ void __launch_bounds__(WL_THREADS, 4)
k_worklist(const WOp* __restrict__ ops, const int2* __restrict__ tiles, int ntiles, unsigned* head,
           unsigned* done, int* err)
{
    __shared__ double red[WL_WARPS][32];
    __shared__ int s_tile;
    int next = 0;
    if (threadIdx.x == 0) next = int(atomicAdd(head, 1u));
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = next;
            if (t < ntiles) next = int(atomicAdd(head, 1u));
            if (t < ntiles) {
                const int pv = ops[tiles[t].x].prev;
                if (pv >= 0) {
                    const unsigned need = unsigned(ops[pv].tiles);
                    volatile unsigned* dv = done + pv;
                    volatile int* ve = err;
                    long long spins = 0;
                    while (*dv < need) {
                        if (*ve || ++spins > WL_SPIN_LIMIT) { atomicExch(err, 1); break; }
                        __nanosleep(40);
                    }
                }
                __threadfence();   // acquire: the finished tiles' writes are visible
            }
            s_tile = t;
        }
        __syncthreads();
        const int t = s_tile;
        if (t >= ntiles) return;
        const int2 tt = tiles[t];
        wl_run(ops[tt.x], tt.y, red);
        __threadfence();   // release this thread's writes before the count
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(done + tt.x, 1u);
    }
}

}  // namespace

struct WorkList {
    DBuf<WOp> ops;
    DBuf<int2> tiles;
    DBuf<unsigned> ctr;   // [head, done per op]
    DBuf<int> err;
    int nops = 0, ntiles = 0, grid = 0;
};

namespace {

struct Chain {
    std::vector<WOp> ops;
};

template <class T>
WOp sell_op(int kind, const Sell<T>& S, int fp32)
{
    WOp o{};
    o.kind = kind;
    o.fp32 = fp32;
    o.K = S.k;
    o.n = S.n_rows;
    o.n_slices = S.n_slices;
    o.unit = S.k == 1 ? WL_SHORT_SLICES : WL_GROUPS * (WL_WARPS / S.k);
    o.tiles = std::max(1, (S.n_slices + o.unit - 1) / o.unit);
    o.sptr = S.sptr.p;
    o.col = S.col.p;
    o.val = S.val.p;
    o.diag = S.ndiag ? S.diag.p : nullptr;
    o.prev = -1;
    return o;
}

WOp vec_op(int kind, long long n, int fp32, int unit = WL_VEC_UNIT)
{
    WOp o{};
    o.kind = kind;
    o.fp32 = fp32;
    o.n = int(n);
    o.unit = unit;
    o.tiles = std::max(1, int((n + unit - 1) / unit));
    o.prev = -1;
    return o;
}

template <class T>
const SolveLevelT<T>& lops(const SolveLevel& L);
template <>
const SolveLevelT<double>& lops<double>(const SolveLevel& L) { return L.d; }
template <>
const SolveLevelT<float>& lops<float>(const SolveLevel& L) { return L.f; }

// The V-cycle of solve.cu's vcycle<T> (F-point smoothing, matrix-free
// polynomial) as a chain of operations, v -> e.
// Algorithmic bytes are those the per-operator kernels report (stored
// entries and each vector read or written once).
template <class T>
void vcycle_ops(const SolveData& S, const T* v, T* e, T* rwork, T* t, T* wa, T* wb, T* cr0, T* cr1, T* ct,
                const Sell<T>& Ac, std::vector<WOp>& out)
{
    const int fp = sizeof(T) == 4 ? 1 : 0;
    constexpr long long VB = sizeof(T);
    const int L = S.nlev;
    for (int l = 0; l < L; ++l) {
        const SolveLevel& lv = *S.lv[l];
        if (!lv.n_c) continue;
        const T* src = l == 0 ? v : rwork;
        WOp o = sell_op(W_RESTRICT, lops<T>(lv).Z, fp);
        o.in = src + lv.off;
        o.in2 = src + lv.off + lv.n_f;
        o.out = rwork + lv.off + lv.n_f;
        o.bytes = mat_bytes32(lops<T>(lv).Z) + (2LL * lv.n_c + lv.n_f + lv.n_c) * VB;
        out.push_back(o);
    }
    {
        const T* rin = (L == 0 ? v : rwork) + S.off_c;
        T* x = e + S.off_c;
        T* bufs[2] = {cr0, cr1};
        int nb = 0;
        const size_t nr = S.roots.size();
        const long long nB = (long long)S.n_coarse * VB, mB = mat_bytes32(Ac);
        for (size_t i = 0; i < nr; ++i) {
            const bool last = i + 1 == nr;
            const Root& q = S.roots[i];
            T* rout = bufs[nb];
            if (q.im == 0.0) {
                WOp o = last ? vec_op(W_NEWTON_LAST, S.n_coarse, fp) : sell_op(W_NEWTON_REAL, Ac, fp);
                o.in = rin;
                if (last) o.out = x;
                else { o.out = rout; o.out2 = x; }
                o.a = double(T(1.0 / q.re));
                o.first = i == 0;
                o.bytes = (last ? 0 : mB + 2 * nB) + (i == 0 ? 2 : 3) * nB;
                out.push_back(o);
            } else {
                const double mod2 = q.re * q.re + q.im * q.im;
                WOp o = sell_op(W_PAIR1, Ac, fp);
                o.in = rin;
                o.out = ct;
                o.out2 = x;
                o.a = double(T(2.0 * q.re));
                o.b = double(T(1.0 / mod2));
                o.first = i == 0;
                o.bytes = mB + (i == 0 ? 3 : 4) * nB;
                out.push_back(o);
                if (!last) {
                    WOp o2 = sell_op(W_PAIR2, Ac, fp);
                    o2.in = ct;
                    o2.in2 = rin;
                    o2.out = rout;
                    o2.b = double(T(1.0 / mod2));
                    o2.bytes = mB + 3 * nB;
                    out.push_back(o2);
                }
            }
            if (!last) { rin = rout; nb ^= 1; }
        }
        if (nr == 0) {
            WOp o = vec_op(W_ZERO, S.n_coarse, fp);
            o.out = x;
            out.push_back(o);
        }
    }
    for (int l = L - 1; l >= 0; --l) {
        const SolveLevel& lv = *S.lv[l];
        const SolveLevelT<T>& o = lops<T>(lv);
        const T* src = l == 0 ? v : rwork;
        const T* rf = src + lv.off;
        const T* ec = e + lv.off + lv.n_f;
        T* ef = e + lv.off;
        const int p = int(lv.alpha.size()) - 1;
        const long long fB = (long long)lv.n_f * VB;
        WOp fr = sell_op(W_FRESID, o.M, fp);
        fr.bytes = mat_bytes32(o.M) + (long long)lv.n_c * VB + 3 * fB;
        fr.in = ec;
        fr.in2 = rf;
        fr.out = t;
        fr.out2 = wa;
        fr.a = double(T(lv.alpha[p]));
        out.push_back(fr);
        if (p == 0) {
            WOp s0 = vec_op(W_SMOOTH0, lv.n_f, fp);
            s0.in = t;
            s0.in3 = ec;
            s0.W = lv.W.p;
            s0.out = ef;
            s0.a = double(T(lv.alpha[0]));
            s0.bytes = 3 * fB + 4LL * lv.n_f;
            out.push_back(s0);
            continue;
        }
        T* win = wa;
        T* wout = wb;
        for (int k = p - 1; k >= 1; --k) {
            WOp h = sell_op(W_HORNER, o.Aff, fp);
            h.in = win;
            h.in2 = t;
            h.out = wout;
            h.a = double(T(lv.alpha[k]));
            h.bytes = mat_bytes32(o.Aff) + 3 * fB;
            out.push_back(h);
            std::swap(win, wout);
        }
        WOp hl = sell_op(W_HORNER_LAST, o.Aff, fp);
        hl.in = win;
        hl.in2 = t;
        hl.in3 = ec;
        hl.W = lv.W.p;
        hl.out = ef;
        hl.a = double(T(lv.alpha[0]));
        hl.bytes = mat_bytes32(o.Aff) + 4 * fB + 4LL * lv.n_f;
        out.push_back(hl);
    }
}

template <class T>
bool sell_ok(const Sell<T>& S)
{
    return S.n_rows == 0 || (S.k >= 1 && S.k <= 8 && S.xs == 0);
}

}  // namespace

bool worklist_supported(const std::vector<Hierarchy*>& hs)
{
    for (Hierarchy* H : hs) {
        const SolveData& S = *H->solve;
        if (H->opt.precision == AIRG_MIXED_FP32_BF16R || S.smooth_type != AIRG_SMOOTH_F) return false;
        if (S.newton_grid[0] || S.newton_grid[1] || S.smooth_grid[0] || S.smooth_grid[1]) return false;
        if (!sell_ok(S.Atop) || !sell_ok(S.Ac) || !sell_ok(S.Ac32)) return false;
        for (const auto& lp : S.lv) {
            const SolveLevel& lv = *lp;
            if (lv.d.Ainv.n_rows || lv.f.Ainv.n_rows) return false;
            if (!sell_ok(lv.d.Z) || !sell_ok(lv.d.M) || !sell_ok(lv.d.Aff)) return false;
            if (!sell_ok(lv.f.Z) || !sell_ok(lv.f.M) || !sell_ok(lv.f.Aff)) return false;
        }
    }
    return true;
}

namespace {

// Problem p's operations of iteration j, in order.
std::vector<WOp> problem_chain(const WlProblem& pr, int j)
{
    std::vector<WOp> ch;
    {
        Hierarchy& H = *pr.H;
        SolveData& S = *H.solve;
        const long long n = S.n0;
        double* vj = S.V.p + size_t(j) * n;
        double* zj = S.Zs.p + size_t(j) * n;
        if (j > 0) {
            WOp o = vec_op(W_SCALE, n, 0);
            o.in = S.w.p;
            o.in2 = pr.nrm;
            o.out = vj;
            o.bytes = 16 * n;
            ch.push_back(o);
        }
        if (mixed_precision(H.opt)) {
            WOp o = vec_op(W_D2F, n, 0);
            o.in = vj;
            o.out = S.vin32.p;
            o.bytes = 12 * n;
            ch.push_back(o);
            vcycle_ops<float>(S, S.vin32.p, S.e32.p, S.rwork32.p, S.t32.p, S.wa32.p, S.wb32.p, S.cr032.p,
                              S.cr132.p, S.ct32.p, S.Ac32, ch);
            WOp f = vec_op(W_F2D, n, 0);
            f.in = S.e32.p;
            f.out = zj;
            f.bytes = 12 * n;
            ch.push_back(f);
        } else {
            vcycle_ops<double>(S, vj, zj, S.rwork.p, S.t.p, S.wa.p, S.wb.p, S.cr0.p, S.cr1.p, S.ct.p, S.Ac, ch);
        }
        WOp sp = sell_op(W_SPMV, S.Atop, 0);
        sp.in = zj;
        sp.out = S.w.p;
        sp.bytes = mat_bytes32(S.Atop) + 16 * n;
        ch.push_back(sp);
        const int unit = std::max<long long>(WL_VEC_UNIT, ((n + WL_MAX_DOT_TILES - 1) / WL_MAX_DOT_TILES + 255) / 256 * 256);
        WOp dot = vec_op(W_DOT, n, 0, unit);
        dot.m = j + 1;
        dot.in = S.V.p;
        dot.in2 = S.w.p;
        dot.ld = n;
        dot.part = S.part.p;
        dot.bytes = 8 * n * (j + 2);
        ch.push_back(dot);
        WOp dfin = vec_op(W_DOT_FIN, 1, 0, 1);
        dfin.n = dot.tiles;
        dfin.m = j + 1;
        dfin.part = S.part.p;
        dfin.out = pr.h1;
        ch.push_back(dfin);
        WOp ax = vec_op(W_AXPY, n, 0, unit);
        ax.m = j + 1;
        ax.in = S.V.p;
        ax.in2 = pr.h1;
        ax.out = S.w.p;
        ax.ld = n;
        ax.part = S.part.p;
        ax.bytes = 8 * n * (j + 3);
        ch.push_back(ax);
        WOp afin = vec_op(W_AXPY_FIN, 1, 0, 1);
        afin.n = ax.tiles;
        afin.part = S.part.p;
        afin.out = pr.nrm;
        ch.push_back(afin);
        for (WOp& o : ch) o.active = pr.active;
        if (size_t(dot.tiles) * size_t(j + 2) > S.part.n) fail(AIRG_ERR_STATE, "work list: partial-sum buffer too small");
    }
    return ch;
}

}  // namespace

long long iteration_bytes(const WlProblem& pr, int j)
{
    long long b = 0;
    for (const WOp& o : problem_chain(pr, j)) b += o.bytes;
    return b;
}

std::shared_ptr<WorkList> build_worklist(const std::vector<WlProblem>& probs, int j, cudaStream_t st)
{
    std::vector<Chain> chains(probs.size());
    for (size_t p = 0; p < probs.size(); ++p) chains[p].ops = problem_chain(probs[p], j);
    // global op indices and the chain dependencies
    std::vector<WOp> all;
    std::vector<std::vector<int>> idx(chains.size());
    size_t maxlen = 0;
    for (size_t p = 0; p < chains.size(); ++p) {
        for (size_t s = 0; s < chains[p].ops.size(); ++s) {
            WOp o = chains[p].ops[s];
            o.prev = s ? idx[p][s - 1] : -1;
            idx[p].push_back(int(all.size()));
            all.push_back(o);
        }
        maxlen = std::max(maxlen, chains[p].ops.size());
    }
    // Queue order of the operations: by the share of its chain's work done
    // before an operation's midpoint (algorithmic bytes), so that every
    // problem advances at the same relative pace and large and small
    // problems finish together; ties by problem, then by position in the
    // chain.  An operation's predecessor always has a smaller key, so its
    // tiles are queued first.
    struct Key {
        double f;
        int p, s;
    };
    std::vector<Key> keys;
    for (size_t p = 0; p < chains.size(); ++p) {
        double tot = 0.0;
        for (int oi : idx[p]) tot += double(std::max<long long>(all[oi].bytes, 1));
        double pre = 0.0;
        for (size_t s = 0; s < idx[p].size(); ++s) {
            const double w = double(std::max<long long>(all[idx[p][s]].bytes, 1));
            keys.push_back(Key{(pre + 0.5 * w) / tot, int(p), int(s)});
            pre += w;
        }
    }
    std::sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
        if (a.f != b.f) return a.f < b.f;
        if (a.p != b.p) return a.p < b.p;
        return a.s < b.s;
    });
    std::vector<int2> tiles;
    for (const Key& k : keys) {
        const int oi = idx[size_t(k.p)][size_t(k.s)];
        for (int t = 0; t < all[oi].tiles; ++t) tiles.push_back(make_int2(oi, t));
    }
    (void)maxlen;
    auto wl = std::make_shared<WorkList>();
    wl->nops = int(all.size());
    wl->ntiles = int(tiles.size());
    wl->ops.alloc(all.size());
    wl->tiles.alloc(tiles.size());
    wl->ctr.alloc(all.size() + 1);
    wl->err.alloc(1);
    CK(cudaMemcpyAsync(wl->ops.p, all.data(), all.size() * sizeof(WOp), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(wl->tiles.p, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(wl->err.p, 0, sizeof(int), st));
    int dev = 0, sms = 0, per = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_worklist, WL_THREADS, 0));
    wl->grid = std::max(1, std::min(per * sms, wl->ntiles));
    CK(cudaStreamSynchronize(st));
    return wl;
}

void launch_worklist(WorkList& wl, cudaStream_t st)
{
    CK(cudaMemsetAsync(wl.ctr.p, 0, wl.ctr.bytes(), st));
    k_worklist<<<wl.grid, WL_THREADS, 0, st>>>(wl.ops.p, wl.tiles.p, wl.ntiles, wl.ctr.p, wl.ctr.p + 1, wl.err.p);
    CK_LAUNCH();
}

bool worklist_timed_out(WorkList& wl, cudaStream_t st)
{
    int e = 0;
    d2h(&e, wl.err.p, 1, st);
    if (e) CK(cudaMemsetAsync(wl.err.p, 0, sizeof(int), st));
    return e != 0;
}

long long worklist_tiles(const WorkList& wl) { return wl.ntiles; }
long long worklist_ops(const WorkList& wl) { return wl.nops; }

}  // namespace airg
