// Many right-hand sides on one hierarchy: the V-cycle of Eq. 6 applied to k
// vectors at once (an SpMM-style V-cycle) inside k independent FGMRES
// iterations advanced in lockstep.
//
// Layout: a batch of k vectors of length n is stored row-major, [row][rhs],
// in the nested F/C order of the single solve.  Every operator kernel runs
// one warp per row with the lanes over right-hand sides (q = lane + 32 j,
// j < KW): each stored entry of the row is read once per warp (broadcast)
// and reused for all k right-hand sides, and the gathers of x read k
// consecutive values of one row -- contiguous, coalesced.  The operator
// bytes of a V-cycle are thus paid once per k right-hand sides.
//
// A right-hand side whose FGMRES residual reaches its tolerance is frozen:
// its next basis vector is zero and its least-squares solution uses only
// the columns built while it was active.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "dev_util.cuh"
#include "handle.h"
#include "solve_internal.cuh"

namespace airg {

namespace {

constexpr int BT = 256;          // threads per block (8 rows of the batch)
constexpr int MAXB = 16;         // restart length of the batched FGMRES
constexpr int MAXK = 128;        // right-hand sides per batch (KW <= 4)


// Rows of operator S times the k right-hand sides x ([row][rhs]): row r is
// handled by PW warps of a block (BT/32/PW rows per block), lanes over the
// right-hand sides (q = lane + 32 j, j < KW).  Warp `part` of a row adds the
// row's stored entries e = part, part + PW, ... in order (after the dense
// diagonal term, part 0); with PW > 1 the partial rows meet in shared memory
// and are added in part order.  PW is fixed per operator from its row
// lengths (1 for short rows, 4 for long ones), so results do not depend on
// timing.  pre(r, lane) loads the row's other operands before the product,
// so those loads overlap the gathers; entries are taken four at a time with
// all their loads issued before their FMAs, which run in entry order.  Then
// epi(r, lane, acc, pre) runs once per row.  `dot` = false skips the product
// (acc = 0).  Every thread of the block reaches the barrier.
template <class T, int KW, int PW, class V, class Pre, class Epi>
__device__ __forceinline__ void bfor_rows(const SellView<T, V>& S, const T* __restrict__ x, int k, bool dot,
                                          const Pre& pre, const Epi& epi, int rev = 0)
{
    using PV = decltype(pre(0, 0));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int part = warp % PW;
    // rev != 0: blocks take the rows in reverse order (serpentine chains)
    const int bx = rev ? int(gridDim.x) - 1 - int(blockIdx.x) : int(blockIdx.x);
    const int r = bx * (BT / 32 / PW) + warp / PW;
    const bool valid = r < S.n_rows;
    const bool lead = valid && part == 0;
    const PV pv = lead ? pre(r, lane) : PV{};
    T acc[KW];
#pragma unroll
    for (int j = 0; j < KW; ++j) acc[j] = T(0);
    if (valid && dot) {
        if (part == 0 && S.diag) {
            const T dg = __ldg(S.diag + r);
#pragma unroll
            for (int j = 0; j < KW; ++j) {
                int q = lane + 32 * j;
                if (q < k) acc[j] = dg * x[size_t(r) * k + q];
            }
        }
        const int s = r >> 5;
        const int b = S.sptr[s] + (r & 31), w = (S.sptr[s + 1] - S.sptr[s]) >> 5;
        int e = part;
        for (; e + 3 * PW < w; e += 4 * PW) {
            T v[4];
            const T* xr[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = b + 32 * (e + u * PW);
                v[u] = ldval<T>(S.val + idx);
                xr[u] = x + size_t(__ldg(S.col + idx)) * k;
            }
            T xv[4][KW];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int j = 0; j < KW; ++j) {
                    int q = lane + 32 * j;
                    xv[u][j] = q < k ? xr[u][q] : T(0);
                }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int j = 0; j < KW; ++j) acc[j] = fma(v[u], xv[u][j], acc[j]);
        }
        for (; e < w; e += PW) {
            const int idx = b + 32 * e;
            const T v = ldval<T>(S.val + idx);
            const T* xr = x + size_t(__ldg(S.col + idx)) * k;
#pragma unroll
            for (int j = 0; j < KW; ++j) {
                int q = lane + 32 * j;
                if (q < k) acc[j] = fma(v, xr[q], acc[j]);
            }
        }
    }
    if constexpr (PW > 1) {
        __shared__ T red[BT / 32][KW * 32];
#pragma unroll
        for (int j = 0; j < KW; ++j) red[warp][j * 32 + lane] = acc[j];
        __syncthreads();
        if (part == 0) {
#pragma unroll
            for (int p = 1; p < PW; ++p)
#pragma unroll
                for (int j = 0; j < KW; ++j) acc[j] += red[warp + p][j * 32 + lane];
        }
    }
    if (lead) epi(r, lane, acc, pv);
}

// this lane's values of row r of v ([row][rhs]); b: a second vector
template <class T, int KW>
struct RowVals {
    T a[KW], b[KW];
};
template <class T, int KW>
__device__ __forceinline__ RowVals<T, KW> row_vals(const T* __restrict__ va, const T* __restrict__ vb,
                                                   long long ra, long long rb, int lane, int k)
{
    RowVals<T, KW> o;
#pragma unroll
    for (int j = 0; j < KW; ++j) {
        int q = lane + 32 * j;
        o.a[j] = (va && q < k) ? va[size_t(ra) * k + q] : T(0);
        o.b[j] = (vb && rb >= 0 && q < k) ? vb[size_t(rb) * k + q] : T(0);
    }
    return o;
}

// blocks for n rows at PW warps per row
inline int grid_rows(long long n, int pw) { return grid_for(n * pw, BT / 32); }

template <class T, int KW, int PW>
__global__ void kb_spmv(SellView<T> S, const T* __restrict__ x, T* __restrict__ y, int k)
{
    bfor_rows<T, KW, PW>(S, x, k, true, [](int, int) { return 0; }, [&](int r, int lane, const T (&a)[KW], int) {
#pragma unroll
        for (int j = 0; j < KW; ++j) {
            int q = lane + 32 * j;
            if (q < k) y[size_t(r) * k + q] = a[j];
        }
    });
}

template <class T, int KW, int PW, class V = T>
__global__ void kb_restrict(SellView<T, V> Z, const T* __restrict__ sf, const T* __restrict__ sc,
                            T* __restrict__ dc, int k)
{
    bfor_rows<T, KW, PW>(Z, sf, k, true,
                         [&](int r, int lane) { return row_vals<T, KW>(sc, nullptr, r, -1, lane, k); },
                         [&](int r, int lane, const T (&a)[KW], const RowVals<T, KW>& pv) {
#pragma unroll
        for (int j = 0; j < KW; ++j) {
            int q = lane + 32 * j;
            if (q < k) dc[size_t(r) * k + q] = pv.a[j] + a[j];
        }
    });
}

template <class T, int KW, int PW>
__global__ void kb_fresid(SellView<T> M, const T* __restrict__ rf, const T* __restrict__ ec,
                          T* __restrict__ t, T* __restrict__ w, T ap, int k)
{
    bfor_rows<T, KW, PW>(M, ec, k, true,
                         [&](int r, int lane) { return row_vals<T, KW>(rf, nullptr, r, -1, lane, k); },
                         [&](int r, int lane, const T (&a)[KW], const RowVals<T, KW>& pv) {
#pragma unroll
        for (int j = 0; j < KW; ++j) {
            int q = lane + 32 * j;
            if (q < k) {
                size_t o = size_t(r) * k + q;
                T tt = pv.a[j] - a[j];
                t[o] = tt;
                w[o] = ap * tt;
            }
        }
    });
}

template <class T, int KW, int PW>
__global__ void kb_horner(SellView<T> A, const T* __restrict__ t, const T* __restrict__ win,
                          T* __restrict__ wout, T ak, int k, int rev)
{
    bfor_rows<T, KW, PW>(A, win, k, true,
                         [&](int r, int lane) { return row_vals<T, KW>(t, nullptr, r, -1, lane, k); },
                         [&](int r, int lane, const T (&a)[KW], const RowVals<T, KW>& pv) {
#pragma unroll
        for (int j = 0; j < KW; ++j) {
            int q = lane + 32 * j;
            if (q < k) wout[size_t(r) * k + q] = fma(ak, pv.a[j], a[j]);
        }
    }, rev);
}

template <class T, int KW, int PW>
__global__ void kb_horner_last(SellView<T> A, const T* __restrict__ t, const T* __restrict__ win,
                               const T* __restrict__ ec, const int* __restrict__ W,
                               T* __restrict__ ef, T a0, int k, int rev)
{
    bfor_rows<T, KW, PW>(A, win, k, true,
                         [&](int r, int lane) { return row_vals<T, KW>(t, ec, r, W[r], lane, k); },
                         [&](int r, int lane, const T (&a)[KW], const RowVals<T, KW>& pv) {
#pragma unroll
        for (int j = 0; j < KW; ++j) {
            int q = lane + 32 * j;
            if (q < k) ef[size_t(r) * k + q] = pv.b[j] + fma(a0, pv.a[j], a[j]);
        }
    }, rev);
}

// last Horner term of an in-place smoother: e += a_0 t + A win (C-point
// smooth, second F-point smooth of FCF; with win = t and a_0 = 0 it applies
// an assembled inverse)
template <class T, int KW, int PW>
__global__ void kb_horner_acc(SellView<T> A, const T* __restrict__ t, const T* __restrict__ win, T* e, T a0,
                              int k, int rev)
{
    bfor_rows<T, KW, PW>(A, win, k, true,
                         [&](int r, int lane) { return row_vals<T, KW>(t, e, r, r, lane, k); },
                         [&](int r, int lane, const T (&a)[KW], const RowVals<T, KW>& pv) {
#pragma unroll
        for (int j = 0; j < KW; ++j) {
            int q = lane + 32 * j;
            if (q < k) e[size_t(r) * k + q] = pv.b[j] + fma(a0, pv.a[j], a[j]);
        }
    }, rev);
}

// degree-0 in-place correction e += a_0 t, and a copy, over m values
template <class T>
__global__ void kb_acc0(long long m, const T* __restrict__ t, T* __restrict__ e, T a0)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) e[i] = e[i] + a0 * t[i];
}
template <class T>
__global__ void kb_copy(long long m, const T* __restrict__ a, T* __restrict__ b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) b[i] = a[i];
}

template <class T>
__global__ void kb_smooth0(long long n, const T* __restrict__ t, const T* __restrict__ ec,
                           const int* __restrict__ W, T* __restrict__ ef, T a0, int k)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * k) return;
    long long r = i / k;
    int q = int(i % k);
    int wc = W[r];
    ef[i] = (wc >= 0 ? ec[size_t(wc) * k + q] : T(0)) + a0 * t[i];
}

// Newton steps of the coarse polynomial (Sec. 2.3) for k right-hand sides
template <class T, int KW, int PW>
__global__ void kb_newton_real(SellView<T> A, const T* __restrict__ rin, T* __restrict__ rout,
                               T* __restrict__ x, T inv, int first, int last, int k, int rev)
{
    bfor_rows<T, KW, PW>(A, rin, k, !last,
                         [&](int r, int lane) { return row_vals<T, KW>(rin, first ? nullptr : x, r, r, lane, k); },
                         [&](int r, int lane, const T (&a)[KW], const RowVals<T, KW>& pv) {
#pragma unroll
        for (int j = 0; j < KW; ++j) {
            int q = lane + 32 * j;
            if (q < k) {
                size_t o = size_t(r) * k + q;
                x[o] = fma(pv.a[j], inv, pv.b[j]);
                if (!last) rout[o] = pv.a[j] - a[j] * inv;
            }
        }
    }, rev);
}

template <class T, int KW, int PW>
__global__ void kb_newton_pair1(SellView<T> A, const T* __restrict__ rin, T* __restrict__ t,
                                T* __restrict__ x, T two_a, T inv2, int first, int k, int rev)
{
    bfor_rows<T, KW, PW>(A, rin, k, true,
                         [&](int r, int lane) { return row_vals<T, KW>(rin, first ? nullptr : x, r, r, lane, k); },
                         [&](int r, int lane, const T (&a)[KW], const RowVals<T, KW>& pv) {
#pragma unroll
        for (int j = 0; j < KW; ++j) {
            int q = lane + 32 * j;
            if (q < k) {
                size_t o = size_t(r) * k + q;
                T tt = two_a * pv.a[j] - a[j];
                t[o] = tt;
                x[o] = fma(tt, inv2, pv.b[j]);
            }
        }
    }, rev);
}

template <class T, int KW, int PW>
__global__ void kb_newton_pair2(SellView<T> A, const T* __restrict__ rin, const T* __restrict__ t,
                                T* __restrict__ rout, T inv2, int k, int rev)
{
    bfor_rows<T, KW, PW>(A, t, k, true,
                         [&](int r, int lane) { return row_vals<T, KW>(rin, nullptr, r, -1, lane, k); },
                         [&](int r, int lane, const T (&a)[KW], const RowVals<T, KW>& pv) {
#pragma unroll
        for (int j = 0; j < KW; ++j) {
            int q = lane + 32 * j;
            if (q < k) rout[size_t(r) * k + q] = pv.a[j] - a[j] * inv2;
        }
    }, rev);
}

__global__ void kb_d2f(long long m, const double* a, float* b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) b[i] = (float)a[i];
}
__global__ void kb_f2d(long long m, const float* a, double* b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) b[i] = (double)a[i];
}

// [q][i] (caller, natural order) <-> [pos(i)][q] (batch, nested order)
// [q][i] (caller: right-hand sides one after the other, natural order) <->
// [pos(i)][q] (batch: rows in nested order, right-hand sides adjacent), a
// transpose with a row permutation.  A block moves a tile of 32 rows x 32
// right-hand sides through shared memory so that both the reads and the
// writes are runs of 32 consecutive doubles.  Block: 32 x 8 threads; grid:
// (ceil(n/32), ceil(k/32)).
constexpr int TT = 32;
__global__ void __launch_bounds__(256)
kb_to_nested(long long n, int k, const int* pos, const double* a, double* b)
{
    __shared__ double tile[TT][TT + 1];
    const long long i0 = (long long)blockIdx.x * TT;
    const int q0 = blockIdx.y * TT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int qq = ty; qq < TT; qq += 8) {              // read: consecutive i
        const long long i = i0 + tx;
        const int q = q0 + qq;
        if (i < n && q < k) tile[qq][tx] = a[size_t(q) * n + i];
    }
    __syncthreads();
    for (int ii = ty; ii < TT; ii += 8) {              // write: consecutive q
        const long long i = i0 + ii;
        const int q = q0 + tx;
        if (i < n && q < k) b[size_t(pos[i]) * k + q] = tile[tx][ii];
    }
}
__global__ void __launch_bounds__(256)
kb_from_nested(long long n, int k, const int* pos, const double* a, double* b)
{
    __shared__ double tile[TT][TT + 1];
    const long long i0 = (long long)blockIdx.x * TT;
    const int q0 = blockIdx.y * TT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int ii = ty; ii < TT; ii += 8) {              // read: consecutive q
        const long long i = i0 + ii;
        const int q = q0 + tx;
        if (i < n && q < k) tile[tx][ii] = a[size_t(pos[i]) * k + q];
    }
    __syncthreads();
    for (int qq = ty; qq < TT; qq += 8) {              // write: consecutive i
        const long long i = i0 + tx;
        const int q = q0 + qq;
        if (i < n && q < k) b[size_t(q) * n + i] = tile[qq][tx];
    }
}

inline dim3 grid_tiles(long long n, int k) { return dim3(unsigned((n + TT - 1) / TT), unsigned((k + TT - 1) / TT)); }

// ----------------------------------------------------- batched Krylov work --
constexpr int RG = 608;   // reduction blocks

// out[i*k + q] = sum_r V_i[r][q] * w[r][q] for i < M, and out[M*k + q] =
// <w_q, w_q> when selfdot, compiled for the exact M; blocks write partial
// sums, the last block adds them in a fixed order.
template <int M>
__global__ void __launch_bounds__(BT)
kb_multidot(long long n, int k, const double* __restrict__ V, long long ldv, const double* __restrict__ w,
            double* __restrict__ part, double* __restrict__ out, unsigned* ticket, int selfdot)
{
    const int m = M + (selfdot ? 1 : 0);
    __shared__ double red[BT];
    __shared__ bool last_block;
    const int ng = BT / k;                 // row groups per block
    const int q = threadIdx.x % k, grp = threadIdx.x / k;
    double acc[M + 1];
#pragma unroll
    for (int i = 0; i < M + 1; ++i) acc[i] = 0.0;
    if (grp < ng) {
        for (long long r = (long long)blockIdx.x * ng + grp; r < n; r += (long long)gridDim.x * ng) {
            const long long t = r * k + q;
            const double wv = __ldg(w + t);
#pragma unroll
            for (int i = 0; i < M; ++i) acc[i] = fma(__ldg(V + i * ldv + t), wv, acc[i]);
            acc[M] = fma(wv, wv, acc[M]);
        }
    }
#pragma unroll
    for (int i = 0; i < M + 1; ++i) {
        if (i < m) {
            red[threadIdx.x] = grp < ng ? acc[i] : 0.0;
            __syncthreads();
            if (threadIdx.x < k) {
                double s = 0.0;
                for (int g = 0; g < ng; ++g) s += red[g * k + threadIdx.x];
                part[((long long)blockIdx.x * m + i) * k + threadIdx.x] = s;
            }
            __syncthreads();
        }
    }
    __threadfence();
    if (threadIdx.x == 0) last_block = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last_block) return;
    __threadfence();
    for (int o = threadIdx.x; o < m * k; o += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) s += part[(long long)b * m * k + o];
        out[o] = s;
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

// w[r][q] -= sum_i h[i*k+q] V_i[r][q] (terms in the order i = 0, 1, ...),
// and out[q] = ||w_q||^2 of the result
template <int M>
__global__ void __launch_bounds__(BT)
kb_multiaxpy_norm(long long n, int k, const double* __restrict__ V, long long ldv, const double* __restrict__ h,
                  double* __restrict__ w, double* __restrict__ part, double* __restrict__ out, unsigned* ticket)
{
    __shared__ double red[BT];
    __shared__ bool last_block;
    const int ng = BT / k;
    const int q = threadIdx.x % k, grp = threadIdx.x / k;
    double c[M];
#pragma unroll
    for (int i = 0; i < M; ++i) c[i] = -h[i * k + q];
    double ss = 0.0;
    if (grp < ng) {
        for (long long r = (long long)blockIdx.x * ng + grp; r < n; r += (long long)gridDim.x * ng) {
            const long long t = r * k + q;
            double v[M];
#pragma unroll
            for (int i = 0; i < M; ++i) v[i] = __ldg(V + i * ldv + t);
            double s = w[t];
#pragma unroll
            for (int i = 0; i < M; ++i) s = fma(c[i], v[i], s);
            w[t] = s;
            ss = fma(s, s, ss);
        }
    }
    red[threadIdx.x] = grp < ng ? ss : 0.0;
    __syncthreads();
    if (threadIdx.x < k) {
        double s = 0.0;
        for (int g = 0; g < ng; ++g) s += red[g * k + threadIdx.x];
        part[(long long)blockIdx.x * k + threadIdx.x] = s;
    }
    __threadfence();
    if (threadIdx.x == 0) last_block = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last_block) return;
    __threadfence();
    for (int o = threadIdx.x; o < k; o += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) s += part[(long long)b * k + o];
        out[o] = s;
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

// x[r][q] += sum_i y[i*k+q] Z_i[r][q] (terms in the order i = 0, 1, ...)
template <int M>
__global__ void kb_update(long long n, int k, const double* __restrict__ Zs, long long ldz,
                          const double* __restrict__ y, double* __restrict__ x)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * k) return;
    int q = int(t % k);
    double v[M];
#pragma unroll
    for (int i = 0; i < M; ++i) v[i] = __ldg(Zs + i * ldz + t);
    double s = x[t];
#pragma unroll
    for (int i = 0; i < M; ++i) s = fma(y[i * k + q], v[i], s);
    x[t] = s;
}

__global__ void kb_scale(long long n, int k, const double* __restrict__ w, const double* __restrict__ inv,
                         double* __restrict__ v)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n * k) v[t] = w[t] * inv[t % k];
}

__global__ void kb_sub(long long m, const double* b, const double* y, double* r)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) r[i] = b[i] - y[i];
}

#define WITH_KW(k, ...)                                                   \
    do {                                                                  \
        if ((k) <= 32) { constexpr int KW = 1; __VA_ARGS__; }             \
        else if ((k) <= 64) { constexpr int KW = 2; __VA_ARGS__; }        \
        else { constexpr int KW = 4; __VA_ARGS__; }                       \
    } while (0)

// Runs the statement with KW (right-hand sides per lane) and PW (warps per
// row: 1 for operators with short rows, 4 for long rows) of operator S.
#define WITH_KWPW(k, S, ...)                                              \
    do {                                                                  \
        if ((S).k == 1) { constexpr int PW = 1; WITH_KW(k, __VA_ARGS__); } \
        else { constexpr int PW = 4; WITH_KW(k, __VA_ARGS__); }           \
    } while (0)

}  // namespace

// Work space of one batch width k.
struct BatchData {
    int k = 0, m = 0;
    long long nk = 0;
    DBuf<double> V, Zs, w, bp, xp, r, part, hdev, inv;
    DBuf<double> rwork, t, wa, wb, cr0, cr1, ct, rcs;          // FP64 V-cycle
    DBuf<float> rwork32, e32, vin32, t32, wa32, wb32, cr032, cr132, ct32, rcs32;  // FP32 V-cycle
    DBuf<unsigned> ticket;
    HBuf<double> hh;
    struct GEntry { const void* v; void* z; cudaGraphExec_t exec; long long kernels; };
    std::vector<GEntry> graphs;
    ~BatchData()
    {
        for (GEntry& g : graphs) cudaGraphExecDestroy(g.exec);
    }
};

namespace {

template <class T>
struct BWork {
    T* rwork; T* t; T* wa; T* wb; T* cr0; T* cr1; T* ct;
    T* rcs;    // saved C residuals, one slot per level l >= 1 (C-point smoothing)
};

template <class T>
const SolveLevelT<T>& bops(const SolveLevel& L);
template <>
const SolveLevelT<double>& bops<double>(const SolveLevel& L) { return L.d; }
template <>
const SolveLevelT<float>& bops<float>(const SolveLevel& L) { return L.f; }

template <class T>
const Sell<T>& bcoarse(const SolveData& S);
template <>
const Sell<double>& bcoarse<double>(const SolveData& S) { return S.Ac; }
template <>
const Sell<float>& bcoarse<float>(const SolveData& S) { return S.Ac32; }

// Prolongation and F-point smooth of level l for k right-hand sides (Eq. 6)
template <class T>
void bf_smooth(SolveData& S, int l, int k, const T* v, T* e, const BWork<T>& wk, cudaStream_t st)
{
    constexpr long long VB = sizeof(T);
    const long long kk = k;
    const SolveLevel& lv = *S.lv[l];
    const T* src = l == 0 ? v : wk.rwork;
    const SolveLevelT<T>& o = bops<T>(lv);
    const T* rf = src + size_t(lv.off) * k;
    const T* ec = e + size_t(lv.off + lv.n_f) * k;
    T* ef = e + size_t(lv.off) * k;
    const int nf = lv.n_f;
    const int p = int(lv.alpha.size()) - 1;
    const long long fB = (long long)nf * VB * kk;
    S.cur_level = l;
    LAUNCH_F(S, PK_FRESID, mat_bytes32(o.M) + (long long)lv.n_c * VB * kk + 3 * fB, (2 * o.M.nnz + 2LL * nf) * kk,
           WITH_KWPW(k, o.M, kb_fresid<T, KW, PW><<<grid_rows(nf, PW), BT, 0, st>>>(view(o.M), rf, ec, wk.t, wk.wa,
                                                                    T(lv.alpha[p]), k)));
    if (o.Ainv.n_rows) {
        // assembled smoother: e_f = W e_c + Ahat^-1 t (last Horner kernel, a0 = 0)
        LAUNCH_F(S, PK_HORNER, mat_bytes32(o.Ainv) + 4 * fB + 4LL * nf, (2 * o.Ainv.nnz + 3LL * nf) * kk,
                 WITH_KWPW(k, o.Ainv, kb_horner_last<T, KW, PW><<<grid_rows(nf, PW), BT, 0, st>>>(view(o.Ainv), wk.t, wk.t, ec,
                                                                               lv.W.p, ef, T(0), k, 0)));
        return;
    }
    if (p == 0) {
        LAUNCH_F(S, PK_HORNER, 3 * fB + 4LL * nf, 3LL * nf * kk,
               kb_smooth0<T><<<grid_for((long long)nf * k, BT), BT, 0, st>>>(nf, wk.t, ec, lv.W.p, ef,
                                                                            T(lv.alpha[0]), k));
        return;
    }
    const long long hB = mat_bytes32(o.Aff) + 3 * fB;
    T* win = wk.wa;
    T* wout = wk.wb;
    for (int kq = p - 1; kq >= 1; --kq) {
        LAUNCH_F(S, PK_HORNER, hB, (2 * o.Aff.nnz + 2LL * nf) * kk,
               WITH_KWPW(k, o.Aff, kb_horner<T, KW, PW><<<grid_rows(nf, PW), BT, 0, st>>>(view(o.Aff), wk.t, win, wout,
                                                                        T(lv.alpha[kq]), k, serpentine(p - 1 - kq))));
        std::swap(win, wout);
    }
    LAUNCH_F(S, PK_HORNER, hB + fB + 4LL * nf, (2 * o.Aff.nnz + 3LL * nf) * kk,
           WITH_KWPW(k, o.Aff, kb_horner_last<T, KW, PW><<<grid_rows(nf, PW), BT, 0, st>>>(view(o.Aff), wk.t, win, ec,
                                                                         lv.W.p, ef, T(lv.alpha[0]), k, serpentine(p - 1))));
}

// e += q(A) t by Horner for k right-hand sides, w = a_p t already in wk.wa
template <class T>
void bhorner_into(SolveData& S, const Sell<T>& A, const std::vector<double>& al, const BWork<T>& wk, T* e,
                  int n, int k, cudaStream_t st)
{
    constexpr long long VB = sizeof(T);
    const long long kk = k, fB = (long long)n * VB * kk;
    const int p = int(al.size()) - 1;
    if (p == 0) {
        LAUNCH_F(S, PK_HORNER, 3 * fB, 2LL * n * kk,
                 kb_acc0<T><<<grid_for((long long)n * k, BT), BT, 0, st>>>((long long)n * k, wk.t, e, T(al[0])));
        return;
    }
    const long long hB = mat_bytes32(A) + 3 * fB;
    T* win = wk.wa;
    T* wout = wk.wb;
    for (int kq = p - 1; kq >= 1; --kq) {
        LAUNCH_F(S, PK_HORNER, hB, (2 * A.nnz + 2LL * n) * kk,
                 WITH_KWPW(k, A, kb_horner<T, KW, PW><<<grid_rows(n, PW), BT, 0, st>>>(view(A), wk.t, win, wout,
                                                                                      T(al[kq]), k, serpentine(p - 1 - kq))));
        std::swap(win, wout);
    }
    LAUNCH_F(S, PK_HORNER, hB + fB, (2 * A.nnz + 3LL * n) * kk,
             WITH_KWPW(k, A, kb_horner_acc<T, KW, PW><<<grid_rows(n, PW), BT, 0, st>>>(view(A), wk.t, win, e,
                                                                                      T(al[0]), k, serpentine(p - 1))));
}

// C-point smooth of level l for k right-hand sides (Sec. 2):
// t_c = r_c - [A_cf A_cc] e_l, e_c += q_c(A_cc) t_c (or Ahat_cc^-1 t_c)
template <class T>
void bc_smooth(SolveData& S, int l, int k, const T* v, T* e, const BWork<T>& wk, cudaStream_t st)
{
    constexpr long long VB = sizeof(T);
    const long long kk = k;
    const SolveLevel& lv = *S.lv[l];
    const SolveLevelT<T>& o = bops<T>(lv);
    const int nc = lv.n_c;
    if (!nc) return;
    const T* rc = l == 0 ? v + size_t(lv.off + lv.n_f) * k : wk.rcs + size_t(lv.rc_off) * k;
    T* el = e + size_t(lv.off) * k;
    T* ec = el + size_t(lv.n_f) * k;
    const int p = int(lv.alpha_c.size()) - 1;
    const long long cB = (long long)nc * VB * kk;
    LAUNCH_F(S, PK_FRESID, mat_bytes32(o.Mc) + (long long)(lv.n_f + nc) * VB * kk + 3 * cB,
             (2 * o.Mc.nnz + 2LL * nc) * kk,
             WITH_KWPW(k, o.Mc, kb_fresid<T, KW, PW><<<grid_rows(nc, PW), BT, 0, st>>>(view(o.Mc), rc, el, wk.t, wk.wa,
                                                                                   T(lv.alpha_c[p]), k)));
    if (o.Ainvc.n_rows) {
        LAUNCH_F(S, PK_HORNER, mat_bytes32(o.Ainvc) + 4 * cB, (2 * o.Ainvc.nnz + 2LL * nc) * kk,
                 WITH_KWPW(k, o.Ainvc, kb_horner_acc<T, KW, PW><<<grid_rows(nc, PW), BT, 0, st>>>(
                                           view(o.Ainvc), wk.t, wk.t, ec, T(0), k, 0)));
        return;
    }
    bhorner_into<T>(S, o.Acc, lv.alpha_c, wk, ec, nc, k, st);
}

// second F-point smooth of FCF for k right-hand sides
template <class T>
void bf_smooth_again(SolveData& S, int l, int k, const T* v, T* e, const BWork<T>& wk, cudaStream_t st)
{
    constexpr long long VB = sizeof(T);
    const long long kk = k;
    const SolveLevel& lv = *S.lv[l];
    const SolveLevelT<T>& o = bops<T>(lv);
    const int nf = lv.n_f;
    if (!nf) return;
    const T* rf = (l == 0 ? v : wk.rwork) + size_t(lv.off) * k;
    T* el = e + size_t(lv.off) * k;
    const int p = int(lv.alpha.size()) - 1;
    const long long fB = (long long)nf * VB * kk;
    LAUNCH_F(S, PK_FRESID, mat_bytes32(o.Mf) + (long long)(nf + lv.n_c) * VB * kk + 3 * fB,
             (2 * o.Mf.nnz + 2LL * nf) * kk,
             WITH_KWPW(k, o.Mf, kb_fresid<T, KW, PW><<<grid_rows(nf, PW), BT, 0, st>>>(view(o.Mf), rf, el, wk.t, wk.wa,
                                                                                   T(lv.alpha[p]), k)));
    if (o.Ainv.n_rows) {
        LAUNCH_F(S, PK_HORNER, mat_bytes32(o.Ainv) + 4 * fB, (2 * o.Ainv.nnz + 2LL * nf) * kk,
                 WITH_KWPW(k, o.Ainv, kb_horner_acc<T, KW, PW><<<grid_rows(nf, PW), BT, 0, st>>>(
                                          view(o.Ainv), wk.t, wk.t, el, T(0), k, 0)));
        return;
    }
    bhorner_into<T>(S, o.Aff, lv.alpha, wk, el, nf, k, st);
}

// e = M^-1 v for k right-hand sides (nested order, [row][rhs])
template <class T>
void bvcycle(SolveData& S, int k, const T* v, T* e, const BWork<T>& wk, cudaStream_t st)
{
    const int L = S.nlev;
    constexpr long long VB = sizeof(T);
    const long long kk = k;
    for (int l = 0; l < L; ++l) {
        const SolveLevel& lv = *S.lv[l];
        const T* src = l == 0 ? v : wk.rwork;
        const Sell<T>& Z = bops<T>(lv).Z;
        const Sell<T, bf16s>& Zb = bops<T>(lv).Zb;
        S.cur_level = l;
        if (l > 0 && lv.n_c && S.smooth_type != AIRG_SMOOTH_F)   // restriction overwrites r_c in place
            LAUNCH_F(S, PK_RESTRICT, 2LL * lv.n_c * VB * kk, 0,
                     kb_copy<T><<<grid_for((long long)lv.n_c * k, BT), BT, 0, st>>>(
                         (long long)lv.n_c * k, src + size_t(lv.off + lv.n_f) * k, wk.rcs + size_t(lv.rc_off) * k));
        if (lv.n_c && Zb.val.n)
            LAUNCH_F(S, PK_RESTRICT, mat_bytes32(Zb) + (2LL * lv.n_c + lv.n_f + lv.n_c) * VB * kk,
                     (2 * Zb.nnz + lv.n_c) * kk,
                     WITH_KWPW(k, Zb, kb_restrict<T, KW, PW, bf16s><<<grid_rows(lv.n_c, PW), BT, 0, st>>>(
                                    view(Zb), src + size_t(lv.off) * k, src + size_t(lv.off + lv.n_f) * k,
                                    wk.rwork + size_t(lv.off + lv.n_f) * k, k)));
        else if (lv.n_c)
            LAUNCH_F(S, PK_RESTRICT, mat_bytes32(Z) + (2LL * lv.n_c + lv.n_f + lv.n_c) * VB * kk,
                     (2 * Z.nnz + lv.n_c) * kk,
                   WITH_KWPW(k, Z, kb_restrict<T, KW, PW><<<grid_rows(lv.n_c, PW), BT, 0, st>>>(
                                  view(Z), src + size_t(lv.off) * k, src + size_t(lv.off + lv.n_f) * k,
                                  wk.rwork + size_t(lv.off + lv.n_f) * k, k)));
    }
    {
        const T* rc = (L == 0 ? v : wk.rwork) + size_t(S.off_c) * k;
        T* x = e + size_t(S.off_c) * k;
        const Sell<T>& A = bcoarse<T>(S);
        SellView<T> Av = view(A);
        const int nco = S.n_coarse;
        const long long nB = (long long)nco * VB * kk, mB = mat_bytes32(A);
        S.cur_level = L;
        const T* rin = rc;
        T* bufs[2] = {wk.cr0, wk.cr1};
        int nb = 0;
        size_t nr = S.roots.size();
        int nsp = 0;   // SpMVs with the coarse operator so far (their direction alternates)
        for (size_t i = 0; i < nr; ++i) {
            bool last = i + 1 == nr;
            const Root& q = S.roots[i];
            T* rout = bufs[nb];
            if (q.im == 0.0) {
                LAUNCH_F(S, PK_NEWTON, (last ? 0 : mB + 2 * nB) + (i == 0 ? 2 : 3) * nB,
                         (last ? 2LL * nco : 2 * A.nnz + 4LL * nco) * kk,
                       WITH_KWPW(k, A, kb_newton_real<T, KW, PW><<<grid_rows(nco, PW), BT, 0, st>>>(
                                      Av, rin, rout, x, T(1.0 / q.re), i == 0, last, k, serpentine(nsp))));
                nsp += 1;
            } else {
                double mod2 = q.re * q.re + q.im * q.im;
                LAUNCH_F(S, PK_NEWTON, mB + (i == 0 ? 3 : 4) * nB, (2 * A.nnz + 4LL * nco) * kk,
                       WITH_KWPW(k, A, kb_newton_pair1<T, KW, PW><<<grid_rows(nco, PW), BT, 0, st>>>(
                                      Av, rin, wk.ct, x, T(2.0 * q.re), T(1.0 / mod2), i == 0, k, serpentine(nsp))));
                if (!last)
                    LAUNCH_F(S, PK_NEWTON, mB + 3 * nB, (2 * A.nnz + 2LL * nco) * kk,
                           WITH_KWPW(k, A, kb_newton_pair2<T, KW, PW><<<grid_rows(nco, PW), BT, 0, st>>>(
                                          Av, rin, wk.ct, rout, T(1.0 / mod2), k, serpentine(nsp + 1))));
                nsp += 2;
            }
            if (!last) { rin = rout; nb ^= 1; }
        }
        if (nr == 0) CK(cudaMemsetAsync(x, 0, sizeof(T) * size_t(nco) * k, st));
    }
    for (int l = L - 1; l >= 0; --l) {
        S.cur_level = l;
        bf_smooth<T>(S, l, k, v, e, wk, st);
        if (S.smooth_type != AIRG_SMOOTH_F) {
            bc_smooth<T>(S, l, k, v, e, wk, st);
            if (S.smooth_type == AIRG_SMOOTH_FCF) bf_smooth_again<T>(S, l, k, v, e, wk, st);
        }
    }
    S.close_run(st);
    S.cur_level = 0;
    CK_LAUNCH();
}

void bprecond_launch(Hierarchy& H, BatchData& B, const double* v, double* z, cudaStream_t st)
{
    SolveData& S = *H.solve;
    long long nk = B.nk;
    if (mixed_precision(H.opt)) {
        LAUNCH(S, PK_LAYOUT, 12 * nk, kb_d2f<<<grid_for(nk, BT), BT, 0, st>>>(nk, v, B.vin32.p));
        BWork<float> wk{B.rwork32.p, B.t32.p, B.wa32.p, B.wb32.p, B.cr032.p, B.cr132.p, B.ct32.p, B.rcs32.p};
        bvcycle<float>(S, B.k, B.vin32.p, B.e32.p, wk, st);
        LAUNCH(S, PK_LAYOUT, 12 * nk, kb_f2d<<<grid_for(nk, BT), BT, 0, st>>>(nk, B.e32.p, z));
    } else {
        BWork<double> wk{B.rwork.p, B.t.p, B.wa.p, B.wb.p, B.cr0.p, B.cr1.p, B.ct.p, B.rcs.p};
        bvcycle<double>(S, B.k, v, z, wk, st);
    }
}

void bprecond(Hierarchy& H, BatchData& B, const double* v, double* z, cudaStream_t st)
{
    SolveData& S = *H.solve;
    if (S.prof || !S.use_graphs) {
        bprecond_launch(H, B, v, z, st);
        return;
    }
    BatchData::GEntry* ge = nullptr;
    for (auto& g : B.graphs)
        if (g.v == v && g.z == z) { ge = &g; break; }
    if (!ge) {
        long long before = S.launches;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        try {
            bprecond_launch(H, B, v, z, st);
        } catch (...) {
            cudaGraph_t g0;
            cudaStreamEndCapture(st, &g0);
            if (g0) cudaGraphDestroy(g0);
            throw;
        }
        cudaGraph_t graph;
        CK(cudaStreamEndCapture(st, &graph));
        cudaGraphExec_t exec;
        cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(e);
        long long nkern = S.launches - before;
        S.launches = before;
        B.graphs.push_back(BatchData::GEntry{v, z, exec, nkern});
        ge = &B.graphs.back();
    }
    CK(cudaGraphLaunch(ge->exec, st));
    S.launches += ge->kernels;
}

void ensure_batch(Hierarchy& H, int k)
{
    SolveData& S = *H.solve;
    if (S.batch && S.batch->k == k) return;
    S.batch.reset();
    auto B = std::make_shared<BatchData>();
    B->k = k;
    B->m = std::min(std::max(1, H.opt.gmres_restart), MAXB);
    long long n = S.n0;
    B->nk = n * k;
    size_t nk = size_t(B->nk);
    int m = B->m;
    B->V.alloc(size_t(m + 1) * nk);
    B->Zs.alloc(size_t(m) * nk);
    B->w.alloc(nk); B->bp.alloc(nk); B->xp.alloc(nk); B->r.alloc(nk);
    B->part.alloc(size_t(RG) * (MAXB + 1) * k);
    B->hdev.alloc(size_t(3 * (MAXB + 2)) * k);
    B->inv.alloc(size_t(k));
    B->hh.alloc(size_t(3 * (MAXB + 2)) * k);
    B->ticket.alloc(1);
    CK(cudaMemset(B->ticket.p, 0, sizeof(unsigned)));
    size_t nf = size_t(std::max({S.max_nf, S.max_nc, 1})) * k, nc = size_t(std::max(S.n_coarse, 1)) * k;
    const size_t nrc = S.smooth_type != AIRG_SMOOTH_F ? size_t(std::max<long long>(S.rc_total, 1)) * k : 0;
    if (mixed_precision(H.opt)) {
        B->rwork32.alloc(nk); B->e32.alloc(nk); B->vin32.alloc(nk);
        B->t32.alloc(nf); B->wa32.alloc(nf); B->wb32.alloc(nf);
        B->cr032.alloc(nc); B->cr132.alloc(nc); B->ct32.alloc(nc);
        if (nrc) B->rcs32.alloc(nrc);
    } else {
        B->rwork.alloc(nk);
        B->t.alloc(nf); B->wa.alloc(nf); B->wb.alloc(nf);
        B->cr0.alloc(nc); B->cr1.alloc(nc); B->ct.alloc(nc);
        if (nrc) B->rcs.alloc(nrc);
    }
    S.batch = B;
}

// per-RHS 2-norms of a batch
void bnorms(SolveData& S, BatchData& B, const double* x, std::vector<double>& out, cudaStream_t st)
{
    long long n = S.n0;
    int k = B.k;
    LAUNCH_F(S, PK_KRYLOV, 8 * B.nk, 2 * B.nk,
           kb_multidot<1><<<RG, BT, 0, st>>>(n, k, x, B.nk, x, B.part.p, B.hdev.p, B.ticket.p, 0));
    out.resize(k);
    d2h(out.data(), B.hdev.p, size_t(k), st);
    for (double& v : out) v = std::sqrt(std::max(v, 0.0));
}

}  // namespace

// Lockstep FGMRES(m) for k right-hand sides (device b, x in the caller's
// layout: k vectors of length n one after the other).
void solve_batched(Hierarchy& H, int k, const double* b, double* x, double rtol, double atol,
                   int maxit, airg_solve_info& info, cudaStream_t st)
{
    SolveData& S = *H.solve;
    ensure_batch(H, k);
    BatchData& B = *S.batch;
    const long long n = S.n0, nk = B.nk;
    const int m = B.m;
    const int g = grid_for(nk, BT);
    SellView<double> A = view(S.Atop);
    const long long topB = mat_bytes32(S.Atop) + 16 * nk;
    LAUNCH(S, PK_LAYOUT, 20 * nk, kb_to_nested<<<grid_tiles(n, k), 256, 0, st>>>(n, k, S.pos0.p, b, B.bp.p));
    LAUNCH(S, PK_LAYOUT, 20 * nk, kb_to_nested<<<grid_tiles(n, k), 256, 0, st>>>(n, k, S.pos0.p, x, B.xp.p));
    std::vector<double> bn, rn, tol(k);
    bnorms(S, B, B.bp.p, bn, st);
    for (int q = 0; q < k; ++q) tol[q] = std::max(rtol * bn[q], atol);
    auto residual = [&]() {
        LAUNCH_F(S, PK_TOPSPMV, topB, 2 * S.Atop.nnz * k,
               WITH_KWPW(k, S.Atop, kb_spmv<double, KW, PW><<<grid_rows(n, PW), BT, 0, st>>>(A, B.xp.p, B.w.p, k)));
        LAUNCH_F(S, PK_KRYLOV, 24 * nk, nk, kb_sub<<<g, BT, 0, st>>>(nk, B.bp.p, B.w.p, B.r.p));
        bnorms(S, B, B.r.p, rn, st);
    };
    residual();
    int its = 0;
    if (H.opt.outer == AIRG_OUTER_RICHARDSON) {
        // lockstep Richardson: x_q += M^-1 r_q for every unconverged q
        std::vector<double> yq(k);
        while (its < maxit) {
            int nact = 0;
            for (int q = 0; q < k; ++q) {
                yq[q] = rn[q] > tol[q] ? 1.0 : 0.0;
                nact += rn[q] > tol[q];
            }
            if (!nact) break;
            bprecond(H, B, B.r.p, B.Zs.p, st);
            h2d(B.hdev.p, yq.data(), size_t(k), st);
            LAUNCH_F(S, PK_KRYLOV, 24 * nk, 2 * nk, kb_update<1><<<g, BT, 0, st>>>(n, k, B.Zs.p, nk, B.hdev.p, B.xp.p));
            residual();
            ++its;
        }
    }
    std::vector<double> Hm(size_t(m + 1) * m * k), cs(size_t(m) * k), sn(size_t(m) * k),
        gv(size_t(m + 1) * k), Y(size_t(m) * k), inv(k);
    std::vector<int> active(k), jdone(k);
    auto hq = [&](int i, int j, int q) -> double& { return Hm[(size_t(i) * m + j) * k + q]; };
    double* hh = B.hh.p;
    while (H.opt.outer == AIRG_OUTER_FGMRES && its < maxit) {
        int nact = 0;
        for (int q = 0; q < k; ++q) {
            active[q] = rn[q] > tol[q];
            nact += active[q];
            jdone[q] = 0;
            inv[q] = active[q] ? 1.0 / rn[q] : 0.0;
        }
        if (!nact) break;
        std::fill(gv.begin(), gv.end(), 0.0);
        for (int q = 0; q < k; ++q) gv[q] = rn[q];
        h2d(B.inv.p, inv.data(), size_t(k), st);
        LAUNCH_F(S, PK_KRYLOV, 16 * nk, nk, kb_scale<<<g, BT, 0, st>>>(n, k, B.r.p, B.inv.p, B.V.p));
        for (int j = 0; j < m; ++j) {
            double* vj = B.V.p + size_t(j) * nk;
            double* zj = B.Zs.p + size_t(j) * nk;
            bprecond(H, B, vj, zj, st);
            LAUNCH_F(S, PK_TOPSPMV, topB, 2 * S.Atop.nnz * k,
                   WITH_KWPW(k, S.Atop, kb_spmv<double, KW, PW><<<grid_rows(n, PW), BT, 0, st>>>(A, zj, B.w.p, k)));
            // CGS with a second pass only if the first cancelled, for some
            // active right-hand side, more than reorth_ratio() allows
            double* h1 = B.hdev.p;
            double* h2 = B.hdev.p + size_t(MAXB + 2) * k;
            double* hnp = B.hdev.p + size_t(2) * (MAXB + 2) * k;
            LAUNCH_F(S, PK_KRYLOV, 8LL * nk * (j + 2), 2LL * nk * (j + 2),
                   WITH_M(j + 1, kb_multidot<MM><<<RG, BT, 0, st>>>(n, k, B.V.p, nk, B.w.p, B.part.p, h1,
                                                                     B.ticket.p, 1)));
            LAUNCH_F(S, PK_KRYLOV, 8LL * nk * (j + 3), 2LL * nk * (j + 2),
                   WITH_M(j + 1, kb_multiaxpy_norm<MM><<<RG, BT, 0, st>>>(n, k, B.V.p, nk, h1, B.w.p, B.part.p,
                                                                           hnp, B.ticket.p)));
            CK(cudaMemcpyAsync(hh, B.hdev.p, sizeof(double) * 3 * (MAXB + 2) * k, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            bool again = false;
            const double ro = reorth_ratio();
            for (int q = 0; q < k; ++q)
                if (active[q] && hh[size_t(2) * (MAXB + 2) * k + q] < ro * hh[size_t(j + 1) * k + q]) again = true;
            for (int q = 0; q < k; ++q)
                for (int i = 0; i <= j; ++i) hq(i, j, q) = hh[size_t(i) * k + q];
            if (again) {
                LAUNCH_F(S, PK_KRYLOV, 8LL * nk * (j + 2), 2LL * nk * (j + 1),
                       WITH_M(j + 1, kb_multidot<MM><<<RG, BT, 0, st>>>(n, k, B.V.p, nk, B.w.p, B.part.p, h2,
                                                                         B.ticket.p, 0)));
                LAUNCH_F(S, PK_KRYLOV, 8LL * nk * (j + 3), 2LL * nk * (j + 2),
                       WITH_M(j + 1, kb_multiaxpy_norm<MM><<<RG, BT, 0, st>>>(n, k, B.V.p, nk, h2, B.w.p, B.part.p,
                                                                               hnp, B.ticket.p)));
                CK(cudaMemcpyAsync(hh, B.hdev.p, sizeof(double) * 3 * (MAXB + 2) * k, cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                for (int q = 0; q < k; ++q)
                    for (int i = 0; i <= j; ++i) hq(i, j, q) += hh[(size_t(MAXB + 2) + i) * k + q];
            }
            ++its;
            int still = 0;
            for (int q = 0; q < k; ++q) {
                inv[q] = 0.0;
                if (!active[q]) continue;
                double hn = std::sqrt(std::max(hh[size_t(2) * (MAXB + 2) * k + q], 0.0));
                hq(j + 1, j, q) = hn;
                for (int i = 0; i < j; ++i) {
                    double a = hq(i, j, q), c = hq(i + 1, j, q);
                    hq(i, j, q) = cs[size_t(i) * k + q] * a + sn[size_t(i) * k + q] * c;
                    hq(i + 1, j, q) = -sn[size_t(i) * k + q] * a + cs[size_t(i) * k + q] * c;
                }
                double a = hq(j, j, q), c = hq(j + 1, j, q);
                double den = std::hypot(a, c);
                cs[size_t(j) * k + q] = den > 0 ? a / den : 1.0;
                sn[size_t(j) * k + q] = den > 0 ? c / den : 0.0;
                hq(j, j, q) = den;
                hq(j + 1, j, q) = 0.0;
                gv[size_t(j + 1) * k + q] = -sn[size_t(j) * k + q] * gv[size_t(j) * k + q];
                gv[size_t(j) * k + q] = cs[size_t(j) * k + q] * gv[size_t(j) * k + q];
                jdone[q] = j + 1;
                if (std::fabs(gv[size_t(j + 1) * k + q]) <= tol[q] || den == 0.0 || hn == 0.0) {
                    active[q] = 0;
                } else {
                    inv[q] = 1.0 / hn;
                    ++still;
                }
            }
            if (!still || its >= maxit || j + 1 == m) break;
            h2d(B.inv.p, inv.data(), size_t(k), st);
            LAUNCH_F(S, PK_KRYLOV, 16 * nk, nk,
                   kb_scale<<<g, BT, 0, st>>>(n, k, B.w.p, B.inv.p, B.V.p + size_t(j + 1) * nk));
        }
        // least squares per right-hand side, zero-padded to the common width
        int jmax = 0;
        std::fill(Y.begin(), Y.end(), 0.0);
        for (int q = 0; q < k; ++q) {
            int jd = jdone[q];
            jmax = std::max(jmax, jd);
            for (int j = jd - 1; j >= 0; --j) {
                double s = gv[size_t(j) * k + q];
                for (int i = j + 1; i < jd; ++i) s -= hq(j, i, q) * Y[size_t(i) * k + q];
                Y[size_t(j) * k + q] = s / hq(j, j, q);
            }
        }
        if (jmax) {
            h2d(B.hdev.p, Y.data(), size_t(jmax) * k, st);
            LAUNCH_F(S, PK_KRYLOV, 8LL * nk * (jmax + 2), 2LL * nk * jmax,
                   WITH_M(jmax, kb_update<MM><<<g, BT, 0, st>>>(n, k, B.Zs.p, nk, B.hdev.p, B.xp.p)));
        }
        residual();
    }
    int conv = 1;
    double worst = 0.0;
    for (int q = 0; q < k; ++q) {
        double rel = bn[q] > 0 ? rn[q] / bn[q] : 0.0;
        worst = std::max(worst, rel);
        if (rn[q] > tol[q]) conv = 0;
    }
    LAUNCH(S, PK_LAYOUT, 20 * nk, kb_from_nested<<<grid_tiles(n, k), 256, 0, st>>>(n, k, S.pos0.p, B.xp.p, x));
    CK_LAUNCH();
    info.iterations = std::max(info.iterations, its);
    info.rel_residual = std::max(info.rel_residual, worst);
    info.converged = info.converged && conv;
}

int batch_max_width() { return MAXK; }

}  // namespace airg
