// AIRG solve phase on the GPU: one V-cycle with up F-point smoothing only
// (Sec. 2, Eq. 6) as the right preconditioner of FP64 flexible GMRES.
//
// Layout ("nested F/C order").  Level l's unknowns are stored as
// [F points of level l | unknowns of level l+1], recursively, so the whole
// hierarchy lives in one vector of the top-level length: level l occupies the
// suffix starting at off_l = n_F,0 + ... + n_F,l-1 and its C points are
// exactly level l+1's block.  Restriction r_{l+1} = r_c + Z r_f (R of Eq. 4)
// therefore updates the C block in place, the coarse-grid correction e_c is
// already where the prolongation reads it, and no gather or scatter runs
// between levels.  The outer FGMRES works on the top operator permuted into
// the same order; b and x are permuted once on entry and exit.
//
// Operators are SELL-32 (slices of 32 rows, column-major inside a slice,
// padded to the slice's longest row) so that a warp reads 32 consecutive
// rows with coalesced loads.  The F-point residual uses M = A_fc + A_ff W
// (the F rows of A P, formed in the setup), so t = r_f - M e_c is one SpMV
// instead of a prolongation followed by two (Eq. 6 with e_f = W e_c).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <mutex>

#include "dev_util.cuh"
#include "handle.h"
#include "solve_internal.cuh"

namespace airg {

namespace {
constexpr int TB = 256;
}
Hierarchy::Hierarchy() = default;
Hierarchy::~Hierarchy() = default;

namespace {

// ----------------------------------------------------------- SELL build --
// Slice widths (x 32).  With `split`, the entry of row r whose (mapped)
// column is r goes to the dense diagonal and is not counted.
__global__ void k_sell_width(int nrows, int nslices, const int* rp, const int* ci, const int* src_row,
                             const int* cmap, int split, int* width)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslices) return;
    int w = 0;
    for (int l = 0; l < 32; ++l) {
        int r = s * 32 + l;
        if (r >= nrows) break;
        int i = src_row ? src_row[r] : r;
        int len = rp[i + 1] - rp[i];
        if (split)
            for (int j = rp[i]; j < rp[i + 1]; ++j)
                if ((cmap ? cmap[ci[j]] : ci[j]) == r) --len;
        w = max(w, len);
    }
    width[s] = w * 32;
}

template <class T>
__global__ void k_sell_fill(int nrows, int nslices, const int* rp, const int* ci, const double* v,
                            const int* src_row, const int* cmap, const int* sptr, int* col, T* val,
                            T* diag, unsigned long long* ndiag)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nslices * 32) return;
    int s = r >> 5, lane = r & 31;
    int w = (sptr[s + 1] - sptr[s]) >> 5;
    int base = sptr[s] + lane;
    if (r >= nrows) {   // columns set by k_sell_pad
        for (int k = 0; k < w; ++k) { col[base + k * 32] = -1; val[base + k * 32] = T(0); }
        return;
    }
    int i = src_row ? src_row[r] : r;
    int k = 0, lastc = -1;   // a row without stored entries: columns set by k_sell_pad
    bool found = false;
    for (int j = rp[i]; j < rp[i + 1]; ++j) {
        int c = cmap ? cmap[ci[j]] : ci[j];
        if (diag && c == r) {
            diag[r] = T(v[j]);
            found = true;
            continue;
        }
        col[base + k * 32] = c;
        val[base + k * 32] = T(v[j]);
        lastc = c;
        ++k;
    }
    for (; k < w; ++k) {
        col[base + k * 32] = lastc;
        val[base + k * 32] = T(0);
    }
    if (diag) {
        if (found) atomicAdd(ndiag, 1ULL);
        else diag[r] = T(0);
    }
}

// Padding of the rows that have no stored entry (and of the rows past the
// end of the last slice): the slice's smallest stored column, so that every
// padded entry gathers a valid element near the slice's others (its value
// is 0).  One warp per slice, lane = row.
__global__ void k_sell_pad(int nslices, const int* __restrict__ sptr, int* col)
{
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (s >= nslices) return;
    const int b = sptr[s] + lane, w = (sptr[s + 1] - sptr[s]) >> 5;
    int m = 0x7fffffff;
    for (int k = 0; k < w; ++k) {
        const int c = col[b + 32 * k];
        if (c >= 0) m = min(m, c);
    }
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (m == 0x7fffffff) m = 0;
    for (int k = 0; k < w; ++k)
        if (col[b + 32 * k] < 0) col[b + 32 * k] = m;
}

template <class T>
void build_sell(const DevCSR& A, const int* src_row, const int* cmap, int n_cols, Sell<T>& S,
                bool split_diag, cudaStream_t st)
{
    S.n_rows = A.n_rows;
    S.n_cols = n_cols;
    S.nnz = A.nnz;
    S.k = choose_parts(A.nnz, A.n_rows);
    S.r = S.k == 1 ? 1 : 4;
    S.n_slices = (A.n_rows + 31) / 32;
    S.sptr.alloc(size_t(S.n_slices) + 1);
    if (S.n_slices)
        k_sell_width<<<grid_for(S.n_slices, TB), TB, 0, st>>>(A.n_rows, S.n_slices, A.rp.p, A.ci.p, src_row,
                                                                cmap, split_diag ? 1 : 0, S.sptr.p);
    CK_LAUNCH();
    S.padded = exclusive_scan(S.sptr.p, S.sptr.p, S.n_slices, st);
    S.col.alloc(std::max<long long>(S.padded, 1));
    S.val.alloc(std::max<long long>(S.padded, 1));
    DBuf<unsigned long long> cnt(1);
    CK(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), st));
    if (split_diag) S.diag.alloc(std::max(A.n_rows, 1));
    if (S.n_slices)
        k_sell_fill<T><<<grid_for((long long)S.n_slices * 32, TB), TB, 0, st>>>(
            A.n_rows, S.n_slices, A.rp.p, A.ci.p, A.v.p, src_row, cmap, S.sptr.p, S.col.p, S.val.p,
            split_diag ? S.diag.p : nullptr, cnt.p);
    if (S.n_slices) k_sell_pad<<<grid_for((long long)S.n_slices * 32, TB), TB, 0, st>>>(S.n_slices, S.sptr.p, S.col.p);
    CK_LAUNCH();
    unsigned long long nd = 0;
    d2h(&nd, cnt.p, 1, st);
    S.ndiag = (long long)nd;
    if (!split_diag) S.diag = DBuf<T>();
}

template <class T>
void sell_to_f32(const Sell<double>& S, Sell<T>& out, cudaStream_t st);

__global__ void k_col16(long long n, const int* __restrict__ col, unsigned short* __restrict__ col16)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) col16[i] = (unsigned short)col[i];
}

// Slice bases and 16-bit offsets: cbase[s] = smallest column of slice s,
// col16 = col - cbase[s]; *span gets the largest offset.  One warp per slice.
__global__ void k_col16_rel(int nslices, const int* __restrict__ sptr, const int* __restrict__ col,
                            int* __restrict__ cbase, unsigned short* __restrict__ col16, int* span)
{
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (s >= nslices) return;
    const int b = sptr[s], e = sptr[s + 1];
    int lo = 0x7fffffff, hi = 0;
    for (int i = b + lane; i < e; i += 32) {
        lo = min(lo, col[i]);
        hi = max(hi, col[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lo == 0x7fffffff) lo = hi = 0;
    if (lane == 0) {
        cbase[s] = lo;
        atomicMax(span, hi - lo);
    }
    if (hi - lo > 65535) return;   // the operator keeps 32-bit indices
    for (int i = b + lane; i < e; i += 32) col16[i] = (unsigned short)(col[i] - lo);
}

// 16-bit copy of an operator's column indices: its single-vector row
// kernels then read 2 instead of 4 bytes of index per entry, and find the
// same column values (the index itself with at most 65536 columns, else the
// offset from the slice's base, where every slice spans at most 65536
// columns; otherwise the operator keeps 32-bit indices only).  AIRG_COL16=0
// keeps 32-bit indices everywhere (for comparison).
template <class T, class V>
void add_col16(Sell<T, V>& S, cudaStream_t st)
{
    const char* e = getenv("AIRG_COL16");
    if ((e && e[0] == '0') || S.padded == 0 || S.n_slices == 0) return;
    S.col16.alloc(size_t(S.padded));
    if (S.n_cols <= 65536) {
        k_col16<<<grid_for(S.padded, TB), TB, 0, st>>>(S.padded, S.col.p, S.col16.p);
        CK_LAUNCH();
        return;
    }
    S.cbase.alloc(size_t(S.n_slices));
    DBuf<int> span(1);
    CK(cudaMemsetAsync(span.p, 0, sizeof(int), st));
    k_col16_rel<<<grid_for((long long)S.n_slices * 32, TB), TB, 0, st>>>(S.n_slices, S.sptr.p, S.col.p, S.cbase.p,
                                                                        S.col16.p, span.p);
    CK_LAUNCH();
    if (read1(span.p, st) > 65535) {
        S.col16 = DBuf<unsigned short>();
        S.cbase = DBuf<int>();
    }
}

__global__ void k_d2f(long long n, const double* a, float* b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}
__global__ void k_f2d(long long n, const float* a, double* b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

// FP64 value -> FP32 (round to nearest) -> bfloat16, rounding the 16
// dropped bits to nearest with ties to even (NaN kept quiet)
__global__ void k_d2bf(long long n, const double* a, bf16s* b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned u = __float_as_uint(__double2float_rn(a[i]));
    unsigned short h;
    if ((u & 0x7fffffffu) > 0x7f800000u) h = (unsigned short)((u >> 16) | 0x0040u);
    else h = (unsigned short)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
    b[i].bits = h;
}

// the FP64 operator S with its values rounded to bfloat16 (no diagonal split)
void copy_sell_bf16(const Sell<double>& S, Sell<float, bf16s>& out, cudaStream_t st)
{
    if (S.ndiag) fail(AIRG_ERR_STATE, "bfloat16 copy of an operator with a dense diagonal");
    out.n_rows = S.n_rows;
    out.n_cols = S.n_cols;
    out.n_slices = S.n_slices;
    out.k = S.k;
    out.r = S.r;
    out.nnz = S.nnz;
    out.padded = S.padded;
    out.ndiag = 0;
    out.sptr.alloc(S.sptr.n);
    out.col.alloc(S.col.n);
    out.val.alloc(S.val.n);
    CK(cudaMemcpyAsync(out.sptr.p, S.sptr.p, S.sptr.bytes(), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(out.col.p, S.col.p, S.col.bytes(), cudaMemcpyDeviceToDevice, st));
    if (S.val.n) k_d2bf<<<grid_for(S.val.n, TB), TB, 0, st>>>((long long)S.val.n, S.val.p, out.val.p);
    CK_LAUNCH();
}

void copy_sell_f32(const Sell<double>& S, Sell<float>& out, cudaStream_t st)
{
    out.n_rows = S.n_rows;
    out.n_cols = S.n_cols;
    out.n_slices = S.n_slices;
    out.k = S.k;
    out.r = S.r;
    out.nnz = S.nnz;
    out.padded = S.padded;
    out.ndiag = S.ndiag;
    out.sptr.alloc(S.sptr.n);
    out.col.alloc(S.col.n);
    out.val.alloc(S.val.n);
    CK(cudaMemcpyAsync(out.sptr.p, S.sptr.p, S.sptr.bytes(), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(out.col.p, S.col.p, S.col.bytes(), cudaMemcpyDeviceToDevice, st));
    if (S.val.n) k_d2f<<<grid_for(S.val.n, TB), TB, 0, st>>>((long long)S.val.n, S.val.p, out.val.p);
    if (S.diag.n) {
        out.diag.alloc(S.diag.n);
        k_d2f<<<grid_for(S.diag.n, TB), TB, 0, st>>>((long long)S.diag.n, S.diag.p, out.diag.p);
    }
    CK_LAUNCH();
}

// ------------------------------------------------------- nested ordering --
// Nested positions.  perm (may be null: identity) places the F points of a
// level, or the coarsest level's unknowns, inside their block.
__global__ void k_pos_coarse(int n, int off, const int* perm, int* pos)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pos[i] = off + (perm ? perm[i] : i);
}

__global__ void k_pos_level(int n, const int8_t* is_f, const int* f_index, const int* c_index,
                            int off, const int* perm_f, const int* pos_next, int* pos)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    pos[i] = is_f[i] ? off + (perm_f ? perm_f[f_index[i]] : f_index[i]) : pos_next[c_index[i]];
}

__global__ void k_rel(int n, const int* pos, int off, int* rel, int* inv)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = pos[i] - off;
    rel[i] = r;
    if (inv) inv[r] = i;
}

// W of F point i (C-local target) -> relative C position, stored at the F
// point's position in its block
__global__ void k_map_w(int nf, const int* W, const int* rel, const int* perm_f, int* out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nf) out[perm_f ? perm_f[i] : i] = W[i] >= 0 ? rel[W[i]] : -1;
}

__global__ void k_invert_perm(int n, const int* perm, int* inv)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) inv[perm[i]] = i;
}

// ------------------------------------------------------- V-cycle kernels --
// Row r of S times x.  K == 1: SELL-32, one thread per row.  K > 1: CSR,
// K consecutive lanes share a row (strided over its entries, so a group's
// loads are contiguous) and reduce with shuffles; the sum is valid in the
// group's first lane.  Every lane of a warp reaches the shuffles.
// Sum of val[idx] * x[col[idx]] over idx = first, first + stride, ... < end.
// The j-th entry of the sequence goes to partial sum j mod 4 (each partial
// in entry order) and the result is (p0 + p1) + (p2 + p3), whatever U is.
// Full chunks of U entries issue their U loads before their gathers, so
// each lane keeps U requests in flight; the remainder runs in chunks of 4,
// so at most 3 issued slots per row carry no entry (predicated slots still
// occupy the FP64 pipe, which is the scarce unit for FP64 on this part).
template <bool C16>
__device__ __forceinline__ int ldcol(const int* __restrict__ col, const unsigned short* __restrict__ col16, int cb,
                                     int i)
{
    if constexpr (C16) return cb + int(__ldg(col16 + i));
    else return __ldg(col + i);
}

// C16: column indices from the 16-bit copy, cb + col16 (the same values)
template <class T, int U = 4, class V = T, bool C16 = false>
__device__ __forceinline__ T strided_dot(const int* __restrict__ col, const unsigned short* __restrict__ col16,
                                         int cb, const V* __restrict__ val, const T* __restrict__ x, int idx,
                                         int end, int stride)
{
    static_assert(U % 4 == 0, "U must be a multiple of 4");
    T a[4] = {T(0), T(0), T(0), T(0)};
    for (; idx + (U - 1) * stride < end; idx += U * stride) {
        int c[U];
        T v[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            c[u] = ldcol<C16>(col, col16, cb, idx + u * stride);
            v[u] = ldval<T>(val + idx + u * stride);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) xv[u] = x[c[u]];
#pragma unroll
        for (int u = 0; u < U; ++u) a[u % 4] = fma(v[u], xv[u], a[u % 4]);
    }
    for (; idx < end; idx += 4 * stride) {
        int c[4];
        T v[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool ok = idx + u * stride < end;
            c[u] = ok ? ldcol<C16>(col, col16, cb, idx + u * stride) : 0;
            v[u] = ok ? ldval<T>(val + idx + u * stride) : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = idx + u * stride < end ? x[c[u]] : T(0);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (idx + u * stride < end) a[u] = fma(v[u], xv[u], a[u]);
    }
    return (a[0] + a[1]) + (a[2] + a[3]);
}

// Row (32*slice + lane) of S times x, computed by the P warps of the block
// that share the slice (part = this warp's index among them).  Every thread
// of the block must call it (it synchronises the block when P > 1).  The
// sum is valid in the part-0 warp, which also adds the dense diagonal.
template <class T, int P, int U = 4, class V = T, bool C16 = false>
__device__ __forceinline__ T row_dot(const SellView<T, V>& S, int slice, int lane, int part,
                                     const T* __restrict__ x)
{
    T acc = T(0);
    if (slice < S.n_slices) {
        int b = S.sptr[slice], w = (S.sptr[slice + 1] - b) >> 5;
        const int cb = C16 && S.cbase ? __ldg(S.cbase + slice) : 0;
        acc = strided_dot<T, U, V, C16>(S.col, S.col16, cb, S.val, x, b + lane + 32 * part, b + lane + 32 * w,
                                        32 * P);
    }
    if (P > 1) {
        __shared__ T red[32][32];
        const int warp = threadIdx.x >> 5;
        red[warp][lane] = acc;
        __syncthreads();
        if (part == 0) {
#pragma unroll
            for (int q = 1; q < P; ++q) acc += red[warp + q][lane];
        }
        __syncthreads();
    }
    const int r = slice * 32 + lane;
    if (S.diag && part == 0 && r < S.n_rows) acc = fma(S.diag[r], x[r], acc);
    return acc;
}

// Rows 32 s + lane, s = s0 .. s0+R-1, of S times x for one warp (short rows,
// one warp per slice).  Per row the arithmetic is fixed: start from
// diag_r x_r (or 0), then add the row's stored entries in slice order with
// one fused multiply-add each.  It does not depend on R or on which path
// below runs, so the slices-per-warp choice never changes a result bit.
// When every slice is at most 4 wide, all loads of the R rows are issued
// (predicated) before their gathers, and all gathers before the sums.
template <class T, int R, class V, bool C16 = false>
__device__ __forceinline__ void dot_slices(const SellView<T, V>& S, const T* __restrict__ x, int s0, int lane,
                                           T (&acc)[R])
{
    int b[R], w[R], cb[R];
    bool fits = true;
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int s = s0 + q;
        const bool ok = s < S.n_slices;
        const int p0 = ok ? __ldg(S.sptr + s) : 0, p1 = ok ? __ldg(S.sptr + s + 1) : 0;
        cb[q] = C16 && ok && S.cbase ? __ldg(S.cbase + s) : 0;
        b[q] = p0 + lane;
        w[q] = (p1 - p0) >> 5;
        fits = fits && w[q] <= 4;
        const int r = s * 32 + lane;
        acc[q] = (S.diag && r < S.n_rows) ? __ldg(S.diag + r) * x[r] : T(0);
    }
    if (fits) {
        int c[R][4];
        T v[R][4], xv[R][4];
#pragma unroll
        for (int q = 0; q < R; ++q)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = u < w[q];
                c[q][u] = ok ? ldcol<C16>(S.col, S.col16, cb[q], b[q] + 32 * u) : 0;
                v[q][u] = ok ? ldval<T>(S.val + b[q] + 32 * u) : T(0);
            }
#pragma unroll
        for (int q = 0; q < R; ++q)
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[q][u] = u < w[q] ? x[c[q][u]] : T(0);
#pragma unroll
        for (int q = 0; q < R; ++q)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (u < w[q]) acc[q] = fma(v[q][u], xv[q][u], acc[q]);
    } else {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            for (int u0 = 0; u0 < w[q]; u0 += 4) {
                int c[4];
                T v[4], xv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool ok = u0 + u < w[q];
                    c[u] = ok ? ldcol<C16>(S.col, S.col16, cb[q], b[q] + 32 * (u0 + u)) : 0;
                    v[u] = ok ? ldval<T>(S.val + b[q] + 32 * (u0 + u)) : T(0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) xv[u] = u0 + u < w[q] ? x[c[u]] : T(0);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (u0 + u < w[q]) acc[q] = fma(v[u], xv[u], acc[q]);
            }
        }
    }
}

// Applies epi(r, (S x)_r, pre(r)) to every row r of S.  pre(r) loads the
// row's other operands; it runs before the row's gathers so that its loads
// overlap them.  K = warps per slice.  R = slices per warp for K = 1, and
// loads in flight per lane (4, 8 or 16) for K > 1; in neither case does R
// change the arithmetic.
template <class T, int K, int R, bool C16 = false, class V, class Pre, class Epi>
__device__ __forceinline__ void for_rows(const SellView<T, V>& S, const T* __restrict__ x, const Pre& pre,
                                         const Epi& epi, int rev = 0)
{
    using PV = decltype(pre(0));
    const int lane = threadIdx.x & 31;
    // A grid smaller than the operator's (a resident grid, Sell::persist)
    // strides over the slices; each row is computed the same way either way.
    // rev != 0 takes the groups of slices in reverse order (block 0 the last
    // group): a chain of steps over one operator that alternates the
    // direction starts each step on the lines the previous one left in L2.
    if constexpr (K == 1) {
        const int nw = (gridDim.x * blockDim.x) >> 5;
        const int ngr = (S.n_slices + R - 1) / R;
        for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < ngr; w += nw) {
            const int s0 = (rev ? ngr - 1 - w : w) * R;
            PV pv[R];
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int r = (s0 + q) * 32 + lane;
                pv[q] = r < S.n_rows ? pre(r) : PV{};
            }
            T acc[R];
            dot_slices<T, R, V, C16>(S, x, s0, lane, acc);
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int r = (s0 + q) * 32 + lane;
                if (r < S.n_rows) epi(r, acc[q], pv[q]);
            }
        }
    } else {
        constexpr int SPB = wpb_for(K) / K;   // slices per block-group
        const int part = (threadIdx.x >> 5) % K;
        const int ngroups = (S.n_slices + SPB - 1) / SPB;
        for (int g0 = blockIdx.x; g0 < ngroups; g0 += gridDim.x) {   // uniform over the block
            const int g = rev ? ngroups - 1 - g0 : g0;
            const int slice = g * SPB + (threadIdx.x >> 5) / K;
            const int r = slice * 32 + lane;
            const bool lead = part == 0 && r < S.n_rows;
            PV pv = lead ? pre(r) : PV{};
            T d = row_dot<T, K, R, V, C16>(S, slice, lane, part, x);
            if (lead) epi(r, d, pv);
        }
    }
}

template <class T>
struct Pair {
    T a, b;
};

// y = S x
template <class T, int K, int R, class V = T, bool C16 = false>
__global__ void k_spmv(SellView<T, V> S, const T* __restrict__ x, T* __restrict__ y)
{
    for_rows<T, K, R, C16>(S, x, [](int) { return 0; }, [&](int r, T d, int) { y[r] = d; });
}

// restriction (R = [Z I] of Eq. 4): dst_c[k] = src_c[k] + (Z src_f)[k]; the
// values of Z may be stored narrower than T (V)
template <class T, int K, int R, class V = T, bool C16 = false>
__global__ void k_restrict(SellView<T, V> Z, const T* __restrict__ src_f, const T* __restrict__ src_c,
                           T* __restrict__ dst_c)
{
    for_rows<T, K, R, C16>(Z, src_f, [&](int r) { return src_c[r]; },
                      [&](int r, T d, T sc) { dst_c[r] = sc + d; });
}

// F-point residual (Eq. 6): t = r_f - M e_c, and the first Horner term w = a_p t
template <class T, int K, int R, bool C16 = false>
__global__ void k_fresid(SellView<T> M, const T* __restrict__ rf, const T* __restrict__ ec,
                         T* __restrict__ t, T* __restrict__ w, T ap)
{
    for_rows<T, K, R, C16>(M, ec, [&](int r) { return rf[r]; },
                      [&](int r, T d, T f) {
                          T tt = f - d;
                          t[r] = tt;
                          w[r] = ap * tt;
                      });
}

// Horner term: wout = a_k t + A_ff win
template <class T, int K, int R, bool C16 = false>
__global__ void k_horner(SellView<T> A, const T* __restrict__ t, const T* __restrict__ win,
                         T* __restrict__ wout, T ak, int rev)
{
    for_rows<T, K, R, C16>(A, win, [&](int r) { return t[r]; },
                      [&](int r, T d, T tr) { wout[r] = fma(ak, tr, d); }, rev);
}

// last Horner term and the correction: e_f = W e_c + (a_0 t + A_ff win)
template <class T, int K, int R, bool C16 = false>
__global__ void k_horner_last(SellView<T> A, const T* __restrict__ t, const T* __restrict__ win,
                              const T* __restrict__ ec, const int* __restrict__ W,
                              T* __restrict__ ef, T a0, int rev)
{
    for_rows<T, K, R, C16>(A, win,
                      [&](int r) {
                          int wc = W[r];
                          return Pair<T>{t[r], wc >= 0 ? ec[wc] : T(0)};
                      },
                      [&](int r, T d, Pair<T> q) { ef[r] = q.b + fma(a0, q.a, d); }, rev);
}

// degree-0 smoother: e_f = W e_c + a_0 t
template <class T>
__global__ void k_smooth0(int n, const T* __restrict__ t, const T* __restrict__ ec,
                          const int* __restrict__ W, T* __restrict__ ef, T a0)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int wc = W[r];
    ef[r] = (wc >= 0 ? ec[wc] : T(0)) + a0 * t[r];
}

// last Horner term of a smoother that corrects in place: e += a_0 t + A win
// (the C-point smooth, and the second F-point smooth of FCF)
template <class T, int K, int R, bool C16 = false>
__global__ void k_horner_acc(SellView<T> A, const T* __restrict__ t, const T* __restrict__ win, T* e, T a0,
                             int rev)
{
    for_rows<T, K, R, C16>(A, win, [&](int r) { return Pair<T>{t[r], e[r]}; },
                      [&](int r, T d, Pair<T> q) { e[r] = q.b + fma(a0, q.a, d); }, rev);
}

// degree-0 in-place correction: e += a_0 t
template <class T>
__global__ void k_acc0(int n, const T* __restrict__ t, T* __restrict__ e, T a0)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) e[r] = e[r] + a0 * t[r];
}

template <class T>
__global__ void k_copy(int n, const T* __restrict__ a, T* __restrict__ b)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) b[r] = a[r];
}

// Newton steps of the coarse polynomial (Sec. 2.3)
// real root, not the last: x += r / theta, r' = r - A r / theta
template <class T, int K, int R, bool C16 = false>
__global__ void k_newton_real(SellView<T> A, const T* __restrict__ rin, T* __restrict__ rout,
                              T* __restrict__ x, T inv_theta, int first, int rev)
{
    for_rows<T, K, R, C16>(A, rin, [&](int r) { return Pair<T>{rin[r], first ? T(0) : x[r]}; },
                      [&](int r, T d, Pair<T> q) {
                          x[r] = fma(q.a, inv_theta, q.b);
                          rout[r] = q.a - d * inv_theta;
                      }, rev);
}

// last real root: x += r / theta (no residual update, no SpMV)
template <class T>
__global__ void k_newton_last(int n, const T* __restrict__ rin, T* __restrict__ x, T inv_theta, int first)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    x[r] = fma(rin[r], inv_theta, first ? T(0) : x[r]);
}

template <class T, int K, int R, bool C16 = false>
__global__ void k_newton_pair1(SellView<T> A, const T* __restrict__ rin, T* __restrict__ t,
                               T* __restrict__ x, T two_a, T inv_mod2, int first, int rev)
{
    for_rows<T, K, R, C16>(A, rin, [&](int r) { return Pair<T>{rin[r], first ? T(0) : x[r]}; },
                      [&](int r, T d, Pair<T> q) {
                          T tt = two_a * q.a - d;
                          t[r] = tt;
                          x[r] = fma(tt, inv_mod2, q.b);
                      }, rev);
}

template <class T, int K, int R, bool C16 = false>
__global__ void k_newton_pair2(SellView<T> A, const T* __restrict__ rin, const T* __restrict__ t,
                               T* __restrict__ rout, T inv_mod2, int rev)
{
    for_rows<T, K, R, C16>(A, t, [&](int r) { return rin[r]; },
                      [&](int r, T d, T ri) { rout[r] = ri - d * inv_mod2; }, rev);
}

// ------------------------------------- coarse steps with x in shared memory --
// The coarsest operator is small and dense-ish (at 1024^2, 17k rows of ~170
// entries), and its input vector fits in shared memory.  In this opt-in
// form (tune_coarse_xs) each block first copies the whole of x there (one
// coalesced pass) and every gather then reads shared memory instead of L2.
// The copy takes most of an SM's shared memory, so blocks are XS_THREADS
// wide, one per SM, and loop over groups of slices.  Each row is computed by
// row_dot exactly as in for_rows with the same K and R, so results are
// bit-identical to the unstaged kernels.
constexpr int XS_THREADS = 1024;

template <class T, int K, int R, class V, class Pre, class Epi>
__device__ __forceinline__ void for_rows_xs(const SellView<T, V>& S, const T* __restrict__ x, int n_x,
                                            const Pre& pre, const Epi& epi)
{
    extern __shared__ __align__(16) unsigned char xs_raw[];
    T* xs = reinterpret_cast<T*>(xs_raw);
    for (int i = threadIdx.x; i < n_x; i += XS_THREADS) xs[i] = x[i];
    __syncthreads();
    using PV = decltype(pre(0));
    constexpr int spb = XS_THREADS / 32 / K;
    const int lane = threadIdx.x & 31;
    const int part = (threadIdx.x >> 5) % K;
    const int ngroups = (S.n_slices + spb - 1) / spb;
    for (int g = blockIdx.x; g < ngroups; g += gridDim.x) {   // uniform over the block
        const int slice = g * spb + (threadIdx.x >> 5) / K;
        const int r = slice * 32 + lane;
        const bool lead = part == 0 && r < S.n_rows;
        PV pv = lead ? pre(r) : PV{};
        T d = row_dot<T, K, R, V>(S, slice, lane, part, xs);
        if (lead) epi(r, d, pv);
    }
}

// y = S x (used to time the staged form against the unstaged one)
template <class T, int K, int R>
__global__ void __launch_bounds__(XS_THREADS, 1)
k_spmv_xs(SellView<T> S, const T* __restrict__ x, int n_x, T* __restrict__ y)
{
    for_rows_xs<T, K, R>(S, x, n_x, [](int) { return 0; }, [&](int r, T d, int) { y[r] = d; });
}

template <class T, int K, int R>
__global__ void __launch_bounds__(XS_THREADS, 1)
k_newton_real_xs(SellView<T> A, const T* __restrict__ rin, int n_x, T* __restrict__ rout,
                 T* __restrict__ x, T inv_theta, int first)
{
    for_rows_xs<T, K, R>(A, rin, n_x, [&](int r) { return Pair<T>{rin[r], first ? T(0) : x[r]}; },
                         [&](int r, T d, Pair<T> q) {
                             x[r] = fma(q.a, inv_theta, q.b);
                             rout[r] = q.a - d * inv_theta;
                         });
}

template <class T, int K, int R>
__global__ void __launch_bounds__(XS_THREADS, 1)
k_newton_pair1_xs(SellView<T> A, const T* __restrict__ rin, int n_x, T* __restrict__ t,
                  T* __restrict__ x, T two_a, T inv_mod2, int first)
{
    for_rows_xs<T, K, R>(A, rin, n_x, [&](int r) { return Pair<T>{rin[r], first ? T(0) : x[r]}; },
                         [&](int r, T d, Pair<T> q) {
                             T tt = two_a * q.a - d;
                             t[r] = tt;
                             x[r] = fma(tt, inv_mod2, q.b);
                         });
}

template <class T, int K, int R>
__global__ void __launch_bounds__(XS_THREADS, 1)
k_newton_pair2_xs(SellView<T> A, const T* __restrict__ rin, const T* __restrict__ t, int n_x,
                  T* __restrict__ rout, T inv_mod2)
{
    for_rows_xs<T, K, R>(A, t, n_x, [&](int r) { return rin[r]; },
                         [&](int r, T d, T ri) { rout[r] = ri - d * inv_mod2; });
}

// blocks of wpb_for(P) warps for n rows with P warps per 32-row slice
inline int gk(long long n, int P) { return grid_for((n + 31) / 32, wpb_for(P) / P); }
inline int bk(int P) { return 32 * wpb_for(P); }

// Runs the statement with the compile-time constant KK = kv (warps per slice).
#define WITH_K(kv, ...)                                                         \
    do {                                                                        \
        switch (kv) {                                                           \
            case 1: { constexpr int KK = 1; __VA_ARGS__; } break;               \
            case 2: { constexpr int KK = 2; __VA_ARGS__; } break;               \
            case 4: { constexpr int KK = 4; __VA_ARGS__; } break;               \
            case 8: { constexpr int KK = 8; __VA_ARGS__; } break;               \
            case 16: { constexpr int KK = 16; __VA_ARGS__; } break;             \
            case 32: { constexpr int KK = 32; __VA_ARGS__; } break;             \
            default: fail(AIRG_ERR_STATE, "bad warps-per-slice");               \
        }                                                                       \
    } while (0)

// WITH_K for the long-row layouts only (KK > 1).
#define WITH_K_LONG(kv, ...)                                                    \
    do {                                                                        \
        switch (kv) {                                                           \
            case 2: { constexpr int KK = 2; __VA_ARGS__; } break;               \
            case 4: { constexpr int KK = 4; __VA_ARGS__; } break;               \
            case 8: { constexpr int KK = 8; __VA_ARGS__; } break;               \
            case 16: { constexpr int KK = 16; __VA_ARGS__; } break;             \
            case 32: { constexpr int KK = 32; __VA_ARGS__; } break;             \
            default: fail(AIRG_ERR_STATE, "bad warps-per-slice");               \
        }                                                                       \
    } while (0)

// Grid and block of the row kernels for operator S: K = S.k warps per slice,
// or (K = 1) S.r slices per warp.
// Blocks of `kernel` that fit on the GPU at once (block size `block`),
// looked up once per kernel.
template <class F>
int resident_grid(F* kernel, int block)
{
    static std::mutex mu;
    static std::unordered_map<const void*, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(reinterpret_cast<const void*>(kernel));
    if (it != cache.end()) return it->second;
    int dev = 0, sms = 0, per = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, block, 0));
    const int g = std::max(1, per * sms);
    cache[reinterpret_cast<const void*>(kernel)] = g;
    return g;
}

// Grid of a row kernel for operator S: one block per group of slices (or
// warp per R slices), or with S.persist the resident blocks of `kernel`.
template <class T, class V, class F>
inline int grid_rows(const Sell<T, V>& S, F* kernel)
{
    int g;
    if (S.k > 1) g = gk(S.n_rows, S.k);
    else g = grid_for((S.n_slices + S.r - 1) / S.r, wpb_for(1));
    if (S.persist) g = std::min(g, resident_grid(kernel, bk(S.k)));
    return g;
}
template <class T, class V>
inline int block_rows(const Sell<T, V>& S) { return bk(S.k); }

// Runs the statement with compile-time KK (warps per slice) and RR (slices
// per warp for KK = 1, loads in flight per lane for KK > 1) of operator S.
#define WITH_KR(S, ...)                                                         \
    do {                                                                        \
        if ((S).k == 1) {                                                       \
            constexpr int KK = 1;                                               \
            switch ((S).r) {                                                    \
                case 1: { constexpr int RR = 1; __VA_ARGS__; } break;           \
                case 2: { constexpr int RR = 2; __VA_ARGS__; } break;           \
                case 4: { constexpr int RR = 4; __VA_ARGS__; } break;           \
                default: fail(AIRG_ERR_STATE, "bad slices-per-warp");           \
            }                                                                   \
        } else {                                                                \
            switch ((S).r) {                                                    \
                case 4: { constexpr int RR = 4; WITH_K_LONG((S).k, __VA_ARGS__); } break;   \
                case 8: { constexpr int RR = 8; WITH_K_LONG((S).k, __VA_ARGS__); } break;   \
                case 16: { constexpr int RR = 16; WITH_K_LONG((S).k, __VA_ARGS__); } break; \
                default: fail(AIRG_ERR_STATE, "bad loads-per-lane");            \
            }                                                                   \
        }                                                                       \
    } while (0)

// WITH_KR with the compile-time flag C16 = whether S's row kernels read
// its 16-bit column indices.
#define WITH_KR_COL(S, ...)                                                     \
    do {                                                                        \
        if ((S).col16.n) {                                                      \
            constexpr bool C16 = true;                                          \
            WITH_KR(S, __VA_ARGS__);                                            \
        } else {                                                                \
            constexpr bool C16 = false;                                         \
            WITH_KR(S, __VA_ARGS__);                                            \
        }                                                                       \
    } while (0)

// WITH_KR for the staged coarse kernels: long rows only (S.k > 1), 4 or 8
// loads in flight per lane (their 1024-thread blocks leave 64 registers a
// thread, too few for 16 FP64 loads in flight).
#define WITH_KR_XS(S, ...)                                                      \
    do {                                                                        \
        switch ((S).r) {                                                        \
            case 4: { constexpr int RR = 4; WITH_K_LONG((S).k, __VA_ARGS__); } break;   \
            case 8: { constexpr int RR = 8; WITH_K_LONG((S).k, __VA_ARGS__); } break;   \
            default: fail(AIRG_ERR_STATE, "bad loads-per-lane");                \
        }                                                                       \
    } while (0)

// Grid of the staged coarse kernels: one block per SM, at most one per
// group of slices.  Their dynamic shared memory holds x (n_cols entries).
template <class T>
int xs_grid_for(const Sell<T>& A)
{
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int spb = XS_THREADS / 32 / A.k;
    const int groups = (A.n_slices + spb - 1) / spb;
    return std::max(1, std::min(groups, sms));
}
template <class T>
size_t xs_smem(const Sell<T>& A) { return sizeof(T) * size_t(A.n_cols); }

// ------------------------------------------ persistent coarse polynomial --
// Grid-wide barrier for a cooperative launch.  Thread 0 of each block
// arrives on a counter; the last arrival resets it and advances the
// generation the others wait on.  The wait is bounded: after
// BARRIER_SPIN_LIMIT polls it records an error flag (AIRG_ERR_TIMEOUT on the
// host) and lets the block continue, so a launch that is not co-resident
// ends instead of hanging.
constexpr long long BARRIER_SPIN_LIMIT = 20000000;   // ~1 s of 50 ns polls

// Bounded wait for `expected` arrivals (gridDim.x for a grid barrier).
__device__ __forceinline__ void grid_barrier_n(unsigned* count, unsigned* gen, int* err,
                                               unsigned expected, long long limit)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = gen;
        unsigned g = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(count, 1u);
        if (arrived == expected - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            long long spins = 0;
            while (*vgen == g) {
                if (++spins > limit) { atomicExch(err, 1); break; }
                __nanosleep(50);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

__device__ __forceinline__ void grid_barrier(unsigned* count, unsigned* gen, int* err)
{
    grid_barrier_n(count, gen, err, gridDim.x, BARRIER_SPIN_LIMIT);
}

// Failure-detection check: one block waits for an arrival that never comes
// (expected = 2 with a single block) and must give up after `limit` polls.
__global__ void k_barrier_timeout_check(unsigned* state, long long limit)
{
    grid_barrier_n(state, state + 1, reinterpret_cast<int*>(state + 2), 2u, limit);
}

// x = q(A) b with the Newton roots of Sec. 2.3 (real: x += r/th, r -= A r/th;
// pair a+-ib: t = 2a r - A r, x += t/|th|^2, r -= A t/|th|^2), all steps in one
// cooperative launch: one SpMV per phase, grid barrier between phases.
// Blocks loop over groups of 8/P slices (same SELL-32 x P mapping as the
// other kernels).  roots[2i], roots[2i+1] = (re, im), im == 0 for real.
template <class T, int P>
__global__ void __launch_bounds__(32 * wpb_for(P))
k_newton_persistent(SellView<T> A, const T* __restrict__ b, T* __restrict__ x,
                    T* __restrict__ r0, T* __restrict__ r1, T* __restrict__ t,
                    const double* __restrict__ roots, int nroots, unsigned* bar_count,
                    unsigned* bar_gen, int* err)
{
    const int lane = threadIdx.x & 31;
    const int part = (threadIdx.x >> 5) % P;
    const int sl = (threadIdx.x >> 5) / P;
    const int spb = wpb_for(P) / P;
    const int ngroups = (A.n_slices + spb - 1) / spb;
    const int n = A.n_rows;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    const T* rin = b;
    T* rbuf[2] = {r0, r1};
    int nb = 0;
    for (int i = 0; i < nroots; ++i) {
        const bool last = i == nroots - 1;
        const T xz = T(0);
        const double re = roots[2 * i], im = roots[2 * i + 1];
        T* rout = rbuf[nb];
        if (im == 0.0) {
            const T inv = T(1.0 / re);
            if (last) {
                for (int q = gt; q < n; q += nt) x[q] = fma(rin[q], inv, i == 0 ? xz : x[q]);
            } else {
                for (int g = blockIdx.x; g < ngroups; g += gridDim.x) {
                    const int slice = g * spb + sl, row = slice * 32 + lane;
                    T d = row_dot<T, P>(A, slice, lane, part, rin);
                    if (part == 0 && row < n) {
                        T ri = rin[row];
                        x[row] = fma(ri, inv, i == 0 ? xz : x[row]);
                        rout[row] = ri - d * inv;
                    }
                }
            }
        } else {
            const T two_a = T(2.0 * re), inv2 = T(1.0 / (re * re + im * im));
            for (int g = blockIdx.x; g < ngroups; g += gridDim.x) {
                const int slice = g * spb + sl, row = slice * 32 + lane;
                T d = row_dot<T, P>(A, slice, lane, part, rin);
                if (part == 0 && row < n) {
                    T tt = two_a * rin[row] - d;
                    t[row] = tt;
                    x[row] = fma(tt, inv2, i == 0 ? xz : x[row]);
                }
            }
            if (!last) {
                grid_barrier(bar_count, bar_gen, err);
                for (int g = blockIdx.x; g < ngroups; g += gridDim.x) {
                    const int slice = g * spb + sl, row = slice * 32 + lane;
                    T d = row_dot<T, P>(A, slice, lane, part, t);
                    if (part == 0 && row < n) rout[row] = rin[row] - d * inv2;
                }
            }
        }
        if (!last) {
            grid_barrier(bar_count, bar_gen, err);
            rin = rout;
            nb ^= 1;
        }
    }
}

// Row dot for a runtime number P of warps per slice (1024-thread blocks).
template <class T>
__device__ __forceinline__ T row_dot_rt(const SellView<T>& S, int slice, int lane, int part, int P,
                                        const T* __restrict__ x, T (*red)[32])
{
    T acc = T(0);
    if (slice < S.n_slices) {
        int b = S.sptr[slice], w = (S.sptr[slice + 1] - b) >> 5;
        acc = strided_dot(S.col, S.col16, 0, S.val, x, b + lane + 32 * part, b + lane + 32 * w, 32 * P);
    }
    if (P > 1) {
        const int warp = threadIdx.x >> 5;
        red[warp][lane] = acc;
        __syncthreads();
        if (part == 0)
            for (int q = 1; q < P; ++q) acc += red[warp + q][lane];
        __syncthreads();
    }
    const int r = slice * 32 + lane;
    if (S.diag && part == 0 && r < S.n_rows) acc = fma(S.diag[r], x[r], acc);
    return acc;
}

struct Coefs {
    double a[32];
};

// F-point smoothing of one level (Eq. 6) in one cooperative launch:
//   phase 0: t = r_f - M e_c, w = a_p t
//   phase k (k = p-1..1): w' = a_k t + A_ff w
//   last:   e_f = W e_c + a_0 t + A_ff w
// with a grid barrier between phases (p barriers).  Blocks of 1024 threads
// loop over groups of 32/P slices of each operator.
template <class T>
__global__ void __launch_bounds__(1024)
k_smooth_persistent(SellView<T> M, int pm, SellView<T> A, int pa, const T* __restrict__ rf,
                    const T* __restrict__ ec, const int* __restrict__ W, T* __restrict__ ef,
                    T* __restrict__ t, T* __restrict__ wa, T* __restrict__ wb, Coefs al, int p,
                    unsigned* bar_count, unsigned* bar_gen, int* err)
{
    __shared__ T red[32][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = A.n_rows;
    {
        const int part = warp % pm, spb = 32 / pm, ng = (M.n_slices + spb - 1) / spb;
        const T ap = T(al.a[p]);
        for (int g = blockIdx.x; g < ng; g += gridDim.x) {
            const int slice = g * spb + warp / pm, row = slice * 32 + lane;
            T d = row_dot_rt(M, slice, lane, part, pm, ec, red);
            if (part == 0 && row < n) {
                T tt = rf[row] - d;
                t[row] = tt;
                if (p > 0) wa[row] = ap * tt;
                else {
                    int wc = W[row];
                    ef[row] = (wc >= 0 ? ec[wc] : T(0)) + T(al.a[0]) * tt;
                }
            }
        }
    }
    const int part = warp % pa, spb = 32 / pa, ng = (A.n_slices + spb - 1) / spb;
    const T* win = wa;
    T* wout = wb;
    for (int k = p - 1; k >= 0; --k) {
        grid_barrier(bar_count, bar_gen, err);
        const T ak = T(al.a[k]);
        for (int g = blockIdx.x; g < ng; g += gridDim.x) {
            const int slice = g * spb + warp / pa, row = slice * 32 + lane;
            T d = row_dot_rt(A, slice, lane, part, pa, win, red);
            if (part == 0 && row < n) {
                T v = fma(ak, t[row], d);
                if (k > 0) wout[row] = v;
                else {
                    int wc = W[row];
                    ef[row] = (wc >= 0 ? ec[wc] : T(0)) + v;
                }
            }
        }
        const T* tmp = wout;
        wout = const_cast<T*>(win);
        win = tmp;
    }
}

// ---------------------------------------------------------- Krylov kernels --
constexpr int RB = 256;          // reduction block
constexpr int RGRID = 1216;      // partial sums per reduction (8 x SMs)

// Basis vectors are handled in chunks of at most MCH per kernel, each
// kernel compiled for its exact chunk size (a predicated maximum-size chunk
// costs as much as a full one).
constexpr int MCH = 16;

// out[i] = <w, V_i> for i < M, and out[M] = <w, w> when selfdot, as one
// pass over the rows.  Blocks write partial sums; the last block to finish
// (atomic ticket) adds them in a fixed order and resets the ticket.
template <int M>
__global__ void __launch_bounds__(RB)
k_multidot(long long n, const double* __restrict__ V, long long ldv, const double* __restrict__ w,
           double* __restrict__ part, double* __restrict__ out, unsigned* ticket, int selfdot)
{
    constexpr int MO = M + 1;
    __shared__ double red[RB / 32][MO];
    __shared__ bool last_block;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m = M + (selfdot ? 1 : 0);
    double acc[MO];
#pragma unroll
    for (int u = 0; u < MO; ++u) acc[u] = 0.0;
    for (long long r = (long long)blockIdx.x * RB + threadIdx.x; r < n; r += (long long)gridDim.x * RB) {
        const double wv = __ldg(w + r);
#pragma unroll
        for (int u = 0; u < M; ++u) acc[u] = fma(__ldg(V + u * ldv + r), wv, acc[u]);
        acc[M] = fma(wv, wv, acc[M]);
    }
#pragma unroll
    for (int u = 0; u < MO; ++u) {
        double v = acc[u];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][u] = v;
    }
    __syncthreads();
    if (threadIdx.x < m) {
        double t = 0.0;
        for (int q = 0; q < RB / 32; ++q) t += red[q][threadIdx.x];
        part[(long long)blockIdx.x * m + threadIdx.x] = t;
    }
    __threadfence();
    if (threadIdx.x == 0) last_block = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last_block) return;
    __threadfence();
    const int nb = gridDim.x;
    for (int i = warp; i < m; i += RB / 32) {
        double v = 0.0;
        for (int q = lane; q < nb; q += 32) v += part[(long long)q * m + i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) out[i] = v;
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

// w += sum_i c_i V_i with c_i = -h_i (neg) or h_i, the terms added in the
// order i = 0, 1, ...; with norm, *out = ||w||^2 of the result (partial sums
// per block, fixed-order sum in the last block).
template <int M>
__global__ void __launch_bounds__(RB)
k_multiaxpy(long long n, const double* __restrict__ V, long long ldv, const double* __restrict__ h, int neg,
            double* __restrict__ w, int norm, double* __restrict__ part, double* __restrict__ out,
            unsigned* ticket)
{
    __shared__ double red[RB / 32];
    __shared__ bool last_block;
    double c[M];
#pragma unroll
    for (int u = 0; u < M; ++u) c[u] = neg ? -h[u] : h[u];
    double ss = 0.0;
    for (long long r = (long long)blockIdx.x * RB + threadIdx.x; r < n; r += (long long)gridDim.x * RB) {
        double v[M];
#pragma unroll
        for (int u = 0; u < M; ++u) v[u] = __ldg(V + u * ldv + r);
        double s = w[r];
#pragma unroll
        for (int u = 0; u < M; ++u) s = fma(c[u], v[u], s);
        w[r] = s;
        ss = fma(s, s, ss);
    }
    if (!norm) return;
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < RB / 32; ++q) t += red[q];
        part[blockIdx.x] = t;
    }
    __threadfence();
    if (threadIdx.x == 0) last_block = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last_block) return;
    __threadfence();
    double s = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += RB) s += part[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < RB / 32; ++q) t += red[q];
        *out = t;
        *ticket = 0u;
    }
}


__global__ void k_scale_into(long long n, const double* __restrict__ w, double inv, double* __restrict__ v)
{
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) v[r] = w[r] * inv;
}

// r = b - y
// x += z, unless *active is 0 (a frozen problem of a batch)
__global__ void k_add_dev(long long n, const double* __restrict__ z, const int* __restrict__ active,
                          double* __restrict__ x)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (active && !*active)) return;
    x[i] += z[i];
}

__global__ void k_sub2(long long n, const double* b, const double* y, double* r)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = b[i] - y[i];
}

// nested <-> natural permutation
__global__ void k_to_nested(long long n, const int* pos, const double* a, double* b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[pos[i]] = a[i];
}
__global__ void k_from_nested(long long n, const int* pos, const double* a, double* b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[pos[i]];
}

// ------------------------------------------------------------ V-cycle ----
template <class T>
struct VWork {
    T* rwork; T* t; T* wa; T* wb; T* cx; T* cr0; T* cr1; T* ct;
    T* rcs;    // C residuals before restriction (C-point smoothing)
};

template <class T>
const SolveLevelT<T>& ops(const SolveLevel& L);
template <>
const SolveLevelT<double>& ops<double>(const SolveLevel& L) { return L.d; }
template <>
const SolveLevelT<float>& ops<float>(const SolveLevel& L) { return L.f; }

template <class T>
const Sell<T>& coarse_op(const SolveData& S);
template <>
const Sell<double>& coarse_op<double>(const SolveData& S) { return S.Ac; }
template <>
const Sell<float>& coarse_op<float>(const SolveData& S) { return S.Ac32; }

// grid of the persistent coarse kernel (0 if no block can be resident)
template <class T>
int newton_persistent_grid(const Sell<T>& A)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (A.n_rows < 1) return 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    WITH_K(A.k, CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_newton_persistent<T, KK>, bk(KK), 0)));
    if (per_sm < 1) return 0;
    int spb = wpb_for(A.k) / A.k;
    int groups = (A.n_slices + spb - 1) / spb;
    return std::min(groups, per_sm * sms);
}

// Prolongation and the F-point smooth of level l (Eq. 6): t = r_f - M e_c
// with M = A_fc + A_ff W, then e_f = W e_c + q(A_ff) t
template <class T>
void f_smooth(SolveData& S, int l, const T* v, T* e, const VWork<T>& wk, cudaStream_t st)
{
    constexpr long long VB = sizeof(T);
    const SolveLevel& lv = *S.lv[l];
    const T* src = l == 0 ? v : wk.rwork;
    const SolveLevelT<T>& o = ops<T>(lv);
    const T* rf = src + lv.off;
    const T* ec = e + lv.off + lv.n_f;
    T* ef = e + lv.off;
    int nf = lv.n_f;
    int g = grid_for(nf, TB);
    int p = int(lv.alpha.size()) - 1;
    const long long fB = (long long)nf * VB;
    const int pidx2 = sizeof(T) == 8 ? 0 : 1;
    S.cur_level = l;
    if (o.Ainv.n_rows) {
        // assembled smoother (Eq. 8 matrix): t = r_f - M e_c, then
        // e_f = W e_c + Ahat^-1 t, the last Horner kernel with a0 = 0
        LAUNCH_F(S, PK_FRESID, mat_bytes(o.M) + (long long)lv.n_c * VB + 3 * fB, 2 * o.M.nnz + 2LL * nf,
                 WITH_KR_COL(o.M, launch_kernel(st, grid_rows(o.M, k_fresid<T, KK, RR, C16>), block_rows(o.M), 0, k_fresid<T, KK, RR, C16>,
                                  view(o.M), rf, ec, wk.t, wk.wa, T(0))));
        LAUNCH_F(S, PK_HORNER, mat_bytes(o.Ainv) + 4 * fB + 4LL * nf, 2 * o.Ainv.nnz + 3LL * nf,
                 WITH_KR_COL(o.Ainv, launch_kernel(st, grid_rows(o.Ainv, k_horner_last<T, KK, RR, C16>), block_rows(o.Ainv), 0, k_horner_last<T, KK, RR, C16>,
                                     view(o.Ainv), wk.t, wk.t, ec, lv.W.p, ef, T(0), 0)));
        return;
    }
    if (S.smooth_grid[pidx2] > 0 && p < 32) {
        Coefs al{};
        for (int q = 0; q <= p; ++q) al.a[q] = lv.alpha[q];
        int need = std::max((o.M.n_slices + 32 / o.M.k - 1) / (32 / o.M.k),
                            (o.Aff.n_slices + 32 / o.Aff.k - 1) / (32 / o.Aff.k));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(std::max(1, std::min(S.smooth_grid[pidx2], need)));
        cfg.blockDim = dim3(1024);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        long long bytes = mat_bytes(o.M) + (long long)lv.n_c * VB + 3 * fB +
                          p * (mat_bytes(o.Aff) + 3 * fB) + fB + 4LL * nf;
        SellView<T> Mv = view(o.M), Av2 = view(o.Aff);
        const long long flops = 2 * o.M.nnz + 2LL * nf + p * (2 * o.Aff.nnz + 2LL * nf) + nf;
        LAUNCH_F(S, PK_HORNER, bytes, flops,
               CK(cudaLaunchKernelEx(&cfg, k_smooth_persistent<T>, Mv, o.M.k, Av2, o.Aff.k, rf, ec,
                                     (const int*)lv.W.p, ef, wk.t, wk.wa, wk.wb, al, p, S.bar.p,
                                     S.bar.p + 1, (int*)(S.bar.p + 2))));
        return;
    }
    LAUNCH_F(S, PK_FRESID, mat_bytes(o.M) + (long long)lv.n_c * VB + 3 * fB, 2 * o.M.nnz + 2LL * nf,
           WITH_KR_COL(o.M, launch_kernel(st, grid_rows(o.M, k_fresid<T, KK, RR, C16>), block_rows(o.M), 0, k_fresid<T, KK, RR, C16>,
                            view(o.M), rf, ec, wk.t, wk.wa, T(lv.alpha[p]))));
    if (p == 0) {
        LAUNCH_F(S, PK_HORNER, 3 * fB + 4LL * nf, 3LL * nf,
               launch_kernel(st, g, TB, 0, k_smooth0<T>, nf, wk.t, ec, lv.W.p, ef, T(lv.alpha[0])));
        return;
    }
    const long long hB = mat_bytes(o.Aff) + 3 * fB;
    T* win = wk.wa;
    T* wout = wk.wb;
    // the p SpMVs with A_ff alternate their direction (serpentine order)
    for (int k = p - 1; k >= 1; --k) {
        LAUNCH_F(S, PK_HORNER, hB, 2 * o.Aff.nnz + 2LL * nf,
               WITH_KR_COL(o.Aff, launch_kernel(st, grid_rows(o.Aff, k_horner<T, KK, RR, C16>), block_rows(o.Aff), 0, k_horner<T, KK, RR, C16>,
                                  view(o.Aff), wk.t, win, wout, T(lv.alpha[k]), serpentine(p - 1 - k))));
        std::swap(win, wout);
    }
    LAUNCH_F(S, PK_HORNER, hB + fB + 4LL * nf, 2 * o.Aff.nnz + 3LL * nf,
           WITH_KR_COL(o.Aff, launch_kernel(st, grid_rows(o.Aff, k_horner_last<T, KK, RR, C16>), block_rows(o.Aff), 0, k_horner_last<T, KK, RR, C16>,
                              view(o.Aff), wk.t, win, ec, lv.W.p, ef, T(lv.alpha[0]), serpentine(p - 1))));
}

// e += q(A) t by Horner, with w = a_p t already in wk.wa (written by the
// residual kernel) and t in wk.t; n rows
template <class T>
void horner_into(SolveData& S, const Sell<T>& A, const std::vector<double>& al, const VWork<T>& wk, T* e,
                 int n, cudaStream_t st)
{
    constexpr long long VB = sizeof(T);
    const int p = int(al.size()) - 1;
    const long long fB = (long long)n * VB;
    if (p == 0) {
        LAUNCH_F(S, PK_HORNER, 3 * fB, 2LL * n, launch_kernel(st, grid_for(n, TB), TB, 0, k_acc0<T>, n, wk.t, e, T(al[0])));
        return;
    }
    const long long hB = mat_bytes(A) + 3 * fB;
    T* win = wk.wa;
    T* wout = wk.wb;
    for (int k = p - 1; k >= 1; --k) {
        LAUNCH_F(S, PK_HORNER, hB, 2 * A.nnz + 2LL * n,
                 WITH_KR_COL(A, launch_kernel(st, grid_rows(A, k_horner<T, KK, RR, C16>), block_rows(A), 0, k_horner<T, KK, RR, C16>, view(A), wk.t, win,
                                       wout, T(al[k]), serpentine(p - 1 - k))));
        std::swap(win, wout);
    }
    LAUNCH_F(S, PK_HORNER, hB + fB, 2 * A.nnz + 3LL * n,
             WITH_KR_COL(A, launch_kernel(st, grid_rows(A, k_horner_acc<T, KK, RR, C16>), block_rows(A), 0, k_horner_acc<T, KK, RR, C16>, view(A), wk.t, win, e,
                                   T(al[0]), serpentine(p - 1))));
}

// C-point smooth of level l (Sec. 2): t_c = r_c - [A_cf A_cc] e_l with the
// level's C residual from before restriction, then e_c += q_c(A_cc) t_c
template <class T>
void c_smooth(SolveData& S, int l, const T* v, T* e, const VWork<T>& wk, cudaStream_t st)
{
    constexpr long long VB = sizeof(T);
    const SolveLevel& lv = *S.lv[l];
    const SolveLevelT<T>& o = ops<T>(lv);
    const int nc = lv.n_c;
    if (!nc) return;
    const T* rc = l == 0 ? v + lv.off + lv.n_f : wk.rcs + lv.rc_off;
    T* el = e + lv.off;
    const int p = int(lv.alpha_c.size()) - 1;
    const long long cB = (long long)nc * VB;
    LAUNCH_F(S, PK_FRESID, mat_bytes(o.Mc) + (long long)(lv.n_f + nc) * VB + 3 * cB, 2 * o.Mc.nnz + 2LL * nc,
             WITH_KR_COL(o.Mc, launch_kernel(st, grid_rows(o.Mc, k_fresid<T, KK, RR, C16>), block_rows(o.Mc), 0, k_fresid<T, KK, RR, C16>,
                              view(o.Mc), rc, el, wk.t, wk.wa, T(lv.alpha_c[p]))));
    if (o.Ainvc.n_rows) {   // assembled: e_c += Ahat_cc^-1 t_c
        LAUNCH_F(S, PK_HORNER, mat_bytes(o.Ainvc) + 4 * cB, 2 * o.Ainvc.nnz + 2LL * nc,
                 WITH_KR_COL(o.Ainvc, launch_kernel(st, grid_rows(o.Ainvc, k_horner_acc<T, KK, RR, C16>), block_rows(o.Ainvc), 0, k_horner_acc<T, KK, RR, C16>,
                                     view(o.Ainvc), wk.t, wk.t, el + lv.n_f, T(0), 0)));
        return;
    }
    horner_into<T>(S, o.Acc, lv.alpha_c, wk, el + lv.n_f, nc, st);
}

// second F-point smooth of FCF: t = r_f - [A_ff A_fc] e_l, e_f += q(A_ff) t
template <class T>
void f_smooth_again(SolveData& S, int l, const T* v, T* e, const VWork<T>& wk, cudaStream_t st)
{
    constexpr long long VB = sizeof(T);
    const SolveLevel& lv = *S.lv[l];
    const SolveLevelT<T>& o = ops<T>(lv);
    const int nf = lv.n_f;
    if (!nf) return;
    const T* rf = (l == 0 ? v : wk.rwork) + lv.off;
    T* el = e + lv.off;
    const int p = int(lv.alpha.size()) - 1;
    const long long fB = (long long)nf * VB;
    LAUNCH_F(S, PK_FRESID, mat_bytes(o.Mf) + (long long)(nf + lv.n_c) * VB + 3 * fB, 2 * o.Mf.nnz + 2LL * nf,
             WITH_KR_COL(o.Mf, launch_kernel(st, grid_rows(o.Mf, k_fresid<T, KK, RR, C16>), block_rows(o.Mf), 0, k_fresid<T, KK, RR, C16>,
                              view(o.Mf), rf, el, wk.t, wk.wa, T(lv.alpha[p]))));
    if (o.Ainv.n_rows) {    // assembled: e_f += Ahat_ff^-1 t
        LAUNCH_F(S, PK_HORNER, mat_bytes(o.Ainv) + 4 * fB, 2 * o.Ainv.nnz + 2LL * nf,
                 WITH_KR_COL(o.Ainv, launch_kernel(st, grid_rows(o.Ainv, k_horner_acc<T, KK, RR, C16>), block_rows(o.Ainv), 0, k_horner_acc<T, KK, RR, C16>,
                                    view(o.Ainv), wk.t, wk.t, el, T(0), 0)));
        return;
    }
    horner_into<T>(S, o.Aff, lv.alpha, wk, el, nf, st);
}

// e = M^-1 v in the nested order.  v is only read; e is written everywhere.
template <class T>
void vcycle(SolveData& S, const T* v, T* e, const VWork<T>& wk, cudaStream_t st)
{
    const int L = S.nlev;
    constexpr long long VB = sizeof(T);
    // restriction, top to bottom (level 0 reads v, deeper levels the work vector)
    for (int l = 0; l < L; ++l) {
        const SolveLevel& lv = *S.lv[l];
        const T* src = l == 0 ? v : wk.rwork;
        const Sell<T>& Z = ops<T>(lv).Z;
        const Sell<T, bf16s>& Zb = ops<T>(lv).Zb;
        S.cur_level = l;
        if (l > 0 && lv.n_c && S.smooth_type != AIRG_SMOOTH_F)   // restriction overwrites r_c in place
            LAUNCH_F(S, PK_RESTRICT, 2LL * lv.n_c * VB, 0,
                     launch_kernel(st, grid_for(lv.n_c, TB), TB, 0, k_copy<T>, lv.n_c, src + lv.off + lv.n_f,
                                                                    wk.rcs + lv.rc_off));
        if (lv.n_c && Zb.val.n)
            LAUNCH_F(S, PK_RESTRICT, mat_bytes(Zb) + (2LL * lv.n_c + lv.n_f + lv.n_c) * VB, 2 * Zb.nnz + lv.n_c,
                   WITH_KR_COL(Zb, launch_kernel(st, grid_rows(Zb, k_restrict<T, KK, RR, bf16s, C16>), block_rows(Zb), 0, k_restrict<T, KK, RR, bf16s, C16>,
                                   view(Zb), src + lv.off, src + lv.off + lv.n_f,
                                   wk.rwork + lv.off + lv.n_f)));
        else if (lv.n_c)
            LAUNCH_F(S, PK_RESTRICT, mat_bytes(Z) + (2LL * lv.n_c + lv.n_f + lv.n_c) * VB, 2 * Z.nnz + lv.n_c,
                   WITH_KR_COL(Z, launch_kernel(st, grid_rows(Z, k_restrict<T, KK, RR, T, C16>), block_rows(Z), 0, k_restrict<T, KK, RR, T, C16>,
                                  view(Z), src + lv.off, src + lv.off + lv.n_f,
                                  wk.rwork + lv.off + lv.n_f)));
    }
    // coarse-grid polynomial
    {
        const T* rc = (L == 0 ? v : wk.rwork) + S.off_c;
        T* x = e + S.off_c;
        const Sell<T>& A = coarse_op<T>(S);
        SellView<T> Av = view(A);
        const int nco = S.n_coarse;
        const T* rin = rc;
        T* bufs[2] = {wk.cr0, wk.cr1};
        int nb = 0;
        size_t nr = S.roots.size();
        const long long nB = (long long)S.n_coarse * VB, mB = mat_bytes(A);
        S.cur_level = L;
        const int pidx = sizeof(T) == 8 ? 0 : 1;
        if (S.newton_grid[pidx] > 0 && nr > 0) {
            // all Newton steps in one cooperative launch
            long long bytes = 0, flops = 0;
            for (size_t i = 0; i < nr; ++i) {
                bool last = i + 1 == nr;
                bytes += S.roots[i].im == 0.0 ? (last ? 3 * nB : mB + 4 * nB) : (last ? mB + 4 * nB : 2 * mB + 8 * nB);
                flops += S.roots[i].im == 0.0 ? (last ? 2LL * nco : 2 * A.nnz + 4LL * nco)
                                              : (last ? 2 * A.nnz + 4LL * nco : 4 * A.nnz + 6LL * nco);
            }
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(S.newton_grid[pidx]);
            cfg.blockDim = dim3(bk(A.k));
            cfg.dynamicSmemBytes = 0;
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nroots = int(nr);
            LAUNCH_F(S, PK_NEWTON, bytes, flops,
                   WITH_K(A.k, CK(cudaLaunchKernelEx(&cfg, k_newton_persistent<T, KK>, Av, rc, x, wk.cr0,
                                                     wk.cr1, wk.ct, (const double*)S.roots_dev.p, nroots,
                                                     S.bar.p, S.bar.p + 1, (int*)(S.bar.p + 2)))));
            goto coarse_done;
        }
        int nsp = 0;   // SpMVs with the coarse operator so far (their direction alternates)
        for (size_t i = 0; i < nr; ++i) {
            bool last = i + 1 == nr;
            const Root& q = S.roots[i];
            T* rout = bufs[nb];
            unsigned* serr = reinterpret_cast<unsigned*>(S.bar.p + 2);
            if (q.im == 0.0) {
                if (last)
                    LAUNCH_F(S, PK_NEWTON, (i == 0 ? 2 : 3) * nB, 2LL * nco,
                           launch_kernel(st, grid_for(nco, TB), TB, 0, k_newton_last<T>, nco, rin, x, T(1.0 / q.re), i == 0));
                else if (A.stream)
                    LAUNCH_F(S, PK_NEWTON, mB + 2 * nB + (i == 0 ? 2 : 3) * nB, 2 * A.nnz + 4LL * nco,
                             coarse_stream_launch<T>(A, CS_REAL, rin, nullptr, rout, x, T(1.0 / q.re), T(0), i == 0,
                                                     serr, st));
                else if (A.xs)
                    LAUNCH_F(S, PK_NEWTON, mB + 2 * nB + (i == 0 ? 2 : 3) * nB, 2 * A.nnz + 4LL * nco,
                           WITH_KR_XS(A, launch_kernel(st, A.xs, XS_THREADS, xs_smem(A), k_newton_real_xs<T, KK, RR>,
                                               Av, rin, A.n_cols, rout, x, T(1.0 / q.re), i == 0)));
                else
                    LAUNCH_F(S, PK_NEWTON, mB + 2 * nB + (i == 0 ? 2 : 3) * nB, 2 * A.nnz + 4LL * nco,
                           WITH_KR_COL(A, launch_kernel(st, grid_rows(A, k_newton_real<T, KK, RR, C16>), block_rows(A), 0, k_newton_real<T, KK, RR, C16>,
                                          Av, rin, rout, x, T(1.0 / q.re), i == 0, serpentine(nsp))));
                if (!last) nsp += 1;
            } else {
                double mod2 = q.re * q.re + q.im * q.im;
                if (A.stream)
                    LAUNCH_F(S, PK_NEWTON, mB + (i == 0 ? 3 : 4) * nB, 2 * A.nnz + 4LL * nco,
                             coarse_stream_launch<T>(A, CS_PAIR1, rin, nullptr, wk.ct, x, T(2.0 * q.re),
                                                     T(1.0 / mod2), i == 0, serr, st));
                else if (A.xs)
                    LAUNCH_F(S, PK_NEWTON, mB + (i == 0 ? 3 : 4) * nB, 2 * A.nnz + 4LL * nco,
                           WITH_KR_XS(A, launch_kernel(st, A.xs, XS_THREADS, xs_smem(A), k_newton_pair1_xs<T, KK, RR>,
                                               Av, rin, A.n_cols, wk.ct, x, T(2.0 * q.re), T(1.0 / mod2), i == 0)));
                else
                    LAUNCH_F(S, PK_NEWTON, mB + (i == 0 ? 3 : 4) * nB, 2 * A.nnz + 4LL * nco,
                           WITH_KR_COL(A, launch_kernel(st, grid_rows(A, k_newton_pair1<T, KK, RR, C16>), block_rows(A), 0, k_newton_pair1<T, KK, RR, C16>,
                                          Av, rin, wk.ct, x, T(2.0 * q.re), T(1.0 / mod2), i == 0, serpentine(nsp))));
                if (!last && A.stream)
                    LAUNCH_F(S, PK_NEWTON, mB + 3 * nB, 2 * A.nnz + 2LL * nco,
                             coarse_stream_launch<T>(A, CS_PAIR2, wk.ct, rin, rout, nullptr, T(0), T(1.0 / mod2), 0,
                                                     serr, st));
                else if (!last && A.xs)
                    LAUNCH_F(S, PK_NEWTON, mB + 3 * nB, 2 * A.nnz + 2LL * nco,
                           WITH_KR_XS(A, launch_kernel(st, A.xs, XS_THREADS, xs_smem(A), k_newton_pair2_xs<T, KK, RR>,
                                               Av, rin, wk.ct, A.n_cols, rout, T(1.0 / mod2))));
                else if (!last)
                    LAUNCH_F(S, PK_NEWTON, mB + 3 * nB, 2 * A.nnz + 2LL * nco,
                           WITH_KR_COL(A, launch_kernel(st, grid_rows(A, k_newton_pair2<T, KK, RR, C16>), block_rows(A), 0, k_newton_pair2<T, KK, RR, C16>,
                                          Av, rin, wk.ct, rout, T(1.0 / mod2), serpentine(nsp + 1))));
                nsp += last ? 1 : 2;
            }
            if (!last) { rin = rout; nb ^= 1; }
        }
        if (nr == 0) CK(cudaMemsetAsync(x, 0, sizeof(T) * S.n_coarse, st));
    }
coarse_done:
    // up: prolongation + smoothing, bottom to top
    for (int l = L - 1; l >= 0; --l) {
        S.cur_level = l;
        f_smooth<T>(S, l, v, e, wk, st);
        if (S.smooth_type != AIRG_SMOOTH_F) {
            c_smooth<T>(S, l, v, e, wk, st);
            if (S.smooth_type == AIRG_SMOOTH_FCF) f_smooth_again<T>(S, l, v, e, wk, st);
        }
    }
    S.close_run(st);
    S.cur_level = 0;
    CK_LAUNCH();
}

long long sell_bytes(const Sell<double>& S, int vbytes)
{
    // values + column indices (none for a dense diagonal) + one read of the
    // gathered input + one write
    return (S.nnz - S.ndiag) * (vbytes + (S.col16.n ? 2 : 4)) + S.ndiag * vbytes + 2LL * S.n_rows * vbytes +
           4LL * (long long)S.cbase.n;
}

// Row-kernel variant of every operator, picked by timing y = S x: slices
// per warp r = 1, 2, 4 for short rows (one warp per slice), loads in flight
// per lane r = 4, 8, 16 for long rows (several warps per slice), each with
// the operator's own grid or a resident grid striding over the slices
// (persist; it removes the partly idle last wave).  None of them changes
// the arithmetic.  forced > 0 (AIRG_ROWS_PER_WARP for short rows,
// AIRG_LOADS_PER_LANE for long rows) fixes r, AIRG_PERSIST_GRID=0|1 the
// grid; with both fixed nothing is timed.
// Returns the time of 3 launches of the chosen variant (0 when not timed).
template <class T, class V>
float tune_rows(Sell<T, V>& A, const T* x, T* y, int forced_short, int forced_long, cudaStream_t st)
{
    if (A.n_rows == 0) return 0.f;
    const int forced = A.k == 1 ? forced_short : forced_long;
    const char* pe = getenv("AIRG_PERSIST_GRID");
    const int forced_p = pe && (pe[0] == '0' || pe[0] == '1') ? pe[0] - '0' : -1;
    if (forced && forced_p >= 0) {
        A.r = forced;
        A.persist = forced_p;
        return 0.f;
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 0.f;
    int best_r = A.k == 1 ? 1 : 4, best_p = 0;
    const int cand_short[3] = {1, 2, 4}, cand_long[3] = {4, 8, 16};
    const int* cand = A.k == 1 ? cand_short : cand_long;
    bool first = true;
    for (int ci = 0; ci < 6; ++ci) {
        A.r = forced ? forced : cand[ci % 3];
        A.persist = ci / 3;
        if ((forced && ci % 3) || (forced_p >= 0 && A.persist != forced_p)) continue;
        SellView<T, V> v = view(A);
        auto launch = [&]() {
            WITH_KR_COL(A, k_spmv<T, KK, RR, V, C16><<<grid_rows(A, k_spmv<T, KK, RR, V, C16>), block_rows(A), 0, st>>>(v, x, y));
        };
        launch();
        CK_LAUNCH();
        CK(cudaEventRecord(e0, st));
        for (int rep = 0; rep < 3; ++rep) launch();
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (first || ms < best) {
            best = ms;
            best_r = A.r;
            best_p = A.persist;
            first = false;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    A.r = best_r;
    A.persist = best_p;
    return best;
}

// Lets staged kernel `f` take the shared memory of any x that fits beside
// its static shared memory; false if `need` bytes do not fit.
template <class F>
bool xs_allow(F* f, size_t need, int optin)
{
    cudaFuncAttributes fa;
    CK(cudaFuncGetAttributes(&fa, f));
    if (fa.sharedSizeBytes + need > size_t(optin)) return false;
    CK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - int(fa.sharedSizeBytes)));
    return true;
}

template <class T, int K, int R>
bool xs_allow_all(size_t need, int optin)
{
    return xs_allow(k_spmv_xs<T, K, R>, need, optin) && xs_allow(k_newton_real_xs<T, K, R>, need, optin) &&
           xs_allow(k_newton_pair1_xs<T, K, R>, need, optin) && xs_allow(k_newton_pair2_xs<T, K, R>, need, optin);
}

// Staged form of the coarsest operator's SpMVs (x in shared memory, for
// long rows when x fits), opt-in: AIRG_COARSE_XS=1 stages whenever x fits,
// with 4 or 8 loads in flight per lane (the faster by timing y = A x);
// AIRG_COARSE_XS=2 stages only when that also times faster than the best
// unstaged form (`unstaged_ms` for 3 launches, 0 when not timed).  Neither
// form changes the arithmetic.  Off by default: on the 1024^2 workload the
// staged step measured 17.6 against 17.0 us, since the step is bound by the
// FP64 pipe and the matrix loads, not by the gathers of x.
template <class T>
void tune_coarse_xs(Sell<T>& A, float unstaged_ms, const T* x, T* y, cudaStream_t st)
{
    A.xs = 0;
    if (A.n_rows == 0 || A.k < 2) return;
    const char* env = getenv("AIRG_COARSE_XS");
    const int mode = env ? atoi(env) : 0;
    if (mode != 1 && mode != 2) return;
    if (mode == 2 && unstaged_ms <= 0.f) return;
    int dev = 0, optin = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t need = xs_smem(A);
    const int r0 = A.r, cand[2] = {4, 8};
    bool fits = true;
    for (int ci = 0; ci < 2 && fits; ++ci) {
        A.r = cand[ci];
        WITH_KR_XS(A, fits = xs_allow_all<T, KK, RR>(need, optin));
    }
    A.r = r0;
    if (!fits) return;
    const int grid = xs_grid_for(A);
    const SellView<T> v = view(A);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = mode == 2 ? unstaged_ms : 0.f;
    int best_r = 0;
    for (int ci = 0; ci < 2; ++ci) {
        A.r = cand[ci];
        WITH_KR_XS(A, k_spmv_xs<T, KK, RR><<<grid, XS_THREADS, need, st>>>(v, x, A.n_cols, y));
        CK_LAUNCH();
        CK(cudaEventRecord(e0, st));
        for (int rep = 0; rep < 3; ++rep)
            WITH_KR_XS(A, k_spmv_xs<T, KK, RR><<<grid, XS_THREADS, need, st>>>(v, x, A.n_cols, y));
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if ((mode == 1 && best_r == 0) || ms < best) {   // mode 1: the faster R
            best = ms;
            best_r = cand[ci];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    A.r = best_r ? best_r : r0;
    A.xs = best_r ? grid : 0;
}

// Streamed form of the coarsest operator's steps (coarse_stream.cu),
// opt-in: AIRG_COARSE_STREAM=1 uses it whenever the layout allows, =2 only
// where it times faster than the best row-kernel form (`unstaged_ms` for 3
// launches of y = A x).  Off by default: on the 4096^2 workload its step
// measured 37.3 against 35.0 us (FP32) and 86.5 against 56.5 us (FP64).
// Neither form changes the arithmetic.
template <class T>
void tune_coarse_stream(Sell<T>& A, float unstaged_ms, const T* x, T* y, cudaStream_t st)
{
    A.stream = 0;
    const char* env = getenv("AIRG_COARSE_STREAM");
    const int mode = env ? atoi(env) : 0;
    if (mode == 0 || A.xs || !coarse_stream_ok(A)) return;
    if (mode == 1) {
        A.stream = 1;
        return;
    }
    if (unstaged_ms <= 0.f) return;
    DBuf<unsigned> err(1);
    CK(cudaMemsetAsync(err.p, 0, sizeof(unsigned), st));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    coarse_stream_launch<T>(A, CS_SPMV, x, nullptr, y, nullptr, T(0), T(0), 0, err.p, st);
    CK(cudaEventRecord(e0, st));
    for (int rep = 0; rep < 3; ++rep)
        coarse_stream_launch<T>(A, CS_SPMV, x, nullptr, y, nullptr, T(0), T(0), 0, err.p, st);
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    unsigned bad = 0;
    d2h(&bad, err.p, 1, st);
    if (bad) fail(AIRG_ERR_TIMEOUT, "a bounded wait of the streamed coarse kernel gave up");
    if (ms < unstaged_ms) A.stream = 1;
}

int env_choice(const char* name, std::initializer_list<int> allowed)
{
    const char* e = getenv(name);
    int v = e ? atoi(e) : 0;
    for (int a : allowed)
        if (v == a) return v;
    return 0;
}

template <class T>
void tune_all(SolveData& S, cudaStream_t st)
{
    const int fs = env_choice("AIRG_ROWS_PER_WARP", {1, 2, 4});
    const int fl = env_choice("AIRG_LOADS_PER_LANE", {4, 8, 16});
    size_t n = std::max(S.n0, 1);
    DBuf<T> x(n), y(n);
    CK(cudaMemsetAsync(x.p, 0, x.bytes(), st));
    for (auto& lp : S.lv) {
        SolveLevelT<T>& o = const_cast<SolveLevelT<T>&>(ops<T>(*lp));
        tune_rows(o.Aff, x.p, y.p, fs, fl, st);
        tune_rows(o.M, x.p, y.p, fs, fl, st);
        tune_rows(o.Z, x.p, y.p, fs, fl, st);
        tune_rows(o.Zb, x.p, y.p, fs, fl, st);
        tune_rows(o.Ainv, x.p, y.p, fs, fl, st);
        tune_rows(o.Mc, x.p, y.p, fs, fl, st);
        tune_rows(o.Acc, x.p, y.p, fs, fl, st);
        tune_rows(o.Mf, x.p, y.p, fs, fl, st);
        tune_rows(o.Ainvc, x.p, y.p, fs, fl, st);
    }
    Sell<T>& Ac = const_cast<Sell<T>&>(coarse_op<T>(S));
    const float unstaged = tune_rows(Ac, x.p, y.p, fs, fl, st);
    tune_coarse_xs(Ac, unstaged, x.p, y.p, st);
    tune_coarse_stream(Ac, unstaged, x.p, y.p, st);
    CK(cudaStreamSynchronize(st));
}

}  // namespace

// Order of the rows of a block inside their window: within each window of
// `win` consecutive rows (in the setup's order), rows sorted by decreasing
// stored-entry count, ties by index.  Rows of one SELL slice then have
// nearly equal lengths, which removes most of the slice padding (bytes and
// the FMAs on padding) while keeping every row near its neighbours, so the
// gathers of x stay local.  perm[i] = position of row i in the block; empty
// for win <= 1.  A row's own arithmetic does not change.
std::vector<int> window_sort_perm(const DevCSR& A, int win, cudaStream_t st)
{
    std::vector<int> perm;
    const int n = A.n_rows;
    if (win <= 1 || n == 0) return perm;
    std::vector<int> rp(size_t(n) + 1);
    d2h(rp.data(), A.rp.p, rp.size(), st);
    perm.resize(n);
    std::vector<int> idx;
    for (int w0 = 0; w0 < n; w0 += win) {
        const int w1 = std::min(n, w0 + win);
        idx.resize(w1 - w0);
        for (int i = w0; i < w1; ++i) idx[i - w0] = i;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
            return rp[a + 1] - rp[a] > rp[b + 1] - rp[b];
        });
        for (int q = 0; q < w1 - w0; ++q) perm[idx[q]] = w0 + q;
    }
    return perm;
}

int sort_window()
{
    const char* e = getenv("AIRG_SORT_WINDOW");
    return e ? std::max(0, atoi(e)) : 256;
}

// ===========================================================================
void build_solve_data(Hierarchy& H, cudaStream_t st)
{
    auto S = std::make_unique<SolveData>();
    const int L = int(H.levels.size());
    S->nlev = L;
    S->n0 = L ? H.levels[0]->n : H.coarse.A.n_rows;
    // offsets
    std::vector<int> off(L + 1, 0);
    for (int l = 0; l < L; ++l) off[l + 1] = off[l] + H.levels[l]->n_f;
    S->off_c = off[L];
    S->n_coarse = H.coarse.A.n_rows;
    // row order inside the F blocks and the coarsest block (window sort)
    const int win = sort_window();
    std::vector<DBuf<int>> perm(L + 1), iperm(L + 1);
    auto upload_perm = [&](const DevCSR& A, int l) {
        std::vector<int> p = window_sort_perm(A, win, st);
        if (p.empty()) return;
        perm[l].alloc(p.size());
        iperm[l].alloc(p.size());
        h2d(perm[l].p, p.data(), p.size(), st);
        k_invert_perm<<<grid_for((long long)p.size(), TB), TB, 0, st>>>(int(p.size()), perm[l].p, iperm[l].p);
        CK_LAUNCH();
    };
    for (int l = 0; l < L; ++l) upload_perm(H.levels[l]->A_ff, l);
    upload_perm(H.coarse.A, L);
    // nested positions, coarsest upward
    std::vector<DBuf<int>> pos(L + 1);
    pos[L].alloc(std::max(S->n_coarse, 1));
    if (S->n_coarse)
        k_pos_coarse<<<grid_for(S->n_coarse, TB), TB, 0, st>>>(S->n_coarse, off[L], perm[L].p, pos[L].p);
    for (int l = L - 1; l >= 0; --l) {
        SetupLevel& lv = *H.levels[l];
        pos[l].alloc(lv.n);
        k_pos_level<<<grid_for(lv.n, TB), TB, 0, st>>>(lv.n, lv.is_f.p, lv.f_index.p, lv.c_index.p,
                                                       off[l], perm[l].p, pos[l + 1].p, pos[l].p);
    }
    CK_LAUNCH();
    // level operators
    long long bytes = 0;
    int max_nc = 0;
    long long rc_total = 0;
    S->smooth_type = H.opt.smooth_type;
    for (int l = 0; l < L; ++l) {
        SetupLevel& lv = *H.levels[l];
        auto sl = std::make_unique<SolveLevel>();
        sl->off = off[l];
        sl->n_f = lv.n_f;
        sl->n_c = lv.n_c;
        sl->alpha = lv.alpha;
        // relative C positions: rel[c] = pos_{l+1}[c] - off_{l+1}; inv: row of Z'
        DBuf<int> rel(std::max(lv.n_c, 1)), inv(std::max(lv.n_c, 1));
        if (lv.n_c)
            k_rel<<<grid_for(lv.n_c, TB), TB, 0, st>>>(lv.n_c, pos[l + 1].p, off[l + 1], rel.p, inv.p);
        // SELL row r of A_ff / M is the F point at position r of the block
        build_sell<double>(lv.A_ff, iperm[l].p, perm[l].p, lv.n_f, sl->d.Aff, true, st);
        build_sell<double>(lv.M, iperm[l].p, rel.p, lv.n_c, sl->d.M, false, st);
        build_sell<double>(lv.Z, inv.p, perm[l].p, lv.n_f, sl->d.Z, false, st);
        if (lv.Ainv.n_rows) build_sell<double>(lv.Ainv, iperm[l].p, perm[l].p, lv.n_f, sl->d.Ainv, true, st);
        sl->W.alloc(std::max(lv.n_f, 1));
        if (lv.n_f) k_map_w<<<grid_for(lv.n_f, TB), TB, 0, st>>>(lv.n_f, lv.W.p, rel.p, perm[l].p, sl->W.p);
        CK_LAUNCH();
        if (!lv.alpha_c.empty()) {
            // C-point smoothing: row blocks of A_l over the level's nested
            // positions (rl = position relative to the level's offset)
            sl->alpha_c = lv.alpha_c;
            DBuf<int> rl(std::max(lv.n, 1)), rinv(std::max(lv.n, 1));
            k_rel<<<grid_for(lv.n, TB), TB, 0, st>>>(lv.n, pos[l].p, off[l], rl.p, rinv.p);
            CK_LAUNCH();
            build_sell<double>(lv.Crows, inv.p, rl.p, lv.n, sl->d.Mc, false, st);
            build_sell<double>(lv.A_cc, inv.p, rel.p, lv.n_c, sl->d.Acc, true, st);
            if (lv.Frows.n_rows) build_sell<double>(lv.Frows, iperm[l].p, rl.p, lv.n, sl->d.Mf, false, st);
            if (lv.Ainv_cc.n_rows) build_sell<double>(lv.Ainv_cc, inv.p, rel.p, lv.n_c, sl->d.Ainvc, true, st);
            max_nc = std::max(max_nc, lv.n_c);
            if (l > 0) {
                sl->rc_off = rc_total;
                rc_total += lv.n_c;
            }
        }
        if (mixed_precision(H.opt)) {
            copy_sell_f32(sl->d.Aff, sl->f.Aff, st);
            copy_sell_f32(sl->d.M, sl->f.M, st);
            if (H.opt.precision == AIRG_MIXED_FP32_BF16R) copy_sell_bf16(sl->d.Z, sl->f.Zb, st);
            else copy_sell_f32(sl->d.Z, sl->f.Z, st);
            if (lv.Ainv.n_rows) copy_sell_f32(sl->d.Ainv, sl->f.Ainv, st);
            if (sl->d.Mc.n_rows) copy_sell_f32(sl->d.Mc, sl->f.Mc, st);
            if (sl->d.Acc.n_rows) copy_sell_f32(sl->d.Acc, sl->f.Acc, st);
            if (sl->d.Mf.n_rows) copy_sell_f32(sl->d.Mf, sl->f.Mf, st);
            if (sl->d.Ainvc.n_rows) copy_sell_f32(sl->d.Ainvc, sl->f.Ainvc, st);
        }
        // 16-bit column copies (the FP64 operators' set the V-cycle's byte count)
        for (Sell<double>* X : {&sl->d.Z, &sl->d.M, &sl->d.Aff, &sl->d.Ainv, &sl->d.Mc, &sl->d.Acc, &sl->d.Mf,
                                &sl->d.Ainvc})
            add_col16(*X, st);
        if (mixed_precision(H.opt)) {
            SolveLevelT<float>& o = sl->f;
            for (Sell<float>* X : {&o.Z, &o.M, &o.Aff, &o.Ainv, &o.Mc, &o.Acc, &o.Mf, &o.Ainvc}) add_col16(*X, st);
            add_col16(o.Zb, st);
        }
        int vb = mixed_precision(H.opt) ? 4 : 8;
        int p = int(lv.alpha.size()) - 1;
        bytes += (H.opt.precision == AIRG_MIXED_FP32_BF16R ? sell_bytes(sl->d.Z, vb) - 2LL * lv.Z.nnz
                                                            : sell_bytes(sl->d.Z, vb)) +
                 sell_bytes(sl->d.M, vb) + 4LL * lv.n_f +
                 (lv.Ainv.n_rows ? sell_bytes(sl->d.Ainv, vb) : p * sell_bytes(sl->d.Aff, vb)) +
                 2LL * lv.n_f * vb;
        if (!lv.alpha_c.empty()) {
            const int pc = int(lv.alpha_c.size()) - 1;
            bytes += sell_bytes(sl->d.Mc, vb) + 2LL * lv.n_c * vb + (l > 0 ? 2LL * lv.n_c * vb : 0) +
                     (sl->d.Ainvc.n_rows ? sell_bytes(sl->d.Ainvc, vb) : pc * sell_bytes(sl->d.Acc, vb));
            if (sl->d.Mf.n_rows)
                bytes += sell_bytes(sl->d.Mf, vb) + 2LL * lv.n_f * vb +
                         (lv.Ainv.n_rows ? sell_bytes(sl->d.Ainv, vb) : p * sell_bytes(sl->d.Aff, vb));
        }
        S->max_nf = std::max(S->max_nf, lv.n_f);
        CK(cudaStreamSynchronize(st));
        S->lv.push_back(std::move(sl));
    }
    build_sell<double>(H.coarse.A, iperm[L].p, perm[L].p, S->n_coarse, S->Ac, true, st);
    if (mixed_precision(H.opt)) copy_sell_f32(S->Ac, S->Ac32, st);
    add_col16(S->Ac, st);
    add_col16(S->Ac32, st);
    S->roots = H.coarse.roots;
    {
        std::vector<double> rr;
        for (const Root& q : S->roots) { rr.push_back(q.re); rr.push_back(q.im); }
        S->roots_dev.alloc(std::max<size_t>(rr.size(), 2));
        h2d(S->roots_dev.p, rr.data(), rr.size(), st);
        S->bar.alloc(4);
        CK(cudaMemsetAsync(S->bar.p, 0, S->bar.bytes(), st));
        // persistent (cooperative, grid-barrier) polynomial kernels: opt-in;
        // graph-launched per-term kernels measured faster on GB300
        const char* pe = getenv("AIRG_PERSISTENT");
        std::string pv = pe ? pe : "";
        bool allow = pv == "1" || pv == "coarse";
        bool allow_s = pv == "1" || pv == "smoother";
        if (allow && !mixed_precision(H.opt)) S->newton_grid[0] = newton_persistent_grid<double>(S->Ac);
        if (allow && mixed_precision(H.opt)) S->newton_grid[1] = newton_persistent_grid<float>(S->Ac32);
        if (allow_s) {
            int dev = 0, sms = 0, per = 0;
            CK(cudaGetDevice(&dev));
            CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            if (!mixed_precision(H.opt)) {
                CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_smooth_persistent<double>, 1024, 0));
                S->smooth_grid[0] = per * sms;
            } else {
                CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_smooth_persistent<float>, 1024, 0));
                S->smooth_grid[1] = per * sms;
            }
        }
    }
    S->ticket.alloc(1);
    CK(cudaMemsetAsync(S->ticket.p, 0, sizeof(unsigned), st));
    {
        int vb = mixed_precision(H.opt) ? 4 : 8;
        long long nsp = 0;
        for (size_t i = 0; i < S->roots.size(); ++i) {
            bool last = i + 1 == S->roots.size();
            nsp += S->roots[i].im == 0.0 ? (last ? 0 : 1) : (last ? 1 : 2);
        }
        bytes += nsp * sell_bytes(S->Ac, vb);
    }
    S->bytes_vcycle = bytes;
    // top operator in the nested order: row pos0[i] <- natural row i
    const DevCSR& A0 = L ? H.levels[0]->A : H.coarse.A;
    S->pos0 = std::move(pos[0]);
    {
        DBuf<int> inv0(std::max(S->n0, 1));
        DBuf<int> dummy(std::max(S->n0, 1));
        if (S->n0) k_rel<<<grid_for(S->n0, TB), TB, 0, st>>>(S->n0, S->pos0.p, 0, dummy.p, inv0.p);
        CK_LAUNCH();
        build_sell<double>(A0, inv0.p, S->pos0.p, S->n0, S->Atop, true, st);
        add_col16(S->Atop, st);
        CK(cudaStreamSynchronize(st));
    }
    // slices per warp of the short-row operators, by timing
    if (mixed_precision(H.opt)) tune_all<float>(*S, st);
    else tune_all<double>(*S, st);
    {
        DBuf<double> x(std::max(S->n0, 1)), y(std::max(S->n0, 1));
        CK(cudaMemsetAsync(x.p, 0, x.bytes(), st));
        tune_rows(S->Atop, x.p, y.p, env_choice("AIRG_ROWS_PER_WARP", {1, 2, 4}),
                  env_choice("AIRG_LOADS_PER_LANE", {4, 8, 16}), st);
        CK(cudaStreamSynchronize(st));
    }
    // work vectors
    S->max_nc = max_nc;
    S->rc_total = rc_total;
    size_t n0 = std::max(S->n0, 1), nf = std::max({S->max_nf, max_nc, 1}), nc = std::max(S->n_coarse, 1);
    S->rwork.alloc(n0);
    S->t.alloc(nf); S->wa.alloc(nf); S->wb.alloc(nf);
    S->cr0.alloc(nc); S->cr1.alloc(nc); S->ct.alloc(nc);
    if (S->smooth_type != AIRG_SMOOTH_F) {
        const size_t nrc = size_t(std::max<long long>(rc_total, 1));
        if (mixed_precision(H.opt)) S->rcs32.alloc(nrc);
        else S->rcs.alloc(nrc);
    }
    if (mixed_precision(H.opt)) {
        S->rwork32.alloc(n0); S->e32.alloc(n0); S->vin32.alloc(n0);
        S->t32.alloc(nf); S->wa32.alloc(nf); S->wb32.alloc(nf);
        S->cr032.alloc(nc); S->cr132.alloc(nc); S->ct32.alloc(nc);
    }
    S->restart = std::max(1, H.opt.gmres_restart);
    int m = S->restart;
    S->V.alloc(size_t(m + 1) * n0);
    S->Zs.alloc(size_t(m) * n0);
    S->w.alloc(n0); S->bp.alloc(n0); S->xp.alloc(n0); S->r.alloc(n0);
    S->part.alloc(size_t(RGRID) * (m + 2));
    S->hdev.alloc(size_t(3 * (m + 2)));
    S->hhost.alloc(size_t(3 * (m + 2)));
    CK(cudaStreamCreateWithFlags(&S->sst, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&S->ev_in, cudaEventDisableTiming));
    const char* ng = getenv("AIRG_NO_GRAPHS");
    S->use_graphs = !(ng && ng[0] == '1');
    H.solve = std::move(S);
}

namespace {

// out[i] = <w, V_i> for i < m, out[m] = <w, w> when selfdot (chunks of MCH)
void launch_multidot(SolveData& S, long long n, int m, const double* V, long long ldv, const double* w,
                     double* out, int selfdot, cudaStream_t st)
{
    if (m == 0) {
        if (selfdot)
            LAUNCH_F(S, PK_KRYLOV, 8 * n, 2 * n,
                   k_multidot<0><<<RGRID, RB, 0, st>>>(n, V, ldv, w, S.part.p, out, S.ticket.p, 1));
        return;
    }
    for (int c0 = 0; c0 < m; c0 += MCH) {
        const int mc = std::min(MCH, m - c0);
        const int self = selfdot && c0 + mc == m;
        LAUNCH_F(S, PK_KRYLOV, 8LL * n * (mc + 1), 2LL * n * (mc + self),
               WITH_M(mc, k_multidot<MM><<<RGRID, RB, 0, st>>>(n, V + c0 * ldv, ldv, w, S.part.p, out + c0,
                                                                S.ticket.p, self)));
    }
}

// w += sum_i (neg ? -h_i : h_i) V_i (chunks of MCH); nrm2 (if not null)
// receives ||w||^2 of the result
void launch_multiaxpy(SolveData& S, long long n, int m, const double* V, long long ldv, const double* h,
                      int neg, double* w, double* nrm2, cudaStream_t st)
{
    for (int c0 = 0; c0 < m; c0 += MCH) {
        const int mc = std::min(MCH, m - c0);
        const int norm = nrm2 && c0 + mc == m;
        LAUNCH_F(S, PK_KRYLOV, 8LL * n * (mc + 2), 2LL * n * (mc + (norm ? 1 : 0)),
               WITH_M(mc, k_multiaxpy<MM><<<RGRID, RB, 0, st>>>(n, V + c0 * ldv, ldv, h + c0, neg, w, norm,
                                                                 S.part.p, nrm2, S.ticket.p)));
    }
}

double dev_norm(SolveData& S, const double* x, long long n, cudaStream_t st)
{
    launch_multidot(S, n, 0, nullptr, n, x, S.hdev.p, 1, st);
    CK_LAUNCH();
    double v = read1(S.hdev.p, st);
    return std::sqrt(v);
}

void precond_launch(Hierarchy& H, const double* v, double* z, cudaStream_t st)
{
    SolveData& S = *H.solve;
    long long n = S.n0;
    if (mixed_precision(H.opt)) {
        LAUNCH(S, PK_LAYOUT, 12 * n, launch_kernel(st, grid_for(n, TB), TB, 0, k_d2f, n, v, S.vin32.p));
        VWork<float> wk{S.rwork32.p, S.t32.p, S.wa32.p, S.wb32.p, nullptr, S.cr032.p, S.cr132.p, S.ct32.p,
                        S.rcs32.p};
        vcycle<float>(S, S.vin32.p, S.e32.p, wk, st);
        LAUNCH(S, PK_LAYOUT, 12 * n, launch_kernel(st, grid_for(n, TB), TB, 0, k_f2d, n, S.e32.p, z));
        CK_LAUNCH();
    } else {
        VWork<double> wk{S.rwork.p, S.t.p, S.wa.p, S.wb.p, nullptr, S.cr0.p, S.cr1.p, S.ct.p, S.rcs.p};
        vcycle<double>(S, v, z, wk, st);
    }
}

// z = M^-1 v: replays the captured V-cycle graph of this (v, z) pair, or
// launches the kernels directly while profiling.
void precond(Hierarchy& H, const double* v, double* z, cudaStream_t st)
{
    SolveData& S = *H.solve;
    if (!S.use_graphs) {
        precond_launch(H, v, z, st);
        return;
    }
    if (S.prof) {
        // profiled V-cycle: captured afresh with its event pairs, so that the
        // kernels run as in an unprofiled solve (no host launch gaps)
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        try {
            precond_launch(H, v, z, st);
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
        S.prof_execs.push_back(exec);
        CK(cudaGraphLaunch(exec, st));
        return;
    }
    SolveData::GEntry* ge = nullptr;
    for (auto& g : S.graphs)
        if (g.v == v && g.z == z) { ge = &g; break; }
    if (!ge) {
        long long before = S.launches;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        try {
            precond_launch(H, v, z, st);
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
        long long nk = S.launches - before;
        S.launches = before;
        S.graphs.push_back(SolveData::GEntry{v, z, exec, nk});
        ge = &S.graphs.back();
    }
    CK(cudaGraphLaunch(ge->exec, st));
    S.launches += ge->kernels;
}

void richardson(Hierarchy& H, double rtol, double atol, int maxit, airg_solve_info& info,
                cudaStream_t st);

// FGMRES(m) on the nested system; bp/xp hold b and x in nested order.
void fgmres(Hierarchy& H, double rtol, double atol, int maxit, airg_solve_info& info,
            cudaStream_t st)
{
    SolveData& S = *H.solve;
    long long n = S.n0;
    int m = S.restart;
    int g = grid_for(n, TB);
    SellView<double> A = view(S.Atop);
    const long long topB = mat_bytes(S.Atop) + 16 * n;
    double bn = dev_norm(S, S.bp.p, n, st);
    double tol = std::max(rtol * bn, atol);
    int its = 0;
    auto residual = [&]() {
        LAUNCH_F(S, PK_TOPSPMV, topB, 2 * S.Atop.nnz,
               WITH_KR_COL(S.Atop, k_spmv<double, KK, RR, double, C16><<<grid_rows(S.Atop, k_spmv<double, KK, RR, double, C16>), block_rows(S.Atop), 0, st>>>(A, S.xp.p, S.w.p)));
        LAUNCH_F(S, PK_KRYLOV, 24 * n, n, k_sub2<<<g, TB, 0, st>>>(n, S.bp.p, S.w.p, S.r.p));
        CK_LAUNCH();
        return dev_norm(S, S.r.p, n, st);
    };
    double rn = residual();
    std::vector<double> Hm(size_t(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
    double* hh = S.hhost.p;
    while (rn > tol && its < maxit) {
        LAUNCH_F(S, PK_KRYLOV, 16 * n, n, k_scale_into<<<g, TB, 0, st>>>(n, S.r.p, 1.0 / rn, S.V.p));
        std::fill(gv.begin(), gv.end(), 0.0);
        gv[0] = rn;
        int jdone = 0;
        for (int j = 0; j < m; ++j) {
            double* vj = S.V.p + size_t(j) * n;
            double* zj = S.Zs.p + size_t(j) * n;
            precond(H, vj, zj, st);
            LAUNCH_F(S, PK_TOPSPMV, topB, 2 * S.Atop.nnz,
                   WITH_KR_COL(S.Atop, k_spmv<double, KK, RR, double, C16><<<grid_rows(S.Atop, k_spmv<double, KK, RR, double, C16>), block_rows(S.Atop), 0, st>>>(A, zj, S.w.p)));
            // classical Gram-Schmidt; a second pass only when the first
            // one cancelled enough of ||w|| to cost orthogonality:
            // ||w'||^2 < reorth_ratio() ||w||^2
            double* h1 = S.hdev.p;
            double* h2 = S.hdev.p + (m + 2);
            double* nrm = S.hdev.p + 2 * (m + 2);
            launch_multidot(S, n, j + 1, S.V.p, n, S.w.p, h1, 1, st);
            launch_multiaxpy(S, n, j + 1, S.V.p, n, h1, 1, S.w.p, nrm, st);
            CK_LAUNCH();
            CK(cudaMemcpyAsync(hh, S.hdev.p, sizeof(double) * 3 * (m + 2), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            double ww = hh[j + 1], w1 = hh[2 * (m + 2)];
            for (int i = 0; i <= j; ++i) Hm[size_t(i) * m + j] = hh[i];
            double hsq = w1;
            if (w1 < reorth_ratio() * ww) {
                launch_multidot(S, n, j + 1, S.V.p, n, S.w.p, h2, 0, st);
                launch_multiaxpy(S, n, j + 1, S.V.p, n, h2, 1, S.w.p, nrm, st);
                CK_LAUNCH();
                CK(cudaMemcpyAsync(hh, S.hdev.p, sizeof(double) * 3 * (m + 2), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                for (int i = 0; i <= j; ++i) Hm[size_t(i) * m + j] += hh[(m + 2) + i];
                hsq = hh[2 * (m + 2)];
            }
            double hn = std::sqrt(std::max(hsq, 0.0));
            Hm[size_t(j + 1) * m + j] = hn;
            for (int i = 0; i < j; ++i) {
                double a = Hm[size_t(i) * m + j], b = Hm[size_t(i + 1) * m + j];
                Hm[size_t(i) * m + j] = cs[i] * a + sn[i] * b;
                Hm[size_t(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
            }
            double a = Hm[size_t(j) * m + j], b = Hm[size_t(j + 1) * m + j];
            double den = std::hypot(a, b);
            cs[j] = den > 0 ? a / den : 1.0;
            sn[j] = den > 0 ? b / den : 0.0;
            Hm[size_t(j) * m + j] = den;
            Hm[size_t(j + 1) * m + j] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            ++its;
            jdone = j + 1;
            if (std::fabs(gv[j + 1]) <= tol || its >= maxit || den == 0.0 || hn == 0.0) break;
            LAUNCH_F(S, PK_KRYLOV, 16 * n, n,
                   k_scale_into<<<g, TB, 0, st>>>(n, S.w.p, 1.0 / hn, S.V.p + size_t(j + 1) * n));
        }
        for (int j = jdone - 1; j >= 0; --j) {
            double s = gv[j];
            for (int i = j + 1; i < jdone; ++i) s -= Hm[size_t(j) * m + i] * y[i];
            y[j] = s / Hm[size_t(j) * m + j];
        }
        h2d(S.hdev.p, y.data(), jdone, st);
        launch_multiaxpy(S, n, jdone, S.Zs.p, n, S.hdev.p, 0, S.xp.p, nullptr, st);
        CK_LAUNCH();
        rn = residual();
    }
    info.iterations = std::max(info.iterations, its);
    double rel = bn > 0 ? rn / bn : 0.0;
    info.rel_residual = std::max(info.rel_residual, rel);
    info.converged = info.converged && (rn <= tol);
}

// Preconditioned Richardson (Sec. 3): x <- x + M^-1 r, r = b - A x, until the
// true residual meets the tolerance.  One V-cycle per iteration.
void richardson(Hierarchy& H, double rtol, double atol, int maxit, airg_solve_info& info,
                cudaStream_t st)
{
    SolveData& S = *H.solve;
    long long n = S.n0;
    int g = grid_for(n, TB);
    SellView<double> A = view(S.Atop);
    const long long topB = mat_bytes(S.Atop) + 16 * n;
    double bn = dev_norm(S, S.bp.p, n, st);
    double tol = std::max(rtol * bn, atol);
    auto residual = [&]() {
        LAUNCH_F(S, PK_TOPSPMV, topB, 2 * S.Atop.nnz,
               WITH_KR_COL(S.Atop, k_spmv<double, KK, RR, double, C16><<<grid_rows(S.Atop, k_spmv<double, KK, RR, double, C16>), block_rows(S.Atop), 0, st>>>(A, S.xp.p, S.w.p)));
        LAUNCH_F(S, PK_KRYLOV, 24 * n, n, k_sub2<<<g, TB, 0, st>>>(n, S.bp.p, S.w.p, S.r.p));
        CK_LAUNCH();
        return dev_norm(S, S.r.p, n, st);
    };
    double rn = residual();
    int its = 0;
    while (rn > tol && its < maxit) {
        precond(H, S.r.p, S.Zs.p, st);
        LAUNCH_F(S, PK_KRYLOV, 24 * n, n, k_add_dev<<<g, TB, 0, st>>>(n, S.Zs.p, nullptr, S.xp.p));
        rn = residual();
        ++its;
    }
    info.iterations = std::max(info.iterations, its);
    double rel = bn > 0 ? rn / bn : 0.0;
    info.rel_residual = std::max(info.rel_residual, rel);
    info.converged = info.converged && (rn <= tol);
}

// v = w / sqrt(nrm2) when *active and nrm2 > 0, else 0 (device-side scaling,
// so that it can sit inside a captured graph)
__global__ void k_scale_dev(long long n, const double* __restrict__ w, const double* __restrict__ nrm2,
                            const int* __restrict__ active, double* __restrict__ v)
{
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double q = *nrm2;
    double inv = (*active && q > 0.0) ? 1.0 / sqrt(q) : 0.0;
    v[r] = w[r] * inv;
}

}  // namespace

// ----------------------------------------- launch helpers for multi.cu ----
void mp_vcycle(Hierarchy& H, const double* v, double* z, cudaStream_t st) { precond_launch(H, v, z, st); }

void mp_top_spmv(Hierarchy& H, const double* x, double* y, cudaStream_t st)
{
    SolveData& S = *H.solve;
    long long n = S.n0;
    SellView<double> A = view(S.Atop);
    LAUNCH_F(S, PK_TOPSPMV, mat_bytes(S.Atop) + 16 * n, 2 * S.Atop.nnz,
           WITH_KR_COL(S.Atop, k_spmv<double, KK, RR, double, C16><<<grid_rows(S.Atop, k_spmv<double, KK, RR, double, C16>), block_rows(S.Atop), 0, st>>>(A, x, y)));
}

void mp_multidot(Hierarchy& H, int m, const double* V, const double* w, double* out, int selfdot,
                 cudaStream_t st)
{
    SolveData& S = *H.solve;
    launch_multidot(S, S.n0, m, V, S.n0, w, out, selfdot, st);
}

void mp_multiaxpy_norm(Hierarchy& H, int m, const double* V, const double* h, double* w, double* out,
                       cudaStream_t st)
{
    SolveData& S = *H.solve;
    launch_multiaxpy(S, S.n0, m, V, S.n0, h, 1, w, out, st);
}

void mp_scale_dev(Hierarchy& H, const double* w, const double* nrm2, const int* active, double* v,
                  cudaStream_t st)
{
    SolveData& S = *H.solve;
    long long n = S.n0;
    LAUNCH_F(S, PK_KRYLOV, 16 * n, n, k_scale_dev<<<grid_for(n, TB), TB, 0, st>>>(n, w, nrm2, active, v));
}

void mp_residual(Hierarchy& H, const double* b, const double* x, double* y, double* r, cudaStream_t st)
{
    SolveData& S = *H.solve;
    long long n = S.n0;
    mp_top_spmv(H, x, y, st);
    LAUNCH_F(S, PK_KRYLOV, 24 * n, n, k_sub2<<<grid_for(n, TB), TB, 0, st>>>(n, b, y, r));
}

void mp_update(Hierarchy& H, int m, const double* Zs, const double* y, double* x, cudaStream_t st)
{
    SolveData& S = *H.solve;
    launch_multiaxpy(S, S.n0, m, Zs, S.n0, y, 0, x, nullptr, st);
}

void mp_add_dev(Hierarchy& H, const double* z, const int* active, double* x, cudaStream_t st)
{
    SolveData& S = *H.solve;
    long long n = S.n0;
    LAUNCH_F(S, PK_KRYLOV, 24 * n, n, k_add_dev<<<grid_for(n, TB), TB, 0, st>>>(n, z, active, x));
}

void mp_permute(Hierarchy& H, const double* a, double* b, bool to_nested, cudaStream_t st)
{
    SolveData& S = *H.solve;
    long long n = S.n0;
    if (to_nested)
        LAUNCH(S, PK_LAYOUT, 20 * n, k_to_nested<<<grid_for(n, TB), TB, 0, st>>>(n, S.pos0.p, a, b));
    else
        LAUNCH(S, PK_LAYOUT, 20 * n, k_from_nested<<<grid_for(n, TB), TB, 0, st>>>(n, S.pos0.p, a, b));
}

// Runs the bounded wait of the grid barrier against an arrival that never
// comes; returns true if the wait gave up (error flag set) as designed.
bool barrier_timeout_check(long long limit, cudaStream_t st)
{
    DBuf<unsigned> state(4);
    CK(cudaMemsetAsync(state.p, 0, state.bytes(), st));
    k_barrier_timeout_check<<<1, 32, 0, st>>>(state.p, limit);
    CK_LAUNCH();
    unsigned h[4];
    d2h(h, state.p, 4, st);
    return h[2] != 0;
}

void solve_system(Hierarchy& H, int nrhs, const double* b, double* x, bool on_device, double rtol,
                  double atol, int maxit, airg_solve_info* info_out, cudaStream_t caller)
{
    auto t0 = std::chrono::steady_clock::now();
    SolveData& S = *H.solve;
    // order after the caller's stream, then work on the private stream
    CK(cudaEventRecord(S.ev_in, caller));
    CK(cudaStreamWaitEvent(S.sst, S.ev_in, 0));
    cudaStream_t st = S.sst;
    long long n = S.n0;
    long long launches0 = S.launches;
    airg_solve_info info{};
    info.converged = 1;
    const double* bdev = b;
    double* xdev = x;
    if (!on_device) {
        // staging buffers grow to the largest call and are reused, so a call
        // with host buffers costs its copies and no allocation
        const size_t need = size_t(n) * nrhs;
        if (S.stage_b.n < need) S.stage_b.alloc(need);
        if (S.stage_x.n < need) S.stage_x.alloc(need);
        h2d(S.stage_b.p, b, need, st);
        h2d(S.stage_x.p, x, need, st);
        bdev = S.stage_b.p;
        xdev = S.stage_x.p;
    }
    int g = grid_for(n, TB);
    const char* nb = getenv("AIRG_NO_BATCH");
    int nseq = nrhs;   // right-hand sides solved one after the other
    if (nrhs > 1 && !(nb && nb[0] == '1')) {
        // many right-hand sides: lockstep outer iteration with the batched V-cycle
        for (int q0 = 0; q0 < nrhs; q0 += batch_max_width()) {
            int kq = std::min(batch_max_width(), nrhs - q0);
            solve_batched(H, kq, bdev + size_t(q0) * n, xdev + size_t(q0) * n, rtol, atol, maxit, info, st);
        }
        nseq = 0;
    }
    for (int q = 0; q < nseq; ++q) {
        LAUNCH(S, PK_LAYOUT, 20 * n, k_to_nested<<<g, TB, 0, st>>>(n, S.pos0.p, bdev + size_t(q) * n, S.bp.p));
        LAUNCH(S, PK_LAYOUT, 20 * n, k_to_nested<<<g, TB, 0, st>>>(n, S.pos0.p, xdev + size_t(q) * n, S.xp.p));
        CK_LAUNCH();
        if (H.opt.outer == AIRG_OUTER_RICHARDSON) richardson(H, rtol, atol, maxit, info, st);
        else fgmres(H, rtol, atol, maxit, info, st);
        LAUNCH(S, PK_LAYOUT, 20 * n, k_from_nested<<<g, TB, 0, st>>>(n, S.pos0.p, S.xp.p, xdev + size_t(q) * n));
        CK_LAUNCH();
    }
    if (!on_device) {
        CK(cudaMemcpyAsync(x, S.stage_x.p, sizeof(double) * n * nrhs, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    S.collect();
    {
        unsigned err = 0;
        d2h(&err, S.bar.p + 2, 1, st);
        if (err) {
            CK(cudaMemsetAsync(S.bar.p, 0, S.bar.bytes(), st));
            CK(cudaStreamSynchronize(st));
            fail(AIRG_ERR_TIMEOUT, "a grid barrier of the coarse-grid kernel gave up waiting");
        }
    }
    info.kernel_launches = S.launches - launches0;
    info.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info_out) *info_out = info;
    if (!info.converged) fail(AIRG_ERR_NOT_CONVERGED, "the outer iteration did not reach the tolerance within maxit");
}

template <class T, class V>
void describe_sell(const Sell<T, V>& A, airg_operator_layout* out)
{
    std::memset(out, 0, sizeof *out);
    if (A.n_rows == 0) return;
    out->n_rows = A.n_rows;
    out->n_cols = A.n_cols;
    out->nnz = A.nnz;
    out->padded = A.padded;
    out->warps_per_slice = A.k;
    out->r = A.r;
    out->resident_grid = A.persist;
    out->index_bytes = A.col16.n ? 2 : 4;
    out->slice_bases = A.cbase.n ? 1 : 0;
    out->value_bytes = int(sizeof(V));
    out->dense_diagonal = A.ndiag ? 1 : 0;
}

template <class T>
bool level_layout(const SolveLevelT<T>& o, bool bf16r, int op, airg_operator_layout* out)
{
    switch (op) {
        case AIRG_OPERATOR_Z:
            if (bf16r) describe_sell(o.Zb, out);
            else describe_sell(o.Z, out);
            return true;
        case AIRG_OPERATOR_M: describe_sell(o.M, out); return true;
        case AIRG_OPERATOR_AFF: describe_sell(o.Aff, out); return true;
        case AIRG_OPERATOR_AINV: describe_sell(o.Ainv, out); return true;
        case AIRG_OPERATOR_C_ROWS: describe_sell(o.Mc, out); return true;
        case AIRG_OPERATOR_ACC: describe_sell(o.Acc, out); return true;
        case AIRG_OPERATOR_AINV_CC: describe_sell(o.Ainvc, out); return true;
        case AIRG_OPERATOR_F_ROWS: describe_sell(o.Mf, out); return true;
        default: return false;
    }
}

bool operator_layout(const Hierarchy& H, int level, int op, airg_operator_layout* out)
{
    if (!H.solve) return false;
    const SolveData& S = *H.solve;
    const bool mixed = mixed_precision(H.opt);
    const int L = int(S.lv.size());   // the coarsest level's index
    if (op == AIRG_OPERATOR_TOP) {
        if (level != 0) return false;
        describe_sell(S.Atop, out);
        return true;
    }
    if (op == AIRG_OPERATOR_COARSE) {
        if (level != L) return false;
        if (mixed) describe_sell(S.Ac32, out);
        else describe_sell(S.Ac, out);
        return true;
    }
    if (level < 0 || level >= L) return false;
    const SolveLevel& lv = *S.lv[size_t(level)];
    return mixed ? level_layout(lv.f, H.opt.precision == AIRG_MIXED_FP32_BF16R, op, out)
                 : level_layout(lv.d, false, op, out);
}

void fill_setup_info(const Hierarchy& H, airg_hierarchy_info* info)
{
    std::memset(info, 0, sizeof *info);
    int L = int(H.levels.size());
    info->levels = L + 1;
    info->truncated = H.coarse.truncated ? 1 : 0;
    info->coarse_roots = int(H.coarse.roots.size());
    info->coarse_krylov = H.coarse.k;
    info->setup_ms = H.setup_ms;
    long long top = L ? H.levels[0]->A.nnz : H.coarse.A.nnz;
    long long store = top, flops = 0;
    for (int l = 0; l < L && l < 63; ++l) {
        const SetupLevel& lv = *H.levels[l];
        info->n[l] = lv.n;
        info->n_f[l] = lv.n_f;
        info->nnz_a[l] = lv.A.nnz;
        int p = int(lv.alpha.size()) - 1;
        // kept for the solve: A_ff, A_fc, R = [Z I], P = [W; I] (Sec. 3)
        store += lv.A_ff.nnz + lv.A_fc.nnz + (lv.Z.nnz + lv.n_c) + (lv.n_f + lv.n_c);
        flops += 2LL * lv.Z.nnz + 2LL * lv.A_fc.nnz;
        if (lv.Ainv.n_rows) {   // assembled smoother: the Eq. 8 matrix is kept and applied once
            store += lv.Ainv.nnz;
            flops += 2LL * lv.A_ff.nnz + 2LL * lv.Ainv.nnz;
        } else {
            flops += 2LL * lv.A_ff.nnz * (p + 1);
        }
        if (!lv.alpha_c.empty()) {   // C-point smoothing keeps A_cf and A_cc
            store += lv.Crows.nnz + lv.Ainv_cc.nnz;
            flops += 2LL * lv.Crows.nnz + (lv.Ainv_cc.n_rows ? 2LL * lv.Ainv_cc.nnz
                                                              : 2LL * lv.A_cc.nnz * (long long)(lv.alpha_c.size() - 1));
        }
        if (lv.Frows.n_rows)
            flops += 2LL * lv.Frows.nnz + (lv.Ainv.n_rows ? 2LL * lv.Ainv.nnz : 2LL * lv.A_ff.nnz * p);
    }
    if (L < 64) {
        info->n[L] = H.coarse.A.n_rows;
        info->nnz_a[L] = H.coarse.A.nnz;
    }
    store += H.coarse.A.nnz;
    long long nsp = 0;
    for (size_t i = 0; i < H.coarse.roots.size(); ++i) {
        bool last = i + 1 == H.coarse.roots.size();
        nsp += H.coarse.roots[i].im == 0.0 ? (last ? 0 : 1) : (last ? 1 : 2);
    }
    flops += 2LL * H.coarse.A.nnz * nsp;
    info->storage_complexity = top ? double(store) / double(top) : 0.0;
    info->cycle_complexity = top ? double(flops) / (2.0 * double(top)) : 0.0;
    info->bytes_per_vcycle = H.solve ? H.solve->bytes_vcycle : 0;
    for (int k = 0; k < AIRG_SETUP_PHASES; ++k) info->setup_phase_ms[k] = H.phase_ms[k];
    info->exact_dots = H.exact_dots;
}

}  // namespace airg

namespace airg {

void set_profiling(Hierarchy& H, bool on, int kind, int level)
{
    SolveData& S = *H.solve;
    S.prof = on;
    S.prof_kind = on ? kind : -1;
    S.prof_level = on ? level : -1;
    S.run_open = false;
    S.recs.clear();
    S.evnext = 0;
    for (int k = 0; k < PROF_KINDS; ++k) {
        S.kind_ms[k] = 0;
        S.kind_launches[k] = 0;
        S.kind_bytes[k] = 0;
        for (int l = 0; l < SolveData::PROF_LEVELS; ++l) {
            S.lev_ms[k][l] = 0;
            S.lev_launches[k][l] = 0;
            S.lev_bytes[k][l] = 0;
            S.lev_flops[k][l] = 0;
        }
    }
}

bool read_profile(const Hierarchy& H, int kind, int level, double* ms, long long* launches, long long* bytes,
                  long long* flops)
{
    if (kind < 0 || kind >= PROF_KINDS || level < -1 || level >= SolveData::PROF_LEVELS) return false;
    const SolveData& S = *H.solve;
    if (level < 0) {
        *ms = S.kind_ms[kind];
        *launches = S.kind_launches[kind];
        *bytes = S.kind_bytes[kind];
        long long f = 0;
        for (int l = 0; l < SolveData::PROF_LEVELS; ++l) f += S.lev_flops[kind][l];
        if (flops) *flops = f;
    } else {
        *ms = S.lev_ms[kind][level];
        *launches = S.lev_launches[kind][level];
        *bytes = S.lev_bytes[kind][level];
        if (flops) *flops = S.lev_flops[kind][level];
    }
    return true;
}

}  // namespace airg
