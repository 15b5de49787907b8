// AIRG setup on the GPU (Sec. 2 of arXiv 2508.17517), level by level:
//   truncation test (Sec. 2.4) -> strength + S+S^T -> PMISR -> DDC (Sec. 2.1)
//   -> block extraction (Eq. 3) -> GMRES polynomial coefficients (Eq. 7)
//   -> fixed-sparsity inverse (Eq. 8) -> Z = -A_cf Ahat^-1 with R drop
//   -> one-point W -> A_coarse = R A P with drop + lumping
// and finally the coarse-grid Newton polynomial (Sec. 2.3).
//
// Reproducibility: every value that feeds a discrete decision (strength,
// DDC bins, drops, one-point choice, truncation) is computed with a fixed
// operation order: row sums run left to right in column order from +0.0
// with explicitly rounded products (__dmul_rn/__dadd_rn, no FMA), sparse
// products accumulate each entry in ascending inner index, and dot products
// are correctly rounded (exact_dot.cuh).  The results are therefore the
// bits of the sequential definitions, whatever the launch shape.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "dev_util.cuh"
#include "exact_dot.cuh"
#include "handle.h"
#include "hostmath.h"

namespace airg {

namespace {

constexpr int TB = 256;
enum { PURPOSE_COEF = 1, PURPOSE_PMISR = 2, PURPOSE_COARSE = 3, PURPOSE_TRUNC = 4, PURPOSE_COEF_C = 5 };

// ------------------------------------------------------------- prefix sum --
constexpr int SCAN_B = 1024;

__global__ void k_scan_block(const int* in, int* out, int* sums, int n)
{
    __shared__ int wsum[32];
    int i = blockIdx.x * SCAN_B + threadIdx.x;
    int v = i < n ? in[i] : 0;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        wsum[lane] = s;
    }
    __syncthreads();
    int incl = x + (w > 0 ? wsum[w - 1] : 0);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == SCAN_B - 1) sums[blockIdx.x] = incl;
}

// single block: exclusive scan of the block sums, in chunks, in 64-bit;
// *total = -1 if any prefix exceeds the int32 index space
__global__ void k_scan_sums(int* sums, int nb, int* total)
{
    __shared__ long long wsum[32];
    __shared__ long long carry;
    __shared__ int overflow;
    if (threadIdx.x == 0) { carry = 0; overflow = 0; }
    __syncthreads();
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < nb; base += SCAN_B) {
        int i = base + threadIdx.x;
        long long v = i < nb ? sums[i] : 0;
        long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            long long s = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                long long y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        long long incl = x + (w > 0 ? wsum[w - 1] : 0);
        long long c = carry;
        long long ex = c + incl - v;
        if (i < nb) {
            if (ex > 0x7fffffffLL) overflow = 1;
            sums[i] = int(ex);
        }
        __syncthreads();
        if (threadIdx.x == SCAN_B - 1) carry = c + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = (overflow || carry > 0x7fffffffLL) ? -1 : int(carry);
}

__global__ void k_scan_add(int* out, const int* sums, int n, const int* total)
{
    int i = blockIdx.x * SCAN_B + threadIdx.x;
    if (i < n) out[i] += sums[blockIdx.x];
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = *total;
}

}  // namespace

void exclusive_scan_async(const int* in, int* out, int n, cudaStream_t st)
{
    int nb = std::max(1, (n + SCAN_B - 1) / SCAN_B);
    DBuf<int> sums(size_t(nb) + 1);
    k_scan_block<<<nb, SCAN_B, 0, st>>>(in, out, sums.p, n);
    k_scan_sums<<<1, SCAN_B, 0, st>>>(sums.p, nb, sums.p + nb);
    k_scan_add<<<nb, SCAN_B, 0, st>>>(out, sums.p, n, sums.p + nb);
    CK_LAUNCH();
    CK(cudaStreamSynchronize(st));   // sums is released on return
}

int exclusive_scan(const int* in, int* out, int n, cudaStream_t st)
{
    exclusive_scan_async(in, out, n, st);
    int total = read1(out + n, st);
    if (total < 0) fail(AIRG_ERR_OOM, "index space of a setup product exceeds 2^31 entries");
    return total;
}

namespace {

// ---------------------------------------------------------- random streams --
__device__ __forceinline__ unsigned long long sm64_mix(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
constexpr unsigned long long SM64_GAMMA = 0x9e3779b97f4a7c15ULL;

inline unsigned long long host_mix(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
inline unsigned long long stream_key(unsigned long long seed, long long level, long long purpose)
{
    unsigned long long tag = ((unsigned long long)level << 8) | (unsigned long long)purpose;
    return host_mix(seed + SM64_GAMMA * (tag + 1ULL));
}

__global__ void k_rng_uniform(unsigned long long key, long long n, double* out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long z = sm64_mix(key + SM64_GAMMA * (unsigned long long)(i + 1));
    out[i] = (double)(z >> 11) * 0x1.0p-53;
}

__global__ void k_rng_u32(unsigned long long key, long long n, unsigned* out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long z = sm64_mix(key + SM64_GAMMA * (unsigned long long)(i + 1));
    out[i] = (unsigned)(z >> 32);
}

// ------------------------------------------------------------- validation --
// Row i of a caller's CSR.  The row pointers are checked first (0 = rp[0] <=
// rp[i] <= rp[i+1] <= rp[n] = nnz); only a row whose bounds pass has its
// entries read.  flags: [0] columns out of range or not strictly
// ascending, [1] no stored diagonal, [2] bad row pointers, [3] a value that
// is not finite.
__global__ void k_validate(int n_rows, int n_cols, int nnz, const int* rp, const int* ci, const double* v,
                           int square, int* flags)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rows) return;
    const int a = rp[i], b = rp[i + 1];
    if (a < 0 || b < a || b > nnz || (i == 0 && a != 0) || (i == n_rows - 1 && b != nnz)) {
        flags[2] = 1;
        return;
    }
    int prev = -1;
    bool diag = false;
    for (int k = a; k < b; ++k) {
        int j = ci[k];
        if (j <= prev || j < 0 || j >= n_cols) flags[0] = 1;
        if (!isfinite(v[k])) flags[3] = 1;
        prev = j;
        if (j == i) diag = true;
    }
    if (square && !diag) flags[1] = 1;
}

// ------------------------------------------------------- strength / graph --
__global__ void k_strength(int n, const int* rp, const int* ci, const double* v, double theta,
                           int8_t* s)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double m = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k)
        if (ci[k] != i && fabs(v[k]) > m) m = fabs(v[k]);
    double thr = __dmul_rn(theta, m);
    for (int k = rp[i]; k < rp[i + 1]; ++k)
        s[k] = (int8_t)(ci[k] != i && m > 0.0 && fabs(v[k]) >= thr);
}

__global__ void k_count_strong_t(int n, const int* rp, const int* ci, const int8_t* s, int* cnt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rp[i]; k < rp[i + 1]; ++k)
        if (s[k]) atomicAdd(cnt + ci[k], 1);
}

__global__ void k_fill_strong_t(int n, const int* rp, const int* ci, const int8_t* s,
                                const int* rpt, int* cursor, int* ct)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rp[i]; k < rp[i + 1]; ++k)
        if (s[k]) {
            int j = ci[k];
            ct[rpt[j] + atomicAdd(cursor + j, 1)] = i;
        }
}

// insertion sort of each row's column list (rows are short)
__global__ void k_sort_rows(int n, const int* rp, int* c)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int a = rp[i] + 1; a < rp[i + 1]; ++a) {
        int key = c[a], b = a - 1;
        while (b >= rp[i] && c[b] > key) { c[b + 1] = c[b]; --b; }
        c[b + 1] = key;
    }
}

// sort each row's (col, val) pairs by column
__global__ void k_sort_rows_kv(int n, const int* rp, int* c, double* v)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int a = rp[i] + 1; a < rp[i + 1]; ++a) {
        int key = c[a];
        double val = v[a];
        int b = a - 1;
        while (b >= rp[i] && c[b] > key) { c[b + 1] = c[b]; v[b + 1] = v[b]; --b; }
        c[b + 1] = key;
        v[b + 1] = val;
    }
}

// row i of S + S^T: merge of the strong columns of row i and the sorted
// row i of S^T, without duplicates
__global__ void k_union(int n, const int* rp, const int* ci, const int8_t* s, const int* rpt,
                        const int* ct, const int* rpg, int* cg, int* cnt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = rp[i], ae = rp[i + 1], b = rpt[i], be = rpt[i + 1];
    int c = 0, o = rpg ? rpg[i] : 0;
    while (true) {
        while (a < ae && !s[a]) ++a;
        if (a >= ae && b >= be) break;
        int ja = a < ae ? ci[a] : 0x7fffffff;
        int jb = b < be ? ct[b] : 0x7fffffff;
        int j = ja < jb ? ja : jb;
        if (ja == j) ++a;
        if (jb == j) ++b;
        if (cg) cg[o + c] = j;
        ++c;
    }
    if (cnt) cnt[i] = c;
}

// ------------------------------------------------------------------ PMISR --
__device__ __forceinline__ bool key_beats(int dj, unsigned wj, int j, int di, unsigned wi, int i)
{
    if (dj != di) return dj > di;
    if (wj != wi) return wj > wi;
    return j > i;
}

__global__ void k_pmisr_select(int n, const int* rpg, const int* cg, const unsigned* w,
                               const int8_t* state, int8_t* newf)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (state[i] != 0) { newf[i] = 0; return; }
    int di = rpg[i + 1] - rpg[i];
    int8_t sel = 1;
    for (int k = rpg[i]; k < rpg[i + 1]; ++k) {
        int j = cg[k];
        if (state[j] == 0 && key_beats(rpg[j + 1] - rpg[j], w[j], j, di, w[i], i)) { sel = 0; break; }
    }
    newf[i] = sel;
}

__global__ void k_pmisr_update(int n, const int* rpg, const int* cg, int8_t* state,
                               const int8_t* newf, int* undecided)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || state[i] != 0) return;
    if (newf[i]) { state[i] = 1; return; }
    for (int k = rpg[i]; k < rpg[i + 1]; ++k)
        if (newf[cg[k]]) { state[i] = 2; return; }
    atomicAdd(undecided, 1);
}

__global__ void k_state_to_f(int n, const int8_t* state, int8_t* is_f)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) is_f[i] = state[i] == 1;
}

// -------------------------------------------------------------------- DDC --
__global__ void k_ddc_ratio(int n, const int* rp, const int* ci, const double* v,
                            const int8_t* is_f, double* ratio, unsigned long long* rmax_bits)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (!is_f[i]) { ratio[i] = -1.0; return; }
    double s = 0.0, d = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        int j = ci[k];
        if (j == i) d = fabs(v[k]);
        else if (is_f[j]) s = __dadd_rn(s, fabs(v[k]));
    }
    double r = d > 0.0 ? __ddiv_rn(s, d) : __longlong_as_double(0x7ff0000000000000LL);
    ratio[i] = r;
    atomicMax(rmax_bits, (unsigned long long)__double_as_longlong(r));   // r >= 0
}

__global__ void k_ddc_bin(int n, const int8_t* is_f, const double* ratio, double rmax, int nbins,
                          int* bins, int* hist)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !is_f[i]) return;
    double t = __dmul_rn(__ddiv_rn(ratio[i], rmax), (double)nbins);
    int b = (int)floor(t);
    if (b > nbins - 1) b = nbins - 1;
    bins[i] = b;
    atomicAdd(hist + b, 1);
}

__global__ void k_ddc_convert(int n, int8_t* is_f, const int* bins, int B)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && is_f[i] && bins[i] >= B) is_f[i] = 0;
}

// ----------------------------------------------------------- local indices --
__global__ void k_flag_eq(int n, const int8_t* is_f, int want, int* flag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (is_f[i] == want);
}

__global__ void k_local_index(int n, const int8_t* is_f, int want, const int* excl, int* idx,
                              int* ids)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (is_f[i] == want) { idx[i] = excl[i]; ids[excl[i]] = i; }
    else idx[i] = -1;
}

// --------------------------------------------------------------- extract --
// rows: list of source rows (nullptr = identity); colmap: new column of each
// source column or -1 to drop (nullptr = keep all, same index)
__global__ void k_sub_count(int nr, const int* rows, const int* rp, const int* ci,
                            const int* colmap, int* cnt)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nr) return;
    int i = rows ? rows[r] : r;
    int c = 0;
    for (int k = rp[i]; k < rp[i + 1]; ++k)
        if (!colmap || colmap[ci[k]] >= 0) ++c;
    cnt[r] = c;
}

__global__ void k_sub_fill(int nr, const int* rows, const int* rp, const int* ci, const double* v,
                           const int* colmap, const int* orp, int* oci, double* ov)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nr) return;
    int i = rows ? rows[r] : r;
    int o = orp[r];
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        int j = colmap ? colmap[ci[k]] : ci[k];
        if (j >= 0) { oci[o] = j; ov[o] = v[k]; ++o; }
    }
}

// -------------------------------------------------------- Arnoldi pieces --
__global__ void k_spmv_det(int n, const int* rp, const int* ci, const double* v,
                           const double* x, double* y)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) s = __dadd_rn(s, __dmul_rn(v[k], x[ci[k]]));
    y[i] = s;
}

__global__ void k_div_dev(long long n, double* out, const double* w, const double* h)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = __ddiv_rn(w[i], *h);
}

__global__ void k_sub(long long n, const double* a, const double* b, double* out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __dsub_rn(a[i], b[i]);
}

__global__ void k_newton_real_x(long long n, double* x, const double* r, double a)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = __dadd_rn(x[i], __ddiv_rn(r[i], a));
}

__global__ void k_newton_r(long long n, double* r, const double* w, double a)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = __dsub_rn(r[i], __ddiv_rn(w[i], a));
}

__global__ void k_newton_pair(long long n, double* x, const double* r, const double* w,
                              double* t, double a2, double mod2)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double tt = __dsub_rn(__dmul_rn(a2, r[i]), w[i]);
    t[i] = tt;
    x[i] = __dadd_rn(x[i], __ddiv_rn(tt, mod2));
}

// --------------------------------------------------- fixed-sparsity powers --
__global__ void k_fsp_init(int n, const int* rp, const int* ci, double a0, double* acc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rp[i]; k < rp[i + 1]; ++k) acc[k] = ci[k] == i ? a0 : 0.0;
}

__device__ __forceinline__ int find_col(const int* ci, int lo, int hi, int j)
{
    while (lo < hi) {
        int mid = lo + ((hi - lo) >> 1);
        if (ci[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Rows of at least FSP_WARP_ROW entries are computed by k_fsp_power_warp.
constexpr int FSP_WARP_ROW = 16;

__global__ void k_fsp_power(int n, const int* rp, const int* ci, const double* a,
                            const double* tprev, double* tout)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (rp[i + 1] - rp[i] >= FSP_WARP_ROW) return;
    for (int q = rp[i]; q < rp[i + 1]; ++q) {
        int j = ci[q];
        double s = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            int l = ci[p];
            int r = find_col(ci, rp[l], rp[l + 1], j);
            if (r < rp[l + 1] && ci[r] == j) s = __dadd_rn(s, __dmul_rn(a[p], tprev[r]));
        }
        tout[q] = s;
    }
}

// The long rows of k_fsp_power, one warp each: lane t computes the entries
// q = rp[i] + t, t + 32, ... of the row, each summed over the row's entries
// p in column order exactly as the one-thread kernel does.
__global__ void k_fsp_power_warp(int n, const int* rp, const int* ci, const double* a,
                                 const double* tprev, double* tout)
{
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const int r0 = rp[i], r1 = rp[i + 1];
    if (r1 - r0 < FSP_WARP_ROW) return;
    for (int q = r0 + lane; q < r1; q += 32) {
        const int j = ci[q];
        double s = 0.0;
        for (int p = r0; p < r1; ++p) {
            const int l = ci[p];
            const int r = find_col(ci, rp[l], rp[l + 1], j);
            if (r < rp[l + 1] && ci[r] == j) s = __dadd_rn(s, __dmul_rn(a[p], tprev[r]));
        }
        tout[q] = s;
    }
}

__global__ void k_fsp_acc(int nnz, double* acc, const double* T, double ak)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nnz) acc[k] = __dadd_rn(acc[k], __dmul_rn(ak, T[k]));
}

__global__ void k_scale(int nnz, double* v, double s)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nnz) v[k] = v[k] * s;
}

// -------------------------------------------------------------- SpGEMM ----
// C = A B.  Each row of C is built by one thread in a private open-addressing
// table: contributions arrive in ascending order of A's column (the inner
// index), so every entry is the left-to-right sum of the definition.
__global__ void k_gemm_bound(int m, const int* arp, const int* aci, const int* brp, int* tsize)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    long long b = 0;
    for (int p = arp[i]; p < arp[i + 1]; ++p) b += brp[aci[p] + 1] - brp[aci[p]];
    int sz = 0;
    if (b > 0) {
        sz = 1;
        while (sz < 2 * b) sz <<= 1;
    }
    tsize[i] = sz;
}

__device__ __forceinline__ unsigned hash_col(int j) { return (unsigned)j * 2654435761u; }

// Rows whose table has at least HASH_WARP_SLOTS slots are accumulated by a
// warp (k_gemm_hash_warp), the others by one thread (k_gemm_hash).
constexpr int HASH_WARP_SLOTS = 64;

__global__ void k_gemm_hash(int m, int row0, const int* arp, const int* aci, const double* av,
                            const int* brp, const int* bci, const double* bv, const int* toff,
                            int* keys, double* vals, int* cnt)
{
    int li = blockIdx.x * blockDim.x + threadIdx.x;   // row within the chunk
    if (li >= m) return;
    int i = row0 + li;
    int base = toff[li], size = toff[li + 1] - base;
    if (size >= HASH_WARP_SLOTS) return;
    int c = 0;
    if (size > 0) {
        unsigned mask = (unsigned)size - 1u;
        for (int p = arp[i]; p < arp[i + 1]; ++p) {
            int l = aci[p];
            double a = av[p];
            for (int q = brp[l]; q < brp[l + 1]; ++q) {
                int j = bci[q];
                double prod = __dmul_rn(a, bv[q]);
                unsigned h = hash_col(j) & mask;
                while (true) {
                    int key = keys[base + h];
                    if (key == j) { vals[base + h] = __dadd_rn(vals[base + h], prod); break; }
                    if (key == -1) {
                        keys[base + h] = j;
                        vals[base + h] = __dadd_rn(0.0, prod);
                        ++c;
                        break;
                    }
                    h = (h + 1u) & mask;
                }
            }
        }
    }
    cnt[li] = c;
}

// The rows with large tables, one warp each.  The entries of A's row are
// taken one at a time, in column order, by the whole warp; the lanes share
// that entry's row of B.  Within one entry of A the columns j of B's row are
// distinct, so no two lanes add to the same j (a lane claims a new slot with
// an atomic compare-and-swap), and the warp synchronises before the next
// entry: every output entry is still summed in ascending inner index with
// the same roundings as the one-thread kernel.
__global__ void k_gemm_hash_warp(int m, int row0, const int* arp, const int* aci, const double* av,
                                 const int* brp, const int* bci, const double* bv, const int* toff,
                                 int* keys, double* vals, int* cnt)
{
    const int lane = threadIdx.x & 31;
    const int li = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (li >= m) return;                       // uniform over the warp
    const int i = row0 + li;
    const int base = toff[li], size = toff[li + 1] - base;
    if (size < HASH_WARP_SLOTS) return;
    const unsigned mask = (unsigned)size - 1u;
    int c = 0;
    for (int p = arp[i]; p < arp[i + 1]; ++p) {
        const int l = aci[p];
        const double a = av[p];
        for (int q = brp[l] + lane; q < brp[l + 1]; q += 32) {
            const int j = bci[q];
            const double prod = __dmul_rn(a, bv[q]);
            unsigned h = hash_col(j) & mask;
            while (true) {
                int key = *(volatile int*)(keys + base + h);
                if (key == -1) {
                    key = atomicCAS(keys + base + h, -1, j);
                    if (key == -1) {
                        vals[base + h] = __dadd_rn(0.0, prod);
                        ++c;
                        break;
                    }
                }
                if (key == j) {
                    vals[base + h] = __dadd_rn(vals[base + h], prod);
                    break;
                }
                h = (h + 1u) & mask;
            }
        }
        __syncwarp();
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[li] = c;
}

__global__ void k_shift_rowptr(int m, const int* prp, int off, int* crp)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) crp[i] = prp[i] + off;
}

// Emit of the rows longer than `skip` entries: one thread per row,
// insertion into column order.
__global__ void k_gemm_emit(int m, const int* toff, const int* keys, const double* vals,
                            const int* crp, int* cci, double* cv, int skip)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || crp[i + 1] - crp[i] <= skip) return;
    int o = crp[i], s = crp[i];
    for (int t = toff[i]; t < toff[i + 1]; ++t) {
        int j = keys[t];
        if (j < 0) continue;
        double v = vals[t];
        int b = o - 1;
        while (b >= s && cci[b] > j) { cci[b + 1] = cci[b]; cv[b + 1] = cv[b]; --b; }
        cci[b + 1] = j;
        cv[b + 1] = v;
        ++o;
    }
}

// Emit of the rows of at most 32 entries: one warp per row, one entry per
// lane, sorted by column with a bitonic network of warp shuffles.
__global__ void k_gemm_emit_small(int m, const int* toff, const int* keys, const double* vals,
                                  const int* crp, int* cci, double* cv)
{
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= m) return;                        // uniform over the warp
    const int n = crp[i + 1] - crp[i];
    if (n > 32) return;
    int k = 0x7fffffff;
    double v = 0.0;
    int filled = 0;
    for (int tb = toff[i]; tb < toff[i + 1]; tb += 32) {
        const int t = tb + lane;
        const int key = t < toff[i + 1] ? keys[t] : -1;
        const unsigned ball = __ballot_sync(0xffffffffu, key >= 0);
        const int pos = filled + __popc(ball & ((1u << lane) - 1u));
        const double val = key >= 0 ? vals[t] : 0.0;
        // lane pos receives this entry
        for (int src = 0; src < 32; ++src) {
            if (!((ball >> src) & 1u)) continue;
            const int sp = __shfl_sync(0xffffffffu, pos, src);
            const int sk = __shfl_sync(0xffffffffu, key, src);
            const double sv = __shfl_sync(0xffffffffu, val, src);
            if (lane == sp) { k = sk; v = sv; }
        }
        filled += __popc(ball);
    }
    for (int size = 2; size <= 32; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int ok = __shfl_xor_sync(0xffffffffu, k, stride);
            const double ov = __shfl_xor_sync(0xffffffffu, v, stride);
            const bool lower = (lane & stride) == 0;
            const bool up = (lane & size) == 0;
            // the lower lane of a pair keeps the smaller key when sorting up
            const bool take = lower == up ? ok < k : ok > k;
            if (take) { k = ok; v = ov; }
        }
    }
    if (lane < n) {
        cci[crp[i] + lane] = k;
        cv[crp[i] + lane] = v;
    }
}

// Emit of the rows of at most EMIT_CAP entries: one warp per row takes the
// valid slots of the row's table into shared memory (ballot / prefix
// count), sorts them by column with a bitonic network and writes them out.
// The values were summed in the hash phase; only their order is set here.
constexpr int EMIT_CAP = 1024;
constexpr int EMIT_WARPS = 4;

__global__ void __launch_bounds__(EMIT_WARPS * 32)
k_gemm_emit_warp(int m, const int* toff, const int* keys, const double* vals, const int* crp, int* cci,
                 double* cv)
{
    __shared__ int sk[EMIT_WARPS][EMIT_CAP];
    __shared__ double sv[EMIT_WARPS][EMIT_CAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * EMIT_WARPS + w;
    if (i >= m) return;
    const int n = crp[i + 1] - crp[i];
    if (n > EMIT_CAP || n <= 32) return;
    int* k = sk[w];
    double* v = sv[w];
    const int t0 = toff[i], t1 = toff[i + 1];
    int filled = 0;
    for (int tb = t0; tb < t1; tb += 32) {
        const int t = tb + lane;
        const int key = t < t1 ? keys[t] : -1;
        const unsigned ball = __ballot_sync(0xffffffffu, key >= 0);
        if (key >= 0) {
            const int pos = filled + __popc(ball & ((1u << lane) - 1u));
            if (pos < EMIT_CAP) {
                k[pos] = key;
                v[pos] = vals[t];
            }
        }
        filled += __popc(ball);
    }
    int P = 1;
    while (P < n) P <<= 1;
    for (int t = n + lane; t < P; t += 32) {
        k[t] = 0x7fffffff;
        v[t] = 0.0;
    }
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < P; t += 32) {
                const int u = t ^ stride;
                if (u > t) {
                    const bool up = (t & size) == 0;
                    const int a = k[t], b = k[u];
                    if ((a > b) == up && a != b) {
                        k[t] = b;
                        k[u] = a;
                        const double x = v[t];
                        v[t] = v[u];
                        v[u] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
    const int o = crp[i];
    for (int t = lane; t < n; t += 32) {
        cci[o + t] = k[t];
        cv[o + t] = v[t];
    }
}

// ------------------------------------------------------------ drop rules --
__global__ void k_drop_rows(int n, const int* rp, const double* v, double tol, int8_t* keep,
                            int* cnt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double m = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k)
        if (fabs(v[k]) > m) m = fabs(v[k]);
    double thr = __dmul_rn(tol, m);
    int c = 0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        int8_t kp = (int8_t)(v[k] != 0.0 && fabs(v[k]) >= thr);
        keep[k] = kp;
        c += kp;
    }
    cnt[i] = c;
}

__global__ void k_drop_lump(int n, const int* rp, const int* ci, const double* v, double tol,
                            int lump, int8_t* keep, double* vout, int* cnt, int* bad)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double m = 0.0;
    int dpos = -1;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        if (ci[k] == i) dpos = k;
        else if (fabs(v[k]) > m) m = fabs(v[k]);
    }
    if (dpos < 0) { *bad = 1; cnt[i] = 0; return; }
    double thr = __dmul_rn(tol, m);
    double d = v[dpos];
    int c = 0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        vout[k] = v[k];
        if (k == dpos) { keep[k] = 1; ++c; continue; }
        if (v[k] == 0.0 || fabs(v[k]) < thr) {
            keep[k] = 0;
            if (lump) d = __dadd_rn(d, v[k]);
        } else {
            keep[k] = 1;
            ++c;
        }
    }
    vout[dpos] = d;
    cnt[i] = c;
}

__global__ void k_compact(int n, const int* rp, const int* ci, const double* v,
                          const int8_t* keep, const int* nrp, int* nci, double* nv)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int o = nrp[i];
    for (int k = rp[i]; k < rp[i + 1]; ++k)
        if (keep[k]) { nci[o] = ci[k]; nv[o] = v[k]; ++o; }
}

// --------------------------------------------------------- one-point W ----
__global__ void k_one_point(int n, const int* rp, const int* ci, const double* v,
                            const int8_t* strong, const int8_t* is_f, const int* c_index,
                            const int* f_index, int* W)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !is_f[i]) return;
    int best = -1;
    for (int pass = 0; pass < 2 && best < 0; ++pass) {
        double bestv = -1.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            int j = ci[k];
            if (j == i || is_f[j]) continue;
            if (pass == 0 && !strong[k]) continue;
            double a = fabs(v[k]);
            if (a > bestv) { bestv = a; best = j; }
        }
    }
    W[f_index[i]] = best >= 0 ? c_index[best] : -1;
}

// P = [W; I] in the fine numbering: one entry (weight 1) per row
__global__ void k_p_count(int n, const int8_t* is_f, const int* f_index, const int* W, int* cnt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cnt[i] = is_f[i] ? (W[f_index[i]] >= 0) : 1;
}

__global__ void k_p_fill(int n, const int8_t* is_f, const int* f_index, const int* c_index,
                         const int* W, const int* prp, int* pci, double* pv)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || prp[i + 1] == prp[i]) return;
    pci[prp[i]] = is_f[i] ? W[f_index[i]] : c_index[i];
    pv[prp[i]] = 1.0;
}

// R = [Z I] in the fine numbering: row c holds Z's row (F columns mapped to
// their fine index) and a 1 at the C point itself, columns ascending
__global__ void k_r_rowptr(int nc, const int* zrp, int* rrp)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c <= nc) rrp[c] = zrp[c] + c;
}

__global__ void k_r_fill(int nc, const int* zrp, const int* zci, const double* zv,
                         const int* f_ids, const int* c_ids, const int* rrp, int* rci, double* rv)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int o = rrp[c], self = c_ids[c];
    bool done = false;
    for (int k = zrp[c]; k < zrp[c + 1]; ++k) {
        int col = f_ids[zci[k]];
        if (!done && self < col) { rci[o] = self; rv[o] = 1.0; ++o; done = true; }
        rci[o] = col;
        rv[o] = zv[k];
        ++o;
    }
    if (!done) { rci[o] = self; rv[o] = 1.0; }
}

// ------------------------------------------------------------- transpose --
__global__ void k_count_cols(int n, const int* rp, const int* ci, int* cnt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rp[i]; k < rp[i + 1]; ++k) atomicAdd(cnt + ci[k], 1);
}

__global__ void k_fill_transpose(int n, const int* rp, const int* ci, const double* v,
                                 const int* trp, int* cursor, int* tci, double* tv)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        int j = ci[k];
        int pos = trp[j] + atomicAdd(cursor + j, 1);
        tci[pos] = i;
        tv[pos] = v[k];
    }
}

// =========================================================================
// host-side building blocks
// =========================================================================
struct Ctx {
    cudaStream_t st;
    DBuf<unsigned long long> xacc;   // exact-dot accumulator
    DBuf<int> xbad;
    DBuf<unsigned> xticket;          // last-block ticket of k_xdot
    long long ndots = 0;             // exact dot products launched
    explicit Ctx(cudaStream_t s) : st(s)
    {
        xacc.alloc(XD_DIGITS);
        xbad.alloc(1);
        xticket.alloc(1);
        CK(cudaMemsetAsync(xacc.p, 0, xacc.bytes(), st));
        CK(cudaMemsetAsync(xbad.p, 0, xbad.bytes(), st));
        CK(cudaMemsetAsync(xticket.p, 0, xticket.bytes(), st));
    }
};

int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    return sms;
}

void xdot(Ctx& c, long long n, const double* x, const double* y, double* out, double* out_sqrt)
{
    int grid = (int)std::min<long long>(std::max<long long>(1, (n + XD_THREADS - 1) / XD_THREADS),
                                        2LL * num_sms());
    k_xdot<<<grid, XD_THREADS, 0, c.st>>>(n, x, y, c.xacc.p, c.xbad.p, c.xticket.p, out, out_sqrt);
    CK_LAUNCH();
    ++c.ndots;
}

// MGS step w -= (*hprev) vprev (skipped when vprev is null) fused with the
// correctly rounded <w, y> (y null: <w, w>) into out / out_sqrt.
void mgs_xdot(Ctx& c, long long n, double* w, const double* vprev, const double* hprev, const double* y,
              double* out, double* out_sqrt)
{
    int grid = (int)std::min<long long>(std::max<long long>(1, (n + XD_THREADS - 1) / XD_THREADS),
                                        2LL * num_sms());
    k_mgs_xdot<<<grid, XD_THREADS, 0, c.st>>>(n, w, vprev, hprev, y, c.xacc.p, c.xbad.p, c.xticket.p, out,
                                               out_sqrt);
    CK_LAUNCH();
    ++c.ndots;
}

// Wall time of one setup phase, added to *acc: the stream is synchronised
// when the phase starts and when it ends, so the time covers the phase's
// kernels and its host work and nothing else.
struct PhaseTimer {
    cudaStream_t st;
    double* acc;
    std::chrono::steady_clock::time_point t0;
    PhaseTimer(cudaStream_t s, double* a) : st(s), acc(a)
    {
        CK(cudaStreamSynchronize(st));
        t0 = std::chrono::steady_clock::now();
    }
    ~PhaseTimer()
    {
        cudaStreamSynchronize(st);   // errors surface at the next checked call
        *acc += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

// Builds CSR from per-row counts already in rp[0..n-1]; returns nnz.
int counts_to_rowptr(DBuf<int>& rp, int n, cudaStream_t st) { return exclusive_scan(rp.p, rp.p, n, st); }

void submatrix(const DevCSR& A, const int* rows, int nr, const int* colmap, int ncols, DevCSR& out,
               cudaStream_t st)
{
    out.n_rows = nr;
    out.n_cols = ncols;
    out.rp.alloc(size_t(nr) + 1);
    if (nr) k_sub_count<<<grid_for(nr, TB), TB, 0, st>>>(nr, rows, A.rp.p, A.ci.p, colmap, out.rp.p);
    CK_LAUNCH();
    out.nnz = counts_to_rowptr(out.rp, nr, st);
    out.ci.alloc(out.nnz);
    out.v.alloc(out.nnz);
    if (nr) k_sub_fill<<<grid_for(nr, TB), TB, 0, st>>>(nr, rows, A.rp.p, A.ci.p, A.v.p, colmap,
                                                          out.rp.p, out.ci.p, out.v.p);
    CK_LAUNCH();
}

// C = A B.  Rows are processed in chunks whose hash tables hold at most
// 2^28 slots (3 GiB) together, so large fill-heavy levels neither overflow
// the int32 table offsets nor exhaust memory; each chunk's rows are emitted
// into a piece that is then copied into C.
void spgemm(const DevCSR& A, const DevCSR& B, DevCSR& C, cudaStream_t st)
{
    int m = A.n_rows;
    C.n_rows = m;
    C.n_cols = B.n_cols;
    DBuf<int> tsize(size_t(m) + 1);
    if (m) k_gemm_bound<<<grid_for(m, TB), TB, 0, st>>>(m, A.rp.p, A.ci.p, B.rp.p, tsize.p);
    CK_LAUNCH();
    std::vector<int> ts(static_cast<size_t>(m));
    d2h(ts.data(), tsize.p, size_t(m), st);
    static long long kLimit = 0;
    if (!kLimit) {
        const char* e = getenv("AIRG_SPGEMM_SLOTS");   // tuning / testing override
        kLimit = e ? std::max(1LL, atoll(e)) : (1LL << 28);
    }
    std::vector<int> cut{0};
    long long acc = 0;
    for (int i = 0; i < m; ++i) {
        if (acc + ts[i] > kLimit && i > cut.back()) { cut.push_back(i); acc = 0; }
        acc += ts[i];
    }
    cut.push_back(m);
    struct Piece {
        int r0 = 0, r1 = 0, nnz = 0;
        DBuf<int> rp, ci;
        DBuf<double> v;
    };
    std::vector<Piece> pieces;
    long long total = 0;
    for (size_t c = 0; c + 1 < cut.size(); ++c) {
        Piece P;
        P.r0 = cut[c];
        P.r1 = cut[c + 1];
        int mc = P.r1 - P.r0;
        DBuf<int> toff(size_t(mc) + 1);
        if (mc) CK(cudaMemcpyAsync(toff.p, tsize.p + P.r0, size_t(mc) * sizeof(int), cudaMemcpyDeviceToDevice, st));
        int tsz = exclusive_scan(toff.p, toff.p, mc, st);
        DBuf<int> keys(std::max(tsz, 1));
        DBuf<double> vals(std::max(tsz, 1));
        CK(cudaMemsetAsync(keys.p, 0xff, keys.bytes(), st));
        P.rp.alloc(size_t(mc) + 1);
        if (mc) {
            k_gemm_hash<<<grid_for(mc, TB), TB, 0, st>>>(mc, P.r0, A.rp.p, A.ci.p, A.v.p, B.rp.p, B.ci.p,
                                                         B.v.p, toff.p, keys.p, vals.p, P.rp.p);
            k_gemm_hash_warp<<<grid_for(mc, TB / 32), TB, 0, st>>>(mc, P.r0, A.rp.p, A.ci.p, A.v.p, B.rp.p,
                                                                   B.ci.p, B.v.p, toff.p, keys.p, vals.p, P.rp.p);
        }
        CK_LAUNCH();
        P.nnz = exclusive_scan(P.rp.p, P.rp.p, mc, st);
        P.ci.alloc(std::max(P.nnz, 1));
        P.v.alloc(std::max(P.nnz, 1));
        if (mc) {
            k_gemm_emit_small<<<grid_for(mc, TB / 32), TB, 0, st>>>(mc, toff.p, keys.p, vals.p, P.rp.p,
                                                                     P.ci.p, P.v.p);
            k_gemm_emit_warp<<<grid_for(mc, EMIT_WARPS), EMIT_WARPS * 32, 0, st>>>(mc, toff.p, keys.p, vals.p,
                                                                                   P.rp.p, P.ci.p, P.v.p);
            k_gemm_emit<<<grid_for(mc, TB), TB, 0, st>>>(mc, toff.p, keys.p, vals.p, P.rp.p, P.ci.p, P.v.p,
                                                         EMIT_CAP);
        }
        CK_LAUNCH();
        CK(cudaStreamSynchronize(st));
        total += P.nnz;
        pieces.push_back(std::move(P));
    }
    if (total > 0x7fffffffLL) fail(AIRG_ERR_OOM, "sparse product exceeds 2^31 entries");
    C.nnz = int(total);
    if (pieces.size() == 1) {
        C.rp = std::move(pieces[0].rp);
        C.ci = std::move(pieces[0].ci);
        C.v = std::move(pieces[0].v);
        return;
    }
    C.rp.alloc(size_t(m) + 1);
    C.ci.alloc(std::max(C.nnz, 1));
    C.v.alloc(std::max(C.nnz, 1));
    int off = 0;
    for (Piece& P : pieces) {
        int mc = P.r1 - P.r0;
        if (mc) k_shift_rowptr<<<grid_for(mc, TB), TB, 0, st>>>(mc, P.rp.p, off, C.rp.p + P.r0);
        CK_LAUNCH();
        if (P.nnz) {
            CK(cudaMemcpyAsync(C.ci.p + off, P.ci.p, size_t(P.nnz) * sizeof(int), cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(C.v.p + off, P.v.p, size_t(P.nnz) * sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
        off += P.nnz;
    }
    CK(cudaMemcpyAsync(C.rp.p + m, &C.nnz, sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
}

void compact(const DevCSR& A, const int8_t* keep, DBuf<int>& cnt, DevCSR& out, cudaStream_t st)
{
    int n = A.n_rows;
    out.n_rows = n;
    out.n_cols = A.n_cols;
    out.rp = std::move(cnt);
    out.nnz = counts_to_rowptr(out.rp, n, st);
    out.ci.alloc(out.nnz);
    out.v.alloc(out.nnz);
    if (n) k_compact<<<grid_for(n, TB), TB, 0, st>>>(n, A.rp.p, A.ci.p, A.v.p, keep, out.rp.p,
                                                       out.ci.p, out.v.p);
    CK_LAUNCH();
}

// Local indices of the rows with is_f == want: idx (n), ids (count); returns count
int local_index(const DBuf<int8_t>& is_f, int n, int want, DBuf<int>& idx, DBuf<int>& ids,
                cudaStream_t st)
{
    DBuf<int> ex(size_t(n) + 1);
    if (n) k_flag_eq<<<grid_for(n, TB), TB, 0, st>>>(n, is_f.p, want, ex.p);
    CK_LAUNCH();
    int cnt = exclusive_scan(ex.p, ex.p, n, st);
    idx.alloc(n);
    ids.alloc(std::max(cnt, 1));
    if (n) k_local_index<<<grid_for(n, TB), TB, 0, st>>>(n, is_f.p, want, ex.p, idx.p, ids.p);
    CK_LAUNCH();
    return cnt;
}

// ---------------------------------------------------------------- Arnoldi --
struct ArnoldiOut {
    std::vector<double> H;   // (k+1) x k row-major
    int k = 0;
    bool broke = false;
    double beta = 0.0;
};

// m steps of MGS Arnoldi from b (device, length n); dots correctly rounded.
ArnoldiOut arnoldi(Ctx& c, const DevCSR& A, const double* b, int m, double tol, double exact_tol)
{
    cudaStream_t st = c.st;
    long long n = A.n_rows;
    DBuf<double> V(size_t(m + 1) * n), w(n), Hd(size_t(m + 1) * m + 1);
    CK(cudaMemsetAsync(Hd.p, 0, Hd.bytes(), st));
    double* beta_d = Hd.p + size_t(m + 1) * m;
    xdot(c, n, b, b, nullptr, beta_d);
    int g = grid_for(n, TB);
    k_div_dev<<<g, TB, 0, st>>>(n, V.p, b, beta_d);
    CK_LAUNCH();
    std::vector<double> Hh(size_t(m + 1) * m, 0.0);
    const double beta_h = read1(beta_d, st);
    ArnoldiOut out;
    out.k = m;
    std::vector<double> col(m + 1);
    for (int j = 0; j < m; ++j) {
        k_spmv_det<<<grid_for(n, TB), TB, 0, st>>>(int(n), A.rp.p, A.ci.p, A.v.p, V.p + size_t(j) * n, w.p);
        CK_LAUNCH();
        // h_ij = <w, v_i> then w -= h_ij v_i, for i = 0..j (modified
        // Gram-Schmidt); each update is fused with the next dot product
        for (int i = 0; i <= j; ++i) {
            double* hij = Hd.p + size_t(i) * m + j;
            const double* hprev = i ? Hd.p + size_t(i - 1) * m + j : nullptr;
            mgs_xdot(c, n, w.p, i ? V.p + size_t(i - 1) * n : nullptr, hprev, V.p + size_t(i) * n, hij, nullptr);
        }
        double* hn = Hd.p + size_t(j + 1) * m + j;
        mgs_xdot(c, n, w.p, V.p + size_t(j) * n, Hd.p + size_t(j) * m + j, nullptr, nullptr, hn);
        // read column j (rows 0..j+1)
        for (int i = 0; i <= j + 1; ++i)
            CK(cudaMemcpyAsync(&col[i], Hd.p + size_t(i) * m + j, sizeof(double),
                               cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int i = 0; i <= j + 1; ++i) Hh[size_t(i) * m + j] = col[i];
        double s = 0.0;
        for (int i = 0; i <= j + 1; ++i) s = s + col[i] * col[i];
        if (col[j + 1] <= tol * std::sqrt(s)) {
            out.k = j + 1;
            out.broke = true;
            break;
        }
        {
            // GMRES residual of the (j+2) x (j+1) least-squares problem
            int kk = j + 1;
            std::vector<double> Hs(size_t(kk + 1) * kk);
            for (int i = 0; i <= kk; ++i)
                for (int q = 0; q < kk; ++q) Hs[size_t(i) * kk + q] = Hh[size_t(i) * m + q];
            if (givens_residual(Hs, kk, beta_h) <= exact_tol * beta_h) {
                out.k = kk;
                break;
            }
        }
        if (j + 1 < m) {
            k_div_dev<<<g, TB, 0, st>>>(n, V.p + size_t(j + 1) * n, w.p, hn);
            CK_LAUNCH();
        }
    }
    out.beta = beta_h;
    int k = out.k;
    out.H.assign(size_t(k + 1) * k, 0.0);
    for (int i = 0; i <= k; ++i)
        for (int j = 0; j < k; ++j) out.H[size_t(i) * k + j] = Hh[size_t(i) * m + j];
    return out;
}

std::vector<double> gmres_poly_coeffs(Ctx& c, const DevCSR& Aff, const airg_options& o, int level,
                                      int& kout, int purpose = PURPOSE_COEF)
{
    int p = o.poly_order;
    long long n = Aff.n_rows;
    DBuf<double> b(n);
    k_rng_uniform<<<grid_for(n, TB), TB, 0, c.st>>>(stream_key(o.seed, level, purpose), n, b.p);
    CK_LAUNCH();
    ArnoldiOut ar = arnoldi(c, Aff, b.p, p + 1, o.breakdown_tol, o.exact_tol);
    std::vector<double> y = givens_lsq(ar.H, ar.k, ar.beta);
    std::vector<double> alpha = power_coefficients(ar.H, ar.k, ar.beta, y);
    alpha.resize(size_t(p) + 1, 0.0);
    kout = ar.k;
    return alpha;
}

// max_i |a_ii| as the bit pattern of a non-negative double (such patterns
// order like the values), so the atomic maximum is exact and order-free
__global__ void k_diag_absmax(int n, const int* rp, const int* ci, const double* v, unsigned long long* out)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    for (int k = rp[r]; k < rp[r + 1]; ++k)
        if (ci[k] == r) {
            atomicMax(out, (unsigned long long)__double_as_longlong(fabs(v[k])));
            break;
        }
}

// nAIR (Sec. 3.3.1): power-basis coefficients of w sum_{k<=p} (I - w A)^k,
// w = 1 / max |a_ii|, i.e. alpha_j = w (-w)^j C(p+1, j+1), with (-w)^j formed
// by repeated products
std::vector<double> neumann_coeffs(const DevCSR& A, const airg_options& o, cudaStream_t st)
{
    const int p = o.poly_order;
    double dmax = 1.0;
    if (A.n_rows) {
        DBuf<unsigned long long> m(1);
        CK(cudaMemsetAsync(m.p, 0, sizeof(unsigned long long), st));
        k_diag_absmax<<<grid_for(A.n_rows, TB), TB, 0, st>>>(A.n_rows, A.rp.p, A.ci.p, A.v.p, m.p);
        CK_LAUNCH();
        unsigned long long bits = 0;
        d2h(&bits, m.p, 1, st);
        std::memcpy(&dmax, &bits, sizeof dmax);
        if (!(dmax > 0.0)) fail(AIRG_ERR_BREAKDOWN, "block without a nonzero diagonal (Neumann polynomial)");
    }
    const double w = 1.0 / dmax;
    // binomial C(p+1, j+1) from Pascal's triangle (exact in 64 bits for p <= 30)
    std::vector<unsigned long long> row(size_t(p) + 2, 0);
    row[0] = 1;
    for (int i = 1; i <= p + 1; ++i)
        for (int j = i; j >= 1; --j) row[j] += row[j - 1];
    std::vector<double> alpha(size_t(p) + 1);
    double pw = 1.0;
    for (int j = 0; j <= p; ++j) {
        alpha[j] = (w * pw) * (double)row[j + 1];
        pw = pw * -w;
    }
    return alpha;
}

std::vector<double> smoother_coeffs(Ctx& c, const DevCSR& A, const airg_options& o, int level, int& kout,
                                    int purpose)
{
    if (o.inverse_type == AIRG_INVERSE_NEUMANN) {
        kout = o.poly_order + 1;
        return neumann_coeffs(A, o, c.st);
    }
    return gmres_poly_coeffs(c, A, o, level, kout, purpose);
}

void fixed_sparsity_inverse(const DevCSR& Aff, const std::vector<double>& alpha, DevCSR& out,
                            cudaStream_t st)
{
    int n = Aff.n_rows, nnz = Aff.nnz;
    out.alloc(n, n, nnz);
    CK(cudaMemcpyAsync(out.rp.p, Aff.rp.p, (n + 1) * sizeof(int), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(out.ci.p, Aff.ci.p, nnz * sizeof(int), cudaMemcpyDeviceToDevice, st));
    if (!n) return;
    k_fsp_init<<<grid_for(n, TB), TB, 0, st>>>(n, Aff.rp.p, Aff.ci.p, alpha[0], out.v.p);
    DBuf<double> T(nnz), Tn(nnz);
    CK(cudaMemcpyAsync(T.p, Aff.v.p, nnz * sizeof(double), cudaMemcpyDeviceToDevice, st));
    for (size_t k = 1; k < alpha.size(); ++k) {
        if (k >= 2) {
            k_fsp_power<<<grid_for(n, TB), TB, 0, st>>>(n, Aff.rp.p, Aff.ci.p, Aff.v.p, T.p, Tn.p);
            k_fsp_power_warp<<<grid_for(n, TB / 32), TB, 0, st>>>(n, Aff.rp.p, Aff.ci.p, Aff.v.p, T.p, Tn.p);
            std::swap(T.p, Tn.p);
        }
        k_fsp_acc<<<grid_for(nnz, TB), TB, 0, st>>>(nnz, out.v.p, T.p, alpha[k]);
        CK_LAUNCH();
    }
    CK(cudaStreamSynchronize(st));
}

// Newton application x = q(A) b (Sec. 2.3), deterministic kernels.
void newton_apply(Ctx& c, const DevCSR& A, const std::vector<Root>& roots, const double* b,
                  double* x)
{
    cudaStream_t st = c.st;
    long long n = A.n_rows;
    DBuf<double> r(n), w(n), t(n);
    CK(cudaMemsetAsync(x, 0, n * sizeof(double), st));
    CK(cudaMemcpyAsync(r.p, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    int g = grid_for(n, TB);
    for (size_t idx = 0; idx < roots.size(); ++idx) {
        bool last = idx + 1 == roots.size();
        double a = roots[idx].re, bi = roots[idx].im;
        if (bi == 0.0) {
            k_newton_real_x<<<g, TB, 0, st>>>(n, x, r.p, a);
            if (!last) {
                k_spmv_det<<<g, TB, 0, st>>>(int(n), A.rp.p, A.ci.p, A.v.p, r.p, w.p);
                k_newton_r<<<g, TB, 0, st>>>(n, r.p, w.p, a);
            }
        } else {
            double mod2 = a * a + bi * bi;
            k_spmv_det<<<g, TB, 0, st>>>(int(n), A.rp.p, A.ci.p, A.v.p, r.p, w.p);
            k_newton_pair<<<g, TB, 0, st>>>(n, x, r.p, w.p, t.p, 2.0 * a, mod2);
            if (!last) {
                k_spmv_det<<<g, TB, 0, st>>>(int(n), A.rp.p, A.ci.p, A.v.p, t.p, w.p);
                k_newton_r<<<g, TB, 0, st>>>(n, r.p, w.p, mod2);
            }
        }
        CK_LAUNCH();
    }
    CK(cudaStreamSynchronize(st));
}

std::vector<Root> coarse_polynomial(Ctx& c, const DevCSR& A, const airg_options& o, int level,
                                    int m, int& kout)
{
    long long n = A.n_rows;
    DBuf<double> b(n);
    k_rng_uniform<<<grid_for(n, TB), TB, 0, c.st>>>(stream_key(o.seed, level, PURPOSE_COARSE), n, b.p);
    CK_LAUNCH();
    ArnoldiOut ar = arnoldi(c, A, b.p, m, o.breakdown_tol, o.exact_tol);
    std::vector<double> wr, wi;
    if (!harmonic_ritz(ar.H, ar.k, ar.broke, wr, wi))
        fail(AIRG_ERR_BREAKDOWN, "harmonic Ritz eigenvalue iteration did not converge");
    kout = ar.k;
    return order_roots(wr, wi, o.addroot_log10, o.addroot_per);
}

double truncation_residual(Ctx& c, const DevCSR& A, const std::vector<Root>& roots,
                           const airg_options& o, int level)
{
    cudaStream_t st = c.st;
    long long n = A.n_rows;
    DBuf<double> b2(n), x(n), y(n), r(n), nrm(2);
    k_rng_uniform<<<grid_for(n, TB), TB, 0, st>>>(stream_key(o.seed, level, PURPOSE_TRUNC), n, b2.p);
    CK_LAUNCH();
    newton_apply(c, A, roots, b2.p, x.p);
    k_spmv_det<<<grid_for(n, TB), TB, 0, st>>>(int(n), A.rp.p, A.ci.p, A.v.p, x.p, y.p);
    k_sub<<<grid_for(n, TB), TB, 0, st>>>(n, b2.p, y.p, r.p);
    CK_LAUNCH();
    xdot(c, n, r.p, r.p, nullptr, nrm.p);
    xdot(c, n, b2.p, b2.p, nullptr, nrm.p + 1);
    double h[2];
    d2h(h, nrm.p, 2, st);
    return h[0] / h[1];
}

// ------------------------------------------------------------- CF split --
void cf_split(Ctx& c, SetupLevel& L, const airg_options& o, int level)
{
    cudaStream_t st = c.st;
    const DevCSR& A = L.A;
    int n = A.n_rows;
    int g = grid_for(n, TB);
    L.strong.alloc(std::max(A.nnz, 1));
    k_strength<<<g, TB, 0, st>>>(n, A.rp.p, A.ci.p, A.v.p, o.strong_threshold, L.strong.p);
    // S^T
    DBuf<int> rpt(size_t(n) + 1), cursor(n);
    CK(cudaMemsetAsync(rpt.p, 0, rpt.bytes(), st));
    CK(cudaMemsetAsync(cursor.p, 0, cursor.bytes(), st));
    k_count_strong_t<<<g, TB, 0, st>>>(n, A.rp.p, A.ci.p, L.strong.p, rpt.p);
    CK_LAUNCH();
    int nst = exclusive_scan(rpt.p, rpt.p, n, st);
    DBuf<int> ct(std::max(nst, 1));
    k_fill_strong_t<<<g, TB, 0, st>>>(n, A.rp.p, A.ci.p, L.strong.p, rpt.p, cursor.p, ct.p);
    k_sort_rows<<<g, TB, 0, st>>>(n, rpt.p, ct.p);
    CK_LAUNCH();
    // G = S + S^T
    DBuf<int> rpg(size_t(n) + 1);
    k_union<<<g, TB, 0, st>>>(n, A.rp.p, A.ci.p, L.strong.p, rpt.p, ct.p, nullptr, nullptr, rpg.p);
    CK_LAUNCH();
    int ng = exclusive_scan(rpg.p, rpg.p, n, st);
    DBuf<int> cg(std::max(ng, 1));
    k_union<<<g, TB, 0, st>>>(n, A.rp.p, A.ci.p, L.strong.p, rpt.p, ct.p, rpg.p, cg.p, nullptr);
    CK_LAUNCH();
    // PMISR rounds
    DBuf<unsigned> w(n);
    DBuf<int8_t> state(n), newf(n);
    DBuf<int> und(1);
    k_rng_u32<<<g, TB, 0, st>>>(stream_key(o.seed, level, PURPOSE_PMISR), n, w.p);
    CK(cudaMemsetAsync(state.p, 0, state.bytes(), st));
    int rounds = 0;
    while (true) {
        ++rounds;
        CK(cudaMemsetAsync(und.p, 0, sizeof(int), st));
        k_pmisr_select<<<g, TB, 0, st>>>(n, rpg.p, cg.p, w.p, state.p, newf.p);
        k_pmisr_update<<<g, TB, 0, st>>>(n, rpg.p, cg.p, state.p, newf.p, und.p);
        CK_LAUNCH();
        if (read1(und.p, st) == 0) break;
        if (rounds > n + 1) fail(AIRG_ERR_STATE, "PMISR made no progress");
    }
    L.pmisr_rounds = rounds;
    L.is_f.alloc(n);
    k_state_to_f<<<g, TB, 0, st>>>(n, state.p, L.is_f.p);
    CK_LAUNCH();
    // DDC passes (Sec. 2.1): 1000 equal bins over [0, max ratio]
    const int nbins = 1000;
    DBuf<double> ratio(n);
    DBuf<int> bins(n), hist(nbins), cnt(size_t(n) + 1);
    DBuf<unsigned long long> rmax(1);
    L.ddc_converted.clear();
    for (int it = 0; it < o.ddc_its; ++it) {
        k_flag_eq<<<g, TB, 0, st>>>(n, L.is_f.p, 1, cnt.p);
        CK_LAUNCH();
        int n_f = exclusive_scan(cnt.p, cnt.p, n, st);
        if (n_f == 0) { L.ddc_converted.push_back(0); continue; }
        CK(cudaMemsetAsync(rmax.p, 0, sizeof(unsigned long long), st));
        k_ddc_ratio<<<g, TB, 0, st>>>(n, A.rp.p, A.ci.p, A.v.p, L.is_f.p, ratio.p, rmax.p);
        CK_LAUNCH();
        unsigned long long rb = read1(rmax.p, st);
        double rm;
        std::memcpy(&rm, &rb, sizeof rm);
        if (!(rm > 0.0)) { L.ddc_converted.push_back(0); continue; }
        if (std::isinf(rm)) fail(AIRG_ERR_BREAKDOWN, "zero diagonal in an F row");
        long long k = (long long)std::ceil(o.ddc_fraction * double(n_f));
        CK(cudaMemsetAsync(hist.p, 0, hist.bytes(), st));
        k_ddc_bin<<<g, TB, 0, st>>>(n, L.is_f.p, ratio.p, rm, nbins, bins.p, hist.p);
        CK_LAUNCH();
        std::vector<int> hh(nbins);
        d2h(hh.data(), hist.p, nbins, st);
        // boundary B whose count at or above it is closest to k (ties: higher B)
        long long above = 0;
        int best_b = nbins;
        long long best_d = k;   // |0 - k|
        std::vector<long long> ab(nbins + 1, 0);
        for (int b = nbins - 1; b >= 0; --b) { above += hh[b]; ab[b] = above; }
        for (int b = nbins - 1; b >= 0; --b) {
            long long d = std::llabs(ab[b] - k);
            if (d < best_d) { best_d = d; best_b = b; }
        }
        L.ddc_converted.push_back(int(best_b < nbins ? ab[best_b] : 0));
        if (best_b < nbins) {
            k_ddc_convert<<<g, TB, 0, st>>>(n, L.is_f.p, bins.p, best_b);
            CK_LAUNCH();
        }
    }
}

}  // namespace

// ===========================================================================
void dot_exact_device(long long n, const double* x, const double* y, double* out,
                      double* out_sqrt, cudaStream_t st)
{
    Ctx c(st);
    xdot(c, n, x, y, out, out_sqrt);
    CK(cudaStreamSynchronize(st));
}

void rng_uniform_device(uint64_t seed, long long level, long long purpose, long long n,
                        double* out, cudaStream_t st)
{
    if (n <= 0) return;
    k_rng_uniform<<<grid_for(n, TB), TB, 0, st>>>(stream_key(seed, level, purpose), n, out);
    CK_LAUNCH();
    CK(cudaStreamSynchronize(st));
}

void validate_csr(const DevCSR& A, bool square, cudaStream_t st)
{
    DBuf<int> flags(4);
    CK(cudaMemsetAsync(flags.p, 0, flags.bytes(), st));
    if (A.n_rows)
        k_validate<<<grid_for(A.n_rows, TB), TB, 0, st>>>(A.n_rows, A.n_cols, A.nnz, A.rp.p, A.ci.p, A.v.p,
                                                            square ? 1 : 0, flags.p);
    CK_LAUNCH();
    int f[4];
    d2h(f, flags.p, 4, st);
    if (f[2]) fail(AIRG_ERR_ARG, "row pointers not monotone within [0, nnz] with rowptr[0] = 0, rowptr[n] = nnz");
    if (f[0]) fail(AIRG_ERR_ARG, "CSR columns out of range or not strictly ascending");
    if (f[1]) fail(AIRG_ERR_ARG, "a row has no stored diagonal");
    if (f[3]) fail(AIRG_ERR_ARG, "a matrix value is not finite");
}

void csr_transpose(const DevCSR& A, DevCSR& T, cudaStream_t st)
{
    int n = A.n_rows, m = A.n_cols;
    T.n_rows = m;
    T.n_cols = n;
    T.nnz = A.nnz;
    T.rp.alloc(size_t(m) + 1);
    DBuf<int> cursor(std::max(m, 1));
    CK(cudaMemsetAsync(T.rp.p, 0, T.rp.bytes(), st));
    CK(cudaMemsetAsync(cursor.p, 0, cursor.bytes(), st));
    if (n) k_count_cols<<<grid_for(n, TB), TB, 0, st>>>(n, A.rp.p, A.ci.p, T.rp.p);
    CK_LAUNCH();
    exclusive_scan(T.rp.p, T.rp.p, m, st);
    T.ci.alloc(A.nnz);
    T.v.alloc(A.nnz);
    if (n) k_fill_transpose<<<grid_for(n, TB), TB, 0, st>>>(n, A.rp.p, A.ci.p, A.v.p, T.rp.p,
                                                              cursor.p, T.ci.p, T.v.p);
    if (m) k_sort_rows_kv<<<grid_for(m, TB), TB, 0, st>>>(m, T.rp.p, T.ci.p, T.v.p);
    CK_LAUNCH();
    CK(cudaStreamSynchronize(st));
}

std::unique_ptr<Hierarchy> build_hierarchy(DevCSR&& A0, const airg_options& o, cudaStream_t st)
{
    auto t0 = std::chrono::steady_clock::now();
    auto H = std::make_unique<Hierarchy>();
    H->opt = o;
    Ctx c(st);
    DevCSR A = std::move(A0);
    int level = 0;
    while (true) {
        int n = A.n_rows;
        bool last = level >= o.max_levels - 1 || n <= o.coarse_min_rows;
        int m_c = std::min(o.coarse_poly_order, n);
        double trunc_rel = NAN;
        const double trunc_before = H->phase_ms[AIRG_PHASE_TRUNCATION];
        if (!last && o.trunc_rtol > 0.0 && level >= o.trunc_start_level) {
            int k = 0;
            std::vector<Root> roots;
            {
                PhaseTimer pt(st, &H->phase_ms[AIRG_PHASE_TRUNCATION]);
                roots = coarse_polynomial(c, A, o, level, m_c, k);
                trunc_rel = truncation_residual(c, A, roots, o, level);
            }
            if (trunc_rel <= o.trunc_rtol) {
                // the test's polynomial becomes the coarse solver
                H->phase_ms[AIRG_PHASE_COARSE_POLY] += H->phase_ms[AIRG_PHASE_TRUNCATION] - trunc_before;
                H->phase_ms[AIRG_PHASE_TRUNCATION] = trunc_before;
                H->coarse.A = std::move(A);
                H->coarse.roots = std::move(roots);
                H->coarse.k = k;
                H->coarse.trunc_rel = trunc_rel;
                H->coarse.truncated = true;
                break;
            }
        }
        auto L = std::make_unique<SetupLevel>();
        L->n = n;
        L->A = std::move(A);
        if (!last) {
            PhaseTimer pt(st, &H->phase_ms[AIRG_PHASE_CF_SPLIT]);
            cf_split(c, *L, o, level);
            L->n_f = local_index(L->is_f, n, 1, L->f_index, L->f_ids, st);
            L->n_c = n - L->n_f;
            if (L->n_f == 0 || L->n_f == n) last = true;
        }
        if (last) {
            PhaseTimer pt(st, &H->phase_ms[AIRG_PHASE_COARSE_POLY]);
            int k = 0;
            H->coarse.roots = coarse_polynomial(c, L->A, o, level, m_c, k);
            H->coarse.k = k;
            H->coarse.trunc_rel = trunc_rel;
            H->coarse.A = std::move(L->A);
            break;
        }
        L->trunc_rel = trunc_rel;
        const DevCSR& Al = L->A;
        DevCSR A_cf;
        {
            PhaseTimer pt(st, &H->phase_ms[AIRG_PHASE_EXTRACT]);
            local_index(L->is_f, n, 0, L->c_index, L->c_ids, st);
            // blocks of Eq. 3
            submatrix(Al, L->f_ids.p, L->n_f, L->f_index.p, L->n_f, L->A_ff, st);
            submatrix(Al, L->f_ids.p, L->n_f, L->c_index.p, L->n_c, L->A_fc, st);
            submatrix(Al, L->c_ids.p, L->n_c, L->f_index.p, L->n_f, A_cf, st);
        }
        // GMRES polynomial (Eq. 7) and fixed-sparsity inverse (Eq. 8)
        {
            PhaseTimer pt(st, &H->phase_ms[AIRG_PHASE_SMOOTHER_POLY]);
            L->alpha = smoother_coeffs(c, L->A_ff, o, level, L->alpha_k, PURPOSE_COEF);
        }
        DevCSR Ainv;
        {
            PhaseTimer pt(st, &H->phase_ms[AIRG_PHASE_FIXED_SPARSITY]);
            fixed_sparsity_inverse(L->A_ff, L->alpha, Ainv, st);
        }
        // Z = -A_cf Ahat^-1, then the relative drop on R
        DevCSR Zfull;
        {
            PhaseTimer pt(st, &H->phase_ms[AIRG_PHASE_RESTRICTOR]);
            spgemm(A_cf, Ainv, Zfull, st);
        }
        if (o.smoother == AIRG_SMOOTH_ASSEMBLED) L->Ainv = std::move(Ainv);
        if (o.smooth_type != AIRG_SMOOTH_F) {
            // C-point smoothing (Sec. 2): the GMRES polynomial of A_cc from
            // its own random stream, and the row blocks its residuals use
            {
                PhaseTimer pt(st, &H->phase_ms[AIRG_PHASE_EXTRACT]);
                submatrix(Al, L->c_ids.p, L->n_c, L->c_index.p, L->n_c, L->A_cc, st);
                submatrix(Al, L->c_ids.p, L->n_c, nullptr, n, L->Crows, st);
                if (o.smooth_type == AIRG_SMOOTH_FCF) submatrix(Al, L->f_ids.p, L->n_f, nullptr, n, L->Frows, st);
            }
            {
                PhaseTimer pt(st, &H->phase_ms[AIRG_PHASE_SMOOTHER_POLY]);
                L->alpha_c = smoother_coeffs(c, L->A_cc, o, level, L->alpha_c_k, PURPOSE_COEF_C);
            }
            PhaseTimer pt(st, &H->phase_ms[AIRG_PHASE_FIXED_SPARSITY]);
            if (o.smoother == AIRG_SMOOTH_ASSEMBLED) fixed_sparsity_inverse(L->A_cc, L->alpha_c, L->Ainv_cc, st);
        }
        {
            PhaseTimer pt(st, &H->phase_ms[AIRG_PHASE_RESTRICTOR]);
            if (Zfull.nnz) k_scale<<<grid_for(Zfull.nnz, TB), TB, 0, st>>>(Zfull.nnz, Zfull.v.p, -1.0);
            DBuf<int8_t> keep(std::max(Zfull.nnz, 1));
            DBuf<int> cnt(size_t(L->n_c) + 1);
            if (L->n_c) k_drop_rows<<<grid_for(L->n_c, TB), TB, 0, st>>>(L->n_c, Zfull.rp.p, Zfull.v.p,
                                                                         o.r_drop, keep.p, cnt.p);
            CK_LAUNCH();
            compact(Zfull, keep.p, cnt, L->Z, st);
        }
        // one-point prolongator
        std::unique_ptr<PhaseTimer> pt_p = std::make_unique<PhaseTimer>(st, &H->phase_ms[AIRG_PHASE_PROLONGATOR]);
        L->W.alloc(std::max(L->n_f, 1));
        k_one_point<<<grid_for(n, TB), TB, 0, st>>>(n, Al.rp.p, Al.ci.p, Al.v.p, L->strong.p,
                                                    L->is_f.p, L->c_index.p, L->f_index.p, L->W.p);
        CK_LAUNCH();
        // P = [W; I] and R = [Z I] in the fine numbering
        DevCSR P, R, AP, Ac;
        P.n_rows = n;
        P.n_cols = L->n_c;
        P.rp.alloc(size_t(n) + 1);
        k_p_count<<<grid_for(n, TB), TB, 0, st>>>(n, L->is_f.p, L->f_index.p, L->W.p, P.rp.p);
        CK_LAUNCH();
        P.nnz = counts_to_rowptr(P.rp, n, st);
        P.ci.alloc(P.nnz);
        P.v.alloc(P.nnz);
        k_p_fill<<<grid_for(n, TB), TB, 0, st>>>(n, L->is_f.p, L->f_index.p, L->c_index.p, L->W.p,
                                                 P.rp.p, P.ci.p, P.v.p);
        CK_LAUNCH();
        R.n_rows = L->n_c;
        R.n_cols = n;
        R.nnz = L->Z.nnz + L->n_c;
        R.rp.alloc(size_t(L->n_c) + 1);
        R.ci.alloc(R.nnz);
        R.v.alloc(R.nnz);
        k_r_rowptr<<<grid_for(L->n_c + 1, TB), TB, 0, st>>>(L->n_c, L->Z.rp.p, R.rp.p);
        k_r_fill<<<grid_for(L->n_c, TB), TB, 0, st>>>(L->n_c, L->Z.rp.p, L->Z.ci.p, L->Z.v.p,
                                                      L->f_ids.p, L->c_ids.p, R.rp.p, R.ci.p, R.v.p);
        CK_LAUNCH();
        pt_p.reset();
        // A_coarse = R (A P), then drop + lump
        {
            PhaseTimer pt(st, &H->phase_ms[AIRG_PHASE_RAP]);
            spgemm(Al, P, AP, st);
            spgemm(R, AP, Ac, st);
            // rows of AP at the F points: A_fc + A_ff W (the solve's residual operator)
            submatrix(AP, L->f_ids.p, L->n_f, nullptr, L->n_c, L->M, st);
        }
        {
            PhaseTimer pt(st, &H->phase_ms[AIRG_PHASE_DROP_LUMP]);
            int nc = Ac.n_rows;
            DBuf<int8_t> keep(std::max(Ac.nnz, 1));
            DBuf<double> vout(std::max(Ac.nnz, 1));
            DBuf<int> cnt(size_t(nc) + 1), bad(1);
            CK(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
            if (nc) k_drop_lump<<<grid_for(nc, TB), TB, 0, st>>>(nc, Ac.rp.p, Ac.ci.p, Ac.v.p, o.a_drop,
                                                                o.a_lump, keep.p, vout.p, cnt.p, bad.p);
            CK_LAUNCH();
            if (read1(bad.p, st)) fail(AIRG_ERR_BREAKDOWN, "coarse row without a diagonal");
            std::swap(Ac.v.p, vout.p);
            DevCSR Acd;
            compact(Ac, keep.p, cnt, Acd, st);
            A = std::move(Acd);
        }
        CK(cudaStreamSynchronize(st));
        H->levels.push_back(std::move(L));
        ++level;
    }
    {
        PhaseTimer pt(st, &H->phase_ms[AIRG_PHASE_SOLVE_LAYOUT]);
        build_solve_data(*H, st);
    }
    H->exact_dots = c.ndots;
    CK(cudaStreamSynchronize(st));
    H->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return H;
}

}  // namespace airg
