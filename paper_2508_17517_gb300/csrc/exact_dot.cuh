// Correctly rounded dot product on the GPU.
//
// <x, y> is defined as the exact sum of the exact products x_i * y_i,
// rounded once to the nearest double (ties to even).  That value does not
// depend on the order of summation, so it is the same however the grid is
// shaped and equals any other correct implementation bit for bit; the setup
// uses it for every Arnoldi inner product and norm (Sec. 2.2-2.4) so that
// the polynomial coefficients, and from them every sparsity decision of the
// hierarchy, are reproducible.
//
// A finite double is m * 2^e with an integer m < 2^53 and e >= -1074, so the
// product of two is an integer below 2^106 (two 64-bit halves from
// __umul64hi / mul) times 2^(ex+ey), ex+ey >= -2148.  The accumulator is a
// signed fixed-point integer with least significant bit 2^-2148 stored as
// 140 digits of 32 bits, each digit held in a 64-bit word so that many
// deposits can wait for one carry pass: a product touches at most 5 digits.
// Warps deposit into shared-memory accumulators with 64-bit atomics
// (two's-complement wrap-around makes signed addition exact), blocks add
// theirs into a global accumulator, and one thread propagates carries and
// rounds.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "exact_dot_limits.h"

namespace airg {

constexpr int XD_DIGITS = 140;   // 140 * 32 = 4480 bits >= 2148 + 2046 + 2
constexpr int XD_BIAS = 2148;    // digit-bit position of 2^0
constexpr int XD_WARPS = 8;      // warps (shared accumulators) per block
constexpr int XD_THREADS = XD_WARPS * 32;

__device__ __forceinline__ bool xd_split(double x, unsigned long long& m, int& e, int& neg)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    neg = int(b >> 63);
    int ex = int((b >> 52) & 0x7ffULL);
    unsigned long long fr = b & ((1ULL << 52) - 1ULL);
    if (ex == 0) { m = fr; e = -1074; }
    else { m = fr | (1ULL << 52); e = ex - 1075; }
    return m != 0ULL;
}

// A thread's register window over six consecutive digits d0 .. d0+5 of the
// accumulator.  A product's five pieces land in digits d .. d+4 with
// d = pos >> 5; products of similar magnitude share d, so most of them are
// added in registers and only a window move (or the end of the thread's
// loop) deposits the window's digits into the shared accumulator.  The
// sums are exact integer sums, so the result does not depend on when they
// are deposited.  Headroom: each slot receives at most one 32-bit piece per
// product, like a digit of the accumulator.
struct XdWin {
    unsigned long long r[6];
    int d0;
};

__device__ __forceinline__ void xd_win_init(XdWin& w)
{
#pragma unroll
    for (int k = 0; k < 6; ++k) w.r[k] = 0ULL;
    w.d0 = -8;
}

__device__ __forceinline__ void xd_win_flush(unsigned long long* acc, XdWin& w)
{
    if (w.d0 < 0) return;
#pragma unroll
    for (int k = 0; k < 6; ++k)
        if (w.r[k]) atomicAdd(acc + w.d0 + k, w.r[k]);
}

__device__ __forceinline__ void xd_win_add(unsigned long long* acc, XdWin& w, double x, double y, int* bad)
{
    unsigned long long mx, my;
    int ex, ey, nx, ny;
    bool zx = !xd_split(x, mx, ex, nx);
    bool zy = !xd_split(y, my, ey, ny);
    if (!isfinite(x) || !isfinite(y)) { *bad = 1; return; }
    if (zx || zy) return;
    unsigned long long lo = mx * my;
    unsigned long long hi = __umul64hi(mx, my);
    const int pos = ex + ey + XD_BIAS;
    const int d = pos >> 5, sh = pos & 31;
    unsigned long long w0 = lo << sh;
    unsigned long long w1 = sh ? ((hi << sh) | (lo >> (64 - sh))) : hi;
    unsigned long long w2 = sh ? (hi >> (64 - sh)) : 0ULL;
    unsigned long long p[5] = {w0 & 0xffffffffULL, w0 >> 32, w1 & 0xffffffffULL, w1 >> 32,
                               w2 & 0xffffffffULL};
    if (nx ^ ny) {
#pragma unroll
        for (int k = 0; k < 5; ++k) p[k] = 0ULL - p[k];
    }
    if (d == w.d0 - 1) {
        // move the window down one digit (depositing its top digit)
        if (w.r[5]) atomicAdd(acc + w.d0 + 5, w.r[5]);
#pragma unroll
        for (int k = 5; k > 0; --k) w.r[k] = w.r[k - 1];
        w.r[0] = 0ULL;
        w.d0 = d;
    } else if (d != w.d0 && d != w.d0 + 1) {
        xd_win_flush(acc, w);
#pragma unroll
        for (int k = 0; k < 6; ++k) w.r[k] = 0ULL;
        w.d0 = d;
    }
    if (d == w.d0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) w.r[k] += p[k];
    } else {
#pragma unroll
        for (int k = 0; k < 5; ++k) w.r[k + 1] += p[k];
    }
}

// Block: XD_THREADS threads.  gacc: XD_DIGITS words, zero on entry of the
// first block (cleared by the caller).  bad: set when an input is inf/nan.
static __global__ void __launch_bounds__(XD_THREADS)
k_xdot_accumulate(long long n, const double* __restrict__ x, const double* __restrict__ y,
                  unsigned long long* __restrict__ gacc, int* bad)
{
    __shared__ unsigned long long sacc[XD_WARPS][XD_DIGITS];
    for (int t = threadIdx.x; t < XD_WARPS * XD_DIGITS; t += blockDim.x)
        (&sacc[0][0])[t] = 0ULL;
    __syncthreads();
    unsigned long long* mine = sacc[threadIdx.x >> 5];
    XdWin win;
    xd_win_init(win);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        xd_win_add(mine, win, x[i], y[i], bad);
    xd_win_flush(mine, win);
    __syncthreads();
    for (int t = threadIdx.x; t < XD_DIGITS; t += blockDim.x) {
        unsigned long long s = 0ULL;
#pragma unroll
        for (int w = 0; w < XD_WARPS; ++w) s += sacc[w][t];
        if (s) atomicAdd(gacc + t, s);
    }
}

// One thread: carry propagation and round-to-nearest-even of an accumulator
// (a copy in shared memory; the callers load the global digits in parallel
// first).  Returns the double and leaves the digits cleared.
static __device__ inline double xd_round(unsigned long long* g)
{
    long long* d = reinterpret_cast<long long*>(g);
    long long carry = 0;
    for (int i = 0; i < XD_DIGITS - 1; ++i) {
        long long v = d[i] + carry;
        long long lo = v & 0xffffffffLL;
        d[i] = lo;
        carry = (v - lo) >> 32;   // v - lo is a multiple of 2^32
    }
    d[XD_DIGITS - 1] += carry;
    int neg = 0;
    if (d[XD_DIGITS - 1] < 0) {
        neg = 1;
        carry = 0;
        for (int i = 0; i < XD_DIGITS; ++i) d[i] = -d[i];
        for (int i = 0; i < XD_DIGITS - 1; ++i) {
            long long v = d[i] + carry;
            long long lo = v & 0xffffffffLL;
            d[i] = lo;
            carry = (v - lo) >> 32;
        }
        d[XD_DIGITS - 1] += carry;
    }
    int top = -1;
    for (int i = XD_DIGITS - 1; i >= 0; --i)
        if (d[i] != 0) { top = i; break; }
    double r = 0.0;
    if (top >= 0) {
        int hb = 63 - __clzll(d[top]);
        int P = top * 32 + hb;                 // most significant bit
        int lsb = P - 52;                      // last bit kept
        if (lsb < XD_BIAS - 1074) lsb = XD_BIAS - 1074;
        unsigned long long M = 0ULL;
        for (int b = P; b >= lsb; --b) M = (M << 1) | (unsigned long long)((d[b >> 5] >> (b & 31)) & 1);
        int rb = (lsb - 1 >= 0) ? int((d[(lsb - 1) >> 5] >> ((lsb - 1) & 31)) & 1) : 0;
        int sticky = 0;
        int lim = lsb - 1;                     // bits [0, lim) are sticky bits
        for (int w = 0; w < (lim >> 5) && !sticky; ++w) sticky = d[w] != 0;
        if (!sticky && lim > 0 && (lim & 31)) {
            long long mask = (1LL << (lim & 31)) - 1;
            sticky = (d[lim >> 5] & mask) != 0;
        }
        if (rb && (sticky || (M & 1ULL))) M += 1ULL;
        r = scalbn((double)M, lsb - XD_BIAS);
    }
    for (int i = 0; i < XD_DIGITS; ++i) d[i] = 0;
    return neg ? -r : r;
}

// One warp: takes the global digits into shared memory (reading and
// clearing each word in one atomic exchange), then one thread rounds.
// Writes the double to *out and optionally its square root to *out_sqrt.
static __global__ void k_xdot_finalize(unsigned long long* gacc, const int* bad, double* out,
                                       double* out_sqrt)
{
    __shared__ unsigned long long d[XD_DIGITS];
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    for (int t = threadIdx.x; t < XD_DIGITS; t += 32) d[t] = atomicExch(gacc + t, 0ULL);
    __syncwarp();
    if (threadIdx.x != 0) return;
    double r = xd_round(d);
    if (*(volatile const int*)bad) r = __longlong_as_double(0x7ff8000000000000LL);
    if (out) *out = r;
    if (out_sqrt) *out_sqrt = __dsqrt_rn(r);
}

// Accumulation and rounding in one launch: blocks deposit as in
// k_xdot_accumulate; the last block to finish (atomic ticket, reset for the
// next call) takes the global digits, clearing them, and rounds.
static __global__ void __launch_bounds__(XD_THREADS)
k_xdot(long long n, const double* __restrict__ x, const double* __restrict__ y,
       unsigned long long* __restrict__ gacc, int* bad, unsigned* ticket, double* out, double* out_sqrt)
{
    __shared__ unsigned long long sacc[XD_WARPS][XD_DIGITS];
    __shared__ bool last;
    for (int t = threadIdx.x; t < XD_WARPS * XD_DIGITS; t += blockDim.x)
        (&sacc[0][0])[t] = 0ULL;
    __syncthreads();
    unsigned long long* mine = sacc[threadIdx.x >> 5];
    XdWin win;
    xd_win_init(win);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        xd_win_add(mine, win, x[i], y[i], bad);
    xd_win_flush(mine, win);
    __syncthreads();
    for (int t = threadIdx.x; t < XD_DIGITS; t += blockDim.x) {
        unsigned long long s = 0ULL;
#pragma unroll
        for (int w = 0; w < XD_WARPS; ++w) s += sacc[w][t];
        if (s) atomicAdd(gacc + t, s);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int t = threadIdx.x; t < XD_DIGITS; t += blockDim.x) sacc[0][t] = atomicExch(gacc + t, 0ULL);
    __syncthreads();
    if (threadIdx.x != 0) return;
    double r = xd_round(sacc[0]);
    if (*(volatile const int*)bad) r = __longlong_as_double(0x7ff8000000000000LL);
    if (out) *out = r;
    if (out_sqrt) *out_sqrt = __dsqrt_rn(r);
    *ticket = 0u;
}

// One modified Gram-Schmidt step fused with the next correctly rounded dot
// product, in one pass: when vprev is given, w_i <- w_i - (h * vprev_i)
// with h = *hprev (product rounded, then the difference: the same two
// roundings as a separate update kernel); then <w, y> (y = w itself when
// null) accumulated exactly and rounded by the last block, as k_xdot.
static __global__ void __launch_bounds__(XD_THREADS)
k_mgs_xdot(long long n, double* __restrict__ w, const double* __restrict__ vprev, const double* hprev,
           const double* __restrict__ y, unsigned long long* __restrict__ gacc, int* bad, unsigned* ticket,
           double* out, double* out_sqrt)
{
    __shared__ unsigned long long sacc[XD_WARPS][XD_DIGITS];
    __shared__ bool last;
    for (int t = threadIdx.x; t < XD_WARPS * XD_DIGITS; t += blockDim.x)
        (&sacc[0][0])[t] = 0ULL;
    __syncthreads();
    unsigned long long* mine = sacc[threadIdx.x >> 5];
    XdWin win;
    xd_win_init(win);
    const double h = vprev ? *hprev : 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double wi = w[i];
        if (vprev) {
            wi = __dsub_rn(wi, __dmul_rn(h, vprev[i]));
            w[i] = wi;
        }
        xd_win_add(mine, win, wi, y ? y[i] : wi, bad);
    }
    xd_win_flush(mine, win);
    __syncthreads();
    for (int t = threadIdx.x; t < XD_DIGITS; t += blockDim.x) {
        unsigned long long s = 0ULL;
#pragma unroll
        for (int q = 0; q < XD_WARPS; ++q) s += sacc[q][t];
        if (s) atomicAdd(gacc + t, s);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int t = threadIdx.x; t < XD_DIGITS; t += blockDim.x) sacc[0][t] = atomicExch(gacc + t, 0ULL);
    __syncthreads();
    if (threadIdx.x != 0) return;
    double r = xd_round(sacc[0]);
    if (*(volatile const int*)bad) r = __longlong_as_double(0x7ff8000000000000LL);
    if (out) *out = r;
    if (out_sqrt) *out_sqrt = __dsqrt_rn(r);
    *ticket = 0u;
}

}  // namespace airg
