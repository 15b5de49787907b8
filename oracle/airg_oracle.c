/*
 * AIRG oracle kernels -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded C in IEEE binary64 that restates the setup and
 * solve steps of AIRG (reduction multigrid with GMRES polynomials, PMISR DDC
 * CF splitting) for the upwind advection operator.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load this file's
 * shared object; the product library never links, loads or calls it.
 *
 * Compiled with -O2 -ffp-contract=off: every product is rounded before it is
 * added, sums run in the order written below, and no FMA is formed, so the
 * results are the same on x86-64 and aarch64.
 *
 * Indices are int64; CSR column indices are strictly ascending in each row.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers: SplitMix64 (Steele, Lea & Flood, "Fast      */
/* splittable pseudorandom number generators", OOPSLA 2014).  The i-th       */
/* output of a stream whose state starts at `key` is mix(key + (i+1)*gamma). */
/* Random vectors drawn during setup (Sec. 2.2 / 2.4: random rhs for the      */
/* polynomial coefficients and for the truncation test; PMISR's Luby         */
/* weights) come from here.                                                   */
/* ------------------------------------------------------------------------ */
#define SM64_GAMMA 0x9e3779b97f4a7c15ULL

static uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Stream key for (seed, level, purpose): output number `tag` of the stream
 * started at `seed`, with tag = (level << 8 | purpose). */
uint64_t orc_rng_key(uint64_t seed, int64_t level, int64_t purpose)
{
    uint64_t tag = ((uint64_t)level << 8) | (uint64_t)purpose;
    return sm64_mix(seed + SM64_GAMMA * (tag + 1));
}

/* Uniform [0,1): top 53 bits of each output, times 2^-53 (exact). */
void orc_rng_uniform(uint64_t key, int64_t n, double* out)
{
    for (int64_t i = 0; i < n; ++i) {
        uint64_t z = sm64_mix(key + SM64_GAMMA * (uint64_t)(i + 1));
        out[i] = (double)(z >> 11) * 0x1.0p-53;
    }
}

/* 32-bit draws: top 32 bits of each output. */
void orc_rng_u32(uint64_t key, int64_t n, uint32_t* out)
{
    for (int64_t i = 0; i < n; ++i) {
        uint64_t z = sm64_mix(key + SM64_GAMMA * (uint64_t)(i + 1));
        out[i] = (uint32_t)(z >> 32);
    }
}

/* ------------------------------------------------------------------------ */
/* Correctly rounded dot product.                                            */
/* The definition of <x,y> is the exact sum of the exact products, rounded   */
/* once to nearest (ties to even).  Each double is m*2^e with an integer     */
/* mantissa m < 2^53 and e >= -1074, so each product is an integer below     */
/* 2^106 times 2^(ea+eb) with ea+eb >= -2148.  All products are added into   */
/* one big signed integer whose least significant bit weighs 2^-2148, stored */
/* in 32-bit limbs (held in int64 so that carries can wait), and the total   */
/* is rounded to a double at the end.                                        */
/* ------------------------------------------------------------------------ */
#define XL 140              /* 140*32 = 4480 bits > 4196 needed            */
#define XBIAS 2148          /* bit position of 2^0                          */

typedef struct {
    int64_t d[XL];
    int64_t since_norm;
    int bad;
} xacc;

static void xacc_normalize(xacc* a)
{
    int64_t carry = 0;
    for (int i = 0; i < XL - 1; ++i) {
        int64_t v = a->d[i] + carry;
        int64_t lo = v & 0xffffffffLL;          /* v mod 2^32, in [0,2^32) */
        a->d[i] = lo;
        carry = (v - lo) / 4294967296LL;        /* exact division          */
    }
    a->d[XL - 1] += carry;                      /* top limb keeps the sign */
    a->since_norm = 0;
}

static int split_double(double x, uint64_t* m, int64_t* e, int* neg)
{
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    *neg = (int)(b >> 63);
    uint64_t ex = (b >> 52) & 0x7ffULL;
    uint64_t fr = b & ((1ULL << 52) - 1ULL);
    if (ex == 0x7ffULL) return -1;              /* inf or nan              */
    if (ex == 0) { *m = fr; *e = -1074; }
    else { *m = fr | (1ULL << 52); *e = (int64_t)ex - 1075; }
    return *m != 0;
}

static void xacc_add_product(xacc* a, double x, double y)
{
    uint64_t mx, my; int64_t ex, ey; int nx, ny;
    int rx = split_double(x, &mx, &ex, &nx);
    int ry = split_double(y, &my, &ey, &ny);
    if (rx < 0 || ry < 0) { a->bad = 1; return; }
    if (rx == 0 || ry == 0) return;
    unsigned __int128 p = (unsigned __int128)mx * (unsigned __int128)my;
    int64_t pos = ex + ey + XBIAS;              /* >= 0                    */
    int64_t limb = pos >> 5;
    int sh = (int)(pos & 31);
    int neg = nx ^ ny;
    for (int k = 0; k < 5; ++k) {
        uint64_t piece;
        int rs = 32 * k - sh;                   /* right shift for piece k */
        if (k == 0) piece = (((uint64_t)p) << sh) & 0xffffffffULL;
        else if (rs >= 128) piece = 0;          /* nothing left up there   */
        else piece = (uint64_t)(p >> rs) & 0xffffffffULL;
        if (piece == 0) continue;
        a->d[limb + k] += neg ? -(int64_t)piece : (int64_t)piece;
    }
    if (++a->since_norm >= (1LL << 24)) xacc_normalize(a);
}

static int xacc_bit(const xacc* a, int64_t b)
{
    if (b < 0) return 0;
    return (int)((a->d[b >> 5] >> (b & 31)) & 1);
}

static double xacc_round(xacc* a)
{
    if (a->bad) return NAN;
    xacc_normalize(a);
    int neg = 0;
    if (a->d[XL - 1] < 0) {
        neg = 1;
        for (int i = 0; i < XL; ++i) a->d[i] = -a->d[i];
        xacc_normalize(a);
    }
    int top = -1;
    for (int i = XL - 1; i >= 0; --i)
        if (a->d[i] != 0) { top = i; break; }
    if (top < 0) return 0.0;
    int hb = 63 - __builtin_clzll((unsigned long long)a->d[top]);
    int64_t P = (int64_t)top * 32 + hb;          /* most significant bit  */
    int64_t lsb = P - 52;                        /* ulp of the result     */
    if (lsb < XBIAS - 1074) lsb = XBIAS - 1074;  /* subnormal floor       */
    uint64_t M = 0;
    for (int64_t b = P; b >= lsb; --b) M = (M << 1) | (uint64_t)xacc_bit(a, b);
    int rb = xacc_bit(a, lsb - 1);
    int sticky = 0;
    for (int64_t b = lsb - 2; b >= 0 && !sticky; --b) sticky = xacc_bit(a, b);
    if (rb && (sticky || (M & 1ULL))) M += 1;
    double r = ldexp((double)M, (int)(lsb - XBIAS));
    return neg ? -r : r;
}

double orc_dot_exact(int64_t n, const double* x, const double* y)
{
    xacc* a = (xacc*)calloc(1, sizeof(xacc));
    for (int64_t i = 0; i < n; ++i) xacc_add_product(a, x[i], y[i]);
    double r = xacc_round(a);
    free(a);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Sparse matrix-vector product y = A x, each row summed left to right in    */
/* column order starting from +0.0, every product rounded before the add.    */
/* ------------------------------------------------------------------------ */
void orc_spmv(int64_t n, const int64_t* rp, const int64_t* ci, const double* v,
              const double* x, double* y)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s = s + v[k] * x[ci[k]];
        y[i] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Strength of connection (Sec. 2.1, PMISR operates on S + S^T).             */
/* Off-diagonal (i,j) is strong iff |a_ij| >= theta * max_{k!=i} |a_ik| and   */
/* that maximum is positive.                                                 */
/* ------------------------------------------------------------------------ */
void orc_strength(int64_t n, const int64_t* rp, const int64_t* ci, const double* v,
                  double theta, int8_t* strong)
{
    for (int64_t i = 0; i < n; ++i) {
        double m = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] != i && fabs(v[k]) > m) m = fabs(v[k]);
        double thr = theta * m;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            strong[k] = (int8_t)(ci[k] != i && m > 0.0 && fabs(v[k]) >= thr);
    }
}

/* ------------------------------------------------------------------------ */
/* DDC diagonal-dominance ratio of each F row (Sec. 2.1):                    */
/*   ratio_i = (sum_{j in F, j != i} |a_ij|) / |a_ii|                         */
/* summed in column order from +0.0.  C rows get -1.  A zero diagonal gives   */
/* +inf.                                                                     */
/* ------------------------------------------------------------------------ */
void orc_ddc_ratio(int64_t n, const int64_t* rp, const int64_t* ci, const double* v,
                   const int8_t* is_f, double* ratio)
{
    for (int64_t i = 0; i < n; ++i) {
        if (!is_f[i]) { ratio[i] = -1.0; continue; }
        double s = 0.0, d = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            int64_t j = ci[k];
            if (j == i) d = fabs(v[k]);
            else if (is_f[j]) s = s + fabs(v[k]);
        }
        ratio[i] = (d > 0.0) ? s / d : INFINITY;
    }
}

/* ------------------------------------------------------------------------ */
/* One power of the fixed-sparsity approximate inverse (Eq. 8):              */
/*   T_k = mask_{pattern(A_ff)}(A_ff T_{k-1})                                 */
/* For each stored (i,j): t_ij = sum over l in row i of A_ff (ascending) with */
/* (l,j) stored, of a_il * t_{k-1,lj}; from +0.0, left to right.             */
/* ------------------------------------------------------------------------ */
static int64_t find_col(const int64_t* ci, int64_t lo, int64_t hi, int64_t j)
{
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (ci[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

void orc_fixed_sparsity_power(int64_t n, const int64_t* rp, const int64_t* ci,
                              const double* a, const double* tprev, double* tout)
{
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
            int64_t j = ci[q];
            double s = 0.0;
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                int64_t l = ci[p];
                int64_t r = find_col(ci, rp[l], rp[l + 1], j);
                if (r < rp[l + 1] && ci[r] == j) s = s + a[p] * tprev[r];
            }
            tout[q] = s;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sparse matrix-matrix product C = A B (rows of A times B, Gustavson).      */
/* Every entry c_ij is the sum over the stored a_il of row i, in ascending l, */
/* of a_il * b_lj, from +0.0 left to right.  Output columns ascending.       */
/* Returns 0, or -1 when out of memory.  Caller frees *crp, *cci, *cv.       */
/* ------------------------------------------------------------------------ */
static int cmp_i64(const void* a, const void* b)
{
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

int orc_spgemm(int64_t m, const int64_t* arp, const int64_t* aci, const double* av,
               int64_t ncols, const int64_t* brp, const int64_t* bci, const double* bv,
               int64_t** crp_out, int64_t** cci_out, double** cv_out)
{
    int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncols > 0 ? ncols : 1));
    double* acc = (double*)malloc(sizeof(double) * (size_t)(ncols > 0 ? ncols : 1));
    int64_t* crp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m + 1));
    if (!mark || !acc || !crp) { free(mark); free(acc); free(crp); return -1; }
    for (int64_t j = 0; j < ncols; ++j) mark[j] = -1;
    crp[0] = 0;
    for (int64_t i = 0; i < m; ++i) {                 /* symbolic */
        int64_t cnt = 0;
        for (int64_t p = arp[i]; p < arp[i + 1]; ++p) {
            int64_t l = aci[p];
            for (int64_t q = brp[l]; q < brp[l + 1]; ++q)
                if (mark[bci[q]] != i) { mark[bci[q]] = i; ++cnt; }
        }
        crp[i + 1] = crp[i] + cnt;
    }
    int64_t nnz = crp[m];
    int64_t* cci = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    double* cv = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    if (!cci || !cv) { free(mark); free(acc); free(crp); free(cci); free(cv); return -1; }
    for (int64_t j = 0; j < ncols; ++j) mark[j] = -1;
    for (int64_t i = 0; i < m; ++i) {                 /* numeric */
        int64_t base = crp[i], cnt = 0;
        for (int64_t p = arp[i]; p < arp[i + 1]; ++p) {
            int64_t l = aci[p];
            for (int64_t q = brp[l]; q < brp[l + 1]; ++q) {
                int64_t j = bci[q];
                if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; cci[base + cnt++] = j; }
                acc[j] = acc[j] + av[p] * bv[q];
            }
        }
        qsort(cci + base, (size_t)cnt, sizeof(int64_t), cmp_i64);
        for (int64_t t = 0; t < cnt; ++t) cv[base + t] = acc[cci[base + t]];
    }
    free(mark); free(acc);
    *crp_out = crp; *cci_out = cci; *cv_out = cv;
    return 0;
}

void orc_free(void* p) { free(p); }

/* ------------------------------------------------------------------------ */
/* Relative drop with lumping for the coarse matrix (Sec. 2, after Eq. 6):   */
/* off-diagonal a_ij is dropped when a_ij == 0 or |a_ij| < tol * max_{k!=i}  */
/* |a_ik|; with lump != 0 the dropped values are added to the diagonal, one  */
/* by one in column order, starting from a_ii.  keep[k] flags survivors;     */
/* vout receives the values with the new diagonal.  Returns -1 when a row    */
/* has no stored diagonal, else 0.                                           */
/* ------------------------------------------------------------------------ */
int orc_drop_lump(int64_t n, const int64_t* rp, const int64_t* ci, const double* v,
                  double tol, int lump, int8_t* keep, double* vout)
{
    for (int64_t i = 0; i < n; ++i) {
        double m = 0.0;
        int64_t dpos = -1;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            if (ci[k] == i) dpos = k;
            else if (fabs(v[k]) > m) m = fabs(v[k]);
        }
        if (dpos < 0) return -1;
        double thr = tol * m;
        double d = v[dpos];
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            vout[k] = v[k];
            if (k == dpos) { keep[k] = 1; continue; }
            if (v[k] == 0.0 || fabs(v[k]) < thr) {
                keep[k] = 0;
                if (lump) d = d + v[k];
            } else {
                keep[k] = 1;
            }
        }
        vout[dpos] = d;
    }
    return 0;
}

/* Relative drop for the restrictor block Z (no diagonal, no lumping):
 * z_ij survives iff z_ij != 0 and |z_ij| >= tol * max_k |z_ik|. */
void orc_drop_rows(int64_t n, const int64_t* rp, const double* v, double tol, int8_t* keep)
{
    for (int64_t i = 0; i < n; ++i) {
        double m = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            if (fabs(v[k]) > m) m = fabs(v[k]);
        double thr = tol * m;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            keep[k] = (int8_t)(v[k] != 0.0 && fabs(v[k]) >= thr);
    }
}

/* ------------------------------------------------------------------------ */
/* Classical one-point prolongator (Sec. 2): each F point takes its value     */
/* from one C point, the C neighbour of largest |a_ij| among its strong       */
/* connections (among all C neighbours when none is strong), lowest column    */
/* on ties, with weight 1.  w[i] = C-local index of that point, or -1 when   */
/* row i is a C point or has no C neighbour.                                  */
/* ------------------------------------------------------------------------ */
void orc_one_point(int64_t n, const int64_t* rp, const int64_t* ci, const double* v,
                   const int8_t* strong, const int8_t* is_f, const int64_t* c_index,
                   int64_t* w)
{
    for (int64_t i = 0; i < n; ++i) {
        w[i] = -1;
        if (!is_f[i]) continue;
        int64_t best = -1;
        for (int pass = 0; pass < 2 && best < 0; ++pass) {
            double bestv = -1.0;
            for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
                int64_t j = ci[k];
                if (j == i || is_f[j]) continue;
                if (pass == 0 && !strong[k]) continue;
                if (fabs(v[k]) > bestv) { bestv = fabs(v[k]); best = j; }
            }
        }
        if (best >= 0) w[i] = c_index[best];
    }
}

/* ------------------------------------------------------------------------ */
/* Sweep (Sec. 1.1): the upwind-ordered substitution that solves a system    */
/* whose matrix is triangular in the given order, exactly up to rounding.    */
/* Returns -1 if a row needs a value that is not yet known, -2 on a missing  */
/* diagonal, else 0.                                                         */
/* ------------------------------------------------------------------------ */
int orc_sweep(int64_t n, const int64_t* rp, const int64_t* ci, const double* v,
              const int64_t* order, const double* b, double* u)
{
    int8_t* done = (int8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    for (int64_t t = 0; t < n; ++t) {
        int64_t i = order[t];
        double s = b[i], d = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            int64_t j = ci[k];
            if (j == i) { d = v[k]; continue; }
            if (!done[j]) { free(done); return -1; }
            s = s - v[k] * u[j];
        }
        if (d == 0.0) { free(done); return -2; }
        u[i] = s / d;
        done[i] = 1;
    }
    free(done);
    return 0;
}
