// Host FP64 dense steps of the AIRG setup.  Compiled with
// -ffp-contract=off: every operation below is one IEEE-rounded operation in
// the order written, so the coefficient computation of Eq. 7 gives the same
// bits as any other implementation that performs the same operations.
#include "hostmath.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <limits>

namespace airg {

namespace {

// Givens QR of the (k+1) x k Hessenberg H (row-major) applied to beta e1:
// R overwrites a copy of H, g is the rotated right-hand side.
void givens_qr(const std::vector<double>& H, int k, double beta, std::vector<double>& R,
               std::vector<double>& g)
{
    R.assign(H.begin(), H.begin() + size_t(k + 1) * k);
    auto at = [&](int i, int j) -> double& { return R[size_t(i) * k + j]; };
    std::vector<double> cs(k, 0.0), sn(k, 0.0);
    g.assign(size_t(k) + 1, 0.0);
    g[0] = beta;
    for (int j = 0; j < k; ++j) {
        for (int i = 0; i < j; ++i) {
            double t1 = cs[i] * at(i, j) + sn[i] * at(i + 1, j);
            double t2 = -sn[i] * at(i, j) + cs[i] * at(i + 1, j);
            at(i, j) = t1;
            at(i + 1, j) = t2;
        }
        double a = at(j, j), b = at(j + 1, j);
        double r = std::sqrt(a * a + b * b);
        cs[j] = a / r;
        sn[j] = b / r;
        at(j, j) = r;
        at(j + 1, j) = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
    }
}

}  // namespace

double givens_residual(const std::vector<double>& H, int k, double beta)
{
    std::vector<double> R, g;
    givens_qr(H, k, beta, R, g);
    return std::fabs(g[k]);
}

std::vector<double> givens_lsq(const std::vector<double>& H, int k, double beta)
{
    std::vector<double> R, g, y(k, 0.0);
    givens_qr(H, k, beta, R, g);
    auto at = [&](int i, int j) -> double& { return R[size_t(i) * k + j]; };
    for (int j = k - 1; j >= 0; --j) {
        double s = g[j];
        for (int i = j + 1; i < k; ++i) s = s - at(j, i) * y[i];
        y[j] = s / at(j, j);
    }
    return y;
}

std::vector<double> power_coefficients(const std::vector<double>& H, int k, double beta,
                                       const std::vector<double>& y)
{
    auto h = [&](int i, int j) { return H[size_t(i) * k + j]; };
    std::vector<std::vector<double>> c(k, std::vector<double>(k, 0.0));
    c[0][0] = 1.0 / beta;
    for (int j = 0; j < k - 1; ++j) {
        double hn = h(j + 1, j);
        for (int t = 0; t < j + 2; ++t) {
            double num = t >= 1 ? c[j][t - 1] : 0.0;
            for (int i = 0; i < j + 1; ++i) num = num - h(i, j) * c[i][t];
            c[j + 1][t] = num / hn;
        }
    }
    std::vector<double> alpha(k, 0.0);
    for (int t = 0; t < k; ++t) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s = s + y[j] * c[j][t];
        alpha[t] = s;
    }
    return alpha;
}

// ---------------------------------------------------------------------------
// Francis double-shift QR on an upper Hessenberg matrix (Golub & Van Loan,
// Matrix Computations, Sec. 7.5): deflate on negligible subdiagonals, take
// the eigenvalues of trailing 1x1 / 2x2 blocks, otherwise chase a 3x3
// Householder bulge with the two eigenvalues of the trailing 2x2 block as
// shifts; every tenth step without deflation uses an ad-hoc shift.
// ---------------------------------------------------------------------------
namespace {

void eig2x2(double a, double b, double c, double d, double& r1, double& i1, double& r2,
            double& i2)
{
    double m = 0.5 * (a + d);
    double p = 0.5 * (a - d);
    double disc = p * p + b * c;
    if (disc >= 0.0) {
        double sq = std::sqrt(disc);
        double l1 = m + (m >= 0.0 ? sq : -sq);
        double det = a * d - b * c;
        double l2 = (l1 != 0.0) ? det / l1 : m - sq;
        r1 = l1; i1 = 0.0; r2 = l2; i2 = 0.0;
    } else {
        double sq = std::sqrt(-disc);
        r1 = m; i1 = sq; r2 = m; i2 = -sq;
    }
}

// Householder reflector P = I - beta v v^T with P x = -sign(x0)||x|| e1.
int householder(const double* x, int len, double* v, double& beta)
{
    double nrm = 0.0;
    for (int i = 0; i < len; ++i) nrm = std::hypot(nrm, x[i]);
    if (nrm == 0.0) { beta = 0.0; return 0; }
    double alpha = x[0] >= 0.0 ? -nrm : nrm;
    v[0] = x[0] - alpha;
    for (int i = 1; i < len; ++i) v[i] = x[i];
    double vtv = 0.0;
    for (int i = 0; i < len; ++i) vtv += v[i] * v[i];
    beta = vtv > 0.0 ? 2.0 / vtv : 0.0;
    return 1;
}

}  // namespace

bool hessenberg_eigvals(int n, std::vector<double> H, std::vector<double>& wr,
                        std::vector<double>& wi)
{
    wr.assign(n, 0.0);
    wi.assign(n, 0.0);
    auto a = [&](int i, int j) -> double& { return H[size_t(i) * n + j]; };
    const double eps = std::numeric_limits<double>::epsilon();
    double anorm = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = std::max(0, i - 1); j < n; ++j) anorm = std::max(anorm, std::fabs(a(i, j)));
    int hi = n - 1;
    int its = 0, total = 0;
    const int max_total = 60 * std::max(n, 1);
    while (hi >= 0) {
        // find the start l of the unreduced block ending at hi
        int l = hi;
        while (l > 0) {
            double s = std::fabs(a(l - 1, l - 1)) + std::fabs(a(l, l));
            if (s == 0.0) s = anorm;
            if (std::fabs(a(l, l - 1)) <= eps * s) { a(l, l - 1) = 0.0; break; }
            --l;
        }
        if (l == hi) {                      // 1x1 block
            wr[hi] = a(hi, hi);
            wi[hi] = 0.0;
            --hi;
            its = 0;
            continue;
        }
        if (l == hi - 1) {                  // 2x2 block
            double r1, i1, r2, i2;
            eig2x2(a(hi - 1, hi - 1), a(hi - 1, hi), a(hi, hi - 1), a(hi, hi), r1, i1, r2, i2);
            wr[hi - 1] = r1; wi[hi - 1] = i1;
            wr[hi] = r2; wi[hi] = i2;
            hi -= 2;
            its = 0;
            continue;
        }
        if (++total > max_total) return false;
        ++its;
        // shifts: eigenvalues of the trailing 2x2 block (sum s, product t)
        double s, t;
        if (its % 10 == 0) {
            double w = std::fabs(a(hi, hi - 1)) + std::fabs(a(hi - 1, hi - 2));
            s = 1.5 * w + a(hi, hi);
            t = w * w;
        } else {
            s = a(hi - 1, hi - 1) + a(hi, hi);
            t = a(hi - 1, hi - 1) * a(hi, hi) - a(hi - 1, hi) * a(hi, hi - 1);
        }
        // first column of (H - s1 I)(H - s2 I) restricted to the block
        double x = a(l, l) * a(l, l) + a(l, l + 1) * a(l + 1, l) - s * a(l, l) + t;
        double y = a(l + 1, l) * (a(l, l) + a(l + 1, l + 1) - s);
        double z = a(l + 1, l) * a(l + 2, l + 1);
        for (int k = l; k <= hi - 2; ++k) {
            double xv[3] = {x, y, z}, v[3], beta;
            householder(xv, 3, v, beta);
            if (beta != 0.0) {
                int c0 = std::max(l, k - 1);
                for (int j = c0; j <= hi; ++j) {            // rows k..k+2
                    double d = v[0] * a(k, j) + v[1] * a(k + 1, j) + v[2] * a(k + 2, j);
                    d *= beta;
                    a(k, j) -= d * v[0];
                    a(k + 1, j) -= d * v[1];
                    a(k + 2, j) -= d * v[2];
                }
                int r1 = std::min(hi, k + 3);
                for (int i = l; i <= r1; ++i) {             // columns k..k+2
                    double d = a(i, k) * v[0] + a(i, k + 1) * v[1] + a(i, k + 2) * v[2];
                    d *= beta;
                    a(i, k) -= d * v[0];
                    a(i, k + 1) -= d * v[1];
                    a(i, k + 2) -= d * v[2];
                }
            }
            x = a(k + 1, k);
            y = a(k + 2, k);
            if (k < hi - 2) z = a(k + 3, k);
        }
        // final 2x2 reflector on rows/columns hi-1, hi
        {
            double xv[2] = {x, y}, v[2], beta;
            householder(xv, 2, v, beta);
            if (beta != 0.0) {
                for (int j = std::max(l, hi - 2); j <= hi; ++j) {
                    double d = beta * (v[0] * a(hi - 1, j) + v[1] * a(hi, j));
                    a(hi - 1, j) -= d * v[0];
                    a(hi, j) -= d * v[1];
                }
                for (int i = l; i <= hi; ++i) {
                    double d = beta * (a(i, hi - 1) * v[0] + a(i, hi) * v[1]);
                    a(i, hi - 1) -= d * v[0];
                    a(i, hi) -= d * v[1];
                }
            }
        }
    }
    return true;
}

bool harmonic_ritz(const std::vector<double>& H, int k, bool broke, std::vector<double>& wr,
                   std::vector<double>& wi)
{
    // H is (k+1) x k; take the leading k x k block
    std::vector<double> T(size_t(k) * k);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) T[size_t(i) * k + j] = H[size_t(i) * k + j];
    if (!broke) {
        // f = H_k^{-T} e_k: LU with partial pivoting of H_k^T
        std::vector<double> M(size_t(k) * k), f(k, 0.0);
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) M[size_t(i) * k + j] = T[size_t(j) * k + i];
        f[k - 1] = 1.0;
        std::vector<int> piv(k);
        for (int c = 0; c < k; ++c) {
            int p = c;
            for (int r = c + 1; r < k; ++r)
                if (std::fabs(M[size_t(r) * k + c]) > std::fabs(M[size_t(p) * k + c])) p = r;
            if (M[size_t(p) * k + c] == 0.0) return false;
            if (p != c) {
                for (int j = 0; j < k; ++j) std::swap(M[size_t(p) * k + j], M[size_t(c) * k + j]);
                std::swap(f[p], f[c]);
            }
            for (int r = c + 1; r < k; ++r) {
                double m = M[size_t(r) * k + c] / M[size_t(c) * k + c];
                if (m == 0.0) continue;
                for (int j = c; j < k; ++j) M[size_t(r) * k + j] -= m * M[size_t(c) * k + j];
                f[r] -= m * f[c];
            }
        }
        for (int r = k - 1; r >= 0; --r) {
            double s = f[r];
            for (int j = r + 1; j < k; ++j) s -= M[size_t(r) * k + j] * f[j];
            f[r] = s / M[size_t(r) * k + r];
        }
        double h = H[size_t(k) * k + (k - 1)];
        for (int i = 0; i < k; ++i) T[size_t(i) * k + (k - 1)] += (h * h) * f[i];
    }
    return hessenberg_eigvals(k, T, wr, wi);
}

std::vector<Root> order_roots(const std::vector<double>& wr, const std::vector<double>& wi,
                              double addroot_log10, double addroot_per)
{
    typedef std::complex<double> C;
    std::vector<C> all, rest;
    for (size_t i = 0; i < wr.size(); ++i) {
        all.push_back(C(wr[i], wi[i]));
        if (wi[i] >= 0.0) rest.push_back(C(wr[i], wi[i]));
    }
    std::vector<C> chosen;
    auto logdist = [](C a, C b) {
        double d = std::abs(a - b);
        return d == 0.0 ? -std::numeric_limits<double>::infinity() : std::log(d);
    };
    if (!rest.empty()) {
        size_t i0 = 0;
        for (size_t i = 1; i < rest.size(); ++i)
            if (std::abs(rest[i]) > std::abs(rest[i0])) i0 = i;
        chosen.push_back(rest[i0]);
        rest.erase(rest.begin() + long(i0));
    }
    while (!rest.empty()) {
        std::vector<C> pts;
        for (C c : chosen) {
            pts.push_back(c);
            if (c.imag() > 0.0) pts.push_back(std::conj(c));
        }
        double best = -std::numeric_limits<double>::infinity();
        size_t bi = 0;
        for (size_t i = 0; i < rest.size(); ++i) {
            double s = 0.0;
            for (C q : pts) s += logdist(rest[i], q);
            if (s > best) { best = s; bi = i; }
        }
        chosen.push_back(rest[bi]);
        rest.erase(rest.begin() + long(bi));
    }
    std::vector<C> extra;
    for (C z : chosen) {
        double lp = 0.0;
        for (C q : all) {
            if (q == z) continue;
            double d = std::abs(1.0 - z / q);
            lp += d == 0.0 ? -std::numeric_limits<double>::infinity() : std::log10(d);
        }
        if (lp > addroot_log10) {
            int nadd = int(std::ceil((lp - addroot_log10) / addroot_per));
            for (int c = 0; c < nadd; ++c) extra.push_back(z);
        }
    }
    std::vector<Root> out;
    for (C z : chosen) out.push_back(Root{z.real(), z.imag() > 0.0 ? z.imag() : 0.0});
    for (C z : extra) out.push_back(Root{z.real(), z.imag() > 0.0 ? z.imag() : 0.0});
    return out;
}

}  // namespace airg
