// Small dense FP64 computations of the AIRG setup that run on the host:
// the GMRES least-squares problem and power-basis coefficients (Eq. 7), and
// the harmonic Ritz roots of the coarse-grid Newton polynomial (Sec. 2.3).
#pragma once

#include <complex>
#include <vector>

namespace airg {

// H is (k+1) x k row-major (column j holds the Arnoldi coefficients of step j).
// Returns y = argmin || beta e1 - H y || by Givens rotations.
std::vector<double> givens_lsq(const std::vector<double>& H, int k, double beta);

// || beta e1 - H y || at the least-squares minimiser (same rotations).
double givens_residual(const std::vector<double>& H, int k, double beta);

// Coefficients alpha_0..alpha_{k-1} of the polynomial with
// sum_j y_j v_j = (sum_t alpha_t A^t) b, from the Arnoldi recurrence
// c_1 = 1/beta, c_{j+1}(z) = (z c_j(z) - sum_{i<=j} h_ij c_i(z)) / h_{j+1,j}.
std::vector<double> power_coefficients(const std::vector<double>& H, int k, double beta,
                                       const std::vector<double>& y);

// Eigenvalues of a real upper Hessenberg matrix (row-major n x n) by the
// Francis double-shift QR iteration.  Returns false if it fails to converge.
bool hessenberg_eigvals(int n, std::vector<double> H, std::vector<double>& wr,
                        std::vector<double>& wi);

// Harmonic Ritz values from an Arnoldi Hessenberg ((k+1) x k row-major):
// eig(H_k + h_{k+1,k}^2 H_k^{-T} e_k e_k^T), or eig(H_k) after a breakdown.
bool harmonic_ritz(const std::vector<double>& H, int k, bool broke, std::vector<double>& wr,
                   std::vector<double>& wi);

struct Root {
    double re, im;   // im > 0: the conjugate pair re +- i im; im == 0: real root
};

// Leja ordering of the roots (conjugates adjacent, represented once) followed
// by the extra copies of roots whose product of other factors exceeds
// 10^addroot_log10 (ceil((log10 pof - addroot_log10) / addroot_per) copies).
std::vector<Root> order_roots(const std::vector<double>& wr, const std::vector<double>& wi,
                              double addroot_log10, double addroot_per);

}  // namespace airg
