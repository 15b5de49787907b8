// C ABI of the AIRG library (declared in include/airg.h).  Every entry point
// converts internal errors into an airg_status and keeps the message for
// airg_last_error(); nothing aborts.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "dev_util.cuh"
#include "exact_dot_limits.h"
#include "handle.h"

struct airg_handle_s {
    std::unique_ptr<airg::Hierarchy> H;
    std::unique_ptr<airg::Hierarchy> HT;   // hierarchy of A^T (adjoint), built lazily
};

namespace {

thread_local std::string g_last_error;

template <class F>
airg_status guarded(F&& f)
{
    try {
        f();
        g_last_error.clear();
        return AIRG_OK;
    } catch (const airg::Error& e) {
        g_last_error = e.msg;
        return e.st;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return AIRG_ERR_OOM;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return AIRG_ERR_STATE;
    }
}

constexpr int TB = 256;

// Node spacing of the unit square's grid, nodes i * h for i = 0 .. nx - 1
// (the non-dimensionalisation of Sec. 3), used when the caller passes h = 0.
double default_spacing(long long nx) { return 1.0 / double(nx - 1); }

__global__ void k_adv_count(long long nx, long long ny, int sx, int sy, int* cnt, int* inflow_flag)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nx * ny) return;
    long long i = idx % nx, j = idx / nx;
    bool in = (sx > 0 && i == 0) || (sx < 0 && i == nx - 1) || (sy > 0 && j == 0) ||
              (sy < 0 && j == ny - 1);
    inflow_flag[idx] = in;
    cnt[idx] = in ? 1 : 1 + (sx != 0) + (sy != 0);
}

__global__ void k_adv_fill(long long nx, long long ny, int sx, int sy, double ax, double ay,
                           const int* rp32, const int* inflow_flag, const int* inflow_pos,
                           int64_t* rowptr, int32_t* col, double* val, int64_t* inflow)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long n = nx * ny;
    if (idx >= n) return;
    double d = __dadd_rn(ax, ay);
    int o = rp32[idx];
    rowptr[idx] = o;
    if (idx == n - 1) rowptr[n] = rp32[n];
    if (inflow_flag[idx]) {
        inflow[inflow_pos[idx]] = idx;
        col[o] = int32_t(idx);
        val[o] = d;
        return;
    }
    long long c[3];
    double v[3];
    int k = 0;
    c[k] = idx; v[k] = d; ++k;
    if (sx != 0) { c[k] = sx > 0 ? idx - 1 : idx + 1; v[k] = -ax; ++k; }
    if (sy != 0) { c[k] = sy > 0 ? idx - nx : idx + nx; v[k] = -ay; ++k; }
    for (int a = 1; a < k; ++a)   // ascending columns
        for (int b = a; b > 0 && c[b - 1] > c[b]; --b) {
            long long tc = c[b]; c[b] = c[b - 1]; c[b - 1] = tc;
            double tv = v[b]; v[b] = v[b - 1]; v[b - 1] = tv;
        }
    for (int a = 0; a < k; ++a) { col[o + a] = int32_t(c[a]); val[o + a] = v[a]; }
}

__global__ void k_rhs_source(long long n, double h, const double* s, double* b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = s ? __dmul_rn(h, s[i]) : 0.0;
}

__global__ void k_rhs_inflow(long long nin, double d, const int64_t* inflow, const double* g, double* b)
{
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nin) b[inflow[k]] = __dmul_rn(d, g[k]);
}

__global__ void k_grad_g(long long nin, double d, const int64_t* inflow, const double* lam, double* gg)
{
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nin) gg[k] = __dmul_rn(d, lam[inflow[k]]);
}

__global__ void k_zero_at(long long nin, const int64_t* idx, double* v)
{
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nin) v[idx[k]] = 0.0;
}

// 64-bit row pointers -> 32-bit; a value outside [0, nnz] becomes -1, which
// the validation rejects before any entry is read
__global__ void k_rp64_to_32(long long n, const int64_t* a, long long nnz, int* b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    const int64_t v = a[i];
    b[i] = (v < 0 || v > nnz) ? -1 : int(v);
}

int sgn(double x) { return x > 0.0 ? 1 : (x < 0.0 ? -1 : 0); }

void check_options(const airg_options& o)
{
    if (o.poly_order < 0 || o.poly_order > 30) airg::fail(AIRG_ERR_ARG, "poly_order must be in [0, 30]");
    if (o.coarse_poly_order < 1 || o.coarse_poly_order > 2000)
        airg::fail(AIRG_ERR_ARG, "coarse_poly_order must be in [1, 2000]");
    if (o.max_levels < 1 || o.max_levels > 64) airg::fail(AIRG_ERR_ARG, "max_levels must be in [1, 64]");
    if (o.gmres_restart < 1 || o.gmres_restart > 30) airg::fail(AIRG_ERR_ARG, "gmres_restart must be in [1, 30]");
    if (o.ddc_its < 0 || !(o.ddc_fraction >= 0.0 && o.ddc_fraction <= 1.0))
        airg::fail(AIRG_ERR_ARG, "bad DDC options");
    if (o.precision != AIRG_FP64 && o.precision != AIRG_MIXED_FP32 && o.precision != AIRG_MIXED_FP32_BF16R)
        airg::fail(AIRG_ERR_ARG, "bad precision");
    if (o.outer != AIRG_OUTER_FGMRES && o.outer != AIRG_OUTER_RICHARDSON) airg::fail(AIRG_ERR_ARG, "bad outer");
    if (o.smoother != AIRG_SMOOTH_POLYNOMIAL && o.smoother != AIRG_SMOOTH_ASSEMBLED)
        airg::fail(AIRG_ERR_ARG, "bad smoother");
    if (o.smooth_type != AIRG_SMOOTH_F && o.smooth_type != AIRG_SMOOTH_FC && o.smooth_type != AIRG_SMOOTH_FCF)
        airg::fail(AIRG_ERR_ARG, "bad smooth_type");
    if (o.inverse_type != AIRG_INVERSE_GMRES && o.inverse_type != AIRG_INVERSE_NEUMANN)
        airg::fail(AIRG_ERR_ARG, "bad inverse_type");
}

airg::DevCSR upload_csr(const airg_csr* A, cudaStream_t st)
{
    if (!A || !A->rowptr || (A->nnz && (!A->col || !A->val)))
        airg::fail(AIRG_ERR_ARG, "null CSR arrays");
    if (A->n_rows <= 0 || A->n_rows != A->n_cols) airg::fail(AIRG_ERR_ARG, "A must be square and non-empty");
    if (A->n_rows >= (1LL << 31) || A->nnz >= (1LL << 31) || A->nnz < 0)
        airg::fail(AIRG_ERR_ARG, "n and nnz must be below 2^31");
    airg::DevCSR D;
    D.alloc(int(A->n_rows), int(A->n_cols), int(A->nnz));
    long long n = A->n_rows;
    if (A->on_device) {
        k_rp64_to_32<<<airg::grid_for(n + 1, TB), TB, 0, st>>>(n, A->rowptr, A->nnz, D.rp.p);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(D.ci.p, A->col, A->nnz * sizeof(int), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(D.v.p, A->val, A->nnz * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
        std::vector<int> rp(n + 1);
        for (long long i = 0; i <= n; ++i) {
            if (A->rowptr[i] < 0 || A->rowptr[i] > A->nnz || (i && A->rowptr[i] < A->rowptr[i - 1]))
                airg::fail(AIRG_ERR_ARG, "row pointers not monotone within [0, nnz]");
            rp[i] = int(A->rowptr[i]);
        }
        CK(cudaMemcpyAsync(D.rp.p, rp.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(D.ci.p, A->col, A->nnz * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(D.v.p, A->val, A->nnz * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
    airg::validate_csr(D, true, st);
    return D;
}

const airg::Hierarchy* level_owner(const airg_handle* h)
{
    if (!h || !h->H) airg::fail(AIRG_ERR_STATE, "null handle");
    return h->H.get();
}

}  // namespace

namespace airg {
// lets entry points outside this file report through airg_last_error()
void set_last_error(const char* msg) { g_last_error = msg; }
// validated device copy of a caller's CSR (multi.cu)
DevCSR upload_csr_checked(const airg_csr* A, cudaStream_t st) { return upload_csr(A, st); }
void check_options_checked(const airg_options& o) { check_options(o); }
}  // namespace airg

extern "C" {

airg_status airg_options_default(airg_options* o)
{
    if (!o) { g_last_error = "null options"; return AIRG_ERR_ARG; }
    std::memset(o, 0, sizeof *o);
    o->strong_threshold = 0.99;
    o->ddc_fraction = 0.01;
    o->ddc_its = 2;
    o->poly_order = 6;
    o->coarse_poly_order = 100;
    o->trunc_rtol = 0.1;
    o->trunc_start_level = 0;
    o->max_levels = 64;
    o->coarse_min_rows = 1;
    o->a_drop = 1e-6;
    o->a_lump = 1;
    o->r_drop = 2e-2;   // not in the paper: chosen on measured solve time (1024^2 and 4096^2)
    o->seed = 2508175ULL;
    o->breakdown_tol = 1e-8;
    o->exact_tol = 1e-12;
    o->addroot_log10 = 4.0;
    o->addroot_per = 14.0;
    o->precision = AIRG_FP64;
    o->gmres_restart = 30;
    o->outer = AIRG_OUTER_FGMRES;
    o->smoother = AIRG_SMOOTH_POLYNOMIAL;
    o->smooth_type = AIRG_SMOOTH_F;
    o->inverse_type = AIRG_INVERSE_GMRES;
    return AIRG_OK;
}

airg_status airg_problem_advection2d(int64_t nx, int64_t ny, double vx, double vy, double h,
                                     int64_t* rowptr, int32_t* col, double* val, int64_t* inflow,
                                     int64_t* nnz_out, int64_t* n_inflow_out, void* stream)
{
    return guarded([&] {
        if (nx < 2 || ny < 2 || nx * ny >= (1LL << 31) / 3 || !rowptr || !col || !val || !inflow ||
            !nnz_out || !n_inflow_out || !(h >= 0.0) || !std::isfinite(h) || !std::isfinite(vx) ||
            !std::isfinite(vy))
            airg::fail(AIRG_ERR_ARG, "bad advection2d arguments");
        if (h == 0.0) h = default_spacing(nx);
        cudaStream_t st = (cudaStream_t)stream;
        long long n = nx * ny;
        airg::DBuf<int> cnt(n + 1), flag(n + 1);
        int sx = sgn(vx), sy = sgn(vy);
        k_adv_count<<<airg::grid_for(n, TB), TB, 0, st>>>(nx, ny, sx, sy, cnt.p, flag.p);
        CK_LAUNCH();
        airg::DBuf<int> fpos(n + 1);
        CK(cudaMemcpyAsync(fpos.p, flag.p, n * sizeof(int), cudaMemcpyDeviceToDevice, st));
        int nin = airg::exclusive_scan(fpos.p, fpos.p, int(n), st);
        int nnz = airg::exclusive_scan(cnt.p, cnt.p, int(n), st);
        k_adv_fill<<<airg::grid_for(n, TB), TB, 0, st>>>(nx, ny, sx, sy, std::fabs(vx), std::fabs(vy),
                                                         cnt.p, flag.p, fpos.p, rowptr, col, val, inflow);
        CK_LAUNCH();
        CK(cudaStreamSynchronize(st));
        *nnz_out = nnz;
        *n_inflow_out = nin;
        (void)h;
    });
}

airg_status airg_assemble_rhs_advection2d(int64_t nx, int64_t ny, double vx, double vy, double h,
                                          int nrhs, const int64_t* inflow, int64_t n_inflow,
                                          const double* g, const double* s, double* b, void* stream)
{
    return guarded([&] {
        if (nx < 2 || ny < 2 || nrhs < 1 || !inflow || !g || !b || n_inflow < 0 || !(h >= 0.0) ||
            !std::isfinite(h))
            airg::fail(AIRG_ERR_ARG, "bad rhs arguments");
        if (h == 0.0) h = default_spacing(nx);
        cudaStream_t st = (cudaStream_t)stream;
        long long n = nx * ny;
        double d = std::fabs(vx) + std::fabs(vy);
        for (int q = 0; q < nrhs; ++q) {
            k_rhs_source<<<airg::grid_for(n, TB), TB, 0, st>>>(n, h, s ? s + size_t(q) * n : nullptr,
                                                               b + size_t(q) * n);
            if (n_inflow)
                k_rhs_inflow<<<airg::grid_for(n_inflow, TB), TB, 0, st>>>(n_inflow, d, inflow,
                                                                          g + size_t(q) * n_inflow,
                                                                          b + size_t(q) * n);
            CK_LAUNCH();
        }
        CK(cudaStreamSynchronize(st));
    });
}

airg_status airg_rhs_adjoint_advection2d(int64_t nx, int64_t ny, double vx, double vy, double h,
                                         int nrhs, const int64_t* inflow, int64_t n_inflow,
                                         const double* lambda, double* grad_g, double* grad_s,
                                         void* stream)
{
    return guarded([&] {
        if (nx < 2 || ny < 2 || nrhs < 1 || !inflow || !lambda || !grad_g || n_inflow < 0 || !(h >= 0.0) ||
            !std::isfinite(h))
            airg::fail(AIRG_ERR_ARG, "bad rhs-adjoint arguments");
        if (h == 0.0) h = default_spacing(nx);
        cudaStream_t st = (cudaStream_t)stream;
        long long n = nx * ny;
        double d = std::fabs(vx) + std::fabs(vy);
        for (int q = 0; q < nrhs; ++q) {
            const double* lam = lambda + size_t(q) * n;
            if (n_inflow)
                k_grad_g<<<airg::grid_for(n_inflow, TB), TB, 0, st>>>(n_inflow, d, inflow, lam,
                                                                      grad_g + size_t(q) * n_inflow);
            if (grad_s) {
                double* gs = grad_s + size_t(q) * n;
                k_rhs_source<<<airg::grid_for(n, TB), TB, 0, st>>>(n, h, lam, gs);
                if (n_inflow) k_zero_at<<<airg::grid_for(n_inflow, TB), TB, 0, st>>>(n_inflow, inflow, gs);
            }
            CK_LAUNCH();
        }
        CK(cudaStreamSynchronize(st));
    });
}

airg_status airg_setup(const airg_csr* A, const airg_options* opt, void* stream, airg_handle** out)
{
    return guarded([&] {
        if (!out) airg::fail(AIRG_ERR_ARG, "null output handle");
        *out = nullptr;
        airg_options o;
        if (opt) o = *opt;
        else airg_options_default(&o);
        check_options(o);
        cudaStream_t st = (cudaStream_t)stream;
        airg::DevCSR D = upload_csr(A, st);
        auto h = new airg_handle_s();
        try {
            h->H = airg::build_hierarchy(std::move(D), o, st);
        } catch (...) {
            delete h;
            throw;
        }
        *out = h;
    });
}

airg_status airg_solve(airg_handle* h, int nrhs, const double* b, double* x, int on_device,
                       double rtol, double atol, int maxit, airg_solve_info* info, void* stream)
{
    return guarded([&] {
        if (!h || !h->H || !h->H->solve) airg::fail(AIRG_ERR_STATE, "handle not set up");
        if (nrhs < 1 || !b || !x || maxit < 0 || !(rtol >= 0.0) || !(atol >= 0.0))
            airg::fail(AIRG_ERR_ARG, "bad solve arguments");
        airg::solve_system(*h->H, nrhs, b, x, on_device != 0, rtol, atol, maxit, info,
                           (cudaStream_t)stream);
    });
}

airg_status airg_solve_adjoint(airg_handle* h, int nrhs, const double* rhs, double* lambda,
                               int on_device, double rtol, double atol, int maxit,
                               airg_solve_info* info, void* stream)
{
    return guarded([&] {
        if (!h || !h->H) airg::fail(AIRG_ERR_STATE, "handle not set up");
        if (nrhs < 1 || !rhs || !lambda) airg::fail(AIRG_ERR_ARG, "bad adjoint arguments");
        cudaStream_t st = (cudaStream_t)stream;
        if (!h->HT) {
            const airg::DevCSR& A0 = h->H->levels.empty() ? h->H->coarse.A : h->H->levels[0]->A;
            airg::DevCSR T;
            airg::csr_transpose(A0, T, st);
            h->HT = airg::build_hierarchy(std::move(T), h->H->opt, st);
        }
        airg::solve_system(*h->HT, nrhs, rhs, lambda, on_device != 0, rtol, atol, maxit, info, st);
    });
}

airg_status airg_setup_info(const airg_handle* h, airg_hierarchy_info* info)
{
    return guarded([&] {
        if (!h || !h->H || !info) airg::fail(AIRG_ERR_ARG, "null handle or info");
        airg::fill_setup_info(*h->H, info);
    });
}

airg_status airg_export_matrix(const airg_handle* h, int level, int what, int64_t* n_rows,
                               int64_t* n_cols, int64_t* nnz, int64_t* rowptr, int32_t* col,
                               double* val)
{
    return guarded([&] {
        const airg::Hierarchy* H = level_owner(h);
        int L = int(H->levels.size());
        if (level < 0 || level > L || !n_rows || !n_cols || !nnz) airg::fail(AIRG_ERR_ARG, "bad level");
        const airg::DevCSR* M = nullptr;
        if (level == L) {
            if (what != 0) airg::fail(AIRG_ERR_ARG, "the coarsest level only has its operator");
            M = &H->coarse.A;
        } else {
            const airg::SetupLevel& lv = *H->levels[level];
            switch (what) {
                case 0: M = &lv.A; break;
                case 1: M = &lv.A_ff; break;
                case 2: M = &lv.A_fc; break;
                case 3: M = &lv.Z; break;
                case 4:
                    if (!lv.Ainv.n_rows && lv.n_f) airg::fail(AIRG_ERR_ARG, "the approximate inverse is kept only with the assembled smoother");
                    M = &lv.Ainv;
                    break;
                case 5:
                    if (H->opt.smooth_type == AIRG_SMOOTH_F) airg::fail(AIRG_ERR_ARG, "A_cc is kept only with C-point smoothing");
                    M = &lv.A_cc;
                    break;
                case 6:
                    if (!lv.Ainv_cc.n_rows && lv.n_c) airg::fail(AIRG_ERR_ARG, "Ahat_cc^-1 is kept only with assembled C-point smoothing");
                    M = &lv.Ainv_cc;
                    break;
                default: airg::fail(AIRG_ERR_ARG, "bad matrix id");
            }
        }
        *n_rows = M->n_rows;
        *n_cols = M->n_cols;
        *nnz = M->nnz;
        if (!rowptr) return;
        std::vector<int> rp(size_t(M->n_rows) + 1);
        airg::d2h(rp.data(), M->rp.p, rp.size(), 0);
        for (size_t i = 0; i < rp.size(); ++i) rowptr[i] = rp[i];
        if (col) airg::d2h(col, M->ci.p, size_t(M->nnz), 0);
        if (val) airg::d2h(val, M->v.p, size_t(M->nnz), 0);
    });
}

airg_status airg_export_vector(const airg_handle* h, int level, int what, int64_t* count, void* out)
{
    return guarded([&] {
        const airg::Hierarchy* H = level_owner(h);
        int L = int(H->levels.size());
        if (level < 0 || level > L || !count) airg::fail(AIRG_ERR_ARG, "bad level");
        if (what == 3) {
            const auto& r = H->coarse.roots;
            *count = int64_t(r.size()) * 2;
            if (out) {
                double* o = (double*)out;
                for (size_t i = 0; i < r.size(); ++i) { o[2 * i] = r[i].re; o[2 * i + 1] = r[i].im; }
            }
            return;
        }
        if (level == L) airg::fail(AIRG_ERR_ARG, "the coarsest level has no CF data");
        const airg::SetupLevel& lv = *H->levels[level];
        switch (what) {
            case 0:
                *count = lv.n;
                if (out) airg::d2h((int8_t*)out, lv.is_f.p, size_t(lv.n), 0);
                break;
            case 1:
                *count = lv.n_f;
                if (out) airg::d2h((int32_t*)out, lv.W.p, size_t(lv.n_f), 0);
                break;
            case 2:
                *count = int64_t(lv.alpha.size());
                if (out) std::memcpy(out, lv.alpha.data(), lv.alpha.size() * sizeof(double));
                break;
            case 4: {
                std::vector<double> s;
                s.push_back(lv.pmisr_rounds);
                for (int c : lv.ddc_converted) s.push_back(c);
                s.push_back(lv.trunc_rel);
                s.push_back(lv.alpha_k);
                *count = int64_t(s.size());
                if (out) std::memcpy(out, s.data(), s.size() * sizeof(double));
                break;
            }
            case 5:
                if (H->opt.smooth_type == AIRG_SMOOTH_F) airg::fail(AIRG_ERR_ARG, "no C-point smoother");
                *count = int64_t(lv.alpha_c.size());
                if (out) std::memcpy(out, lv.alpha_c.data(), lv.alpha_c.size() * sizeof(double));
                break;
            default: airg::fail(AIRG_ERR_ARG, "bad vector id");
        }
    });
}

airg_status airg_profile(airg_handle* h, int enable)
{
    return guarded([&] {
        if (!h || !h->H || !h->H->solve) airg::fail(AIRG_ERR_STATE, "handle not set up");
        airg::set_profiling(*h->H, enable != 0);
    });
}

airg_status airg_profile_group(airg_handle* h, int kind, int level)
{
    return guarded([&] {
        if (!h || !h->H || !h->H->solve) airg::fail(AIRG_ERR_STATE, "handle not set up");
        if (kind < 0 || kind > 6 || level < 0 || level > 64) airg::fail(AIRG_ERR_ARG, "bad kernel kind or level");
        airg::set_profiling(*h->H, true, kind, level);
    });
}

airg_status airg_profile_read(const airg_handle* h, int kind, double* ms, int64_t* launches,
                              int64_t* bytes)
{
    return guarded([&] {
        if (!h || !h->H || !h->H->solve || !ms || !launches || !bytes)
            airg::fail(AIRG_ERR_ARG, "bad profile arguments");
        long long l = 0, b = 0;
        if (!airg::read_profile(*h->H, kind, -1, ms, &l, &b, nullptr)) airg::fail(AIRG_ERR_ARG, "bad kernel kind");
        *launches = l;
        *bytes = b;
    });
}

airg_status airg_profile_read_level(const airg_handle* h, int kind, int level, double* ms, int64_t* launches,
                                    int64_t* bytes, int64_t* flops)
{
    return guarded([&] {
        if (!h || !h->H || !h->H->solve || !ms || !launches || !bytes || !flops)
            airg::fail(AIRG_ERR_ARG, "bad profile arguments");
        long long l = 0, b = 0, f = 0;
        if (!airg::read_profile(*h->H, kind, level, ms, &l, &b, &f))
            airg::fail(AIRG_ERR_ARG, "bad kernel kind or level");
        *launches = l;
        *bytes = b;
        *flops = f;
    });
}

airg_status airg_operator_layout_info(const airg_handle* h, int level, int op, airg_operator_layout* out)
{
    return guarded([&] {
        if (!h || !h->H || !out) airg::fail(AIRG_ERR_ARG, "null handle or out");
        if (!airg::operator_layout(*h->H, level, op, out))
            airg::fail(AIRG_ERR_ARG, "no operator slot for this level and op");
    });
}

airg_status airg_check_wait_timeout(int64_t spin_limit, void* stream)
{
    bool gave_up = false;
    airg_status st = guarded([&] {
        if (spin_limit < 1) airg::fail(AIRG_ERR_ARG, "spin_limit must be positive");
        gave_up = airg::barrier_timeout_check(spin_limit, (cudaStream_t)stream);
        if (!gave_up) airg::fail(AIRG_ERR_STATE, "the bounded wait did not report its timeout");
    });
    if (st == AIRG_OK && gave_up) {
        g_last_error = "bounded device wait gave up after spin_limit polls (as intended)";
        return AIRG_ERR_TIMEOUT;
    }
    return st;
}

void airg_free(airg_handle* h) { delete h; }

const char* airg_last_error(void) { return g_last_error.c_str(); }

airg_status airg_dot_exact(int64_t n, const double* x, const double* y, double* out, void* stream)
{
    return guarded([&] {
        if (n < 0 || !out || (n && (!x || !y))) airg::fail(AIRG_ERR_ARG, "bad dot arguments");
        if (n > airg::XD_MAX_N) airg::fail(AIRG_ERR_ARG, "airg_dot_exact: n exceeds 2^31 - 1 (accumulator limit)");
        cudaStream_t st = (cudaStream_t)stream;
        airg::DBuf<double> r(1);
        airg::dot_exact_device(n, x, y, r.p, nullptr, st);
        airg::d2h(out, r.p, 1, st);
    });
}

airg_status airg_rng_uniform(uint64_t seed, int64_t level, int64_t purpose, int64_t n, double* out,
                             void* stream)
{
    return guarded([&] {
        if (n < 0 || (n && !out)) airg::fail(AIRG_ERR_ARG, "bad rng arguments");
        airg::rng_uniform_device(seed, level, purpose, n, out, (cudaStream_t)stream);
    });
}

airg_status airg_host_gmres_coeffs(int k, const double* H, double beta, double* alpha)
{
    return guarded([&] {
        if (k < 1 || !H || !alpha) airg::fail(AIRG_ERR_ARG, "bad coefficient arguments");
        std::vector<double> Hv(H, H + size_t(k + 1) * k);
        std::vector<double> y = airg::givens_lsq(Hv, k, beta);
        std::vector<double> a = airg::power_coefficients(Hv, k, beta, y);
        std::copy(a.begin(), a.end(), alpha);
    });
}

airg_status airg_host_eigvals(int n, const double* H, double* wr, double* wi)
{
    return guarded([&] {
        if (n < 1 || !H || !wr || !wi) airg::fail(AIRG_ERR_ARG, "bad eigenvalue arguments");
        std::vector<double> Hv(H, H + size_t(n) * n), r, i;
        if (!airg::hessenberg_eigvals(n, Hv, r, i)) airg::fail(AIRG_ERR_BREAKDOWN, "QR iteration did not converge");
        std::copy(r.begin(), r.end(), wr);
        std::copy(i.begin(), i.end(), wi);
    });
}

}  // extern "C"
