// The AIRG hierarchy object behind airg_handle: setup products in each
// level's own numbering (kept for export and checking) and the solve-phase
// operators in the nested F/C layout (see solve.cu).
#pragma once

#include <cmath>
#include <memory>
#include <vector>

#include "dev_util.cuh"
#include "hostmath.h"

namespace airg {

// Setup products of one non-coarsest level, in the level's numbering.
struct SetupLevel {
    int n = 0, n_f = 0, n_c = 0;
    DevCSR A;                 // level operator A_l
    DBuf<int8_t> strong;      // per stored entry of A_l
    DBuf<int8_t> is_f;        // per row: 1 = F point
    DBuf<int> f_index, c_index;   // F-/C-local index of each row, -1 otherwise
    DBuf<int> f_ids, c_ids;       // row of each F / C point
    DevCSR A_ff, A_fc, Z;     // blocks of Eq. 3; Z = -A_cf Ahat_ff^-1 after drop
    DevCSR M;                 // rows of A P at the F points = A_fc + A_ff W
    DevCSR Ainv;              // fixed-sparsity Ahat_ff^-1 (Eq. 8), kept for the assembled smoother
    // C-point smoothing only: A_cc, the C rows [A_cf A_cc] and the F rows
    // [A_ff A_fc] of A_l with the level's own column numbering, and the
    // GMRES polynomial of A_cc
    DevCSR A_cc, Crows, Frows;
    DevCSR Ainv_cc;           // fixed-sparsity Ahat_cc^-1 (assembled C-point smoother)
    std::vector<double> alpha_c;
    int alpha_c_k = 0;
    DBuf<int> W;              // one-point prolongator: C-local index or -1
    std::vector<double> alpha;    // p+1 smoother coefficients (zero-padded)
    int alpha_k = 0;              // Krylov dimension reached (p+1 unless breakdown)
    int pmisr_rounds = 0;
    std::vector<int> ddc_converted;
    double trunc_rel = NAN;
};

struct CoarseLevel {
    DevCSR A;
    std::vector<Root> roots;
    int k = 0;
    double trunc_rel = NAN;
    bool truncated = false;
};

struct SolveData;   // solve.cu

struct Hierarchy {
    airg_options opt{};
    std::vector<std::unique_ptr<SetupLevel>> levels;
    CoarseLevel coarse;
    double setup_ms = 0.0;
    double phase_ms[AIRG_SETUP_PHASES] = {};   // setup breakdown (AIRG_PHASE_*)
    long long exact_dots = 0;                  // correctly rounded dots of the setup
    std::unique_ptr<SolveData> solve;
    Hierarchy();
    ~Hierarchy();
};

// setup.cu
std::unique_ptr<Hierarchy> build_hierarchy(DevCSR&& A0, const airg_options& opt,
                                           cudaStream_t st);
void dot_exact_device(long long n, const double* x, const double* y, double* out,
                      double* out_sqrt, cudaStream_t st);
void rng_uniform_device(uint64_t seed, long long level, long long purpose, long long n,
                        double* out, cudaStream_t st);
void csr_transpose(const DevCSR& A, DevCSR& T, cudaStream_t st);
void validate_csr(const DevCSR& A, bool square, cudaStream_t st);

// solve.cu
void build_solve_data(Hierarchy& H, cudaStream_t st);
void solve_system(Hierarchy& H, int nrhs, const double* b, double* x, bool on_device,
                  double rtol, double atol, int maxit, airg_solve_info* info, cudaStream_t st);
void fill_setup_info(const Hierarchy& H, airg_hierarchy_info* info);
// layout and tuned row-kernel variant of one solve-phase operator
// (AIRG_OPERATOR_*); false for an op or level that names no operator slot
bool operator_layout(const Hierarchy& H, int level, int op, airg_operator_layout* out);
// on: time the solve kernels; kind >= 0 restricts the timing to the
// launches of that kind on `level` (consecutive V-cycle launches of the
// group share one event pair)
void set_profiling(Hierarchy& H, bool on, int kind = -1, int level = -1);
bool barrier_timeout_check(long long limit, cudaStream_t st);
bool read_profile(const Hierarchy& H, int kind, int level, double* ms, long long* launches, long long* bytes,
                  long long* flops);

}  // namespace airg
