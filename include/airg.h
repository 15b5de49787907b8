/*
 * airg.h -- C ABI of the GB300 (sm_103a) AIRG solver.
 *
 * AIRG is the reduction multigrid of Dargaville, Smedley-Stevenson, Smith &
 * Pain, "Solving advection equations with reduction multigrids on GPUs"
 * (arXiv 2508.17517): approximate ideal restriction built from GMRES
 * polynomials (Sec. 2.2, Eq. 7-8), one-point prolongation and up F-point
 * smoothing only (Sec. 2, Eq. 6), a PMISR DDC coarse/fine splitting
 * (Sec. 2.1), a high-order GMRES polynomial in Newton form as the coarse-grid
 * solver (Sec. 2.3) on a hierarchy truncated automatically by that
 * polynomial's quality (Sec. 2.4).  Setup and solve run on the GPU; the
 * outer iteration is flexible GMRES in FP64.
 *
 * Conventions (every entry point):
 *  - Return an airg_status; never abort, never trap on the device.  The text
 *    of the last error on the calling thread is airg_last_error().
 *  - "device" pointers are CUDA global-memory addresses on the current
 *    device; "host" pointers are ordinary CPU memory.  Each pointer argument
 *    says which it takes.  Pointers are borrowed for the duration of the call
 *    only, unless stated otherwise.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    stream-ordered on it and return after the work they launched has
 *    finished, unless stated otherwise.
 *  - Index types: row pointers int64, column indices int32; n < 2^31 and
 *    nnz < 2^31 (AIRG_ERR_ARG otherwise).  Columns strictly ascending per row.
 */
#ifndef AIRG_H
#define AIRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AIRG_OK = 0,
    AIRG_ERR_ARG = 1,            /* invalid argument or malformed matrix        */
    AIRG_ERR_CUDA = 2,           /* a CUDA runtime call failed                  */
    AIRG_ERR_OOM = 3,            /* device or host allocation failed            */
    AIRG_ERR_BREAKDOWN = 4,      /* zero diagonal / singular polynomial step    */
    AIRG_ERR_NOT_CONVERGED = 5,  /* maxit reached; x and info are still valid   */
    AIRG_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up          */
    AIRG_ERR_STATE = 7           /* handle not in a state that allows the call  */
} airg_status;

/* Precision of the V-cycle: FP64; FP32 (vectors, operators, polynomials);
 * FP32 with the restrictor values Z (R = [Z I], Eq. 4) stored in bfloat16.
 * The outer iteration, its orthogonalisation and residuals stay FP64. */
enum { AIRG_FP64 = 0, AIRG_MIXED_FP32 = 1, AIRG_MIXED_FP32_BF16R = 2 };
/* Outer iteration around the V-cycle: flexible GMRES (default), or the
 * preconditioned Richardson iteration x <- x + M^-1 (b - A x) of Sec. 3. */
enum { AIRG_OUTER_FGMRES = 0, AIRG_OUTER_RICHARDSON = 1 };
/* F-point smoother: the matrix-free GMRES polynomial q(A_ff) by Horner
 * (Eq. 6-7), or the assembled fixed-sparsity approximation of Eq. 8 applied
 * as one SpMV (the alternative timed in Sec. 2.2; stores one more matrix per
 * level). */
enum { AIRG_SMOOTH_POLYNOMIAL = 0, AIRG_SMOOTH_ASSEMBLED = 1 };
/* Which points are smoothed on the way up (Sec. 2; the options listed in
 * Sec. 3.3.2): F points only (the paper's default, Eq. 6); F then C points;
 * F, C, then F again.  A C-point smooth applies a GMRES polynomial of A_cc
 * of the same degree, matrix-free, to r_c - A_cf e_f - A_cc e_c, where r_c
 * is the level's C residual before restriction; it keeps A_cf and A_cc on
 * every level.  With AIRG_SMOOTH_ASSEMBLED the C-point smooth applies the
 * fixed-sparsity Ahat_cc^-1 of Eq. 8 instead (one more matrix per level).
 * Every solve entry point (one or many right-hand sides, batches of grids,
 * adjoint) supports all three. */
enum { AIRG_SMOOTH_F = 0, AIRG_SMOOTH_FC = 1, AIRG_SMOOTH_FCF = 2 };
/* Block approximate inverse behind the smoother and the restrictor: the
 * GMRES polynomial of Eq. 7 (AIRG), or the Neumann polynomial of nAIR
 * (Sec. 3.3.1), read as q(A) = w sum_{k<=p} (I - w A)^k with w = 1 / max_i
 * |a_ii|: the Jacobi-scaled Neumann series whenever the block's diagonal is
 * constant.  The coarse-grid polynomial is the GMRES one in both. */
enum { AIRG_INVERSE_GMRES = 0, AIRG_INVERSE_NEUMANN = 1 };

/* Compressed sparse row matrix (n_rows x n_cols).  Caller-owned, read-only. */
typedef struct {
    int64_t n_rows, n_cols, nnz;
    const int64_t* rowptr;   /* n_rows + 1 entries                          */
    const int32_t* col;      /* nnz entries, ascending within each row      */
    const double* val;       /* nnz entries                                 */
    int on_device;           /* 1: the three arrays are device pointers     */
} airg_csr;

/* Solver options.  airg_options_default() fills the values of the command
 * line in Sec. 3 of the paper (strong threshold 0.99, DDC fraction 0.01 with
 * 2 passes, smoother polynomial order 6, coarse polynomial order 100,
 * truncation tolerance 0.1, A drop 1e-6 with lumping). */
typedef struct {
    double strong_threshold;   /* PMISR strength threshold                   */
    double ddc_fraction;       /* share of F points converted per DDC pass    */
    int ddc_its;               /* DDC passes                                  */
    int poly_order;            /* smoother GMRES polynomial degree p          */
    int coarse_poly_order;     /* Arnoldi steps m_c of the coarse polynomial  */
    double trunc_rtol;         /* truncation tolerance alpha_trunc; <=0: off  */
    int trunc_start_level;     /* first level tested for truncation           */
    int max_levels;            /* hard cap on levels (coarsest included)      */
    int coarse_min_rows;       /* a level this small is the coarsest          */
    double a_drop;             /* relative drop tolerance on A_coarse         */
    int a_lump;                /* 1: add dropped A_coarse entries to diagonal */
    double r_drop;             /* relative drop tolerance on R                */
    uint64_t seed;             /* seed of all random streams of the setup     */
    double breakdown_tol;      /* Arnoldi rank threshold on h_{j+1,j}         */
    double exact_tol;          /* Arnoldi stops once the GMRES residual of its
                                  least-squares problem is <= exact_tol*||b||
                                  (the polynomial already inverts exactly)   */
    double addroot_log10;      /* extra-root threshold on log10(pof)          */
    double addroot_per;        /* decades of pof per extra root               */
    int precision;             /* AIRG_FP64, AIRG_MIXED_FP32, _BF16R           */
    int gmres_restart;         /* outer FGMRES restart length                 */
    int outer;                 /* AIRG_OUTER_FGMRES or AIRG_OUTER_RICHARDSON  */
    int smoother;              /* AIRG_SMOOTH_POLYNOMIAL or _ASSEMBLED        */
    int smooth_type;           /* AIRG_SMOOTH_F, _FC or _FCF                  */
    int inverse_type;          /* AIRG_INVERSE_GMRES or AIRG_INVERSE_NEUMANN  */
} airg_options;

typedef struct airg_handle_s airg_handle;
typedef struct airg_batch_s airg_batch;

typedef struct {
    int iterations;            /* outer FGMRES iterations (= V-cycles)        */
    double rel_residual;       /* true ||b - A x||_2 / ||b||_2 at exit        */
    int converged;             /* 1 if rel_residual test met                  */
    double solve_ms;           /* wall time of the call                       */
    int64_t kernel_launches;   /* CUDA kernels this call launched             */
} airg_solve_info;

/* Phases of airg_setup timed in airg_hierarchy_info.setup_phase_ms (the
 * setup breakdown of Sec. 3.1), summed over levels: the truncation test
 * (coarse polynomial and its residual on levels that were not truncated,
 * Sec. 2.4); CF splitting (strength, PMISR, DDC, Sec. 2.1); extraction of
 * the blocks of Eq. 3; the smoother's GMRES polynomial coefficients
 * (Arnoldi, Eq. 7); the fixed-sparsity inverse (Eq. 8); the restrictor
 * Z = -A_cf Ahat^-1 and its drop; the one-point prolongator and the P/R
 * assembly; the RAP sparse products; the drop and lumping of A_coarse; the
 * coarse-grid Newton polynomial (Sec. 2.3); the solve layout (SELL
 * conversion, row-kernel tuning and buffers). */
enum {
    AIRG_PHASE_TRUNCATION = 0, AIRG_PHASE_CF_SPLIT = 1, AIRG_PHASE_EXTRACT = 2,
    AIRG_PHASE_SMOOTHER_POLY = 3, AIRG_PHASE_FIXED_SPARSITY = 4, AIRG_PHASE_RESTRICTOR = 5,
    AIRG_PHASE_PROLONGATOR = 6, AIRG_PHASE_RAP = 7, AIRG_PHASE_DROP_LUMP = 8,
    AIRG_PHASE_COARSE_POLY = 9, AIRG_PHASE_SOLVE_LAYOUT = 10, AIRG_SETUP_PHASES = 11
};

typedef struct {
    int levels;                /* number of levels, coarsest included         */
    int truncated;             /* 1 if the hierarchy was truncated (Sec. 2.4) */
    int coarse_roots;          /* Newton roots of the coarse solver           */
    int coarse_krylov;         /* Arnoldi steps taken for those roots         */
    double cycle_complexity;   /* V-cycle flops / top SpMV flops (Sec. 3)     */
    double storage_complexity; /* solve-time nnz / nnz(A_top) (Sec. 3)        */
    double setup_ms;           /* wall time of airg_setup                     */
    int64_t n[64];             /* unknowns per level                          */
    int64_t n_f[64];           /* F points per level (0 on the coarsest)      */
    int64_t nnz_a[64];         /* nnz of the level operator A_l               */
    int64_t bytes_per_vcycle;  /* algorithmic bytes of one V-cycle            */
    double setup_phase_ms[16]; /* wall time of each AIRG_PHASE_* (stream
                                  synchronised at every phase boundary)      */
    int64_t exact_dots;        /* correctly rounded dot products the setup ran */
} airg_hierarchy_info;

/* Fills `opt` with the defaults above.  AIRG_ERR_ARG if opt is NULL. */
airg_status airg_options_default(airg_options* opt);

/*
 * Upwind finite-difference operator of v.grad(u) = s on an nx-by-ny node grid
 * with spacing h (Eq. 1-2, Sec. 3).  Nodes (i, j) have index i + nx*j.  Each
 * equation is multiplied by h (the non-dimensionalisation of Sec. 3):
 * interior rows d*u_ij - |vx| u_(upwind x) - |vy| u_(upwind y) = h s_ij with
 * d = |vx| + |vy|; inflow nodes (v.n < 0) keep their unknowns with the row
 * d*u = d*g (boundary DOFs not eliminated).  Zero velocity components store
 * no entry.  h = 0 selects the spacing of the unit square's node grid,
 * 1 / (nx - 1), here and in the two right-hand-side calls below.  All
 * pointers are DEVICE pointers, caller-allocated:
 *   rowptr: n+1, col: 3n, val: 3n, inflow: nx+ny (sorted node indices).
 * *nnz_out and *n_inflow_out (HOST pointers) receive the counts.
 * AIRG_ERR_ARG unless nx, ny >= 2, 3 nx ny < 2^31, h >= 0 finite and vx, vy
 * finite (a smaller system can be passed to airg_setup as a CSR matrix
 * directly).
 */
airg_status airg_problem_advection2d(int64_t nx, int64_t ny, double vx, double vy, double h,
                                     int64_t* rowptr, int32_t* col, double* val,
                                     int64_t* inflow, int64_t* nnz_out,
                                     int64_t* n_inflow_out, void* stream);

/*
 * Right-hand sides b = B g + h s for the operator above (Eq. 1-2):
 * b = d*g on inflow nodes (g ordered as `inflow`), h*s elsewhere.  nrhs
 * systems stored one after the other (b: nrhs*n, g: nrhs*n_inflow,
 * s: nrhs*n, s may be NULL for zero source).  DEVICE pointers.
 */
airg_status airg_assemble_rhs_advection2d(int64_t nx, int64_t ny, double vx, double vy,
                                          double h, int nrhs, const int64_t* inflow,
                                          int64_t n_inflow, const double* g, const double* s,
                                          double* b, void* stream);

/*
 * Transpose of airg_assemble_rhs_advection2d, for gradients through a solve:
 * with lambda = A^-T dL/du (airg_solve_adjoint), dL/dg = B^T lambda and
 * dL/ds = h lambda: grad_g[k] = d * lambda[inflow[k]], grad_s[i] = h *
 * lambda[i] on nodes that are not inflow nodes and 0 on inflow nodes (the
 * source does not enter their rows).  nrhs systems one after the other;
 * grad_s may be NULL.  DEVICE pointers.
 */
airg_status airg_rhs_adjoint_advection2d(int64_t nx, int64_t ny, double vx, double vy, double h,
                                         int nrhs, const int64_t* inflow, int64_t n_inflow,
                                         const double* lambda, double* grad_g, double* grad_s,
                                         void* stream);

/*
 * AIRG setup (Sec. 2): the level loop of truncation test (Sec. 2.4), CF
 * splitting (Sec. 2.1), block extraction, GMRES polynomial coefficients
 * (Eq. 7), fixed-sparsity inverse (Eq. 8), restrictor with drop, one-point
 * prolongator, RAP with drop and lumping, then the coarse-grid Newton
 * polynomial (Sec. 2.3), all on the GPU.  A is copied; the handle owns every
 * device buffer it allocates.  Setup values are reproducible: sums run in a
 * fixed order and dot products are correctly rounded.
 * A is validated before use (host or device arrays alike): square, n and
 * nnz below 2^31, rowptr[0] = 0 <= rowptr[i] <= rowptr[i+1] <= rowptr[n] =
 * nnz, columns strictly ascending within [0, n), a stored diagonal in every
 * row, finite values.  A row's entries are read only after its row pointers
 * pass.  Errors: AIRG_ERR_ARG (any of these), AIRG_ERR_OOM, AIRG_ERR_CUDA,
 * AIRG_ERR_BREAKDOWN.
 */
airg_status airg_setup(const airg_csr* A, const airg_options* opt, void* stream,
                       airg_handle** out);

/*
 * Solve A x = b with FGMRES(restart) right-preconditioned by one AIRG V-cycle
 * per iteration (Eq. 6: restriction, coarse Newton polynomial, one-point
 * prolongation, one up F-point smooth with the matrix-free GMRES
 * polynomial).  Converged when ||b - A x||_2 <= max(rtol ||b||_2, atol), the
 * unpreconditioned norm of Sec. 3.  b and x hold nrhs vectors of length n,
 * one after the other; x is the initial guess on entry and the solution on
 * exit.  on_device = 1: b and x are DEVICE pointers; 0: HOST pointers (the
 * copies in and out are part of the call; they go through device buffers
 * that the handle keeps, grown to the largest call, so pinned host memory
 * gives copies at link speed and no allocation per call).  info (HOST, may be NULL)
 * receives the worst iteration count / residual over the right-hand sides.
 * AIRG_ERR_NOT_CONVERGED still returns x and info.
 */
airg_status airg_solve(airg_handle* h, int nrhs, const double* b, double* x, int on_device,
                       double rtol, double atol, int maxit, airg_solve_info* info,
                       void* stream);

/*
 * Adjoint solve A^T lambda = rhs (the reversed-flow operator) with its own
 * AIRG hierarchy, built on the first call from the transpose of A and kept in
 * the handle.  Arguments as for airg_solve.
 */
airg_status airg_solve_adjoint(airg_handle* h, int nrhs, const double* rhs, double* lambda,
                               int on_device, double rtol, double atol, int maxit,
                               airg_solve_info* info, void* stream);

/*
 * Many separate problems (different operators, e.g. grids of uneven size),
 * one AIRG hierarchy each, solved together.  airg_setup_batch builds the
 * nprob hierarchies (As: HOST array of nprob CSR descriptors, same options
 * for all).  airg_solve_batch runs FGMRES in lockstep across the problems.
 * Each iteration of all problems -- scale v_j, V-cycle, SpMV, Gram-Schmidt
 * pass -- is one CUDA graph launch (captured once per iteration index and
 * replayed) in which every problem forms an independent branch of
 * per-operator kernels.  With the environment variable AIRG_MULTI=worklist
 * it is instead one persistent kernel launch (also captured) whose blocks
 * take the tiles of every problem's operations from a device work list in
 * dependency order, except for layouts the work list does not implement
 * (C-point smoothing, the assembled smoother, bfloat16 restrictor values,
 * the opt-in persistent or staged kernels), which stay in the graph form.
 * A bounded wait of the work list that gives up returns AIRG_ERR_TIMEOUT.
 * bvec, xvec: HOST arrays of nprob pointers
 * to vectors of each problem's length (DEVICE pointers if on_device, else
 * HOST); x is the initial guess on entry.  infos: HOST array of nprob
 * entries (may be NULL).  AIRG_ERR_NOT_CONVERGED if any problem misses the
 * tolerance; every x and info is still written.
 */
airg_status airg_setup_batch(int nprob, const airg_csr* As, const airg_options* opt, void* stream,
                             airg_batch** out);
airg_status airg_solve_batch(airg_batch* b, const double* const* bvec, double* const* xvec,
                             int on_device, double rtol, double atol, int maxit,
                             airg_solve_info* infos, void* stream);
/* Levels, sizes, complexities and V-cycle bytes of problem i (0 <= i <
 * nprob) of a batch, as airg_setup_info gives them for one hierarchy.  info
 * is a HOST pointer.  AIRG_ERR_ARG for a null batch or info or i out of
 * range. */
airg_status airg_batch_setup_info(const airg_batch* b, int i, airg_hierarchy_info* info);
/*
 * Timing of the lockstep iterations of airg_solve_batch: with profiling
 * enabled (which clears the totals), a CUDA event pair brackets each
 * iteration's launch -- the one work-list kernel, or the graph of
 * per-problem branches -- on the batch's stream.  airg_batch_profile_read
 * returns the summed event time (ms), the number of such launches and the
 * algorithmic bytes of the operations of the problems still active in them
 * (stored entries, column indices and each vector read or written once).
 * Outputs are HOST pointers.  AIRG_ERR_ARG for a null batch or output.
 */
airg_status airg_batch_profile(airg_batch* b, int enable);
airg_status airg_batch_profile_read(const airg_batch* b, double* ms, int64_t* launches, int64_t* bytes);
void airg_batch_free(airg_batch* b);

/* Levels, sizes and the complexities of Sec. 3.  info is a HOST pointer. */
airg_status airg_setup_info(const airg_handle* h, airg_hierarchy_info* info);

/*
 * Export one setup product of level `level` in the level's own numbering
 * (points in increasing index, F/C-local indices in increasing index), for
 * checking against an independent implementation.  `what`:
 *   0 A_l (the level operator)   1 A_ff   2 A_fc   3 Z (restrictor block, after drop)
 *   4 the fixed-sparsity Ahat_ff^-1 of Eq. 8 (kept only with AIRG_SMOOTH_ASSEMBLED)
 *   5 A_cc (kept only with C-point smoothing)
 *   6 the fixed-sparsity Ahat_cc^-1 (C-point smoothing with AIRG_SMOOTH_ASSEMBLED)
 * Two-call protocol with HOST buffers: pass NULL arrays to get *n_rows,
 * *n_cols, *nnz; then pass arrays of those sizes.  `what` = 0 on the coarsest
 * level returns the coarse operator.
 */
airg_status airg_export_matrix(const airg_handle* h, int level, int what, int64_t* n_rows,
                               int64_t* n_cols, int64_t* nnz, int64_t* rowptr, int32_t* col,
                               double* val);

/*
 * Export per-level vectors (HOST buffers, two-call protocol as above):
 *   what 0: CF marker, int8, n entries (1 = F, 0 = C)
 *   what 1: one-point prolongator W, int32 per F point (C-local index, -1 none)
 *   what 2: smoother coefficients alpha_0..alpha_p, double
 *   what 3: coarse Newton roots, double pairs (re, im), im > 0 for a
 *           conjugate pair, im == 0 for a real root (coarsest level only)
 *   what 4: per-level scalars, double: [pmisr_rounds, ddc_converted_pass1,
 *           ddc_converted_pass2.., trunc_rel, alpha_k]
 * *count receives the number of elements.
 */
airg_status airg_export_vector(const airg_handle* h, int level, int what, int64_t* count,
                               void* out);

/*
 * Per-kernel timing of the solve phase.  airg_profile(h, 1) makes every
 * kernel that airg_solve launches record a CUDA event before and after it on
 * the solve's stream, and clears the totals; airg_profile(h, 0) stops
 * recording.  airg_profile_read returns, for one kind of kernel, the summed
 * event time (ms), the number of launches and the algorithmic bytes those
 * launches move (stored entries, column indices and each vector read or
 * written once; padding excluded).  Kinds: 0 restriction, 1 F-point
 * residual, 2 F-point smoother (Horner terms), 3 coarse Newton steps,
 * 4 top-level SpMV of FGMRES, 5 FGMRES vector work, 6 layout / precision
 * conversions.  Outputs are HOST pointers.
 */
airg_status airg_profile(airg_handle* h, int enable);
/*
 * Like airg_profile(h, 1), but times only the launches of one kernel kind on
 * one level (the group that dominates the solve, say), so that the timed
 * solve carries as few event records as possible: consecutive launches of
 * the group inside one V-cycle (a kind 0-3 group: the restriction, F-point
 * residual, smoother or coarse Newton steps of a level) share one event
 * pair, while groups of kinds 4-6 get one pair per launch.  The totals are
 * read with airg_profile_read_level; airg_profile(h, 0) stops.  AIRG_ERR_ARG
 * for a kind outside 0..6 or a level outside 0..64.
 */
airg_status airg_profile_group(airg_handle* h, int kind, int level);
airg_status airg_profile_read(const airg_handle* h, int kind, double* ms, int64_t* launches,
                              int64_t* bytes);

/*
 * The same totals restricted to one level of the hierarchy: level l's
 * restriction, F-point residual and smoother launches, level = number of
 * levels - 1 for the coarse Newton steps, 0 for the top-level FGMRES, layout
 * and conversion kernels.  *flops receives the floating-point operations
 * those launches perform on stored entries and vectors (an FMA counts as
 * two; padding excluded).  0 <= level < 65; AIRG_ERR_ARG otherwise.
 */
airg_status airg_profile_read_level(const airg_handle* h, int kind, int level, double* ms,
                                    int64_t* launches, int64_t* bytes, int64_t* flops);

/*
 * Storage and row-kernel variant of one solve-phase operator, as the setup
 * laid it out (SELL-32: slices of 32 rows, padded to their longest row) and
 * as its timing of y = S x picked the variant (the product of Sec. 3's
 * solve-phase SpMVs is the same whichever variant runs).
 */
typedef struct {
    int64_t n_rows, n_cols;
    int64_t nnz;              /* stored entries, diagonal included            */
    int64_t padded;           /* SELL slots of the off-diagonal entries,
                                 padding included                             */
    int32_t warps_per_slice;  /* 1: short rows, one warp per slice or more    */
    int32_t r;                /* short rows: slices per warp (1, 2, 4); long
                                 rows: loads in flight per lane (4, 8, 16)    */
    int32_t resident_grid;    /* 1: the row kernels run on a grid of resident
                                 blocks that stride over the slices           */
    int32_t index_bytes;      /* column index bytes per entry that the
                                 single-vector row kernels read: 2 or 4       */
    int32_t slice_bases;      /* 1: those 16-bit indices are offsets from each
                                 slice's smallest column                      */
    int32_t value_bytes;      /* 8 FP64, 4 FP32, 2 bfloat16                   */
    int32_t dense_diagonal;   /* 1: the diagonal is a dense vector, outside
                                 the slices                                   */
} airg_operator_layout;

/* Operators of airg_operator_layout_info, in the precision the V-cycle runs
 * in (bfloat16 values for the restrictor with AIRG_MIXED_FP32_BF16R):
 * the top-level FP64 operator of the outer iteration (level 0); level l's
 * restrictor block Z (Eq. 4), F-point residual operator M = A_fc + A_ff W
 * (Eq. 6 with the one-point P), A_ff (Horner terms, Eq. 7), the assembled
 * Ahat_ff^-1 of Eq. 8 (AIRG_SMOOTH_ASSEMBLED); the C rows [A_cf A_cc], A_cc,
 * Ahat_cc^-1 and the F rows [A_ff A_fc] of C-point / FCF smoothing; and the
 * coarsest operator (level = number of levels - 1, Sec. 2.3). */
enum {
    AIRG_OPERATOR_TOP = 0, AIRG_OPERATOR_Z = 1, AIRG_OPERATOR_M = 2, AIRG_OPERATOR_AFF = 3,
    AIRG_OPERATOR_AINV = 4, AIRG_OPERATOR_C_ROWS = 5, AIRG_OPERATOR_ACC = 6,
    AIRG_OPERATOR_AINV_CC = 7, AIRG_OPERATOR_F_ROWS = 8, AIRG_OPERATOR_COARSE = 9
};

/*
 * Fills *out (a HOST struct) with the layout of operator `op` of level
 * `level`.  An operator that the hierarchy does not keep (Ahat^-1 without
 * the assembled smoother, the C-point operators without C-point smoothing)
 * is reported with n_rows = 0 and AIRG_OK.  AIRG_ERR_ARG for a NULL handle
 * or out, an `op` outside the enum, AIRG_OPERATOR_TOP on a level other than
 * 0, AIRG_OPERATOR_COARSE on another level than the coarsest, or a level
 * operator asked of the coarsest level or beyond it.
 */
airg_status airg_operator_layout_info(const airg_handle* h, int level, int op, airg_operator_layout* out);

/*
 * Failure-detection check of the device-side waits: launches one block that
 * waits, through the same bounded wait as the grid barrier of the
 * persistent kernels, for an arrival that never comes.  The wait must give
 * up after `spin_limit` polls of ~50 ns, record the error flag and let the
 * kernel finish; the call then returns AIRG_ERR_TIMEOUT (the designed
 * outcome) and the CUDA context stays usable.  Any other status means the
 * mechanism is broken.  Nothing hangs or faults.
 */
airg_status airg_check_wait_timeout(int64_t spin_limit, void* stream);

/* Releases every device and host buffer of the handle.  NULL is a no-op. */
void airg_free(airg_handle* h);

/* Text of the last error raised on the calling thread ("" if none). */
const char* airg_last_error(void);

/*
 * Building blocks exposed for testing (same contracts as their use inside
 * the setup):
 *  airg_dot_exact: <x, y> correctly rounded from the exact sum of exact
 *    products; x, y DEVICE (length n), result to *out (HOST).  n must be
 *    <= 2^31 - 1 (the accumulator's carry headroom); AIRG_ERR_ARG beyond.
 *  airg_rng_uniform: uniform [0,1) counter stream (SplitMix64, Steele, Lea &
 *    Flood 2014) of (seed, level, purpose) into out (DEVICE, length n).
 *  airg_host_gmres_coeffs: power-basis coefficients alpha (length k, HOST) of
 *    the GMRES polynomial from an Arnoldi Hessenberg H ((k+1) x k, row-major,
 *    HOST) and beta = ||b|| (Eq. 7), by Givens least squares; CPU only.
 *  airg_host_eigvals: eigenvalues (wr, wi; HOST, length n) of a real upper
 *    Hessenberg matrix (row-major n x n, HOST) by the Francis double-shift QR
 *    iteration; CPU only.  AIRG_ERR_BREAKDOWN if it does not converge.
 */
airg_status airg_dot_exact(int64_t n, const double* x, const double* y, double* out,
                           void* stream);
airg_status airg_rng_uniform(uint64_t seed, int64_t level, int64_t purpose, int64_t n,
                             double* out, void* stream);
airg_status airg_host_gmres_coeffs(int k, const double* H, double beta, double* alpha);
airg_status airg_host_eigvals(int n, const double* H, double* wr, double* wi);

/*
 * airg_dot_exact_noalloc: the same correctly rounded <x, y> as
 * airg_dot_exact, for callers that cannot allocate device memory: code
 * inside a framework whose caching pool has reserved the device's memory (a
 * cudaMalloc behind its back can fail or fragment it), or a latency-critical
 * loop where cudaMalloc / cudaFree would synchronise the device.  The paper
 * has no counterpart: it is a service of this library.
 *  - Allocates nothing: its scratch is a file-scope __device__ array of
 *    141 x 8 bytes (accumulator + inf/nan flag) that every GPU loading the
 *    library keeps until the process exits.
 *  - x, y: DEVICE pointers, length n; out: DEVICE pointer to one double.
 *    Asynchronous: the result is in *out when `stream` reaches that point.
 *  - n must be <= 2^31 - 1 (the accumulator's carry headroom);
 *    AIRG_ERR_ARG beyond that, before any GPU work.
 *  - The first call on a device looks up the scratch array's device address
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *    The address is kept per device ordinal for the life of the process: it
 *    does not survive cudaDeviceReset or a switch to another context on the
 *    same device: after either, this entry point must not be called again
 *    in the process.
 *  - All calls on a device share the scratch: each call clears it first, and
 *    calls that overlap on the GPU (different streams, no ordering) race.
 */
airg_status airg_dot_exact_noalloc(int64_t n, const double* x, const double* y, double* out,
                                   void* stream);

#ifdef __cplusplus
}
#endif

#endif /* AIRG_H */
