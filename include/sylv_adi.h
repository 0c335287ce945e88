/*
 * sylv_adi.h - C ABI of the GB300 inexact low-rank Sylvester ADI solver.
 *
 * Solves  A X + X B = -f g^*  (paper eq. (sylv)) for large sparse real A (n x n),
 * B (m x m) and low-rank f (n x r), g (m x r), returning X ~ Z Gamma Y^* by the
 * inexact LR-ADI iteration (Algorithm 1, M = I, C = I).  Each outer step solves
 * the shifted systems (A + beta_k I) z_k = w_{k-1} and (B + alpha_k I)^* y_k =
 * t_{k-1} (eq. (lradi_basic)) with restarted, right-Jacobi-preconditioned
 * GMRES(m) per column, stopped at the tolerances delta^A_k / r, delta^B_k / r
 * chosen by the paper's controller (Sec. 3.3: eqs. (ADI_relax1_prak),
 * (upd_resgap), (ADI_relax2_prak), (simple_tols), (one_side)).  All of it runs
 * on the GPU; the host only launches work and reads a status word.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: SYLV_OK (0) or a negative SYLV_ERR_* code.  Nothing aborts,
 *   nothing traps.  sylv_last_error() gives a message for the calling thread.
 * - Dense blocks are column-major with leading dimension = number of rows.
 * - Complex numbers are pairs of doubles (re, im), i.e. C99 double complex.
 * - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Work is enqueued on it; calls that return results to the host synchronise it.
 * - Input pointers are borrowed for the duration of the call only; objects copy
 *   what they keep.  Objects own the device memory they allocate and release it
 *   in their destroy call.
 * - Indices are 0-based int32; values float64.
 */
#ifndef SYLV_ADI_H
#define SYLV_ADI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SYLV_OK                 0
#define SYLV_ERR_INVALID       -1   /* bad argument (null pointer, size, CSR structure) */
#define SYLV_ERR_CUDA          -2   /* a CUDA runtime call failed, or a bounded wait in a kernel gave up */
#define SYLV_ERR_NOMEM         -3   /* device or host allocation failed */
#define SYLV_ERR_MAXIT         -4   /* kmax outer steps without reaching tau; factors valid */
#define SYLV_ERR_INNER_STALL   -5   /* an inner solve hit max_inner before its tolerance */
#define SYLV_ERR_NONFINITE     -6   /* NaN or Inf met in a norm */
#define SYLV_ERR_NOT_SOLVED    -7   /* results asked for before sylv_adi_solve */
#define SYLV_ERR_UNSUPPORTED   -8   /* option combination not built */

/* ---- inner-tolerance strategies (Sec. 3.3 and Sec. 4's list of settings) ---- */
#define SYLV_STRAT_FIXED        0   /* delta^A = delta^B = fixed_tol (Sec. 4, "fixed") */
#define SYLV_STRAT_NOBL_MID     1   /* eq. (ADI_relax1_prak) + eq. (simple_tols) */
#define SYLV_STRAT_BL_MID       2   /* eq. (ADI_relax2_prak) + eq. (simple_tols) */
#define SYLV_STRAT_NOBL_A       3   /* eq. (ADI_relax1_prak) + eq. (one_side): delta^A = delta^A_min */
#define SYLV_STRAT_BL_A         4   /* eq. (ADI_relax2_prak) + eq. (one_side) */
#define SYLV_STRAT_NOBL_B       5   /* mirror of eq. (one_side): delta^B = delta^B_min */
#define SYLV_STRAT_BL_B         6

/* ---- precision of the inner Krylov solves ---- */
#define SYLV_PREC_FP64          0   /* everything in float64 (complex128 for complex shifts) */
#define SYLV_PREC_FP32          1   /* Krylov basis and its sweeps in float32 (complex64); the
                                       restart residual, the Hessenberg least squares, the
                                       solutions, the factors and the outer iteration in float64 */
#define SYLV_PREC_BF16          2   /* as FP32 with the Krylov basis stored in bfloat16 */

/* Sparse square matrix in CSR form.  Borrowed; copied by the create calls. */
typedef struct sylv_csr {
    int32_t n_rows, n_cols;      /* must be equal */
    int64_t nnz;
    const int32_t* rowptr;       /* n_rows + 1 entries, rowptr[0] = 0, nondecreasing */
    const int32_t* colind;       /* nnz entries in [0, n_cols) */
    const double*  val;          /* nnz entries */
    int32_t on_device;           /* 0: host pointers, 1: device pointers */
} sylv_csr;

typedef struct sylv_shift { double re, im; } sylv_shift;

/* Solver options; sylv_opts_default() fills the paper's defaults (Sec. 4):
 * xi = 1, delta_min = tau/20 (set at create when left <= 0), delta_max = 0.1,
 * kmax = 50, strategy BL_MID, fixed_tol = tau/20 (when <= 0), GMRES(30),
 * max_inner = 20000, float64, right Jacobi on, inner = SYLV_INNER_GMRES. */
typedef struct sylv_opts {
    double  xi;                  /* safeguard xi in (0, 1] of eqs. (ADI_relax1/2_prak) */
    double  dmin_A, dmin_B;      /* eq. (bound_tols) lower clamps; <= 0 means tau/20 */
    double  dmax_A, dmax_B;      /* eq. (bound_tols) upper clamps */
    int32_t kmax;                /* maximum number of outer steps (divisor in hat-eps) */
    int32_t strategy;            /* SYLV_STRAT_* */
    double  fixed_tol;           /* tolerance of SYLV_STRAT_FIXED; <= 0 means tau/20 */
    int32_t restart;             /* GMRES restart length m, 1..SYLV_MAX_RESTART */
    int32_t max_inner;           /* cap on Arnoldi steps per column solve */
    int32_t precision;           /* SYLV_PREC_* */
    int32_t jacobi;              /* 1: right preconditioner P = diag(Op) + shift diag(Mass)
                                    (Mass = I unless the generalized equation gives one) */
    int32_t bl_clamp;            /* 0: eq. (ADI_relax2_prak) literally, |.|;
                                    1: max(., 0) in place of |.| (paper silent) */
    int32_t rows_per_chunk;      /* work-unit size of the vector kernels; 0 = auto */
    int32_t driver;              /* 0: each solve is one CUDA graph whose conditional nodes
                                    the kernels set (no host round trip inside a solve);
                                    1: the host launches every device iteration.  Profiling
                                    (sylv_adi_profile) always uses the host-driven loop.
                                    The host-driven loop launches the kernels of an iteration
                                    with programmatic stream serialization (each kernel waits
                                    for its predecessor on the device; the next one is
                                    scheduled early), falling back to plain launches if the
                                    attribute is refused; the environment variable
                                    SYLV_NO_PDL, when set, selects plain launches (results
                                    are the same; profilers that cannot follow programmatic
                                    launches need it). */
    int32_t ortho;               /* Arnoldi orthogonalisation of the inner GMRES:
                                    SYLV_ORTHO_CGS2: classical Gram-Schmidt twice, three
                                    sweeps over the basis and three reductions per step;
                                    SYLV_ORTHO_DCGS2: the second pass delayed into the next
                                    step (Swirydowicz et al., Numer. Linear Algebra Appl. 28,
                                    2021): two sweeps, one reduction per step */
    int32_t restart_every;       /* host driver only: launch the restart kernels (update of x,
                                    true residual, new cycle) in the first device iteration
                                    of an outer step and then every restart_every-th one
                                    (0 or 1: every iteration; default 4).  A system whose
                                    cycle ended waits for the next such iteration; results
                                    are the same, idle launches fewer (measured on the 2D
                                    benchmark workload: 1.59 s -> 1.45 s).  The graph driver
                                    launches them only when a cycle has ended. */
    int32_t inner;               /* inner solver of the shifted systems (Sec. 3.3 "Further
                                    implementation aspects": any Krylov method whose residual
                                    norm is available, right preconditioned):
                                    SYLV_INNER_GMRES: restarted GMRES(restart), ortho as above;
                                    SYLV_INNER_BICGSTAB: BiCGstab (van der Vorst 1992), the
                                    short-recurrence solver of the paper's experiments (Sec. 4):
                                    no Krylov basis, two products per step; restart and ortho
                                    are unused and precision SYLV_PREC_BF16 is not built (there
                                    is no basis to store) */
    int32_t real_pairs;          /* complex shifts only: 0: the complex formulation (two complex
                                    steps per conjugate pair, complex factors, as the paper's
                                    experiments keep it); 1: the real double step per conjugate
                                    pair (Sec. 3.3 "Complex shift parameters"): one complex solve
                                    per column for a side whose shift is complex (the second
                                    solution follows from the first), two real-shift solves for a
                                    side whose shift is real, real factors Z, Y and a real core
                                    with 2 x 2 blocks (sylv_adi_core).  Runs the host-driven loop;
                                    not built for batches with complex shifts. */
    int32_t autotune;            /* with rows_per_chunk = 0: 1 times a bounded set of work-chunk
                                    sizes (the default rule's size and 512 .. 8192 rows) on the
                                    actual systems at create - synthetic vectors and a stencil of
                                    the operators' shape, CUDA events over a few device
                                    iterations - and keeps the fastest (sylv_adi_tuning reports
                                    them); 0 (the default) uses the default rule, so that results
                                    do not depend on timing: GMRES one wave of resident blocks
                                    over all rows, BiCGstab at most 768 rows (at least 256) */
} sylv_opts;

#define SYLV_INNER_GMRES     0
#define SYLV_INNER_BICGSTAB  1

#define SYLV_ORTHO_CGS2  0
#define SYLV_ORTHO_DCGS2 1

#define SYLV_MAX_RESTART 30
#define SYLV_MAX_RANK    4

typedef struct sylv_info {
    int32_t status;              /* last solve's status (SYLV_OK or SYLV_ERR_*) */
    int32_t steps;               /* outer steps taken (k - 1 at exit) */
    int32_t kr;                  /* columns of Z and Y = steps * r */
    int32_t is_complex;          /* factors are complex (complex shifts) */
    double  rel_res_comp;        /* ||w_k t_k^*|| / ||f g^*|| at exit (the stop test) */
    double  norm_fg;             /* ||f g^*||_2 */
    int64_t inner_its_A;         /* sum of Arnoldi steps over all A-side column solves */
    int64_t inner_its_B;
    int64_t inner_restarts;      /* GMRES cycles over all solves */
    int32_t stalled_solves;      /* inner solves that hit max_inner */
    int32_t ticks;               /* device iterations launched (for diagnostics) */
    int64_t launches;            /* kernel launches of the last solve */
} sylv_info;

/* Columns of one row of sylv_adi_history() (doubles, row-major). */
#define SYLV_HIST_COLS 14
/* k, alpha_re, beta_re, delta_A, delta_B, hat_eps, ||r^A_k||, ||r^B_k||,
 * its_A, its_B, u_k, v_k, ||w_k t_k^*||/||fg^*||, ||w_{k-1}||              */

typedef struct sylv_handle sylv_handle;
typedef struct sylv_op sylv_op;

/* Message describing the last error on the calling thread ("" if none). */
const char* sylv_last_error(void);

/* Fill *o with the defaults above.  Returns SYLV_ERR_INVALID for o == NULL. */
int sylv_opts_default(sylv_opts* o);

/* ------------------------------------------------------------------------ */
/* Shifted sparse operator (steps a2/a3 of the hot path)                     */
/* ------------------------------------------------------------------------ */

/* Upload a CSR matrix (or its transpose, transpose = 1) as a device operator.
 * A matrix whose nonzeros lie on at most 9 fixed diagonals (finite-difference
 * stencils, Sec. 4 eq. (ex:convdiff)) is stored by diagonals so the product
 * reads no column indices; any other CSR is kept as CSR.  The main diagonal is
 * kept for the Jacobi preconditioner.  Errors: SYLV_ERR_INVALID for a
 * malformed CSR (non-square, rowptr not monotone, column out of range). */
int sylv_op_create(const sylv_csr* csr, int32_t transpose, sylv_op** out);
/* The same for the shifted operators of the generalized equation
 * A X C + M X B = -f g^* (eq. (gsylv), Algorithm 1 with M, C): Op + sigma Mass
 * with a mass matrix of the same size (mass = NULL: Mass = I).  Both are
 * stored by diagonals when their nonzeros together lie on at most 9 fixed
 * offsets (the 2D finite element mass matrices of the Q1 elements), else as
 * two CSR matrices.  transpose = 1 stores Op^T and Mass^T.  The Jacobi
 * preconditioner becomes P = diag(Op) + sigma diag(Mass). */
int sylv_op_create_g(const sylv_csr* csr, const sylv_csr* mass, int32_t transpose, sylv_op** out);
/* Storage format chosen: 1 = by diagonals (*ndiag set), 0 = CSR. */
int sylv_op_format(const sylv_op* op, int32_t* is_stencil, int32_t* ndiag, int32_t* n);
/* Y = (Op + sigma I) P^{-1} X for ncols columns (device pointers, n x ncols,
 * column-major), P = diag(Op) + sigma I when jacobi = 1, else P = I.  This is
 * the operator of the inner systems of Algorithm 1 (A + beta_k I, or B^T +
 * conj(alpha_k) I) under right preconditioning (Sec. 3.3).  is_complex = 1
 * treats X, Y as complex (interleaved) vectors; sigma must be real otherwise. */
int sylv_op_apply(const sylv_op* op, sylv_shift sigma, int32_t jacobi, int32_t is_complex,
                  const void* X, void* Y, int32_t ncols, void* stream);
int sylv_op_destroy(sylv_op* op);

/* ------------------------------------------------------------------------ */
/* One CGS2 orthogonalisation step (step a4)                                 */
/* ------------------------------------------------------------------------ */

/* Given k orthonormal columns V (n x k, device, ld = n) and w (n, device):
 * h = V^* w, w -= V h, h2 = V^* w, w -= V h2 (classical Gram-Schmidt applied
 * twice); on return w holds the orthogonalised vector divided by its norm,
 * h_out (host, k + 1 entries) holds h + h2 followed by the norm.  1 <= k <= 30.
 * is_complex as for sylv_op_apply; h_out then holds k + 1 complex entries.
 * The Arnoldi step of the inner GMRES solves uses the same device code. */
int sylv_cgs2(const void* V, int32_t n, int32_t k, void* w, void* h_out,
              int32_t is_complex, void* stream);

/* The same CGS2 step for callers that cannot let a library allocate GPU
 * memory (a pool or arena that owns the device budget, loops that must not
 * allocate after start-up, custom memory managers).  The paper has no
 * counterpart; this is a library service.  Real data only.
 * V: device, n x (k + 1), column-major (ld = n); columns 0..k-1 hold the
 * orthonormal basis, column k receives the orthogonalised w divided by its
 * norm.  w: device, n entries, read only.  h_out: host, k + 1 entries, as for
 * sylv_cgs2.  1 <= k <= 30 and n <= sylv_cgs2_noalloc_max_rows().
 * Scratch lives in one static device array of SYLV_NOALLOC_SCRATCH_BYTES
 * that every GPU loading this library holds until the process exits; no
 * cudaMalloc/cudaFree or other allocating call is made.  Each call looks up
 * that array's device address on the current device, copies its small
 * descriptors from host memory and synchronises the stream before it
 * returns: the call is synchronous and must not be made while its stream is
 * being captured into a CUDA graph.  All calls share the array and each call
 * re-initialises what it reads, so calls that overlap on the GPU (other
 * streams, other host threads) race: serialise them.  Sizes beyond the
 * limit return SYLV_ERR_INVALID with a message. */
#define SYLV_NOALLOC_SCRATCH_BYTES (1 << 20)
int sylv_cgs2_noalloc(double* V, int32_t n, int32_t k, const double* w, double* h_out, void* stream);
/* Largest n sylv_cgs2_noalloc accepts. */
int sylv_cgs2_noalloc_max_rows(void);

/* ------------------------------------------------------------------------ */
/* Batched shifted GMRES (steps a2-a7)                                       */
/* ------------------------------------------------------------------------ */

/* Solve (Op + sigma I) x_l = b_l for l = 0..ncols-1 (device, n x ncols), each
 * column by restarted GMRES(restart) with x0 = 0, right Jacobi when jacobi =
 * 1, stopping when the Givens residual estimate is <= tol and confirming with
 * the recomputed true residual ||b_l - (Op + sigma I) x_l|| <= tol (a new cycle
 * starts otherwise), or after max_iters Arnoldi steps.  The columns run
 * concurrently in one set of launches.  Outputs (host arrays of ncols):
 * iters_out (Arnoldi steps), resnorm_out (true residual norms).
 * Returns SYLV_ERR_INNER_STALL if some column stopped at max_iters.
 * Optional hist_out (host, ncols x max_iters doubles, may be NULL): the Givens
 * residual estimate after each Arnoldi step.  precision = SYLV_PREC_*: with
 * FP32/BF16 the basis and its sweeps run in float32 while B, X, the restart
 * residual and the least squares stay float64 (iterative refinement across
 * restarts), so tol is still met in float64. */
int sylv_gmres(const sylv_op* op, sylv_shift sigma, int32_t jacobi, int32_t is_complex,
               const void* B, void* X, int32_t ncols, double tol, int32_t restart,
               int32_t max_iters, int32_t precision, int32_t* iters_out, double* resnorm_out,
               double* hist_out, void* stream);

/* One Arnoldi cycle of k steps (1 <= k <= SYLV_MAX_RESTART) of the inner
 * GMRES exactly as the solver runs it (steps a2-a4): the operator
 * (Op + sigma I) P^{-1} (right Jacobi when jacobi = 1), the Krylov basis in
 * the storage and sweep precision of precision (SYLV_PREC_*), classical
 * Gram-Schmidt twice (ortho = SYLV_ORTHO_CGS2) or with the second pass
 * delayed (SYLV_ORTHO_DCGS2), from the unit start vector v0 (device, n
 * entries).  Outputs: V_out (device, n x (k + 1), column-major) the basis
 * vectors v_0..v_k (with DCGS2 the cycle does not complete v_k: that column
 * is zero), H_out (host, (k + 1) x k, column-major) the Hessenberg matrix as
 * formed, with Op' V_k = V_{k+1} H.  Values are float64 (complex128 when
 * is_complex).  SYLV_ERR_NONFINITE if the cycle ended early (breakdown). */
int sylv_arnoldi(const sylv_op* op, sylv_shift sigma, int32_t jacobi, int32_t is_complex, const void* v0,
                 int32_t k, int32_t precision, int32_t ortho, void* V_out, void* H_out, void* stream);

/* Solve (Op + sigma I) x_l = b_l for l = 0..ncols-1 by BiCGstab (van der
 * Vorst, SIAM J. Sci. Stat. Comput. 13, 1992; the inner solver of the paper's
 * experiments, Sec. 4) with x0 = 0, right Jacobi when jacobi = 1.  Each
 * column stops when its recurrence residual (||s|| or ||r||) is <= tol, at a
 * breakdown (rhat^* v = 0, rho = 0 or omega = 0) or after max_iters steps;
 * the true residual ||b_l - (Op + sigma I) x_l|| is then recomputed in
 * float64 and, if it is above tol, a new cycle starts from x with a fresh
 * shadow vector rhat = r.  Arguments and outputs as sylv_gmres (iters_out
 * counts BiCGstab steps, two operator applications each; hist_out the
 * recurrence residual norm after each step).  The columns of one call share
 * each launch, with the operator read once per row for up to four columns.
 * precision = SYLV_PREC_FP64 or SYLV_PREC_FP32 (vectors and products in
 * float32, x and the restart residual in float64).  Returns
 * SYLV_ERR_INNER_STALL if a column stopped at max_iters. */
int sylv_bicgstab(const sylv_op* op, sylv_shift sigma, int32_t jacobi, int32_t is_complex,
                  const void* B, void* X, int32_t ncols, double tol, int32_t max_iters,
                  int32_t precision, int32_t* iters_out, double* resnorm_out, double* hist_out,
                  void* stream);

/* ------------------------------------------------------------------------ */
/* Inner-tolerance controller (step a1), evaluated by the device code         */
/* ------------------------------------------------------------------------ */

/* For each of count inputs, in[i*11 + 0..10] = {k, kmax, eps, xi, u_prev,
 * v_prev, N_w, N_t, fixed_tol, (unused), (unused)}, with clamps from o, write
 * out[i*3 + 0..2] = {delta^A_k, delta^B_k, hat-eps_k} (host arrays).  Runs
 * the same device function the solver runs at the start of every step. */
int sylv_controller_eval(const sylv_opts* o, int32_t count, const double* in, double* out);

/* ------------------------------------------------------------------------ */
/* Full solver (Algorithm 1)                                                 */
/* ------------------------------------------------------------------------ */

/* Create a solver for A X + X B = -f g^*.
 * A: n x n, B: m x m (CSR, borrowed, copied).  f: n x r, g: m x r (host,
 * column-major, real).  alpha[i], beta[i] (i < n_shifts) is the i-th shift
 * pair, reused cyclically when the iteration runs past n_shifts; complex pairs
 * must be followed immediately by their conjugate pair.  tol = tau of
 * Algorithm 1 (stop when ||w t^*|| < tau ||f g^*||).  opts may be NULL.
 * Allocates all device memory the solve needs (factors for kmax steps, Krylov
 * bases for the 2r column solves).  Errors: SYLV_ERR_INVALID, SYLV_ERR_NOMEM,
 * SYLV_ERR_UNSUPPORTED (r > SYLV_MAX_RANK, restart > SYLV_MAX_RESTART). */
int sylv_adi_create(const sylv_csr* A, const sylv_csr* B, const double* f, const double* g,
                    int32_t r, const sylv_shift* alpha, const sylv_shift* beta,
                    int32_t n_shifts, double tol, const sylv_opts* opts, void* stream,
                    sylv_handle** out);
/* The generalized equation A X C + M X B = -f g^* (eq. (gsylv)) with
 * nonsingular M (n x n) and C (m x m); M = NULL or C = NULL means identity.
 * Algorithm 1 as printed: inner systems (A + beta_k M) z = w_{k-1} and
 * (B + alpha_k C)^* y = t_{k-1}, updates w_k = w_{k-1} + gamma_k M z_k and
 * t_k = t_{k-1} + conj(gamma_k) C^* y_k (eq. (lradi_g)), and the residual-gap
 * estimate of eq. (upd_resgap) with ||M z_k||, ||C^T y_k||; X = Z Gamma Y^*
 * as before.  Other arguments, errors and ownership as sylv_adi_create;
 * SYLV_ERR_UNSUPPORTED with real_pairs = 1 and complex shifts. */
int sylv_adi_create_g(const sylv_csr* A, const sylv_csr* B, const sylv_csr* M, const sylv_csr* C,
                      const double* f, const double* g, int32_t r, const sylv_shift* alpha,
                      const sylv_shift* beta, int32_t n_shifts, double tol, const sylv_opts* opts,
                      void* stream, sylv_handle** out);
/* Replace f and g (same shapes) before the next solve; host pointers. */
int sylv_adi_set_rhs(sylv_handle* h, const double* f, const double* g);
/* Same, from device pointers (n x r and m x r float64, column-major). */
int sylv_adi_set_rhs_device(sylv_handle* h, const double* f, const double* g);
/* Run Algorithm 1 from w_0 = f, t_0 = g.  Blocks until done; returns the
 * solve's status (SYLV_OK, SYLV_ERR_MAXIT, SYLV_ERR_INNER_STALL as a warning,
 * SYLV_ERR_NONFINITE). */
int sylv_adi_solve(sylv_handle* h);
int sylv_adi_info(const sylv_handle* h, sylv_info* info);
/* Per-step metrics, rows of SYLV_HIST_COLS doubles (see above); writes
 * min(cap, steps) rows to buf and the row count to *rows. */
int sylv_adi_history(const sylv_handle* h, double* buf, int32_t cap, int32_t* rows);
/* Copy Z (n x kr), Y (m x kr) and gamma (kr) to caller buffers (host when
 * on_device = 0, device otherwise).  Complex factors are written as
 * interleaved pairs.  Any of Z, Y, gamma may be NULL to skip it. */
int sylv_adi_factors(const sylv_handle* h, void* Z, void* Y, void* gamma, int32_t on_device,
                     int32_t* kr_out, int32_t* is_complex);
int sylv_adi_destroy(sylv_handle* h);
/* The real core of X = Z G Y^T when the factors are real (real shifts, or
 * real_pairs = 1): G is kr x kr (host, column-major, leading dimension
 * ld >= kr), diagonal for plain steps (gamma_k I_r) and with a 2 x 2 block
 * P diag(gamma, conj gamma) Q^* (kron I_r) per conjugate pair.  G may be NULL
 * to query kr.  With complex factors (the complex formulation) the core is
 * the diagonal returned by sylv_adi_factors and this call returns
 * SYLV_ERR_UNSUPPORTED.  With real_pairs = 1, sylv_adi_factors returns real
 * Z, Y and must be given gamma = NULL. */
int sylv_adi_core(const sylv_handle* h, double* G, int32_t ld, int32_t* kr_out);

/* The work-chunk size (rows per work item of the inner-solver kernels) a
 * handle uses, and with opts.autotune the candidates timed at create with
 * their milliseconds per device iteration (at most cap of them; *count gets
 * their number). */
int sylv_adi_tuning(const sylv_handle* h, int32_t* rows_per_chunk, int32_t* cand, double* ms, int32_t cap,
                    int32_t* count);

/* Kernel statistics of a handle.  SYLV_NUM_KERNELS entries, in this order:
 * shifted product + first Gram-Schmidt sweep, second sweep, third sweep with
 * the Givens update, restart update, restart residual, controller,
 * step initialisation, factor update + Gram.  sylv_adi_profile(h, 1) resets
 * the counters and times the launches of every fourth device iteration (and
 * every outer-step kernel) with CUDA events on the handle's stream; 0 stops
 * the timing and resets too.  sylv_adi_kernel_stats copies, per kernel, the
 * estimated milliseconds (mean event-timed duration of the timed launches
 * times the number of launches; 0 when not profiling), the algorithmic bytes
 * moved and floating-point operations (accumulated by the kernels from each
 * system's size, Krylov index and the matrix's nonzeros) and the number of
 * launches, since the last reset.  Any pointer may be NULL. */
#define SYLV_NUM_KERNELS 8
int sylv_adi_profile(sylv_handle* h, int32_t enable);
int sylv_adi_kernel_stats(const sylv_handle* h, double* ms, double* bytes, double* flops,
                          int64_t* launches);

/* ------------------------------------------------------------------------ */
/* Batched solves: many independent equations in one device loop            */
/* ------------------------------------------------------------------------ */
/* One equation A X + X B = -f g^* of a batch, with its own sizes, rank,
 * shift pairs and tolerance (the arguments of sylv_adi_create). */
typedef struct sylv_problem {
    const sylv_csr* A;
    const sylv_csr* B;
    const double* f;            /* n x r, host */
    const double* g;            /* m x r, host */
    int32_t r;
    const sylv_shift* alpha;    /* n_shifts pairs, host */
    const sylv_shift* beta;
    int32_t n_shifts;
    double tol;
} sylv_problem;

typedef struct sylv_batch sylv_batch;

/* Every instance runs Algorithm 1 with the same options (opts may be NULL;
 * dmin and fixed_tol defaults follow each instance's tol).  The 2 r_i column
 * systems of all instances share each sweep launch and instances move
 * between outer steps independently.  opts->driver = 0: a solve is one CUDA
 * graph launch with no host round trip; 1: the host launches every device
 * iteration (outer kernel, step set-up, inner kernels) and reads a mapped
 * word that the device clears when the last instance finishes (used while
 * profiling).  If any instance has complex shifts the whole batch runs in
 * complex arithmetic.  Pointers are borrowed for the call.  Errors as
 * sylv_adi_create, the message naming the instance. */
int sylv_adi_batch_create(int32_t count, const sylv_problem* probs, const sylv_opts* opts, void* stream,
                          sylv_batch** out);
/* Solve all instances (blocks until done).  SYLV_OK when every instance
 * reached its tolerance, else the status of the first instance that did not
 * (sylv_adi_batch_info gives each instance's status). */
int sylv_adi_batch_solve(sylv_batch* b);
/* Per instance i (0 <= i < count): as sylv_adi_info / _history / _factors.
 * ticks and launches in the info are those of the whole batch solve. */
int sylv_adi_batch_info(const sylv_batch* b, int32_t i, sylv_info* info);
int sylv_adi_batch_history(const sylv_batch* b, int32_t i, double* buf, int32_t cap, int32_t* rows);
int sylv_adi_batch_factors(const sylv_batch* b, int32_t i, void* Z, void* Y, void* gamma, int32_t on_device,
                           int32_t* kr_out, int32_t* is_complex);
/* Whole-batch counters since create: kernel launches and device iterations
 * of the last solve; algorithmic bytes and flops of all kernels. */
int sylv_adi_batch_stats(const sylv_batch* b, int64_t* launches, double* bytes, double* flops,
                         int64_t* ticks);
/* Replace instance i's f (n_i x r_i) and g (m_i x r_i), host pointers,
 * before the next solve. */
int sylv_adi_batch_set_rhs(sylv_batch* b, int32_t i, const double* f, const double* g);
/* As sylv_adi_profile / sylv_adi_kernel_stats for the whole batch (the
 * outer-step counter holds the batch's outer kernel, the step counter its
 * set-up kernel); profiling runs the host-driven loop. */
int sylv_adi_batch_profile(sylv_batch* b, int32_t enable);
int sylv_adi_batch_kernel_stats(const sylv_batch* b, double* ms, double* bytes, double* flops, int64_t* launches);
/* As sylv_adi_tuning for a batch. */
int sylv_adi_batch_tuning(const sylv_batch* b, int32_t* rows_per_chunk, int32_t* cand, double* ms, int32_t cap,
                          int32_t* count);
int sylv_adi_batch_destroy(sylv_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* SYLV_ADI_H */
