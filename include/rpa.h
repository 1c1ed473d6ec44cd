/*
 * rpa.h -- C interface of librpa, a single-GPU (GB300, sm_103a) implementation of the
 * hot path of the real-space RPA correlation-energy method of B. Zhang, S. Shah,
 * J. E. Pask, E. Chow and P. Suryanarayana, "Random Phase Approximation Correlation
 * Energy using Real-Space Density Functional Perturbation Theory" (arXiv 2504.01816).
 *
 * Discrete model (the paper's Formulation and Implementation sections):
 *   grid        nx*ny*nz points, spacing h, zero (Dirichlet) values outside the box;
 *               point (i,j,k) at index i + nx*(j + ny*k).  N_d = nx*ny*nz.
 *   H           -1/2 L_h + diag(V_loc); L_h the 12th-order centred FD Laplacian
 *               (Section "Implementation": high-order centred finite differences,
 *               matrix-free application).
 *   orbitals    u_n, n < N_s, l2-orthonormal eigenvectors of H (u = psi h^{3/2}) with
 *               eigenvalues eps_n (the ground state the paper reads from files).
 *   nu^p        (4 pi)^p (-L_h)^{-p}, applied by the Kronecker-product formalism
 *               (per-axis eigendecompositions of the 1D second-difference matrices;
 *               Section "Implementation"; Poisson equation, Eq. 5).
 *   chi0(iw) dV = (4/h^3) Re sum_n u_n (.) x_n,  (H - eps_n + i w) x_n = -P_c(u_n (.) dV),
 *               P_c = I - U U^T  (Eqs. 7-9; the Galerkin initial guess of Section
 *               "Implementation" removes exactly the occupied components that P_c removes).
 *   E_c         (1/2pi) int_0^inf sum_{i<N_r} [log(1-lambda_i) + lambda_i] dw over the
 *               lowest N_r eigenvalues lambda_i of nu^1/2 chi0 nu^1/2 (Eq. 10), by
 *               subspace iteration with Rayleigh-Ritz (Algorithm 1) and Gauss-Legendre
 *               frequencies mapped to [0, inf) by w = w0 (1+x)/(1-x).
 *
 * Conventions shared by every entry point:
 *   - Pointers named *_dev are device pointers on the current CUDA device; *_host are host
 *     pointers.  The caller owns every buffer it passes; the library never frees, keeps or
 *     aliases them beyond the call (rpa_setup copies what it needs).
 *   - A block of K grid functions is an N_d x K column-major matrix of doubles: column c
 *     starts at c*N_d.  Complex vectors are interleaved (re, im) doubles.
 *   - stream is a cudaStream_t passed as void* (NULL = the legacy default stream).  Work
 *     is enqueued on it; calls that return host results synchronise it.
 *   - Every call returns an rpa_status; nothing throws across this interface.  On any
 *     status other than RPA_OK, rpa_last_error() gives a message (thread-local).
 *     RPA_ERR_NOT_CONVERGED still fills every output.
 *   - A context is not thread-safe: calls on one context must not overlap.
 */
#ifndef RPA_H
#define RPA_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rpa_ctx rpa_ctx;

typedef enum {
    RPA_OK = 0,
    RPA_ERR_INVALID = 1,        /* bad argument (size, pointer, option) */
    RPA_ERR_CUDA = 2,           /* a CUDA runtime error */
    RPA_ERR_OOM = 3,            /* device allocation failed */
    RPA_ERR_NOT_CONVERGED = 4,  /* a COCG solve hit maxit; outputs are still written */
    RPA_ERR_BREAKDOWN = 5,      /* COCG breakdown: p^T A p or r^T r vanished */
    RPA_ERR_NOT_SPD = 6         /* the overlap matrix R^T R is not positive definite */
} rpa_status;

typedef enum {
    RPA_FP64 = 0,   /* plain form: complex FP64 COCG */
    RPA_MIXED = 1   /* complex FP32 COCG inside FP64 iterative refinement */
} rpa_precision;

typedef struct {
    int prec;                  /* rpa_precision */
    double tol;                /* COCG: stop when ||b - A x||_2 <= tol ||b||_2 (Hermitian norm) */
    int maxit;                 /* COCG: iteration limit per system (FP64) or per inner solve (mixed) */
    int max_refine;            /* mixed: limit on FP64 residual evaluations per system */
    double inner_tol;          /* mixed: relative residual reduction asked of each FP32 inner solve */
    double eps_c;              /* subspace iteration: stop when |dE_c,m| <= eps_c * n_atoms / n_omega (Ha/atom) */
    int n_omega;               /* Gauss-Legendre frequency count (<= 64) */
    double omega0;             /* frequency map scale w0 (Ha) */
    int max_subspace_iters;    /* subspace iteration limit per frequency */
    int fixed_subspace_iters;  /* > 0: run exactly this many iterations per frequency */
    int n_atoms;               /* divides eps_c and the reported per-atom energy */
    int batch_systems;         /* Sternheimer systems in flight at once (0 = automatic; with
                                  block_cocg rounded down to whole groups, at least one) */
    int profile;               /* != 0: time every launch of the COCG kernels with CUDA events and
                                  count the grid points they process (filled into rpa_stats.prof_*) */
    int project_solution;      /* != 0: also remove the occupied components of every Sternheimer
                                  solution (x <- P_c x).  The same chi0 when the orbitals are exact
                                  eigenvectors of H; when V_loc differs from the potential the
                                  orbitals belong to, it is the response of the fixed occupied space
                                  (the function rpa_ec_gradient differentiates) */
    int z_chunks;              /* stencil work items per grid column along z (0 or 1 = whole columns);
                                  more chunks give more parallel items when few systems are in flight,
                                  at the price of re-reading a 6-plane overlap per chunk */
    int stencil_shape;         /* COCG kernels of the mixed form.  1..3: two kernels per iteration
                                  (direction update + stencil, then x/r update) with xy tiles and z
                                  marching: 1 = one grid column per thread, up to 640 threads per
                                  block; 2 = one column per thread, up to 320 threads, two blocks per
                                  SM; 3 = two columns per thread, up to 384 threads.  4 = one fused
                                  kernel per iteration, one block per system with whole xy planes in
                                  a shared-memory ring (grids whose nx*ny plane fits, about 1800
                                  points); where a plane does not fit, its cluster form (below); where
                                  neither fits, as 1.  5 = the fused kernel warp-specialised: producer
                                  threads form the next plane while consumer threads apply the
                                  stencil (planes of up to ~416 blocks of 2 x 2 points; else as 4).
                                  6 = the fused kernel's cluster form: the 2..8 blocks of a thread-
                                  block cluster split every plane into bands of row pairs and read
                                  the rows past their band from each other's shared memory, here
                                  with rings small enough for two blocks per SM (else as 4).
                                  0 = automatic: as 4.  rpa_autotune sets it.  The plain FP64 form
                                  always uses 1; periodic grids run 4 (even nx) or 1. */
    int independent_frequencies; /* != 0: every frequency starts from V0 instead of the subspace of
                                  the next higher frequency (no warm start, Algorithm 1 carries it);
                                  with fixed_subspace_iters = 1 E_c is then the Rayleigh-Ritz energy
                                  of the fixed subspace span(V0) at every frequency */
    int sq_order;              /* 0: E_c,m = (w_m/2pi) sum_i g(lambda_i) over the Rayleigh-Ritz values;
                                  N_o in 1..32: E_c,m = (w_m/2pi) Tr g(V^T chi~0 V) by Gauss spectral
                                  quadrature of order N_o (Lanczos from each basis vector, the paper's
                                  evaluation; exact for N_o >= N_r).  The Ritz values are returned
                                  either way.  rpa_ec_gradient requires 0 (it differentiates the
                                  Rayleigh-Ritz energy). */
    int contractions;          /* dense contractions of the chi0 application and the Rayleigh-Ritz
                                  step -- the Kronecker per-axis transforms of nu^1/2, the P_c
                                  coefficients and C = V^T R: 0 = automatic (tensor cores in the mixed
                                  form, FP64 in the plain form); 1 = FP64 on CUDA cores; 2 = tensor
                                  cores (tcgen05: in every k chunk of 64 each row of each operand is
                                  scaled by a power of two and cut into four integer pieces of at most
                                  8 bits; the ten products of pieces that matter accumulate exactly in
                                  FP32 and are combined in FP64; ~1e-8 relative); 3 = tensor cores
                                  except the Kronecker transforms.  The overlap R^T R, the rotation
                                  V = R L^-T, Cholesky, the eigensolve and rpa_coulomb_apply always
                                  use FP64. */
    int omega_first;           /* frequency range of this call (ascending index into the n_omega   */
    int omega_count;           /* Gauss-Legendre nodes): rpa_ec / rpa_ec_gradient evaluate only the
                                  frequencies omega_first .. omega_first + omega_count - 1 (count 0 =
                                  all) and report zero for the others (lambdas, ec_per_omega; E_c sums
                                  only the range).  With independent_frequencies set, the ranges of a
                                  partition of the frequencies give, summed, exactly the E_c of one
                                  call over all of them: frequency sharding across processes (the
                                  paper's frequencies are independent but for the warm start). */
    int periodic;              /* boundary conditions, fixed at rpa_setup (rpa_set_options rejects a
                                  change): 0 = zero values outside the box (Dirichlet); 1 = periodic
                                  in x, y and z (a bulk cell, the paper's Section "Results"): the
                                  stencil takes the periodic continuation of every grid function,
                                  and nu^p acts with the G = 0 mode removed (the constant function
                                  maps to zero: the neutralising background of a periodic cell). */
    int precondition;          /* 1: COCG preconditioned by M = (-1/2 L_h + s)^-1, s = mean(V_loc) -
                                  eps_n + i omega, applied through the Kronecker eigendecomposition
                                  of L_h (the paper's Laplacian-based preconditioning, Section
                                  "Implementation"): fewer iterations, each with three extra passes
                                  over the vectors.  Runs the split COCG kernels (stencil_shape 1..3;
                                  the fused kernels 4..6 stand in with 1).  Needs a plane's two
                                  complex copies and the x and y factors in one block's shared
                                  memory (FP32: planes up to ~80 x 80; FP64: ~64 x 64) and
                                  nz <= 96.  0 (default): plain COCG. */
    int block_cocg;            /* s in 1..16: the chi0 applications (rpa_apply_nuchi0, rpa_ec) and
                                  rpa_sternheimer_solve take the systems of one orbital s at a time
                                  (consecutive systems with the same orbital for the latter) and
                                  solve each group by block COCG, the paper's block variant of COCG
                                  (Section "Implementation"): X += P alpha, R -= Q alpha, P = R +
                                  P beta with s x s matrices alpha = (P^T A P)^-1 R^T R and beta =
                                  (R^T R)^-1 R'^T R' (unconjugated products), to the same per-system
                                  stopping rule, inside the same FP64 refinement for the mixed form.
                                  The block iterations restart from the true residual where an s x s
                                  matrix turns singular to working precision, and leave out columns
                                  already converged.  Not with precondition or project_solution;
                                  rpa_ec_gradient's adjoint solves stay single.  0 (default): off. */
} rpa_options;

#define RPA_PROF_SLOTS 8

typedef struct {
    long long sternheimer_solves;   /* systems solved */
    long long cocg_iterations;      /* COCG iterations summed over systems (inner ones for mixed) */
    long long refinement_steps;     /* FP64 residual evaluations summed over systems (mixed) */
    long long stencil_points;       /* grid points x stencil applications in COCG (work measure) */
    int subspace_iterations[64];    /* per frequency, ascending omega */
    double omegas[64];              /* frequency nodes, ascending */
    double weights[64];             /* frequency weights */
    double ms_coulomb;              /* device time per phase (CUDA events), milliseconds */
    double ms_projection;           /* P_c coefficients and right-hand sides */
    double ms_cocg;                 /* Sternheimer solves including refinement */
    double ms_density;              /* drho accumulation */
    double ms_subspace;             /* Gram/projection, Cholesky, Rayleigh-Ritz, rotation */
    double ms_total;
    int worst_status;               /* largest per-system COCG status seen */
    /* with rpa_options.profile: one entry per COCG kernel (name, launches, summed device time,
     * grid points processed, algorithmic bytes moved = points x the kernel's bytes per point) */
    int prof_count;
    char prof_name[RPA_PROF_SLOTS][32];
    long long prof_launches[RPA_PROF_SLOTS];
    double prof_ms[RPA_PROF_SLOTS];
    double prof_points[RPA_PROF_SLOTS];
    double prof_bytes[RPA_PROF_SLOTS];
    long long launches;             /* kernels launched by the call (all of the library's kernels) */
    long long near_breakdowns;      /* mixed form: FP32 COCG steps at which r^T r or p^T A p fell to
                                       rounding level (the recurrence restarted or the inner solve
                                       ended early), summed over systems */
    long long host_syncs;           /* host synchronisations of the call: with CUDA graphs and without
                                       profile, one per subspace iteration (its read-back of the Ritz
                                       values), plus the adjoint's per-frequency steps */
} rpa_stats;

/* Fill *opt with defaults: FP64, tol 1e-8, maxit 20000, max_refine 20, inner_tol 1e-4,
 * eps_c 1e-5, n_omega 8, omega0 1, max_subspace_iters 100, fixed 0, n_atoms 1, batch 0,
 * profile 0, project_solution 0, z_chunks 0, stencil_shape 0 (automatic), independent_frequencies 0,
 * sq_order 0, contractions 0 (automatic), omega_first 0, omega_count 0 (all frequencies), periodic 0,
 * precondition 0. */
void rpa_default_options(rpa_options *opt);

/* Create a context for one system (the inputs of Algorithm 1: H, P = the orbitals, eps).
 * nx,ny,nz >= 1, h > 0, fd_order must be 12.  vloc_dev: N_d doubles.  psi_dev: N_d x n_s
 * column-major, l2-orthonormal columns.  eps_host: n_s doubles.  opt may be NULL
 * (defaults).  The library copies all inputs; the caller may free them on return.
 * The per-axis eigendecompositions of the Kronecker Coulomb operator are computed here. */
rpa_status rpa_setup(rpa_ctx **out, int nx, int ny, int nz, double h, int fd_order,
                     const double *vloc_dev, const double *psi_dev, const double *eps_host,
                     int n_s, const rpa_options *opt, void *stream);

/* Replace the context's options (tolerances, precision, frequency count ...). */
rpa_status rpa_set_options(rpa_ctx *ctx, const rpa_options *opt);

/* out = nu^power in for ncols columns (N_d x ncols, column-major), with
 * nu = 4 pi (-L_h)^{-1} (Poisson, Eq. 5) by the Kronecker-product formalism.  Any real
 * power is accepted (0.5 and 1 are the ones the method uses).  in and out may alias. */
rpa_status rpa_coulomb_apply(rpa_ctx *ctx, double power, const double *in_dev, double *out_dev,
                             int ncols, void *stream);

/* Solve nsys Sternheimer systems (H - eps_n + i omega) x_s = b_s (Eq. 9) by COCG, with n =
 * orbital_idx_host[s].  rhs_dev: N_d x nsys real right-hand sides.  project != 0 replaces
 * b_s by P_c b_s first (removes the occupied components, as the Galerkin initial guess
 * does); the equation then lives in the unoccupied space, and in the mixed form the stopping
 * test is on ||P_c (b - A x)|| and x is returned with its occupied components removed (to
 * FP64 rounding for tol < 1e-9, else to ~1e-9 of ||x||).  x_dev: N_d x nsys complex
 * (interleaved), written.  iters_dev/status_dev: nsys
 * ints on the device (iterations, per-system rpa_status), may be NULL.  Returns the worst
 * per-system status. */
rpa_status rpa_sternheimer_solve(rpa_ctx *ctx, double omega, const int *orbital_idx_host, int nsys,
                                 const double *rhs_dev, int project, double *x_dev,
                                 int *iters_dev, int *status_dev, void *stream);

/* R = nu^1/2 chi0(i omega) nu^1/2 V (symmetric = 1) or R = nu chi0(i omega) V (symmetric = 0)
 * for n_r columns (N_d x n_r, column-major).  One application of Algorithm 1's loop over
 * trial vectors: Coulomb half-apply, N_s x n_r Sternheimer solves, drho accumulation,
 * Coulomb half-apply.  V and R must not alias. */
rpa_status rpa_apply_nuchi0(rpa_ctx *ctx, double omega, const double *V_dev, double *R_dev, int n_r,
                            int symmetric, void *stream);

/* E_c by Algorithm 1 with Rayleigh-Ritz.  V0_dev: N_d x n_r starting vectors (need not be
 * orthonormal; they are orthonormalised through the Cholesky factor of V0^T V0).  Frequencies run from
 * the highest to the lowest, the subspace carried over.  Outputs (host, each may be NULL):
 * lambdas_host n_omega x n_r (row m = ascending Ritz values of the last iteration at the
 * m-th frequency, ascending omega); ec_host[0] = E_c (Ha), ec_host[1] = E_c / n_atoms;
 * ec_per_omega_host n_omega weighted contributions (w_m/2pi) sum_i g(lambda_i); stats. */
rpa_status rpa_ec(rpa_ctx *ctx, int n_r, const double *V0_dev, double *lambdas_host, double *ec_host,
                  double *ec_per_omega_host, rpa_stats *stats, void *stream);

/* dE_c/dV_loc(r) at fixed occupied orbitals and eigenvalues (the adjoint of rpa_ec).
 *
 * Runs rpa_ec with project_solution on, then at every frequency takes the Ritz pairs
 * (lambda_i, y_i) of the last subspace iteration and, by Hellmann-Feynman,
 *     dE_c/dV(r) = (1/2pi) sum_m w_m sum_i g'(lambda_i) d lambda_i/dV(r),  g'(x) = -x/(1-x),
 *     d lambda_i/dV(r) = (4/h^3) Re sum_n x_{n,i}(r)^2,
 * where x_{n,i} is the projected Sternheimer solution for dV = nu^1/2 y_i.  The Sternheimer
 * operator is complex symmetric, so the adjoint solve is the forward solve; the solutions are
 * recomputed (one extra Sternheimer pass per frequency), never stored.  This derivative is not
 * in the paper; it differentiates the method's E_c (Eq. 10).
 * grad_dev: N_d doubles (written).  V_out_dev: N_d x n_r, the final subspace (may be NULL).
 * The other arguments and outputs are those of rpa_ec. */
rpa_status rpa_ec_gradient(rpa_ctx *ctx, int n_r, const double *V0_dev, double *grad_dev, double *V_out_dev,
                           double *lambdas_host, double *ec_host, double *ec_per_omega_host, rpa_stats *stats,
                           void *stream);

/* Uneven batch: several independent systems, one context each, in one set of launches.
 *
 * rpa_apply_nuchi0_batch does for every context k what rpa_apply_nuchi0 does for one: R_dev[k] =
 * nu^1/2 chi0(i omega) nu^1/2 V_dev[k] (symmetric != 0) or nu chi0 V_dev[k], ncols[k] columns in
 * [0, 1024] (N_d x ncols[k], column-major, no aliasing).  The Sternheimer systems (Eq. 9) of all the
 * contexts run together in the block COCG kernels (block size max(1, block_cocg)): one launch per
 * kernel and iteration for the whole batch, every system with its own grid, operator, orbitals and
 * stopping rule.  The contexts must be distinct, on one device, with equal prec, tol, inner_tol,
 * maxit, max_refine and block_cocg, and without precondition or project_solution (else
 * RPA_ERR_INVALID); the first context's batch_systems and profile apply.  Synchronises `stream`.
 * Returns the worst per-system status. */
rpa_status rpa_apply_nuchi0_batch(rpa_ctx *const *ctxs, int n, double omega, const double *const *V_dev,
                                  double *const *R_dev, const int *ncols, int symmetric, void *stream);

/* rpa_ec for every context k of a batch: n_r[k] trial vectors V0_dev[k], each context with its own
 * frequencies, subspace iteration and stopping rule (Algorithm 1), and the chi0 applications of
 * the contexts still iterating run together as in rpa_apply_nuchi0_batch (one host thread per
 * context drives its subspace iteration; the last to reach its chi0 application runs the batch,
 * and a context that has finished drops out of later batches).  Outputs per context, each pointer
 * may be NULL: lambdas_host[k] (n_omega x n_r[k] Ritz values), ec_host[2k] and ec_host[2k + 1]
 * (E_c and E_c per atom), ec_per_omega_host[k] (n_omega values), stats[k] (the launches and
 * synchronisations of a batch are counted in
 * the context whose thread ran it).  Same conditions on the contexts as rpa_apply_nuchi0_batch.
 * Work starts after what is already queued on `stream`; the call returns when every context is
 * done.  Returns the worst per-system status; a failure of one context fails the call with that
 * context's message. */
rpa_status rpa_ec_batch(rpa_ctx *const *ctxs, int n, const int *n_r, const double *const *V0_dev,
                        double *const *lambdas_host, double *ec_host, double *const *ec_per_omega_host,
                        rpa_stats *stats, void *stream);

/* Size of the fixed device scratch array used by rpa_coulomb_apply_noalloc (64 MiB).  Every
 * GPU on which the library is loaded keeps this much memory reserved until the process exits. */
#define RPA_STATIC_SCRATCH_BYTES (64u << 20)

/* rpa_coulomb_apply without any device allocation inside the call.
 *
 * For callers that cannot let the library call cudaMalloc at that point: applications whose
 * device memory is already fully reserved by their own allocator or memory pool, so that a
 * fresh cudaMalloc would fail (or would fragment the pool they manage).  The paper has no
 * counterpart of this entry point; it computes exactly what rpa_coulomb_apply computes.
 *
 * Scratch: the library's own statically sized device array of RPA_STATIC_SCRATCH_BYTES.  A call
 * needs 2 * ncols * N_d + N_d doubles (each of the two column blocks rounded up to 256 bytes);
 * larger requests return RPA_ERR_INVALID with a message and do nothing.  The caller still
 * provides in_dev and out_dev (N_d x ncols, column-major; they may alias).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current, and later calls reuse it.  The context's device must be the current
 * device.  Like rpa_coulomb_apply, the call synchronises `stream` before
 * it returns.
 * All calls share the one array and it keeps the last call's contents; every scratch word is
 * written before it is read, so nothing needs clearing.  Calls whose work overlaps on the GPU
 * (different streams or threads, any context) race on the array and give wrong results:
 * serialise them. */
rpa_status rpa_coulomb_apply_noalloc(rpa_ctx *ctx, double power, const double *in_dev, double *out_dev,
                                     int ncols, void *stream);

/* Number of configurations rpa_autotune times. */
#define RPA_AUTOTUNE_CANDIDATES 9

/* Autotuner: times one application of nu^1/2 chi0(i omega) nu^1/2 to the n_r columns of V_dev
 * for each candidate configuration of the COCG kernels and keeps the fastest for this context by
 * setting its stencil_shape and z_chunks options.  Candidates 0..5: the two-kernel variants
 * stencil_shape = 1, 2, 3 (columns per thread and threads per block, i.e. the xy tile shape)
 * crossed with one or two z chunks per column, index 2 (stencil_shape - 1) + (z_chunks - 1);
 * candidate 6: the fused single-pass kernel (stencil_shape 4); candidate 7: its warp-specialised
 * form (stencil_shape 5); candidate 8: its cluster form with two blocks per SM (stencil_shape 6).
 * The plain FP64 form has one configuration (candidate 0).  times_ms_host (may be NULL) receives RPA_AUTOTUNE_CANDIDATES
 * timings, -1 for a candidate that does not apply; *chosen_host (may be NULL) the index of the
 * chosen one.  The context's results do not depend on the choice beyond rounding. */
rpa_status rpa_autotune(rpa_ctx *ctx, double omega, const double *V_dev, int n_r, int *chosen_host,
                        double *times_ms_host, void *stream);

/* Release the context and its device workspaces.  NULL is ignored. */
void rpa_destroy(rpa_ctx *ctx);

/* Message of the last failing call on this thread ("" if none). */
const char *rpa_last_error(void);

/* Library version string. */
const char *rpa_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RPA_H */
