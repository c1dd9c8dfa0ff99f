/*
 * htd.h -- C ABI of the GB300 time-domain Helmholtz preconditioner library
 * (libhtd.so).  Method: C. C. Stolk, "A time-domain preconditioner for the
 * Helmholtz equation" (arXiv 2006.16861).
 *
 * The library solves H U = F for the damped Helmholtz operator of Sec. 1,
 *     -Delta U - (omega/c)^2 U + i omega R U = F,   zero Dirichlet data,
 * discretised on a regular grid by the compact-stencil cell form of App. A
 * (9 points in 2-D, 27 in 3-D).  The preconditioner is Table 1
 * (TimeDomainPreconditioner): T n_P steps of the frequency-adapted leapfrog
 * recurrence I_acd (Def. of I_acd) driven by the windowed time-harmonic
 * forcing (Def. approx_solver), used inside restarted GMRES (Sec. 2.4).
 * Options (htd_options) select the exact operator S_T instead of Table 1's
 * read-out, a windowed projection read-out, the backward-differences scheme
 * I_abd of Sec. 6, FP32 or FP64 recurrence, the stencil, and right-hand-side
 * batching; htd_grad and htd_grad_td return misfit gradients.
 *
 * Conventions (all entry points):
 *  - Plain C types only.  Pointers named *_dev are CUDA device pointers on the
 *    handle's device; pointers named *_host are host pointers.
 *  - Grid: n[a] unknown nodes per axis at x_i = i h (a < ndim), zero ghost
 *    ring at i = -1 and i = n[a].  Node arrays have prod(n[a]) entries,
 *    row-major with the last axis fastest.  Cell arrays have prod(n[a] + 1)
 *    entries; cell a (lower-corner node index a = -1 .. n-1 per axis) is stored
 *    at a + 1, its wave speed applies on [a h, (a+1) h].
 *  - Complex vectors are complex128, interleaved (re, im), node layout.
 *  - The caller owns every buffer it passes; the handle owns its internal
 *    device workspaces (allocated by htd_create, freed by htd_destroy).
 *  - Every call returns an htd_status.  No exception or abort crosses the ABI.
 *    On error, outputs are unspecified; the handle stays usable except after
 *    HTD_ERR_CUDA.
 *  - A handle is not thread-safe.  Work is enqueued on the given CUDA stream
 *    (NULL = the legacy default stream); calls that return host values
 *    (htd_gmres_solve, htd_residual_norm) synchronise that stream.
 */
#ifndef HTD_H
#define HTD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct htd_ctx *htd_handle;
typedef struct htd_batch_s *htd_batch;

typedef enum {
    HTD_OK = 0,
    HTD_ERR_ARG = 1,            /* invalid argument (null pointer, bad size or option) */
    HTD_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    HTD_ERR_OOM = 3,            /* device allocation failed */
    HTD_ERR_UNSTABLE = 4,       /* requested n_P violates the CFL bound, or not a multiple of 4 */
    HTD_ERR_NONFINITE = 5,      /* NaN/Inf in an input or a residual norm */
    HTD_ERR_NOT_CONVERGED = 6,  /* iteration cap reached before the tolerance */
    HTD_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up */
    HTD_ERR_SIZE = 8            /* problem larger than a fixed-size buffer allows */
} htd_status;

enum { HTD_FP64 = 0, HTD_MIXED = 1 };            /* recurrence precision */
enum { HTD_MODE_TABLE1 = 0, HTD_MODE_EXACT = 1, HTD_MODE_PROJECT = 2 }; /* preconditioner form */
enum { HTD_ACD = 0, HTD_ABD = 1 };               /* time integrator */
enum { HTD_DAMP_NODE = 0, HTD_DAMP_CELL = 1 };   /* form of Im H */
enum { HTD_FGMRES = 0, HTD_LEFT_GMRES = 1 };     /* Krylov method */
enum { HTD_STENCIL_Q1MIX = 0, HTD_STENCIL_FD5 = 1, HTD_STENCIL_FAMILY = 2 };
enum { HTD_BC_DIRICHLET = 0 };

typedef struct {
    int ndim;          /* 2 or 3 */
    int64_t n[3];      /* unknown nodes per axis, n[a] >= 1 for a < ndim */
    double h;          /* grid spacing > 0 */
} htd_grid;

typedef struct {
    int precision;     /* HTD_FP64: recurrence in double; HTD_MIXED: recurrence in
                          float, Krylov, residual and Givens in double */
    int mode;          /* HTD_MODE_TABLE1: Table 1, one real run, U = u_{T n_P} +
                          i u_{(T-1/4) n_P}.  HTD_MODE_EXACT: S_T^acd F of
                          Def. approx_solver, two real runs (forcings F and -iF).
                          HTD_MODE_PROJECT (not in the paper): Table 1's run read
                          out by projection onto e^{-i omega t} over its last
                          proj_periods whole periods, U = (2/n_acc) sum_j
                          e^{-i 2 pi j/n_P} u_j, n_acc = proj_periods n_P, summed
                          with compensated (Kahan) additions in the recurrence
                          precision; like Table 1 only R-linear (use FGMRES) */
    int krylov;        /* HTD_FGMRES (flexible right preconditioning, default) or
                          HTD_LEFT_GMRES (left preconditioning, Sec. 2.4) */
    int T;             /* periods per preconditioner application, >= 1 */
    double rho;        /* window parameter in [0, 1]; 0 means a ramp over one
                          period (rho = 1/T), as in Sec. 5.1 */
    int nP;            /* time steps per period; 0 = smallest stable multiple of 4 */
    int stencil;       /* cell kernel of App. A (per Hamming distance s between two
                          corners of a cell: h^2 H_cell = S_s - (h k)^2 M_s).
                          HTD_STENCIL_Q1MIX: Q1 element stiffness, half consistent
                          Q1 mass + half lumped mass (the stand-in for the paper's
                          optimized coefficients, which it does not print).
                          HTD_STENCIL_FD5: edge stiffness and lumped mass (the
                          5-/7-point operator of Sec. 3.1 for constant k).
                          HTD_STENCIL_FAMILY: S = stencil_gamma S(Q1) +
                          (1 - stencil_gamma) S(FD5), M = stencil_a M(consistent Q1)
                          + (1 - stencil_a) M(lumped); (a, gamma) = (0.5, 1) is
                          Q1MIX and (0, 0) is FD5.  Every member has a PSD cell
                          stiffness and 0 <= cell mass <= 2^-d I, the properties
                          the bounds of App. A use */
    int restart;       /* Krylov restart length m for htd_gmres_solve, 1..64 */
    int max_rhs;       /* right-hand sides one batched application may carry for
                          this handle (htd_batch_*), 1..256; 0 means 1.  The
                          per-rhs device arrays (two states, two forcing planes,
                          and two more states for the blocked 2-D kernel) are
                          allocated max_rhs times */
    int proj_periods;  /* HTD_MODE_PROJECT: whole periods projected, 1..T; 0
                          means 1.  Adds four planes per right-hand side */
    int integrator;    /* HTD_ACD: frequency-adapted central differences
                          (Def. of I_acd, default).  HTD_ABD: frequency-adapted
                          backward differences (Def. of I_abd, Sec. 6), explicit
                          also for non-diagonal damping, with its omega and n_P
                          from Sec. 6.1 (stricter: it needs lambda_max(Im H)
                          below about 2 k_max^2) */
    int damping;       /* HTD_DAMP_NODE: (Im H)_ii = omega_phys R_i (Eq. damped
                          Helmholtz equation, diagonal).  HTD_DAMP_CELL: Im H =
                          omega_phys sum over cells of R_cell times the cell mass
                          of App. A (non-diagonal; R_cell the mean of R over the
                          cell's grid corners); needs HTD_ABD */
    double stencil_a;  /* HTD_STENCIL_FAMILY: weight of the consistent Q1 mass, in
                          [0, 1] (default 0.5) */
    double stencil_gamma; /* HTD_STENCIL_FAMILY: weight of the Q1 element stiffness,
                          in [0, 1] (default 1) */
    int tblock;        /* recurrence steps per launch of the 2-D FP32 kernel:
                          0 = chosen at create by timing the one-step kernel,
                          the blocked configurations and the resident-grid
                          kernel (default), 1 = one step per launch, 4 or 8 =
                          temporally blocked with that depth.  Ignored for
                          other precisions, dimensions and I_abd */
    /* Kernel selection.  The defaults (all 0) let htd_create pick by timing;
       the other values restrict or force a kernel variant, for tuning and for
       tests that compare variants.  Every variant computes the same recurrence;
       the tests hold them to bit-identity or to the FP32 tolerance. */
    int tb_rows;       /* blocked 2-D kernel: rows per thread the create-time
                          tuner may pick (6, 8, 10, 12 or 20); 0 = any */
    int tb_form;       /* blocked 2-D kernel: HTD_TB_ANY (tuned), HTD_TB_COLUMN
                          (one column per thread), HTD_TB_PAIR (two columns per
                          thread in paired FP32 instructions, d in registers),
                          HTD_TB_PAIR_SD (pairs, d staged in shared memory),
                          HTD_TB_RESIDENT (the resident-grid kernel whenever
                          the handle qualifies, else as HTD_TB_ANY).  The
                          resident-grid kernel runs a whole run in one
                          cooperative launch: the grid is cut into at most one
                          tile per SM, each CTA keeps its tile's states and
                          coefficients in shared memory for all T n_P steps
                          and swaps edge values with its neighbours through
                          global memory every step (in projection mode it
                          also accumulates the window's states).  It
                          qualifies for a handle with max_rhs 1 and a grid
                          whose tiles fit the shared memory of one SM (about
                          1.1 M nodes on 152 SMs with the FP32 recurrence,
                          0.5 M with FP64); the FP64 recurrence times it
                          against the one-step kernel when tblock is 0.  A
                          handle that joins a batch leaves it for its tuned
                          blocked configuration */
    int s3_kernel;     /* 3-D FP32 step kernel: HTD_S3_PAIR (TMA-streamed z
                          planes, node pairs; default), HTD_S3_ZMARCH (one step
                          per launch, register z-march), HTD_S3_NODE_32x8,
                          HTD_S3_NODE_64x4, HTD_S3_NODE_128x2 (TMA-streamed, one
                          node per thread on that column tile) */
    int s3_stages;     /* ring stages of the streamed 3-D kernels: 0 = 5, or 4, 6, 7 */
    int s3_zchunk;     /* z planes per CTA of the streamed 3-D kernels: 0 = chosen
                          at create by timing, else that many */
    int s3_rhs_per_cta; /* right-hand sides per CTA of the streamed 3-D pair kernel
                          for handles with max_rhs > 1: 0 = 1 or 2, whichever is
                          faster when timed at create with every rhs slot active;
                          1; 2 (one CTA streams a column tile for two rhs slots,
                          loading q*kappa and d once and computing every stencil
                          coefficient once for both; 4 ring stages) */
    int launch;        /* bit flags: HTD_LAUNCH_NO_OVERLAP (consecutive step
                          launches do not overlap by programmatic dependent
                          launch), HTD_LAUNCH_NO_GRAPH (steps launched one by one
                          instead of replaying a captured CUDA graph),
                          HTD_LAUNCH_NO_GROUP (in a batch, this handle keeps its
                          own step sequence instead of joining the persistent
                          launch of the batch's 2-D handles) */
    long long wait_limit_ns; /* bound of the device-side waits between the row
                          groups of the blocked 2-D kernel; 0 = 1 s.  A wait that
                          runs out makes the call return HTD_ERR_TIMEOUT (see
                          htd_set_wait_limit) */
} htd_options;

enum { HTD_TB_ANY = 0, HTD_TB_COLUMN = 1, HTD_TB_PAIR = 2, HTD_TB_PAIR_SD = 3,
       HTD_TB_RESIDENT = 4 };
enum { HTD_S3_PAIR = 0, HTD_S3_ZMARCH = 1, HTD_S3_NODE_32x8 = 2, HTD_S3_NODE_64x4 = 3,
       HTD_S3_NODE_128x2 = 4 };
enum { HTD_LAUNCH_NO_OVERLAP = 1, HTD_LAUNCH_NO_GRAPH = 2, HTD_LAUNCH_NO_GROUP = 4 };

typedef struct {
    int iterations;           /* Arnoldi steps taken */
    int restarts;             /* Krylov cycles started */
    int precond_applies;      /* preconditioner applications */
    int converged;            /* 1 if the true relative residual <= tol */
    long long steps;          /* recurrence steps run (all applications) */
    double rel_res_true;      /* ||F - H U|| / ||F|| at exit (FP64) */
    double rel_res_est;       /* last Arnoldi residual estimate */
    double ms_total;          /* wall time of the call, host clock */
    double ms_precond;        /* device time inside preconditioner applications,
                                 CUDA events on the call's stream */
    long long launches;       /* kernels launched by the call (graph nodes counted) */
    int reorth;               /* Arnoldi steps that needed the second Gram-Schmidt
                                 pass (||w|| fell below 1/sqrt(2) of itself in the
                                 first) */
    int hist_len;
    double hist[256];         /* Arnoldi estimate after each step (first 256) */
} htd_solve_info;

/* Fill *opt with the defaults: FP64, TABLE1, FGMRES, T = 10, rho = 0.25,
 * nP = 0 (automatic), Q1MIX stencil, restart 20, max_rhs 1, proj_periods 1,
 * HTD_ACD, HTD_DAMP_NODE, stencil_a 0.5, stencil_gamma 1, tblock 0, and 0 for
 * every kernel-selection field. */
void htd_default_options(htd_options *opt);

/*
 * Create a solver for one problem on the current CUDA device.
 *   grid        grid description (see conventions).
 *   c_cell_host wave speed per cell, prod(n+1) doubles > 0, host memory.
 *   R_node_host damping per node, prod(n) doubles >= 0, host memory
 *               ((Im H)_ii = omega_phys * R_i, Sec. 1 damped Helmholtz eq.).
 *   omega_phys  physical angular frequency > 0.
 *   bc          HTD_BC_DIRICHLET (the only boundary condition).
 *   opt         options (NULL = defaults).
 * Parameter selection (Sec. 2.2 with the bounds of App. A): omega = k_max =
 * max omega_phys / c; lambda_max(Re H) bounded by the constant-coefficient
 * symbol at k_min; n_P the smallest multiple of 4 with
 * sin^2(pi / n_P) < omega^2 / lambda_max(A) (Eq. define_Deltat_ImH_diagonal);
 * dt = 2 pi / (omega n_P); alpha, beta of Eq. define_alpha_beta.
 * Errors: HTD_ERR_ARG, HTD_ERR_UNSTABLE (bad requested nP), HTD_ERR_NONFINITE,
 * HTD_ERR_OOM, HTD_ERR_CUDA.  *out is set only on success.
 */
htd_status htd_create(const htd_grid *grid, const double *c_cell_host,
                      const double *R_node_host, double omega_phys, int bc,
                      const htd_options *opt, htd_handle *out);

/* Release the handle and its device memory.  NULL is accepted. */
htd_status htd_destroy(htd_handle h);

/* Parameters selected for a problem (see htd_plan). */
typedef struct {
    double k_min, k_max;     /* min / max of omega_phys / c over cells */
    double omega_c;          /* computational omega (= k_max, App. A bound; with
                                HTD_ABD the Sec. 6.1 value, above k_max) */
    double lam_max_reH;      /* upper bound for lambda_max(Re H) */
    double lam_max_A;        /* lam_max_reH + omega_c^2 */
    double dt, alpha, beta;  /* time step, Eq. define_alpha_beta */
    double rho;              /* window parameter used (1/T when 0 was asked) */
    int nP;                  /* time steps per period */
    int T;                   /* periods */
    long long steps;         /* recurrence steps per real run: T * nP */
    int steps_per_launch;    /* recurrence steps per kernel launch (temporal
                                blocking; 1 = one step per launch; T * nP for the
                                resident-grid kernel; 0 in htd_plan, which does not
                                look at the device) */
    int tile[3];             /* owned tile (x, y) of the blocked or resident-grid
                                2-D step kernel and its columns per thread (1, or
                                2: node pairs in paired FP32 instructions), or
                                column tile and z chunk of the streamed 3-D one; 0
                                if unused */
    int ctas_per_sm;         /* resident CTAs per SM of that kernel */
    int waves;               /* waves of CTAs per launch of that kernel */
    int step_kernel;         /* recurrence kernel in use: 0 one step per launch
                                (gather / z-march), 1 temporally blocked 2-D
                                (TMA tiles), 2 TMA-streamed 3-D, 3 one-step
                                backward differences (HTD_ABD), 4 resident-grid
                                2-D (one launch per run); -1 in htd_plan */
    int rhs_per_cta;         /* right-hand sides one CTA of the step kernel works
                                on (1 or 2); 0 in htd_plan */
} htd_params;

/*
 * Host-only parameter selection (no CUDA call, no allocation): validates the
 * arguments exactly as htd_create does and fills *out.  Same arguments as
 * htd_create; errors HTD_ERR_ARG, HTD_ERR_UNSTABLE, HTD_ERR_NONFINITE.
 */
htd_status htd_plan(const htd_grid *grid, const double *c_cell_host, const double *R_node_host,
                    double omega_phys, int bc, const htd_options *opt, htd_params *out);

/* Parameters chosen by htd_create. */
htd_status htd_get_params(htd_handle h, htd_params *out);

/*
 * U = P F: one application of the preconditioner (Table 1 or the exact S_T,
 * per the handle's mode), in the handle's recurrence precision.
 *   F_dev, U_dev  complex128[N] device vectors; they may not overlap.
 *   stream        cudaStream_t (as void*), NULL = default stream.
 * Asynchronous: returns after enqueueing.
 */
htd_status htd_apply_precond(htd_handle h, const void *F_dev, void *U_dev, void *stream);

/*
 * Y = H X, the true operator in complex128 (App. A cell form plus
 * i omega_phys R on the diagonal).  X_dev, Y_dev complex128[N], no overlap.
 * Asynchronous.
 */
htd_status htd_apply_H(htd_handle h, const void *X_dev, void *Y_dev, void *stream);

/*
 * r = F - H U (complex128) and *rel = ||r|| / ||F|| (host double; 0 if F = 0).
 * r_dev may be NULL (the residual is then kept in handle workspace).
 * Synchronises the stream.  HTD_ERR_NONFINITE if the norm is not finite.
 */
htd_status htd_residual_norm(htd_handle h, const void *F_dev, const void *U_dev,
                             void *r_dev, double *rel, void *stream);

/*
 * Allocation-free variant of htd_residual_norm: *rel = ||F - H U|| / ||F||
 * (0 if F = 0), with the residual vector and the reduction partial sums kept
 * in a fixed buffer inside the library instead of the handle's workspace.
 * The paper has no counterpart.  It is for callers that cannot let a library
 * allocate device memory when they call it: applications whose device memory
 * is handed out by their own pool (a framework's caching allocator that has
 * reserved most of the GPU, so that a library's cudaMalloc would fail or
 * fragment it), and solve loops that cannot afford the device-wide
 * synchronisation that cudaMalloc/cudaFree may imply while other streams run.
 * The call makes no cudaMalloc, cudaFree or other allocating call.
 *   Limit: N = prod(n) <= HTD_NOALLOC_MAX_NODES; larger problems return
 *   HTD_ERR_SIZE and compute nothing.
 *   The buffer is a static __device__ array of HTD_NOALLOC_MAX_NODES complex128
 *   values plus 2 * 1216 + 2 partial sums (about 4.04 MiB); every GPU that
 *   loads the library holds it until the process exits.
 *   All calls on a device share the one buffer and it keeps the last call's
 *   contents; every value a call reads is written by that call first, so no
 *   clearing is needed.  Calls whose GPU work overlaps (several streams or
 *   host threads at once) race on the buffer: serialise them.
 *   The first call on each device looks up the buffer's device address
 *   (cudaGetSymbolAddress, which may load the module); the address is cached
 *   per device and looked up again after a call that returned HTD_ERR_CUDA
 *   (after cudaDeviceReset, make such a call or expect stale addresses until
 *   one fails).  The handle's device must be current.
 *   The call returns a host value, so it copies the two sums to the host and
 *   synchronises `stream`: it cannot be recorded into a CUDA graph, and
 *   `stream` must not be capturing.
 *   A CUDA error already pending when the call starts is reported as
 *   HTD_ERR_CUDA and left pending; nothing is launched then.
 * Errors: HTD_ERR_ARG, HTD_ERR_SIZE, HTD_ERR_NONFINITE, HTD_ERR_CUDA.
 */
#define HTD_NOALLOC_MAX_NODES 262144
htd_status htd_residual_norm_noalloc(htd_handle h, const void *F_dev, const void *U_dev,
                                     double *rel, void *stream);

/*
 * Solve H U = F with restarted GMRES(m), m = opt.restart (Sec. 2.4): flexible
 * right preconditioning (default) or left preconditioning, preconditioner P of
 * the handle, Arnoldi by classical Gram-Schmidt in FP64 with a second
 * (re-orthogonalisation) pass in the steps where the first pass removed more
 * than half of the new vector's squared norm ("twice is enough"), Givens least
 * squares on the host.
 *   F_dev      complex128[N] right-hand side (device).
 *   U_dev      complex128[N] (device): initial guess on entry, solution on exit.
 *   tol        stop when the Arnoldi estimate and the true relative residual
 *              ||F - H U|| / ||F|| are <= tol.  tol <= 0: run exactly
 *              max_iters Arnoldi steps with no early exit (returns HTD_OK).
 *   max_iters  cap on Arnoldi steps (>= 0).
 *   info       optional statistics (NULL allowed).
 * Synchronises the stream.  HTD_ERR_NOT_CONVERGED if the cap is reached
 * first (U holds the last iterate), HTD_ERR_NONFINITE on NaN/Inf.
 */
htd_status htd_gmres_solve(htd_handle h, const void *F_dev, void *U_dev, double tol,
                           int max_iters, void *stream, htd_solve_info *info);

/*
 * Same as htd_gmres_solve with host buffers: copies F_host (complex128[N],
 * pinned memory recommended) and the initial guess U_host to handle-owned
 * device buffers, solves, and copies the solution back to U_host.
 */
htd_status htd_gmres_solve_host(htd_handle h, const void *F_host, void *U_host, double tol,
                                int max_iters, void *stream, htd_solve_info *info);

/*
 * Receiver misfit and its gradient (adjoint-state method for H U = F):
 *   J = 1/2 sum_s || P U_s - d_s ||^2,   H U_s = F_s  (s < nsrc),
 * P the sampling at the nodes rec_idx.  H is complex symmetric, so the adjoint
 * field is mu_s = H^{-1} conj(r_s), r_s = P^T (P U_s - d_s), and
 *   dJ/dm_alpha = omega_phys^2 sum_s Re sum_{beta,gamma in cell alpha}
 *                 mu_{s,beta} M_{|beta-gamma|} U_{s,gamma}     (m = c^{-2} per cell),
 *   dJ/dR_i     = omega_phys sum_s Im(mu_{s,i} U_{s,i})        (R per node),
 * from the dependence of H on m (through -(omega/c)^2 in Sec. 1's damped
 * Helmholtz equation, discretised with the cell mass M of App. A) and on R
 * ((Im H)_ii = omega_phys R_i).  The paper has no gradient; this is the
 * standard adjoint of its problem statement.  Both solves use
 * htd_gmres_solve with the handle's preconditioner and tolerance `tol`.
 *   F_dev       complex128[nsrc][N] right-hand sides (device).
 *   rec_idx_host int64[nrec] receiver node indices in [0, N) (host).
 *   d_dev       complex128[nsrc][nrec] data (device; may be NULL if nrec = 0).
 *   grad_m_dev  double[prod(n+1)] (device, cell order of c_cell) or NULL.
 *   grad_R_dev  double[N] (device) or NULL.  Both NULL: misfit only (no
 *               adjoint solves).  Outputs are overwritten, not accumulated.
 *   misfit      host double, J.
 *   info        optional: iterations, applications, steps and times summed
 *               over all solves; rel_res_true is the worst of them.
 * Synchronises the stream.  Errors: HTD_ERR_ARG (bad sizes or indices), the
 * solve errors of htd_gmres_solve (HTD_ERR_NOT_CONVERGED stops at the first
 * solve that fails), HTD_ERR_CUDA, HTD_ERR_OOM (first call allocates the
 * handle's gradient workspace: three complex vectors and the receiver buffers).
 */
htd_status htd_grad(htd_handle h, int nsrc, const void *F_dev, int nrec,
                    const int64_t *rec_idx_host, const void *d_dev, double tol, int max_iters,
                    void *grad_m_dev, void *grad_R_dev, double *misfit, void *stream,
                    htd_solve_info *info);

/*
 * Misfit of the preconditioner's own approximate solution and its gradient
 * through the recurrence (reverse-time discrete adjoint with checkpoints; the
 * paper has no gradient, this differentiates its Table 1 / S_T^acd run):
 *   J = 1/2 sum_s sum_r |(P F_s)[rec_r] - d_{s,r}|^2,
 * P = one application of the handle's preconditioner (mode TABLE1 or EXACT).
 * Each real run of P is the recurrence (1 + L/2) u_{j+1} = (2 - K) u_j -
 * (1 - L/2) u_{j-1} + g_j (Def. of I_acd); its adjoint is the same recurrence
 * run backwards in time with -dJ/du_k injected at the read-out steps, and
 *   dJ/dm_alpha = -(dt^2/alpha) omega_phys^2 sum_k lam_k^T M_alpha u_{k-1},
 *   dJ/dR_i     = (beta dt omega_phys / (2 alpha omega)) sum_k lam_{k,i} (u_{k,i} - u_{k-2,i}),
 * with m = c^{-2} per cell, M_alpha the cell mass of App. A, and omega, dt,
 * n_P held at the handle's values (they are chosen from c at create).
 *   nsrc, F_dev, nrec, rec_idx_host, d_dev, grad_m_dev, grad_R_dev, misfit:
 *               as in htd_grad.
 *   checkpoint_every  C: (u_j, u_{j-1}) are kept every C steps and each
 *               segment is recomputed once on the way back; 0 chooses
 *               ceil(sqrt(2 T n_P)).  Device memory 2 ceil(T n_P / C) + C + 6
 *               state planes (the handle keeps the largest workspace asked).
 * The states and multipliers are in the handle's recurrence precision (FP32 in
 * mixed mode), the gradient sums in FP64.  Synchronises the stream.  Errors:
 * HTD_ERR_ARG (bad sizes or indices, mode PROJECT), HTD_ERR_OOM, HTD_ERR_CUDA,
 * HTD_ERR_NONFINITE, HTD_ERR_TIMEOUT.
 */
htd_status htd_grad_td(htd_handle h, int nsrc, const void *F_dev, int nrec,
                       const int64_t *rec_idx_host, const void *d_dev, int checkpoint_every,
                       void *grad_m_dev, void *grad_R_dev, double *misfit, void *stream);

/*
 * Batches.  The paper solves one right-hand side of one problem at a time
 * (Sec. 5); these calls run many independent systems together: several
 * right-hand sides of one handle (sharing its coefficient arrays) and several
 * handles of different sizes and step counts.  Each system is the problem of
 * htd_gmres_solve; only the scheduling differs.
 *
 * htd_batch_create: ninst distinct handles on the current device, instance i
 * carrying nrhs[i] right-hand sides (1 <= nrhs[i] <= its max_rhs option).  The
 * batch owns the Krylov workspace of every system (2 m + 2 complex vectors of
 * the instance's N each); the handles stay owned by the caller and must
 * outlive the batch.  Errors: HTD_ERR_ARG (null, repeated handle, bad nrhs,
 * a LEFT_GMRES handle), HTD_ERR_OOM, HTD_ERR_CUDA.
 */
htd_status htd_batch_create(int ninst, const htd_handle *handles, const int *nrhs,
                            htd_batch *out);
htd_status htd_batch_destroy(htd_batch b);

/*
 * U_i[r] = P_i F_i[r] for every system: F_dev[i], U_dev[i] are complex128
 * [nrhs[i]][N_i] (device, distinct).  One application of every preconditioner
 * (both runs in mode EXACT) as one CUDA-graph launch per run, in the batch's
 * current form (htd_batch_desc): every handle's captured step sequence as a
 * child graph, each step kernel covering all right-hand sides of its handle;
 * or, when at least two handles are 2-D with FP32 recurrence (I_acd, Table 1
 * or exact read-out), those handles as ONE persistent launch -- a queue of
 * tasks (level = 8 steps, handle, rhs slot, tile) of the blocked kernel's
 * work, ordered by level, each tile starting a level once its 3 x 3 tile
 * neighbourhood has finished the previous one -- beside the other handles'
 * sequences.  Every output equals the handle's own htd_apply_precond bit for
 * bit in either form.  Asynchronous on stream.
 */
htd_status htd_batch_apply_precond(htd_batch b, const void *const *F_dev, void *const *U_dev,
                                   void *stream);

/*
 * Solve every system H_i U_i[r] = F_i[r] by FGMRES(m_i) with the handle's
 * preconditioner, all systems in lockstep: each Arnoldi step applies the
 * preconditioners of all systems still running in one graph launch, then
 * runs the FP64 Krylov updates of each system; a system leaves when its true
 * relative residual <= tol (or after max_iters steps) and its slots go idle.
 * U_dev[i] holds the initial guesses on entry.  info: sum(nrhs) entries in
 * instance-major order, or NULL.  Synchronises the stream.  Returns
 * HTD_ERR_NOT_CONVERGED if any system did not converge (all are still
 * solved as far as they went), HTD_ERR_NONFINITE, HTD_ERR_TIMEOUT,
 * HTD_ERR_CUDA.
 */
htd_status htd_batch_gmres_solve(htd_batch b, const void *const *F_dev, void *const *U_dev,
                                 double tol, int max_iters, void *stream, htd_solve_info *info);

/*
 * Test and tuning hooks.
 *
 * htd_set_wait_limit: bound (ns) of the device-side waits between the row
 * groups of the blocked 2-D kernel for this handle's later launches (0 = 1 s,
 * the default); the copy-completion waits keep their fixed 1 s bound so that
 * no CTA exits with a copy in flight.  stall_test != 0 makes the first such
 * wait of every CTA wait on a barrier that nothing arrives on, so it runs out
 * after limit_ns: the kernel records the timeout, skips its remaining waits,
 * finishes, and the call that ran it returns HTD_ERR_TIMEOUT (its outputs are
 * then unspecified).  This exercises the timeout path without a fault or a
 * hang.  Synchronous.  Errors: HTD_ERR_ARG (limit_ns < 0), HTD_ERR_CUDA.
 */
htd_status htd_set_wait_limit(htd_handle h, long long limit_ns, int stall_test);

/*
 * Host-side allocation-failure injection for tests: the library's device
 * allocations numbered 0 .. after-1 from this call on succeed, allocation
 * number `after` fails as if the device were out of memory (the calling entry
 * point returns HTD_ERR_OOM after releasing what it took), later ones succeed.
 * after < 0 switches it off.  Process-wide, not thread-safe.
 */
void htd_test_fail_alloc(long long after);

/* How a batch runs its preconditioner applications (filled after the first
 * application or solve; zeros before).  A batch with a group of 2-D handles
 * has two forms of a run that give the same bits: every handle's own step
 * sequence as a child graph (plain), or the group's persistent launch beside
 * the other handles' sequences (group).  The first two rounds of a solve run
 * one form each; the one with the smaller device time per point update is
 * kept for the batch from then on. */
typedef struct {
    int instances;           /* handles in the batch */
    int systems;             /* (handle, right-hand side) pairs */
    int grouped;             /* 2-D FP32 handles the persistent launch would run
                                (0: no group) */
    int group_ctas;          /* persistent CTAs of that launch */
    long long group_tasks;   /* its tasks per run: levels x tiles x rhs slots */
    int group_steps_per_task; /* recurrence steps per task (the blocked depth B) */
    int form;                /* 0 not yet decided, 1 plain, 2 group */
    double ns_per_update_plain; /* device time per point update of the timed round
                                   in each form (0 until timed) */
    double ns_per_update_group;
} htd_batch_desc;
htd_status htd_batch_describe(htd_batch b, htd_batch_desc *out);

/* Set the batch's form: 0 = decide by timing the first rounds of the next
 * solve (the default), 1 = every handle's own step sequence, 2 = the group's
 * persistent launch (HTD_ERR_ARG if the batch has no group).  Either form
 * gives the same bits. */
htd_status htd_batch_set_form(htd_batch b, int form);

/* Static string for a status code. */
const char *htd_status_string(htd_status s);

#ifdef __cplusplus
}
#endif

#endif /* HTD_H */
