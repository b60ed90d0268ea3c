/*
 * cmg.h — C ABI of the collective multigrid solver for the saddle-point
 * optimality system S x = f of a linear-quadratic elliptic optimal control
 * problem under uncertainty (Ciaramella, Nobile, Vanzan, arXiv 2302.13680).
 *
 * Discrete problem (Sec. 2, full-space optimality system, in its symmetric
 * scaling; generic block form Eq. (2)): on the unit square with n x n
 * interior nodes, h = 1/(n+1), N samples of the diffusion field,
 *     (h^2/N) y_j + A_j p_j        = f_y,j      (state-row block, C_j = M/N)
 *     nu h^2 u   - h^2 sum_j p_j   = f_u        (control row,  G = nu M, D_j = -M)
 *     A_j y_j    - h^2 u           = f_p,j      (adjoint-row block, E_j = -M)
 * with M = h^2 I (lumped mass) and A_j the integrated 5-point stiffness of
 * -div(kappa_j grad), face coefficients the harmonic mean of the two nodal
 * values, zero Dirichlet data.  kappa_j(x,y) = exp(amp sum_k xi_jk
 * sin(k pi x) sin(pi y) / k), the sine-mode stand-in for the log-normal
 * field of Eq. (15).
 *
 * Vector layout (all levels): a full-space vector is three arrays
 *     y [n*n][N]   state, node-major, sample index fastest
 *     u [n*n]      control
 *     p [n*n][N]   adjoint
 * node index i = iy*n + ix (x fastest).  Level 0 is the finest grid; level
 * l has n_l = (n_{l-1} - 1)/2 nodes per side.
 *
 * Memory and streams: every vector argument is a DEVICE pointer, borrowed
 * for the duration of the call, 16-byte aligned.  The handle owns the
 * device memory it allocates (hierarchy coefficients, coarse factors,
 * work vectors) and frees it in cmg_destroy.  All work is enqueued on the
 * stream given to cmg_create; calls return after enqueueing except those
 * documented as synchronising (cmg_solve, cmg_norm).
 *
 * Errors: every call returns a cmg_status; on failure a message is kept in
 * the handle (cmg_last_error).  No call aborts the process; a failed call
 * leaves the handle usable.  Invalid sizes, null pointers or a level out of
 * range give CMG_ERR_INVALID_ARG before anything is enqueued.
 */
#ifndef CMG_H_
#define CMG_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cmg_handle cmg_handle;

typedef enum {
  CMG_OK = 0,
  CMG_ERR_INVALID_ARG = 1,
  CMG_ERR_CUDA = 2,
  CMG_ERR_OOM = 3,
  CMG_ERR_NOT_CONVERGED = 4,
  CMG_ERR_NONFINITE = 5,
  CMG_ERR_TIMEOUT = 6,
  CMG_ERR_UNSUPPORTED = 7
} cmg_status;

enum { CMG_SMOOTH_RBGS = 0, CMG_SMOOTH_JACOBI = 1 };
enum { CMG_FP64 = 0, CMG_FP32 = 1 };
enum { CMG_METHOD_CYCLE = 0, CMG_METHOD_FGMRES = 1 };
enum { CMG_COARSE_AVERAGED = 0, CMG_COARSE_NODAL = 1, CMG_COARSE_GALERKIN = 2 };

/* Problem description (Sec. 2; field of Sec. 3.2). */
typedef struct {
  int n;            /* interior nodes per side, finest grid: 2^L - 1, 3 <= n <= 4095 */
  int N;            /* samples (quadrature nodes, Monte Carlo weights 1/N): 1 <= N <= 256, or up
                       to 512 when N is a multiple of 4 (a lane holds at most 8 chunks of the
                       16-byte, or for other N 1-sample, vectors: see cmg_sample_map); other N
                       return CMG_ERR_UNSUPPORTED */
  int K;            /* field modes, 0 <= K <= 64 */
  double nu;        /* control cost nu > 0 */
  double amp;       /* field amplitude */
  int coarsest_n;   /* nodes per side of the coarsest grid: 1, 3 or 7 (<= n) */
  int coarse_coeff; /* face coefficients of the rediscretised coarse grids:
                       CMG_COARSE_AVERAGED (default): each coarse face averages the finer
                       grid's faces, harmonic along it (two fine faces in series) and
                       arithmetic across it (weights 1/4, 1/2, 1/4);
                       CMG_COARSE_NODAL: the field is sampled at each grid's own nodes and
                       faces are harmonic means of the two endpoint values;
                       CMG_COARSE_GALERKIN: no rediscretisation -- the coarse matrices are the
                       Galerkin products S_l = P^T S_{l-1} P of Sec. 3 (the operator of the
                       paper's experiments): 9-point A_j and a 9-point mass M_l on every grid
                       below the finest.  Cycles in FP64 or FP32 with the control updated
                       (freeze_u = 0; FP32 with ctl32 = 0: on the 9-point grids the per-sample
                       arithmetic is FP32 on FP32 copies of the FP64 Galerkin planes, the control
                       row and the coarsest elimination FP64; tail_n is ignored);
                       CMG_SMOOTH_JACOBI as on any grid, and CMG_SMOOTH_RBGS = red-black
                       Gauss-Seidel on the finest grid and four-colour (iy mod 2, ix mod 2)
                       collective Gauss-Seidel on the 9-point grids; distributed control only
                       (ctl_box all zero), no semismooth Newton and no batches: those return
                       CMG_ERR_UNSUPPORTED */
  double ctl_box[4]; /* local control (Sec. 3.1 after Eq. (13); the local-control test case of
                       Sec. 3.2): the closed region [x0, x1] x [y0, y1] = {ctl_box[0], ctl_box[1],
                       ctl_box[2], ctl_box[3]} inside the unit square.  Nodes of every grid inside
                       it carry a control basis function; at the others u_i = 0, the control row
                       is absent (its residual is zero) and the smoothers use Eq. (14) with
                       u_i = 0.  All four zero = control everywhere (distributed control).
                       Other values with x1 <= x0 or y1 <= y0, or outside [0, 1]:
                       CMG_ERR_INVALID_ARG. */
} cmg_problem;

/* Cycle options (Algorithm 1). */
typedef struct {
  int smoother;     /* CMG_SMOOTH_RBGS (red = (ix+iy) even first) | CMG_SMOOTH_JACOBI */
  double theta;     /* damping of collective Jacobi, Eq. (11); the paper uses 0.5 */
  int n1, n2;       /* pre- and post-smoothing sweeps */
  int gamma;        /* recursive calls per level: 1 = V-cycle, 2 = W-cycle */
  int precision;    /* arithmetic of the cycle: CMG_FP64, or CMG_FP32: FP32 vectors and
                       FP32 per-sample arithmetic in the smoothing, residual and transfer
                       sweeps, while the per-node Schur scalar of Eq. (13) (the sum over
                       samples for u_i, 1/sigma_i and u_i) is FP64 from the lanes' FP32
                       partial sums, 1/sigma_i being computed in FP64 from the FP32 faces;
                       the coarsest solve takes the per-sample products A_j^{-1} f in FP32
                       and the sums over samples and the control Schur solve in FP64 */
  int tail_n;       /* grids with at most tail_n nodes per side (and the coarsest solve)
                       run as ONE launch of a thread-block cluster whose phases are
                       separated by cluster barriers; 0 = one launch per step on every
                       grid (faster inside the refinement graph on GB300).  The same
                       algorithm either way, results equal up to rounding (the
                       per-launch path computes the residual after red-black
                       pre-smoothing at colour 0 only and fuses the prolongation into
                       the next half-sweep).  Ignored (one launch per step) when N
                       needs more than 4 chunks per lane or the coarsest grid is 7 x 7. */
  int freeze_u;     /* 1: keep the control fixed: each node solves only its state and
                       adjoint rows for the current u_i (Eq. (14) with u_i given instead
                       of zero) and the coarse corrections of u are zero.  Cycles then
                       solve the 2N PDEs for a given control (used to complete a
                       predicted control into a consistent initial iterate); 0 = the
                       collective smoother of Eq. (13). */
  int ctl32;        /* CMG_FP32 cycles only: 1 = the per-node Schur scalar of Eq. (13) in
                       FP32 as well (sum over samples, 1/sigma_i rounded to FP32, u_i):
                       an all-FP32 option, off by default (0); ignored by FP64 cycles. */
} cmg_cycle;

/* Solve statistics filled by cmg_solve. */
typedef struct {
  int iters;        /* outer iterations: cycles (CMG_METHOD_CYCLE) or FGMRES steps */
  int cycles;       /* fine-grid cycles applied */
  double relres0;   /* ||W (f - S x0)||_2 / ||W f||_2 (see cmg_solve) */
  double relres;    /* final ||W (f - S x)||_2 / ||W f||_2, recomputed from x */
} cmg_stats;

/* ---- hierarchy ------------------------------------------------------- */

/* Build the grid hierarchy n, (n-1)/2, ..., coarsest_n and, on the device,
 * the nodal field, face coefficients, diag(A_j) and the Schur denominators
 * of Eq. (13) on every grid (coarse operators rediscretised, Sec. 3, with
 * faces per prob->coarse_coeff), plus
 * the coarsest-grid factors used by the direct solve of Algorithm 1.
 * xi_host: host array [N][K] of field coefficients (copied).  stream: a
 * cudaStream_t (NULL = legacy default stream).  On success *out owns all
 * device memory it allocated.  Synchronises the stream once.
 * Errors: INVALID_ARG (sizes), UNSUPPORTED (N above the kernels' limit),
 * OOM, CUDA. */
cmg_status cmg_create(const cmg_problem* prob, const double* xi_host, void* stream,
                      cmg_handle** out);

/* Recompute every level's coefficients and the coarsest factors from new
 * field coefficients xi_dev (DEVICE [N][K]), same sizes.  Enqueued only. */
cmg_status cmg_set_samples(cmg_handle* h, const double* xi_dev);

void cmg_destroy(cmg_handle* h);
const char* cmg_last_error(const cmg_handle* h);
int cmg_num_levels(const cmg_handle* h);
int cmg_level_n(const cmg_handle* h, int level);   /* -1 if out of range */

/* Mean over samples of log kappa_j at the finest grid's n*n interior nodes
 * (DEVICE out[n*n], FP64); an input of the warm-start network. */
cmg_status cmg_mean_log_kappa(cmg_handle* h, double* out);

/* ---- right-hand side -------------------------------------------------- */

/* f = ((h^2/N) y_d, 0, h^2 f_src) on the finest grid (right side of the
 * full-space system, Sec. 2).  yd, fsrc: device [n*n] (fsrc may be NULL
 * for zero forcing). */
cmg_status cmg_rhs(cmg_handle* h, const double* yd, const double* fsrc,
                   double* fy, double* fu, double* fp);

/* ---- level operators (FP64; *_f32 take float vectors) ------------------ */

/* r = f - S x on grid `level` (Eq. (2) with this problem's blocks).  With
 * fy, fu, fp all NULL the call computes r = S x (operator apply).  On a
 * CMG_COARSE_GALERKIN handle S on the grids below the finest is the Galerkin
 * product P^T S P (9-point blocks); the _f32 variant reads FP32 copies of
 * its planes and forms the control row's sums in FP64. */
cmg_status cmg_residual(cmg_handle* h, int level,
                        const double* y, const double* u, const double* p,
                        const double* fy, const double* fu, const double* fp,
                        double* ry, double* ru, double* rp);
cmg_status cmg_residual_f32(cmg_handle* h, int level,
                            const float* y, const float* u, const float* p,
                            const float* fy, const float* fu, const float* fp,
                            float* ry, float* ru, float* rp);

/* `sweeps` collective smoothing steps in place on grid `level`:
 * red-black collective Gauss-Seidel (each node solves its reduced system
 * Eq. (12) by Eq. (13) with current neighbour values; all red nodes, then
 * all black) or damped collective Jacobi Eq. (11).  Only opts->smoother and
 * opts->theta are read.  On the Galerkin grids of a CMG_COARSE_GALERKIN
 * handle CMG_SMOOTH_RBGS sweeps in four colours (iy mod 2, ix mod 2). */
cmg_status cmg_smooth(cmg_handle* h, int level, const cmg_cycle* opts, int sweeps,
                      double* y, double* u, double* p,
                      const double* fy, const double* fu, const double* fp);
cmg_status cmg_smooth_f32(cmg_handle* h, int level, const cmg_cycle* opts, int sweeps,
                          float* y, float* u, float* p,
                          const float* fy, const float* fu, const float* fp);

/* Coarse right side c = P^T r from grid `level` to `level`+1, P the
 * bilinear prolongation (Algorithm 1, restriction step; weights 1, 1/2,
 * 1/4, i.e. four times the 1/16 full-weighting stencil because every block
 * row is in integrated form). */
cmg_status cmg_restrict(cmg_handle* h, int level,
                        const double* ry, const double* ru, const double* rp,
                        double* cy, double* cu, double* cp);
cmg_status cmg_restrict_f32(cmg_handle* h, int level,
                            const float* ry, const float* ru, const float* rp,
                            float* cy, float* cu, float* cp);

/* x += P e: bilinear prolongation of the correction e on grid `level`+1
 * added to x on grid `level` (Algorithm 1, coarse correction step). */
cmg_status cmg_prolong_add(cmg_handle* h, int level,
                           const double* ey, const double* eu, const double* ep,
                           double* y, double* u, double* p);
cmg_status cmg_prolong_add_f32(cmg_handle* h, int level,
                               const float* ey, const float* eu, const float* ep,
                               float* y, float* u, float* p);

/* x = S^{-1} f on the coarsest grid (Algorithm 1, direct solver): the
 * per-sample PDE blocks are eliminated with precomputed A_j^{-1} and the
 * n_c^2 x n_c^2 Schur system for u is solved with its precomputed inverse.
 * Always computed in FP64 (the f32 variant converts on load and store).  On
 * a CMG_COARSE_GALERKIN handle the elimination carries the non-diagonal
 * Galerkin mass (x and f must not overlap). */
cmg_status cmg_coarse_solve(cmg_handle* h, const double* fy, const double* fu, const double* fp,
                            double* y, double* u, double* p);
cmg_status cmg_coarse_solve_f32(cmg_handle* h, const float* fy, const float* fu, const float* fp,
                                float* y, float* u, float* p);

/* ---- cycles and solves ------------------------------------------------ */

/* One cycle of Algorithm 1 on the finest grid, in place on x, for rhs f.
 * opts->precision must match the vector type (cmg_cycle_f32 for FP32). */
cmg_status cmg_cycle_apply(cmg_handle* h, const cmg_cycle* opts,
                           double* y, double* u, double* p,
                           const double* fy, const double* fu, const double* fp);
cmg_status cmg_cycle_apply_f32(cmg_handle* h, const cmg_cycle* opts,
                               float* y, float* u, float* p,
                               const float* fy, const float* fu, const float* fp);

/* Solve S x = f on the finest grid to ||W (f - S x)||_2 <= tol ||W f||_2,
 * x in/out (initial guess in, solution out), FP64 vectors.  This is the
 * relative unpreconditioned residual of Sec. 3.2 measured on the paper's
 * own form of the system (Sec. 2), whose state rows are N times the
 * symmetric ones used here: W = diag(N I, 1, 1) on the (y, u, p) rows.
 * (In the symmetric scaling the FP64 rounding floor of ||f - S x|| / ||f||
 * grows like N (n+1)^2 eps and lies above 1e-10 for n = 255, N = 64.)
 * method CMG_METHOD_CYCLE: repeated cycles (stationary iteration, Algorithm 1
 *   repeated); with opts->precision == CMG_FP32 it is iterative refinement
 *   with residual replacement: each step runs e = cycle_FP32(0; r), updates
 *   the FP32 residual recursively (r -= S e) and sums the corrections in
 *   FP32; an anchor adds the sum to x and recomputes r = f - S x in FP64
 *   once the recursive norm has dropped by 1e-3 since the last anchor, after
 *   8 steps, or at the tolerance, and the stopping test is made on that
 *   FP64 residual.  The environment variables CMG_ANCHOR_DROP (in (0, 1))
 *   and CMG_ANCHOR_MAX (1..1000), read at cmg_create, change the two limits.
 * method CMG_METHOD_FGMRES: right-preconditioned flexible GMRES(restart)
 *   on W S x = W f with one cycle (FP64 or FP32) applied to W^{-1} v as
 *   preconditioner; Arnoldi by classical Gram-Schmidt applied twice, all
 *   Krylov vectors FP64.
 * With CMG_FP32 and CMG_METHOD_CYCLE the refinement loop runs on the device
 * as one CUDA graph with a conditional while node (the host synchronises
 * once per solve); it runs eagerly, one synchronisation per outer
 * iteration, while a profiling window is open or when the environment held
 * CMG_GRAPHS=0 at cmg_create (the same kernels; for tools that replay
 * kernels one by one).  The other forms synchronise once per outer
 * iteration to test convergence.  Returns
 * CMG_ERR_NOT_CONVERGED if maxit is reached (x holds the last iterate),
 * CMG_ERR_NONFINITE if a residual norm is not finite. */
cmg_status cmg_solve(cmg_handle* h, const cmg_cycle* opts, int method, double tol,
                     int maxit, int restart,
                     const double* fy, const double* fu, const double* fp,
                     double* y, double* u, double* p, cmg_stats* stats);

/* L1 + box constrained problem (Sec. 4): minimise
 *   1/2 E[||y(u) - y_d||^2] + nu/2 ||u||^2 + beta ||u||_1  over  a <= u <= b
 * (the handle's field, samples and nu; forcing f = 0) by the globalised
 * semismooth Newton method of Algorithm 2: F(u) = 0 with the optimality map
 * of Sec. 4, active sets I+ u I-, each Newton system solved by cmg_solve
 * (opts, method; stopping at inner_tol, at most 200 cycles / iterations)
 * with the control row's coupling restricted to the active sets, a
 * backtracking line search on phi(u) = sqrt(F' M F) (sigma = 1e-4,
 * rho = 1/2), stop when phi <= tol or after maxit Newton steps.  Algorithm
 * 2's initial states y0, p0 for u0 come from one solve of the same system
 * with no control coupling.
 * yd [n*n]: target at the finest grid's nodes (DEVICE, 16-byte aligned);
 * u [n*n]: u0 in, control out; y, p [n*n][N]: states out (the adjoint in this
 * library's symmetric scaling, 1/N times the paper's).  All DEVICE pointers.
 * Requires a < 0 < b, beta >= 0, tol > 0, inner_tol > 0, opts->freeze_u = 0.
 * The handle's operators are back to the linear-quadratic problem on return.
 * Returns CMG_ERR_NOT_CONVERGED if phi > tol after maxit steps. */
typedef struct {
  int newton;        /* Newton steps taken */
  int inner_total;   /* cycles / FGMRES iterations over all linear solves (initial states included) */
  double merit0;     /* phi(u0) */
  double merit;      /* phi at return */
} cmg_ssn_stats;
cmg_status cmg_ssn_solve(cmg_handle* h, const cmg_cycle* opts, int method, double beta, double a, double b,
                         double tol, double inner_tol, int maxit, const double* yd, double* y, double* u,
                         double* p, cmg_ssn_stats* stats);

/* ||(y,u,p)||_2 over all (2N+1) n_l^2 entries of a level vector, written to
 * *out_host.  Synchronises. */
cmg_status cmg_norm(cmg_handle* h, int level, const double* y, const double* u,
                    const double* p, double* out_host);

/* Wait for all work enqueued on the handle's stream. */
cmg_status cmg_sync(cmg_handle* h);

/* ---- batches of independent instances ---------------------------------- */

typedef struct cmg_batch cmg_batch;

/* Create `count` independent instances (own grid size, samples, field,
 * nu), each as by cmg_create with prob[i] and xi_host[i] (host [N_i][K_i]),
 * all enqueueing on `stream`.  Errors as cmg_create (nothing is kept). */
cmg_status cmg_batch_create(const cmg_problem* probs, const double* const* xi_host, int count, void* stream,
                            cmg_batch** out);
void cmg_batch_destroy(cmg_batch* b);
const char* cmg_batch_last_error(const cmg_batch* b);
/* The i-th instance's handle (owned by the batch) for the level calls. */
cmg_handle* cmg_batch_instance(cmg_batch* b, int i);

/* Solve every instance to its own tolerance (as cmg_solve with
 * CMG_METHOD_CYCLE: each instance runs FP64 refinement around FP32 cycles of
 * Algorithm 1 and stops at its own tolerance or maxit, decided on the
 * device).  Arguments are HOST arrays of `count` DEVICE pointers (instance
 * i's vectors sized by its own n_i, N_i); stats: host array of `count`.
 * With opts->precision == CMG_FP32, two forms:
 *   CMG_BATCH_PERSISTENT (used when the options and instances allow it:
 *     red-black V-cycles with n1, n2 >= 1 and the control updated, averaged
 *     coarse grids, one coarsest size, N <= 128): the instances advance in
 *     lockstep, their grids aligned by depth from the finest.  Per cycle, ONE
 *     persistent cooperative launch per grid depth runs every instance's
 *     down-leg (pre-smoothing from zero, residual, restriction) phase by
 *     phase over a work list of (instance, warp of nodes) items with a
 *     grid-wide barrier between phases, one launch runs every coarsest
 *     solve (a CTA per instance), and one persistent launch per depth runs
 *     the up-legs; the refinement steps are one launch each for all
 *     instances.  Per-instance masks skip instances that have stopped.  The
 *     loop is one CUDA graph with a while node that runs while any instance
 *     iterates (eager, one synchronisation per iteration, while a profiling
 *     window is open or graphs are off).  A barrier wait that exceeds its
 *     poll limit (cmg_batch_set_wait_limit) aborts the solve with
 *     CMG_ERR_TIMEOUT and leaves the batch usable.
 *   CMG_BATCH_BRANCHES (otherwise): ONE graph launch in which every instance
 *     is an independent branch with its own device-side while node.
 * Graphs are captured on first use and reused while the pointers and
 * options stay the same.  With CMG_FP64 the instances are solved one after
 * another.  Returns CMG_ERR_NOT_CONVERGED if any instance missed its
 * tolerance (stats say which), CMG_ERR_NONFINITE if any norm is not finite. */
cmg_status cmg_batch_solve(cmg_batch* b, const cmg_cycle* opts, double tol, int maxit,
                           const double* const* fy, const double* const* fu, const double* const* fp,
                           double* const* y, double* const* u, double* const* p, cmg_stats* stats);

/* ---- launch-shape autotuning ------------------------------------------- */

/* Choose, per grid, the launch shape of the node kernels of `precision`
 * (CMG_FP64 or CMG_FP32): how many sample chunks one lane takes (1, 2 or 4,
 * which fixes how many lanes share a node) and, for CMG_FP32 with N a
 * multiple of 4, whether the red-black half-sweep stages its loads through
 * shared memory (CMG_TUNE_STAGED | 1 or 2 chunks), and for CMG_FP32 with N
 * even and at most 64 the layout with two samples per lane and N/2 lanes
 * (rounded up to a power of two) per node (CMG_TUNE_WIDE | 1), which applies
 * to every node kernel of that grid.  Each candidate is timed
 * with CUDA events on a few red+black sweeps on the handle's own
 * work vectors, three times in turn, and the one with the fastest median
 * time is kept in the handle.  chosen (host, may
 * be NULL) receives the target per grid (num_levels entries; the coarsest
 * is not tuned: 0).  Synchronises.  Numerical results do not depend on the
 * choice except for the order of the sample sums (rounding). */
cmg_status cmg_autotune(cmg_handle* h, int precision, int* chosen);
/* Set the per-grid targets directly (e.g. from a cache of earlier
 * cmg_autotune runs): num_levels entries of 0 (size heuristic), 1, 2 or 4,
 * and for CMG_FP32 also CMG_TUNE_STAGED | 1, CMG_TUNE_STAGED | 2 or
 * CMG_TUNE_WIDE | 1 (ignored where N is odd or above 64) or CMG_TUNE_FUSED |
 * 1, 2 or 4 or CMG_TUNE_TMA | 1, 2 or 4, each possibly with CMG_TUNE_UNFUSED; NULL resets all to 0.  Other values return
 * CMG_ERR_INVALID_ARG. */
#define CMG_TUNE_STAGED 16
#define CMG_TUNE_WIDE 32
/* FP32 flag, combinable with any FP32 target: on this grid the cycle adds
 * the prolonged coarse correction in its own pass and then runs the plain
 * post-smoothing half-sweeps, instead of fusing the prolongation into the
 * first of them (cmg_autotune times both and sets it where the pass is
 * faster). */
#define CMG_TUNE_UNFUSED 64
/* FP32 flag with 1, 2 or 4 chunks per lane: each red-black sweep on this
 * grid (colour 0, then colour 1; Eq. (13) per node) runs as one launch over
 * tiles of the grid, reading the old iterate from one buffer and writing
 * the new one to a second (allocated with the handle when N % 4 == 0), so
 * the faces, f and old values are read once per sweep instead of once per
 * half-sweep.  Sweeps run in pairs (into the second buffer and back); the
 * results equal the half-sweeps' bit for bit.  Ignored where the shape is
 * not covered (N % 4 != 0, a frozen control, fewer than two sweeps).  Set
 * by cmg_set_tuning only: cmg_autotune does not choose it (its tiles walk
 * their rows one after another, so a sweep that reads less, from the zero
 * iterate, takes as long as a full one). */
#define CMG_TUNE_FUSED 128
/* FP32 flag with 1, 2 or 4 chunks per lane (N % 4 == 0, N <= 256): the
 * plain red-black half-sweeps on this grid bring their operands into a ring
 * of shared-memory stages by TMA tensor loads that gather every other node
 * of a grid row (a segment of one colour's nodes, its neighbours in the
 * rows above and below, its left/right neighbours, its faces and right
 * sides); one producer thread per CTA issues them and consumer warps
 * update the nodes from there, so the bytes in flight are set by the ring,
 * not by registers.  The results equal the direct half-sweep's bit for
 * bit.  Ignored where the shape is not covered (frozen control, 16-byte
 * misaligned arrays); the zero-iterate and prolongation-fused sweeps keep
 * their direct kernels. */
#define CMG_TUNE_TMA 256
/* The TMA half-sweep (CMG_TUNE_TMA) bounds every wait on its shared-memory
 * barriers; a wait that runs out (never, unless a load or a warp fails to
 * complete) adds one to a process-wide counter and returns.  *count = that
 * counter for the current device (synchronises the device).
 * CMG_ERR_INVALID_ARG for a null pointer, CMG_ERR_CUDA if the read fails. */
cmg_status cmg_sweep_wait_timeouts(unsigned int* count);
/* The launch shape the node kernels use for N samples of elem_bytes (4 or 8)
 * over `items` nodes (0: as many lanes per node as allowed) with a tuning
 * target as above: *lanes_per_node (a power of two <= 32, consecutive lanes of
 * one warp), *vec_width (samples per vector load: 16 / elem_bytes when it
 * divides N, else 1; 2 for CMG_TUNE_WIDE in FP32) and *chunks_per_lane (a
 * power of two; lanes x chunks x width >= N).  Host arithmetic only (no
 * device call, no handle).  CMG_ERR_INVALID_ARG for N < 1, elem_bytes not 4
 * or 8, or a null output; CMG_ERR_UNSUPPORTED when the chunks per lane exceed
 * the kernels' limit of 8 (the outputs are still written). */
cmg_status cmg_sample_map(int N, int elem_bytes, long long items, int target, int* lanes_per_node, int* vec_width,
                          int* chunks_per_lane);
cmg_status cmg_set_tuning(cmg_handle* h, int precision, const int* spl_targets);

/* Forms of cmg_batch_solve for FP32 cycles. */
enum { CMG_BATCH_AUTO = 0, CMG_BATCH_PERSISTENT = 1, CMG_BATCH_BRANCHES = 2 };
/* Choose the form: CMG_BATCH_AUTO (the default: the branches, which solve
 * the 96-instance workload of n up to 255 and N in [16, 128] faster),
 * CMG_BATCH_PERSISTENT (cmg_batch_solve returns CMG_ERR_UNSUPPORTED where it
 * is not supported) or CMG_BATCH_BRANCHES. */
cmg_status cmg_batch_set_form(cmg_batch* b, int form);
/* The form the last FP32 cmg_batch_solve used (0 before any). */
int cmg_batch_form(const cmg_batch* b);
/* Persistent form, per grid depth: each leg (down or up) runs either as the
 * persistent kernel (one cooperative launch, barriers between phases) or as
 * one ordinary launch per phase and map class (no barrier; every SM's warps
 * resident).  CMG_BATCH_LEGS_BY_WORK (default): the persistent kernel where
 * a depth has fewer than 19,456 warp items (152 SMs x 32 warps x 4), one
 * launch per phase elsewhere; CMG_BATCH_LEGS_PERSISTENT / _PHASES: that form
 * at every depth.  Takes effect on the next solve. */
enum { CMG_BATCH_LEGS_BY_WORK = -1, CMG_BATCH_LEGS_PERSISTENT = 0, CMG_BATCH_LEGS_PHASES = 1 };
cmg_status cmg_batch_set_legs(cmg_batch* b, int legs);
/* Polls per grid-wide barrier wait of the persistent form before the solve
 * is abandoned with CMG_ERR_TIMEOUT (0 = the default, 2^26 polls of at
 * least 64 ns, several seconds).  Takes effect on the next solve. */
cmg_status cmg_batch_set_wait_limit(cmg_batch* b, long long polls);

/* cmg_autotune on every instance of a batch (the batch graph is re-captured
 * on the next solve). */
cmg_status cmg_batch_autotune(cmg_batch* b, int precision);

/* ---- learned warm start: network kernels --------------------------------- */

/* C = A B^T (+ bias[N]) (then max(., 0) if relu) on the 5th-generation
 * tensor cores: A [M][K] and B [N][K] BF16 row-major (K contiguous, row
 * strides lda, ldb >= K), FP32 accumulation in tensor memory; C32 [M][ldc]
 * FP32 and/or C16 [M][ldc] BF16 outputs (either may be NULL).  K, lda and
 * ldb must be multiples of 8; A, B 16-byte aligned.  Operands are loaded
 * by TMA (tensor maps made per call); with the environment variable
 * CMG_GEMM_TMA=0, or if no tensor map can be made, by cp.async instead
 * (same results).  status (DEVICE int) is set to 1 if a tensor-core
 * completion wait exceeded its limit (the output is then incomplete); it is
 * never cleared by the call.  Enqueued on `stream`.  Used for the
 * convolution layers of the warm-start network (not part of the paper). */
cmg_status cmg_nn_gemm_bf16(const void* A, long long lda, const void* B, long long ldb, int M, int N, int K,
                            const float* bias, int relu, float* C32, void* C16, int ldc, int* status,
                            void* stream);

/* Layer kernels (activations NHWC BF16 [B][H][W][C]; weights [Cout][9 Cin]
 * BF16, column t*Cin + c for tap t = 3 dy + dx; all DEVICE pointers,
 * enqueued on `stream`; CMG_ERR_INVALID_ARG on null pointers or sizes out
 * of range, nothing enqueued):
 *   im2col      3x3 patches [B*H*W][9C] (transposed = 1: [9C][B*H*W]), zero
 *               outside the image; C a multiple of 8;
 *   col2im      data gradient dX from patch gradients dcol [B*H*W][9C] FP32;
 *   transpose   BF16 [R][Cc] -> [Cc][R];
 *   relu_bwd    dz = dy where y > 0 else 0;
 *   avgpool     2x2 mean (backward = 1: spread dY/4 over [B][H][W][C]);
 *   upsample_add  Y = nearest 2x upsampling of X [B][H/2][W/2][C] plus S;
 *   upsample_bwd  dX [B][H][W][C] = sum over each 2x2 block of dY;
 *   add, to_bf16, sum_slices (fixed-order sum of split-K partials), colsum
 *               (per-channel sums, bias gradients);
 *   mse         masked mean squared error on the interior m x m of [B][S][S]
 *               FP32 images: BF16 gradient and per-CTA partial sums;
 *   adamw       AdamW step on FP32 master weights, BF16 copy refreshed;
 *   pack_input / pack_target / unpack_output  between solver grids
 *               ([B][n*n] FP64) and S x S network images. */
/* Poll limit of the TMA kernel's waits for operands and accumulators
 * (process-wide; 0 = the default of 2^22 polls).  A wait that runs out sets
 * the call's status word to 1 and the CTA stops issuing work; it still
 * drains the tensor-core operations and copies it has in flight (those
 * waits keep the default limit), frees its tensor memory and returns, so the
 * next call runs normally.  A tiny limit makes every call give up: a way to
 * exercise that path.  Takes effect for calls enqueued after it. */
cmg_status cmg_nn_set_wait_limit(long long polls);
/* 3x3 convolution with zero padding 1 as an implicit GEMM on the tensor
 * cores: Y[p][co] = relu?(bias[co] + sum over taps t = 3 dy + dx and channels
 * c of X[b][y + dy - 1][x + dx - 1][c] Wt[co][t C + c]) for output pixel
 * p = (b, y, x); X NHWC BF16 [B][H][W][C], Wt [Cout][9 C] BF16 (both 16-byte
 * aligned), bias FP32 [Cout] or NULL, Y [B H W][Cout] BF16, all device
 * pointers.  The tensor cores read X directly through a TMA im2col map (no
 * im2col matrix in memory); the result equals cmg_nn_im2col followed by
 * cmg_nn_gemm_bf16 bit for bit.  Covers C a multiple of 32 (per K step of
 * 64, one tensor-map load of 64 channels of a tap, or two of 32) and C = 8,
 * 16, 24 (one load per 8 channels of a tap); returns CMG_ERR_UNSUPPORTED,
 * with nothing enqueued, for other C, Cout > 64, where no tensor map can be
 * made or with CMG_GEMM_TMA=0 (use im2col + GEMM then).  status as for cmg_nn_gemm_bf16.
 * Enqueued on `stream`. */
cmg_status cmg_nn_conv3x3_bf16(const void* X, int B, int H, int W, int C, const void* Wt, int Cout,
                               const float* bias, int relu, void* Y, int* status, void* stream);
/* Split-K form of cmg_nn_gemm_bf16 for long reductions (weight gradients):
 * slice z of ksplit reads columns [z Kslice, (z+1) Kslice) of A and B and
 * writes the FP32 partial product to partials + z*M*ldc (sum the slices
 * with cmg_nn_sum_slices). */
cmg_status cmg_nn_gemm_bf16_splitk(const void* A, long long lda, const void* B, long long ldb, int M, int N,
                                   int Kslice, int ksplit, float* partials, int ldc, int* status, void* stream);
/*   outer       out[p][c] = a[p] w[c] (data gradient of a 1x1 convolution to one channel). */
cmg_status cmg_nn_outer(const void* a, const float* w, void* out, long long P, int C, void* stream);
cmg_status cmg_nn_im2col(const void* X, void* col, int B, int H, int W, int C, int transposed, void* stream);
cmg_status cmg_nn_col2im(const float* dcol, void* dX, int B, int H, int W, int C, void* stream);
cmg_status cmg_nn_transpose(const void* in, void* out, long long R, long long Cc, void* stream);
/* Weights of the data-gradient convolution of a 3x3 layer: Wf [C][9 Cout]
 * with Wf[c][t Cout + co] = W[co][(8 - t) C + c] (W [Cout][9 C]); then
 * cmg_nn_conv3x3_bf16(dZ, ..., C = Cout, Wf, Cout = C, no bias, no ReLU)
 * gives the gradient of the layer's input, the col2im of dZ W. */
cmg_status cmg_nn_flip3x3(const void* W, void* Wf, int Cout, int C, void* stream);
cmg_status cmg_nn_relu_bwd(const void* y, const void* dy, void* dz, long long n, void* stream);
cmg_status cmg_nn_avgpool(const void* X, void* Y, int B, int H, int W, int C, int backward, void* stream);
cmg_status cmg_nn_upsample_add(const void* X, const void* S, void* Y, int B, int H, int W, int C, void* stream);
cmg_status cmg_nn_upsample_bwd(const void* dY, void* dX, int B, int H, int W, int C, void* stream);
cmg_status cmg_nn_add(const void* a, const void* b, void* out, long long n, void* stream);
cmg_status cmg_nn_to_bf16(const float* in, void* out, long long n, void* stream);
cmg_status cmg_nn_sum_slices(const float* part, int slices, float* out, long long n, void* stream);
cmg_status cmg_nn_colsum(const void* in, long long P, int C, float* out, void* stream);
cmg_status cmg_nn_mse(const float* pred, const float* tgt, int B, int S, int m, void* grad, float* partial,
                      int max_partials, int* used_partials, void* stream);
cmg_status cmg_nn_adamw(float* w, const float* g, float* m1, float* m2, void* w16, long long n, float lr,
                        float b1, float b2, float eps, float wd, int step, void* stream);
cmg_status cmg_nn_pack_input(const double* f0, const double* f1, int B, int n, int S, int Cp, float s0,
                             float s1, void* X, void* stream);
cmg_status cmg_nn_unpack_output(const float* img, int B, int n, int S, double scale, double* out,
                                void* stream);
cmg_status cmg_nn_pack_target(const double* u, int B, int n, int S, double scale, float* img, void* stream);

/* ---- Neumann boundary control ---------------------------------------------- */

/* The control problem of Sec. 2 with the control acting as a Neumann
 * condition on Gamma = (0,1) x {0} (the boundary-control test case of
 * Sec. 3.2), solved by collective multigrid with Galerkin coarse operators
 * (Sec. 3) and damped collective Jacobi (Eq. (11); each node's block by
 * Eq. (13) on Gamma and Eq. (14) elsewhere), all FP64.
 *
 * Grid l has n_l interior columns (x = (ix+1) h, Dirichlet at x = 0, 1) and
 * n_l + 1 rows (y = r h, row 0 on Gamma, Dirichlet at y = 1): (n_l + 1) n_l
 * nodes, node r n_l + ix.  Vectors: y, p [(n_l+1) n_l][N] (sample fastest),
 * u [n_l] on the row-0 nodes.  System (symmetric scaling):
 *     (M/N) y_j + A_j p_j = f_y,j;  G u - B^T sum_j p_j = f_u;  A_j y_j - B u = f_p,j
 * with, on the finest grid, A_j the dual-cell 5-point stiffness (harmonic-
 * mean faces; the x-faces of row 0 halved and no south face there), lumped
 * M = h^2 (h^2/2 on row 0), G = nu h I and B = h I on Gamma; coarse blocks
 * P^T S P with P bilinear in x and, in y, keeping row 0 on Gamma (fine row
 * 2R = coarse row R).  Pointers are DEVICE, 16-byte aligned, borrowed for
 * the call; work is enqueued on the handle's stream (cmg_bnd_rhs and
 * cmg_bnd_solve synchronise).  Errors as for cmg_handle. */
typedef struct cmg_bnd cmg_bnd;
/* n = 2^L - 1 columns (rows n + 1), N samples (<= 1024), K field modes
 * (xi_host [N][K], host), coarsest_n 1, 3 or 7 (<= n).  Builds the field,
 * the finest blocks, every Galerkin coarse block, the Jacobi diagonals and
 * the coarsest factors; synchronises once.  INVALID_ARG, UNSUPPORTED (the
 * coarsest factors above 200 KB of shared memory), OOM, CUDA. */
cmg_status cmg_bnd_create(int n, int N, int K, double nu, double amp, int coarsest_n, const double* xi_host,
                          void* stream, cmg_bnd** out);
void cmg_bnd_destroy(cmg_bnd* h);
const char* cmg_bnd_last_error(const cmg_bnd* h);
int cmg_bnd_num_levels(const cmg_bnd* h);
int cmg_bnd_level_n(const cmg_bnd* h, int level);   /* columns of grid `level`, -1 if out of range */
/* f = ((M y_d)/N, 0, M f_src) on the finest grid; yd, fsrc [(n+1) n] (fsrc
 * may be NULL: zero). */
cmg_status cmg_bnd_rhs(cmg_bnd* h, const double* yd, const double* fsrc, double* fy, double* fu, double* fp);
/* r = f - S_l x (r = S_l x when fy, fu, fp are all NULL) on grid `level`. */
cmg_status cmg_bnd_residual(cmg_bnd* h, int level, const double* y, const double* u, const double* p,
                            const double* fy, const double* fu, const double* fp, double* ry, double* ru,
                            double* rp);
/* `sweeps` damped collective Jacobi steps x += theta S~^{-1} (f - S x), theta in (0, 1]. */
cmg_status cmg_bnd_smooth(cmg_bnd* h, int level, double theta, int sweeps, double* y, double* u, double* p,
                          const double* fy, const double* fu, const double* fp);
/* c = P^T r from grid `level` to `level`+1; x += P e from `level`+1 to `level`. */
cmg_status cmg_bnd_restrict(cmg_bnd* h, int level, const double* ry, const double* ru, const double* rp, double* cy,
                            double* cu, double* cp);
cmg_status cmg_bnd_prolong_add(cmg_bnd* h, int level, const double* ey, const double* eu, const double* ep,
                               double* y, double* u, double* p);
/* x = S^{-1} f on the coarsest grid (block elimination: per-sample A_j^{-1},
 * the control Schur system G + B^T (sum_j A_j^{-1} (M/N) A_j^{-1}) B). */
cmg_status cmg_bnd_coarse_solve(cmg_bnd* h, const double* fy, const double* fu, const double* fp, double* y,
                                double* u, double* p);
/* One cycle of Algorithm 1 on the finest grid (gamma 1: V, 2: W), in place. */
cmg_status cmg_bnd_cycle(cmg_bnd* h, double theta, int n1, int n2, int gamma, double* y, double* u, double* p,
                         const double* fy, const double* fu, const double* fp);
/* Repeated cycles until ||W (f - S x)|| <= tol ||W f|| (W = diag(N I, 1, 1):
 * the relative residual of the paper's scaling, Sec. 3.2) or maxit; x in/out.
 * CMG_ERR_NOT_CONVERGED / CMG_ERR_NONFINITE as cmg_solve. */
cmg_status cmg_bnd_solve(cmg_bnd* h, double theta, int n1, int n2, int gamma, double tol, int maxit,
                         const double* fy, const double* fu, const double* fp, double* y, double* u, double* p,
                         cmg_stats* stats);

/* ---- learned warm start: the network as one handle ------------------------ */

/* The warm-start network (not part of the paper; multigrid always finishes
 * the solve, Algorithm 1): a BF16 U-Net mapping (y_d, sample mean of
 * log kappa_j) on an S x S image to a control u0.  Four resolutions S, S/2,
 * S/4, S/8 with 32, 64, 64, 64 channels; two 3x3 convolutions + ReLU per
 * encoder level, 2x2 average pooling, nearest upsampling with additive
 * skips, one 3x3 convolution + ReLU per decoder level, a 1x1 linear head;
 * input images [B][S][S][8] BF16 NHWC (channels 0, 1 = y_d and mean
 * log kappa, the rest zero).  Layers 0..10 are the 3x3 convolutions c0a,
 * c0b, c1a, c1b, c2a, c2b, c3a, c3b, d2, d1, d0 (weights [Cout][9 Cin],
 * column t*Cin + c for tap t = 3 dy + dx, bias [Cout]); layer 11 is the
 * head (weights [1][32], bias [1]).
 *
 * The handle owns FP32 master weights, their BF16 copies, the AdamW moments,
 * the gradients, the activations of the last forward pass and the work
 * buffers of the largest layer, all sized at create for at most max_batch
 * images; every call enqueues on the stream given at create.  Device
 * pointers passed in are borrowed for the call (the input X of
 * cmg_unet_forward until the matching cmg_unet_backward).  Errors are
 * status codes with a per-handle message (cmg_unet_last_error); a failed
 * call leaves the handle usable. */
typedef struct cmg_unet cmg_unet;
enum {
  CMG_UNET_W = 0,     /* FP32 master weights */
  CMG_UNET_B = 1,     /* bias */
  CMG_UNET_GW = 2,    /* gradient of the weights (last backward pass) */
  CMG_UNET_GB = 3,    /* gradient of the bias */
  CMG_UNET_MW = 4,    /* AdamW first moment of the weights */
  CMG_UNET_VW = 5,    /* AdamW second moment of the weights */
  CMG_UNET_MB = 6,    /* AdamW moments of the bias */
  CMG_UNET_VB = 7,
  CMG_UNET_W16 = 8    /* the BF16 weights the kernels use (read only, widened to FP32) */
};

/* S: image side, a multiple of 32 in [32, 4096]; max_batch in [1, 1024];
 * seed: initial weights (He-normal for the convolutions, N(0, 1e-4) for the
 * head, zero biases and moments) from a host generator.  Synchronises the
 * stream once.  INVALID_ARG, OOM, CUDA. */
cmg_status cmg_unet_create(int S, int max_batch, unsigned long long seed, void* stream, cmg_unet** out);
void cmg_unet_destroy(cmg_unet* net);
const char* cmg_unet_last_error(const cmg_unet* net);
/* Input and output normalisation (also stored in checkpoints): network
 * channels 0 and 1 are in_yd * y_d and in_logk * mean log kappa; the
 * network predicts u / out. */
cmg_status cmg_unet_set_scales(cmg_unet* net, float in_yd, float in_logk, double out);
cmg_status cmg_unet_get_scales(const cmg_unet* net, float* in_yd, float* in_logk, double* out);
/* Solver grids to images: yd, mlk [B][n*n] FP64 -> X [B][S][S][8] BF16
 * (zero padded outside the n x n interior, n <= S); u [B][n*n] FP64 ->
 * T [B][S][S] FP32 normalised targets; pred [B][S][S] FP32 (NULL = the
 * handle's last prediction) -> out [B][n*n] FP64 controls.  DEVICE. */
cmg_status cmg_unet_pack_inputs(cmg_unet* net, const double* yd, const double* mlk, int B, int n, void* X);
cmg_status cmg_unet_pack_targets(cmg_unet* net, const double* u, int B, int n, float* T);
cmg_status cmg_unet_unpack(cmg_unet* net, const float* pred, int B, int n, double* out);
/* Forward pass of B <= max_batch images X (DEVICE, 16-byte aligned); the
 * prediction is kept in the handle and copied to pred [B][S][S] FP32 when
 * pred is not NULL.  Activations are kept for cmg_unet_backward. */
cmg_status cmg_unet_forward(cmg_unet* net, const void* X, int B, float* pred);
/* Masked mean squared error of the last prediction against target
 * [B][S][S] FP32 over the interior m x m pixels of each image:
 * *loss (DEVICE double) = sum (pred - target)^2 / (B m^2); its gradient
 * (BF16) is kept in the handle for cmg_unet_backward. */
cmg_status cmg_unet_loss(cmg_unet* net, const float* target, int m, double* loss);
/* Gradients of every weight and bias for the last forward pass, from the
 * loss gradient dpred [B][S][S] BF16 (DEVICE), or from the one cmg_unet_loss
 * kept when dpred is NULL. */
cmg_status cmg_unet_backward(cmg_unet* net, const void* dpred);
/* One AdamW step on every layer (decoupled weight decay wd on the weights,
 * none on the biases; bias-corrected moments); refreshes the BF16 weights. */
cmg_status cmg_unet_step(cmg_unet* net, float lr, float beta1, float beta2, float eps, float wd);
/* Parameters: cmg_unet_num_params layers; layer i has weights [rows][cols]
 * and a bias [rows].  cmg_unet_get / cmg_unet_set copy array `which`
 * (CMG_UNET_*) to / from HOST memory and synchronise; setting CMG_UNET_W
 * refreshes the BF16 copy; CMG_UNET_W16 can only be read. */
int cmg_unet_num_params(const cmg_unet* net);
int cmg_unet_steps_taken(const cmg_unet* net);
cmg_status cmg_unet_param_shape(const cmg_unet* net, int layer, int* rows, int* cols);
cmg_status cmg_unet_get(cmg_unet* net, int layer, int which, float* host);
cmg_status cmg_unet_set(cmg_unet* net, int layer, int which, const float* host);
/* *host = 1 if a tensor-core completion wait of any layer's GEMM exceeded
 * its limit since create (results then incomplete), else 0.  Synchronises. */
cmg_status cmg_unet_status(cmg_unet* net, int* host);
/* Checkpoints: a binary file with the FP32 weights, biases, both AdamW
 * moments of each, the AdamW step count and the scales (format 1, checked
 * with the layer shapes on load; S need not match: the network is fully
 * convolutional).  Both synchronise.  A failed load leaves the network
 * unchanged. */
cmg_status cmg_unet_save(cmg_unet* net, const char* path);
cmg_status cmg_unet_load(cmg_unet* net, const char* path);

/* ---- measurement ------------------------------------------------------- */

/* Kernel kinds for cmg_profile_begin. */
enum {
  CMG_KERNEL_SMOOTH = 1,     /* red-black half-sweep or Jacobi update */
  CMG_KERNEL_RESIDUAL = 2,   /* residual / operator apply */
  CMG_KERNEL_RESTRICT = 4,
  CMG_KERNEL_PROLONG = 8,    /* prolongation; in the FP32 red-black cycle the colour-0 half-sweep with it fused in */
  CMG_KERNEL_COARSE = 16,
  CMG_KERNEL_TAIL = 32       /* the cluster launch of the coarse-grid cycle (level = its first grid) */
};

/* Bracket every subsequent launch of the kernel kinds in `kinds` (a bit
 * mask) on grid `level` with CUDA events on the handle's stream (at most
 * 16384 launches are recorded).  Not part of the algorithm: used to time a
 * kernel inside a longer run. */
cmg_status cmg_profile_begin(cmg_handle* h, int kinds, int level);

/* Stop recording, synchronise, and return the summed device time (ms) and
 * the number of recorded launches since cmg_profile_begin. */
cmg_status cmg_profile_end(cmg_handle* h, double* total_ms, int* launches);

/* Number of CUDA kernels this library has launched in the process so far. */
long long cmg_kernel_launches(void);

/* ---- allocation-free entry point ---------------------------------------- */

/* For callers that cannot call cudaMalloc where they need a norm (code
 * running under a host application that owns every device allocation, or
 * a loop that must not allocate between steps).  The paper has no
 * counterpart; this is a service of the library.
 *
 * Writes sqrt(wy^2 ||y||^2 + ||u||^2 + ||p||^2) to out[0] (DEVICE pointer,
 * one double), y and p of length ny, u of length nu (DEVICE, FP64).  With
 * wy = 1 and the level-0 sizes (ny = n*n*N, nu = n*n) it equals cmg_norm;
 * with wy = N it is the norm of the paper's scaling used by cmg_solve.
 * Needs no handle and allocates nothing: the per-block partial sums live in
 * a file-scope device array of 3 x 65536 doubles (1.5 MiB) that every GPU
 * loading this library holds until the process exits.  Its device address
 * is looked up on the FIRST call made on each device (with that device
 * current); make that first call before any stream capture.  Enqueued on
 * `stream` (a cudaStream_t, NULL = legacy default stream) and not
 * synchronised.
 * Every call on a device shares that one array: calls whose work overlaps
 * on the GPU (different streams, or different host threads) race and give
 * wrong results; order them on one stream.  Each call writes every partial
 * it reads, so nothing needs clearing between calls.
 * Errors: CMG_ERR_INVALID_ARG for a null pointer, negative length or
 * non-finite / negative wy; CMG_ERR_UNSUPPORTED if ny or nu exceeds 2^28
 * (268,435,456) elements, the size the array covers (nothing is enqueued);
 * CMG_ERR_CUDA if the launch fails. */
cmg_status cmg_norm_noalloc(const double* y, const double* u, const double* p, long long ny,
                            long long nu, double wy, double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CMG_H_ */
