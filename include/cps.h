/*
 * cps.h -- C ABI of the GB300 corrector-step solver library (libcps.so).
 *
 * The library assembles and solves the sparse symmetric positive definite
 * M-matrix systems of the two corrector problems of the mesoscopic one-domain
 * Navier-Stokes-Brinkman scheme of Aricò, Helmig, Puleo and Schneider
 * (arXiv 2309.03543):
 *
 *   CP2 (Sec. 3.2.3, Eq. CS2_sys_coeff):  A_ee  =  sum_j l_j d_{j,n} / d_{e,ep}
 *                                          A_e,ep = -l_j d_{j,n} / d_{e,ep}
 *        with d_{j,n} = n_j . Xi_j n_j, Xi = eps M^-1 = eps dt (I + nu eps Kinv dt)^-1
 *        (Eq. Cs2_4, M = M0/dt, M0 = I + nu eps Kinv dt from Sec. 3.1);
 *   CP1 (Sec. 3.2.2, Eq. CS1_sys_coeff):  A_ee  = Mbar_kk A_e + nu sum_j l_j / d_{e,ep}
 *                                          A_e,ep = -nu l_j / d_{e,ep}.
 *
 * One unknown per triangle (cell); at most three neighbours per cell.  The
 * systems are solved by preconditioned conjugate gradients (Sec. 3.2.2:
 * "PCG with an incomplete Cholesky factorization"), assembled and factored
 * once and then solved for many right-hand sides (Sec. 3.1).
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers on the context's device unless the
 *     comment says "host".  The caller owns them; the library never frees or
 *     keeps them after the call returns.
 *   - Floating point arrays are IEEE binary64, row-major, contiguous.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     enqueued on it; calls that return a result the host needs (assemble,
 *     solve, adjoint, the CP1 and CP2 steps and their set-ups) synchronise that
 *     stream before they return.
 *   - The return value is a status: CPS_OK (0) or a negative CPS_ERR_* code.
 *     No entry point aborts, traps or throws.  cps_last_error() gives a
 *     human-readable message for the last failing call on a context.
 *   - Handles are not thread-safe: use one handle from one host thread at a
 *     time.
 */
#ifndef CPS_H
#define CPS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define CPS_OK 0
#define CPS_ERR_ARG (-1)            /* bad argument: NULL, size, range, kind */
#define CPS_ERR_NONMANIFOLD (-2)    /* a side shared by more than two cells */
#define CPS_ERR_NONDELAUNAY (-3)    /* some d_{e,ep} <= 1e-12 l_j (Sec. 3.1) */
#define CPS_ERR_ORIENTATION (-4)    /* a triangle is not counter-clockwise */
#define CPS_ERR_NOT_SPD (-5)        /* PCG saw p.Ap <= 0 or a NaN */
#define CPS_ERR_NOT_CONVERGED (-6)  /* max_iter reached; x holds the last iterate */
#define CPS_ERR_SINGULAR (-7)       /* CP2 without a Dirichlet side, or a zero row */
#define CPS_ERR_NOMEM (-8)          /* device allocation failed */
#define CPS_ERR_CUDA (-9)           /* a CUDA runtime call failed */
#define CPS_ERR_TIMEOUT (-10)       /* a bounded device-side wait gave up */

/* ------------------------------------------------------------- constants */
#define CPS_KIND_CP2 0      /* pressure-increment system (Eq. CS2_sys_coeff) */
#define CPS_KIND_CP1_X 1    /* viscous x-velocity system (Eq. CS1_sys_coeff) */
#define CPS_KIND_CP1_Y 2    /* viscous y-velocity system */

#define CPS_PER_VERTEX 0    /* eps, Kinv given at the mesh nodes (Sec. 3.2) */
#define CPS_PER_CELL 1      /* eps, Kinv given per triangle */
#define CPS_PER_CELL_LOGK 2 /* eps per triangle; kinv[nt] holds the log-permeability
                               theta, K = exp(theta) I (isotropic), Kinv = exp(-theta) I */

#define CPS_PC_JACOBI 1     /* diagonal preconditioner */
#define CPS_PC_IC0 2        /* IC(0) in a multicolour order of the cells */
#define CPS_PC_REDUCED 3    /* two-colourable cell graphs: eliminate one colour
                               exactly, CG on the other colour's Schur complement */

#define CPS_FP64 0          /* all storage and arithmetic in binary64 */
#define CPS_MIXED 1         /* binary32 matrix/vectors inside FP64 refinement */

typedef struct cps_ctx_s* cps_ctx;
typedef struct cps_sys_s* cps_sys;

typedef struct {
    int64_t iters;        /* PCG iterations run (summed over refinements) */
    double rel_res;       /* true ||b - A x||_2 / ||b||_2 at return, in FP64 */
    int32_t status;       /* same value as the call's return */
    int32_t refinements;  /* outer FP64 residual steps (CPS_MIXED), else 1 */
    int64_t launches;     /* kernels this call enqueued (graph nodes counted) */
} cps_stats;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  *out receives the handle. */
int cps_create(cps_ctx* out, int device);

/* Destroy a context.  Systems made from it that are still live are freed
 * with it; their handles become invalid. */
int cps_destroy(cps_ctx ctx);

/* Message of the last failing call on this context (never NULL; owned by
 * the context, valid until the next call on it). */
const char* cps_last_error(cps_ctx ctx);

/* ------------------------------------------------------------- assembly */

/* Build one corrector system from a counter-clockwise triangle mesh.
 *
 *   xy[nv*2]        vertex coordinates (x, y)
 *   tri[nt*3]       vertex ids of each triangle, counter-clockwise; local
 *                   side j joins vertices (j+1)%3 and (j+2)%3
 *   dirichlet[nb]   boundary sides with eta = 0 at the side midpoint, given as
 *                   tri*3 + j; all other boundary sides are no-flux.  May be
 *                   NULL when nb = 0 (then CP2 is singular: CPS_ERR_SINGULAR)
 *   eps[nf]         porosity, nf = nv (CPS_PER_VERTEX) or nt (CPS_PER_CELL,
 *                   CPS_PER_CELL_LOGK)
 *   kinv[nf*3]      inverse permeability tensor (xx, xy, yy), symmetric PSD;
 *                   kinv[nt] = theta for CPS_PER_CELL_LOGK
 *   field_loc       CPS_PER_VERTEX: side tensor = mean of the tensors Xi at the
 *                   side's two nodes (Sec. 3.2 side averages); CPS_PER_CELL:
 *                   mean of the two cells' Xi, a boundary side uses its cell's
 *   kind            CPS_KIND_CP2, CPS_KIND_CP1_X or CPS_KIND_CP1_Y
 *   nu, dt          kinematic viscosity and time step (> 0)
 *
 * Geometry (Sec. 3.1, Eq. cs1_discr): circumcentres c_e, side lengths l_j,
 * outward unit normals n_j, d_{e,ep} = (c_ep - c_e) . n_j.  A Dirichlet side
 * adds l_j d_{j,n} / delta_j (CP1: nu l_j / delta_j) to the diagonal, with
 * delta_j = (m_j - c_e) . n_j the distance from the circumcentre to the side.
 * The Jacobi preconditioner is ready on return (cps_set_precond switches).
 * Errors: CPS_ERR_ARG, _NONMANIFOLD, _NONDELAUNAY, _ORIENTATION, _SINGULAR,
 * _NOMEM, _CUDA.  On error *out is NULL. */
int cps_assemble(cps_ctx ctx, const double* xy, int64_t nv, const int32_t* tri, int64_t nt,
                 const int32_t* dirichlet, int64_t nb, const double* eps,
                 const double* kinv, int field_loc, int kind, double nu, double dt,
                 cps_sys* out, void* stream);

/* Select the preconditioner (Sec. 3.2.2 uses incomplete Cholesky):
 * CPS_PC_JACOBI, or CPS_PC_IC0 = IC(0) factored once on the pattern of A in a
 * multicolour order of the cells (two colours on the lattice's bipartite cell
 * graph).  The factor is computed here, once, on the device.
 * CPS_PC_REDUCED (FP64 solves only): for a cell graph with two colours R, B
 * (no two neighbours share a colour), the R unknowns are eliminated exactly
 * from the diagonally scaled system and CG runs on S = I - E^T E over the B
 * cells (E = the scaled R-B couplings); x_R is recovered afterwards.  The
 * solution is that of A x = b; CPS_ERR_ARG if the graph needs more than two
 * colours. */
int cps_set_precond(cps_sys sys, int precond, void* stream);

/* Free a system and all device memory it owns.  A handle that was already
 * freed (or whose context was destroyed) must not be passed again. */
int cps_sys_free(cps_sys sys);

/* Host outputs (any may be NULL): number of cells, number of interior sides,
 * smallest diagonal entry, 1 if every row has a positive diagonal and
 * non-positive off-diagonals (the M-matrix sign pattern), and the number of
 * kernels the assembly (and preconditioner set-up) launched. */
int cps_sys_info(cps_sys sys, int64_t* nt, int64_t* n_interior_sides, double* diag_min,
                 int* is_mmatrix, int64_t* setup_launches);

/* Copy the assembled matrix out in padded ELL form (device pointers):
 * diag[nt]; col[3*nt], val[3*nt] slot-major (entry s*nt + e is slot s of row
 * e; an unused slot has col = e, val = 0).  Row/column order is the mesh's. */
int cps_export_matrix(cps_sys sys, double* diag, int32_t* col, double* val, void* stream);

/* ---------------------------------------------------------------- solves */

/* Solve A x = b by PCG.
 *   b[nt]       right-hand side (not modified)
 *   x[nt]       in: initial guess (warm start; zeros for a cold start),
 *               out: solution
 *   rtol        stop when ||b - A x||_2 <= rtol ||b||_2; the true residual is
 *               recomputed in FP64 at the end and the solve continues if it is
 *               still above rtol
 *   max_iter    bound on PCG iterations (summed over refinements)
 *   precision   CPS_FP64 or CPS_MIXED (binary32 matrix, vectors and SpMV in
 *               the inner PCG; binary64 dot products, alpha/beta, and the
 *               outer residual b - A x and update of x)
 *   stats       host pointer, may be NULL
 * b = 0 gives x = 0.  Errors: CPS_ERR_ARG, _NOT_SPD, _NOT_CONVERGED (x holds
 * the last iterate; CPS_MIXED: the iterate with the least true residual, with
 * that residual in stats -- where kappa(A) times the binary32 unit roundoff
 * approaches 1 the binary32 corrections stop reducing the FP64 residual, and
 * the solve ends there instead of letting refinement drive it up), _CUDA. */
int cps_solve(cps_sys sys, const double* b, double* x, double rtol, int64_t max_iter,
              int precision, cps_stats* stats, void* stream);

/* Solve nsys independent systems (each with its own matrix, b and x) together.
 * systems, b, x and stats are HOST arrays of length nsys holding handles and
 * device pointers (b[i], x[i] of system i's size; x[i] is the initial guess
 * and receives the solution).  All systems must come from the same context.
 * CPS_FP64 (Jacobi, whatever each system's preconditioner setting): by
 * default one cooperative kernel launch for the whole ensemble -- the
 * larger systems (estimated work cells^1.5 above half a block's fair
 * share) are each solved by a static team of blocks that split the rows and
 * combine their sums through bounded device-side waits, and every other
 * block takes whole systems from a device work queue (largest first) and
 * solves each with block-level reductions only; a team's blocks join the
 * queue when their system is done, and every system stops as soon as it
 * converges.  The iteration is the single-reduction (Chronopoulos-Gear) form
 * of Jacobi CG, restarted from the true residual up to 8 times.  A team
 * wait that runs out (about one second) gives CPS_ERR_TIMEOUT.  With
 * cps_set_batch_path(ctx, CPS_BATCH_GRAPH) instead one launch per phase for
 * all systems, a per-system convergence mask, and iteration chunks replayed
 * from a CUDA graph (a system of more than 33,554,432 cells is rejected there
 * with CPS_ERR_ARG -- solve it alone).  CPS_MIXED: by default the same one
 * launch, each system (or team) running the single solve's refinement with
 * every decision on the device -- binary32 textbook CG inner iterations with
 * FP64 inner products, an FP64 true residual after each, the best FP64
 * iterate kept (stats.refinements = residual replacements); with
 * CPS_BATCH_GRAPH instead each system's solve (whose residual replacements
 * are decided on the host) runs whole on one of up to 8 internal streams,
 * fed by as many host threads, so that the systems' launches overlap on the
 * GPU; the call returns after ordering `stream` behind all of them (it
 * blocks the calling thread until every system has finished).  The return
 * value is the first non-OK per-system status, or CPS_OK. */
int cps_solve_batch(const cps_sys* systems, int nsys, const double* const* b,
                    double* const* x, double rtol, int64_t max_iter, int precision,
                    cps_stats* stats, void* stream);

/* How cps_solve_batch runs ensembles on this context (no counterpart in
 * the paper; both are for the ensemble workload): CPS_BATCH_ONE_LAUNCH (the
 * default) or CPS_BATCH_GRAPH (see cps_solve_batch).  Errors: CPS_ERR_ARG. */
#define CPS_BATCH_ONE_LAUNCH 0
#define CPS_BATCH_GRAPH 1
int cps_set_batch_path(cps_ctx ctx, int path);

/* Adjoint of one solve x = A^-1 b (A symmetric, so the same matrix and
 * preconditioner serve): lambda = A^-1 g, then for every local side slot
 * (slot-major, s*nt + e)
 *   dT[s*nt+e] += -(lambda_e - lambda_ep)(x_e - x_ep)   interior side
 *   dT[s*nt+e] += -lambda_e x_e                         Dirichlet side
 * which is dL/dT for the side coefficient T of A (each interior side appears
 * in both of its cells' slots with the same value).  If dtheta is not NULL
 * (CP2 with CPS_PER_CELL_LOGK, or CPS_PER_CELL with isotropic Kinv, read as
 * Kinv = exp(-theta) I) the chain rule
 * through Xi_e = eps dt / (1 + nu eps dt exp(-theta_e)) is applied and
 * dL/dtheta is ADDED to dtheta[nt].  dT may be NULL if only dtheta is wanted.
 * lambda[nt] is overwritten (its input is the initial guess).
 * Errors: as cps_solve, plus CPS_ERR_ARG for dtheta on an unsupported system. */
int cps_adjoint(cps_sys sys, const double* x, const double* g, double* lambda, double* dT,
                double* dtheta, double rtol, int64_t max_iter, cps_stats* stats,
                void* stream);

/* ------------------------------------------- CP2 step around the solves */

/* Prepare the CP2 step (Sec. 3.2.3) on an assembled CP2 system: pass the same
 * xy, tri, eps and kinv (device pointers, same sizes and field_loc) that built
 * it; nothing of them is kept.  Stores per side slot the mean-flux geometry
 * l_j n_j, T_j, four co-normal weights and cell indices of the tangential flux
 * (App. C), per cell the RT0 weights and Mbar_e (about 376 bytes per cell).
 * A second call replaces the data.  Errors: CPS_ERR_ARG (not CP2, null
 * pointer), _NONDELAUNAY, _NONMANIFOLD, _ORIENTATION (inputs that do not
 * match the system), _NOMEM, _CUDA. */
int cps_cp2_setup(cps_sys sys, const double* xy, const int32_t* tri, const double* eps,
                  const double* kinv, void* stream);

/* One CP2 step: from the cell velocity u^{k+2/3} of the first corrector to the
 * divergence-free u^{k+1} and the updated eps grad(Psi).
 *   u23[2*nt]     u^{k+2/3} per cell: x components, then y components
 *   g_k[2*nt]     eps grad(Psi^k) per cell, same layout
 *   eta_tilde[nt] out: first solution eta~ (may be NULL, or eta itself, in
 *                 which case eta ends as the second solution)
 *   eta[nt]       out: second solution eta
 *   u_next[2*nt]  out: u^{k+1}, the RT0 field at the centroid (Eq. RT0)
 *   g_next[2*nt]  out: eps grad(Psi^{k+1}) = g_k + Mbar_e (u_next - u23) (Eq. grad_PSI)
 *   flux[3*nt]    out (may be NULL): outward flux Q of u^{k+1} through local
 *                 side j of cell e at j*nt + e; sum_j Q = 0 per cell to the
 *                 solve tolerance and Q is antisymmetric across a side
 *   rtol, max_iter, precision as cps_solve, for both solves
 *   stats         host array of 2 (first and second solve), may be NULL
 * Steps: Fbar_j = ((u_e.n_j) A_ep + (u_ep.n_j) A_e)/(A_e + A_ep) l_j
 * (Eq. flux_k_+_2/3; a Dirichlet side carries (u_e.n_j) l_j, a no-flux side
 * nothing); A eta~ = sum_j Fbar_j (Eq. Cs2_7_1); tau_j(eta~), the tangential
 * flux of Xi_j grad(eta) from the co-normal decomposition (Eq. Cs2_6, App. C);
 * A eta = sum_j (Fbar_j + tau_j) from eta~ (Eq. Cs2_7_2); Q_j = Fbar_j -
 * T_j (eta_e - eta_ep) + tau_j.  Fluxes are physical and outward.  Needs
 * cps_cp2_setup.  The outputs must not overlap the inputs.  Errors: as
 * cps_solve (CPS_ERR_NOT_CONVERGED still completes the step), CPS_ERR_ARG. */
int cps_cp2_step(cps_sys sys, const double* u23, const double* g_k, double* eta_tilde,
                 double* eta, double* u_next, double* g_next, double* flux, double rtol,
                 int64_t max_iter, int precision, cps_stats* stats, void* stream);

/* ------------------------------------------------ CP1 step (two systems) */

typedef struct {
    int64_t outer;        /* outer sweeps after the uncoupled first one */
    int64_t solve_iters;  /* PCG iterations of all solves */
    double err;           /* last min(err_x, err_y) (App. B) */
    double rel_res_max;   /* largest final relative residual of the solves */
} cps_cp1_stats;

/* Prepare the CP1 step (Sec. 3.2.2) on a pair of systems assembled with
 * CPS_KIND_CP1_X (sys_x) and CPS_KIND_CP1_Y (sys_y) from the same mesh, fields
 * and Dirichlet sides; pass the same xy, tri, eps and kinv (device pointers).
 * Stores on sys_x the side coefficients nu l_j/d (nu l_j/delta on Dirichlet
 * sides) and per cell Mbar_11 A_e, Mbar_12 A_e, Mbar_22 A_e (Mbar the mean over
 * the cell's nodes of (I + nu eps Kinv dt)/dt).  Errors: CPS_ERR_ARG (kinds,
 * sizes, contexts, null pointers), _NONDELAUNAY, _NOMEM, _CUDA. */
int cps_cp1_setup(cps_sys sys_x, cps_sys sys_y, const double* xy, const int32_t* tri,
                  const double* eps, const double* kinv, void* stream);

/* The CP1 solves of one time step with the outer iteration of App. B (Eq. A1):
 *   du_breve[2*nt]  predictor increment u^{k+1/3} - u^{k-1/3} per cell (x
 *                   components, then y)
 *   du[2*nt]        in: initial guess of the first solves (zeros for a cold
 *                   start); out: the increment u^{k+2/3} - u^{k+1/3}
 *   toll            outer tolerance (the paper uses 1e-4 .. 1e-3)
 *   max_outer       bound on the outer sweeps after the first (0: the
 *                   uncoupled first sweep only)
 *   rtol, max_iter, precision   as cps_solve, for every solve
 *   stats           host, may be NULL
 * Each component solves (Mbar_kk A_e + nu L) du_k = -nu L du_breve_k -
 * Mbar_12 A_e du_other, nu L the off-diagonal operator of the CP1 matrix
 * (Eq. cs1_sys2, Eq. CS1_sys_coeff with the sign of Eq. CS1_2).  Sweep 0 drops
 * the coupling; each later sweep solves both components with the other's
 * previous iterate, warm-started, until min(err_x, err_y) <= toll, err_k =
 * ||du_k^{i+1} - du_k^i||_2 / ||du_k^i||_2.  Needs cps_cp1_setup.  When both
 * systems use the Jacobi preconditioner the whole outer iteration runs by
 * default in one cooperative launch: each sweep's right-hand sides, both
 * solves (the single-reduction Jacobi CG of cps_solve_batch, FP64 or mixed,
 * by all the launch's blocks), the change test and the stop decision on the
 * device, the statistics read once at the end; otherwise (or after
 * cps_set_cp1_path(sys_x, CPS_CP1_HOST)) each solve is a cps_solve and the
 * change sums are read back after every sweep.  Errors: as cps_solve
 * (CPS_ERR_TIMEOUT: a device-side wait of the one launch ran out);
 * CPS_ERR_NOT_CONVERGED also when max_outer sweeps end above toll (du holds
 * the last iterate). */
int cps_cp1_step(cps_sys sys_x, cps_sys sys_y, const double* du_breve, double* du, double toll,
                 int64_t max_outer, double rtol, int64_t max_iter, int precision,
                 cps_cp1_stats* stats, void* stream);

/* How cps_cp1_step runs on the pair prepared on sys_x (no counterpart in the
 * paper): CPS_CP1_ONE_LAUNCH (the default; Jacobi systems) or CPS_CP1_HOST
 * (see cps_cp1_step).  Errors: CPS_ERR_ARG (bad path, or no cps_cp1_setup). */
#define CPS_CP1_ONE_LAUNCH 0
#define CPS_CP1_HOST 1
int cps_set_cp1_path(cps_sys sys_x, int path);

/* Device durations in milliseconds (host ms[3]) of the last cps_cp2_step's
 * three step kernels -- mean flux, tangential flux, update -- from CUDA events
 * recorded around each on the step's stream (-1 if unavailable).
 * Errors: CPS_ERR_ARG (no CP2 step data). */
int cps_cp2_kernel_times(cps_sys sys, float* ms);

/* Choose how FP64 Jacobi and reduced-system solves run:
 *   CPS_PATH_AUTO (default): the autotuner times the applicable paths on the
 *     system's first solve of that kind and keeps the fastest;
 *   CPS_PATH_STREAM: graph-replayed streaming kernels, any size;
 *   CPS_PATH_CLUSTER (FP64 Jacobi only): the whole solve in one launch of a
 *     single thread-block cluster whose shared memory holds the system;
 *     CPS_ERR_ARG if the system does not fit, see cps_sys_info;
 *   CPS_PATH_PERSISTENT: the whole solve in one cooperative launch of one
 *     resident grid, iterations separated by software grid barriers (every
 *     wait bounded: a wait that runs out ends the solve with
 *     CPS_ERR_TIMEOUT);
 *   CPS_PATH_STREAM_L2: streaming kernels with the vectors r, p, q held in
 *     persisting L2 during the solve; CPS_ERR_ARG if the GPU's persisting
 *     set-aside cannot hold them;
 *   CPS_PATH_PERSISTENT_L2: the persistent launch with r, p, q in persisting
 *     L2 (CPS_ERR_ARG as above);
 *   CPS_PATH_STREAM_1RED, CPS_PATH_STREAM_1RED_L2 (FP64 Jacobi only):
 *     graph-replayed streaming kernels with the single-reduction
 *     (Chronopoulos-Gear) recurrences -- two kernels and one grid reduction
 *     per iteration instead of three and two -- without / with its vectors
 *     in persisting L2 (all five where the set-aside holds them, else r, p,
 *     q; CPS_ERR_ARG as above when it cannot hold r, p, q);
 *   CPS_PATH_CLUSTER_1RED (FP64 Jacobi only): the one-cluster launch with the
 *     single-reduction (Chronopoulos-Gear) recurrences -- s = A p and w = A r
 *     are carried so that both inner products of an iteration come from one
 *     SpMV (two cluster barriers per iteration instead of three; one more
 *     vector in shared memory, so a somewhat smaller size limit);
 *   CPS_PATH_CLUSTER_PIPE (FP64 Jacobi only): the one-cluster launch with the
 *     pipelined (Ghysels-Vanroose) single-reduction recurrences -- z = A s
 *     is carried as well, so that the SpMV of an iteration runs while its
 *     reduction is in flight: one split cluster barrier per iteration (two
 *     more vectors in shared memory, a smaller size limit).  Pinned only:
 *     CPS_PATH_AUTO does not take it, since its recurrences lose accuracy
 *     sooner and need more iterations than the per-iteration gain repays;
 *   CPS_PATH_CLUSTER_SSTEP2, CPS_PATH_CLUSTER_SSTEP3 (FP64 Jacobi only): the
 *     one-cluster launch with s-step CG, s = 2 or 3 -- per outer step a
 *     Chebyshev basis of s + 1 powers of the matrix applied to p and s
 *     applied to r, their Gram matrix in one reduction, then s CG steps on
 *     the basis coordinates: s + 1 cluster barriers per s iterations instead
 *     of 2s, for more arithmetic per row (2s + 1 vectors in shared memory,
 *     a smaller size limit); the stop test runs once per outer step, so the
 *     count may exceed the single-reduction one by up to s - 1.  Pinned
 *     only: CPS_PATH_AUTO does not take it;
 *   CPS_PATH_PERSISTENT_1RED, CPS_PATH_PERSISTENT_1RED_L2 (FP64 Jacobi,
 *     FP64 IC(0) in a two-colour order, and the reduced system): the
 *     persistent launch with the single-reduction recurrences -- per
 *     iteration one grid reduction and waits on the neighbouring blocks only
 *     (Jacobi: one; IC(0): two, in Eisenstat's form of the preconditioned
 *     iteration, which applies the two-colour IC(0) factor and the matrix in
 *     one pass over the matrix, with the same iterates; reduced system: two,
 *     around the two halves of the Schur product) -- without / with its
 *     vectors in persisting L2 (Jacobi and the reduced system: five,
 *     CPS_ERR_ARG when the set-aside cannot hold them; IC(0): six where they
 *     fit, else five, else none).
 * FP64 IC(0) in a two-colour order runs on the streaming kernels for every
 * other pin, and CPS_PATH_AUTO times both ways on the first such solve; with
 * more colours it always streams.
 * Mixed precision always streams. */
#define CPS_PATH_AUTO 0
#define CPS_PATH_STREAM 1
#define CPS_PATH_CLUSTER 2
#define CPS_PATH_PERSISTENT 3
#define CPS_PATH_STREAM_L2 4
#define CPS_PATH_PERSISTENT_L2 5
#define CPS_PATH_CLUSTER_1RED 6
#define CPS_PATH_STREAM_1RED 7
#define CPS_PATH_STREAM_1RED_L2 8
#define CPS_PATH_PERSISTENT_1RED 9
#define CPS_PATH_PERSISTENT_1RED_L2 10
#define CPS_PATH_CLUSTER_PIPE 11
#define CPS_PATH_CLUSTER_SSTEP2 12
#define CPS_PATH_CLUSTER_SSTEP3 13
int cps_set_solver_path(cps_sys sys, int path);

/* Pin the launch shapes of the iteration kernels of one precision instead of
 * letting the autotuner time them (for reproducible measurements, e.g. under
 * a profiler whose replay would skew the tuner's timings).  unroll, grid and
 * block are host arrays of 3 entries (SpMV, residual update, direction
 * update; the third is ignored for CPS_MIXED): unroll 1, 2 or 4 rows per
 * thread per trip (also 8 for the two FP64 update kernels), grid 1..4096
 * blocks, block 256 (or, CPS_FP64 only, 1024) threads.  CPS_ERR_ARG for
 * anything else. */
int cps_set_kernel_shapes(cps_sys sys, int precision, const int32_t* unroll, const int32_t* grid,
                          const int32_t* block);

/* Test hook for failure detection (no counterpart in the paper).  With
 * CPS_TEST_STALL_BARRIER, the next persistent launch on this system (see
 * CPS_PATH_PERSISTENT) waits at its first grid barrier for one arrival that
 * never comes: every block's bounded wait runs out after about a second, the
 * kernel ends, and the solve returns CPS_ERR_TIMEOUT.  The same holds for the
 * team waits of the next one-launch cps_solve_batch whose first system this
 * is (every team of blocks stalls; systems solved by single blocks finish),
 * and of the next one-launch cps_cp1_step whose sys_x this is.  The context
 * stays usable.  One-shot; 0 clears a pending fault.  CPS_ERR_ARG for an
 * unknown fault. */
#define CPS_TEST_STALL_BARRIER 1
int cps_test_inject(cps_sys sys, int fault);

/* Launch configuration the autotuner chose for the iteration kernels of one
 * precision (host outputs of 3 entries each; zeros before the first solve in
 * that precision): rows per thread per trip of the grid-stride loop, the
 * grid in blocks and the threads per block (block may be NULL; 256, or 1024
 * for the FP64 kernels), for the SpMV kernel, the residual update and
 * (CPS_FP64 only) the direction update.  The tuner times every candidate on
 * the system's own data at its first solve; systems below 131072 cells keep
 * the defaults (unroll 2, 8 blocks per SM).  For CPS_FP64 Jacobi solves it
 * also times the ways of running the loop: flags (may be NULL, 8 entries)
 * receives {one-cluster launch chosen (0 no, 1 textbook recurrences, 2 the
 * single-reduction recurrences, 3 the pipelined ones), persisting-L2 window (0 none, 1 the
 * matrix, 2 the vectors r, p, q, 3 the five vectors of the single-reduction
 * loop), persistent launch chosen (either recurrence), reduced system:
 * persistent launch chosen (0 no, 1 textbook recurrences, 2 single-reduction
 * recurrences), reduced system: window (0, 2, or 3 the five vectors of its
 * single-reduction loop), single-reduction
 * streaming chosen, single-reduction persistent launch chosen, IC(0):
 * persistent single-reduction launch chosen (0 no, 1 without a window, 2
 * with its first five vectors, 3 with all six in persisting L2)}, flags
 * then taking 8 entries; probe_us (may be
 * NULL, 18 entries) the microseconds per iteration measured for {streaming,
 * one cluster (the best of its three recurrences), streaming + matrix in L2, persistent, streaming + vectors in
 * L2, persistent + vectors in L2, reduced system: streaming, persistent,
 * streaming + vectors in L2, persistent + vectors in L2, single-reduction
 * streaming, single-reduction streaming + vectors in L2, single-reduction
 * persistent, single-reduction persistent + vectors in L2, IC(0): streaming,
 * persistent single-reduction (the better window), reduced system:
 * persistent single-reduction, the same + its vectors in L2} (0 where not tried; the
 * persistent figures are the best over the grid sizes tried, the one-cluster
 * figure the better of its two recurrences).
 * The context remembers what the tuner chose per mesh size (cells,
 * vertices): a system assembled later on the same context with the same
 * sizes starts from those choices and is not timed again.  A path forced by
 * cps_set_solver_path applies to that system only. */
/* Launch shape (host outputs: rows per thread per trip, blocks, threads per
 * block) of the single-reduction loop's update kernel, which the FP64 path
 * probe tunes on its own once it has chosen that loop (the residual update's
 * shape before; 0s before the first FP64 solve).  Errors: CPS_ERR_ARG. */
int cps_get_gear_shape(cps_sys sys, int32_t* unroll, int32_t* grid, int32_t* block);

int cps_get_tuning(cps_sys sys, int precision, int32_t* unroll, int32_t* grid, int32_t* block,
                   int32_t* flags, double* probe_us);

/* Allocation-free solve of a matrix the caller already holds in the padded
 * ELL form that cps_export_matrix writes (no counterpart in the paper; it is
 * an interface for callers that cannot allocate device memory).  Such callers
 * exist: code running inside a host that owns all device memory through its
 * own pool, code that must not call cudaMalloc/cudaFree because those calls
 * synchronise the device, and code whose memory budget is already spent.
 * This call needs no handle and allocates nothing (no cudaMalloc, cudaFree,
 * pinned host memory, events or graphs): its working vectors live in one
 * fixed device array inside libcps.so (about 4.3 MB, held on every device
 * that loads the library until the process exits).
 *   n                 rows, 0 <= n <= 65536; a larger n returns CPS_ERR_ARG
 *                     before any work is enqueued
 *   diag[n], col[3n], val[3n]   device arrays: diagonal, then slot-major
 *                     neighbour columns and values (s*n + e is slot s of row
 *                     e; an unused slot has col = e, val = 0); A must be
 *                     symmetric with a positive diagonal
 *   b[n], x[n]        device arrays: right-hand side; initial guess in,
 *                     solution out
 *   rtol, max_iter    as cps_solve (FP64 Jacobi-PCG, true-residual stop)
 *   stats             host pointer, may be NULL
 *   stream            cudaStream_t on the current device
 * The first call on a device looks up the device address of the array
 * (cudaGetSymbolAddress) for that device, which is the current device of the
 * calling thread; make that first call before any stream capture.  Under
 * CUDA's default lazy module loading that first call is also the moment the
 * library's device code and data, this array included, are loaded onto the
 * device: it is the one call that commits device memory and may synchronise
 * the device.  Callers with a spent memory budget or a no-synchronisation
 * rule should therefore make the first call during their start-up (or run
 * with CUDA_MODULE_LOADING=EAGER, which loads everything at context
 * creation).  Every call waits for its stream: it reads the iteration state
 * back to the host after the set-up and after each chunk of 32 iterations.
 * Every call on a device shares the same array and resets the parts that
 * must start at zero, so calls whose work overlaps on the GPU (different
 * streams or host threads at the same time) race with each other: serialise
 * them.
 * Errors: CPS_ERR_ARG (size, NULL, column out of range), CPS_ERR_NOT_SPD
 * (diagonal <= 0 or p.Ap <= 0), CPS_ERR_NOT_CONVERGED, CPS_ERR_CUDA (also
 * returned, without clearing it, when a CUDA error from the caller's earlier
 * work is still pending on entry).  stats->status always equals the return
 * value; rel_res is NaN when the call returned before computing a residual. */
int cps_solve_ell_noalloc(int64_t n, const double* diag, const int32_t* col, const double* val,
                          const double* b, double* x, double rtol, int64_t max_iter,
                          cps_stats* stats, void* stream);

/* y = A x for the assembled matrix (device pointers, FP64). */
int cps_matvec(cps_sys sys, const double* x, double* y, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CPS_H */
