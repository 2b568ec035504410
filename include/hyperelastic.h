/*
 * hyperelastic.h -- C ABI of libhyperelastic: matrix-free finite-strain hyperelasticity with
 * geometric multigrid on one GB300 GPU (arXiv 1904.13131, "A matrix-free approach for finite-strain
 * hyperelastic problems using geometric multigrid").
 *
 * Problem class: compressible neo-Hookean solid (Sec. 2.3) on the unit square (dim 2, plane strain)
 * or unit cube (dim 3), uniform m^dim mesh of Q_k Lagrange cells (k = 1..4) with GLL nodes and the
 * (k+1)^dim Gauss rule (Sec. 7, Tables 1-2: q = p + 1); homogeneous or prescribed Dirichlet values on
 * selected components of selected faces.
 *
 * Conventions for every call:
 *  - Vectors are caller-owned DEVICE buffers (e.g. a torch tensor's data pointer) on the context's
 *    device, in the canonical layout: nodes of the (k m + 1)^dim lattice in lexicographic order with
 *    x fastest, the dim displacement components of a node interleaved (dof = node * dim + comp).
 *    "Level" l counts from 0 (coarsest, m / 2^(L-1) cells per direction) to L-1 (finest, m cells).
 *  - The library owns everything else (caches, level vectors, hierarchy) and frees it in
 *    hy_destroy. It never frees caller buffers.
 *  - Work is enqueued on the stream given to hy_create (borrowed, not owned); calls that return
 *    scalars or reports synchronise that stream before returning.
 *  - Every call returns a hy_status, never throws across the ABI and never aborts the process.
 *    On error, hy_last_error() holds a one-line description. A kernel-side failure (J <= 0, NaN)
 *    is reported through the status of the call that checks it, with the device left usable.
 *  - Faces are numbered (-x, +x, -y, +y, -z, +z); a face mask is a bitmask of constrained
 *    components (bit c = component c).
 */
#ifndef HYPERELASTIC_H
#define HYPERELASTIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hy_ctx hy_ctx;

typedef enum {
  HY_OK = 0,
  HY_ERR_ARG = 1,          /* invalid argument (size, degree, pointer, NaN input, ...) */
  HY_ERR_STATE = 2,        /* call out of order (e.g. apply before set_displacement) */
  HY_ERR_OOM = 3,          /* device allocation failed */
  HY_ERR_CUDA = 4,         /* a CUDA runtime call failed */
  HY_ERR_JNEG = 5,         /* J = det F <= 0 at some Gauss point (Sec. 2.1 requires J > 0) */
  HY_ERR_NOCONV = 6,       /* an iteration reached its cap */
  HY_ERR_TIMEOUT = 7,      /* a bounded device wait gave up */
  HY_ERR_UNSUPPORTED = 8   /* valid but not built (e.g. degree 5) */
} hy_status;

/* Arithmetic of a tangent action. HY_FF (double-float): FP64 vectors and an FP64-accurate result (about
 * 48 significant bits, within 1e-12 of the FP64 action in relative L2 norm), computed as unevaluated sums
 * of two floats on the FP32 pipe, which GB300 issues at 64 times its FP64 rate. Not IEEE FP64: a
 * service of this library for the finest level (see fine_dtype), not a step of the paper's method. */
typedef enum { HY_F64 = 0, HY_F32 = 1, HY_FF = 2 } hy_dtype;

/* Tangent-operator variants (Sec. 5):
 *   HY_T4  cache F^{-1}, tau and the fourth-order tangent J*C per Gauss point (Algorithm 3)
 *   HY_T2  cache F^{-1}, tau and two scalars of the neo-Hooke action (Algorithm 2)
 *   HY_FC  cache F only; J, ln J, tau and the action recomputed in every application
 *   HY_SC  cache mu - 2 lambda ln J only; F recomputed from the displacement (Algorithm 1)
 *   HY_NC  cache nothing; everything recomputed from the displacement */
typedef enum { HY_T4 = 0, HY_T2 = 1, HY_FC = 2, HY_SC = 3, HY_NC = 4 } hy_variant;

/* Create a context on CUDA device `device`, enqueuing all work on `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream). The stream is borrowed: it must outlive the context. */
hy_status hy_create(hy_ctx **out, int device, void *cuda_stream);
/* Free every device buffer the context owns. NULL is accepted. */
void hy_destroy(hy_ctx *ctx);
/* Name of a status code ("HY_OK", ..., "HY_ERR_UNKNOWN" for other values); a static string. */
const char *hy_status_str(hy_status s);
/* Message of the context's most recent failed call (empty if none failed yet; a later success does not
 * clear it); owned by the context, valid until its next call. NULL context: "null context". */
const char *hy_last_error(const hy_ctx *ctx);

/* Mesh and level hierarchy (Sec. 6: a hierarchy of uniformly refined meshes; Sec. 3: Q_k space).
 * dim 2|3, degree 1..4, cells_per_dir m >= 1; n_levels >= 1 levels with m / 2^(L-1-l) cells on level l
 * (m must stay even while halving). face_masks[2*dim] gives the constrained components of each
 * face; the same homogeneous constraints hold on every level (Sec. 6). Replaces any previous mesh. */
hy_status hy_mesh_setup(hy_ctx *ctx, int dim, int degree, int cells_per_dir, int n_levels,
                        const uint32_t *face_masks);

/* Number of dofs of level `level` (-1 = finest). */
hy_status hy_num_dofs(const hy_ctx *ctx, int level, int64_t *n);

/* Materials of level `level` (-1 = finest): HOST arrays cell_mat[m_l^dim] (ids < n_mat, cells in
 * lexicographic order, x fastest) and mu[n_mat], lambda[n_mat] (Sec. 2.3). Every level needs one
 * call before hy_set_displacement; n_mat <= 16. */
hy_status hy_set_material(hy_ctx *ctx, int level, const uint8_t *cell_mat, const double *mu,
                          const double *lambda, int n_mat);

/* Volumetric function of the compressible neo-Hooke law, on every level; the isochoric part and the
 * -mu ln J term are the paper's (Sec. 2.3). HY_LAW_LOG2 (default): U = lambda ln^2 J, the paper's;
 * HY_LAW_J2: U = lambda/4 (J^2 - 1 - 2 ln J). With p = J U'(J) both give tau = mu b - (mu - p) I and
 * J*C = 2 (mu - p) S + J p'(J) I (x) I. The law enters where the Gauss-point state is formed (the state
 * build, residual, diagonal and dense coarse assembly), so it goes through the caching variants T4 and
 * T2 unchanged. The recomputing variants FC, SC and NC form the state in every application: under
 * HY_LAW_J2 they run their general build, which evaluates the volumetric function chosen at run time
 * (and reads the reference map of every Gauss point from the cache: d^2 + 1 more cached values per point,
 * see hy_set_geometry). The double-float action of FC/SC/NC has no general build (HY_ERR_UNSUPPORTED with
 * fine_dtype = HY_FF). Takes effect at the next hy_set_displacement (and for hy_residual at once).
 * HY_ERR_ARG for another value. */
typedef enum { HY_LAW_LOG2 = 0, HY_LAW_J2 = 1 } hy_law;
hy_status hy_set_material_law(hy_ctx *ctx, int law);

/* Curved cells (the paper's meshes are curved, Sec. 7): X_dev holds the finest level's nodal coordinates
 * (device FP64, n_dofs values interleaved like a displacement) of an isoparametric Q_k map of the lattice
 * cells; coarser levels get their coordinates by the same nodal interpolation that carries the
 * displacement down (Sec. 6). Gradients use dxi/dX = (dX/dxi)^{-1} and the volume weights w_q det(dX/dxi)
 * at every Gauss point. The map enters where the Gauss-point state is formed (state build, residual,
 * diagonal, dense coarse assembly), so it goes through the caching variants T4 and T2 with unchanged
 * applications. FC, SC and NC (the paper's Algorithm 1 is SC) run their general build on curved cells: the
 * state build caches the inverse Jacobian dxi/dX and the weight w_q det(dX/dxi) of every Gauss point (as
 * the paper's matrix-free operators keep the mapping data of curved cells per quadrature point), d^2 + 1
 * values beside the variant's own; the application maps its unit-cell gradients with them. Not with the
 * double-float action (HY_ERR_UNSUPPORTED with fine_dtype = HY_FF). Dead tractions keep the
 * reference measure of the lattice faces (exact for maps that keep the faces in place). NULL returns to
 * the uniform lattice. The coordinates take sum over levels of n_dofs(l) * 8 bytes beyond hy_footprint,
 * and so do the extra cached values of FC/SC/NC.
 * Takes effect at the next hy_set_displacement (and for hy_residual at once). */
hy_status hy_set_geometry(hy_ctx *ctx, const double *X_dev);

/* Failure-path check of the bounded device waits (no counterpart in the paper). Every wait of the
 * tangent-action kernels on a bulk copy is bounded by GPU wall time (4 s) and a poll count; when one
 * gives up, the kernel flags the context's error word, lets its copies land and returns, and the next
 * synchronising call reports HY_ERR_TIMEOUT. This call runs one thread block whose wait can never
 * complete (nothing arrives on its barrier), with the wall-time bound limit_s in [1e-3, 10] seconds.
 * It returns HY_ERR_TIMEOUT once the wait has given up, with the error word cleared and the context
 * usable; HY_ERR_STATE before hy_mesh_setup; HY_ERR_ARG for limit_s out of range. */
hy_status hy_check_bounded_wait(hy_ctx *ctx, double limit_s);

/* Linearisation point (Sec. 6). u_dev: fine-level FP64 displacement (device). The displacement is
 * carried down to every level by nodal interpolation and each level's Gauss-point cache is built
 * for `variant` from FP64 kinematics (F, J, ln J). level_dtype = HY_F32 selects the mixed-precision
 * V-cycle (FP32 caches, smoother, transfers on every level but the coarsest, which stays FP64; the
 * finest level gets both an FP64 and an FP32 cache). Also builds the level diagonals and the
 * smoother / coarse-solver eigenvalue estimates. Returns HY_ERR_JNEG if J <= 0 anywhere. */
hy_status hy_set_displacement(hy_ctx *ctx, const double *u_dev, hy_variant variant, hy_dtype level_dtype);

/* y = A(u) x on the finest level (Eq. algebraic_tangent applied as in Eq. mf_vmult), with the
 * Dirichlet treatment A~ = Z A Z + (I - Z): x is read as zero on constrained dofs and y equals x
 * there. dtype selects the FP64 or FP32 cache (the FP32 one exists after set_displacement with
 * HY_F32), or HY_FF the double-float one (exists after set_displacement with the solver parameter
 * fine_dtype = HY_FF; FP64 vectors). x_dev and y_dev are device arrays of n_dofs elements of that type
 * (FP64 for HY_FF); they must not alias. HY_ERR_STATE if the requested cache does not exist. */
hy_status hy_apply_tangent(hy_ctx *ctx, const void *x_dev, void *y_dev, hy_dtype dtype);

/* Same on any level (the level operators of the V-cycle, Sec. 6). */
hy_status hy_vmult(hy_ctx *ctx, int level, const void *x_dev, void *y_dev, hy_dtype dtype);

/* r = F(u) of Eq. weak_form (no traction term), FP64, zero on constrained rows; u_dev and r_dev are
 * fine-level FP64 device vectors. HY_ERR_JNEG if J <= 0 at a Gauss point. */
hy_status hy_residual(hy_ctx *ctx, const double *u_dev, double *r_dev);

/* Diagonal of the constrained level operator (1 on constrained dofs), as used by the Chebyshev
 * smoother (Sec. 7); d_dev holds n_dofs(level) elements of dtype. */
hy_status hy_diagonal(hy_ctx *ctx, int level, void *d_dev, hy_dtype dtype);

/* One V-cycle of the geometric multigrid preconditioner (Secs. 6-7) on the finest level:
 * z = V r for FP64 device vectors r, z (zero initial guess, constrained entries of z zero). */
hy_status hy_gmg_vcycle(hy_ctx *ctx, const double *r_dev, double *z_dev);

/* Solver knobs (Sec. 7 defaults in brackets). */
typedef struct {
  int cheb_degree;          /* [4]   Chebyshev degree of the level smoother */
  int cheb_sweeps;          /* [1]   smoother applications per pre-/post-smoothing */
  double cheb_lo;           /* [0.6] lower end of the smoothing range, times lambda_max */
  double cheb_hi;           /* [1.2] upper end, times lambda_max */
  int eig_iters;            /* [30]  CG iterations of the lambda_max estimate */
  int coarse_eig_iters;     /* [0 = number of free coarse dofs] CG iterations on the coarsest level */
  double coarse_reduction;  /* [1e-3] residual reduction of the coarse Chebyshev solve */
  int coarse_solver;        /* [0] 0 = Chebyshev as a solver (Sec. 7); 1 = exact: the coarsest tangent
                               assembled densely and inverted (Gauss-Jordan) once per linearisation,
                               applied as one matrix-vector product (coarsest level <= 6000 dofs,
                               any degree); 2 = as 1 with the inversion in double-float
                               arithmetic on the FP32 pipe (about 48 significant bits; the applied inverse
                               and the matrix-vector product are FP64) */
  int kernel_form;          /* [-1] tangent-action kernel: 0 = one thread per (cell, Gauss point), 1 = one
                               thread per x-line of a cell, 2 = as 1 on a persistent grid whose thread
                               blocks copy their next cache chunk in while finishing the current one (FP32;
                               runs as 1 in the other precisions), 3 = one thread per z-plane of a cell, only
                               the z direction exchanged through shared memory (FP32 in 3D, degrees 1-2;
                               runs as 1 elsewhere), -1 = autotuned: the first linearisation
                               of each (dim, degree, variant, precision, mesh size) times the forms on the
                               level's own cache and keeps the fastest (process-wide; when the environment variable
                               HY_TUNE_FILE names a file, the decisions are read from it at the first tuning
                               and it is rewritten, as a JSON array, with every new decision) */
  hy_dtype fine_dtype;      /* [HY_F64] tangent action of the finest level inside the solver (outer CG, and the
                               finest level of an FP64 V-cycle): HY_F64, or HY_FF to build a double-float
                               cache of the finest level at hy_set_displacement and use it there (every
                               degree; with curved cells or the second law only for T4/T2: the general
                               builds of FC/SC/NC have no double-float action); HY_FF also sums the level
                               diagonals' (node, Gauss point) pairs in double-float */
  int level_variant;        /* [-1] tangent variant of the V-cycle's level operators (every level below the
                               finest, and the finest level's FP32 cache): -1 = the variant given to
                               hy_set_displacement, else a hy_variant. The variants are implementations of
                               one operator (Sec. 5): a cheaper one speeds up the smoother without changing
                               the preconditioner beyond rounding. */
  double setup_reuse;       /* [0 = off] reuse of the V-cycle's setup across linearisations: when the
                               coarsest level's carried-down displacement differs from the one of the last
                               full setup by at most setup_reuse (relative, Euclidean norm), hy_set_displacement
                               keeps that setup's eigenvalue estimates (smoother ranges, Chebyshev coarse
                               bounds) and exact coarse inverse; the level caches, diagonals and the V-cycle
                               graph are rebuilt as always. The V-cycle stays a fixed SPD preconditioner of
                               the current tangent, so the outer CG converges to the same tolerance; only its
                               iteration count can change. Not in the paper, which sets up every
                               linearisation. */
} hy_solver_params;

/* Replace the context's solver parameters (copied); they take effect at the next hy_set_displacement.
 * HY_ERR_ARG for a value out of the ranges above. */
hy_status hy_set_solver_params(hy_ctx *ctx, const hy_solver_params *p);
/* Copy the context's current solver parameters (the defaults above before any hy_set_solver_params). */
hy_status hy_get_solver_params(const hy_ctx *ctx, hy_solver_params *p);

/* Estimates held by the context after set_displacement: lmax of level `level` (levels >= 1), and
 * for the coarsest level its Chebyshev interval [lo, hi] and degree. Any output may be NULL. */
hy_status hy_level_info(const hy_ctx *ctx, int level, double *lmax, double *coarse_lo, double *coarse_hi,
                        int *coarse_degree);
/* Override the estimates (levels >= 1: lmax; level 0: lo, hi), e.g. to mirror another solver. */
hy_status hy_set_level_info(hy_ctx *ctx, int level, double lmax, double coarse_lo, double coarse_hi);

/* Tangent-action kernel form used on a level for a precision (0 point, 1 line, 2 persistent line, 3 plane;
 * see kernel_form), or -1
 * when that level has no cache of that precision. */
hy_status hy_kernel_form(const hy_ctx *ctx, int level, hy_dtype dtype, int *form);

/* Copy the level-`level` displacement (the carried-down linearisation point) into u_dev (FP64). */
hy_status hy_level_displacement(const hy_ctx *ctx, int level, double *u_dev);

/* Transfers between level l-1 (coarse) and l (fine), constrained entries zeroed (Sec. 6):
 * fine += P coarse (prolongate_add) and coarse = P^T fine (restrict). dtype as for the level. */
hy_status hy_prolongate_add(hy_ctx *ctx, int fine_level, const void *coarse_dev, void *fine_dev, hy_dtype dtype);
/* (restrict: see above) */
hy_status hy_restrict(hy_ctx *ctx, int fine_level, const void *fine_dev, void *coarse_dev, hy_dtype dtype);

/* Preconditioned CG (FP64) on the finest level: A~ x = b with the V-cycle preconditioner, zero
 * initial guess, stop at ||r|| <= rtol ||b||. iterations may be NULL. HY_ERR_NOCONV at max_iter. */
hy_status hy_pcg(hy_ctx *ctx, const double *b_dev, double *x_dev, double rtol, int max_iter, int *iterations);

/* Newton-Raphson with load steps (Sec. 3, Sec. 7). */
typedef struct {
  int load_steps;            /* [5] prescribed values reached in equal increments */
  int max_newton;            /* [25] per load step */
  double newton_rtol;        /* [1e-10] ||R_free|| <= rtol * ||first right-hand side of the step|| */
  double newton_atol;        /* [1e-14] or ||R_free|| <= atol */
  double cg_rtol;            /* [1e-8] */
  int cg_max_iter;           /* [1000] */
  hy_variant variant;        /* [HY_T4] tangent variant of every level */
  hy_dtype level_dtype;      /* [HY_F64] HY_F32 = mixed-precision V-cycle */
  double face_values[6][3];  /* final prescribed displacement per face and component */
  double face_traction[6][3]; /* final dead traction per face (reference configuration, per unit reference
                                 area), reached in the same increments; [0] = none. The paper loads its
                                 benchmark this way (Sec. 7); the tangent is unchanged by a dead load. */
  int first_step;            /* [0 = 1] checkpoint / resume: run load steps first_step .. last_step of the
                                load_steps increments only. u_inout_dev then holds on entry the converged
                                state after step first_step - 1 (zero for step 1); a solve stopped after a
                                step and resumed from its u (saved anywhere, in any context of the same
                                problem) continues the same load path. */
  int last_step;             /* [0 = load_steps] */
} hy_newton_params;

typedef struct {
  int load_steps_done;        /* the last load step completed (an absolute step number) */
  int newton_iterations[64];  /* per load step (first 64 steps) */
  int cg_iterations_total;
  int cg_iterations_max;
  double final_residual;      /* ||R_free|| at the end */
  int backtracks;             /* J <= 0 halvings taken */
  int n_solves;               /* linear (PCG) solves performed; the first 256 are recorded below */
  int solve_cg_iterations[256];
  double solve_ms[256];       /* host wall time of each PCG solve (stream synchronised) */
  double setup_ms_total;      /* time spent linearising (caches, diagonals, eigenvalue estimates) */
  double total_ms;            /* whole call */
  int setups_reused;          /* linearisations that kept the previous V-cycle setup (solver setup_reuse) */
  double setup_phase_ms[6];   /* device time of the linearisations' phases, summed: carry the displacement
                                 down; Gauss-point states and diagonals; kernel-form autotuning; smoother
                                 eigenvalue estimates; coarse setup on the context's stream (the wait for the
                                 exact inverse, or the coarse eigenvalue estimate); and, measured on the side
                                 stream where it overlaps the others, the exact coarse inverse itself */
} hy_newton_report;

/* Fill p with the defaults in brackets above (zero tractions and prescribed values). */
void hy_newton_default_params(hy_newton_params *p);
/* Solve for the equilibrium displacement: u_inout_dev (fine FP64, device) holds the start state on
 * entry (its constrained values are overwritten by the load path) and the solution on return; on
 * error it holds the last accepted iterate. rep may be NULL. */
hy_status hy_newton_solve(hy_ctx *ctx, const hy_newton_params *p, double *u_inout_dev, hy_newton_report *rep);

/* External force of dead tractions on the finest level: f_dev = sum over faces of t_face * int_face N_a dA
 * (the surface term of Eq. weak_form), t_face = traction[face][component] (HOST, faces -x, +x, -y, +y, -z,
 * +z). f_dev: device FP64 vector of n_dofs, overwritten (constrained dofs included). */
hy_status hy_face_load(hy_ctx *ctx, const double traction[6][3], double *f_dev);

/* Deterministic FP64 dot product of two fine-level device vectors (fixed reduction order, so
 * repeated calls give identical bits). Uses a scratch buffer owned by the context. */
hy_status hy_dot(hy_ctx *ctx, const double *a_dev, const double *b_dev, int64_t n, double *result);

/* Allocation-free dot product, for callers that must not allocate device memory while they run
 * (for example code that works inside a device-memory budget another framework has fully claimed,
 * or a real-time loop in which a cudaMalloc/cudaFree could stall on a device synchronisation). The
 * paper has no counterpart: it is a service of this library, not a step of the method. It needs no
 * context: it runs on `device` and enqueues on `cuda_stream` (NULL = legacy default stream), writes
 * a . b for the FP64 device vectors a_dev, b_dev of n elements to the HOST double *result and
 * synchronises the stream before returning. Its scratch is a fixed array inside the library (about
 * 128 KiB per device, held until the process exits); n > HY_DOT_NOALLOC_MAX_N returns HY_ERR_ARG.
 * The first call on each device looks up that array's device address, so make it before any stream
 * capture. All calls share the array: calls that overlap on the GPU (different streams without
 * ordering) race; serialise them. The summation order is fixed, so repeated calls agree bitwise. The
 * calling thread's current device is the same after the call as before it. */
#define HY_DOT_NOALLOC_MAX_N (16384LL * 4096LL) /* 67,108,864 elements */
hy_status hy_dot_noalloc(int device, void *cuda_stream, const double *a_dev, const double *b_dev, int64_t n,
                         double *result);

/* Device bytes a context will own for this problem after mesh setup and set_displacement (the
 * admission measure of the solve server); pure host arithmetic, no GPU needed. sp: the solver parameters
 * the context will use (NULL: the defaults). face_masks[2*dim] (may be NULL: then an upper bound) fixes the
 * free dofs of an exact coarse solve. */
hy_status hy_footprint(int dim, int degree, int cells_per_dir, int n_levels, hy_variant variant,
                       hy_dtype level_dtype, const hy_solver_params *sp, const uint32_t *face_masks, int64_t *bytes);

/* Device bytes currently owned by the context (its hierarchy, caches and work vectors). */
hy_status hy_ctx_bytes(const hy_ctx *ctx, int64_t *bytes);

/* Number of kernels this context has launched since creation (for accounting). */
hy_status hy_kernel_launches(const hy_ctx *ctx, int64_t *count);

/* ---- Work-list batches ---------------------------------------------------------------------------
 * Several independent problems of the same dimension and degree (each a context with its own mesh size,
 * material and linearisation) advanced together. Not a step of the paper's method: it batches the
 * method's operator action (Eq. mf_vmult) and its preconditioned CG (Sec. 6) across problems, so that
 * many problems too small to fill the GPU share its SMs.
 *  - The finest-level tangent actions of all problems run as ONE kernel launch over a work list of
 *    per-problem arguments (thread blocks are dealt to the problems in order, each problem keeping the
 *    cell blocks and Gauss-point cache layout of its own context).
 *  - hy_batch_pcg advances every not-yet-converged problem by one PCG iteration per replay of a CUDA
 *    graph (the list launch, then one branch per problem with its dot products, updates and V-cycle,
 *    all CG scalars on the device), with one host synchronisation per iteration for the whole batch; the
 *    graph is captured again only when a problem leaves the resident set (converged or failed).
 * The batch borrows the contexts (it does not own them; destroy it first) and runs on a stream of its
 * own, ordered after the work queued on each context's stream at each call and before work queued
 * there afterwards. A batch is not thread-safe; the contexts must not be used by another thread during
 * a batch call. All contexts must have had hy_set_displacement with the same variant. */
typedef struct hy_batch hy_batch;
#define HY_BATCH_MAX 1024

/* Group count distinct contexts (same device, dimension and degree, mesh set up). HY_ERR_ARG for an
 * empty, oversized, mixed or repeated list; HY_ERR_STATE for a context without a mesh. */
hy_status hy_batch_create(hy_batch **out, hy_ctx *const *ctxs, int count);
/* Free the batch's graphs, streams and buffers (the contexts stay). NULL is accepted. */
void hy_batch_destroy(hy_batch *b);
/* Message of the batch's most recent failed call; owned by the batch. NULL batch: "null batch". */
const char *hy_batch_last_error(const hy_batch *b);

/* y_i = A~_i x_i on the finest level of every context i, in one list launch (as hy_apply_tangent,
 * dtype HY_F64 or HY_F32; the context needs a finest-level cache of that precision). x_dev[i], y_dev[i]:
 * device vectors of context i's finest level (distinct). The kernel form of the list launch is timed on
 * the first call per precision unless the first context's kernel_form parameter forces one. */
hy_status hy_batch_apply(hy_batch *b, const void *const *x_dev, void *const *y_dev, hy_dtype dtype);

/* hy_pcg for every context i at once: A~_i x_i = b_i, zero initial guess, ||r_i|| <= rtol ||b_i||.
 * iterations[count] and status[count] receive each problem's iteration count and outcome (HY_OK,
 * HY_ERR_NOCONV at max_iter or for a non-SPD operator, HY_ERR_TIMEOUT, ...), with the message in that
 * context's hy_last_error. The return value reports failures of the batch itself (launch, capture). */
hy_status hy_batch_pcg(hy_batch *b, const double *const *b_dev, double *const *x_dev, double rtol, int max_iter,
                       int *iterations, hy_status *status);

/* Kernels launched by the batch's own calls (list launches and graph replays). */
hy_status hy_batch_kernel_launches(const hy_batch *b, int64_t *count);
/* Kernel form chosen for the list launch of a precision (0 point, 1 line, -1 not chosen yet). */
hy_status hy_batch_kernel_form(const hy_batch *b, hy_dtype dtype, int *form);

/* ---- Solve server (continuous batching of many independent solves on one GPU) --------------------
 * Not a step of the paper's method: a request loop around hy_newton_solve. Requests are queued in
 * arrival order; `max_active` worker threads, each with its own CUDA stream, admit the head of the
 * queue as soon as a worker is free and its hy_footprint fits the remaining `hbm_budget_bytes` (the head
 * is never bypassed). An admitted request keeps its hierarchy and Newton state resident on the device
 * until its solve ends; requests admitted while others run overlap with them on the device. */
typedef struct hy_server hy_server;

typedef struct {
  int dim, degree, cells_per_dir, n_levels;
  uint32_t face_masks[6];
  const uint8_t *cell_mat_levels; /* HOST: material ids of every level, coarsest first, concatenated */
  const double *mu, *lambda;      /* HOST: per material id */
  int n_mat;
  hy_newton_params newton;        /* load path, tolerances, variant, V-cycle precision */
  hy_solver_params solver;
  int law;                        /* hy_law of the material */
  const double *u_start;          /* HOST, NULL = zero: the start state (n_dofs values, copied at submit);
                                     with newton.first_step > 1 it re-admits a checkpoint, e.g. the u of an
                                     earlier request that stopped at newton.last_step */
} hy_request;

typedef struct {
  int64_t submitted, completed, failed, active, queued;
  int64_t bytes_in_use, bytes_peak, budget;
  int64_t retried;  /* solves run again with the coarsest level dropped: a solve that fails only on a
                       coarsest-level tangent that is not positive definite (a coarse mesh that does not
                       resolve the inclusion, Sec. 6) reruns from its start state with one level fewer, while
                       two levels remain and the budget holds the larger coarse level (Chebyshev coarse
                       solve when it exceeds the dense-inverse limit) */
  int64_t batched_solves; /* batched serving: outer linear solves that went through the batcher */
  int64_t batch_runs;     /* batched serving: work-list batches run (batched_solves / batch_runs = the mean
                             number of solves fused per batch) */
} hy_server_stats;

/* Start a server on `device` with `max_active` workers (1..64), admitting requests while their summed
 * footprints stay within hbm_budget_bytes. HY_ERR_ARG for a bad device, budget or worker count. */
hy_status hy_server_create(hy_server **out, int device, int64_t hbm_budget_bytes, int max_active);
/* Batched serving (call before the first submit; HY_ERR_STATE afterwards or when already enabled). Not a
 * step of the paper: it fuses the paper's matrix-free operator action (Eq. mf_vmult) and its GMG-
 * preconditioned CG (Secs. 6-7) across requests. Each worker still linearises its own request on its own
 * stream, but its outer CG solves go to a batcher, which waits until every running Newton solve has a
 * solve waiting or window_ms (0..1000) has passed since the oldest arrived, groups the waiting solves by
 * dimension, degree, cache variants, finest-level precision, CG tolerance and cap and size (within a factor
 * of 4 in dofs: a batch returns when its slowest member has converged), and runs every group as
 * one work-list batch (hy_batch_pcg: one graph replay per PCG iteration with ONE kernel launch for the
 * finest-level tangent actions of all members and their V-cycles as concurrent branches). Groups of
 * different degree run side by side. Results are those of the requests' own PCG (the same arithmetic per
 * problem). HY_ERR_ARG for a bad window. */
hy_status hy_server_set_batching(hy_server *s, int enable, double window_ms);
/* Running requests finish; queued ones are dropped. */
void hy_server_destroy(hy_server *s);
/* Copies the request and returns at once. HY_ERR_OOM if its footprint exceeds the whole budget. */
hy_status hy_server_submit(hy_server *s, const hy_request *r, uint64_t *ticket);
/* state: 0 queued, 1 running, 2 done, 3 failed (the call then returns the solve's status). When done,
 * rep, the solution u_host (n_u doubles, may be NULL) and the submit-to-completion latency are filled. */
hy_status hy_server_poll(hy_server *s, uint64_t ticket, int *state, hy_newton_report *rep, double *u_host,
                         int64_t n_u, double *latency_ms);
/* Block the calling thread until the request has finished, or HY_ERR_TIMEOUT after timeout_s seconds. */
hy_status hy_server_wait(hy_server *s, uint64_t ticket, double timeout_s);
/* Forget a finished request (frees its host copy of the solution). */
hy_status hy_server_release(hy_server *s, uint64_t ticket);
/* Counters and device bytes of the server (a consistent snapshot). */
hy_status hy_server_stats_get(hy_server *s, hy_server_stats *st);

#ifdef __cplusplus
}
#endif
#endif /* HYPERELASTIC_H */
