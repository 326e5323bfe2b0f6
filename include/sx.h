/*
 * sx.h -- C ABI of libsx, a GB300 (sm_103a) implementation of the hot path
 * of the energy-based optimization time integrator of "SymX:
 * Energy-based Simulation from Symbolic Expressions" (arXiv 2303.02156).
 *
 * The calls follow the paper's statement of the problem: register degrees
 * of freedom (§5.1, Fig. 2 "add_dof_array"), add energies over element
 * lists with per-element parameters (§3 Eq. 5; §5.1 "add_energy"),
 * evaluate the global energy, gradient and Hessian at three levels
 * (§5.2 "Data-Symbol Mapping": E for the line search, E+grad for the
 * convergence test, E+grad+Hessian for the Newton system), with optional
 * per-element projection to positive semi-definiteness (§5.2, Algorithm 1),
 * assembled into a 3x3 block CRS matrix (§5.3, Eq. 11), and take a
 * backward-Euler step by Newton's method (§3, Eqs. 2-3) with a 3x3
 * block-Jacobi PCG linear solve (§7.2).
 *
 * Conventions (all calls):
 *  - Every call returns an int status: SX_OK (0) or a negative SX_E* code;
 *    sx_last_error(ctx) gives a one-line description of the last failure.
 *    No C++ exception crosses this boundary.
 *  - Input arrays may be host or device pointers (any address CUDA's
 *    unified addressing resolves, pinned or pageable host memory included);
 *    outputs of sx_eval_elements and the sx_get_* views are device memory.
 *  - Inputs are copied into library-owned device memory; the library never
 *    keeps a caller pointer past the call.
 *  - Pointers returned by sx_get_* are views into library memory, valid
 *    until the next call that mutates that scene.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Calls that
 *    return a host-side value (energy, report, footprint) synchronize that
 *    stream; the others are asynchronous unless stated.
 *  - Node arrays are AoS: node n's coordinates at [3n, 3n+2]. Stencils are
 *    int32[n][4]. Per-element parameters are one value per element.
 *  - A context is not thread-safe; use one context per host thread.
 *  - All scenes of a context live on the device that was current at
 *    sx_create.
 */
#ifndef SX_H
#define SX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define SX_OK 0
#define SX_EINVAL (-1)        /* bad argument */
#define SX_ENOMEM (-2)        /* device allocation failed */
#define SX_ECUDA (-3)         /* a CUDA runtime call failed */
#define SX_ENAN (-4)          /* non-finite energy, gradient or Hessian */
#define SX_ENOTCONV (-5)      /* PCG or Newton iteration limit reached */
#define SX_ESTATE (-6)        /* state outside the energy's domain (barrier d <= 0) */
#define SX_EDEGENERATE (-7)   /* a rest element has non-positive volume */
#define SX_EBUDGET (-8)       /* request can never fit the server's memory budget */
#define SX_ELINESEARCH (-9)   /* line search found no decrease */
#define SX_EORDER (-10)       /* call out of order (e.g. eval before finalize) */

/* ---- evaluation levels (§5.2: three global evaluation functions) ------ */
#define SX_E 0      /* energy */
#define SX_EG 1     /* energy + gradient */
#define SX_EGH 2    /* energy + gradient + Hessian */

/* ---- element-math precision ------------------------------------------ */
#define SX_FP64 0   /* all arithmetic in double */
#define SX_FP32 1   /* element E/g/H and SpMV in float; the PSD projection,
                       gradient assembly, energy sums, residual norms and PCG
                       dot products stay in double */

/* PSD projection modes (sx_eval) */
#define SX_PROJECT_NONE 0
#define SX_PROJECT_ELEMENT 1
#define SX_PROJECT_MATERIAL 2

/* ---- energy kinds ----------------------------------------------------- */
#define SX_KIND_SNH_TET4 0     /* linear tets of any SX_MODEL_* density */
#define SX_KIND_TET4 SX_KIND_SNH_TET4
#define SX_KIND_HINGE4 1
#define SX_KIND_PT_BARRIER 2
#define SX_KIND_PT_FRICTION 3
#define SX_KIND_TET_HO 4       /* 10- or 20-node tets (sx_add_tet_ho) */
#define SX_HO_MAX_QP 64        /* quadrature points per high-order rule */

/* ---- tet4 densities (§6.1 "Non-Linear Material Models", App. B) -------
 * SNH    Stable Neo-Hookean (§3.1 Eq. 7), parameters mu', lambda' as in
 *        sx_add_snh_tet4;
 * NH     Neo-Hookean mu/2 (Ic - 3) - mu ln J + lambda/2 ln^2 J (the text
 *        form of §3.1 prints +mu ln J; the minus sign is the one whose rest
 *        state is stress-free); J <= 0 is an invalid state (SX_ESTATE, like
 *        a barrier pair at d <= 0);
 * STVK   St. Venant-Kirchhoff mu |E|^2 + lambda/2 tr(E)^2, E = (F^T F - I)/2;
 * COROT  fixed co-rotational mu |F - R|^2 + lambda/2 (J - 1)^2;
 * ARAP   as-rigid-as-possible with a volume term
 *        mu/2 |F - R|^2 + lambda/2 (J - 1)^2.
 * COROT and ARAP use a lagged rotation R per tet (constant within a time
 * step, §6.1; not differentiated): the rotation of the polar decomposition
 * of F, taken at the start of every Newton step and by
 * sx_update_rotations; the identity when the block is added. */
#define SX_MODEL_SNH 0
#define SX_MODEL_NH 1
#define SX_MODEL_STVK 2
#define SX_MODEL_COROT 3
#define SX_MODEL_ARAP 4

typedef struct sx_ctx sx_ctx;
typedef struct sx_scene sx_scene;
typedef struct sx_server sx_server;

typedef struct {
    int device;          /* CUDA device ordinal; -1 = the current device */
    int share_sms;       /* 1: the register-heavy kernels (element evaluation,
                            projection) leave room on every SM -- one block of
                            each per SM less than fits -- so that work of other
                            contexts on higher-priority streams (the serving
                            lanes of smaller scenes) is not held behind their
                            long-lived blocks; costs throughput. 0: default. */
    int reserved[6];
} sx_options;

/* Create / destroy a context. */
int sx_create(sx_ctx** ctx, const sx_options* opt);
int sx_destroy(sx_ctx* ctx);
const char* sx_last_error(sx_ctx* ctx);

/* Fault injection for tests of the failure paths (the paper has no
 * counterpart): the n-th device allocation that a scene of this context
 * makes from now on fails as if the device were out of memory (n = 0
 * disarms). The call that meets it returns SX_ENOMEM and leaves the context
 * and its other scenes usable; a finalize that fails this way leaves its
 * scene unfinalized, so it can be retried. Host-side only: no GPU fault is
 * involved. */
int sx_inject_alloc_failure(sx_ctx* ctx, int n);
/* Library build string (arch, version); never NULL. */
const char* sx_version(void);

/* ---- scenes and DOF registration (§5.1 Fig. 2 "add_dof_array";
 *      §5.3 concatenated DOF sets, Eq. 11) ---------------------------------
 * A scene holds one global DOF vector of n_nodes 3D nodes; several DOF
 * sets (a tet mesh, a shell, free points) are registered by stacking them
 * into one node range, as §5.3 concatenates DOF sets. X_rest: rest
 * positions, n_nodes x 3 doubles, node stride `stride` doubles (>= 3);
 * host or device. The deformed state starts at X_rest with zero velocity. */
int sx_scene_create(sx_ctx* ctx, int64_t n_nodes, const double* X_rest,
                    int64_t stride, void* stream, sx_scene** scene);
int sx_scene_destroy(sx_scene* scene);

/* Stable Neo-Hookean linear tets (§3.1 Eq. 7; App. B density). tets: n x 4
 * node ids; young, poisson: per-element Young's modulus (Pa) and Poisson
 * ratio. Rest precompute on the device: Dm = [X1-X0,
 * X2-X0, X3-X0], Dm^-1, V = det(Dm)/6 > 0 (else SX_EDEGENERATE and the
 * block is not added), lumped mass rho V / 4 per vertex, and the density's
 * parameters mu' = 4 mu / 3, lambda' = lambda + 5 mu / 6 from the
 * isotropic Lame pair (literal_params != 0: mu' = mu, lambda' = lambda).
 * Synchronous. energy_id (may be NULL) receives the block's id. */
int sx_add_snh_tet4(sx_scene* scene, const int32_t* tets, int64_t n,
                    const double* young, const double* poisson, double density,
                    int literal_params, void* stream, int* energy_id);

/* Linear tets of density `model` (SX_MODEL_*). Arguments and rest
 * precompute as sx_add_snh_tet4; SX_MODEL_SNH takes the re-parameterized
 * (mu', lambda'), the other models the plain Lame pair (mu, lambda).
 * SX_EINVAL for an unknown model. Synchronous. */
int sx_add_tet4(sx_scene* scene, int model, const int32_t* tets, int64_t n,
                const double* young, const double* poisson, double density, void* stream,
                int* energy_id);

/* High-order Lagrange tets (§6.2 Eq. 12; App. A shape functions)
 * with the Stable Neo-Hookean density (mu', lambda' as in sx_add_snh_tet4):
 * E_e = sum_q w_q det J0(xi_q) psi(F(xi_q)) over a quadrature rule given by
 * the caller (the fixed-value summation of §5), J0 = sum_a X_a dN_a^T,
 * F = (sum_a x_a dN_a^T) J0^-1. order 2: 10 nodes per tet (the vertices,
 * then one node per edge in the order 01, 12, 20, 03, 13, 23: App. A);
 * order 3: 20 nodes (the vertices; two per edge in that order, first the
 * one nearer the edge's first vertex; one per face in the order 012, 013,
 * 123, 023). tets: n x K node ids; rule: nq x 4 doubles (w, xi0, xi1, xi2)
 * on the reference tet of volume 1/6, 1 <= nq <= SX_HO_MAX_QP; host
 * arrays. Lumped mass rho V_e / K per node (V_e = sum_q w_q det J0);
 * det J0 <= 0 at a point: SX_EDEGENERATE. With projection (sx_eval
 * project != 0) the material Hessian is clamped at every point in closed
 * form (as SX_PROJECT_MATERIAL does for linear SNH tets), so the element
 * Hessian is PSD. For the fixed pattern an element is S four-node
 * sub-stencils that together cover its node pairs (S = 10 for order 2, 38
 * for order 3): sx_block_info and sx_eval_elements count n S stencils, and
 * an element's E, g and H are the sums over its S sub-stencils (each pair
 * block and node gradient is held by exactly one of them). Synchronous. */
int sx_add_tet_ho(sx_scene* scene, int order, const int32_t* tets, int64_t n,
                  const double* young, const double* poisson, double density,
                  const double* rule, int nq, void* stream, int* energy_id);

/* Lagged rotations of the COROT / ARAP blocks of a scene (§6.1).
 * sx_update_rotations: R of every tet of those blocks := the rotation of
 * the polar decomposition of F at the current state (F = U S V^T with
 * singular values in descending order, R = U V^T, the column of U of the
 * smallest singular value negated if that makes R a rotation; the identity
 * for F = 0). Stream-ordered.
 * sx_get_rotations / sx_set_rotations: n x 9 doubles (row-major 3x3 per
 * tet) of block `energy_id` (COROT / ARAP, else SX_EINVAL), host or
 * device; get synchronizes `stream`. */
int sx_update_rotations(sx_scene* scene, void* stream);
int sx_get_rotations(sx_scene* scene, int energy_id, double* R, void* stream);
int sx_set_rotations(sx_scene* scene, int energy_id, const double* R, void* stream);

/* Quadratic hinge bending E = k_b/2 x^T Q x (§6.3, Eq. 13) over 4-node
 * stencils (e0, e1, o0, o1): shared edge then the two opposite vertices.
 * Q = c (q q^T kron I3) with q (n x 4) the per-stencil weights and c (n)
 * the per-stencil scale (for Bergou et al.'s form, cotangent
 * weights and 3/(A0+A1)). Q is constant and PSD, so it is never projected.
 * Synchronous. */
int sx_add_hinge4(sx_scene* scene, const int32_t* stencils, int64_t n,
                  const double* q, const double* c, double k_b, void* stream,
                  int* energy_id);

/* Point-triangle IPC barrier E = -kappa (d - dhat)^2 ln(d / dhat) of the
 * unsigned distance d between point p and triangle (t0, t1, t2) (§6.4,
 * Eq. 15); active only for 0 < d < dhat (conditional evaluation, §5.2
 * Eq. 9), inactive pairs contribute zero and keep their (zero) blocks in
 * the fixed pattern. pairs: n x 4 = (p, t0, t1, t2). A state with
 * d <= 0 makes sx_eval return SX_ESTATE. Synchronous. */
int sx_add_pt_barrier(sx_scene* scene, const int32_t* pairs, int64_t n,
                      double dhat, double kappa, void* stream, int* energy_id);

/* Lagged IPC friction on point-triangle pairs (§6.4, friction potential).
 * Per pair (p, t0, t1, t2): E = mu fn f0(|T (dx - dx_lag)|), where
 * dx = p - sum_i beta_i t_i is the separation at the lagged contact point,
 * f0(s) = dt f(s / dt) and f(y) = -y^3/(3 yh^2) + y^2/yh + yh/3 for
 * y <= yh, y otherwise (yh = yhat: the stick/slide velocity threshold), so
 * that a sliding pair feels the Coulomb force mu fn. Lagged per pair by
 * sx_update_friction and at the start of every Newton step (with the
 * step's dt): the closest point's barycentric weights beta, an orthonormal
 * basis T (2 x 3) of the plane normal to p - c, the contact force
 * fn = -b'(d) of the barrier b(d) = -kappa (d - dhat)^2 ln(d / dhat) at
 * d = |p - c| (0 outside 0 < d < dhat) and dx_lag = p - c. Until the first
 * lag fn = 0 (no friction). The Hessian is PSD by construction and never
 * projected. mu >= 0, yhat > 0, dhat > 0, kappa >= 0. Synchronous. */
int sx_add_pt_friction(sx_scene* scene, const int32_t* pairs, int64_t n, double mu,
                       double yhat, double dhat, double kappa, void* stream, int* energy_id);
/* Lag every friction block of the scene at its current state with time
 * step dt > 0 (stream-ordered). */
int sx_update_friction(sx_scene* scene, double dt, void* stream);
/* The lag of friction block `energy_id` (host or device arrays, any may be
 * NULL): beta n x 3, T n x 6 (two rows), fn n, dx_lag n x 3. Synchronizes
 * `stream`. */
int sx_get_friction_lag(sx_scene* scene, int energy_id, double* beta, double* T, double* fn,
                        double* dx_lag, void* stream);

/* Add per-node mass (n_nodes doubles) to the lumped mass, e.g. for shell
 * vertices or free points that belong to no tet. Synchronous. */
int sx_add_node_mass(sx_scene* scene, const double* mass, void* stream);

/* Pinned (Dirichlet) nodes: their DOFs are eliminated from the Newton
 * system (identity rows) and never move. nodes: n node ids; replaces any
 * earlier set. Synchronous. */
int sx_set_pinned(sx_scene* scene, const int32_t* nodes, int64_t n, void* stream);

/* Constant external acceleration (M^-1 f_ext of Eq. 2), host double[3]. */
int sx_set_gravity(sx_scene* scene, const double g[3]);

/* Build the fixed 3x3-block CRS pattern (union of all stencils' node pairs
 * plus every diagonal; columns ascending; full storage), the per-stencil
 * slot maps and the assembly lists (§5.3). Must follow the last add_* call
 * and precede any evaluation. Synchronous. */
int sx_finalize(sx_scene* scene, void* stream);

/* ---- changing contact pairs (§5.3: the pattern of a barrier block follows
 *      the active pairs; §6.4, Eq. 15: a pair contributes only while
 *      0 < d < dhat) ------------------------------------------------------
 * Both calls keep the scene's state (x, v), masses, pins and inertia
 * setting, replace the pairs of point-triangle block `energy_id` and, if
 * the scene was finalized, rebuild its pattern, index maps and buffers (a
 * new fixed pattern: blocks of pairs that left disappear, blocks of new
 * pairs appear). Earlier sx_get_* views and assembled outputs are invalid
 * afterwards. Synchronous on `stream`.
 * sx_set_pairs: n new pairs (point, t0, t1, t2), host or device, n >= 0.
 * sx_compact_pairs: keeps, in their order, the pairs that are active at the
 *   current state (0 < d < dhat) or in the error state d <= 0 (so that the
 *   next evaluation still reports SX_ESTATE); *n_active (may be NULL)
 *   receives their number. */
int sx_set_pairs(sx_scene* scene, int energy_id, const int32_t* pairs, int64_t n, void* stream);
int sx_compact_pairs(sx_scene* scene, int energy_id, int64_t* n_active, void* stream);

/* ---- state ------------------------------------------------------------ */
/* x, v: n_nodes x 3 doubles (either may be NULL). */
int sx_set_state(sx_scene* scene, const double* x, const double* v, void* stream);
int sx_get_state(sx_scene* scene, double* x, double* v, void* stream);

/* Enable the inertia term of the incremental potential (Eq. 2):
 * m/(2 dt^2) |x - x_tilde|^2 per node. x_tilde: n_nodes x 3; NULL
 * disables the term. */
int sx_set_inertia(sx_scene* scene, double dt, const double* x_tilde, void* stream);

/* ---- evaluation (§5.2; Algorithm 1) -----------------------------------
 * level: SX_E, SX_EG or SX_EGH. project: SX_PROJECT_NONE, SX_PROJECT_ELEMENT
 * (1: every non-convex element Hessian -- SNH, barrier -- projected to PSD
 * by clamping the eigenvalues of its 12x12 at 0, FP64 always) or
 * SX_PROJECT_MATERIAL (2: for SNH tets the material Hessian d2psi/dF2 is
 * clamped instead, H = V B^T proj(d2psi/dF2) B, in closed form in the frame
 * of the signed SVD of F (FP64) -- a different PSD Hessian, above the plain
 * one, cheaper than the 12x12 clamp; tets of the other models and barriers
 * as in 1). precision: SX_FP64
 * or SX_FP32. E_out (host, may be NULL)
 * receives the total energy; the assembled gradient (FP64) and BSR values
 * stay on the device (sx_get_grad, sx_get_bsr). Synchronous when E_out is
 * given. */
int sx_eval(sx_scene* scene, int level, int project, int precision,
            double* E_out, void* stream);

/* The same for several scenes of one context in one fused launch sequence
 * (persistent element kernel over a tile queue of all their stencils).
 * E_out: host array of n (may be NULL). */
int sx_eval_batch(sx_ctx* ctx, sx_scene* const* scenes, int n, int level,
                  int project, int precision, double* E_out, void* stream);

/* Views of the assembled system after an SX_EG / SX_EGH evaluation.
 * dtype: SX_FP64 (double vals) or SX_FP32 (float vals), the precision of
 * the last SX_EGH evaluation. vals: nnzb blocks x 9, row-major 3x3. */
int sx_get_bsr(sx_scene* scene, const int32_t** row_ptr, const int32_t** col,
               const void** vals, int64_t* nnzb, int* dtype);
int sx_get_grad(sx_scene* scene, const double** grad);
/* Diagonal block index of every node (n_nodes int32). */
int sx_get_diag_slots(sx_scene* scene, const int32_t** diag_slot);

/* Copies of the same data into caller buffers (host or device): row_ptr
 * (n_nodes+1), col (nnzb), vals (nnzb x 9 of the last SX_EGH precision;
 * dtype receives it); grad (n_nodes x 3). Any pointer may be NULL.
 * Asynchronous on `stream` for device or pinned destinations. */
int sx_copy_bsr(sx_scene* scene, int32_t* row_ptr, int32_t* col, void* vals, int* dtype,
                void* stream);
int sx_copy_grad(sx_scene* scene, double* grad, void* stream);

/* Scene shape: node count, BSR block count (0 before sx_finalize), total
 * stencils and energy blocks. Any pointer may be NULL. */
int sx_scene_info(sx_scene* scene, int64_t* n_nodes, int64_t* nnzb, int64_t* n_stencils,
                  int* n_blocks);
/* Kind (SX_KIND_*) and element count of energy block `energy_id`. */
int sx_block_info(sx_scene* scene, int energy_id, int* kind, int64_t* n);
/* Counters of the last evaluation: elements whose Hessian was projected
 * (SX_EGH with project), stencils in an invalid state (barrier pairs with
 * d <= 0, Neo-Hookean tets with J <= 0), non-finite flag.
 * Synchronizes `stream`. */
int sx_eval_stats(sx_scene* scene, int* clamped, int* bad_state, int* nonfinite,
                  void* stream);

/* ---- element-level outputs with global indices (§5.3 last paragraph;
 *      §5.2 low-level API) ---------------------------------------------
 * For energy block `energy_id`, write per element E (n doubles), g
 * (n x 12 doubles), H (n x 144 doubles, row-major 12x12, projected when
 * project != 0) to device buffers, and the block's slot map (n x 16 int32:
 * BSR block index of local node pair (a, b) at 4a + b). Any of E, g, H,
 * slots may be NULL. */
int sx_eval_elements(sx_scene* scene, int energy_id, int project, int precision,
                     double* E, double* g, double* H, int32_t* slots, void* stream);

/* ---- element-level outputs without device allocation -------------------
 * The paper has no counterpart: this entry point exists for callers that
 * cannot let a call allocate device memory -- for example an application
 * whose device memory is already reserved by its own caching allocator,
 * or a fixed-latency simulation loop that must not take the implicit
 * device-wide synchronization of cudaMalloc/cudaFree. It computes exactly
 * what sx_eval_elements computes (same kernels), but all of its scratch
 * (tile table, projection queue of SX_NOALLOC_MAX_ELEMENTS x 45 doubles,
 * counters, scene descriptor) lives in static device arrays of this
 * library, about 25 MB that every GPU which loads the library holds until
 * the process exits. It makes no cudaMalloc/cudaFree call and calls no
 * allocating routine.
 *  - Blocks with more than SX_NOALLOC_MAX_ELEMENTS elements (stencils;
 *    sub-stencils for high-order tets) are rejected with SX_EINVAL, and so
 *    are high-order blocks whose element-kernel tiles (whole elements, up
 *    to 128 threads each) would exceed the static tile table of 512.
 *  - E, g, H: device outputs as in sx_eval_elements (n, n x 12,
 *    n x 144); a NULL E or g sends that output to the scene's own staging
 *    buffers instead. The call synchronizes `stream`.
 *  - The first call on a device looks up the addresses of the static
 *    arrays (cudaGetSymbolAddress) for that device; make that first call
 *    before capturing any stream.
 *  - Every call shares the same static arrays: calls that overlap on the
 *    GPU (other streams, other host threads) race and must be serialized
 *    by the caller. Counters are cleared by each call. */
#define SX_NOALLOC_MAX_ELEMENTS 65536
int sx_eval_elements_noalloc(sx_scene* scene, int energy_id, int project, int precision,
                             double* E, double* g, double* H, void* stream);

/* ---- backward-Euler Newton step (§3 Eqs. 2-3; §7.2 solver) ------------ */
typedef struct {
    double newton_tol;   /* stop when ||g_free|| <= tol * ||g_free(x0)|| */
    double pcg_tol;      /* stop when ||r|| <= tol * ||b|| */
    int max_newton;      /* Newton iteration cap */
    int max_pcg;         /* PCG iteration cap per solve */
    int max_halvings;    /* line-search halvings cap */
    int project;         /* SX_PROJECT_* (see sx_eval) */
    int precision;       /* SX_FP64 or SX_FP32 */
    double armijo_c;     /* sufficient-decrease constant */
    int forcing;         /* 1: PCG stops at ||r|| <= eta_k ||b|| with the forcing
                            sequence eta_k = min(1/2, sqrt(||g_k|| / ||g_0||))
                            (the paper's solver, §7.2; Nocedal-Wright), never
                            below pcg_tol; 0: fixed pcg_tol */
    int graphs;          /* 1: PCG runs in chunks of 8 iterations replayed from
                            one CUDA graph per batch (built from kernel nodes
                            on first use, no stream capture; not while
                            sx_profile is on); 0: plain launches. Results are
                            the same either way. */
} sx_newton_opts;

/* Defaults: 1e-8, 1e-10, 100, 10000, 30, 1, SX_FP64, 1e-4, forcing 0,
 * graphs 1. */
void sx_newton_opts_default(sx_newton_opts* o);

typedef struct {
    int status;          /* SX_OK or the failing code */
    int newton_iters;
    int pcg_iters;       /* total over the step */
    int ls_halvings;     /* total over the step */
    double g0_norm;      /* ||g_free(x0)|| */
    double g_norm;       /* final ||g_free|| */
    double energy;       /* final E_BE */
    double ms;           /* wall time of the step */
} sx_step_report;

/* One step: x_tilde = x + dt v + dt^2 g_ext; x0 = x; Newton with PCG and
 * Armijo backtracking; v = (x - x_t)/dt. A step that fails (any status but
 * SX_OK: non-finite values, an invalid state, an iteration cap, a line search
 * without decrease) is not taken: the scene keeps the x and v it had at the
 * call. Synchronous. */
int sx_newton_step(sx_scene* scene, double dt, const sx_newton_opts* opts,
                   sx_step_report* report, void* stream);

/* Advance a scene by dt with the time-step halving restart of a failed
 * step (§7 experiments: a step whose Newton iteration or line search fails
 * is redone as two steps of half the size): substeps are taken in time
 * order; when one fails to converge (SX_ENOTCONV, SX_ELINESEARCH, SX_ENAN or
 * SX_ESTATE) the scene's x and v are restored to that substep's start and
 * its interval is covered by two substeps of half its size, at most
 * max_dt_halvings levels deep. Other errors return at once. On any failure
 * the state is that of the start of the failed substep (the whole call's
 * start when nothing succeeded), restored from a device snapshot taken
 * before each substep. A successful call clears sx_last_error's text, also
 * when substeps failed on the way. report (may be NULL): status, Newton / PCG /
 * line-search counts summed over the successful substeps, g0_norm of the
 * first, g_norm and energy of the last, ms of the whole call; substeps (may
 * be NULL) receives their number. A checkpoint of a scene is its x and v
 * (sx_get_state / sx_set_state): lagged rotations and friction data are
 * retaken at every step, the rest is fixed at registration. Synchronous. */
int sx_advance(sx_scene* scene, double dt, const sx_newton_opts* opts, int max_dt_halvings,
               sx_step_report* report, int* substeps, void* stream);

/* One step for each of n scenes, batched: every kernel of the Newton and
 * PCG loops covers all still-active scenes in one launch, with per-scene
 * scalars (step sizes, convergence) kept on the device. reports: host
 * array of n. A scene whose step fails keeps its state (as sx_newton_step);
 * the others are stepped. */
int sx_newton_step_batch(sx_ctx* ctx, sx_scene* const* scenes, int n, double dt,
                         const sx_newton_opts* opts, sx_step_report* reports,
                         void* stream);

/* ---- tracing: per-phase device time and launch counts ------------------
 * Phases of the path, each timed with CUDA events recorded on the stream
 * the phase's kernels are launched on. */
#define SX_PH_ELEMENTS 0   /* element E/g/H kernel (+ PSD test)            */
#define SX_PH_CLAMP 1      /* eigen-decomposition of queued stencils       */
#define SX_PH_ASSEMBLE 2   /* BSR value gather + inertia diagonal          */
#define SX_PH_GRAD 3       /* gradient gather, inertia energy, norms       */
#define SX_PH_REDUCE 4     /* per-scene deterministic reductions           */
#define SX_PH_SPMV 5       /* PCG: q = A p                                 */
#define SX_PH_PCG 6        /* PCG: setup, vector updates, scalar steps     */
#define SX_PH_NEWTON 7     /* predictor, line-search vectors, velocity     */
#define SX_PH_OTHER 8      /* control writes and copies                    */
#define SX_PH_COUNT 9

/* enable != 0 starts recording (and clears the accumulators); 0 stops. */
int sx_profile(sx_ctx* ctx, int enable);
/* Synchronizes the recorded streams and returns, per phase, the summed
 * device milliseconds (ms[SX_PH_COUNT], may be NULL) and the kernel
 * launches since the last reset (launches[SX_PH_COUNT], may be NULL; counted
 * whether or not timing is enabled). reset != 0 clears both. */
int sx_profile_read(sx_ctx* ctx, double* ms, int64_t* launches, int reset);
/* Diagnostics of the projection of the context's last batched evaluation
 * (sx_eval, sx_eval_batch, a Newton step's evaluations; the paper has no
 * counterpart: it shows which paths of phase 2 ran). counts must hold
 * SX_PROJ_BINS ints: counts[k], k = 0..9, the queued stencils whose float
 * eigen-solve left an N block of k columns (9 also when its Gershgorin test
 * failed), except those of k >= 4 with 1..3 clearly negative modes, which
 * are counted in counts[16 + k'] (k' = 1..3, the deflation of those modes);
 * counts[10 + k], k = 1..3, the stencils of k that the refinement's first
 * pass did not certify. A stencil that a later pass hands on is counted
 * again where it goes (bin 9, or its own k for a deflation not certified).
 * The other entries are 0; before any projection all counts are 0.
 * Synchronizes `stream`. */
#define SX_PROJ_BINS 20
int sx_projection_bins(sx_ctx* ctx, int* counts, void* stream);

/* ---- launch shapes and the autotuner -----------------------------------
 * (No counterpart in the paper: these pick GPU launch configurations.)
 * Per context and precision: the projection kernel's block size (32, 64,
 * 128 or 256 threads; default 128) and the element kernel's grid (-1: a
 * persistent launch with as many blocks per SM as fit -- the default;
 * k >= 1: k blocks per SM, capped at what fits; 0: one 128-element tile per
 * block). Every shape computes bit-identical results. */
typedef struct {
    int clamp_threads;        /* chosen projection block size */
    int elem_blocks_per_sm;   /* chosen element grid (-1, k >= 1 or 0, as above) */
    double default_ms;        /* one E+g+projected H+assembly pass, default shape */
    double tuned_ms;          /* the same pass with the chosen shape */
    int candidates;           /* shapes timed */
} sx_tune_report;

/* Times one E+g+projected-H+assembly pass of the batch (best of 3 after a
 * warm-up, CUDA events on `stream`) under the default shape, each other
 * projection block size, and each element-grid choice, and keeps the
 * fastest for `precision` in the context (used by every later call of the
 * context). Overwrites the scenes' assembled outputs. Synchronous. */
int sx_autotune(sx_ctx* ctx, sx_scene* const* scenes, int n, int precision,
                sx_tune_report* report, void* stream);
/* Sets / reads a shape directly (SX_EINVAL for an unsupported block size
 * or an element grid below -1). */
int sx_set_launch_shape(sx_ctx* ctx, int precision, int clamp_threads, int elem_blocks_per_sm);
int sx_get_launch_shape(sx_ctx* ctx, int precision, int* clamp_threads, int* elem_blocks_per_sm);

/* ---- footprint (for admission by memory) ------------------------------ */
typedef struct {
    int64_t n_nodes;
    int64_t n_tets;
    int64_t n_hinges;
    int64_t n_pairs;
    int64_t nnzb_hint;   /* 0: estimate from the counts */
} sx_scene_desc;

/* Device bytes a finalized scene of this shape holds (upper estimate),
 * including its share of the context's projection scratch. */
int sx_scene_footprint(const sx_scene_desc* desc, int64_t* bytes);
/* Device bytes this scene holds now. */
int sx_scene_bytes(sx_scene* scene, int64_t* bytes);

/* ---- serving: continuous batching of backward-Euler steps -------------
 * (No counterpart in the paper, which takes one step of one scene; this
 * is the request-loop form of the §3 time step.)
 * Requests are split by tet count into size-class lanes (default 3:
 * n_tets < 20,000, < 120,000, the rest). Each lane has its own context,
 * CUDA stream (smaller classes at higher stream priority) and worker
 * thread, all on the device current at sx_server_create. Per tick a lane
 * (1) admits its waiting requests in arrival order while their device
 * footprint fits the memory budget shared by all lanes (registration, rest
 * precompute and pattern build happen at admission), (2) runs one batched
 * Newton step (sx_newton_step_batch) over every scene resident in the lane
 * -- requests that arrived while others were on the GPU join the lane's
 * next tick at their own step 0 -- and (3) retires finished requests,
 * keeping their final state on the host and freeing their device memory.
 * Lanes run concurrently, so a small scene's step does not wait for the
 * PCG of a large one. Each scene's result does not depend on what it is
 * batched with (all reductions are per scene and in a fixed order). The
 * ctx passed to sx_server_create only names the device; it stays free for
 * other calls. Step latency is measured from a step's eligibility (request
 * admitted and its previous step done) to the end of the tick that
 * completed it. */
#define SX_SERVER_MAX_LANES 8
typedef struct {
    int64_t n_nodes;
    const double* X;          /* n_nodes x 3 rest positions (host) */
    int64_t n_tets;
    const int32_t* tets;      /* n_tets x 4 (host) */
    const double* young;      /* n_tets (host) */
    const double* poisson;    /* n_tets (host) */
    double density;
    int64_t n_pinned;
    const int32_t* pinned;    /* n_pinned node ids (host, may be NULL) */
    double gravity[3];
} sx_snh_scene_spec;

typedef struct {
    int64_t req_id;
    int status;               /* SX_OK or the failing code */
    int steps;                /* steps taken */
    int64_t n_tets;
    double submit_ms;         /* times on the server clock (ms since create) */
    double admit_ms;
    double done_ms;
    double mean_step_ms;
    char error[120];          /* the library's message for a failed request
                                 (empty when status is SX_OK) */
} sx_completion;

typedef struct {
    int64_t submitted, admitted, completed, rejected;
    int64_t element_steps;    /* sum over completed steps of the scene's tets */
    double wall_ms;           /* since create */
    double busy_ms;           /* time spent in ticks */
    double step_p50_ms, step_p99_ms;
    double request_p50_ms, request_p99_ms;   /* submit -> done */
    int64_t bytes_in_use, peak_bytes;
    int active, pending, ticks;
} sx_serve_stats;

/* opts: Newton options for every step (NULL = defaults). Synchronous. */
int sx_server_create(sx_ctx* ctx, int64_t hbm_budget_bytes, const sx_newton_opts* opts,
                     sx_server** srv);
/* Replaces the lanes: n_lanes in [1, SX_SERVER_MAX_LANES], bounds the
 * n_lanes - 1 increasing tet-count limits (lane i takes n_tets < bounds[i],
 * the last lane the rest; NULL if n_lanes == 1). Only before the first
 * submit (else SX_EORDER). Synchronous. */
int sx_server_set_lanes(sx_server* srv, int n_lanes, const int64_t* bounds);
/* At most max_resident scenes resident in one lane (0, the default: no
 * limit other than the memory budget). A lane then admits a waiting request
 * only when one of its scenes retires: its ticks stay short (lower step
 * latency for the admitted scenes) at the price of longer queueing (higher
 * request latency) and smaller batches. May be changed at any time; takes
 * effect at the lanes' next admissions. */
int sx_server_set_lane_cap(sx_server* srv, int max_resident);
/* Copies the spec (the caller's arrays may be freed on return) and queues
 * the request; SX_EBUDGET if its footprint alone exceeds the budget. */
int sx_server_submit(sx_server* srv, const sx_snh_scene_spec* spec, int n_steps, double dt,
                     int64_t* req_id);
/* Up to `max` completions not yet returned; *n receives their number. */
int sx_server_poll(sx_server* srv, sx_completion* out, int max, int* n);
/* Final state of a completed request (host buffers, n_nodes x 3 each; either
 * may be NULL); releases it. SX_EINVAL if unknown or not complete. */
int sx_server_result(sx_server* srv, int64_t req_id, double* x, double* v);
/* Blocks until nothing is pending or active (or timeout_ms elapses: then
 * SX_ENOTCONV). */
int sx_server_drain(sx_server* srv, double timeout_ms);
int sx_server_stats(sx_server* srv, sx_serve_stats* st);
/* Stops the lanes after their current ticks and frees everything. */
int sx_server_destroy(sx_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* SX_H */
