/*
 * libpff: GB300-native hot path of the matrix-free, GMG-preconditioned
 * Newton-GMRES solver for quasi-static phase-field fracture of Kolditz & Wick,
 * "Matrix-free geometric multigrid preconditioning of combined Newton-GMRES for
 * solving phase-field fracture with local mesh refinement" (arXiv 2404.03265).
 *
 * Conventions
 * -----------
 * - Every call returns pff_status (0 = PFF_OK).  No exception crosses the ABI.
 *   pff_last_error() returns a thread-local message for the last failure.
 * - Handles (pff_mesh, pff_problem) are owned by the library; destroy them with
 *   the matching *_destroy call.  Device tables of a mesh are allocated by the
 *   library (cudaMalloc) on the CUDA device current at pff_problem_create.
 * - Vectors are caller-owned DEVICE pointers in the library's node layout:
 *   n_slots entries (pff_mesh_info.n_slots), one per node slot.  Slots that hold
 *   no node ("holes", pff_mesh_slots flags bit0 clear) are ignored on input and
 *   written as 0 on output.  A displacement vector is stored in block layout:
 *   n_slots values of u_x followed by n_slots values of u_y (2*n_slots values);
 *   a phase-field vector has one value per slot.
 *   Values of hanging nodes are ignored on input (they follow from the
 *   constraint) and written as 0 by operators.
 * - stream is a cudaStream_t passed as void* (NULL = legacy default stream);
 *   device work is stream-ordered and asynchronous unless stated otherwise.
 */
#ifndef PFF_H
#define PFF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pff_status;
enum {
  PFF_OK = 0,
  PFF_ERR_INVALID_ARG = 1,
  PFF_ERR_CUDA = 2,
  PFF_ERR_OOM = 3,
  PFF_ERR_NOT_CONVERGED = 4,
  PFF_ERR_GMRES_BREAKDOWN = 5,
  PFF_ERR_NONFINITE = 6,
  PFF_ERR_LINESEARCH = 7,
  PFF_ERR_TIMEOUT = 8,
  PFF_ERR_STATE = 9
};

enum { PFF_F64 = 0, PFF_F32 = 1 };

/* Operator selector of pff_apply. */
enum {
  PFF_OP_JACOBIAN = 0,   /* y = G~ x  (constrained Jacobian, Sec. 3.1 / 3.2)           */
  PFF_OP_TRANSPOSE = 1,  /* y = G~^T x (vector-Jacobian product)                        */
  PFF_OP_CONDENSED = 2   /* y = M_f C^T G C x: fixed inputs NOT masked, fixed rows 0     */
};

typedef struct pff_mesh pff_mesh;
typedef struct pff_problem pff_problem;
typedef struct pff_mg pff_mg;

typedef struct pff_mesh_info {
  int64_t n_slots;       /* length of a node vector                                   */
  int64_t n_nodes;       /* leaf-mesh nodes (incl. hanging); DoFs = 3 * n_nodes        */
  int64_t n_leaf_cells;
  int64_t n_hanging;
  int64_t n_partials;    /* interface partial sums of one apply                       */
  int64_t n_bricks;
  int64_t n_irregular;   /* bricks that read explicit index tables                    */
  int64_t x_max, y_max;  /* integer node coordinates run over 0..x_max, 0..y_max       */
  double h_min;          /* diagonal of the finest leaf cell                          */
  int32_t fe_degree;
  int32_t finest_level;  /* levels 0..finest_level                                    */
} pff_mesh_info;

/* Material and solver parameters (Table 1 of the paper; Problems 1 and 2). */
typedef struct pff_params {
  double E;       /* Young's modulus                                       */
  double nu;      /* Poisson ratio (plane strain Lame constants)            */
  double Gc;      /* critical energy release rate G_c                        */
  double eps;     /* length scale l                                          */
  double kappa;   /* regularisation in g(phi) = (1-kappa) phi^2 + kappa      */
  double p;       /* pressure                                                */
  double c;       /* primal-dual active set constant; c <= 0 selects the
                     per-DoF c_i = 2 |lambda_i / (phi_i - phi_old_i)| of Sec. 2 */
} pff_params;

const char* pff_last_error(void);

/* ---- mesh (host) ----------------------------------------------------------
 * Quadtree on [x0,x1] x [y0,y1] with ncx x ncy coarse cells (level 0).
 * Refinement keeps a 2:1 face balance (Sec. 3: hanging nodes).  Marks refer to
 * leaves in canonical order: ascending (level, j, i).
 * rule 0: refine leaves whose centre x0 + (i + 1/2) hx_l lies in the closed box;
 * rule 1: refine leaves whose closed cell meets the closed box.
 * pff_mesh_finalize builds nodes, hanging constraints, the brick layout and the
 * multigrid level meshes for Q_k elements, k = fe_degree in {1, 2}.
 * Errors: PFF_ERR_INVALID_ARG on bad sizes, PFF_ERR_STATE on refine after
 * finalize.                                                                   */
pff_status pff_mesh_create(double x0, double x1, double y0, double y1, int32_t ncx, int32_t ncy,
                           pff_mesh** out);
pff_status pff_mesh_refine_global(pff_mesh* m, int32_t times);
pff_status pff_mesh_refine_box(pff_mesh* m, int32_t rule, double bx0, double bx1, double by0,
                               double by1);
pff_status pff_mesh_refine_marked(pff_mesh* m, const uint8_t* marks_host, int64_t n_leaves);
pff_status pff_mesh_n_leaves(const pff_mesh* m, int64_t* n);
pff_status pff_mesh_finalize(pff_mesh* m, int32_t fe_degree);
pff_status pff_mesh_info_get(const pff_mesh* m, pff_mesh_info* out);
/* Host arrays of n_slots entries: integer node coordinates (-1 for holes) and
 * flags (bit0 node, bit1 on the boundary (Dirichlet u), bit2 hanging).         */
pff_status pff_mesh_slots(const pff_mesh* m, int32_t* X, int32_t* Y, uint8_t* flags);
/* Host array 3*n_leaf_cells: (level, i, j) per leaf cell, canonical order.       */
pff_status pff_mesh_leaf_cells(const pff_mesh* m, int32_t* lij);
void pff_mesh_destroy(pff_mesh* m);

/* ---- problem --------------------------------------------------------------
 * Binds parameters to a finalized mesh and uploads its device tables.          */
pff_status pff_problem_create(pff_mesh* m, const pff_params* prm, pff_problem** out);
void pff_problem_destroy(pff_problem* pb);

/* Linearisation point U^k = (u, phi) and phi_tilde (Sec. 2: the degradation of
 * the u-equation uses phi_tilde).  u: 2*n_slots doubles, phi, phi_tilde:
 * n_slots doubles (device).  Hanging entries are replaced by their constraint.
 * The library keeps FP64 and FP32 copies.                                      */
pff_status pff_set_state(pff_problem* pb, const double* u, const double* phi, const double* phi_tilde,
                         void* stream);

/* Active set of the phase field (Algorithm 2): active[s] != 0 marks the phi DoF
 * of slot s as fixed (identity row and column).  Device array of n_slots bytes;
 * entries on hanging nodes and holes are ignored.                              */
pff_status pff_set_active(pff_problem* pb, const uint8_t* active, void* stream);

/* Matrix-free operator (Sec. 3.1 Jacobian, Sec. 3.3 matrix-free cell loop):
 *   PFF_OP_JACOBIAN  y = G~ x,   G~ = M_f C^T G C M_f + I_fixed
 *   PFF_OP_TRANSPOSE y = G~^T x
 *   PFF_OP_CONDENSED y = M_f C^T G C x
 * G: unconstrained Jacobian at the state; C: hanging-node constraints; M_f:
 * free (not Dirichlet, not active, not hanging) DoFs; I_fixed: identity on
 * Dirichlet u and active phi DoFs.  precision PFF_F64: double vectors, PFF_F32:
 * float vectors (state cast to float).  xu/yu: 2*n_slots, xp/yp: n_slots.
 * x and y must not overlap.                                                    */
pff_status pff_apply(pff_problem* pb, int32_t precision, int32_t op, const void* xu, const void* xp,
                     void* yu, void* yp, void* stream);

/* phi_tilde of load step n by extrapolation (Sec. 2: the degradation of the
 * u-equation uses phi_tilde, "the old incremental step solution or an
 * extrapolation"): phi_tilde = clip(2 phi_prev - phi_prev2, 0, 1) per slot, the
 * linear extrapolation in the step index from the two previous steps' converged
 * phase fields, clipped to the phase field's range.  n_slots doubles each
 * (device); phi_tilde may alias neither input.  Pass the result as
 * pff_newton_opts.phi_tilde.  Errors: PFF_ERR_INVALID_ARG on NULL pointers.     */
pff_status pff_extrapolate_phi(pff_problem* pb, const double* phi_prev, const double* phi_prev2,
                               double* phi_tilde, void* stream);

/* Shape of the Q1 cell loop (Sec. 3.3's matrix-free cell-by-cell evaluation;
 * the shape changes the schedule, not the arithmetic: every cell and every nodal
 * sum is evaluated in the same order, so results are bitwise the same).  A warp
 * sweeps a strip of 2 * strip_half_rows node rows of a 30 x 30 brick, its lower
 * and upper halves side by side.  strip_half_rows: 15 (one strip per brick), 5
 * or 1 (3 or 15 shorter strips: more warps for small level meshes of the
 * V-cycle), or 0 (default: chosen per call from the number of bricks).  It acts
 * on the Jacobian (pff_apply) and the multigrid level block operators; the other
 * Q1 operators always use 15; Q2 meshes ignore it.  V-cycles captured by an
 * earlier pff_mg_setup keep their shape until the next one.
 * Errors: PFF_ERR_INVALID_ARG for other values.                               */
pff_status pff_set_cell_loop(pff_problem* pb, int32_t strip_half_rows);

/* ---- multigrid preconditioner (Sec. 3.2) -----------------------------------
 * One V-cycle per diagonal block of G~: block 0 = u-u (2 components, vectors of
 * 2*n_slots doubles), block 1 = phi-phi (n_slots doubles).  Levels are all cells
 * of one refinement level (local smoothing); Chebyshev-accelerated Jacobi
 * smoothing of degree 3 on [0.08, 1.2] * lambda_max, lambda_max from 12 steps of
 * Jacobi-preconditioned CG (FP64 vectors and coefficients; its operator applies
 * in the V-cycle's precision on levels >= 1); inverse diagonal from cell-local
 * assembly (FP64); direct FP64 solve on level 0.  precision selects the V-cycle
 * arithmetic (PFF_F32: applies, smoothing and transfers in FP32).
 * pff_mg_setup uses the problem's current state and active set (call it after
 * pff_set_state / pff_set_active); it synchronises the stream.  Its per-level
 * work (inverse diagonals, eigenvalue estimates) runs on an internal pool of
 * streams that is joined back into `stream` before it returns (from the second
 * set-up on, replayed as one captured graph while the material, the modulus, the
 * cell-loop shape and the coarse mode are unchanged); the level-0 blocks are
 * assembled by probing and inverted on the device (blocked Gauss-Jordan, two
 * launches per 32 pivots).
 * pff_vcycle: z = MG(r) for one block; fixed leaf DoFs (Dirichlet u, active phi)
 * get z = r, hanging entries and holes 0.  r and z are device vectors.          */
pff_status pff_mg_create(pff_problem* pb, int32_t precision, pff_mg** out);
pff_status pff_mg_setup(pff_mg* mg, void* stream);
pff_status pff_vcycle(pff_mg* mg, int32_t block, const double* r, double* z, void* stream);
/* Inverse diagonal of block `block` on `level` (Sec. 3.2 Chebyshev-Jacobi):
 * 1/diag(A_l) on interior rows, 0 on refinement-edge, Dirichlet and active
 * rows and holes, FP64, as set up by the last pff_mg_setup.  Written to out
 * (device, ncomp * n_slots_l doubles, components in blocks; ncomp = 2 for block
 * 0, 1 for block 1) if out is not NULL and capacity suffices; *n_out (may be
 * NULL) receives that count.  X_host, Y_host (may be NULL): n_slots_l finest-grid
 * integer coordinates of the level's slots (-1 for holes).                     */
pff_status pff_inverse_diagonal(const pff_mg* mg, int32_t level, int32_t block, double* out, int32_t* X_host,
                                int32_t* Y_host, int64_t capacity, int64_t* n_out, void* stream);
/* lambda_max estimates per level (host array of finest_level + 1 doubles; entry 0 unused) */
pff_status pff_mg_lambda(const pff_mg* mg, int32_t block, double* lam_host, int32_t n);
/* Coarse-level solver of the V-cycle: mode 0 (default) a direct FP64 solve of the
 * level-0 block; mode 1 Chebyshev-Jacobi on level 0 (Sec. 3.2: the extreme
 * eigenvalues of the same CG run give the interval [0.9 lambda_min, 1.2
 * lambda_max]; the degree is the smallest with a Chebyshev error bound of 1e-3,
 * at most 64).  Takes effect at the next pff_mg_setup.                         */
pff_status pff_mg_set_coarse(pff_mg* mg, int32_t mode);
/* Fused smoother (on = 1, the default): each Chebyshev step of the V-cycle
 * (Sec. 3.2) is the store of the level apply that it needs, one launch instead
 * of two (Q1 and Q2); on = 0 runs the apply and the update as separate kernels.
 * The two round the same expressions; they may differ in the last bit where the
 * compiler contracts the update differently.  No paper counterpart: a
 * launch-count choice.  Takes effect at the next V-cycle; PFF_ERR_INVALID_ARG
 * for other values of on.                                                      */
pff_status pff_mg_set_fused_smoother(pff_mg* mg, int32_t on);
void pff_mg_destroy(pff_mg* mg);

/* ---- residual, GMRES, Newton / primal-dual active set ---------------------
 * Full vectors hold three blocks of n_slots doubles (u_x, u_y, phi).        */
typedef struct pff_solve_info {
  int32_t newton_iterations;
  int32_t converged;           /* 1 if the stopping rule was met                */
  int32_t linesearch_failures; /* Newton steps whose line search found no decrease */
  int32_t gmres_total;         /* linear iterations, summed over Newton steps     */
  int32_t gmres_max;
  int32_t pad;
  int64_t active_size;         /* size of the final active set                   */
  double residual0;            /* ||R~(U^{n,0})|| (GMRES: initial preconditioned residual) */
  double residual;             /* final ||R~|| (GMRES: final estimate)            */
  double margin;               /* min |R_i / B_ii + c (phi_i - phi_i^old)| over DoFs */
  int32_t gmres_per_newton[128];
  double residual_history[129];
  double time_mg_setup;        /* seconds in multigrid set-up (Newton step)      */
  double time_gmres;           /* seconds in GMRES (Newton step); the rest of the
                                  step is residuals, active sets, line search     */
  /* device seconds inside the GMRES iterations (CUDA events on the solve stream):
     operator applies (with their precision conversions), block V-cycles (with
     their staging copies), and Gram-Schmidt orthogonalisation plus the norm of
     the new basis vector.  time_gmres minus their sum is host work and waits. */
  double time_gmres_apply;
  double time_gmres_vcycle;
  double time_gmres_orth;
} pff_solve_info;

typedef struct pff_newton_opts {
  double tol;         /* relative Newton tolerance on ||R~|| (1e-8)           */
  double atol;        /* absolute floor (1e-13)                               */
  double gmres_rtol;  /* GMRES tolerance on the preconditioned residual (1e-6) */
  double omega;       /* line-search damping (0.5)                            */
  int32_t restart;    /* GMRES restart length (50)                            */
  int32_t gmres_maxiter;
  int32_t max_newton; /* Newton iteration cap (100)                           */
  int32_t ls_max;     /* line-search trials (10)                              */
  int32_t matvec_precision; /* Jacobian applies inside GMRES: PFF_F64 (default,
                               0) or PFF_F32 (FP64 Krylov vectors rounded in
                               and out; the residual, line search, active set,
                               orthogonalisation and Givens rotations stay FP64) */
  int32_t reserved;   /* 0                                                    */
  const double* phi_tilde; /* device, n_slots: phi_tilde of the u-equation (Sec. 2,
                              "old step or extrapolation"); NULL: phi_old      */
} pff_newton_opts;

/* ---- allocation-free variant of pff_apply (no counterpart in the paper) ----
 * Same operators, arguments, layout and results as pff_apply.  The difference is
 * where the apply keeps its scratch: the interface partial sums (one triple per
 * interface node of an irregular brick, condensed by a second kernel) and, on Q1
 * meshes, the input resolved on each hanging node (one triple each).  pff_apply
 * uses buffers made by pff_problem_create; this call uses one fixed device array
 * of PFF_NOALLOC_MAX_PARTIALS triples (1.5 MiB) that is part of the library
 * image.  No device or pinned memory is allocated by the call, directly or
 * through a library.  It serves callers that must not allocate while they run: a
 * host whose caching allocator has reserved nearly all device memory (a library
 * cudaMalloc could fail at any time there), or a latency-bound loop that cannot
 * afford cudaFree's implicit device synchronisation.
 * Set-up: pff_problem_create loads the module holding the array on the current
 * device and caches the array's address (cudaGetSymbolAddress), so that loading
 * the module, which reserves the array, does not happen inside this call.  On a
 * device where no problem was created the first call does that look-up itself;
 * make it outside any stream capture there.  The cached address does not
 * survive cudaDeviceReset (which invalidates every problem as well).
 * Limits and hazards:
 *  - a mesh with pff_mesh_info.n_partials, plus n_hanging for fe_degree 1, above
 *    PFF_NOALLOC_MAX_PARTIALS is rejected with PFF_ERR_INVALID_ARG (use
 *    pff_apply);
 *  - the array is shared by all problems and streams of a device and keeps the
 *    previous call's contents (nothing in it has to start at zero: every value
 *    that is read is written earlier in the same call); calls that may execute
 *    at the same time on one device race on it, so order them on one stream or
 *    with events;
 *  - the problem must live on the current device.                              */
#define PFF_NOALLOC_MAX_PARTIALS 65536
pff_status pff_apply_noalloc(pff_problem* pb, int32_t precision, int32_t op, const void* xu, const void* xp,
                             void* yu, void* yp, void* stream);

/* Active set of Algorithm 2 at (R, phi, phi_old): A = { i : R_i / B_ii +
 * c (phi_i - phi_old_i) > 0 } with R the condensed residual (3 blocks of
 * n_slots doubles, as from pff_residual; its phi block is used), B the lumped
 * phi mass and c from pff_params; never on hanging nodes or holes.  active
 * (device, n_slots bytes): the previous set on input, the new one on output.
 * n_changed, n_active, margin (host, may be NULL): entries that changed, size of
 * the set, min |indicator| over nodes.  Synchronises.                         */
pff_status pff_active_set(pff_problem* pb, const double* R, const double* phi, const double* phi_old,
                          uint8_t* active, int64_t* n_changed, int64_t* n_active, double* margin, void* stream);

/* Pressure p of the current load step (Problem 1).                           */
pff_status pff_set_pressure(pff_problem* pb, double p);
/* R = -A(U)(psi) (Problem 2, residual form; sigma^+ read as sigma) for every
 * basis function, hanging contributions condensed onto their parents,
 * Dirichlet u rows 0.  u: 2*n_slots, phi, phi_tilde: n_slots (device).  R: 3 blocks. */
pff_status pff_residual(pff_problem* pb, const double* u, const double* phi, const double* phi_tilde, double* R,
                        void* stream);
/* B: lumped phi mass, integral of each (constrained) basis function; n_slots.   */
pff_status pff_lumped_mass(pff_problem* pb, double* B, void* stream);
/* Total crack volume integral of u . grad phi (Sec. 4) into *out_host (synchronises). */
pff_status pff_tcv(pff_problem* pb, const double* u, const double* phi, double* out_host, void* stream);
/* Crack opening displacement (Sec. 4): COD(x) = integral over y of u . grad phi
 * along the vertical line at each x_host[i] (host, n_x values), by the
 * (k+1)-point Gauss rule in y on every leaf cell the line crosses (a cell
 * [x0, x0 + hx) contains x when x0 <= x < x0 + hx).  u: 2*n_slots, phi: n_slots
 * (device).  cod_host: n_x doubles (host).  Synchronises.                    */
pff_status pff_cod(pff_problem* pb, const double* u, const double* phi, const double* x_host, int32_t n_x,
                   double* cod_host, void* stream);
/* Left-preconditioned GMRES on G~ x = rhs (transpose != 0: G~^T) with the block
 * V-cycle preconditioner of mg, x0 = 0; synchronises.  The Krylov basis (FP64,
 * restart + 1 vectors) holds the node rows only; rhs and x are slot-layout
 * vectors (x is 0 on holes).  Errors:
 * PFF_ERR_NOT_CONVERGED, PFF_ERR_GMRES_BREAKDOWN, PFF_ERR_NONFINITE (info filled). */
pff_status pff_gmres_solve(pff_problem* pb, pff_mg* mg, int32_t transpose, const double* rhs, double* x,
                           double rtol, int32_t restart, int32_t maxiter, pff_solve_info* info, void* stream);
/* One load step of Algorithm 2 at the problem's pressure: Newton iterations with
 * the primal-dual active set, multigrid-preconditioned GMRES and line search;
 * phi_tilde = opts->phi_tilde when set (e.g. from pff_extrapolate_phi), else
 * phi_old.  u, phi: updated in place; active: n_slots bytes, the
 * previous step's final set on input, this step's on output.  opts may be NULL
 * (defaults above).  Synchronises.  Errors: PFF_ERR_NOT_CONVERGED,
 * PFF_ERR_NONFINITE, PFF_ERR_GMRES_BREAKDOWN (info filled).                   */
pff_status pff_newton_pdas_step(pff_problem* pb, pff_mg* mg, double* u, double* phi, const double* phi_old,
                                uint8_t* active, const pff_newton_opts* opts, pff_solve_info* info, void* stream);

/* ---- differentiation: per-cell modulus, TCV gradient, adjoint --------------
 * Sec. 4 quantity of interest J = TCV = integral of u . grad phi; parameters p,
 * G_c (Problem 1) and a per-cell Young's modulus E_K (sigma = E_K sigma_1, the
 * Lame constants of each cell scaled by E_K).                                  */

/* Per-cell modulus: E_cells is a device array of n_leaf_cells doubles in the
 * canonical leaf-cell order of pff_mesh_leaf_cells (positive values), or NULL to
 * return to the uniform pff_params.E.  Level operators of the multigrid use the
 * leaf value on leaf cells and the mean of the four children on refined cells;
 * call pff_mg_setup again afterwards.  The array is copied (stream-ordered).   */
pff_status pff_set_cell_modulus(pff_problem* pb, const double* E_cells, void* stream);

/* Replace the problem's parameters (E is ignored while a cell modulus is set).
 * Takes effect for later calls; an existing pff_mg needs pff_mg_setup again.   */
pff_status pff_set_params(pff_problem* pb, const pff_params* prm);

/* g = M_f C^T dJ/dU at U = (u, phi): 3 blocks of n_slots doubles (device),
 * rows of Dirichlet u, active phi (pff_set_active) and hanging nodes 0.        */
pff_status pff_tcv_gradient(pff_problem* pb, const double* u, const double* phi, double* g, void* stream);

/* Vector-Jacobian product of the residual with respect to the parameters at the
 * problem's state (pff_set_state: u, phi, phi_tilde) and active set:
 *   g_theta = (C M_f w) . dR/dtheta,  R = -A (Problem 2),
 * w: 3 blocks of n_slots doubles (device; fixed entries ignored, hanging entries
 * taken from their parents).  gE_cells: device, n_leaf_cells doubles in
 * canonical leaf order (may be NULL); g_host[0] = g_p, g_host[1] = g_Gc (host).
 * Synchronises.                                                               */
pff_status pff_param_vjp(pff_problem* pb, const double* w, double* gE_cells, double* g_host, void* stream);

/* Adjoint gradient of J at a converged load step (u, phi, active from
 * pff_newton_pdas_step, phi_old its obstacle and phi_tilde):
 *   G~^T lambda = M_f C^T dJ/dU (left-preconditioned GMRES with the block V-cycle
 *   of mg, relative tolerance rtol on the preconditioned residual),
 *   dJ/dtheta = (C M_f lambda) . dR/dtheta.
 * Sets the problem's state and active set to (u, phi, phi_old) / active and
 * re-runs pff_mg_setup.  Outputs as in pff_param_vjp: gE_cells (device, may be
 * NULL), g_host[0] = dJ/dp, g_host[1] = dJ/dG_c.  info: GMRES count and
 * residuals.  Synchronises.  Errors: PFF_ERR_NOT_CONVERGED,
 * PFF_ERR_GMRES_BREAKDOWN, PFF_ERR_NONFINITE.                                 */
pff_status pff_tcv_adjoint(pff_problem* pb, pff_mg* mg, const double* u, const double* phi, const double* phi_old,
                           const uint8_t* active, double rtol, int32_t restart, int32_t maxiter, double* gE_cells,
                           double* g_host, pff_solve_info* info, void* stream);

/* phi_tilde of the load steps that pff_tcv_adjoint_steps differentiates. */
#define PFF_PHIT_PREVIOUS 0     /* phi_tilde of step k = phi[k-1] (the obstacle)          */
#define PFF_PHIT_EXTRAPOLATED 1 /* step k >= 2: clip(2 phi[k-1] - phi[k-2], 0, 1), as
                                   pff_extrapolate_phi; step 1: phi[0]                     */

/* Checkpointed adjoint of J = TCV(U^N) over n_steps load steps of Algorithm 2,
 * step k (1..N) solved from phi_old = phi[k-1] (its obstacle) at pressure
 * p_host[k-1] with final active set active[k-1], and phi_tilde per
 * phi_tilde_mode (PFF_PHIT_PREVIOUS or PFF_PHIT_EXTRAPOLATED, the choice the
 * steps were solved with; Sec. 2 allows the old step or an extrapolation):
 *   u[k], phi[k] (k = 0..N): host arrays of device pointers to the converged
 *   states (u: 2*n_slots, phi: n_slots doubles; k = 0 is the initial state);
 *   active[k] (k = 0..N-1): host array of device pointers (n_slots bytes).
 * Backwards from G~_N^T mu = C^T dJ/dU^N, each step passes its phi-sensitivity
 * to the previous one through phi_tilde (the degradation and pressure terms of
 * the u-equation) and through its active rows (obstacle phi[k-1]); the free rows
 * of a step still see the active values, which the active-row adjoint accounts
 * for.  Extrapolated, the phi_tilde share reaches step k-1 with weight 2 and step
 * k-2 with weight -1 on the slots strictly inside the clip (the derivative of
 * the clip there; 0 on clipped slots, the one-sided choice at the kinks); the
 * share that reaches phi[0] is dropped (the initial state is parameter-free).
 * Outputs: gp_host[k-1] = dJ/dp_k (host, n_steps), *gGc_host = dJ/dG_c,
 * gE_cells (device, n_leaf_cells, may be NULL) = dJ/dE_K.  Leaves the problem's
 * state, active set and multigrid at step 1; restores the pressure.
 * Synchronises.  Errors as pff_tcv_adjoint; PFF_ERR_INVALID_ARG on another
 * phi_tilde_mode.                                                            */
pff_status pff_tcv_adjoint_steps(pff_problem* pb, pff_mg* mg, int32_t n_steps, const double* const* u,
                                 const double* const* phi, const uint8_t* const* active, const double* p_host,
                                 int32_t phi_tilde_mode, double rtol, int32_t restart, int32_t maxiter,
                                 double* gE_cells, double* gp_host, double* gGc_host, pff_solve_info* info,
                                 void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PFF_H */
