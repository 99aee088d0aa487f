/*
 * hf.h - C ABI of the GB300 hydraulic-fracture Newton step.
 *
 * The library advances the fully-coupled hydro-mechanical system of
 * Giovanardi, Serebrinsky & Radovitzky, "A fully-coupled computational
 * framework for large-scale simulation of fluid-driven fracture propagation on
 * parallel computers" (arXiv 1911.10275):
 *   - linear elasticity on discontinuous P2 elements (Sec. 3, Eq.
 *     weakElastoStatics), with IIPG-type DG consistency + stability terms on
 *     intact interior facets;
 *   - a linear-decreasing cohesive law on activated facets (Eq. tsl);
 *   - continuous P2 lubrication flow, cubic law q = -w^3/(12 mu) grad p, on
 *     fluid-filled facets (Eq. lubrication, Eq. weakPressure), backward Euler
 *     in time (Eq. discreteElastoStatics, Eq. discreteLubrication);
 *   - one Newton iteration per hf_newton_step: assembly of the residual and of
 *     the Jacobian blocks [A B; C D] (Eq. fully-coupled-fully-discrete) into a
 *     fixed-pattern element-block CSR, then ILU(0) block-Jacobi preconditioned
 *     GMRES (FP64, or FP32 inner solves inside FP64 iterative refinement).
 *
 * Conventions shared with every caller:
 *   - 2D: 6-node triangles, vertices 0,1,2 counter-clockwise, mid-nodes
 *     3=(0,1), 4=(1,2), 5=(2,0).  Plane strain.
 *   - 3D: 10-node tetrahedra with positive volume, vertices 0..3, mid-nodes
 *     4=(0,1), 5=(1,2), 6=(0,2), 7=(0,3), 8=(1,3), 9=(2,3).
 *   - Local facet i of an element is the facet opposite vertex i.  Its
 *     face-node order is: its vertices in ascending local index, then the
 *     mid-nodes of its edges in ascending local index (3 nodes in 2D, 6 in 3D).
 *   - face_elems[2f] = e_minus, face_elems[2f+1] = e_plus (-1: boundary).  The
 *     jump is [[u]] = u(e_plus) - u(e_minus); the facet normal n is the outward
 *     normal of e_minus (Eq. displacementJump); the opening is w = [[u]].n.
 *   - Facet quadrature points are generated in e_minus's face-vertex order
 *     (collapsed-coordinate Gauss rules, 5 points per direction).
 *   - Displacement unknown (element e, local node a, component k) has index
 *     e*nen*dim + a*dim + k in every host array of this API.
 *   - Pressure unknowns live on every node of a crackable facet; pressure DOF
 *     j is the j-th smallest such global node id.
 *
 * Error behaviour: every call returns an hf_status; nothing throws or exits.
 * A failed call leaves the state as it was unless it returns HF_ERR_CUDA, in
 * which case the handle is poisoned and later calls return HF_ERR_STATE.
 * hf_last_error() describes the last failure.  One handle = one CUDA stream;
 * a handle is not thread-safe.  Host arrays passed in are copied; output
 * arrays are caller-allocated with the sizes stated.
 */
#ifndef HF_H
#define HF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int hf_status;
enum {
  HF_OK = 0,
  HF_ERR_INVALID_ARG = -1,
  HF_ERR_OOM = -2,
  HF_ERR_CUDA = -3,
  HF_ERR_NOT_CONVERGED = -4,
  HF_ERR_NONFINITE = -5,
  HF_ERR_TIMEOUT = -6,
  HF_ERR_DEVICE_ASSERT = -7,
  HF_ERR_STATE = -8
};

typedef struct hf_mesh hf_mesh; /* opaque; owns all device memory */

/* Mesh, interface list and boundary data (Sec. 3: partition of the domain,
 * interior boundary, every interior facet carries an interface element).
 * All arrays are host memory owned by the caller and copied at create. */
typedef struct {
  int dim;                        /* 2 or 3 */
  int order;                      /* polynomial order; must be 2 */
  int64_t n_nodes;
  const double* xyz;              /* n_nodes*dim */
  int64_t n_elems;
  const int32_t* elem_nodes;      /* n_elems*(6|10), node order above */
  int64_t n_faces;                /* all facets, interior and boundary */
  const int32_t* face_elems;      /* n_faces*2: e_minus, e_plus (-1 boundary) */
  const int8_t* face_local;       /* n_faces*2: local facet ids (-1 boundary) */
  const int8_t* face_crackable;   /* n_faces: 1 = may become cohesive/fluid */
  int64_t n_dirichlet;
  const int64_t* dir_dof;         /* displacement unknowns held fixed */
  const double* dir_val;          /* their values (strong, nodal) */
  int64_t n_neumann;
  const int32_t* neu_face;        /* boundary facets carrying a traction */
  const double* neu_traction;     /* n_neumann*dim, constant per facet */
} hf_mesh_desc;

/* Solver options.  Defaults come from hf_default_solver_opts. */
enum { HF_PREC_FP64 = 0, HF_PREC_MIXED = 1 };
enum { HF_SCHEME_COUPLED = 0, HF_SCHEME_STAGGERED = 1 };
typedef struct {
  int precision;        /* HF_PREC_FP64 or HF_PREC_MIXED (FP32 SpMV/ILU in FP64 IR) */
  int restart;          /* GMRES restart length m (1..96; default 60) */
  int max_iters;        /* cap on GMRES iterations per Newton step (all cycles) */
  double rtol;          /* GMRES: ||J d + R|| <= rtol ||R|| */
  double inner_rtol;    /* mixed: reduction asked of each FP32 inner solve (default 1e-4); after
                           two sweeps in a row that do not halve the FP64 residual the solve
                           goes on in FP64, so a value >= 1 (no reduction asked) makes every
                           mixed solve finish in FP64 */
  int jacobi_block;     /* elements per block-Jacobi subdomain (>= 1) */
  int fluid_scaling;    /* 1: scale pressure rows by c^n (remark in Sec. 3) */
  double newton_tol;    /* relative-increment tolerance of hf_newton_step */
  int use_graphs;       /* 1: capture each GMRES cycle in a CUDA graph */
  int coarse;           /* 1: add the rigid-body coarse correction to the preconditioner */
  int coarse_max;       /* bound on the coarse unknowns (16..4096): sets the aggregate size */
  int reorth;           /* classical Gram-Schmidt passes: 0 one; 1 a second, re-orthogonalising
                           pass when the first removed more than 30% of the vector; 2 always
                           two; 3 (default) two, the second delayed by one Arnoldi step and fused
                           with the next step's first (two basis sweeps and one global reduction
                           per step).  FP32 cycles lose orthogonality with one */
  int scheme;           /* HF_SCHEME_COUPLED (default): one Newton iteration of the fully-coupled
                           system; HF_SCHEME_STAGGERED: one iteration of the staggered scheme of
                           Sec. 4.3 (FP64 only) */
} hf_solver_opts;

/* Report of one Newton iteration (Sec. 3: convergence on the Euclidean norms
 * of the relative increments of both nodal arrays). */
typedef struct {
  double du_rel;        /* ||dU||_2 / ||U||_2 after the update */
  double dp_rel;        /* ||dP||_2 / ||P||_2 after the update */
  double res_norm;      /* ||R||_2 at the start of the iteration */
  double lin_res;       /* ||J d + R||_2 / ||R||_2 reached by GMRES */
  int gmres_iters;      /* inner (Arnoldi) iterations taken */
  int refinements;      /* mixed mode: outer refinement steps */
  int converged;        /* du_rel <= tol && dp_rel <= tol */
  int lin_converged;    /* lin_res <= rtol */
  int fp64_fallback;    /* mixed mode: FP32 sweeps stalled, the solve finished in FP64 */
} hf_newton_report;

void hf_default_solver_opts(hf_solver_opts* o);

/* Builds the fixed-topology discretisation: facet geometry, pressure DOF map,
 * element-block pattern, block-Jacobi subdomains and their level schedule.
 * cuda_stream: a cudaStream_t (NULL = a new stream owned by the handle).
 * Errors: HF_ERR_INVALID_ARG on malformed input (bad ids, dim/order, a facet
 * whose elements do not share it), HF_ERR_OOM, HF_ERR_CUDA. */
hf_status hf_mesh_create(const hf_mesh_desc* desc, void* cuda_stream, hf_mesh** out);
hf_status hf_mesh_destroy(hf_mesh* h);

/* Elastic and cohesive material (Sec. 2, Eq. tsl; stability b of Eq.
 * weakElastoStatics).  Rebuilds the cached linear blocks (bulk B^T D B and
 * the intact-facet DG blocks).  E > 0, -1 < nu < 0.5, sigma_c > 0,
 * delta_c > 0, b_stab > 0. */
hf_status hf_set_material(hf_mesh* h, double E, double nu, double sigma_c, double delta_c,
                          double b_stab);

/* Fluid and injection (Eq. lubrication, Eq. discreteLubrication): viscosity mu,
 * total injection rate Q0 split over n_inj pressure DOFs with the given
 * weights (a point source: one DOF, weight 1), fluid-activation opening
 * delta_f, time step dt, vapour pressure p_v, pressure cut-off switch, and the
 * length L of the fluid-row scaling c^n = 12 mu (L / max w^n)^3. */
hf_status hf_set_injection(hf_mesh* h, double mu, double Q0, int64_t n_inj,
                           const int64_t* p_dofs, const double* weights, double delta_f,
                           double dt, double p_vapor, int cutoff_on, double L_ref);

hf_status hf_set_solver(hf_mesh* h, const hf_solver_opts* o);

/* State (U, P, alpha, beta, w^n, t).  U: n_elems*nen*dim, P: n_p,
 * alpha/beta: n_faces, w_old: n_faces*nfn face-node openings at t^n (NULL:
 * take the opening of U).  Rescales the fluid rows from w_old. */
hf_status hf_set_state(hf_mesh* h, const double* U, const double* P, const int8_t* alpha,
                       const int8_t* beta, const double* w_old, double t);
hf_status hf_get_state(hf_mesh* h, double* U, double* P, int8_t* alpha, int8_t* beta,
                       double* w_old, double* t);

/* One Newton iteration of Sec. 3 (assemble R and J, solve J d = -R, update).
 * Returns HF_OK even if the iteration did not converge (see rep->converged);
 * HF_ERR_NONFINITE if a norm is not finite (state then unchanged).
 * With scheme HF_SCHEME_STAGGERED it is instead one iteration of the
 * staggered scheme of Sec. 4.3 ("Fully-coupled vs. staggered"): the
 * mechanical equation solved for U with the pressure of the previous
 * iteration, A dU = -R_u(U, P), then the lubrication equation for P at the
 * updated opening, D dP = -R_p(U + dU, P) (A, D the diagonal blocks of Eq.
 * fully-coupled-fully-discrete); du_rel and dp_rel are those two increments.
 * The decoupled fluid problem is elliptic and needs an essential pressure
 * (hf_set_fixed_pressure). */
hf_status hf_newton_step(hf_mesh* h, hf_newton_report* rep);

/* Essential pressure condition (Sec. 4.3: the decoupled fluid equation of
 * the staggered scheme needs the pressure given at least at one point):
 * pressure DOF p_dofs[i] is held at values[i] by an identity row, in both
 * schemes.  Replaces any earlier set; n = 0 clears it.  HF_ERR_INVALID_ARG
 * on a DOF out of range or a non-finite value. */
hf_status hf_set_fixed_pressure(hf_mesh* h, int64_t n, const int64_t* p_dofs, const double* values);

/* Fracture criterion (Sec. 3, activation of the TSL): on crackable intact
 * facets, alpha := 1 where the normal DG traction n.<sigma>n + (b/h)(lambda +
 * 2 mu) w exceeds sigma_c at a facet quadrature point.  Irreversible.
 * n_new_alpha: number of facets switched. */
hf_status hf_check_fracture_criterion(hf_mesh* h, int64_t* n_new_alpha);

/* End of a time step (Sec. 3: beta lagged to the end of the step; Remark on
 * delta_f): beta := 1 on cohesive facets whose opening exceeds delta_f at a
 * quadrature point, w^n := w^{n+1}, t += dt, c^n recomputed. */
hf_status hf_accept_step(hf_mesh* h, int64_t* n_new_beta);

/* Openings at the face nodes of every facet (n_faces*nfn, 0 on boundary
 * facets), pressures (n_p), alpha, beta (n_faces).  Any pointer may be NULL. */
hf_status hf_get_opening_pressure(hf_mesh* h, double* w_face_nodes, double* p, int8_t* alpha,
                                  int8_t* beta);

/* Sizes fixed by the mesh. */
hf_status hf_get_sizes(const hf_mesh* h, int64_t* n_u, int64_t* n_p, int64_t* nfn);

/* Diagnostics used by the parity tests: residual R at the current state
 * (n_u + n_p, host layout), and y = J x for a host vector x (same layout).
 * Both include the row scaling and the identity rows of the Newton system. */
hf_status hf_eval_residual(hf_mesh* h, double* R);
hf_status hf_apply_jacobian(hf_mesh* h, const double* x, double* y);
/* Largest normal DG traction over the quadrature points of each crackable
 * intact facet (-inf elsewhere), as tested by hf_check_fracture_criterion. */
hf_status hf_get_criterion_traction(hf_mesh* h, double* tmax);
/* z = M^-1 x with the block-Jacobi ILU(0) preconditioner of the current state. */
hf_status hf_apply_preconditioner(hf_mesh* h, const double* x, double* z);
/* Solve J d = rhs with the configured GMRES (no state change); host vectors. */
hf_status hf_solve_linear(hf_mesh* h, const double* rhs, double* d, hf_newton_report* rep);

/* Profiling.  on = 1: every kernel class of the Newton step is bracketed by
 * CUDA events on the handle's stream (GMRES cycles are then launched without
 * graphs, the coarse level on the handle's stream).  on = 2: only each whole
 * GMRES cycle is bracketed (graph replay or eager launches, as configured),
 * nothing inside it.  on = 0: off.  hf_get_kernel_times returns the
 * accumulated milliseconds and counts since profiling was switched on, per
 * class: 0 SpMV (Krylov precision), 1 preconditioner apply, 2 Gram-Schmidt +
 * norm, 3 ILU factorisation (and the coarse matrix), 4 assembly (facet terms
 * + residual), 5 FP64 SpMV of the refinement residual, 6 Newton update, 7 the
 * rest of the preconditioner (coarse restriction, solve and prolongation;
 * pressure rows), each with its launch count; 8 whole GMRES cycles (mode 2)
 * with the Arnoldi steps they finalised.  Class 1 is the ILU(0) apply
 * alone.  ms and launches hold 9. */
hf_status hf_set_profiling(hf_mesh* h, int on);
hf_status hf_get_kernel_times(hf_mesh* h, double* ms, int64_t* launches);
/* Structure counts: [0] elements, [1] interior facet slots (element-side pairs
 * with a neighbour), [2] slots inside block-Jacobi subdomains, [3] deepest
 * level schedule, [4] subdomains, [5] nonlinear facets, [6] pressure
 * unknowns, [7] facets, [8] kernel launches issued by the library in this
 * process so far, [9] CUDA error met when reading timing events recorded
 * inside a captured GMRES cycle (0: none; graph cycles then go untimed),
 * [10] device bytes the handle holds, [11] coarse unknowns in use (0: one
 * level), [12] elements per coarse aggregate, [13] second Gram-Schmidt passes
 * taken by GMRES since the handle was created, [14] basis vectors swept by
 * first Gram-Schmidt passes (the sum of j + 1 over Arnoldi steps j), [15] basis
 * vectors swept by second passes.  st holds 16. */
hf_status hf_get_stats(const hf_mesh* h, int64_t* st);

const char* hf_last_error(const hf_mesh* h);

/* Failure detection without a fault.  The ILU(0) apply and the streamed
 * Gram-Schmidt kernels wait on mbarriers for their bulk copies with a
 * bounded number of polls (default 2^22); a wait that runs out raises a
 * device flag holding the first site that gave up (1 ILU(0) apply; 2-4 the
 * Gram-Schmidt dot kernel's producer, u/w and consumer waits; 5-6 the update
 * kernel's producer and consumer waits; 7 the drain at kernel exit; 8 the
 * self-test below), the kernel goes on, and the solve returns HF_ERR_TIMEOUT
 * with the context intact and the site in hf_last_error.  hf_set_wait_limit sets
 * that bound (1..2^30 polls).  hf_check_wait_timeout runs the same bounded
 * wait on a barrier that nothing ever completes (no copies issued) and
 * returns HF_ERR_TIMEOUT once it has given up (HF_OK would mean the wait
 * never gave up); the flag is cleared again, so the handle stays usable.
 * The paper has no counterpart: this is the library's own robustness. */
hf_status hf_set_wait_limit(hf_mesh* h, int64_t polls);
hf_status hf_check_wait_timeout(hf_mesh* h);

/* Allocation-free Newton convergence norms.  The paper has no counterpart:
 * this exists for callers that cannot allocate device memory (a process whose
 * device memory belongs to a pool or arena, code that must not allocate while
 * a CUDA graph is built around it, hosts that allocate only at start-up).
 * Computes out[0..3] = ||dx_u||^2, ||x_u||^2, ||dx_p||^2, ||x_p||^2, the sums
 * hf_newton_step uses for its relative increments, where the first n_u
 * entries of the device vectors d_dx and d_x are displacements and the next
 * n_p pressures.  d_out is device memory for 4 doubles, written on the given
 * stream (a cudaStream_t, NULL = legacy default stream); the call does not
 * synchronise.  It calls no cudaMalloc, cudaFree or allocating library
 * routine: its scratch is a fixed array of 128 KiB + 256 B in the library's
 * own device memory, which every GPU that loads the library keeps until the
 * process exits.  n_u + n_p must not exceed 67,108,864 (the scratch holds the
 * partial sums of at most 4096 blocks of 16,384 unknowns); larger sizes,
 * negative sizes and null pointers return HF_ERR_INVALID_ARG.  The first call
 * on each device looks up the scratch address with the device current (make
 * that first call before any stream capture); every later call whose stream
 * is not being captured looks it up again, so an address cached before a
 * device reset is not reused (a call inside a capture uses the address of the
 * last call made outside one).  Every call shares the one
 * scratch array and clears its counter first, so calls that overlap on the
 * GPU (different streams, or host threads racing) give wrong results.  err
 * (may be NULL) receives a message of at most err_len bytes. */
hf_status hf_increment_norms_noalloc(const double* d_dx, const double* d_x, int64_t n_u, int64_t n_p,
                                     double* d_out, void* cuda_stream, char* err, int64_t err_len);

/* ------------------------------------------------------------ time step */

/* Options of hf_advance_step. */
typedef struct {
  int newton_max;        /* Newton iterations per attempt before the step is cut (default 8); past
                           it, iterations go on while the increments at least halve each time, up
                           to 4 newton_max */
  int criterion_rounds;  /* criterion / Newton-again rounds per sub-step (default 4) */
  int max_cutbacks;      /* consecutive failed attempts (each halving the sub-step) before the call
                           gives up (default 10); at most 256 attempts in all */
  int max_new_facets;    /* an attempt whose fracture criterion switches more than this many facets
                           in one round fails like a non-converged one (undone, sub-step halved):
                           the criterion is checked on the converged state of a sub-step at fixed
                           crack, and a sub-step that injects far more fluid than the crack holds
                           overshoots the pressure and switches a whole region at once.  0 (the
                           default): no limit */
} hf_step_opts;

typedef struct {
  int64_t newton_iters;  /* Newton iterations, failed attempts included */
  int64_t gmres_iters;   /* Arnoldi iterations over those Newton iterations */
  int64_t substeps;      /* accepted sub-steps (1 when the full step converged) */
  int64_t cutbacks;      /* attempts undone and halved */
  int64_t new_alpha;     /* facets switched to cohesive */
  int64_t new_beta;      /* facets switched to fluid-filled */
  double t;              /* time reached (t + dt on success) */
  double du_rel, dp_rel; /* relative increments of the last Newton iteration */
} hf_step_report;

void hf_default_step_opts(hf_step_opts* o);

/* One time step of length dt (hf_set_injection) as Sec. 3 drives it: Newton
 * iterations (hf_newton_step) until the relative increments meet the
 * tolerance, then the fracture criterion; if it switched facets, Newton
 * again (at most criterion_rounds rounds); then the end of the step
 * (hf_accept_step).  An attempt that does not converge within newton_max
 * iterations, whose linear solve misses its tolerance by more than a factor
 * of 10 (the FP64 solve ends early when five restarts in a row each reduce
 * the residual by less than 1%), or whose state turns
 * non-finite, or whose criterion switches more than max_new_facets facets in
 * one round, is undone from a device copy of the start-of-step state and
 * retried with half the sub-step; after a success the sub-step grows by 1.5
 * up to dt, until t + dt is reached.  dt itself is left unchanged.  Errors:
 * HF_ERR_NOT_CONVERGED after max_cutbacks consecutive failures or 256
 * attempts (state = the last accepted sub-step), any CUDA or state error as
 * returned by the calls above. */
hf_status hf_advance_step(hf_mesh* h, const hf_step_opts* opts, hf_step_report* rep);

/* Block-Jacobi subdomains of the preconditioner (diagnostics): for each
 * element (caller's order), its subdomain and its position in that
 * subdomain's elimination order (n_elems each; either may be NULL).  Within a
 * subdomain the block ILU(0) of the element blocks of A eliminates elements
 * in increasing position: L_ik = A_ik D_k^-1 for earlier neighbours k,
 * D_i = A_ii - sum_k L_ik A_ki. */
hf_status hf_get_subdomains(const hf_mesh* h, int32_t* sd_of_elem, int32_t* order_in_sd);

/* Aggregate of each element (caller's element order) in the coarse level of
 * the preconditioner: the preconditioner is M^-1 = B^-1 + Phi A0^-1 Phi^T,
 * B the block-Jacobi ILU(0) of the subdomains, Phi the rigid-body modes of
 * each aggregate (translations and infinitesimal rotations about its
 * centre) on its elements' displacement unknowns, zero on Dirichlet rows,
 * and A0 = Phi^T J_base Phi with J_base the linear part of the tangent
 * (bulk and intact-facet blocks).  The paper has no coarse level (its
 * subdomain solver is direct, Sec. 3); it is added here because the
 * one-level iteration count grows with the mesh.  agg_of_elem holds n_elems. */
hf_status hf_get_aggregates(const hf_mesh* h, int32_t* agg_of_elem);

/* The coarse operator of the preconditioner (diagnostics): *nc coarse
 * unknowns (call with NULL arrays first), A0 and its inverse as used
 * (nc x nc, row-major, row/column index = aggregate * n_modes + mode), and per
 * aggregate its centre (dim values, padded to 3) and size H, in geo (4 per
 * aggregate).  Mode k < dim is the translation along axis k; the rotations
 * (in the planes (0,1) [, (1,2), (2,0)]) take u_a = -X_b, u_b = X_a with
 * X = (x - centre) / H. */
hf_status hf_get_coarse_operator(hf_mesh* h, int64_t* nc, double* A0, double* A0inv, double* geo);

/* Unknown counts of the system a descriptor defines, without a handle:
 * n_u = n_elems * nen * dim displacements, n_p pressure unknowns (the
 * distinct nodes of crackable interior facets). */
hf_status hf_mesh_sizes(const hf_mesh_desc* desc, int64_t* n_u, int64_t* n_p);

/* Upper bound on the device memory a handle for this mesh holds once it has
 * been created, given these solver options (NULL: the defaults) and stepped
 * (both solver precisions, the step snapshot included); read with
 * hf_get_stats [10]. */
hf_status hf_estimate_device_bytes(const hf_mesh_desc* desc, const hf_solver_opts* opts, int64_t* bytes);

/* ------------------------------------------------------------ serving */

/* A request loop over many independent fracture problems.  The paper solves
 * one problem at a time; this runtime keeps several on the device at once.
 * `slots` worker threads each own a CUDA stream; a submitted request waits
 * in a FIFO queue until a slot is free and its device-memory bound
 * (hf_estimate_device_bytes) fits in what the budget has left; smaller
 * requests may pass a waiting larger one at most `max_bypass` times.  An
 * admitted request builds its handle on the slot's stream, runs n_steps calls
 * of hf_advance_step with its mesh, state, crack state and Krylov workspace
 * resident, copies its final state to host memory and frees its device
 * memory.  Requests on different slots overlap on the GPU. */
typedef struct hf_runtime hf_runtime;

typedef struct {
  int slots;                 /* concurrent requests (1..64) */
  int64_t hbm_budget_bytes;  /* bound on the summed estimates of admitted requests */
  int max_bypass;            /* times the head of the queue may be passed (default 8) */
  int device;                /* CUDA device ordinal */
} hf_runtime_opts;

/* A request: every array is host memory owned by the caller and copied by
 * hf_runtime_submit.  Material, injection and solver options as in
 * hf_set_material / hf_set_injection / hf_set_solver; the initial state as in
 * hf_set_state (NULL U0, P0, alpha0, beta0: zeros). */
typedef struct {
  const hf_mesh_desc* mesh;
  double E, nu, sigma_c, delta_c, b_stab;
  double mu, Q0;
  int64_t n_inj;
  const int64_t* inj_dofs;
  const double* inj_weights;
  double delta_f, dt, p_vapor;
  int cutoff_on;
  double L_ref;
  hf_solver_opts solver;
  hf_step_opts step;
  int n_steps;
  const double* U0;
  const double* P0;
  const int8_t* alpha0;
  const int8_t* beta0;
  double t0;
} hf_request;

typedef struct {
  hf_status status;        /* HF_OK, or the first error of the request */
  int64_t n_u, n_p, n_faces;
  int64_t steps_done;
  int64_t newton_iters, gmres_iters, cutbacks;
  int64_t device_bytes;    /* the handle's device memory after its last step */
  int64_t estimate_bytes;  /* the bound admission used */
  double t_submit, t_admit, t_done;  /* seconds on the runtime's clock */
  double t_final;          /* simulated time reached */
} hf_result;

hf_status hf_runtime_create(const hf_runtime_opts* opts, hf_runtime** out);
/* Waits for running requests, drops queued ones, joins the workers. */
hf_status hf_runtime_destroy(hf_runtime* rt);
/* Queues a copy of the request; *id identifies it. HF_ERR_INVALID_ARG on a
 * malformed request; one whose estimate exceeds the budget completes at once
 * with status HF_ERR_OOM. */
hf_status hf_runtime_submit(hf_runtime* rt, const hf_request* req, int64_t* id);
/* Waits up to timeout_s seconds (< 0: without limit) for request id to
 * finish and fills *res; HF_ERR_TIMEOUT if it has not finished by then. */
hf_status hf_runtime_wait(hf_runtime* rt, int64_t id, double timeout_s, hf_result* res);
/* Copies the final state of a finished request (sizes from hf_result; any
 * pointer may be NULL) and forgets the request. */
hf_status hf_runtime_fetch(hf_runtime* rt, int64_t id, double* U, double* P, int8_t* alpha, int8_t* beta);
/* [0] queued, [1] running, [2] finished and not fetched, [3] device bytes
 * admitted now, [4] peak admitted bytes, [5] peak running requests,
 * [6] requests completed so far, [7] requests that failed.  st holds 8. */
hf_status hf_runtime_stats(hf_runtime* rt, int64_t* st);
/* Seconds since hf_runtime_create on the runtime's clock. */
double hf_runtime_now(const hf_runtime* rt);

#ifdef __cplusplus
}
#endif
#endif /* HF_H */
