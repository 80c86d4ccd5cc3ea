/*
 * uf.h -- C ABI of the GB300-native UrbanFlow RANS step.
 *
 * The library advances the Reynolds-averaged Navier-Stokes equations with a
 * k-omega closure and a porosity drag on a uniform staggered 3D grid, as in
 * "UrbanFlow: Designing Comfortable Outdoor Areas" (arXiv 2204.01117), Sec. 3:
 *   momentum      : Eq. (momen_drag), RANS with eddy viscosity and drag f_d
 *   drag          : Sec. 3 footnote + forward-Euler drag equation,
 *                   u <- max(0, 1 - dt C_d a ((1-phi)/(phi+e))^b |u|) u
 *   turbulence    : k and omega equations, P_k, nu_t = k / omega~ (Sec. 3),
 *                   Table 1 coefficients, viscosity limiter (Sec. 3)
 *   discretisation: staggered MAC grid, operator splitting, MacCormack
 *                   semi-Lagrangian advection, pressure Poisson projection
 *                   solved by preconditioned CG (Sec. 3, App. A.3)
 *   boundaries    : inlet Dirichlet, outlet zero normal derivative, walls,
 *                   outlet pressure 0, dp/dn = 0 elsewhere (Sec. 3)
 *
 * Conventions shared by every entry point:
 *   - All functions return a uf_status and never throw or abort.  On failure
 *     uf_last_error() returns a message for the calling thread.
 *   - Device memory is owned by the caller.  The library never calls
 *     cudaMalloc or cudaFree: the caller allocates one workspace of
 *     uf_workspace_bytes() bytes (any device allocator; 256-byte aligned) and
 *     keeps it alive until uf_destroy().  The library owns only small host-side
 *     objects (the grid handle, CUDA graphs, one internal capture stream).
 *   - Work is enqueued on the CUDA stream given at creation and is
 *     asynchronous unless a stats pointer is passed.
 *   - Field buffers exchanged through uf_set_state / uf_get_state /
 *     uf_set_porosity are dense arrays, x fastest then y then z, in the grid's
 *     precision (float for UF_F32, double for UF_F64).  They may live in host
 *     memory (pageable or pinned) or device memory; the copy direction is
 *     inferred from the pointer.
 *   - Field extents: u (nx+1)*ny*nz, v nx*(ny+1)*nz, w nx*ny*(nz+1);
 *     p, k, omega, phi, nu_t nx*ny*nz.
 */
#ifndef UF_H
#define UF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct uf_grid uf_grid;

typedef enum {
  UF_OK = 0,
  UF_ERR_ARG = 1,            /* invalid argument or description            */
  UF_ERR_CUDA = 2,           /* a CUDA runtime call failed                  */
  UF_ERR_NOMEM = 3,          /* workspace too small                         */
  UF_ERR_NOT_CONVERGED = 4,  /* pressure CG hit its iteration cap           */
  UF_ERR_NAN = 5,            /* non-finite residual in the pressure solve   */
  UF_ERR_TIMEOUT = 6,        /* a bounded device wait gave up               */
  UF_ERR_STATE = 7,          /* call out of order (e.g. step before init)   */
  UF_ERR_BOUNDS = 8          /* an index left its array (only in a library
                                built with -DUF_BOUNDS_CHECK)              */
} uf_status;

enum { UF_F32 = 0,   /* FP32 fields, FP64 reductions and coarsest MG solve */
       UF_F64 = 1 }; /* FP64 throughout                                     */

enum { UF_PRECOND_MG = 0,      /* geometric multigrid V-cycle (default)       */
       UF_PRECOND_AI1 = 1,     /* approximate inverse, 1st order (Sec. 3)     */
       UF_PRECOND_JACOBI = 2,
       UF_PRECOND_NONE = 3,
       UF_PRECOND_AI2 = 4 };   /* approximate inverse, 2nd order (Sec. 3)     */

enum { UF_STOP_RESIDUAL = 0,   /* ||r|| <= cg_tol ||b|| (default)            */
       UF_STOP_PAPER = 1 };    /* r.z <= cg_tol ||b||^2 with z = M^-1 r, the
                                  rule of App. A.3 (cg_tol 1e-5 there); only
                                  with the AI, Jacobi and no preconditioner  */

enum { UF_FIELD_U = 0, UF_FIELD_V = 1, UF_FIELD_W = 2, UF_FIELD_P = 3,
       UF_FIELD_K = 4, UF_FIELD_OMEGA = 5, UF_FIELD_PHI = 6, UF_FIELD_NUT = 7 };

/* Grid and physics description.  uf_default_desc() fills the paper's
 * constants: Table 1 (C_mu 0.09, alpha 0.52, beta 0.0708, sigma 0.5,
 * sigma* 0.6, C_lim 7/8), drag a = 0.62, b = 2.5, e = 1e-10 (Sec. 3
 * footnote), C_d = 1.0 (App. A.2), and the readings of what the paper leaves
 * open: rho = 1.225 kg/m^3, nu = 1.5e-5 m^2/s, I = 0.1, L = 10 m, CFL 0.5,
 * k >= 1e-10, omega >= 1e-6, CG stop ||r|| <= 1e-7 ||b|| (FP32) or 1e-12
 * (FP64) when cg_tol is 0 (the default), at most 200 iterations, AI relaxation w = 1.65 (App. A.3: best
 * w lies in 1.6-1.7). */
typedef struct {
  int nx, ny, nz;          /* cells; nx, ny >= 2, nz >= 1                   */
  double h;                /* cell size [m]                                 */
  int precision;           /* UF_F32 or UF_F64                              */
  double wind_dir_deg;     /* horizontal wind direction, 0 = +x, 90 = +y     */
  double u_ref;            /* inflow speed [m/s] (at z_ref for the log law)  */
  double z_ref, z0;        /* log-law reference height and roughness [m]    */
  int inflow_loglaw;       /* 0: uniform u_ref; 1: log law (Sec. 6.1)       */
  int ground_noslip;       /* 1: no-slip ground; 0: slip ground             */
  double rho, nu, Cd, a, b, e;
  double I, L;             /* inlet turbulence intensity and length scale   */
  double C_mu, alpha, beta, sigma, sigma_star, C_lim;
  double cfl;              /* dt = cfl h / max|u| unless fixed_dt > 0       */
  double fixed_dt;
  double k_min, omega_min;
  int precond;             /* UF_PRECOND_*                                   */
  double cg_tol;           /* ||r||/||b|| to stop at; 0 = by precision      */
  int cg_max_iter;
  double ai_omega;         /* relaxation of the AI preconditioner           */
  double mg_jacobi_omega;  /* damping of the MG Jacobi smoother (6/7)       */
  int mg_coarse_max;       /* coarsest MG level has at most this many cells */
  int mg_smoother;         /* UF_SMOOTH_CHEBY (default), _JACOBI or _RBGS   */
  int cg_stop_rule;        /* UF_STOP_RESIDUAL (default) or UF_STOP_PAPER   */
  int mg_transfer;         /* UF_TRANSFER_LINEAR (default) or _CONSTANT      */
} uf_grid_desc;

enum { UF_SMOOTH_JACOBI = 0,   /* damped Jacobi, 2 sweeps before + 2 after        */
       UF_SMOOTH_RBGS = 1,     /* red-black Gauss-Seidel, red-black / black-red   */
       UF_SMOOTH_CHEBY = 2 };  /* 2 weighted-Jacobi sweeps before + 2 after with
                                  the degree-2 Chebyshev weights for [1/3, 2]   */

/* Multigrid transfers between levels.  Between the finest level and level 1
 * the V-cycle always uses piecewise-constant prolongation and the summed
 * restriction (its transpose).  LINEAR (default): between coarser levels,
 * cell-centred linear prolongation (3/4 of the parent, 1/4 of its neighbour
 * per halved axis; mirrored ghosts at walls, negated at outlets) and its
 * transpose as the restriction: fewer CG iterations for a little more work
 * on the small levels.  CONSTANT: piecewise constant on every level. */
enum { UF_TRANSFER_CONSTANT = 0, UF_TRANSFER_LINEAR = 1 };

typedef struct {
  double dt;               /* time step taken                                */
  int cg_iters;            /* CG iterations of the pressure solve            */
  double cg_rel_residual;  /* ||r||/||b|| at exit (recursive residual)      */
  int status;              /* uf_status of the device-side checks           */
  long long cg_iters_total;/* CG iterations since the grid was created      */
} uf_step_stats;

/* Per-kernel timing of one profiled step (uf_profile_step). */
typedef struct {
  char name[40];           /* kernel label, e.g. "cg_direction_spmv"         */
  int launches;            /* launches in the profiled step                  */
  double total_ms;         /* summed CUDA-event time of those launches      */
  double bytes_per_launch; /* algorithmic HBM bytes one launch must move    */
} uf_kernel_time;

/* Fills *d with the paper's constants and the stated readings (see above);
 * sizes default to 64 x 32 x 16, h = 2 m, 5 m/s uniform inflow along +x. */
void uf_default_desc(uf_grid_desc* d);

/* Bytes of device workspace the grid needs (0 if the description is
 * invalid).  The value includes 256 bytes of alignment slack. */
size_t uf_workspace_bytes(const uf_grid_desc* d);

/* Creates a grid on the current CUDA device.  d_workspace: device pointer to
 * at least uf_workspace_bytes(d) bytes, owned by the caller.  stream: a
 * cudaStream_t (NULL = legacy default stream is rejected; pass a created
 * stream).  The workspace is zeroed; porosity defaults to 1 (open air) and
 * the state to zero until uf_set_state or uf_init_state.
 * Errors: UF_ERR_ARG (bad description or NULL pointers), UF_ERR_NOMEM (bytes
 * too small), UF_ERR_CUDA. */
uf_status uf_create_grid(const uf_grid_desc* d, void* d_workspace, size_t bytes, void* stream, uf_grid** out);

/* Releases host-side objects and graphs; the workspace stays the caller's. */
uf_status uf_destroy(uf_grid* g);

/* Sets the porosity field phi (nx*ny*nz values in [0,1], grid precision,
 * host or device pointer) and derives the per-cell drag coefficient
 * C_d a ((1-phi)/(phi+e))^b (Sec. 3 footnote). */
uf_status uf_set_porosity(uf_grid* g, const void* phi);

/* Copies one field (UF_FIELD_*) in or out, dense layout, grid precision.
 * Setting U, V or W expects every face, boundary faces included. */
uf_status uf_set_state(uf_grid* g, int field, const void* buf);
uf_status uf_get_state(uf_grid* g, int field, void* buf);

/* Several fields in (uf_set_fields) or out (uf_get_fields) in one call:
 * fields[i] (UF_FIELD_*) from / to bufs[i], dense layout as uf_set_state
 * (setting PHI also derives the drag coefficient).  A host buffer moves with
 * one contiguous copy through a device staging array and is repacked to the
 * padded layout by a kernel; a device buffer is repacked directly.  The
 * staging arrays are scratch buffers of the step: call between steps, not
 * concurrently with one.  uf_set_fields returns once the copies are
 * enqueued (a pinned host buffer must stay valid until the stream has
 * consumed it); uf_get_fields synchronises once, after the last field. */
uf_status uf_set_fields(uf_grid* g, int n, const int* fields, const void* const* bufs);
uf_status uf_get_fields(uf_grid* g, int n, const int* fields, void* const* bufs);

/* Snapshot of the complete time-stepping state, for checkpoint and resume
 * (the paper has no counterpart).  Besides the fields uf_set_fields
 * writes, the time integration carries the pressure history: each step's
 * solve starts from the guess 2 p^n - p^{n-1}, and the pressure is held in
 * twice the working precision.  uf_set_fields cannot restore either, so a
 * run restarted from its fields takes a different (equally converged) CG
 * path.  uf_save_state copies the face velocities, k, omega, p^n and the
 * next guess (both in the pressure store) into a caller-owned device
 * buffer of uf_state_bytes(g) bytes; uf_load_state puts them back, after
 * which the steps reproduce the uninterrupted run bit for bit.  The layout
 * is private to the grid's size and precision.  Both are asynchronous on
 * the grid's stream; UF_ERR_NOMEM if the buffer is smaller than
 * uf_state_bytes, UF_ERR_STATE if there is no state to save. */
size_t uf_state_bytes(uf_grid* g);
uf_status uf_save_state(uf_grid* g, void* d_buf, size_t bytes);
uf_status uf_load_state(uf_grid* g, const void* d_buf, size_t bytes);

/* Initial state: the inflow profile on every face (Dirichlet values on the
 * boundary faces), k and omega at the inlet values of Sec. 3
 * (k = 1.5 (I U)^2, omega = k^1/2 / (C_mu^1/4 L)), one drag step with the
 * CFL time step, the BCs, and one pressure projection from p = 0. */
uf_status uf_init_state(uf_grid* g);

/* One time step: dt -> eddy viscosity -> MacCormack advection -> diffusion
 * -> drag + velocity BCs -> pressure solve (for the correction to the
 * pressure extrapolated in time, 2 p^n - p^{n-1}) -> projection -> k-omega
 * update.  The pressure state is held in twice the working precision (an
 * unevaluated pair of FP32 values for FP32 grids, FP64 for FP64 grids): it
 * grows upstream of the outlet far beyond the differences the projection
 * uses.  UF_FIELD_P reads and writes it rounded to the grid precision, and
 * a pressure written from outside has no history (p^{n-1} = p^n).  Replays a
 * captured CUDA graph;
 * the CG loop runs in a conditional (while) graph node, so the host never
 * waits inside the step.  stats == NULL: asynchronous.  stats != NULL: the
 * call synchronises the stream and fills *stats; a failed device check is
 * returned (UF_ERR_NOT_CONVERGED, UF_ERR_NAN). */
uf_status uf_step(uf_grid* g, uf_step_stats* stats);

/* nsteps calls of uf_step; stats (may be NULL) describe the last step and,
 * when given, the call synchronises and reports the first device error of
 * any of the steps. */
uf_status uf_run(uf_grid* g, int nsteps, uf_step_stats* last);

/* Pedestrian-level comfort objective on the current state: over cells whose
 * centre height lies in [z_lo, z_hi], the sum of max(|u_c| - u_hi, 0)^2 +
 * max(u_lo - |u_c|, 0)^2 with the cell-centre velocity averaged from the
 * faces; FP64 accumulation.  Synchronises. */
uf_status uf_objective(uf_grid* g, double z_lo, double z_hi, double u_hi, double u_lo, double* J_out);

/* Divergence diagnostic ||h div u||_2 / ||u_cell||_2 of the current
 * velocity.  Synchronises. */
uf_status uf_divergence(uf_grid* g, double* out);

/* Applies the pressure operator A (matrix-free 7-point, BC aware) to a cell
 * field x (device pointer, grid precision, dense) into y.  Synchronises. */
uf_status uf_apply_poisson(uf_grid* g, const void* x, void* y);

/* Solves A p = b with the grid's preconditioned CG starting from the grid's
 * current pressure; b is a dense cell field (host or device).  The result
 * replaces the grid's pressure.  Synchronises; fills iterations and the
 * final relative residual. */
uf_status uf_poisson_solve(uf_grid* g, const void* b, int* iters, double* rel_residual);

/* One time step computed by the same kernels as uf_step, but launched one
 * by one on the grid's stream with a CUDA event pair around every launch and
 * the CG loop polled from the host (the step advances the state exactly like
 * uf_step).  Writes up to `capacity` entries, one per kernel label, and the
 * number of labels to *count.  Synchronises.  Used to measure kernel
 * durations and for per-kernel profilers, which cannot see inside graphs that
 * hold conditional nodes. */
uf_status uf_profile_step(uf_grid* g, uf_kernel_time* out, int capacity, int* count, uf_step_stats* stats);

/* Kernel launches per step of the captured graph, counting every CG
 * iteration of the last step; 0 before the first step. */
int uf_last_step_launches(uf_grid* g);

/* Kernel launches of one graph step: *fixed outside the CG loop (including
 * the solver set-up) and *per_iter per CG iteration; with the cumulative
 * iteration count of uf_step_stats this counts every kernel a run launched.
 * Builds the step graphs if needed. */
uf_status uf_launch_counts(uf_grid* g, int* fixed, int* per_iter);

/* ---- Objectives ----------------------------------------------------------
 * UF_OBJ_COMFORT: the pedestrian comfort band of uf_objective, sum over the
 *   cells with centre height in [z_lo, z_hi] of max(|u_c| - u_hi, 0)^2 +
 *   max(u_lo - |u_c|, 0)^2.
 * UF_OBJ_REGIONS: the region-average objective of Sec. 6 ("Avoiding Heat
 *   Pockets in Early Design Stages"), L = sum_i (ubar_i - u_t)^2, ubar_i the
 *   mean of |u_c| over the cells whose centres lie in box i (regions[6i ..
 *   6i+5] = x0, x1, y0, y1, z0, z1 in m, host array); every box must hold at
 *   least one cell centre.
 * |u_c|: speed from the face averages at the cell centre. */
#define UF_MAX_REGIONS 8
enum { UF_OBJ_COMFORT = 0, UF_OBJ_REGIONS = 1 };
typedef struct {
  int kind;                  /* UF_OBJ_*                                      */
  double z_lo, z_hi, u_hi, u_lo;   /* comfort band                            */
  int nreg;                  /* regions: 1..UF_MAX_REGIONS                    */
  const double* regions;     /* 6 * nreg values                               */
  double u_t;                /* target speed [m/s] (0.55 in Sec. 6)           */
} uf_objective_desc;

/* The objective of the current state (synchronises).  Errors: UF_ERR_ARG
 * for a NULL descriptor or output, an unknown kind, nreg outside
 * 1..UF_MAX_REGIONS, a NULL region array or a box with no cell centre. */
uf_status uf_objective_ex(uf_grid* g, const uf_objective_desc* obj, double* J_out);

/* ---- Discrete adjoint and design gradients ----------------------------
 * The paper obtains design gradients by forward differences, N+1 forward
 * simulations per gradient (Sec. 4, "Automatic Design Optimization";
 * Sec. 6); these
 * entry points give the same gradient from one forward and one reverse
 * sweep: the hand-written transpose of every sub-step of uf_step (a1-a9 in
 * reverse; the pressure solve is self-adjoint because A is symmetric) and of
 * the comfort objective of uf_objective, with checkpointing every
 * ckpt_every steps and recomputation of each segment.  Non-smooth points
 * (clamps, limiters, upwind side, the drag cut-off, the MacCormack clamp)
 * take the branch of the forward pass.  The initial state is held fixed. */

/* Bytes of the caller-allocated device workspace uf_adjoint_run needs for
 * nsteps steps with checkpoints every ckpt_every steps (0 on bad input):
 * one taped segment of ckpt_every steps, the checkpoints and the adjoint
 * fields. */
size_t uf_adjoint_workspace_bytes(uf_grid* g, int nsteps, int ckpt_every);

/* From the grid's current state X0, runs nsteps steps (the grid needs
 * fixed_dt > 0), evaluates J = uf_objective(z_lo, z_hi, u_hi, u_lo) on the
 * final state, and sweeps back to give dJ/dphi, the gradient with respect
 * to the porosity field last set (dense cell field, grid precision, host or
 * device pointer; may be NULL).  Afterwards the grid holds the final state,
 * as after uf_run.  d_ws: device workspace of uf_adjoint_workspace_bytes().
 * Synchronises.  Errors: UF_ERR_ARG (no fixed dt, bad sizes), UF_ERR_NOMEM,
 * UF_ERR_STATE, and the solver errors of uf_step. */
uf_status uf_adjoint_run(uf_grid* g, void* d_ws, size_t bytes, int nsteps, int ckpt_every, double z_lo, double z_hi,
                         double u_hi, double u_lo, void* dJ_dphi, double* J_out);

/* uf_adjoint_run for any objective of uf_objective_ex; the descriptor is
 * checked, with the errors of uf_objective_ex, before any step runs. */
uf_status uf_adjoint_run_ex(uf_grid* g, void* d_ws, size_t bytes, int nsteps, int ckpt_every,
                            const uf_objective_desc* obj, void* dJ_dphi, double* J_out);

/* Vector-Jacobian product of one step (uf_step with the grid's fixed dt) at
 * the grid's current state X: given lam_out, the cotangent of the step's
 * output state, fills lam_in = (dX'/dX)^T lam_out and, if lam_phi is not
 * NULL, lam_phi = (dX'/dphi)^T lam_out.  lam_out and lam_in are arrays of
 * five dense field buffers in the order u, v, w, k, omega (grid precision,
 * host or device); the pressure is not an input (it only warm-starts the
 * solve).  The grid's state is restored afterwards.  d_ws: device workspace
 * of at least uf_adjoint_workspace_bytes(g, 1, 1) bytes.  Synchronises.
 * Errors as uf_adjoint_run. */
uf_status uf_step_vjp(uf_grid* g, void* d_ws, size_t bytes, const void* const* lam_out, void* const* lam_in,
                      void* lam_phi);

/* ---- Sub-steps and their transposes (test support) --------------------
 * One sub-step of uf_step applied in isolation to dense inputs (grid
 * precision, host or device, in the order listed), or, with transpose = 1,
 * its hand-written transpose at those inputs: out = J^T cot, the adjoints of
 * the inputs from cotangents `cot` of the outputs.  Face fields are u
 * (nx+1, ny, nz), v (nx, ny+1, nz), w (nx, ny, nz+1); cell fields (nx, ny,
 * nz); x fastest.
 *   UF_SUB_EDDY     (a1)  in u, v, w, k, omega  -> nu_t
 *   UF_SUB_ADVECT   (a2)  in u, v, w            -> u~, v~, w~ (interior faces; others 0)
 *   UF_SUB_DIFFUSE  (a3)  in u~, v~, w~, nu_t   -> u2, v2, w2 (interior faces; others 0)
 *   UF_SUB_DRAG_BC  (a4, a5) in u2, v2, w2, phi -> u3, v3, w3 (every face)
 *   UF_SUB_PROJECT  (a6-a8) in u3, v3, w3       -> u1, v1, w1 (pressure solved from 0)
 *   UF_SUB_TURB     (a9)  in u1, v1, w1, k, omega -> k', omega'
 * The grid needs fixed_dt > 0.  The call allocates and frees a scratch
 * block, synchronises, and leaves the grid without a usable state (set one
 * before stepping).  Errors: UF_ERR_ARG (no fixed dt, unknown sub-step, a
 * NULL list or buffer), UF_ERR_CUDA. */
enum { UF_SUB_EDDY = 0, UF_SUB_ADVECT = 1, UF_SUB_DIFFUSE = 2, UF_SUB_DRAG_BC = 3, UF_SUB_PROJECT = 4,
       UF_SUB_TURB = 5 };
uf_status uf_substep(uf_grid* g, int which, int transpose, const void* const* in, const void* const* cot,
                     void* const* out);

/* Parametric design -> porosity (smoothed cut-cell idea of Sec. 3, "Urban
 * model resolving"): nbox (<= 64) boxes with base footprints
 * boxes[4i..4i+3] = (x_a, x_b, y_a, y_b) [m] and parameters
 * theta[3i..3i+2] = (height, x shift, y shift) [m];
 * phi = prod_i (1 - chi_i), chi_i = s((x - x_a - dx)/w) s((x_b + dx - x)/w)
 * s((y - y_a - dy)/w) s((y_b + dy - y)/w) s((H - z)/w) at cell centres, s the
 * logistic function, w = width [m].  phi_out == NULL: sets the grid's
 * porosity (as uf_set_porosity); else writes the dense field there (host or
 * device).  boxes and theta are host arrays. */
uf_status uf_design_to_phi(uf_grid* g, int nbox, const double* boxes, const double* theta, double width,
                           void* phi_out);

/* Porosity from closed triangle meshes (Sec. 3, "Urban model resolving"):
 * tris = 9 * ntri doubles (three vertices x, y, z per triangle, m, host
 * array); object o is triangles [obj_first[o], obj_first[o] + obj_count[o])
 * with porosity obj_phi[o] inside (0 for a building, the canopy's value for a
 * tree).  A point is inside an object when it lies in the object's bounding
 * box and a ray from it crosses the object's triangles an odd number of
 * times (even-odd rule, Moller-Trumbore crossings, along the fixed direction
 * (0.5741, 0.6219, 0.5327)); a cell's porosity is the mean over sub^3
 * uniformly placed points of the minimum inside porosity of the objects
 * containing the point, 1 in the open (the cut-cell volume fraction).  The
 * decisions are made in FP64 with every operation rounded separately, so
 * they are reproducible.  phi_out == NULL: sets the grid's porosity (as
 * uf_set_porosity); else writes the dense field there (host or device).
 * Allocates and frees device memory for the mesh; synchronises.  Errors:
 * UF_ERR_ARG (NULL arrays, sub outside 1..16, a triangle range outside the
 * mesh, a porosity outside [0, 1], a non-finite vertex). */
uf_status uf_mesh_to_phi(uf_grid* g, int ntri, const double* tris, int nobj, const int* obj_first,
                         const int* obj_count, const double* obj_phi, int sub, void* phi_out);

/* Vector-Jacobian product of uf_design_to_phi: dJ/dtheta (host, 3*nbox
 * doubles) from dJ/dphi (dense cell field, grid precision, host or device).
 * Synchronises. */
uf_status uf_design_vjp(uf_grid* g, int nbox, const double* boxes, const double* theta, double width,
                        const void* dJ_dphi, double* dJ_dtheta);

/* ---- Launch tuning -----------------------------------------------------
 * Two knobs of the multigrid-preconditioned solve change only its speed, not
 * the iteration it computes: where the single-block shared-memory tail of
 * the V-cycle starts (the multigrid depth handled by per-level kernels) and
 * how many z planes each block of a per-level kernel marches over (the tile
 * depth).  Other preconditioners ignore them.  Results stay equal up to the
 * order of FP64 partial sums. */
#define UF_MAX_LEVELS 16
#define UF_UNFUSED_ADVECT 1
#define UF_UNFUSED_MOMENTUM 2
typedef struct {
  int tail_level;             /* first level of the tail; 0 = automatic (the
                                 shallowest level whose levels fit 64 KB of
                                 shared memory); values above the coarsest
                                 level, or below the shallowest level whose
                                 levels fit 220 KB, are clamped */
  int march_zc[UF_MAX_LEVELS];/* z planes per block of level l; 0 = automatic;
                                 otherwise even, 2..64 */
  int advect_zc;              /* z planes per block of the fused MacCormack
                                 advection; 0 = automatic (16), else 1..64 */
  int unfused;                /* bit mask of the step's fused kernels to run as
                                 their separate sub-step kernels instead:
                                 1 = the advection as its two passes
                                 (forward, backward); 2 = diffusion, drag +
                                 BCs and the pressure right-hand side as
                                 three kernels.  Both forms give the same
                                 values bit for bit.  0 = all fused (default) */
  int coarse_start;           /* first multigrid level of the V-cycle run as one
                                 thread-block-cluster launch (down legs, the
                                 tail, up legs); the levels above it use one
                                 launch per level and leg.  0 = automatic
                                 (per-level launches: on the coarse grids
                                 measured so far the cluster, which holds
                                 16 SMs at most, is no faster), -1 =
                                 per-level launches only.  Both give the same
                                 values bit for bit */
} uf_tuning;

/* The knobs in use, resolved (no zeros).  levels: number of MG levels. */
uf_status uf_get_tuning(uf_grid* g, uf_tuning* out, int* levels);

/* Sets the knobs (NULL: back to automatic) and drops the captured graphs,
 * which are rebuilt on the next call that needs them. */
uf_status uf_set_tuning(uf_grid* g, const uf_tuning* t);

/* Autotuner: times `reps` pressure solves of a fixed synthetic right-hand
 * side from a zero guess for each candidate (tail level x uniform tile
 * depth), keeps the fastest and returns it in *chosen (may be NULL) with its
 * mean solve time in *best_ms (may be NULL).  Uses only the grid's scratch
 * buffers: the state is untouched.  Synchronises. */
uf_status uf_autotune(uf_grid* g, int reps, uf_tuning* chosen, double* best_ms);

/* ---- Batched execution ---------------------------------------------------
 * Many independent grids -- design variants, wind directions, uneven sizes --
 * advance together: every phase of the step (a0-a9) is one persistent launch
 * over a work list of (instance, tile) items, sized to the SMs, and one
 * captured CUDA graph holds the whole step, with a single conditional WHILE
 * node for all instances' CG loops (instances that have converged skip their
 * items until the last one has).  Each instance computes exactly what it
 * computes alone with the same tuning.  Instances share the precision, the
 * MG preconditioner and the smoother. */
typedef struct uf_batch uf_batch;

#define UF_MAX_BATCH 64

/* Bytes of the device workspace of a batch of n (<= UF_MAX_BATCH) grids:
 * every grid's uf_workspace_bytes plus the batch's work lists. 0 on error. */
size_t uf_batch_workspace_bytes(int n, const uf_grid_desc* descs);

/* Creates the batch and its n grids inside d_workspace (caller-owned, as for
 * uf_create_grid); all work runs on `stream`. */
uf_status uf_batch_create(int n, const uf_grid_desc* descs, void* d_workspace, size_t bytes, void* cuda_stream,
                          uf_batch** out);

/* Handle of instance i, owned by the batch (do not uf_destroy it): set its
 * porosity and state, read fields, evaluate objectives, tune it. */
uf_status uf_batch_grid(uf_batch* b, int i, uf_grid** out);

/* nsteps batched steps of every instance (each needs a state).  stats: NULL
 * or n entries, filled after the last step (synchronises).  Errors of any
 * instance are reported (the first one wins). */
uf_status uf_batch_run(uf_batch* b, int nsteps, uf_step_stats* stats);

/* Kernel launches of one batched step: *fixed outside the CG loop and
 * *per_iter per CG iteration of the slowest instance. */
uf_status uf_batch_launch_counts(uf_batch* b, int* fixed, int* per_iter);

/* One batched step launched eagerly (no graph), each launch bracketed by
 * CUDA events on the batch's stream; the host polls the unfinished-instance
 * count before every CG iteration.  Fills per-kernel aggregates as
 * uf_profile_step does (names prefixed "b_"; bytes_per_launch summed over
 * the instances of the launch).  Advances every instance by one step. */
uf_status uf_batch_profile_step(uf_batch* b, uf_kernel_time* out, int capacity, int* count);

/* Autotunes per size class: instances with the same number of multigrid
 * levels and cell counts within a factor sqrt(2) (one half-octave bin) share
 * one tuning, chosen by uf_autotune on the first of them; the batch graphs
 * are rebuilt.  classes: number of size classes
 * (may be NULL). */
uf_status uf_batch_autotune(uf_batch* b, int reps, int* classes);

uf_status uf_batch_destroy(uf_batch* b);

/* ---- Pressure solve without any device allocation ---------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc or hand the library a workspace: code running
 * inside another framework's memory pool, plug-ins in a host application
 * that owns the CUDA context and forbids allocations after start-up, and
 * real-time loops that must never take the allocator's locks or fail with
 * out-of-memory mid-run.
 *
 * Solves A p = b with the operator of uf_poisson_solve (7-point, outlet
 * sides from wind_dir_deg get p = 0 ghosts, other sides dp/dn = 0) by CG
 * preconditioned with the paper's first-order approximate inverse (w = 1.65),
 * FP32 vectors, FP64 inner products, stopping at ||r|| <= tol ||b|| or after
 * max_iter iterations.  b (input) and p (warm start in, solution out) are
 * dense device arrays of nx*ny*nz floats, x fastest; stream is a created
 * cudaStream_t.  Synchronises; fills *iters and *rel_residual (may be NULL).
 *
 * Scratch: a file-scope __device__ array of UF_STATIC_SCRATCH_BYTES, which
 * every GPU that loads the library holds until the process exits.  Grids
 * above UF_STATIC_MAX_CELLS cells are rejected with UF_ERR_ARG.  The first
 * call on each device looks the array's address up (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream
 * capture.  Every call uses the same array and resets its solver state
 * first; calls that overlap on the GPU (other threads or streams) race on
 * it, so serialise them.  Calls no cudaMalloc or cudaFree. */
#define UF_STATIC_SCRATCH_BYTES (16u << 20)
#define UF_STATIC_MAX_CELLS 800000
uf_status uf_poisson_solve_static(int nx, int ny, int nz, double wind_dir_deg, const float* b, float* p,
                                  double tol, int max_iter, void* stream, int* iters, double* rel_residual);

/* Thread-local message of the last failure. */
const char* uf_last_error(void);

/* 1 if this library was built with -DUF_BOUNDS_CHECK (the debug build whose
 * kernels check every global index they form against its array and whose
 * calls then return UF_ERR_BOUNDS on a violation), else 0. */
int uf_bounds_checked(void);

#ifdef __cplusplus
}
#endif
#endif /* UF_H */
