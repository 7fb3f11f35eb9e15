/*
 * mpm.h -- C ABI of the GB300 implicit-MPM Newton step.
 *
 * One implicit material-point-method load step (Zhao, Li, Jiang & Choo,
 * "GeoWarp", arXiv 2507.09435, Sec. 2.2): the residual
 *   r(u^{n+1}) = assembled (f_int,p - f_ext,p)          (paper Sec. 2.2, residual eq.)
 * is driven to zero by Newton's method
 *   -J^{n+1,k} du^{n+1,k} = r(u^{n+1,k}),  J = dr/du     (paper Sec. 2.2, Newton eqs.)
 * until ||r^k|| / ||r^0|| <= tol                          (paper Sec. 2.2, criterion)
 * after which the particle state is updated and the grid reset (the paper's
 * four-stage procedure, Sec. 2.2).  Each Newton iteration runs, on the GPU:
 *   G2P of the nodal increment through quadratic B-spline gradients, the
 *   constitutive update (Neo-Hookean elasticity, optionally Drucker-Prager or
 *   modified Cam-Clay return mapping in principal logarithmic strain), P2G of
 *   the internal force into the FP64 residual, assembly of each particle's
 *   consistent tangent into a node-block sparse Jacobian (block size dim x dim,
 *   coupling +-2 nodes per axis: the 5^dim block neighbourhood of the paper's
 *   Sec. 3.2 / Table 1 for quadratic B-splines), and a block-Jacobi
 *   preconditioned BiCGStab or GMRES(m) solve.
 *
 * Conventions
 *   - Units SI; stress positive in tension; pressure p = tr(tau)/3.
 *   - Grid: n[a] cells per axis (n[2] ignored in 2D), spacing h, nodes at
 *     origin + i*h, 0 <= i <= n[a].  Node index ix + (nx+1)*(iy + (ny+1)*iz);
 *     a DOF index is node*B + component with B values per node: B = dim for
 *     MPM_SOLID, B = dim + 1 for MPM_UP (component dim is the pore pressure,
 *     positive in compression).  2D is plane strain.
 *   - Particle arrays passed in are HOST arrays in the caller's order; they
 *     are copied at the call.  The library keeps particles sorted by cell on
 *     the device; every getter returns them in the caller's original order.
 *   - Output buffers are caller-owned host arrays of the documented size.
 *   - The scene owns all device memory it allocates; mpm_destroy_scene frees it.
 *   - Every call returns an mpm_status; on error the scene keeps a message
 *     readable with mpm_last_error.  No C++ exception crosses this ABI.
 *   - A scene is used by one host thread at a time.  Distinct scenes may be
 *     driven concurrently, each on its own CUDA stream.
 */
#ifndef MPM_H
#define MPM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpm_scene mpm_scene;

typedef enum {
  MPM_OK = 0,
  MPM_ERR_INVALID_ARG = 1,
  MPM_ERR_OOM = 2,
  MPM_ERR_CUDA = 3,
  MPM_ERR_NOT_CONVERGED = 4,     /* Newton hit newton_maxit before tol        */
  MPM_ERR_KRYLOV_MAXIT = 5,      /* linear solve hit krylov_maxit             */
  MPM_ERR_KRYLOV_BREAKDOWN = 6,  /* BiCGStab/GMRES breakdown (zero divisor)   */
  MPM_ERR_NONFINITE = 7,         /* NaN/Inf in residual or state              */
  MPM_ERR_TIMEOUT = 8,           /* host-side wall-clock budget exceeded      */
  MPM_ERR_BOUNDS = 9,            /* a particle's support left the grid        */
  MPM_ERR_RETURN_MAP = 10,       /* local return-map Newton did not converge  */
  MPM_ERR_STATE = 11             /* call out of order (e.g. newton before begin) */
} mpm_status;

enum { MPM_NH = 0, MPM_NH_DP = 1, MPM_NH_MCC = 2 };        /* material models   */
enum { MPM_FP64 = 0, MPM_MIXED = 1 };                       /* precision modes   */
enum { MPM_BICGSTAB = 0, MPM_GMRES = 1 };                   /* Krylov methods    */
enum { MPM_FORCING_FIXED = 0, MPM_FORCING_EW = 1 };         /* linear tolerances */
enum { MPM_SOLID = 0, MPM_UP = 1 };                         /* formulations      */
enum { MPM_PC_AUTO = 0, MPM_PC_NODE = 1, MPM_PC_SEG4 = 2, MPM_PC_MG = 3 };  /* preconditioners */

typedef struct {
  int dim;                 /* 2 (plane strain) or 3                              */
  int n[3];                /* cells per axis                                     */
  double h;                /* grid spacing                                       */
  double origin[3];
  int precision;           /* MPM_FP64: Jacobian + Krylov in FP64;
                              MPM_MIXED: Jacobian + Krylov in FP32 (residual,
                              return map, eigen-decomposition and the Newton
                              check stay FP64 in both modes)                   */
  int krylov;              /* MPM_BICGSTAB or MPM_GMRES                          */
  int gmres_restart;       /* GMRES(m) restart length (default 30)               */
  double newton_tol;       /* relative residual tolerance (paper criterion)      */
  int newton_maxit;
  int forcing;             /* MPM_FORCING_FIXED: linear rtol = krylov_rtol;
                              MPM_FORCING_EW: Eisenstat-Walker choice 2,
                              clamped to [krylov_rtol, 0.01]                     */
  double krylov_rtol;
  int krylov_maxit;
  int formulation;         /* MPM_SOLID: dim displacement values per node;
                              MPM_UP (2D only): displacements and the pore
                              pressure, B = dim + 1 values per node (the
                              coupled formulation of the paper's Sec. 2.2
                              remark, verified in Sec. 4.4)                   */
  double dt;               /* MPM_UP: time step of a load step, s (> 0)          */
  double p_scale;          /* MPM_UP: weight of the mass-balance rows in the
                              Newton and Krylov norms and inverse scale of the
                              pressure unknown inside the solver; 0 = max over
                              materials of mu / h                              */
  int precond;             /* block-Jacobi blocks: MPM_PC_NODE one node's
                              B x B diagonal block; MPM_PC_SEG4 the 4B x 4B
                              diagonal block of four consecutive active nodes
                              (row order, mostly x-neighbours); MPM_PC_AUTO
                              (0): SEG4 for MPM_UP, NODE otherwise;
                              MPM_PC_MG: geometric multigrid V-cycle on the
                              background grid (every second node per level,
                              linear interpolation, Galerkin coarse operators
                              P^T J P, damped block-Jacobi smoothing, dense
                              coarsest level); BiCGStab only (MPM_GMRES with
                              MPM_PC_MG is MPM_ERR_INVALID_ARG)               */
  int jacobian_reuse;      /* 0 or 1: the Jacobian is assembled at every Newton
                              iteration (Newton's method, Sec. 2.2); k > 1: at
                              the first iteration of a load step and then at
                              every k-th one, the iterations between reusing
                              the last assembled Jacobian and its
                              preconditioner (modified Newton); negative:
                              MPM_ERR_INVALID_ARG                              */
} mpm_scene_desc;

typedef struct {
  int model;               /* MPM_NH, MPM_NH_DP, MPM_NH_MCC                       */
  double E, nu, rho;       /* Young's modulus, Poisson ratio, density           */
  double phi, psi, c;      /* DP friction / dilation angle (degrees), cohesion    */
  double M, lambda_cc, kappa_cc; /* MCC critical-state slope, compression indices */
  double pc0;              /* MCC initial preconsolidation pressure (negative)    */
  double k_hyd;            /* MPM_UP: hydraulic conductivity, m/s (Darcy flux
                              q = -(k_hyd / gamma_w) grad p)                   */
  double gamma_w;          /* MPM_UP: unit weight of the pore fluid, N/m^3      */
} mpm_material;

typedef struct {
  int status;              /* mpm_status of this iteration                       */
  int krylov_iters;        /* linear iterations spent in this Newton iteration   */
  double krylov_rel;       /* achieved relative linear residual (recurrence)    */
  double krylov_rtol;      /* requested relative linear tolerance               */
  double r_norm;           /* ||r^k|| over free DOFs after the update            */
  double rel_residual;     /* ||r^k|| / ||r^0||                                  */
  int n_plastic;           /* particles on the plastic branch at this iterate    */
} mpm_newton_report;

typedef struct {
  int status;
  int newton_iters;
  int converged;
  int krylov_iters_total;
  double r0_norm;
  double rel_residual;
  double hist[33];         /* relative residual after 0..newton_iters iterations */
  int krylov_iters[32];
  int n_active_nodes;
  long long nnzb;          /* structurally present Jacobian blocks              */
  double t_setup_ms, t_residual_ms, t_assembly_ms, t_krylov_ms, t_commit_ms;
} mpm_step_report;

/* Create a scene from host particle arrays.
 *   x[np*3] positions (z ignored in 2D); vol0[np], mass[np] (> 0);
 *   mat_id[np] in [0, nmat); E_p, phi_p: optional per-particle Young's
 *   modulus / friction angle overriding the material's (NULL = none);
 *   pc0_p: optional per-particle initial preconsolidation (NULL = material's);
 *   stream: a cudaStream_t to run on, or NULL for a stream the scene creates.
 * Errors: MPM_ERR_INVALID_ARG (bad sizes, a particle outside the grid's
 * interior, non-positive mass), MPM_ERR_OOM, MPM_ERR_CUDA. */
mpm_status mpm_create_scene(const mpm_scene_desc* desc, int np, const double* x,
                            const double* vol0, const double* mass, const int* mat_id,
                            const double* E_p, const double* phi_p, const double* pc0_p,
                            const mpm_material* mats, int nmat, void* stream,
                            mpm_scene** out);

/* Gravity vector used by the following load steps (f_ext = sum_p w_ip m_p g). */
mpm_status mpm_set_gravity(mpm_scene* s, const double g[3]);

/* Prescribed values for the following load steps: dof[k] = node*B + comp on
 * the dense node grid; value[k] is the displacement increment per load step,
 * or, for a pore-pressure DOF (MPM_UP), the pressure at the end of the step.
 * Replaces the previous set.  DOFs on nodes without mass are ignored.
 * Errors: MPM_ERR_INVALID_ARG for an index outside the grid. */
mpm_status mpm_set_dirichlet(mpm_scene* s, int n, const long long* dof, const double* value);

/* External forces carried by particles for the following load steps (the
 * Neumann term of the paper's weak form, Sec. 2.1: a surface traction times
 * the area of the particle's share of the loaded face), spread to the nodes
 * with w_ip like gravity.  particle[k] is a caller-order index, f[3k..3k+2]
 * the force in N (2D: N per unit thickness).  Replaces the previous set (all
 * other particles carry none).  Errors: MPM_ERR_INVALID_ARG. */
mpm_status mpm_set_traction(mpm_scene* s, int n, const int* particle, const double* f);

/* Stage a load step: sort particles by cell, find the active nodes
 * (nodal mass > 1e-12 * max particle mass) and the Jacobian pattern, apply the
 * prescribed increments, evaluate r^0.  `rep` (nullable) gets ||r^0||. */
mpm_status mpm_begin_step(mpm_scene* s, mpm_newton_report* rep);

/* One Newton iteration of the staged step: assemble J, solve J d = -r with
 * the configured Krylov method, update du += d, evaluate the new residual.
 * Returns MPM_ERR_STATE if no step is staged.  Does not commit. */
mpm_status mpm_newton_step(mpm_scene* s, mpm_newton_report* rep);

/* Replace the iterate of the staged step by du (host, nnode*B) and
 * re-evaluate the residual and the per-particle tangents there; prescribed
 * DOFs keep their prescribed increments.  For checks at chosen states and
 * for warm starts.  MPM_ERR_STATE if no step is staged. */
mpm_status mpm_set_du(mpm_scene* s, const double* du);

/* Assemble the Jacobian J = dr/du at the current iterate of the staged step
 * (readable with mpm_get_jacobian_bsr) without solving.  mpm_newton_step
 * does this itself; the call exists for inspection and external solvers. */
mpm_status mpm_assemble(mpm_scene* s);

/* Commit the staged step's converged increment to the particles
 * (x += sum_i w_ip du_i, F <- dF F, elastic strain and hardening variable). */
mpm_status mpm_commit_step(mpm_scene* s);

/* Whole load step: begin, Newton to newton_tol (at most newton_maxit), commit.
 * Returns MPM_ERR_NOT_CONVERGED (state not committed) when tol is missed.
 * Reproducibility: with MPM_BICGSTAB (any preconditioner) every sum of the
 * step (residual, nodal mass, Jacobian, norms, Krylov dot products) is taken
 * in an order that depends only on the inputs, so the same scene and steps
 * give the same results bit for bit, iteration counts included, on the same
 * GPU model and build; MPM_GMRES sums its dot products with atomics. */
mpm_status mpm_solve_step(mpm_scene* s, mpm_step_report* rep);

/* FP64 residual of the current iterate on the dense node grid, nnode*B
 * entries; prescribed and inactive DOFs read 0.  For MPM_UP the pressure rows
 * hold the fluid mass balance multiplied by dt (m^3; m^2 in 2D). */
mpm_status mpm_get_residual(const mpm_scene* s, double* r);
/* Current nodal iterate du (nnode*B: displacement increments, and for MPM_UP
 * the pore pressure) and nodal mass (nnode). */
mpm_status mpm_get_du(const mpm_scene* s, double* du);
mpm_status mpm_get_mass(const mpm_scene* s, double* mass);

/* Number of active nodes and of structurally present Jacobian blocks of the
 * staged step (the blocks whose node pair shares an occupied cell). */
mpm_status mpm_get_counts(const mpm_scene* s, int* n_active, long long* nnzb);

/* The Jacobian assembled for the latest Newton iteration, in block CSR:
 * row_node[n_active] node index of each block row, row_ptr[n_active+1],
 * col_node[nnzb] node index of each block, val[nnzb*B*B] row-major
 * blocks converted to double.  Rows and columns of prescribed DOFs hold the
 * identity.  Capacity `cap` in blocks; MPM_ERR_INVALID_ARG if too small. */
mpm_status mpm_get_jacobian_bsr(const mpm_scene* s, long long cap, int* row_node,
                                long long* row_ptr, int* col_node, double* val);

/* Multigrid hierarchy of the last assembly (MPM_PC_MG), for inspection.
 * *levels: levels in use (level 0 is the Jacobian itself, the last level is
 * solved with a dense inverse).  For 1 <= level < *levels: dims[3] the
 * level's node counts per axis (dims[2] = 1 in 2D), *nrow its active nodes;
 * when `nodes` is not NULL (room for `cap` rows): nodes[nrow] the active node
 * indices (x fastest), vals[nrow * S * B * B] the Galerkin operator P^T A P
 * as stencil blocks (S = 5^dim slots per row, slot (dx+2) + 5(dy+2)
 * [+ 25(dz+2)] for the neighbour at offset (dx, dy, dz); block row-major;
 * solver units: u-p pressure rows and columns carry p_scale), fixed[nnode*B]
 * (may be NULL) the level's prescribed-DOF flags, and *lambda_max (may be
 * NULL) the power-iteration estimate of lambda_max(D^-1 A) that sets the
 * smoother damping.  MPM_ERR_STATE without a hierarchy; MPM_ERR_INVALID_ARG
 * for a level out of range or `cap` too small. */
mpm_status mpm_get_mg_level(const mpm_scene* s, int level, int* levels, int dims[3], int* nrow, int cap,
                            int* nodes, double* vals, unsigned char* fixed, double* lambda_max);

/* One application of the multigrid preconditioner of the last assembly
 * (MPM_PC_MG): z = M^-1 b, the V-cycle the Krylov solve applies (its first
 * sweep from zero, the remaining sweeps, the coarse levels and the dense
 * solve), on the scene's stream and in its precision.  b and z: host arrays
 * of nnode*B doubles (node-major, x fastest; u-p in solver units, pressure
 * rows scaled by p_scale); b is rounded to the scene's precision, and z is 0
 * on nodes without a row.  Synchronises the scene's stream.  MPM_ERR_STATE
 * without a hierarchy (precond other than MPM_PC_MG, or before an assembly
 * of the staged step); MPM_ERR_INVALID_ARG for NULL pointers. */
mpm_status mpm_mg_apply(mpm_scene* s, const double* b, double* z);

/* Device-pointer variants: the caller's DEVICE buffers (for example the data
 * pointers of CUDA tensors on the scene's device), written on the scene's
 * stream without synchronising the host (order later work on that stream, or
 * synchronise it, before reading).  Same layouts and units as the host calls:
 * d_du and d_r hold nnode*B doubles (u-p pressure in physical units), d_x
 * np*3 doubles in the caller's particle order (z = 0 in 2D).  The scene's
 * own device memory is never handed out. */
mpm_status mpm_get_du_dev(const mpm_scene* s, double* d_du);
mpm_status mpm_get_residual_dev(const mpm_scene* s, double* d_r);
mpm_status mpm_get_positions_dev(const mpm_scene* s, double* d_x);
/* mpm_set_dirichlet with the DOF indices (int64) and values in device memory;
 * synchronises the scene's stream to report an index outside [0, nnode*B)
 * (MPM_ERR_INVALID_ARG; the out-of-range entries are skipped). */
mpm_status mpm_set_dirichlet_dev(mpm_scene* s, int n, const long long* d_dof, const double* d_value);

/* Particle state in the caller's original order (any pointer may be NULL):
 * x[np*3], be[np*6] elastic left Cauchy-Green (xx,yy,zz,xy,yz,xz),
 * pc[np] preconsolidation, F[np*9] deformation gradient (row-major),
 * tau[np*9] Kirchhoff stress of the committed state. */
mpm_status mpm_get_particles(const mpm_scene* s, double* x, double* be, double* pc, double* F,
                             double* tau);

/* Per-particle material parameters for the following load steps (caller
 * order, np values each; NULL keeps a field): Young's modulus E_p (> 0),
 * friction angle phi_p (degrees, Drucker-Prager), hydraulic conductivity
 * k_p (m/s, MPM_UP only).  Unstages a staged step. */
mpm_status mpm_set_params(mpm_scene* s, const double* E_p, const double* phi_p, const double* k_p);

/* Particle displacement increments of the staged step's current iterate,
 * du_p = sum_i w_ip du_i (caller order, np*3; z = 0 in 2D). */
mpm_status mpm_get_particle_increment(const mpm_scene* s, double* du_p);

/* Adjoint of the staged step at its current iterate (call it after the
 * Newton iterations have converged, before mpm_commit_step).  For a loss L
 * of the step's converged increment it solves J^T lambda = dL/du with the
 * Jacobian at that iterate and returns dL/dtheta = -lambda^T dr/dtheta
 * (the implicit-function adjoint of r(du; theta) = 0; the paper's inverse
 * analysis, Sec. 4.5, differentiates through its implicit steps the same
 * way).  The start-of-step particle state is held fixed: this is the
 * gradient of one load step.
 *   dL_dU   host, nnode*B: dL/du on the nodal DOFs in physical units (NULL = 0)
 *   dL_dx   host, np*3 (caller order): dL/d(du_p) on the particle
 *           increments of mpm_get_particle_increment (NULL = 0)
 *   grad_E, grad_phi  host, np (caller order) or NULL: dL/dE_p, dL/dphi_p
 *           (phi in degrees; zero for models without friction)
 *   grad_k  host, nmat or NULL: dL/dk_hyd per material (MPM_UP)
 * The linear solve uses the scene's Krylov method to a relative tolerance of
 * 1e-12 (FP64) or 1e-6 (mixed); a solve that stops early is accepted at a
 * relative residual of 1e-8 (FP64) or 1e-5 (mixed).  Afterwards the scene's matrix holds J^T
 * (mpm_get_jacobian_bsr would return it); a following mpm_newton_step
 * reassembles J.  Errors: MPM_ERR_STATE without a staged step,
 * MPM_ERR_KRYLOV_MAXIT / MPM_ERR_KRYLOV_BREAKDOWN if the solve fails. */
mpm_status mpm_adjoint(mpm_scene* s, const double* dL_dU, const double* dL_dx, double* grad_E,
                       double* grad_phi, double* grad_k);

/* Reverse chain through a sequence of load steps.  Step n maps the committed
 * particle state s_{n-1} = (x, be, pc, F) and the parameters to its converged
 * increment U_n and to the committed state s_n.  To differentiate a loss of
 * several steps, record s_{n-1} (mpm_get_particles) and U_n (mpm_get_du) on
 * the way forward; then, for n = N .. 1: restore s_{n-1} (mpm_set_state),
 * stage step n (mpm_set_dirichlet, mpm_set_gravity, mpm_begin_step), set its
 * converged increment (mpm_set_du) and call this.  On entry sbar_* hold the
 * adjoint dL/ds_n of the end-of-step state (caller order: x np*3, be np*6,
 * pc np, F np*9; zeros for the last step of a loss on increments only); on
 * exit they hold dL/ds_{n-1}.  dL_dU / dL_dx are the loss's direct gradients
 * on this step's increment as in mpm_adjoint.  The parameter gradients are
 * ADDED to grad_E, grad_phi (np) and grad_k (nmat) (each may be NULL).  The
 * per-particle partial derivatives of the commit map and of the residual
 * contribution with respect to the particle state and parameters are central
 * differences of the FP64 particle update (relative steps 1e-6 to 1e-7); the
 * transposed solve is as in mpm_adjoint.  Errors as mpm_adjoint. */
mpm_status mpm_adjoint_step(mpm_scene* s, const double* dL_dU, const double* dL_dx, double* sbar_x,
                            double* sbar_be, double* sbar_pc, double* sbar_F, double* grad_E,
                            double* grad_phi, double* grad_k);

/* Overwrite the committed particle state including positions (caller order;
 * x np*3, then as mpm_set_particles; any pointer may be NULL).  Unstages a
 * staged step.  MPM_ERR_INVALID_ARG for a position outside the grid
 * interior or an invalid be / F. */
mpm_status mpm_set_state(mpm_scene* s, const double* x, const double* be, const double* pc, const double* F);

/* MPM_UP: pore pressure of each particle after the last commit,
 * p_p = sum_i w_ip p_i (caller's order, np values).  MPM_ERR_INVALID_ARG for a
 * single-phase scene. */
mpm_status mpm_get_pressure(const mpm_scene* s, double* pp);

/* Number of CUDA kernels this scene has launched so far (including those
 * inside CUDA-graph launches). */
mpm_status mpm_kernel_launches(const mpm_scene* s, long long* out);

/* Newton globalisation counters of this scene since it was created:
 * *limited Newton corrections scaled down by the step-length limit (a node
 * moved by more than one cell width h), *halvings halved steps (a return map
 * left its domain, a state became non-finite or inverted, or the residual
 * norm did not decrease).  Either pointer may be NULL.  The paper's Newton
 * (Sec. 2.2) takes full steps; these safeguards are this library's. */
mpm_status mpm_get_newton_counters(const mpm_scene* s, long long* limited, long long* halvings);

/* Measured arithmetic peak of the current device (a measurement helper; the
 * paper has no counterpart): fused multiply-add throughput in TFLOP/s (2
 * flops per FMA) of a kernel of independent FMA chains timed with CUDA
 * events, FP64 (precision MPM_FP64) or FP32 (MPM_MIXED).  The FP64 residual
 * pass and the FP32 assembly are reported against it.  Synchronises the
 * device; allocates 8 bytes.  Errors: MPM_ERR_INVALID_ARG, MPM_ERR_CUDA. */
mpm_status mpm_fma_peak(int precision, double* tflops);

/* Time the Jacobian-vector product kernel of the staged step's assembled
 * Jacobian: `reps` launches on the scene's stream between CUDA events.
 * ms_per_launch: average duration; bytes_per_launch: algorithmic bytes of
 * one launch (present blocks, the input and output vectors, the row list). */
mpm_status mpm_time_spmv(mpm_scene* s, int reps, double* ms_per_launch, double* bytes_per_launch);

/* Overwrite the committed particle state (caller's particle order, host
 * arrays; any pointer may be NULL to keep that field): be[np*6] elastic left
 * Cauchy-Green (xx,yy,zz,xy,yz,xz), pc[np] preconsolidation, F[np*9].  With
 * mpm_get_particles this checkpoints and resumes a scene; it also sets an
 * initial (e.g. geostatic) stress state.  Unstages a staged step.
 * MPM_ERR_INVALID_ARG for a non-positive-definite be or det(F) <= 0. */
mpm_status mpm_set_particles(mpm_scene* s, const double* be, const double* pc, const double* F);

/* Free-DOF residual norm that allocates nothing (the paper has no counterpart;
 * this is a convenience of this library).  For callers that cannot call
 * cudaMalloc where they need the Newton convergence check: code running while
 * a host framework owns every device allocation, or a loop that forbids
 * allocation after start-up.
 *   r      device pointer, nnode*dim FP64 residual on the dense node grid
 *   rows   device pointer, nrow int32 node indices (the rows to include);
 *          each rows[k] must lie in [0, nnode): the call cannot check this
 *          (it is not given nnode), and an index outside is an out-of-bounds
 *          device read (undefined behaviour)
 *   fixed  device pointer, nnode*dim uint8 prescribed-DOF flags (1 = skip)
 *   dim    values per node, 2 or 3 (a 2D u-p residual has 3: u_x, u_y, p)
 *   out_norm  host pointer, receives sqrt(sum of r^2 over the free DOFs);
 *          nrow = 0 gives 0
 *   stream cudaStream_t to run on (NULL = legacy default stream); the call
 *          synchronises this stream and copies the result to the host, so
 *          it must not be called on a stream that is being captured into a
 *          CUDA graph (that would invalidate the capture).
 * Its only scratch is a file-scope device array of 8192 FP64 partial sums
 * (64 KiB per GPU that loads the library, held until exit), so nrow is
 * limited to 8192*256 = 2,097,152 rows; larger nrow returns
 * MPM_ERR_INVALID_ARG.  No cudaMalloc, cudaFree or allocating library call is
 * made.  The first call on a device looks up that array's device address with
 * cudaGetSymbolAddress (once per device, with that device current).  Every
 * call shares the array, so calls that overlap on the GPU race; order them on
 * one stream or with events.
 * Errors: MPM_ERR_INVALID_ARG, MPM_ERR_CUDA (a launch or copy failed, or a
 * CUDA error was already pending on this thread from earlier work: the call
 * then reports and clears it without launching); message from
 * mpm_noalloc_last_error. */
mpm_status mpm_residual_norm_noalloc(const double* r, const int* rows, int nrow,
                                     const unsigned char* fixed, int dim, double* out_norm,
                                     void* stream);
/* Message of the last failed mpm_residual_norm_noalloc call on this thread. */
const char* mpm_noalloc_last_error(void);

/* Device memory a scene of this size would take (for admission control): an
 * upper bound over particles, grid, tangents, Krylov vectors (the GMRES(m)
 * basis included), the stencil-BSR Jacobian with its block-Jacobi inverses
 * and the multigrid levels; the adjoint's transposed Jacobian is not
 * included.  Host arithmetic only.  MPM_ERR_INVALID_ARG for a bad desc. */
mpm_status mpm_footprint_bytes(const mpm_scene_desc* desc, int np, size_t* out);

void mpm_destroy_scene(mpm_scene* s);
const char* mpm_status_string(mpm_status st);
/* Last error message of a scene; with s == NULL, the message of the last
 * failed mpm_create_scene on this thread. */
const char* mpm_last_error(const mpm_scene* s);

#ifdef __cplusplus
}
#endif
#endif /* MPM_H */
