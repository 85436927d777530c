/*
 * jf.h - C ABI of libjf.so, a GB300 (sm_103a) implementation of the
 * finite-volume Runge-Kutta stage of the compressible Euler / Navier-Stokes
 * equations for an ideal gas, following JAX-FLUIDS (Bezgin, Buhendwa, Adams,
 * arXiv 2203.13760).
 *
 * What one RK3 step computes (all steps in hand-written CUDA kernels):
 *   conservative -> primitive variables      Section 2 (W, U, Eq. StiffenedGas, B = 0)
 *   WENO5-JS face reconstruction of W        Section 3.3, "High-order Godunov approach"
 *   HLLC flux with Einfeldt signal speeds    Section 3.3, Eq. (ApproxRiemannSolver)
 *   C4 viscous and heat fluxes               Sections 2 and 3.4
 *   flux divergence                          Section 3.1, Eq. (FVD)
 *   TVD-RK3 stage combination                Section 3.2 (Gottlieb & Shu 1998)
 *   CFL time step (FP64 max-reduction)       Section 3.2
 *
 * Conventions shared by every entry point
 *   - A field U is a caller-owned, contiguous device array of 5 components
 *     U[5][nz][ny][nx] (x fastest): rho, rho u, rho v, rho w, E.  Its element
 *     type is float when jf_scheme.dtype == JF_F32 and double for JF_F64, and it
 *     must be 16-byte aligned.  Only interior cells are stored; boundary
 *     conditions are applied inside the kernels.
 *   - Active axes are a prefix: (nx), (nx, ny) or (nx, ny, nz); an axis with one
 *     cell is inactive.  An active axis needs at least 5 cells.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every call only enqueues work on it and returns; nothing
 *     synchronises the host except jf_status_sync.
 *   - Device scalars (dt_dev, dt_used_dev) are FP64 device pointers.
 *   - Argument errors return synchronously (JF_ERR_ARG / JF_ERR_UNSUPPORTED)
 *     and enqueue nothing.  Conditions found on the device (non-physical
 *     state: rho <= 0, p <= 0 or not finite) set a device flag that
 *     jf_status_sync reports.  No call throws, traps or aborts.
 *   - The library owns its workspace (stage buffers, reduction scratch),
 *     allocated in jf_init / jf_batch_create; the step calls never allocate,
 *     except that the adjoint workspace is allocated at the first
 *     jf_rk3_step_vjp call of a handle.
 *   - A handle is used by one host thread at a time.  Two steps on one handle
 *     in different streams race on the shared workspace.
 */
#ifndef JF_H
#define JF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct jf_ctx* jf_handle; /* opaque, owned by the library */

typedef enum {
  JF_OK = 0,
  JF_ERR_ARG = -1,          /* invalid argument (null pointer, bad size or option) */
  JF_ERR_CUDA = -2,         /* a CUDA runtime call failed; see jf_last_error */
  JF_ERR_OOM = -3,          /* workspace allocation failed */
  JF_ERR_NONPHYSICAL = -4,  /* a kernel met rho <= 0, p <= 0 or a non-finite value */
  JF_ERR_TIMEOUT = -5,      /* reserved: a bounded device wait gave up */
  JF_ERR_UNSUPPORTED = -6   /* valid but unsupported configuration */
} jf_status;

typedef enum { JF_BC_PERIODIC = 0, JF_BC_ZERO_GRADIENT = 1, JF_BC_WALL = 2 } jf_bc;
enum { JF_F32 = 0, JF_F64 = 1 };
/* Scheme options (Table 2 of the paper; 0 is the Appendix A configuration). */
enum { JF_EINFELDT = 0, JF_DAVIS = 1, JF_TORO = 2 };           /* signal speed estimates */
enum { JF_FLUX_HLLC = 0, JF_FLUX_HLL = 1, JF_FLUX_RUSANOV = 2, /* Riemann solvers */
       JF_FLUX_ROE = 3,                                           /* flux splitting (ROE setup) */
       JF_FLUX_RUSANOV_NN = 4 };                                  /* Section 7.4 learned dissipation */
enum { JF_WENO5_JS = 0, JF_WENO5_Z = 1, JF_WENO3_JS = 2 };       /* reconstructions */

/* The Rusanov-NN dissipation network (Section 7.4): parameters per handle. */
#define JF_NN_HIDDEN 32
#define JF_NN_PARAMS (JF_NN_HIDDEN * 4 + JF_NN_HIDDEN + 2 * (JF_NN_HIDDEN * JF_NN_HIDDEN + JF_NN_HIDDEN) + JF_NN_HIDDEN + 1)
enum { JF_RK3 = 0, JF_RK2 = 1, JF_EULER = 2 };                   /* time integrators */

/* Cartesian grid of nx*ny*nz cells on [lo, hi] (Section 3.1: cuboid cells).
 * bc[] = {x-lo, x-hi, y-lo, y-hi, z-lo, z-hi} (west, east, south, north,
 * bottom, top; Section 3.7), each a jf_bc; periodic must be set on both sides
 * of an axis.  Zero gradient copies the nearest interior cell into the halo
 * (the "neumann"/transmissive boundary of Appendix A).  JF_BC_WALL is a slip
 * (symmetry) wall: the halo holds the mirror image of the cells inside, with
 * the momentum normal to the wall negated (the wall boundary of Table 2 for
 * inviscid flow; with viscosity the mirror makes it a free-slip wall).  Grids
 * with walls run in the run-time-scheme kernels; the adjoint does not
 * support them (JF_ERR_UNSUPPORTED). */
typedef struct {
  int nx, ny, nz;
  double lo[3], hi[3];
  int bc[6];
} jf_grid;

/* Ideal gas (Eq. StiffenedGas with B = 0) and transport (Section 2).
 * mu = 0 makes the run inviscid.  Heat conductivity
 * lambda = mu gamma R / ((gamma - 1) Pr). */
typedef struct {
  double gamma, R, mu, Pr;
} jf_gas;

/* Scheme options.  dtype: JF_F32 or JF_F64 (arithmetic and storage type of
 * the fields; the CFL reduction and dt are always FP64).  weno_eps: WENO5
 * epsilon (1e-6).  cfl: CFL number.  viscous / heat: include the viscous
 * stresses / heat flux (both need mu > 0).  safe_recon: 1 = a face side whose
 * reconstructed density or pressure is not positive falls back to its cell
 * value (the paper's "is_safe_reconstruction" flag, which it does not define
 * further).  Table 2 variants (a zero-initialised struct gives the Appendix A
 * configuration):
 *   signal_speed  JF_EINFELDT (Roe-averaged, Einfeldt 1988), JF_DAVIS (Davis
 *                 1988), JF_TORO (Toro 1994: PVRS star pressure)
 *   flux          JF_FLUX_HLLC (Toro 1994), JF_FLUX_HLL (Harten, Lax, van Leer
 *                 1983), JF_FLUX_RUSANOV (local Lax-Friedrichs); the signal
 *                 speeds apply to HLLC and HLL.  JF_FLUX_ROE selects the
 *                 flux-splitting formulation of Section 3.3 with the Roe
 *                 eigensystem and Roe splitting (the paper's "ROE" setup):
 *                 `recon` then reconstructs the split characteristic
 *                 fluxes, and safe_recon has no effect
 *                 JF_FLUX_RUSANOV_NN is Section 7.4's Rusanov flux with the
 *                 dissipation alpha = exp(NN(x)) of a network whose
 *                 parameters jf_set_nn gives (inputs x = (|u_R - u_L|,
 *                 (u_L + u_R)/2, (c_L + c_R)/2, |s_R - s_L|) along the face
 *                 normal, s = ln(p / rho^gamma) / (gamma - 1); three hidden
 *                 layers of JF_NN_HIDDEN ReLU units)
 *   recon         JF_WENO5_JS (Jiang & Shu 1996), JF_WENO5_Z (Borges et al.
 *                 2008, power 1), JF_WENO3_JS (Jiang & Shu 1996, third order:
 *                 weights 1/3 and 2/3)
 *   integrator    JF_RK3 / JF_RK2 (TVD Runge-Kutta of Gottlieb & Shu 1998,
 *                 Shu-Osher form) or JF_EULER, used by jf_rk3_step,
 *                 jf_rk3_run and jf_batch_step (the names keep the default).
 * The adjoint (jf_rk3_step_vjp) covers the default configuration (viscous
 * and heat fluxes included, no walls) with a tiled kernel, and inviscid runs
 * with any boundary condition, WENO5-JS or WENO3-JS, HLLC with Einfeldt
 * speeds or Rusanov-NN, and any of the three integrators with a per-face
 * kernel; other configurations return JF_ERR_UNSUPPORTED.  An option out of
 * range is JF_ERR_ARG. */
typedef struct {
  int dtype;
  double weno_eps;
  double cfl;
  int viscous, heat;
  int signal_speed;
  int safe_recon;
  int flux;
  int recon;
  int integrator;
} jf_scheme;

/* Create a solver for one grid.  Validates the configuration and allocates
 * the workspace (two stage buffers of 5*nx*ny*nz elements plus scalars) on
 * the current CUDA device.  On success *out owns them until jf_destroy.
 * Paper: the InputReader / Initializer / SimulationManager set-up of
 * Section 4.4. */
jf_status jf_init(const jf_grid* grid, const jf_gas* gas, const jf_scheme* scheme, jf_handle* out);

/* Release a handle (single-grid or batch) and its workspace.  Waits for the
 * device to finish work that uses the workspace.  NULL is accepted. */
jf_status jf_destroy(jf_handle h);

/* dUdt = L(U): the right-hand side of Eq. (FVD) (Section 3.1), i.e. the
 * Algorithm 3 loop over active axes (inviscid, viscous and heat fluxes) for
 * the field U.  U and dUdt are device arrays of the handle's dtype and must
 * not overlap. */
jf_status jf_rhs(jf_handle h, const void* U, void* dUdt, void* stream);

/* *dt_dev = CFL time step of U (Section 3.2; formula of this library):
 *   dt = CFL min(dt_c, dt_v), dt_c = min_d dx_d / max_cells max_d (|u_d| + c),
 *   dt_v = 3/14 min_d dx_d^2 / max_cells max(mu / rho, lambda / (rho c_v))
 *   (dt_v only when viscous or heat is on), computed in FP64.  U is a
 * 16-byte aligned device array of the handle's dtype (JF_ERR_ARG otherwise);
 * dt_dev receives one FP64 value. */
jf_status jf_compute_dt(jf_handle h, const void* U, double* dt_dev, void* stream);

/* One TVD-RK3 step in place (Section 3.2, Algorithm 2):
 *   U1 = Un + dt L(Un); U2 = 3/4 Un + 1/4 (U1 + dt L(U1));
 *   U^{n+1} = 1/3 Un + 2/3 (U2 + dt L(U2)).
 * dt_dev != NULL: fixed step read from device memory.  dt_dev == NULL: the
 * CFL step of Un (jf_compute_dt) is computed first.  dt_used_dev (may be
 * NULL) receives the step used. */
jf_status jf_rk3_step(jf_handle h, void* U_inout, const double* dt_dev, double* dt_used_dev, void* stream);

/* One Shu-Osher stage (Section 3.2): out = a Un + b (Us + dt L(Us)), with L
 * as in jf_rhs; Un may be NULL when a == 0, and out may equal Un (it is read
 * point-wise before it is written) but must not overlap Us.  jf_rk3_step is
 * three of these calls (a, b) = (0, 1), (3/4, 1/4), (1/3, 2/3); custom
 * Runge-Kutta schemes of the same form (Euler, TVD-RK2) use the same call.
 * dt_dev is an FP64 device scalar and must not be NULL. */
jf_status jf_stage(jf_handle h, const void* Us, const void* Un, void* out, double a, double b, const double* dt_dev,
                   void* stream);

/* n independent RK3 steps of host-resident states (the end-to-end form: a
 * serving loop of states that live in host memory): for k = 0 .. n-1, copy
 * U_in_host[k] to the device, advance it one step as jf_rk3_step does (dt_dev
 * as there; NULL = its own CFL step) and copy the result to U_out_host[k].
 * U_in_host / U_out_host: HOST arrays of n host pointers, each to a whole
 * state [5][nz][ny][nx] of the handle's dtype; pinned (page-locked) memory
 * lets the copies overlap the steps: the upload of state k + 1 and the
 * download of state k - 1 run on two internal streams while state k steps
 * on `stream`, in two device buffers of the handle (allocated, with the
 * streams, at the first call).  `stream` waits for the last download, so a
 * synchronisation of it makes every U_out_host[k] readable.  In and out
 * pointers may be equal (state k is read before it is written). */
jf_status jf_rk3_step_host(jf_handle h, const void* const* U_in_host, void* const* U_out_host, int n,
                           const double* dt_dev, void* stream);

/* nsteps RK3 steps in place, enqueued as one CUDA graph (captured at the
 * first call for a given (U, nsteps, dt mode) and replayed afterwards).
 * dt_dev as for jf_rk3_step (a fixed step is read at every step).
 * dt_hist_dev (may be NULL) receives the nsteps steps used. */
jf_status jf_rk3_run(jf_handle h, void* U_inout, int nsteps, const double* dt_dev, double* dt_hist_dev,
                     void* stream);

/* Adjoint of one fixed-dt RK3 step (vector-Jacobian product, Section 7.2:
 * gradients backpropagated through the solver):
 *   lam_in = (dU^{n+1} / dU^n)^T lam_out,
 * with U^{n+1} = RK3(U^n; dt) as in jf_rk3_step (the scheme's integrator:
 * TVD-RK3, TVD-RK2 or Euler) and dt held fixed (not
 * differentiated).  Un is the state at the start of the step (not modified);
 * the step is recomputed inside.  lam_out and lam_in are device arrays shaped
 * like U; they may not overlap.  dt_dev must not be NULL.  The first call of
 * a handle allocates its adjoint workspace: two states, and on 3D grids an
 * accumulator of 6 values per cell. */
jf_status jf_rk3_step_vjp(jf_handle h, const void* Un, const double* dt_dev, const void* lam_out, void* lam_in,
                          void* stream);

/* One fixed-dt TVD-RK3 step of U_inout in place (the same launches and
 * result as jf_rk3_step with dt_dev), keeping the stage states: U1_out and
 * U2_out (device arrays shaped like U, caller-owned, distinct from U_inout and
 * from each other) receive U1 = Un + dt L(Un) and
 * U2 = 3/4 Un + 1/4 (U1 + dt L(U1)) (Section 3.1, TVD-RK3).  They let the
 * adjoint of the step skip its recomputation (jf_rk3_step_vjp_stages).
 * JF_ERR_UNSUPPORTED unless the scheme's integrator is TVD-RK3. */
jf_status jf_rk3_step_keep(jf_handle h, void* U_inout, const double* dt_dev, void* U1_out, void* U2_out,
                           void* stream);

/* jf_rk3_step_vjp from the stage states of the step (Un, U1, U2 as kept by
 * jf_rk3_step_keep; not modified) instead of recomputing them: the three
 * stage-VJP launches only.  lam_in must differ from every other array.
 * JF_ERR_UNSUPPORTED unless the scheme is the default one (HLLC, Einfeldt
 * speeds, WENO5-JS, TVD-RK3) on a grid without walls; the other schemes use
 * jf_rk3_step_vjp. */
jf_status jf_rk3_step_vjp_stages(jf_handle h, const void* Un, const void* U1, const void* U2, const double* dt_dev,
                                 const void* lam_out, void* lam_in, void* stream);

/* jf_rk3_step_vjp for a handle whose flux is JF_FLUX_RUSANOV_NN, adding the
 * gradient of the step with respect to the network parameters (Section 7.4:
 * the learned dissipation trained through the solver):
 *   lam_in = (dU^{n+1}/dU^n)^T lam_out,  theta_bar += (dU^{n+1}/dtheta)^T lam_out,
 * with dt fixed.  theta_bar is a device array of JF_NN_PARAMS elements of the
 * handle's dtype in the layout of jf_set_nn; the call adds to it (the caller
 * zeroes it).  Supported: inviscid grids with any boundary condition,
 * WENO5-JS or WENO3-JS, and the scheme's integrator (TVD-RK3, TVD-RK2 or
 * Euler).  The contributions are summed with atomics, so the last bits may
 * vary from run to run. */
jf_status jf_rk3_step_vjp_params(jf_handle h, const void* Un, const double* dt_dev, const void* lam_out, void* lam_in,
                                 void* theta_bar, void* stream);

/* Adjoint of one fixed-dt step of every simulation of a batch in the same
 * launches (the per-face adjoint of jf_rk3_step_vjp's run-time schemes;
 * inviscid, WENO5-JS or WENO3-JS, HLLC with Einfeldt speeds or Rusanov-NN,
 * the scheme's integrator):
 *   lam_in[s] = (dU_s^{n+1}/dU_s^n)^T lam_out[s] + add[s],
 *   theta_bar += sum_s (dU_s^{n+1}/dtheta)^T lam_out[s]   (Rusanov-NN, if theta_bar != NULL).
 * Un_ptrs, lam_out_ptrs, lam_in_ptrs: HOST arrays of nsim device pointers
 * (the states at the start of the step, not modified; lam_in may not alias
 * lam_out or Un); add_ptrs: NULL or a HOST array of nsim device pointers
 * (NULL entries add nothing), the cotangent of a loss at U^n in a trajectory
 * sweep; dt_dev: nsim FP64 device values.  The step states are recomputed
 * inside; the adjoint buffers are allocated at the first call.  theta_bar as
 * in jf_rk3_step_vjp_params.  Paper: Section 7.4 (training over batches of
 * trajectory windows). */
jf_status jf_batch_step_vjp(jf_handle batch, void* const* Un_ptrs, const double* dt_dev, void* const* lam_out_ptrs,
                            void* const* lam_in_ptrs, void* const* add_ptrs, void* theta_bar, void* stream);

/* Deferred parameter gradient of a Rusanov-NN batch over a backward sweep
 * (Section 7.4: the gradient of a training loss sums over every face of
 * every stage of every step).  After jf_batch_param_grad_begin, each
 * jf_batch_step_vjp call with a non-NULL theta_bar (its value is not read)
 * keeps its face records (network inputs and cotangents) in a store owned by
 * the handle instead of adding to theta_bar, for at most max_steps calls
 * (JF_ERR_ARG beyond).  jf_batch_param_grad_end then adds the sum over all
 * kept records to theta_bar (a device array of JF_NN_PARAMS elements of the
 * batch's dtype) in one launch and leaves the deferred mode.  The result
 * equals the per-call gradients up to the order of the floating-point sums.
 * begin allocates the store (5 values per face per stage per step) when it
 * is smaller than needed; the other calls do not allocate. */
jf_status jf_batch_param_grad_begin(jf_handle batch, int max_steps);
jf_status jf_batch_param_grad_end(jf_handle batch, void* theta_bar, void* stream);

/* Loss of the adjoint workload: *loss_dev = sum_cells (rho - rho_target)^2 dV
 * (FP64 accumulation) and, if seed != NULL, seed = dloss/dU (the cotangent
 * that starts the backward pass: 2 (rho - rho_target) dV in the density
 * component, 0 elsewhere).  target is a device array of nx*ny*nz densities
 * of the handle's dtype. */
jf_status jf_loss_density_l2(jf_handle h, const void* U, const void* target, double* loss_dev, void* seed,
                             void* stream);

/* Training loss of Section 7.4 (the mean squared error of the primitive
 * state vectors of a predicted and a reference trajectory):
 *   *loss_dev = 1/(nstates ncomp ncells) sum (W(U) - W(Uref))^2,
 * over nstates states of ncells cells each, stored one after another as
 * [nstates][5][ncells] in U and Uref (device arrays of the handle's dtype,
 * 16-byte aligned), and over the primitive components (rho, u, v, p) for
 * ncomp = 4 (two-dimensional states) or (rho, u, v, w, p) for ncomp = 5;
 * FP64 accumulation.  If grad != NULL (same layout as U) it receives
 * dloss/dU through the transposed Jacobian of W(U).  h (a single-grid or
 * batch handle) supplies gamma and the reduction scratch; its grid is not
 * used.  Errors: JF_ERR_ARG for a null pointer, ncomp outside {4, 5} or a
 * non-positive count. */
jf_status jf_loss_primitive_mse(jf_handle h, const void* U, const void* Uref, long long nstates, long long ncells,
                                int ncomp, double* loss_dev, void* grad, void* stream);

/* Batch of nsim independent simulations with their own grid sizes (Section
 * 4.5, feed_forward over a batch of initial buffers; here sizes may differ).
 * All share gas and scheme and have the same number of active axes (1D, 2D
 * or 3D; JF_ERR_UNSUPPORTED otherwise); 1 <= nsim <= 65535.  The work list
 * holds the simulations' tiles, and for 3D grids and the row tiles of 2D
 * grids chunks of 32 planes (rows) along the march (jf_set_variant selects
 * 16 or 64).  Allocates each simulation's stage buffers and the work list. */
jf_status jf_batch_create(const jf_grid* grids, int nsim, const jf_gas* gas, const jf_scheme* scheme,
                          jf_handle* out);

/* Advance every simulation of a batch by nsteps RK3 steps in place, each
 * with its own CFL step (dt_dev == NULL is not allowed: dt_dev is an array of
 * nsim FP64 device values that receives the last step of each simulation).
 * U_ptrs is a HOST array of nsim device pointers to the simulations' fields
 * (same order as in jf_batch_create).  One persistent kernel launch per RK
 * stage covers all simulations; the nsteps steps are captured in a CUDA graph
 * at the first call for a given (U_ptrs, nsteps) and replayed afterwards. */
jf_status jf_batch_step(jf_handle batch, void* const* U_ptrs, int nsteps, double* dt_dev, void* stream);

/* feed_forward of Section 4.5: the solution trajectories of a batch for
 * nsteps steps of a FIXED step per simulation.  U0_ptrs: HOST array of nsim
 * device pointers to the initial states (read only).  traj_ptrs: HOST array of
 * nsim device pointers, simulation s owning (nsteps + 1) * 5 * N_s elements
 * of the batch's dtype laid out [t][5][nz][ny][nx]: slot 0 receives U0, slot
 * t + 1 one step of slot t (the paper's (N_b, N_T + 1, 5, ...) trajectory,
 * per simulation since sizes may differ).  dt_dev: device array of nsim FP64
 * steps.  The integrator of the scheme is used; the arithmetic is that of
 * jf_batch_step and jf_rk3_step, so slot t equals t fixed-dt steps of the
 * single-grid path bit for bit.  Asynchronous on `stream` except for the
 * upload of the per-call pointer tables (a stream-ordered allocation, freed
 * on the stream). */
jf_status jf_batch_feed_forward(jf_handle batch, void* const* U0_ptrs, void* const* traj_ptrs, int nsteps,
                                const double* dt_dev, void* stream);

/* Parameters of the Rusanov-NN network of a handle (single grid or batch)
 * whose scheme has flux == JF_FLUX_RUSANOV_NN (Section 7.4).  theta is a
 * caller-owned device array of nparams == JF_NN_PARAMS elements of the
 * handle's dtype: W1[32][4], b1[32], W2[32][32], b2[32], W3[32][32], b3[32],
 * W4[32], b4 (row-major, outputs by inputs).  The library keeps the pointer
 * and reads the values at every launch (in CUDA graphs too), so a caller
 * that updates theta in place between steps needs no new call; theta must
 * stay valid while work that uses it is in flight.  A new pointer drops the
 * handle's cached graphs.  Steps with that flux before this call return
 * JF_ERR_ARG.  Other schemes: JF_ERR_ARG. */
jf_status jf_set_nn(jf_handle h, const void* theta, int nparams);

/* Choose the launch variant of a handle (autotuner hook): `variant` indexes
 * the tile/schedule table of jf_variant_info; -1 restores the default (the
 * first entry, except for 2D grids whose rows padded to whole 128-cell row
 * tiles cover at most 8 % more cells than the first entry's tiles and give
 * at least 12 rows of row tiles per resident CTA: then the row tiles, which
 * march along y).  Returns JF_ERR_ARG for an index outside the table. */
jf_status jf_set_variant(jf_handle h, int variant);

/* Describe launch variant `variant` for the handle's dimensionality and
 * precision into buf (NUL-terminated, at most len bytes).  Returns the number
 * of variants (>= 1), or a negative jf_status. */
int jf_variant_info(jf_handle h, int variant, char* buf, int len);

/* Planes per CTA of the default launch variant of a 3D grid (host logic, no
 * GPU needed; the "auto" z chunk that jf_variant_info reports).  Inputs: the
 * grid's cells nx, ny, nz; the tile bx x by of the kernel; ctas_per_sm, the
 * CTAs of that tile resident on one SM; sms, the GPU's SM count.  With
 * tiles = ceil(nx/bx) ceil(ny/by) CTAs per plane and slots = sms x
 * ctas_per_sm: if one wave of 32-plane CTAs covers the grid, the chunk is
 * ceil(nz tiles / slots) (>= 1); otherwise it is the length z in 20..40
 * (the longest on ties) whose launch finishes first in a greedy schedule of
 * the CTAs in launch order (tiles CTAs per chunk, chunk after chunk, the
 * last chunk nz - (ceil(nz/z) - 1) z planes, each CTA costing its planes
 * plus half a plane of prologue) over `slots` identical slots; launches of
 * more than 400000 CTAs at z = 20 keep 32.  Returns the chunk (>= 1), or 0
 * if an argument is not positive. */
int jf_auto_zchunk(int nx, int ny, int nz, int bx, int by, int ctas_per_sm, int sms);

/* Wait for the handle's stream work (cudaDeviceSynchronize), then read and
 * clear the device error flag.  Returns JF_ERR_NONPHYSICAL if a kernel met a
 * non-physical state since the last call, JF_ERR_CUDA on a CUDA error,
 * JF_OK otherwise. */
jf_status jf_status_sync(jf_handle h);

/* Text of the last error on this handle ("" if none).  With h == NULL, the
 * last error of a call that had no valid handle (e.g. a failed jf_init).
 * The string is owned by the library and valid until the next call. */
const char* jf_last_error(jf_handle h);

/* Largest grid (cells) jf_rk3_step_noalloc accepts. */
#define JF_NOALLOC_MAX_CELLS 65536

/* One RK3 step exactly like jf_rk3_step, but with no handle and no device
 * memory allocation (the paper has no counterpart: this serves callers that
 * may not call cudaMalloc / cudaFree while they run, e.g. under a device
 * memory budget fixed at start-up or inside another library's hot loop).
 * The stage buffers, the CFL reduction scratch, dt and the error flag live in
 * one fixed device array compiled into libjf (about 5.2 MB, held by every GPU
 * that loads the library until the process exits), sized for
 * JF_NOALLOC_MAX_CELLS cells in FP64; larger grids are rejected with
 * JF_ERR_ARG and an explanatory jf_last_error(NULL).
 * grid / gas / scheme / U_inout / dt_dev / dt_used_dev / stream mean what
 * they mean for jf_init and jf_rk3_step.  The first call on a device resolves
 * the array's address and sets kernel attributes for that device (make that
 * first call before any stream capture).  Every call shares the array: calls
 * whose work overlaps on the GPU race and must be serialised by the caller.
 * Device-side non-physical states are not reported (there is no handle for
 * jf_status_sync). */
jf_status jf_rk3_step_noalloc(const jf_grid* grid, const jf_gas* gas, const jf_scheme* scheme, void* U_inout,
                              const double* dt_dev, double* dt_used_dev, void* stream);

/* Measurement helper (not part of the method): the fused-multiply-add rate
 * of the device in FLOP/s (2 per FMA) for dtype JF_F32 or JF_F64, from one
 * launch of a kernel of independent FMA chains at full occupancy (iters
 * loop trips of 128 FMAs per thread), timed with CUDA events on `stream`
 * after one shorter warm-up launch.  This is the ALU roofline of the stage
 * kernels.  Blocks the host until the timed launch ends; errors go to
 * jf_last_error(NULL). */
jf_status jf_fma_peak(int dtype, int iters, double* flops_per_s, void* stream);

/* Library version string. */
const char* jf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* JF_H */
