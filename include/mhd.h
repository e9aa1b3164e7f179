/*
 * mhd.h — C ABI of the B300 library for one explicit hydrodynamic-magnetic-
 * hydrodynamic (H-M-H) Strang step of 2.5D ideal MHD on periodic uniform
 * Cartesian meshes: an entropy-stable DGSEM hydro stage (§3.2, Algorithm 1)
 * and a compatible finite-element magnetic-velocity stage (§3.3, Algorithm 2),
 * composed by Strang splitting (§3.4, Algorithm 3, eq. strang-composition).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Return value: 0 = OK, > 0 informational, < 0 error (see MHD_* codes);
 * mhd_last_error() gives a thread-local message for the last error.  No C++
 * exception crosses this boundary.
 *
 * Ownership: a context owns all of its device memory.  Inputs are copied in,
 * outputs are written to caller-owned buffers.  Pointers flagged `on_device`
 * are device addresses (for example torch tensors' data_ptr) and are accessed
 * on the context's stream; otherwise they are host addresses and the call
 * copies synchronously.
 *
 * Host layouts (all double, FP64):
 *   DG nodal fields  U[5][K][(p+1)^2], components (rho, m_x, m_y, m_z, E_mech),
 *                    K = ey*nx + ex, node j*(p+1)+i with i the x index; nodes
 *                    are the GLL(p) points of each element (§3.2).
 *   Bx               [ny*(k+1)][nx*(k+1)]: column ex*(k+1)+a, a = GLL(k+1)
 *                    node 0..k in x (node k+1 is node 0 of the next element),
 *                    row ey*(k+1)+b, b = Gauss(k) node in y  (R_h^k, x-comp).
 *   By               same shape, column = Gauss(k) node in x, row = GLL(k+1)
 *                    node in y (R_h^k, y-comp).
 *   Bz               [K][(k+1)^2] at the GLL(k) nodes of each element (V_h^k).
 *   Az (potential)   [ny*(k+1)][nx*(k+1)] at the GLL(k+1) nodes 0..k (W_h^{k+1}).
 * Here k is the magnetic base degree m of the paper, k in {p-1, p}.
 */
#ifndef MHD_H
#define MHD_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MHD_OK = 0,
  MHD_RETRIED = 1,          /* a rejected step succeeded after halving dt      */
  MHD_EINVAL = -1,          /* invalid argument                                 */
  MHD_ENOMEM = -2,          /* device allocation failed                         */
  MHD_ECUDA = -3,           /* a CUDA call failed (message in mhd_last_error)   */
  MHD_INADMISSIBLE = -4,    /* halvings exhausted; state restored to step start */
  MHD_NONFINITE = -5,       /* a non-finite value was produced                  */
  MHD_TIMEOUT = -6          /* a bounded device wait gave up                    */
};

typedef struct { int nx, ny; double x0, x1, y0, y1; } mhd_mesh_t;

/* Stabilisation switches and constants (§3.2.2, §3.3.3, §4 of the paper):
 * oe_hydro / oe_vel: hydro and velocity oscillation elimination; pp: Zhang-Shu
 * positivity limiter; ar: artificial resistivity; s_H, s_M: OE scale factors;
 * C_s, C_eta: A.R. sensor response and strength; cfl: CFL number of the
 * time-step reading; max_halvings: retries of a rejected step.
 * strang_order: 0 (default) the H-M-H composition of eq. strang-composition
 * and Algorithm 3, Phi_H^{dt/2} Phi_M^{dt} Phi_H^{dt/2}; 1 the M-H-M
 * composition Phi_M^{dt/2} Phi_H^{dt} Phi_M^{dt/2}, which reproduces the
 * printed temporal Cauchy differences of the paper's Table 3 digit for digit
 * (not supported by the adjoint).
 * reduced_2d2v: 1 selects the reduced magnetic stage of 2D2V configurations
 * (§4: u_z = B_z = 0, so the in-plane components of E_h and J_h vanish and are
 * not formed); it needs u_z = B_z = 0, which every step then keeps exactly.
 * On such states the result equals that of the full stage (0, default).  A
 * step that meets a nonzero m_z or B_z (or NaN) restores the state and
 * returns MHD_EINVAL.  The adjoint recomputes with the full stage. */
typedef struct {
  int oe_hydro, oe_vel, pp, ar;
  double s_H, s_M, C_s, C_eta, cfl;
  int max_halvings;
  int strang_order;
  int reduced_2d2v;
} mhd_params_t;

/* Diagnostics (DG-GLL quadrature for the fluid, exact magnetic product for
 * E_mag).  div_B is max_K min(hx,hy) max_{Gauss(k)^2} |dBx/dx + dBy/dy|.
 * n_rejections: rejected step attempts since the context was created.
 * stab_active: which stabilisation maps acted since the previous diagnostics
 * call (bit 1 a hydro OE factor D_p below 0.99, 2 the limiter scaled or
 * collapsed an element, 4 a positive A.R. coefficient, 8 a velocity-OE factor
 * below 0.99); reading clears it. */
typedef struct {
  double mass, mom[3], E_kin, E_int, E_mag, entropy, div_B, B_max, rho_min, p_min, eta_max;
  int n_rejections;
  int stab_active;
} mhd_diag_t;

typedef struct mhd_ctx mhd_ctx;

/* Create a context for a periodic nx x ny mesh of [x0,x1]x[y0,y1] with DGSEM
 * degree p (1..4) and magnetic base degree k (k = p-1 or k = p, k >= 0),
 * ratio of specific heats gamma > 1.  Allocates all device memory on the
 * current device.  Errors: MHD_EINVAL, MHD_ENOMEM, MHD_ECUDA. */
int mhd_create(const mhd_mesh_t* mesh, int p, int k, double gamma, mhd_ctx** out);
void mhd_destroy(mhd_ctx* ctx);

/* Reflecting walls by the method of images (§4.5 mirror boundaries, §4.7
 * reflecting walls; the paper gives no discrete wall treatment, reading R24).
 * The physical domain is the mesh given; the context stores and steps the
 * periodic domain doubled in every walled direction (walls: bit 0 the pair of
 * x-walls at x0, x1, bit 1 the y-walls), with the physical elements at
 * ex < nx, ey < ny and their mirror images beyond.  Every operator of the step
 * is reflection-equivariant, so a mirror-symmetric state stays so, and its
 * physical part is the solution with walls: no mass crosses a wall and the
 * normal velocity is odd across it.  The image parity of B per wall pair:
 * `conducting` bit set = a conducting wall (B_n odd, B_t even, so B_n = 0 on
 * the wall), clear = a symmetry plane (B_n even, B_t odd, field lines cross the
 * wall normally).  All state layouts, coordinates and sizes of the context
 * are those of the doubled periodic mesh; set the physical part, then call
 * mhd_mirror_fill.  mhd_diagnostics reports the physical part only.
 * Errors as mhd_create; walls outside 1..3 or conducting bits outside walls:
 * MHD_EINVAL. */
int mhd_create_walled(const mhd_mesh_t* mesh, int p, int k, double gamma, int walls, int conducting,
                      mhd_ctx** out);

/* Overwrite the image part of a walled context's state with the mirror images
 * of its physical part (normal velocity odd, B with the wall pair's parity;
 * on a conducting wall the normal B on the wall is set to 0).  MHD_EINVAL on a
 * context without walls.  Synchronises. */
int mhd_mirror_fill(mhd_ctx* ctx);

/* Stabilisation parameters (default: all off, s_H = s_M = 0.02, C_s = 5,
 * C_eta = 0.2, cfl = 0.4, max_halvings = 20, strang_order = 0,
 * reduced_2d2v = 0).  A negative constant, cfl <= 0, max_halvings < 0 or a
 * strang_order / reduced_2d2v outside {0, 1} is refused with MHD_EINVAL and
 * the previous parameters stay in force. */
int mhd_set_params(mhd_ctx* ctx, const mhd_params_t* prm);

/* Stream on which all work of the context is enqueued (a cudaStream_t). */
int mhd_set_stream(mhd_ctx* ctx, void* stream);

/* Sizes: K elements, N = K (p+1)^2 DG nodes, G = K (k+1)^2 magnetic grid
 * points per in-plane array, Z = K (k+1)^2 B_z values. */
int mhd_sizes(const mhd_ctx* ctx, long long* K, long long* N, long long* G, long long* Z);

/* Physical coordinates of the nodes into host buffers: which = 0 DG nodes
 * [N], 1 W nodes of the potential layout [G], 2 B_z nodes [Z]. */
int mhd_node_coords(const mhd_ctx* ctx, int which, double* X, double* Y);

/* Conservative state in (U [5][N]) and the magnetic field (host layouts). */
int mhd_set_state(mhd_ctx* ctx, const double* U, const double* Bx, const double* By, const double* Bz,
                  int on_device);
int mhd_get_state(mhd_ctx* ctx, double* U, double* Bx, double* By, double* Bz, int on_device);

/* Fluid state from nodal primitives rho [N], u [3][N], p [N] (m = rho u,
 * E_mech = p/(gamma-1) + rho|u|^2/2); the magnetic field is left unchanged. */
int mhd_set_primitive(mhd_ctx* ctx, const double* rho, const double* u, const double* p, int on_device);

/* The same exchange into a caller buffer, without touching the context's
 * state: rho [N], u [3][N], p [N] -> U [5][N] (m = rho u,
 * E_mech = p/(gamma-1) + rho|u|^2/2; the nodal variable exchange of §3.4.1
 * written for the pressure).  Synchronises the context's stream. */
int mhd_primitive_to_conservative(mhd_ctx* ctx, const double* rho, const double* u, const double* p, double* U,
                                  int on_device);

/* Vector-Jacobian product of mhd_primitive_to_conservative at (rho, u): for
 * lamU [5][N] = dJ/dU writes g_rho [N], g_u [3][N], g_p [N] = dJ/d(rho, u, p)
 * (the paper has no adjoint; this differentiates the exchange above).
 * Synchronises the context's stream. */
int mhd_primitive_to_conservative_vjp(mhd_ctx* ctx, const double* rho, const double* u, const double* lamU,
                                      double* g_rho, double* g_u, double* g_p, int on_device);

/* Magnetic field B = (Bx0 + (-dAz/dy), By0 + dAz/dx, Bz) from the nodal
 * W_h^{k+1} interpolant of a potential Az (exactly divergence-free). */
int mhd_set_B_from_potential(mhd_ctx* ctx, const double* Az, double Bx0, double By0, const double* Bz,
                             int on_device);

/* Physical coordinates of the nq x nq Gauss-Legendre points of every element
 * into host buffers X, Y [K][nq][nq] (x fastest, element K = ey*nx + ex),
 * 1 <= nq <= 16.  These are the points at which mhd_set_Bz_projected takes
 * its data. */
int mhd_quad_coords(const mhd_ctx* ctx, int nq, double* X, double* Y);

/* Out-of-plane field B_z set to the element-wise L2 projection onto V_h^k
 * (Q^k in the GLL(k) nodal basis of §3.1.3) of values fq [K][nq][nq] given at
 * the points of mhd_quad_coords (host or device memory per on_device).  The
 * element mass is exact for nq >= k+1; the data integral uses the nq-point
 * rule, exact when the data are polynomials of degree <= 2 nq - 1 - k.  The
 * paper does not state its initial B_z; this projection reproduces its
 * Table 1 (§4.1).  k+1 <= nq <= 16, else MHD_EINVAL.  The in-plane field and
 * the fluid state are unchanged. */
int mhd_set_Bz_projected(mhd_ctx* ctx, const double* fq, int nq, int on_device);

/* CFL time step of the current state (written to *dt). */
int mhd_compute_dt(mhd_ctx* ctx, double* dt);

/* One Strang step S^dt = Phi_H^{dt/2} o Phi_M^{dt} o Phi_H^{dt/2}
 * (Algorithm 3).  dt <= 0 means "use the CFL step".  A step whose raw stage
 * averages are inadmissible is restored and retried with dt/2 up to
 * max_halvings times: returns MHD_RETRIED with *dt_taken the reduced step, or
 * MHD_INADMISSIBLE with the state restored. */
int mhd_strang_step(mhd_ctx* ctx, double dt, double* dt_taken);

/* Several Strang steps at a fixed dt as one CUDA-graph launch (captured on the
 * first call for a given nsteps and replayed afterwards; parameter or stream
 * changes invalidate it); the status of the whole sequence is checked once at
 * the end.  If a raw average became inadmissible the state is restored to the
 * start of the sequence and MHD_INADMISSIBLE is returned with *steps_done = 0. */
int mhd_strang_steps(mhd_ctx* ctx, double dt, int nsteps, int* steps_done);

/* Batches of independent runs (the paper has no counterpart): every run has its own context (mesh, p, k, gamma, parameters
 * and state) and stream.  mhd_batch_step advances every run by nsteps Strang
 * steps with its own fixed dt (dt[i]) as ONE CUDA-graph launch holding a
 * parallel branch per run, then checks every run's status once.  The graph
 * is captured on the first call and re-captured when nsteps or a run's
 * parameters change; each run's result is bitwise that of mhd_strang_steps on
 * the run alone.  A run whose raw averages become inadmissible is restored to
 * the start of the call and reported MHD_INADMISSIBLE in status[i] (may be
 * NULL); the other runs keep their results. */
typedef struct mhd_batch mhd_batch;
int mhd_batch_create(int nruns, const mhd_mesh_t* meshes, const int* p, const int* k, const double* gamma,
                     mhd_batch** out);
void mhd_batch_destroy(mhd_batch* batch);
int mhd_batch_size(const mhd_batch* batch);
/* Context of run i (owned by the batch): use it to set states and parameters
 * and to read states and diagnostics. */
mhd_ctx* mhd_batch_run(mhd_batch* batch, int i);
int mhd_batch_step(mhd_batch* batch, const double* dt, int nsteps, int* status);
/* Kernel launches enqueued by the batch and its runs since creation. */
long long mhd_batch_launch_count(const mhd_batch* batch);

/* Tile autotuner (batching of independent problems; the paper has none): times the
 * elements-per-CTA variants of the volume kernel and of each of the three
 * magnetic-stage kernels (the E kernel first, then J, then the curl, the
 * others held) on the context's own mesh and CURRENT state (set a state first)
 * and keeps the fastest for every later launch (cached graphs are re-captured).
 * choices (may be NULL) receives [volume elements per CTA, elements per CTA of
 * the magnetic E kernel].  Synchronises; leaves the state unchanged. */
int mhd_autotune(mhd_ctx* ctx, int* choices);
/* Set the tile variants directly (0 = default, 1, 2; see mhd_autotune).
 * mag_variant 0..2 applies to all three magnetic kernels; 3..26 is the code
 * vE + 3 vJ + 9 vB of one variant per kernel (E, J, curl).  Errors:
 * MHD_EINVAL (a variant out of range or too large for the device). */
int mhd_set_tiles(mhd_ctx* ctx, int vol_variant, int mag_variant);
/* mhd_autotune for every run of a batch (each run keeps its own choice). */
int mhd_batch_autotune(mhd_batch* batch);

/* A single substep: which = 0 hydro Phi_H^tau (Algorithm 1), 1 magnetic
 * Phi_M^tau (Algorithm 2, with the nodal variable exchange around it). */
int mhd_substep(mhd_ctx* ctx, int which, double tau);

/* Test hook: hydro residual L_E (eq. euler-semidiscrete, mass-inverted) of a
 * conservative state U [5][N] into L [5][N]. */
int mhd_hydro_rhs(mhd_ctx* ctx, const double* U, double* L, int on_device);

/* Test hook: the hydro stage map P = P_PP o P_OE (eqs. euler-oe-map and
 * euler-pp-density/-pressure, §3.2.2-§3.2.3) of the enabled maps applied to a
 * conservative state U [5][N] with stage length tau >= 0 (the OE factors
 * D_l = exp(-s_H tau Theta_l)); the result goes to out [5][N] (host or
 * device per on_device, may alias U).  No residual, no stage combination and
 * no admissibility check: every element average must be admissible (rho > 0,
 * p > 0), as it is for the candidates the substeps pass to the map.  The
 * context's state is not touched; the map's activity bits are recorded as in a
 * step (mhd_diag_t.stab_active). */
int mhd_hydro_stage_map(mhd_ctx* ctx, const double* U, double tau, double* out, int on_device);

/* Test hook: magnetic residual L_M (eq. magnetic-dae) of a primitive state
 * (rho, e [N], u [3][N], B in host layouts, eta [K]) into de [N], du [3][N],
 * dBx, dBy [G], dBz [Z]. */
int mhd_mag_rhs(mhd_ctx* ctx, const double* rho, const double* e, const double* u, const double* Bx,
                const double* By, const double* Bz, const double* eta, double* de, double* du, double* dBx,
                double* dBy, double* dBz, int on_device);

/* ---- Adjoint (differentiation of the step; the paper has none) ----
 * Packed state vector of a context: [U 5N | Bx G | By G | Bz Z] in the host
 * layouts above (G = Z); its length is mhd_state_size().  An adjoint vector
 * lam has the same packing and holds dJ/d(state) of a scalar objective J. */
long long mhd_state_size(const mhd_ctx* ctx);

/* Vector-Jacobian product of one Strang step S^dt (Algorithm 3) at fixed dt:
 * lam_n = (dS^dt/dx)(state_n)^T lam_np1, written by hand in reverse mode
 * (transposed flux differencing with the Jacobians of the entropy-conservative
 * two-point flux and of the LLF flux, the adjoint SSP-RK(3,3) stages, the
 * transposed discrete curl, the adjoint lumped reconstructions of E_h and
 * J_h, and the adjoint nodal exchange).  The step's intermediate states are
 * recomputed from state_n on the device; the context's own state is not
 * touched.  Stabilisation: the maps that are enabled are differentiated
 * with their coefficients frozen at the values of the recomputed step (the
 * OE factors D_l and limiter factors theta of the hydro stage maps, the
 * factors and rho-weighted projector of the velocity OE, the A.R.
 * coefficient eta; the resistive Ohm load and the Ohmic heating themselves
 * are differentiated), and *flags (may be NULL) reports which are active (bit
 * 1 hydro OE, bit 2 limiter, bit 4 A.R., bit 8 velocity OE); the call returns
 * MHD_OK.  lam_n may alias lam_np1.
 * The first call allocates the adjoint's device buffers (about 14
 * state-sized vectors).  Errors: MHD_EINVAL, MHD_ENOMEM, MHD_ECUDA,
 * MHD_INADMISSIBLE or MHD_NONFINITE if the recomputed step leaves the
 * admissible set. */
int mhd_adjoint_step(mhd_ctx* ctx, const double* state_n, const double* lam_np1, double* lam_n, double dt,
                     int on_device, int* flags);

/* Adjoint of a checkpoint segment of nsteps fixed-dt Strang steps from the
 * packed state_0: one forward pass records the stage states of every step of
 * the segment in device memory (about 60 state-sized vectors per step; the
 * tapes stay allocated for later calls), then the step adjoints run from the
 * last step to the first: lam_0 = (d(S^dt)^nsteps/dx)(state_0)^T lam_end.
 * mhd_adjoint_step is the nsteps = 1 case.  Flags, frozen coefficients,
 * aliasing and errors as for mhd_adjoint_step. */
int mhd_adjoint_segment(mhd_ctx* ctx, const double* state_0, int nsteps, const double* lam_end, double* lam_0,
                        double dt, int on_device, int* flags);

/* Test hook: (dL_E/dU)(U)^T nu for the hydro residual of mhd_hydro_rhs
 * (U, nu, out [5][N]). */
int mhd_hydro_rhs_vjp(mhd_ctx* ctx, const double* U, const double* nu, double* out, int on_device);

/* Test hook: vector-Jacobian product of the ideal magnetic residual of
 * mhd_mag_rhs (eta = 0, where de/dt = 0 and nothing depends on e) with
 * respect to (rho [N], u [3][N], B): inputs w_u [3][N] and w_B (host layouts)
 * weight (du/dt, dB/dt); outputs g_rho [N], g_u [3][N], g_B. */
int mhd_mag_rhs_vjp(mhd_ctx* ctx, const double* rho, const double* u, const double* Bx, const double* By,
                    const double* Bz, const double* w_u, const double* w_Bx, const double* w_By, const double* w_Bz,
                    double* g_rho, double* g_u, double* g_Bx, double* g_By, double* g_Bz, int on_device);

/* Diagnostics of the current state. */
int mhd_diagnostics(mhd_ctx* ctx, mhd_diag_t* out);

/* Resistivity eta_K [K] of the last magnetic substep into a host buffer. */
int mhd_get_eta(mhd_ctx* ctx, double* eta);

/* Number of kernel launches enqueued by the context since creation. */
long long mhd_launch_count(const mhd_ctx* ctx);

/* Instrumentation (no counterpart in the paper): with enable != 0 every
 * subsequent launch group is bracketed by CUDA events on the context stream,
 * grouped in classes 0 face flux, 1 volume + stage combination, 2-4 magnetic
 * stage (one group per SSP stage: J loads, E loads + velocity, curl update),
 * 5 nodal exchange, 6 hydro stabilisation, 7 A.R. coefficient, 8 velocity
 * OE.  Enabling clears previous records. */
int mhd_profile_kernels(mhd_ctx* ctx, int enable);

/* Total event time in ms and number of groups per class since profiling was
 * enabled (arrays of nclasses entries); returns the number of classes. */
int mhd_kernel_times(mhd_ctx* ctx, double* ms, long long* counts, int nclasses);

/* Hydro residual L_E of a conservative state without any device allocation.
 * The paper has no counterpart: this exists for callers that cannot allocate
 * device memory themselves, for example code running while all device memory
 * belongs to a caching allocator or to a fixed budget of the host application,
 * or a latency-critical loop where a cudaMalloc/cudaFree pair is not
 * acceptable.  It computes what mhd_hydro_rhs computes, without a context: U
 * and L are caller-owned DEVICE buffers [5][K (p+1)^2] in the DG layout above;
 * the work is enqueued on `stream` (a cudaStream_t, 0 = legacy default stream)
 * and the call returns without synchronising.
 * Scratch: the face fluxes live in one file-scope device array of 2^20
 * doubles (8 MiB) that every GPU using the library keeps until the process
 * exits.  Meshes needing more than 10 K (p+1) <= 2^20 doubles are rejected
 * with MHD_EINVAL (p = 3: K <= 26,214 elements).  All calls share the array:
 * calls whose kernels overlap on the GPU race and must be serialised by the
 * caller.  Nothing in it needs to start at zero (each call writes what it
 * reads first).  Set-up: every call looks up the array's device address in
 * the current context (a cheap runtime query, so the address never goes stale
 * after cudaDeviceReset); the first call in a context also uploads the 1D
 * tables for degree p (synchronous copies to device symbols, repeated in a
 * context created after a reset).  Make that first call before any stream
 * capture.  U and L must be distinct, non-overlapping buffers of exactly
 * 5 K (p+1)^2 doubles on the current device: the call cannot check this, and
 * the Python binding does so before calling.
 * Errors: MHD_EINVAL, MHD_ECUDA (message in mhd_last_error). */
int mhd_hydro_rhs_static(const mhd_mesh_t* mesh, int p, double gamma, const double* U, double* L, void* stream);

/* Instrumentation (no counterpart in the paper): measured FP64 FMA issue rate
 * of the current device in TFLOP/s (FMA = 2 flops), from a probe kernel with
 * every lane active.  Allocates and frees a small buffer. */
int mhd_fp64_peak(double* tflops);

/* Test hook (no counterpart in the paper): y[i] = the library's FP64
 * reciprocal of x[i] for n device doubles, enqueued on `stream` without
 * synchronising.  The kernels use this reciprocal (the PTX seed
 * rcp.approx.ftz.f64 refined by one cubic Newton step) in place of division
 * for densities, pressures and their sums; it is specified for normal |x| in
 * [2^-1000, 2^1000].  Errors: MHD_EINVAL, MHD_ECUDA. */
int mhd_rcp_check(const double* x, double* y, long long n, void* stream);

/* Test hook (no counterpart in the paper): y[i] = the square root the kernels
 * use for sound speeds, Alfven speeds and the sensor's face-jump norms, for
 * n device doubles x (asynchronous on `stream`; x and y device pointers of n
 * doubles each, owned by the caller).  It is Heron's iteration seeded by the
 * PTX approximation rsqrt.approx.ftz.f64 (two steps, each one FMA residual),
 * within 1 ulp of IEEE sqrt for normal x >= 0; zero, subnormal, infinite and
 * NaN inputs follow IEEE sqrt, negative ones give NaN.  Errors: MHD_EINVAL,
 * MHD_ECUDA. */
int mhd_sqrt_check(const double* x, double* y, long long n, void* stream);

/* Debug build only (no counterpart in the paper; libmhd_debug.so, compiled
 * with MHD_BOUNDS_CHECK): the number of out-of-range global-memory indices the
 * checked kernels met since the last reset (each such access was redirected
 * to element 0 instead of being made); reset != 0 clears the counts.  The
 * release library returns -1.  Synchronises the device. */
long long mhd_debug_oob(int reset);

const char* mhd_status_string(int status);
const char* mhd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MHD_H */
