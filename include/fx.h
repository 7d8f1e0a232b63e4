/* fx.h -- C ABI of the GB300 (sm_103a) multigroup two-moment (M1) radiation-hydrodynamics
 * stage update.
 *
 * The method is the explicit transport + implicit interaction update of Skinner, Dolence,
 * Burrows, Radice & Vartanyan (2019), "FORNAX: a Flexible Code for Multiphysics Astrophysical
 * Simulations":
 *   - covariant Newtonian hydrodynamics and comoving multigroup radiation moments (Sec. 3,
 *     Eqs. 1-5, 11-12), finite-volume discretisation (Sec. 4, Eqs. 8-9);
 *   - coordinate-moment, TVD-limited parabolic reconstruction (Sec. 5.1, Eqs. 13-16), linear
 *     reconstruction of the radiation moments (Sec. 2);
 *   - HLLC gas fluxes, M1-closure HLL radiation fluxes with the diffusion-limit correction and
 *     contact-velocity upwinded advection (Sec. 5.2, Eqs. 17-19);
 *   - SSP-RK2 (Sec. 4) with the operator-split implicit energy and momentum coupling (Sec. 5.3,
 *     Eqs. 24-32; Sec. 6) after each stage.
 *
 * Every call returns an fx_status.  No exception or signal crosses the boundary.  Errors are
 * sticky per handle: once a call fails, later calls return the same status until
 * fx_clear_error().  fx_last_error() gives a human-readable reason.
 *
 * Threading: a handle is not thread-safe; use one handle per host thread.  All device work of a
 * handle runs on the CUDA stream given to fx_bind_workspace().
 */
#ifndef FX_H
#define FX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fx_grid fx_grid; /* opaque; created and owned by the library */

typedef enum {
  FX_OK = 0,
  FX_ERR_ARG = -1,         /* invalid argument or parameter combination                    */
  FX_ERR_CUDA = -2,        /* a CUDA runtime call or kernel launch failed                  */
  FX_ERR_WORKSPACE = -3,   /* no workspace bound, or the bound one is too small/misaligned */
  FX_ERR_NEWTON = -4,      /* the coupling's Newton and bisection failed in some cell      */
  FX_ERR_FLOOR = -5,       /* a density, pressure or radiation-energy floor was applied   */
  FX_ERR_NONFINITE = -6,   /* a non-finite value appeared in the state                     */
  FX_ERR_UNSUPPORTED = -7, /* parameters outside what this build supports                  */
  FX_ERR_BOUNDS = -8       /* debug build (FX_BOUNDS_CHECK) only: a kernel index fell outside
                              its buffer; the access went to the buffer's first element instead
                              and fx_last_error() names the first such index and its site      */
} fx_status;

enum { FX_OUTFLOW = 0, FX_PERIODIC = 1, FX_REFLECT = 2, FX_AXIS = 3 }; /* Sec. 7.5 */
enum { FX_CART = 0, FX_SPH = 1 };       /* Cartesian, or spherical (x1 -> r, x2 -> theta)  */
/* radial map (Appendix A): r = x1, r = exp(x1), or r = r_t sinh(x1 / r_t) (r_t = map_rt) */
enum { FX_MAP_ID = 0, FX_MAP_EXP = 1, FX_MAP_SINH = 2 };
enum { FX_FP64 = 0, FX_FP32 = 1, FX_FP32_F64NEWTON = 2 }; /* precision forms (see fx_params)  */
enum { FX_HLLC = 0, FX_HLLE = 1, FX_LLF = 2 };            /* gas Riemann solvers (Sec. 5.2)   */
enum { FX_NTOTALS = 6, FX_NBUDGET = 9 };

/* Grid, physics and solver parameters (plain data, copied at fx_grid_create).
 *   dims, n[d]         number of dimensions (1..3) and cells per direction (n[d] ignored for
 *                      d >= dims); each direction is uniform in its generic coordinate x^d
 *                      on [x_lo[d], x_hi[d]].
 *   geom, map1         FX_CART, or FX_SPH with dims == 2: x1 -> r through map1, x2 = theta.
 *   map_rt             r_t of FX_MAP_SINH (> 0; ignored by the other maps): nearly uniform in r
 *                      for r << r_t, logarithmic for r >> r_t.
 *   bc_lo/bc_hi        boundary condition per direction and side.
 *   ngroups            energy groups (1..32), logarithmically spaced edges
 *                      eps_min (eps_max/eps_min)^(g/ngroups) (Sec. 4).
 *   gamma              ideal-gas adiabatic index; c_v = 1/(gamma-1), T = p/rho.
 *   c_light, a_rad     (reduced) speed of light and radiation constant.
 *   kappa0, kap_*_exp  absorption opacity kappa_g = kappa0 rho^a T^b eps_g^d with
 *                      eps_g = sqrt(edge_g edge_g+1); a and b must be multiples of 1/2.
 *   sigma0             scattering opacity sigma = sigma0 rho.
 *   precision          FX_FP64: plain FP64 path.
 *                      FX_FP32: FP32 state, reconstruction, fluxes and coupling (the Newton
 *                      iterates on T - T^- so that FP32 resolves the change of T); FP64
 *                      conserved totals.
 *                      FX_FP32_F64NEWTON: as FX_FP32, but the temperature iterate, residual
 *                      and energy/momentum bookkeeping of the coupling in FP64.
 *                      State buffers are double for FX_FP64 and float otherwise.
 *   rad_recon_order    1 = linear + MC limiter (the paper's choice for radiation); 2 = the
 *                      gas's n = 2 parabola with its limiters, per group and moment (the
 *                      forward step only: fx_adjoint returns FX_ERR_UNSUPPORTED).
 *   couple             1 = apply the implicit interaction after each RK stage.
 *   newton_maxit, bisect_maxit, newton_rtol
 *                      coupling iteration caps and the relative temperature step tolerance.
 *   rho_floor, p_floor, E_floor
 *                      floors; applying the density or pressure floor sets FX_ERR_FLOOR, the
 *                      radiation-energy floor is a silent positivity floor.
 *   map_rt             see geom, map1.
 *   riemann            gas Riemann solver (Sec. 5.2): FX_HLLC (0, the paper's default), FX_HLLE
 *                      or FX_LLF (local Lax-Friedrichs).  The radiation advection is upwinded on
 *                      the HLLC contact speed of the face's states with every solver.
 *   shock_guard        carbuncle guard (Sec. 5.2), 0 = off: a face lies in a shock when the
 *                      pressures of its two cells differ by more than the factor 1 + shock_guard,
 *                      and with FX_HLLC a face of direction d takes HLLE when one of its cells
 *                      has such a face in another direction.  The adjoint needs FX_HLLC without
 *                      the guard (otherwise FX_ERR_UNSUPPORTED).
 *   vterms             1 = the velocity-dependent radiation terms of the comoving-frame moment
 *                      equations (Sec. 3.2, their group form; Sec. 5.2; Step 2 of Sec. 6) in
 *                      each stage's explicit operator: the work terms -v^i_;j P^j_i (energy) and
 *                      -v^i_;j F_i (flux), and the upwind frequency-space fluxes of nu P and
 *                      nu Q (Q: the M1 heat-flux tensor, Q_ijk = cE [(f-q)/2 (n_i d_jk + n_j d_ik
 *                      + n_k d_ij) + (5q-3f)/2 n_i n_j n_k], q = f (2 + 3 chi)/5), with
 *                      <v^i_;j> from the face velocities (v* normal, the upwind state's
 *                      transverse components).  Cartesian grids: the face differences over dx.
 *                      Spherical grids: the coordinate components' differences plus the
 *                      volume-averaged connection coefficients times the centroid velocity, in
 *                      physical components with the phi-phi entry (3-d tensors, F_phi = 0).
 *                      The adjoint returns FX_ERR_UNSUPPORTED with it.  0 = off.
 *   species, xi0       0 or 1: one radiation species (photons).  3: neutrinos (nu_e, anti-nu_e,
 *                      nu_x), each with the ngroups groups (3 ngroups <= 32 channels, species-
 *                      major), the composition rho Y_e advected with the gas, and the two-equation
 *                      interaction in (T, Y_e) of Sec. 5.3: the equilibrium channel energy
 *                      w_s(Y_e) B_g(T) with w = 2 Y_e, 2 (1 - Y_e), 1 (synthetic emissivities,
 *                      every species with the opacity law above), and the lepton number per unit
 *                      energy xi = -xi0/eps_g, +xi0/eps_g, 0, so that rho Y_e - sum xi E is
 *                      conserved.  Cartesian and spherical grids.  With vterms each species'
 *                      groups form their own chain in frequency; the terms leave rho Y_e
 *                      unchanged while moving energy between groups of different xi, so they do
 *                      not conserve rho Y_e - sum xi E.  Without boundary layers or the adjoint
 *                      (FX_ERR_UNSUPPORTED); in the FP32 forms the interaction iterates in FP64
 *                      on the FP32 Planck band table with FP32 channel arithmetic, to FP32
 *                      resolution, and stores the FP32 state.
 */
typedef struct {
  int dims;
  int64_t n[3];
  int geom;
  int map1;
  double x_lo[3], x_hi[3];
  int bc_lo[3], bc_hi[3];
  int ngroups;
  double eps_min, eps_max;
  double gamma, c_light, a_rad;
  double kappa0, kap_rho_exp, kap_T_exp, kap_eps_exp, sigma0;
  int precision;
  int rad_recon_order;
  int couple;
  int newton_maxit, bisect_maxit;
  double newton_rtol;
  double rho_floor, p_floor, E_floor;
  double map_rt;
  int riemann;
  double shock_guard;
  int vterms;
  int species;
  double xi0;
} fx_params;

/* State layout (upload, download, and the device copy inside the workspace): ncell = prod n[d],
 * cells in x-fastest order.  Gas block [2+dims][ncell]: rho, covariant momentum rho v_1..v_D,
 * total energy rho e.  Then the radiation block [1+dims][ncell][channels] (channel innermost;
 * channels = ngroups, or 3 ngroups species-major with three species): E, covariant F_1..F_D.
 * With three species, then the composition block [1][ncell]: rho Y_e.  fx_state_elems() gives
 * the element count. */

/* Validate parameters, build the geometry and reconstruction tables (host, FP64) and return the
 * workspace size in bytes the caller must provide.  *out receives the new handle (NULL on
 * error).  No device memory is allocated by the library for the state; small read-only
 * geometry tables are copied to the device at fx_bind_workspace. */
fx_status fx_grid_create(const fx_params* params, fx_grid** out, size_t* workspace_bytes);

/* Bind caller-owned device memory (e.g. a torch tensor) of at least `bytes` as the workspace,
 * 256-byte aligned, and the CUDA stream (cudaStream_t, may be NULL for the default stream) on
 * which all later work of this handle is enqueued.  The caller keeps ownership and must keep
 * the memory alive until fx_grid_destroy.  A handle may be bound again to other memory: the
 * tables and the boundary layers (at the handle's current time) are set in it, the status, the
 * budgets and the objective J start from zero, and the state must be uploaded again. */
fx_status fx_bind_workspace(fx_grid* h, void* dev_ptr, size_t bytes, void* cuda_stream);

/* Number of elements of the state in the layout above. */
size_t fx_state_elems(const fx_grid* h);

/* Copy a full state into the workspace.  src holds fx_state_elems() elements of type
 * src_precision (FX_FP64 = double, FX_FP32 = float) in host memory (src_is_device = 0,
 * synchronous) or device memory (src_is_device = 1, enqueued on the bound stream). */
fx_status fx_state_upload(fx_grid* h, const void* src, int src_precision, int src_is_device);

/* Build the state from primitives (Sec. 5.1 variables): prim is [3+dims][ncell] doubles ([4+dims]
 * with three species) with
 * rows rho, p, vhat_1..vhat_D (physical velocity), T_rad (and Y_e with three species: channel
 * energies w_s(Y_e) B_g(T_rad), composition rho Y_e).  Radiation starts in local
 * equilibrium, E_g = B_g(T_rad) (Planck group energy), F_g = 0.  Host or device pointer: host
 * primitives are staged through the second state buffer, as many cells at a time as fit, and the
 * call synchronises; device primitives are read on the bound stream. */
fx_status fx_state_init_equilibrium(fx_grid* h, const double* prim, int prim_is_device);

/* Enqueue nsteps SSP-RK2 steps of size dt on the bound stream (asynchronous).  Returns FX_OK
 * unless arguments are invalid, a launch fails or an earlier error is pending; device-side
 * conditions (Newton failure, floors, non-finite values) are reported by fx_sync().  Without
 * per-kernel timing and the objective, a step is captured once as a CUDA graph (on a stream the
 * library creates) and replayed per step; the capture is kept while dt, the workspace, the
 * budgets flag, kappa0, the march chunk and the boundary layers stay the same.  If capture
 * fails the kernels are launched one by one, with no status set. */
fx_status fx_step(fx_grid* h, double dt, int nsteps);

/* Wait for the bound stream and return the sticky status, including device-side conditions
 * raised by earlier fx_step calls. */
fx_status fx_sync(fx_grid* h);

/* Conserved totals over the grid (synchronises): out[0] mass, out[1..3] momentum components
 * including the radiation momentum sum_g F_g/c^2, out[4] total energy rho e + sum_g E_g,
 * out[5] radiation energy sum_g E_g; each sum_cells V (...) in FP64 with compensated
 * summation. */
fx_status fx_conserved_totals(fx_grid* h, double out[FX_NTOTALS]);

/* Budgets of the conserved totals (reading R13 of the paper's update: the comoving-frame
 * momentum coupling, Eqs. 31-32, does not conserve the total energy, and open boundaries let
 * every total change).  While enabled, every fx_step stage accumulates, in FP64 on the device:
 *   out[0] mass, out[1..3] momentum components (gas momentum plus the radiation momentum
 *   sum_g F_g/c^2) and out[4] total energy rho e + sum_g E_g, out[5] radiation energy, that
 *   leave through the faces of the non-periodic boundaries (outward flux times face area,
 *   weighted dt/2 per stage as the SSP-RK2 update weighs them; momentum components are
 *   covariant, meaningful as a budget on Cartesian grids);
 *   out[6] the energy the gas gives up to the flux absorption, sum_cells V (1/c^2) v . sum_g
 *   (F_g^new - F_g^-) (weight 1/2 after stage 1, 1 after stage 2);
 *   out[7] the radiation energy the silent positivity floor of E_g adds (same weights);
 *   out[8] the radiation energy the velocity-dependent terms add (vterms; weighted as out[4]).
 * Then, from the totals T of fx_conserved_totals at two times, T_mass(0) - T_mass(n) = out[0],
 * T_mom(0) - T_mom(n) = out[1..3] (Cartesian, without vterms: the flux equations' velocity
 * terms are not momentum-conservative), T_E(0) - T_E(n) = out[4] + out[6] - out[7] - out[8],
 * to round-off in FX_FP64 (in the FP32 forms, to the FP32 state's rounding).
 * fx_budgets_enable(h, 1) zeroes the accumulators (enqueued on the bound stream) and starts
 * accumulating; fx_budgets_enable(h, 0) stops (the default: the accumulation costs the kernels
 * registers and reductions, and the adjoint passes never add to it).  fx_budgets synchronises
 * and returns the sums since the last enable.  Both return FX_ERR_ARG for a null argument,
 * FX_ERR_WORKSPACE without a workspace, FX_ERR_CUDA on a failed copy, and the sticky status
 * first. */
fx_status fx_budgets_enable(fx_grid* h, int on);
fx_status fx_budgets(fx_grid* h, double out[FX_NBUDGET]);

/* Boundary layers: fixed and time-dependent boundary states, and reflecting walls on part of a
 * side, as boxes of grid cells that the library overwrites before each stage and after each
 * step (the double Mach reflection of Sec. 8.4 puts two such layers of cells on its fixed and
 * moving-shock sides).  A layer is one box [lo, hi) of cells and one rule:
 *   FX_LAYER_FRONT: state A where x - x0 - (y - y0) cot_alpha - speed t <= 0, else state B,
 *     with x, y the cell centre (y = 0 in 1-d) and t the time of the overwritten state.  A and B
 *     are primitives (rho, p, v_1..v_D, T_rad): E_g = B_g(T_rad), F_g = 0.  A fixed state is a
 *     front far away (x0 = 1e30, A = B).
 *   FX_LAYER_MIRROR: cell i along direction d takes the values of cell 2m - 1 - i, with the d
 *     components of momentum and radiation flux negated (a reflecting wall at the face m - 1/2).
 * Boxes may not overlap, and no mirror may read a cell of a box (otherwise FX_ERR_ARG).  The
 * layers apply at time t0 + the sum of the dt of the fx_step calls since: the stage-1 input at
 * t, the stage-2 input and the step's result at t + dt.  n = 0 removes them; at most 8 layers;
 * Cartesian grids only (FX_ERR_UNSUPPORTED); the adjoint returns FX_ERR_UNSUPPORTED while layers
 * are set.  Totals and budgets include the layer cells.  Returns the sticky status first,
 * FX_ERR_WORKSPACE without a workspace. */
enum { FX_LAYER_FRONT = 0, FX_LAYER_MIRROR = 1 };
typedef struct {
  int kind;
  int d, m;
  int64_t lo[3], hi[3];
  double x0, y0, cot_alpha, speed;
  double A[6], B[6];
} fx_layer;
fx_status fx_boundary_layers(fx_grid* h, const fx_layer* layers, int n, double t0);

/* Copy the state out, converting to dst_precision, to host (synchronous) or device memory. */
fx_status fx_state_download(fx_grid* h, void* dst, int dst_precision, int dst_is_device);

/* Number of kernel launches enqueued by one fx_step(dt, 1) call (per RK stage: the gas face
 * kernel, the radiation/update kernel, with the interaction on the interaction kernel (the
 * two-equation one with three species), with the carbuncle guard on the shock-flag kernel, with
 * vterms the velocity-term kernel, with three species the composition kernel, and the
 * objective's reduction while it is enabled; per step, with boundary layers, three layer
 * launches and the advance of the layers' time).  A step replayed as a captured graph launches
 * the same kernels. */
int fx_launches_per_step(const fx_grid* h);

/* Planes of the slowest axis that one block of the radiation/update kernel marches over: 32 (or
 * the axis length) until the workspace is bound, then fitted to the bound device by
 * fx_bind_workspace (fewest waves of blocks times planes per block).  0 for 1-d grids, -1 for a
 * null handle. */
int fx_march_chunk(const fx_grid* h);

/* Per-kernel device timing (instrumentation, not part of the method).  While enabled, every
 * stage that fx_step enqueues records four CUDA events on the bound stream: before the gas face
 * kernel, after it, after the radiation/update kernel, and after the interaction kernel (one
 * thread per cell, in every form; with the interaction off the last two events coincide; with
 * vterms the velocity-term kernel runs between the last two events).
 * fx_kernel_timing_enable(h, on) switches this on or off and discards what was recorded.
 * fx_kernel_timing_read(h, out) waits for the last recorded event and writes
 * out[0] = total milliseconds of the radiation/update kernel, out[1] = its launches,
 * out[2] = total milliseconds of the gas face kernel, out[3] = its launches,
 * out[4] = total milliseconds of the interaction kernel (with vterms, plus the velocity-term
 * kernel), out[5] = its launches (0 with both off), summed over the stages recorded since
 * enable or the previous read; it then starts a new record.  Each duration includes the launch
 * gap between the bracketing events (~1 us).  Both return FX_ERR_ARG for a null handle or output
 * and FX_ERR_CUDA when an event call fails. */
fx_status fx_kernel_timing_enable(fx_grid* h, int on);
fx_status fx_kernel_timing_read(fx_grid* h, double out[6]);

/* Host-side inspection (no GPU needed): the FP64 reconstruction/divergence table of direction d,
 * fx_debug_ntab() entries of n[d] + 4 rows each (padded cells -2 .. n+1), entry-major.  Returns
 * the number of doubles (copied only when cap is large enough), or -1 for a bad argument. */
int fx_debug_table(const fx_grid* h, int d, double* out, size_t cap);
int fx_debug_ntab(void);

/* Host-side inspection of the FP32 Planck band tables: for group g and node i (u = log2 T =
 * *u0 + i/32), with L = log2 of the band integral Int t^3/(e^t-1) dt over the group's edges
 * divided by T: out[4(g*nu + i) + {0,1,2,3}] = L - floor(L), (dL/du)/32, floor(L), and 2^floor(L)
 * (0 where floor(L) < -126).  Returns
 * the number of floats (copied only when cap is large enough), or -1 for a null handle. */
int fx_debug_planck_table(const fx_grid* h, float* out, size_t cap, int* nu, float* u0);

/* Equilibrium initialisation for callers that cannot allocate device memory: code running inside
 * a host that owns the allocator (a plugin, or a process under a memory pool that forbids
 * cudaMalloc) may have no workspace to stage host data in.  This call allocates nothing: it
 * stages the host primitives in a fixed device array that the library defines at file scope,
 * of FX_NOALLOC_STAGE_BYTES bytes (64 MiB, held by every GPU that loads the library until the
 * process exits; 1 KiB of it holds the group constants), then builds the state exactly as
 * fx_state_init_equilibrium does, but into the caller's device buffer `state` (fx_state_elems()
 * elements of state_precision, FX_FP64 or FX_FP32) on the given CUDA stream (NULL for the
 * default stream).  The paper has no counterpart; this is an interface convenience.
 *   - h may be unbound (no workspace): only its parameters and host tables are used.
 *   - prim: host array [3+dims][ncell] as for fx_state_init_equilibrium; at most
 *     FX_NOALLOC_STAGE_BYTES - 1024 bytes, otherwise FX_ERR_UNSUPPORTED with a message.
 *   - The first call on a device resolves the array's device address on the current device;
 *     make that first call before any stream capture.
 *   - Every call uses the same array and leaves its contents behind; calls that overlap on the
 *     GPU (other streams, other host threads) race on it.  Order them on one stream.
 *   - Asynchronous: the copies are enqueued on the stream; the host array may be reused when
 *     the call returns when it is pageable (the staging copy is then synchronous); page-locked
 *     (pinned) host memory is read by the copy engine later, so it must stay unchanged until
 *     the stream has executed the copy (synchronise the stream before reusing it).
 *   - Like every other entry point, returns the sticky status of an earlier device failure of
 *     the handle without enqueuing anything. */
#define FX_NOALLOC_STAGE_BYTES (64u << 20)
fx_status fx_state_init_equilibrium_noalloc(fx_grid* h, const double* prim, void* state,
                                            int state_precision, void* cuda_stream);

/* ---- Objective and adjoint (Cartesian grids) --------------------------------------------
 *
 * Objective J (the paper defines no objective; the one here is the boundary outflow that the
 * discrete update applies, so that its gradient is exact for the discrete map): the radiation
 * energy that the update itself
 * moves out through the upper x boundary, J = sum over steps of dt (Phi(U^n) + Phi(U^(1)))/2,
 * Phi = sum over groups and upper-x faces of face area x (corrected HLL energy flux + v* E
 * upwind term), Sec. 4 and Eqs. 17-19 of the paper.  Its gradient with respect to the initial
 * state and to the opacity normalisation kappa0 comes from a hand-written adjoint of the stage
 * (interaction: implicit-function derivative of the Newton system, Eqs. 25-28), run backwards
 * over checkpoints taken every k steps and recomputed segment by segment. */

/* Accumulate J during subsequent fx_step calls (on != 0; resets J to 0) or stop (on == 0).
 * While on, each stage enqueues one more small reduction kernel.  FX_ERR_UNSUPPORTED on
 * curvilinear grids. */
fx_status fx_objective_enable(fx_grid* h, int on);
/* J accumulated since fx_objective_enable (synchronises). */
fx_status fx_boundary_energy_out(fx_grid* h, double* J);
/* Set the opacity normalisation kappa0 (>= 0) used by subsequent steps. */
fx_status fx_set_kappa0(fx_grid* h, double kappa0);
/* Replace the density of the current state by rho (ncell values in the state's precision, host
 * or device), holding pressure, velocity, E_g and F_g fixed: m = rho v, rho e adjusted by the
 * kinetic energy change.  Host sources synchronise; device sources are stream-ordered. */
fx_status fx_state_set_density(fx_grid* h, const void* rho, int rho_precision, int rho_is_device);

/* Bytes of the caller-owned adjoint workspace for nsteps steps with a checkpoint every k steps:
 * ceil(nsteps/k) checkpoints, k + 1 segment states, 3k stage records, adjoint buffers. */
fx_status fx_adjoint_workspace_bytes(const fx_grid* h, int nsteps, int k, size_t* bytes);
/* Forward pass: from the current state, nsteps steps of size dt accumulating J (written to *J)
 * and storing the checkpoints in adj_ws (device memory, 256-byte aligned, at least the size
 * fx_adjoint_workspace_bytes gives).  The handle's state is left unchanged.  Synchronises. */
fx_status fx_adjoint_forward(fx_grid* h, double dt, int nsteps, int k, void* adj_ws, size_t adj_bytes,
                             double* J);
/* Backward pass over the checkpoints a preceding fx_adjoint_forward (same dt, nsteps, k, adj_ws
 * and kappa0) stored: gradients of seed * J.  grad_state (device, fx_state_elems() values of the
 * state's precision, state layout) receives dJ/dU^0 in conserved variables; grad_rho (device,
 * ncell values) receives dJ/drho(x, 0) at fixed pressure, velocity, E_g and F_g; *dJ_dkappa0 the
 * kappa0 derivative.  Any output may be NULL.  Synchronises; returns the sticky status of the
 * recomputed steps (FX_ERR_NEWTON etc.) like fx_sync. */
fx_status fx_adjoint_backward(fx_grid* h, double dt, int nsteps, int k, void* adj_ws, size_t adj_bytes,
                              double seed, void* grad_state, void* grad_rho, double* dJ_dkappa0);
/* Both passes (seed 1). */
fx_status fx_adjoint(fx_grid* h, double dt, int nsteps, int k, void* adj_ws, size_t adj_bytes,
                     void* grad_state, void* grad_rho, double* J, double* dJ_dkappa0);

const char* fx_last_error(const fx_grid* h);
void fx_clear_error(fx_grid* h);
void fx_grid_destroy(fx_grid* h);

#ifdef __cplusplus
}
#endif
#endif /* FX_H */
