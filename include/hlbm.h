/*
 * hlbm.h - C ABI of the GB300 library for one full time step of the hybrid low-Mach
 * lattice Boltzmann / finite-difference combustion solver of Hosseini, Darabiha and Thevenin,
 * "Low Mach number lattice Boltzmann model for turbulent combustion: flow in confined
 * geometries" (Section 2).
 *
 * One step (lbm_step) is, for every cell:
 *   1. the finite-difference update of temperature and species (Section 2.3: explicit Euler,
 *      third-order WENO advection, centred second-order diffusion) with Arrhenius chemistry and
 *      the thickened-flame factor, producing rho and the dilatation Lambda of Eq. 3;
 *   2. in a closed domain, the thermodynamic-pressure update (a reduction over all cells);
 *   3. the lattice Boltzmann pull-stream and collide of Eq. 1, with the source Xi of Eq. 2,
 *      the moments of Eq. 7, the pre-conditioning of Eq. 13, the cumulant collision of
 *      Eq. 9-12 (or the single-rate special case) with a Smagorinsky eddy viscosity, and the
 *      post-collision populations of Eq. 8; bounce-back on solid cells.
 *
 * Conventions
 *   - Grid: nx * ny * nz cells (nz = 1 when dim == 2); cell index r = x + nx*(y + ny*z).
 *     Every field is structure-of-arrays, x fastest.
 *   - Lattice: D2Q9 (dim 2) or D3Q27 (dim 3). Direction i has velocity (cx, cy[, cz]) with
 *     i = (cx+1) + 3*(cy+1) [+ 9*(cz+1)]; the opposite of i is Q-1-i; weights are tensor
 *     products of (1/6, 2/3, 1/6).
 *   - Units: the configuration is SI; internally lattice units (dr = dt = 1, c_s^2 = 1/3).
 *     Velocities, pressures P_h and population values exchanged through this ABI are in lattice
 *     units; temperatures in kelvin; densities in units of cfg.rho_ref; P_th in pascal.
 *   - Masks: uint8 per cell, 0 = fluid, anything else = solid (never updated).
 *   - Boundaries per face: LBM_BC_PERIODIC, LBM_BC_WALL (halfway bounce-back, zero-gradient
 *     scalars), LBM_BC_INLET (low-x face only: bounce-back from a wall moving with the inlet
 *     velocity, Dirichlet T_in / Y_in), LBM_BC_OUTLET (high-x face only: anti-bounce-back
 *     pressure outlet at the half-way face, g_i = -g*_opp + 2 w_i (P_ref + rho (1.5 (c_i.u)^2
 *     - 0.5 u^2)) with u of the outlet cell from the previous step, i.e. twice the even part of
 *     the Eq. 6 equilibrium at the outlet pressure P_ref; zero-gradient T and Y).
 *   - Ownership: the caller owns every pointer it passes; the library copies inputs during the
 *     call and owns its internal device buffers (allocated through cfg.alloc/cfg.free when given,
 *     else cudaMalloc/cudaFree).
 *   - Streams: all work is enqueued on cfg.stream. With NULL the library creates its own blocking
 *     stream (which orders itself with the legacy default stream); step pairs are captured in
 *     CUDA graphs, which the legacy default stream does not allow. Calls that return data to
 *     host memory synchronise the stream.
 *   - Errors: nothing aborts or traps. Every call returns an lbm_status; lbm_last_error gives
 *     a one-line message. A context that returned LBM_ERR_CUDA should be destroyed.
 */
#ifndef HLBM_H
#define HLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = 1,         /* invalid argument or configuration                       */
  LBM_ERR_ALLOC = 2,       /* device allocation failed (or the allocator returned NULL) */
  LBM_ERR_CUDA = 3,        /* a CUDA runtime call failed                               */
  LBM_ERR_STATE = 4,       /* call out of order (e.g. step before set_fields)          */
  LBM_ERR_NONFINITE = 5,   /* a non-finite velocity was produced by a step             */
  LBM_ERR_UNSUPPORTED = 6, /* valid request this build does not implement              */
  LBM_ERR_TIMEOUT = 7      /* a bounded wait inside a kernel ran out (a data tile of the
                              tiled FD update did not arrive); the kernel returned early */
} lbm_status;

enum { LBM_BC_PERIODIC = 0, LBM_BC_WALL = 1, LBM_BC_INLET = 2, LBM_BC_OUTLET = 3 };
/* population storage: all arithmetic is FP64 for LBM_STORE_F64, FP32 otherwise. Populations are
 * stored shifted, h_i = (g_i - w_i P_ref) / w_i. */
enum { LBM_STORE_F64 = 0, LBM_STORE_F32 = 1, LBM_STORE_F16 = 2 };
enum { LBM_COLL_BGK = 0, LBM_COLL_CUMULANT = 1 };

#define LBM_MAX_SPECIES 8
#define LBM_MAX_REACTIONS 4

typedef struct {
  double W;   /* molar mass, kg/mol                     */
  double Le;  /* Lewis number (constant)                */
  double hf;  /* enthalpy of formation, J/kg            */
} lbm_species;

/* Irreversible Arrhenius step: q = A T^beta exp(-E/(R T)) prod_k [X_k]^order[k], [X] in mol/m^3,
 * q in mol/(m^3 s); omega_k = W_k nu[k] q (kg/(m^3 s)). Unused entries are 0. */
typedef struct {
  double A, beta, E;
  double nu[LBM_MAX_SPECIES];
  double order[LBM_MAX_SPECIES];
} lbm_reaction;

typedef void* (*lbm_alloc_fn)(size_t bytes, void* user);
typedef void (*lbm_free_fn)(void* ptr, void* user);

typedef struct {
  int dim, nx, ny, nz;
  int storage;    /* LBM_STORE_* */
  int collision;  /* LBM_COLL_*  */
  int bc_lo[3], bc_hi[3];
  int thermal;    /* 0: isothermal lattice Boltzmann only (rho = 1, Lambda = 0)           */
  double dx, dt;  /* grid spacing (m) and time step (s)                                  */
  double nu_ref;  /* kinematic viscosity at T_ref and density rho_ref, m^2/s               */
  double T_ref, mu_exp, Pr, cp, rho_ref; /* mu = rho_ref nu_ref (T/T_ref)^mu_exp; J/(kg K)  */
  double P_th0;   /* initial thermodynamic pressure, Pa                                  */
  double P_ref;   /* lattice pressure gauge of the shifted population storage            */
  double smag_cs; /* Smagorinsky constant (0 = off)                                      */
  double omega_bulk;  /* relaxation rate of the second-order trace                        */
  double omega_hi[4]; /* rates of cumulant orders 3, 4, 5, 6                              */
  double thicken_F;   /* thickened-flame factor                                           */
  int flame_sensor;   /* 1: F_loc = 1 + (F-1) tanh(beta Omega / wref), Omega =
                         max(Y_fuel,0) max(Y_ox,0) exp(-sensor_Ta / T)                      */
  int sensor_species, sensor_oxidizer;  /* fuel and oxidizer indices                        */
  double sensor_beta, sensor_wref, sensor_Ta; /* -, -, K                                    */
  int closed_domain;  /* 1: the global mass balance is reduced every step (FP64): M += inlet
                         minus outlet mass flux, I = sum W / (R T rho_ref); without a pressure
                         outlet P_th = M / I (a confined domain), with an outlet (bc_hi[0] =
                         LBM_BC_OUTLET) the domain is open to the ambient there and P_th stays at
                         P_th0 while M is still tracked. 0: P_th = P_th0, nothing reduced      */
  int n_species, n_reactions;
  lbm_species sp[LBM_MAX_SPECIES];
  lbm_reaction rx[LBM_MAX_REACTIONS];
  double T_in;                   /* inlet temperature, K                                   */
  double Y_in[LBM_MAX_SPECIES];  /* inlet mass fractions                                   */
  void* stream;                  /* cudaStream_t, NULL = a stream owned by the library      */
  lbm_alloc_fn alloc;            /* optional device allocator                              */
  lbm_free_fn free;
  void* alloc_user;
} lbm_config;

typedef struct lbm_ctx lbm_ctx;

/* Validate cfg, convert to lattice units (Eq. 12: tau = nu/c_s^2 + 1/2) and allocate the state.
 * Returns LBM_ERR_ARG for an invalid configuration, LBM_ERR_ALLOC if allocation fails. */
lbm_status lbm_init(const lbm_config* cfg, lbm_ctx** out);
void lbm_destroy(lbm_ctx* ctx);
const char* lbm_last_error(const lbm_ctx* ctx);

/* Geometry (Section 3: solid walls, obstacles, inlets). mask: N bytes. inlet_u: dim * ny * nz
 * doubles, the lattice velocity of each element (y + ny z) of the low-x inlet face, component
 * major; may be NULL when there is no inlet. on_device: 1 if both pointers are device memory.
 * Builds the per-cell link words (see lbm_get_links). */
lbm_status lbm_set_geometry(lbm_ctx* ctx, const uint8_t* mask, const double* inlet_u, int on_device);

/* Replace the inlet-face velocities only (same layout as in lbm_set_geometry), between steps;
 * fields, link words and captured graphs stay. on_device: 1 if inlet_u is device memory. Pinned
 * host memory is read in place by the device: keep it unchanged until the stream has passed the
 * call; pageable host memory may be reused on return. Requires lbm_set_geometry first. */
lbm_status lbm_set_inlet(lbm_ctx* ctx, const double* inlet_u, int on_device);

/* Variable heat capacities (Section 2.3 couples the solver to a thermochemistry library for the
 * mixture properties; that library is not available, and this is the reading used in its place):
 * cp: host array [n_species][5], c_p,k(T) = sum_m cp[k][m] T^m in J/(kg K); the species
 * enthalpies are h_k(T) = hf_k + integral from T0 to T of c_p,k (T0 in K: the temperature at
 * which the formation enthalpies hold). The temperature update then uses the mixture
 * c_p = sum_k Y_k c_p,k(T), the conductivity lambda = F mu c_p / Pr per cell (face value the
 * arithmetic mean), the heat release -sum_k h_k(T) omega_k and the species-enthalpy flux
 * sum_k (c_p,k - c_p) rho D_k grad Y_k . grad T (centred gradients), all divided by rho c_p; the
 * species equations are unchanged (constant Lewis numbers). cp = NULL returns to the constant
 * cfg.cp. Thermal runs only; takes effect from the next step (captured graphs are rebuilt). The
 * adjoint calls return LBM_ERR_UNSUPPORTED while it is on. */
lbm_status lbm_set_thermo(lbm_ctx* ctx, const double* cp, double T0);

/* Mixture-averaged species diffusion (Section 2.3: the paper evaluates its transport properties
 * with mixture-averaged approximations). Le_pair: host array [n_species][n_species] of pair Lewis
 * numbers, rho D_kj = mu / (Pr Le_kj) (binary diffusion data expressed against the conductivity;
 * the diagonal is not used); NULL returns to the constant Lewis numbers of cfg. Per cell the
 * Hirschfelder-Curtiss coefficient rho D_k = (mu / Pr) / Le_k^mix with
 * Le_k^mix = sum_{j!=k} (X_j + 1e-10) Le_kj / sum_{j!=k} (X_j + 1e-10), X_j = max(Y_j W / W_j, 0);
 * per face the mass flux is that of the mole-fraction gradient with a correction velocity,
 * J_k = G_k,f (dY_k + Y_k,f dlnW) - Y_k,f sum_j G_j,f (dY_j + Y_j,f dlnW) (arithmetic face means,
 * dlnW = (W_n - W) / mean W), so that the fluxes sum to zero and equal Le_kj give the constant-Lewis
 * update. The temperature equation is unchanged (constant c_p). The library allocates one
 * [(n_species + 1)][N] coefficient array on the first call. LBM_ERR_UNSUPPORTED together with
 * variable heat capacities or interpolated walls; the adjoint calls return LBM_ERR_UNSUPPORTED
 * while it is on. */
lbm_status lbm_set_transport(lbm_ctx* ctx, const double* Le_pair);

/* Initial fields: T [N] (K), Y [n_species][N], u [dim][N], P_h [N] (lattice), g_pert [Q][N]
 * (lattice, may be NULL). Populations are set to the equilibrium of Eq. 6 plus g_pert. T and Y
 * are ignored (may be NULL) when cfg.thermal == 0. Requires lbm_set_geometry first. */
lbm_status lbm_set_fields(lbm_ctx* ctx, const double* T, const double* Y, const double* u,
                          const double* P_h, const double* g_pert, int on_device);

/* Advance n_steps full steps of the hybrid scheme (Section 2), asynchronously on the context's
 * stream. Each step, in this order: the finite-difference update of T and Y_k (Section 2.3) with
 * the Arrhenius sources, the thickened-flame factor and the flame sensor, which also gives rho
 * and Lambda (Eq. 3) at the current level; in a closed domain the thermodynamic-pressure update
 * (P = M / I, a reduction over all fluid cells); the lattice Boltzmann stream and collide
 * (Eq. 1, 2, 7, 13, 9-12, 8) with that rho and Lambda. n_steps >= 0; LBM_ERR_STATE before
 * lbm_set_fields. Failures inside a kernel are reported by the next lbm_get_fields
 * (LBM_ERR_NONFINITE, LBM_ERR_TIMEOUT). */
lbm_status lbm_step(lbm_ctx* ctx, int n_steps);

/* Field selection bits for lbm_get_fields. Output is FP64, concatenated in bit order:
 * T [N], Y [n_species][N], u [dim][N], P_h [N] (Eq. 7a, last step), rho [N], Lambda [N]
 * (both at the level used by the last step), g [Q][N] (post-collision populations, unshifted).
 * Solid cells hold unspecified values. */
enum { LBM_F_T = 1, LBM_F_Y = 2, LBM_F_U = 4, LBM_F_PH = 8, LBM_F_RHO = 16, LBM_F_LAM = 32,
       LBM_F_G = 64 };
/* Number of doubles lbm_get_fields writes for these bits. */
size_t lbm_fields_size(const lbm_ctx* ctx, unsigned bits);
/* Reports LBM_ERR_NONFINITE if any step since the last check produced a non-finite velocity, and
 * LBM_ERR_TIMEOUT if a kernel's bounded wait for its data ran out (the fields are then invalid). */
lbm_status lbm_get_fields(lbm_ctx* ctx, unsigned bits, double* dst, int dst_on_device);

/* Thermodynamic pressure state: out[0] = P_th (Pa), out[1] = last increment of P_th (Pa per
 * step), out[2] = mass M (lattice units), out[3] = steps taken. Synchronises the stream. */
lbm_status lbm_get_scalars(lbm_ctx* ctx, double out[4]);

/* Per-cell link words (uint32, N): for a fluid cell bit i is set when direction i is a
 * bounce-back link (solid, wall or inlet source) and bit 31 is set; bit 30 marks cells with
 * interpolated bounce-back links (lbm_set_wall_fractions); solid cells hold 0. */
lbm_status lbm_get_links(lbm_ctx* ctx, uint32_t* dst, int dst_on_device);

/* Per-cell stencil words of the finite-difference update (uint32, N): for axis a and side s
 * (0: minus, 1: plus) the four bits at 4*(2a+s) hold the kind of the distance-1 point (bits 0-1:
 * 0 fluid, 1 wall or solid, 2 inlet, 3 outlet) and of the distance-2 point (bits 2-3: 0 fluid,
 * 1 zero-gradient copy of the distance-1 value, 2 inlet); bit 30 marks a cell with ghost-point
 * wall weights (see lbm_set_wall_fractions); bit 31 marks a fluid cell, solid cells
 * hold 0. Integer output, comparable bit for bit. */
lbm_status lbm_get_stencil_words(lbm_ctx* ctx, uint32_t* dst, int dst_on_device);

/* Curved or offset walls (the paper's curved-boundary treatment of the lattice Boltzmann solver,
 * Section 1; formulas are a reading: linearly interpolated bounce-back). q: host array [Q][N]
 * of doubles: for a fluid cell r and pull direction i whose source r - c_i is solid or outside
 * a wall face, the fraction in (0, 1] of the link r -> r - c_i at which the wall lies; other
 * entries are ignored, and q = 1/2 is half-way bounce-back (the default). A link with q < 1/2
 * whose node r + c_i is not fluid, and links of the inlet and outlet faces, stay half-way.
 * NULL clears the data. Must follow lbm_set_geometry (which clears it); synchronises the
 * stream. The finite-difference update uses the same fractions for its walls (ghost points): where
 * the distance-1 point along an axis is a wall or solid, the link toward it has fraction q and the
 * opposite point is fluid, the ghost value is phi_r + w (phi_opposite - phi_r) with
 * w = (1 - 2q) / (1 + 2q) (zero slope of the parabola through the two points at the wall); a
 * distance-2 wall point copies that ghost, or past a fluid neighbour takes the neighbour's. Cells
 * with such weights carry bit 30 of their stencil word (lbm_get_stencil_words). */
lbm_status lbm_set_wall_fractions(lbm_ctx* ctx, const double* q);

/* The same as a list of n_links links (host arrays): cell index r, pull direction i and the wall
 * fraction q of the link r -> r - c_i. Entries that are not bounce-back links of fluid cells, or
 * with q outside (0, 1], are ignored; n_links = 0 clears the data. For large grids, where a dense
 * [Q][N] array would not fit in host memory. */
lbm_status lbm_set_wall_links(lbm_ctx* ctx, long long n_links, const int* cell, const int* dir, const double* q);

/* Running statistics (the paper's diagnostics, Section 3: time-averaged and RMS fields).
 * op 0: reset the accumulators (allocated on first use); op 1: sample after every `interval`-th
 * step from now on (steps counted since set_fields; sampled steps run without CUDA graphs);
 * op 2: stop sampling. Per fluid cell and field (u components, P_h, and T for thermal runs):
 * mean and sum of squared deviations in FP32 by Welford's update. */
lbm_status lbm_stats_control(lbm_ctx* ctx, int op, int interval);

/* Statistics so far: dst holds 2 * nf * N doubles, the nf mean fields then the nf RMS
 * fluctuation fields (population standard deviation over the samples), fields in the order
 * u_x, u_y[, u_z], P_h[, T]; solid cells hold 0. n_samples (may be NULL) receives the count.
 * Synchronises the stream when dst is host memory. */
lbm_status lbm_get_stats(lbm_ctx* ctx, double* dst, int dst_on_device, long long* n_samples);

/* Flame surface in 2-D (Section 3.1 tracks the c = 0.2 and 0.8 iso-lines): length, in cells, of
 * the iso-line c = level of the progress variable c = (T - T_u) / (T_b - T_u) of the current
 * state, by marching squares over squares of four fluid cell centres (a corner equal to the
 * level counts as above; saddles are split by the mean of the corners). 2-D thermal runs only;
 * synchronises the stream. */
lbm_status lbm_flame_length(lbm_ctx* ctx, double level, double T_u, double T_b, double* length);

/* Properties of a planar flame propagating along x (Section 3.1 takes the burnt state, adiabatic
 * temperature and interface thickness from a 1-D freely propagating flame; Section 3.2.2 gives its
 * speed S_L and thickness delta_L = (T_max - T_min) / max dT/dx). From the current state, with
 * column means over the fluid cells of each x column (y, z):
 *   props[0] S_c, consumption speed (m/s): sum over fluid cells of (-omega_F / F_loc) dx /
 *            (rho_u Y_F,u A), A = ny nz cross-section cells, rho_u = P_th W_u / (R T_in) and
 *            Y_F,u = Y_in[fuel] the inlet state, omega_F the fuel rate of the Arrhenius law the
 *            update uses and F_loc its thickening factor (the flame sensor's value at the
 *            current state when the sensor is on), so that thickening leaves S_c unchanged;
 *   props[1] delta_L (m), (T_max - T_min) / max |centred difference of the column-mean T|
 *            (0 when the profile is flat);
 *   props[2] x_f (m), first crossing of (T_min + T_max) / 2 from low x, linear between column
 *            centres at x dx (-1 when there is none);
 *   props[3] T_min, props[4] T_max (K) of the column means;
 *   props[5] T_b, props[6 .. 6+K) Y_b: column means of the last column holding fluid.
 * props: host array of 6 + n_species doubles. profile: NULL or host array [2 + n_species][nx] that
 * receives the column means of T, of -omega_F / F_loc (kg/(m^3 s)) and of each Y_k (0 where a column holds
 * no fluid). Thermal runs with Y_in[fuel] > 0; synchronises the stream. */
lbm_status lbm_flame_properties(lbm_ctx* ctx, int fuel_species, double* props, double* profile);

/* Probes (Section 3.2 finds the precessing vortex core from the pressure recorded at points and
 * its spectrum). After every `interval`-th step the values u_x, u_y[, u_z], P_h[, T] (nf = dim + 1
 * [+ 1 thermal]) of each probe cell are appended to a ring of `capacity` samples; when it is full
 * the oldest sample is overwritten. cells: host array of n_probes fluid cell indices (LBM_ERR_ARG
 * for a solid or out-of-range cell). n_probes = 0 stops recording. Recording steps launch directly
 * (no graphs) and write P_h. Resets the sample count; synchronises the stream. */
lbm_status lbm_set_probes(lbm_ctx* ctx, int n_probes, const int* cells, long long capacity, int interval);

/* The recorded samples, oldest first: dst [n_samples][n_probes][nf] doubles (may be NULL to query
 * the count); n_samples (may be NULL) receives min(samples taken, capacity). Synchronises the
 * stream when dst is host memory. */
lbm_status lbm_get_probes(lbm_ctx* ctx, double* dst, int dst_on_device, long long* n_samples);

/* Welch estimate of the one-sided power spectral density of the device series x[i * stride],
 * i < n, sampled every dt seconds: segments of seg_len samples (even, >= 4, <= n) advancing by
 * seg_len / 2, each with its mean removed and the periodic Hann window (1 - cos(2 pi j / seg_len))/2
 * applied; |DFT|^2 averaged over the segments, times dt / sum(window^2), doubled except at
 * frequency 0 and seg_len / 2. psd: host array of seg_len / 2 + 1 doubles, bin f at frequency
 * f / (seg_len dt) Hz, in units^2 / Hz. Synchronises the stream. */
lbm_status lbm_welch_psd(lbm_ctx* ctx, const double* x, long long n, long long stride, double dt, int seg_len,
                         double* psd);

/* lbm_welch_psd of one probe's field (0 .. nf-1 in the order above) over the recorded samples,
 * oldest first, dt = interval * cfg.dt. */
lbm_status lbm_probe_spectrum(lbm_ctx* ctx, int probe, int field, int seg_len, double* psd);

/* Checkpoint: bytes of device memory needed, save into / load from caller-owned device memory. */
size_t lbm_state_bytes(const lbm_ctx* ctx);
lbm_status lbm_save_state(lbm_ctx* ctx, void* dst_device);
lbm_status lbm_load_state(lbm_ctx* ctx, const void* src_device);

/* Kernel timing (CUDA events on the context's stream). enable=1 starts recording each
 * kernel launch of lbm_step; lbm_kernel_times returns, per kernel kind, the summed device time
 * in ms and the launch count since the last reset:
 *   kind 0 finite-difference update, 1 flame sensor, 2 thermodynamic pressure, 3 lattice
 *   Boltzmann stream-collide. The flame-sensor pass runs only for the first step after the state
 *   was set from outside (lbm_set_fields, lbm_load_state); afterwards each finite-difference
 *   update writes the sensor's F_loc of the state it produces. Synchronises the stream. */
#define LBM_KERNEL_KINDS 4
lbm_status lbm_profile(lbm_ctx* ctx, int enable);
lbm_status lbm_kernel_times(lbm_ctx* ctx, double ms[LBM_KERNEL_KINDS], long long launches[LBM_KERNEL_KINDS]);

/* Algorithmic bytes of one launch of each kernel kind (each array touched once). */
lbm_status lbm_kernel_bytes(const lbm_ctx* ctx, double bytes[LBM_KERNEL_KINDS]);

/* Adjoint of one step (discrete reverse mode; the paper has no adjoint, this is the exact
 * transpose of lbm_step's update: LB stream-collide, bounce-back, inlet and outlet rules,
 * FD transport and chemistry). Supported: 2-D, FP32 or FP64 storage, cumulant collision with the
 * default higher-order rates, open domain, constant thickening factor (LBM_ERR_UNSUPPORTED
 * otherwise). state_n: device copy of state n in the lbm_save_state layout. adj: device buffer
 * in the same layout and types holding the adjoint of state n+1 (populations in the stored
 * shifted form); overwritten with the adjoint of state n. grad_inlet: device array [dim][ny] of
 * the field type to which the adjoint of the inlet-face velocity is added. The context's own
 * state is replaced by state_n (used to recompute the forward step). Upwind choices and the
 * max(Y, 0) of the rate law are held fixed (derivative 0 across their switches). Workspace owned
 * by the library, allocated at the first adjoint call: (9 + 18 (n_species + 1)) N values of the
 * field type plus one state (per-cell adjoints of the LB step's rho, Lambda, T and u, and two
 * arrays of stencil-point adjoints through which consecutive reverse steps pass the T and Y
 * adjoints). */
lbm_status lbm_adjoint_step(lbm_ctx* ctx, const void* state_n, void* adj, void* grad_inlet);

/* Reverse sweep over one checkpoint segment (same support as lbm_adjoint_step): from the state
 * `checkpoint` (device, lbm_save_state layout, state n0) the library recomputes n_steps steps,
 * keeping every state of the segment and its rho, Lambda in device workspace it owns
 * (n_steps x (state + 2 N) values of the field type), then applies the adjoint step from
 * n0 + n_steps - 1 down to n0. adj: device buffer in the lbm_save_state layout, holding the
 * adjoint of state n0 + n_steps on entry and that of state n0 on return (populations of solid
 * cells are set to zero); grad_inlet: as in lbm_adjoint_step (accumulated). Equivalent to
 * n_steps calls of lbm_adjoint_step with the saved states, without host round trips. The
 * context's current state is left as it was. */
lbm_status lbm_adjoint_segment(lbm_ctx* ctx, const void* checkpoint, int n_steps, void* adj, void* grad_inlet);

/* Reverse sweep over a whole checkpointed run (same support as lbm_adjoint_step): checkpoints is a
 * host array of n_segments device pointers, checkpoints[s] the state s * seg_len in the
 * lbm_save_state layout; the run has n_steps steps, (n_segments - 1) seg_len < n_steps <=
 * n_segments seg_len (the last segment may be shorter). adj: adjoint of state n_steps on entry,
 * of state 0 on return; grad_inlet accumulated. Equivalent to lbm_adjoint_segment over the
 * segments from the last to the first, with identical results: the same kernels in the same
 * order on the context's stream, while the recompute of the next segment runs on a second stream
 * of the library (the two overlap; at small grids each kernel fills a fraction of the GPU).
 * Workspace: 2 seg_len segment slots (lbm_adjoint_segment's, grown). */
lbm_status lbm_adjoint_sweep(lbm_ctx* ctx, const void* const* checkpoints, int n_segments, int seg_len, int n_steps,
                             void* adj, void* grad_inlet);

/* Objective J = sum over fluid cells of the fuel consumption rate -omega_F (kg/(m^3 s), lattice
 * cell volume 1) of the context's current state, written to *J (host), and its gradient with
 * respect to the state written to adj_out (device, lbm_save_state layout: T and Y parts filled,
 * populations and velocity zero). Same support as lbm_adjoint_step. Synchronises the stream. */
lbm_status lbm_fuel_objective(lbm_ctx* ctx, int fuel_species, double* J, void* adj_out);

/* Gradient with respect to the initial temperature field: reverse of lbm_set_fields, whose
 * populations are the equilibrium of Eq. 6 with rho = P_th W / (R T) (Eq. 13), so that T enters
 * both T itself and the populations. state0: device copy of the state lbm_set_fields produced
 * (lbm_save_state layout; it becomes the context's state); adj0: device adjoint of that state;
 * grad_T0: device array [N] of the field type, overwritten with dJ/dT0. Same support as
 * lbm_adjoint_step, thermal runs only. */
lbm_status lbm_initial_T_adjoint(lbm_ctx* ctx, const void* state0, const void* adj0, void* grad_T0);

/* 1: capture pairs of steps in CUDA graphs (default), 0: launch directly. */
lbm_status lbm_use_graphs(lbm_ctx* ctx, int enable);

/* Allocation-free thermodynamic-pressure integral. The paper has no counterpart of this call;
 * it serves callers that cannot allocate device memory (a host framework that owns every
 * allocation through its own pool, code where cudaMalloc is forbidden or would synchronise the
 * device, a monitor holding only pointers to fields made elsewhere).
 * Computes I = sum over cells with mask == 0 of W / (R T rho_ref), W = (sum_k Y_k / W_k)^-1,
 * with the kernel and exact fixed-point partial sums that lbm_step uses every step, and writes
 * it to I_out. T [n_cells] and Y [n_species][n_cells] are FP32, mask [n_cells] uint8, I_out one
 * double: all device pointers. W: n_species molar masses (kg/mol) in host memory. Work is
 * enqueued on `stream` (NULL = legacy default stream of the current device) and runs on the
 * stream's device, which the call makes current while it enqueues and then restores; the call
 * returns before the work completes. Per cell the term T_ref W / (max_k W_k T) is formed in FP32
 * and summed exactly in 64-bit fixed point (resolution 2^-32); if any cell's term is non-finite
 * or 2^30 and above (e.g. T = 0 in a fluid cell), I_out receives NaN (the status cannot report
 * it, since the call does not wait for the GPU).
 * It calls no allocator: per-block partial sums go to a static device array of 1 MiB that every
 * GPU loading this library holds until the process exits, which limits n_cells to 16777216
 * (larger sizes return LBM_ERR_ARG). The first call on a device resolves that array's device
 * address (cudaGetSymbolAddress) and should therefore come before any stream capture on that
 * device. All calls on a device share the array, so calls that overlap on the GPU (on
 * different streams) race; each call overwrites every slot it reads and clears its counter of
 * out-of-range cells before use. err (may be NULL) receives a one-line message. */
lbm_status lbm_pth_integral_noalloc(const float* T, const float* Y, const uint8_t* mask, int n_cells,
                                   int n_species, const double* W, double T_ref, double rho_ref,
                                   double* I_out, void* stream, char* err, size_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* HLBM_H */
