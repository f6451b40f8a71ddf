/*
 * lbm.h -- C ABI of the B300 (sm_103a) LBM-LES urban-wind step.
 *
 * One call advances a lattice by n time steps of the fused D3Q19 stream-and-collide update of
 * the paper's solver (App. D): SRT-BGK collision (Eq. D.2) with the Smagorinsky-Lilly closure
 * evaluated locally from the non-equilibrium momentum flux (Eqs. D.8-D.11), streaming (Eq. D.3),
 * mid-grid bounce-back at solid cells and no-slip faces (App. D, last paragraph), equilibrium
 * velocity boundary cells on inflow faces (Sec. 3, boundary-condition paragraph), zero-gradient
 * outflow, free-slip and periodic faces, all applied in the same pass over the lattice.
 *
 * Conventions shared by every entry point
 *   - Lattice: nx * ny * nz cells, cell index c = (z * ny + y) * nx + x (x fastest).  z is up;
 *     the ground wall lies half a spacing below z = 0.  Lattice units (dx = dt = 1).
 *   - Ownership: the caller owns every device buffer and the CUDA stream.  The library never
 *     allocates device memory: the whole domain state lives in a caller-provided workspace of
 *     lbm_workspace_bytes() bytes (e.g. a torch uint8 CUDA tensor).  Host memory for the opaque
 *     handle comes from malloc.
 *   - Streams: every call is enqueued on the stream given to lbm_create_domain (a cudaStream_t
 *     passed as void*, NULL = legacy default stream) and returns without waiting for the GPU,
 *     except lbm_diagnostics, which synchronises that stream.
 *   - Errors: every call returns an lbm_status; on failure the domain keeps a message readable
 *     with lbm_last_error().  Invalid arguments are detected on the host before any launch;
 *     launch failures return LBM_ECUDA.  No call aborts or traps.
 *   - Direction order of exported populations (lbm_direction_table): 0 = rest, 1..6 = +x -x +y
 *     -y +z -z, 7..18 = the twelve face diagonals, opposite directions in pairs (2k-1, 2k).
 */
#ifndef LBM_B300_H
#define LBM_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_domain lbm_domain; /* opaque */

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,    /* bad argument (sizes, NULL pointer, face combination, parameter range) */
    LBM_ENOMEM = -2,    /* workspace smaller than lbm_workspace_bytes(), or host malloc failed */
    LBM_ECUDA = -3,     /* a CUDA call or kernel launch failed (message holds cudaGetErrorString) */
    LBM_EUNSTABLE = -4, /* watchdog: non-finite populations found (see lbm_params.watchdog_every) */
    LBM_ESTATE = -5     /* call not valid in the domain's current state */
} lbm_status;

/* Face kinds, per face in the order x-, x+, y-, y+, z-, z+.
 *   PERIODIC    wrap to the opposite face (both faces of the axis must be periodic)
 *   INFLOW_EQ   the face layer consists of equilibrium cells f = f^eq(rho_b, u_b(z))
 *               (Sec. 3: equilibrium-based open velocity boundaries)
 *   OUTFLOW_ZG  zero gradient: a population entering from outside equals the same-direction
 *               population that left the adjacent in-domain cell (the paper's own outlet is an
 *               equilibrium face, Sec. 3; zero gradient is this library's open outlet)
 *   FREESLIP    specular reflection half a spacing outside the face
 *   NOSLIP      mid-grid bounce-back half a spacing outside the face (App. D)  */
typedef enum {
    LBM_FACE_PERIODIC = 0,
    LBM_FACE_INFLOW_EQ = 1,
    LBM_FACE_OUTFLOW_ZG = 2,
    LBM_FACE_FREESLIP = 3,
    LBM_FACE_NOSLIP = 4
} lbm_face;

/* Population storage.  Arithmetic is always FP32; populations are stored shifted by their
 * lattice weight, g_i = f_i - w_i, to keep the stored values small:
 *   LBM_F32    g as float
 *   LBM_F16S   g * 2^14 as IEEE binary16, round-to-nearest-even
 *   LBM_BF16S  g as bfloat16, round-to-nearest-even */
typedef enum { LBM_F32 = 0, LBM_F16S = 1, LBM_BF16S = 2 } lbm_store;

typedef struct {
    float tau;            /* molecular relaxation time, > 1/2; nu_0 = (tau - 1/2)/3 (Eq. D.5) */
    float cs_smag;        /* Smagorinsky constant C (Eq. D.7), >= 0; filter width Delta = 1 */
    float rho_b;          /* density of the equilibrium boundary cells, > 0 */
    int store;            /* lbm_store */
    int face[6];          /* lbm_face, order x- x+ y- y+ z- z+ */
    float force[3];       /* uniform body-force density, Guo forcing; {0,0,0} = none */
    int watchdog_every;   /* > 0: lbm_step scans for non-finite populations every that many
                             steps (synchronises the stream); 0 = off */
    float coriolis[3];    /* rotation vector Omega^lbm (lattice units, e.g. lbm_coriolis_omega);
                             each fluid cell adds the Coriolis force 2 rho Omega^lbm x u, u = sum c f
                             / rho, to the body force of Guo's forcing (App. E); {0,0,0} = none */
    /* Relaxation zones next to the outer faces (Sec. 3: a top sponge layer and buffer nudging toward
     * the target boundary state next to the lateral faces).  After its collision, a fluid cell at
     * distance d (cells) from a zone's face layer, d < width, relaxes toward the equilibrium of its
     * own density and the profile velocity u_b(z):  f* <- f* - s (f* - f^eq(rho, u_b(z))),
     * s = sigma ((width - d) / width)^2, the largest s where zones overlap.  Mass is kept; the
     * velocity deviation from u_b shrinks by the factor (1 - s) per step. */
    int sponge_top;       /* width of the zone under the top face layer (z = nz - 1); 0 = none */
    float sponge_sigma;   /* its rate at the face layer, 0 <= sigma <= 1 */
    int buffer_width;     /* width of the zones next to the open lateral faces (INFLOW_EQ or
                             OUTFLOW_ZG among x-, x+, y-, y+); 0 = none */
    float buffer_sigma;   /* their rate at the face layer, 0 <= sigma <= 1 */
    int flux_balance;     /* 1: mass-flux consistency (Sec. 2.1, Sec. 3): every equilibrium boundary cell's
                             velocity gets the same shift along the inward normal of the face owning
                             it (x-, x+, y-, y+, z-, z+: the first inflow face holding the cell), the
                             smallest uniform shift that makes the net volume inflow of all equilibrium
                             cells zero; recomputed by lbm_set_inflow_profile.  0 = off */
} lbm_params;

/* Fill p with defaults: tau 0.52, C 0.16, rho_b 1, F32, x- inflow, x+ outflow, periodic y,
 * no-slip ground, free-slip top, no force, no rotation, no watchdog, no relaxation zones, no flux
 * balancing.  Returns LBM_EINVAL if p is NULL. */
lbm_status lbm_params_default(lbm_params *p);

/* Earth rotation in the local east-north-up frame at latitude lat_deg, in lattice units (App. E):
 * Omega^lbm = Omega dt_si (0, cos lat, sin lat) with Omega = 7.292115e-5 rad/s.  out: 3 floats. */
lbm_status lbm_coriolis_omega(double lat_deg, double dt_si, float *out);

/* Net volume inflow of the equilibrium boundary cells (sum over them of u . n_in, n_in the inward
 * normal of the face owning the cell, one cell face of area 1 each) before and after the flux
 * balancing of the current profile, and the normal shift applied (0 when flux_balance is off).
 * HOST outputs, any may be NULL. */
lbm_status lbm_flux_balance_info(const lbm_domain *d, double *before, double *after, double *shift);

/* Lattice units of a physical setup by Mach scaling (Sec. 3 run parameters, App. D: velocities
 * scale with dt/dx, viscosities with dt/dx^2):
 *   dx_si     cell size [m], > 0
 *   u_ref_si  reference wind speed [m/s], > 0
 *   ma_lbm    lattice Mach number of the reference speed, u_lbm / c_s with c_s = 1/sqrt(3), > 0
 *   nu_si     kinematic viscosity [m^2/s], >= 0
 * out (HOST double[4]): out[0] = dt_si = ma_lbm c_s dx_si / u_ref_si [s]; out[1] = u_ref in
 * lattice units = ma_lbm c_s; out[2] = nu_lbm = nu_si dt_si / dx_si^2; out[3] = tau = 3 nu_lbm + 1/2
 * (Eq. D.5 with dt = dx = 1).  LBM_EINVAL on out-of-range arguments. */
lbm_status lbm_lattice_units(double dx_si, double u_ref_si, double ma_lbm, double nu_si, double *out);

/* Lateral face kinds for a wind direction theta (radians, 0 = +x, counter-clockwise): a lateral
 * face is INFLOW_EQ when the wind enters through it (u . n_in > 1e-6 |u|), OUTFLOW_ZG otherwise;
 * z- = NOSLIP, z+ = FREESLIP.  face must hold 6 ints. */
lbm_status lbm_faces_for_direction(float theta, int *face);

/* Bytes of device workspace a domain of this size and storage needs (0 if the arguments are
 * invalid).  Layout (all regions 256-byte aligned): populations 19 * N * sizeof(store) between
 * two guard regions, cell flags N bytes, cell info 4 N bytes, inflow profile nz * 3 floats, exit
 * buffers for outflow faces, precomputed boundary tables of the face cells (58 * 4 bytes per
 * face cell; omitted above 2^30 cells), reduction scratch. */
size_t lbm_workspace_bytes(int nx, int ny, int nz, const lbm_params *p);

/* Create a domain in the caller's workspace.
 *   solid      HOST array of nx*ny*nz bytes, x fastest, nonzero = solid (voxelised buildings,
 *              Sec. 2.1); copied during the call, may be freed afterwards
 *   nx,ny,nz   lattice size; >= 2 on every non-periodic axis, >= 1 on periodic ones,
 *              nx*ny*nz + 2 (nx*ny + nx + 1) + 1024 < 2^31 (32-bit cell offsets in the kernels)
 *   workspace  DEVICE pointer, 256-byte aligned, ws_bytes >= lbm_workspace_bytes()
 *   stream     cudaStream_t as void* (NULL = default stream); all later calls use it
 *   out        receives the handle
 * Cell kinds: solid where the mask is set; otherwise equilibrium cell on an INFLOW_EQ face
 * layer; otherwise fluid.  The populations start at rest (rho = 1, u = 0) and the inflow profile
 * at zero; call lbm_set_inflow_profile and lbm_init_fields before stepping. */
lbm_status lbm_create_domain(const uint8_t *solid, int nx, int ny, int nz, const lbm_params *p,
                             void *workspace, size_t ws_bytes, void *stream, lbm_domain **out);

/* Replace the stream used by later calls (the caller orders the hand-over). */
lbm_status lbm_set_stream(lbm_domain *d, void *stream);

/* Set the equilibrium-boundary velocity profile u_b(z) from L level speeds (HOST array) and a
 * direction theta (radians, 0 = +x, counter-clockwise): u_b = s(z) (cos theta, sin theta, 0).
 * L divides nz: level l covers the cells z in [l nz/L, (l+1) nz/L).  Otherwise s(z) is linear in
 * height between level centres (cell z sits at height z + 1/2, level l is centred at
 * (l + 1/2) nz / L) and constant beyond the outermost centres.  The host array may be reused as
 * soon as the call returns.  The upload is asynchronous through a small ring of pinned host
 * slots; the call waits only when the slot it reuses still has a copy in flight, four profile
 * updates back.  (The paper's per-cell boundary field comes from Kriging of lidar
 * profiles, Sec. 3 and App. A; this entry point takes the per-height profile directly.) */
lbm_status lbm_set_inflow_profile(lbm_domain *d, const float *speed, int L, float theta);

/* Initialise the populations to equilibrium, f = f^eq(rho, u) (Eq. D.4), and reset the step
 * counter to 0.
 *   rho  DEVICE float[N] or NULL (rho = 1)
 *   u    DEVICE float[N][3] (u, v, w interleaved per cell) or NULL (u = u_b(z))
 * Equilibrium cells take f^eq(rho_b, u_b(z)); solid cells are ignored. */
lbm_status lbm_init_fields(lbm_domain *d, const float *rho, const float *u);

/* Advance n >= 0 time steps (asynchronous).  Each step is one fused kernel over all cells:
 * gather (Eq. D.3 with the face rules above), moments (D.1), equilibrium (D.4), LES closure
 * (D.8-D.11), collision (D.2), store.  Streaming is in place on one lattice (odd/even step
 * pattern), so each step reads and writes every population of every non-solid cell once. */
lbm_status lbm_step(lbm_domain *d, int n);

/* Number of steps taken since the last lbm_init_fields. */
long long lbm_steps_done(const lbm_domain *d);

/* Sample (u, v, w, rho) of the current post-collision state at ncol columns and nh heights
 * (virtual lidar profiles, Sec. 4.4).
 *   ij   DEVICE int[ncol][2] = (x, y) of each column
 *   k    DEVICE int[nh] heights (cell z index)
 *   out  DEVICE float[ncol][nh][4]
 * Solid cells give (0,0,0,0); equilibrium cells give (u_b(z), rho_b).  An index outside the
 * lattice gives NaN in all four entries (indices are not checked on the host). */
lbm_status lbm_sample_columns(lbm_domain *d, const int *ij, int ncol, const int *k, int nh,
                              float *out);

/* Full macroscopic fields of the current post-collision state (same rules as above).
 *   rho  DEVICE float[N] (may be NULL);  u  DEVICE float[N][3] (may be NULL) */
lbm_status lbm_macroscopic(lbm_domain *d, float *rho, float *u);

/* Export the current post-collision populations, shifted, as FP32: g[i * N + c] = f*_i(c) - w_i
 * in the direction order of lbm_direction_table; solid cells export 0.  DEVICE float[19 * N]. */
lbm_status lbm_export_populations(lbm_domain *d, float *g);

/* Resume from a saved state (checkpoint / restart): g is a DEVICE float[19 * N] in the format of
 * lbm_export_populations (post-collision populations, shifted, library direction order; solid
 * cells ignored), written into the domain's in-place layout in its storage kind (rounded to 16 bits
 * for FP16S / BF16S) together with the outflow side buffers; the step counter becomes `step`, which
 * must be even (a state exported after an odd step can be resumed one step later, or as an even
 * count).  Asynchronous; g may be reused once the stream has passed the call.  Exporting after an
 * even number of steps, importing into a domain with the same mask, faces and parameters, and
 * stepping on reproduces the uninterrupted run bit for bit. */
lbm_status lbm_import_populations(lbm_domain *d, const float *g, long long step);

/* The library's direction order: c[3*i + a] (int) and w[i] (float), i = 0..18.  Returns 19. */
int lbm_direction_table(int *c, float *w);

/* FP64 reductions over the current state, computed on the GPU and copied to HOST out[4]:
 *   out[0] = total mass sum rho over fluid cells
 *   out[1] = net mass flux rho u . n_out summed over the cells of every open (inflow or
 *            outflow) face layer
 *   out[2] = max |u| over fluid cells
 *   out[3] = number of fluid cells with a non-finite population
 * Each GPU thread sums the density deviations rho - 1 of its cells in FP32 (they are ~1e-3, so
 * its partial keeps ~1e-10 of the mass) and max |u| in FP32; every sum across threads and blocks,
 * and the flux, is FP64.  Synchronises the domain's stream. */
lbm_status lbm_diagnostics(lbm_domain *d, double *out);

/* The same reductions as lbm_diagnostics, for callers that must not allocate device memory and
 * cannot wait on the host (a stream-ordered serving or assimilation loop under a fixed memory
 * budget, or a workspace sized without reduction scratch).  No counterpart in the paper.
 *   out  DEVICE double[4], written asynchronously on the domain's stream (same meaning as
 *        lbm_diagnostics' out); nothing is copied to the host and the stream is not synchronised
 * Allocates nothing: the partial sums live in a fixed 512 KiB array inside the library (kept by
 * every GPU that loads it until the process exits), which limits the lattice to 2^28 cells;
 * larger lattices return LBM_EINVAL.  All calls share that array: calls whose kernels overlap on
 * the GPU (different streams or host threads) race, so keep them in one stream order.  The first
 * call on a device looks up the array's device address; make it before any stream capture.  The
 * current CUDA device must be the one that was current at lbm_create_domain (else LBM_EINVAL):
 * the array's address differs per device.  The threads take their cells in a different order
 * than in lbm_diagnostics, so the masses agree to the rounding of the per-thread FP32 partials
 * (~1e-10 relative), the flux to FP64 rounding, max |u| and the count exactly. */
lbm_status lbm_diagnostics_noalloc(lbm_domain *d, double *out);

/* ---------------------------------------------------------------------------------------------
 * Synthetic von Karman inflow turbulence (App. F).
 *
 * Once configured, every lbm_step sets the velocity of the equilibrium cells of the inflow faces
 * x-, x+, y-, y+ and z+ (never the ground) to
 *     U_i(t) = U_b,i + sigma_i q^(f)(x_i, t),   q_a = sum_m A_m,a cos(k_m . x_i + omega_m t + phi_m,a)
 * for the step t about to be taken (t = lbm_steps_done); that step's equilibrium cells then hold
 * f^eq(rho_b, U_i(t)).  One extra kernel evaluates the sum at each anchor t_a (every step with
 * stride 1, every s steps otherwise); between anchors the step kernel itself blends the two
 * anchor fields (interpolation) or keeps the last one (hold).  x_i are the integer cell indices.
 * Each cell
 * belongs to the first inflow face holding it in the order x-, x+, y-, y+, z+.  Per face f:
 * cells = its equilibrium cells, restricted to U_b . n_f > 0 (n_f inward) if inflow_only; the face
 * is dropped (its cells keep U_b) when it has none or U_c,f = |mean U_b| (|mean U_b . n_f| with
 * char_normal) is <= 1e-7.  Over the kept cells: u_ref = mean |U_b|, e_c = sum U_b / |sum U_b|
 * ((1,0,0) if the sum is 0), omega_m = u_ref k_m . e_c.  Wavenumbers k_m = exp(ln k_min + xi_m
 * (ln k_max - ln k_min)), xi_m = (m - 1 + r_m)/N_m, k_min = 2 pi/(10 L), k_max = pi (k_min -> 0.1
 * k_max if k_min >= k_max); directions (sqrt(1-mu^2) cos theta, sqrt(1-mu^2) sin theta, mu); von
 * Karman weights W = k^4 / (1 + (k L)^2)^(17/6), A_m = sqrt(W_m) / sqrt(1/2 sum W), A_m,a = g_a A_m;
 * sigma_i = I u_char (I > 0; u_char = |U_b,i| or |U_b,i . n_f|) else sigma0.  With a stride s the
 * field is evaluated at anchors t_a = floor(t/s) s and held, or interpolated linearly to t_a + s.
 * The step's velocity readouts (lbm_macroscopic, lbm_sample_columns, lbm_diagnostics) report U_i of
 * the last step taken; right after lbm_init_fields (which uses U_b) they report U_b.
 * --------------------------------------------------------------------------------------------- */
typedef struct {
    int n_modes;        /* N_m, 1 .. 1024 (same for every face) */
    float length;       /* integral length scale L, lattice units, > 0 */
    float intensity;    /* I > 0: sigma_i = I u_char; I <= 0: sigma_i = sigma0 */
    float sigma0;       /* constant fluctuation level (lattice velocity), >= 0 */
    float gain[3];      /* component gains g_x, g_y, g_z */
    int char_normal;    /* 0: U_c,f and u_char from |U_b|; 1: from the face-normal component */
    int inflow_only;    /* 1: only cells with U_b . n_f > 0 are turbulent */
    int stride;         /* temporal stride s >= 1 */
    int interpolate;    /* 1: interpolate between anchors, 0: hold the anchor's field */
} lbm_stg_params;

/* Defaults: 64 modes, L = 20, I = 0.1, sigma0 = 0, gains 1, |U_b| speeds, every cell, stride 1,
 * interpolation on.  LBM_EINVAL if p is NULL. */
lbm_status lbm_stg_params_default(lbm_stg_params *p);

/* Device bytes lbm_stg_configure needs for n_modes modes on this domain's inflow faces (tables
 * and per-face velocity planes); 0 if d is NULL, n_modes is out of range or the domain has no
 * inflow face among x-, x+, y-, y+, z+. */
size_t lbm_stg_workspace_bytes(const lbm_domain *d, int n_modes);

/* Switch the synthetic inflow on (or reconfigure it) for later steps.
 *   p          parameters (host), checked: LBM_EINVAL with a message when out of range
 *   uniforms   HOST double[6][n_modes][6], values in [0, 1): for face f (x-, x+, y-, y+, z-, z+;
 *              the z- entries are unused) and mode m: r_m, (mu_m + 1)/2, theta_m / 2 pi, and
 *              phi_m,x, phi_m,y, phi_m,z / 2 pi.  The paper draws them from a base seed mixed
 *              with the face id; here the caller draws them (the same numbers on every face give
 *              one shared realisation).  Copied during the call.
 *   workspace  DEVICE memory, 256-byte aligned, ws_bytes >= lbm_stg_workspace_bytes; owned by
 *              the caller, used until lbm_stg_disable / lbm_destroy or the next configure
 * The tables depend on the inflow profile: lbm_set_inflow_profile rebuilds them.  Builds the
 * tables on the host (O(N_m x face cells)) and uploads them on the domain's stream. */
lbm_status lbm_stg_configure(lbm_domain *d, const lbm_stg_params *p, const double *uniforms,
                             void *workspace, size_t ws_bytes);

/* Switch the synthetic inflow off: the equilibrium cells take U_b again from the next step on. */
lbm_status lbm_stg_disable(lbm_domain *d);

/* The configuration's global convection quantities: u_ref, e_c[3] (HOST) and a bit mask of the
 * turbulent faces (bit k = face k).  Any output may be NULL.  LBM_EINVAL when not configured. */
lbm_status lbm_stg_reference(const lbm_domain *d, double *u_ref, double *e_c, int *faces);

/* ---------------------------------------------------------------------------------------------
 * Boundary assimilation: virtual-lidar misfit and its discrete-adjoint gradient with respect to
 * the inflow parameters.  (The paper fits the inflow to Doppler-lidar profiles by Kriging, Sec. 3
 * and App. A; these calls give the gradient of the same fit, so the inflow can be recovered by
 * gradient descent.)
 *
 * Forward model (FP32 storage, no body force, no rotation, no relaxation zones, no flux balancing,
 * synthetic inflow off):
 *   1. lbm_set_inflow_profile(speed, L, theta) and lbm_init_fields(NULL, NULL): every non-solid
 *      cell starts at f^eq of the profile velocity u_b(z) (rho = 1, equilibrium cells rho_b);
 *   2. n_steps fused steps (lbm_step); the domain is left at step n_steps;
 *   3. the lidar samples (u, v, w, rho) at cells (ij[c], k[h]) after each of the last n_avg
 *      states (the states n_steps - n_avg + 1 .. n_steps; state 0 is the initial state) and
 *      averages them in FP64: mean[c][h][4];
 *   4. J = sum over c, h of (mean_u - target_u)^2 + (mean_v - target_v)^2.
 * Gradient (lbm_lidar_misfit_grad): the exact derivative of the discrete forward model (up to
 * FP32 rounding) with respect to speed[0..L-1] and theta, by the discrete adjoint of every step
 * (streaming with every face rule, the LES collision D.1-D.11, equilibrium boundary cells, the
 * initial state), run backwards in segments of checkpoint_every steps that are recomputed from
 * checkpoints, with FP64 accumulation of the parameter gradient.  At a cell with Q = 0 the
 * derivative of the Smagorinsky term is taken as 0.
 * --------------------------------------------------------------------------------------------- */
typedef struct {
    int n_steps;            /* T >= 1 */
    int n_avg;              /* 1 <= n_avg <= T + 1: the last n_avg states are averaged */
    int checkpoint_every;   /* K >= 1: gradient only; a checkpoint every K states, segments of
                               K steps recomputed in the reverse sweep */
} lbm_adjoint_params;

/* Device workspace bytes for ncol x nh samples; gradient != 0: for lbm_lidar_misfit_grad, which
 * holds ceil(T/K) checkpoints, min(K, T) segment states and two adjoint lattices of 19 N floats
 * each (plus O(N) bytes); gradient == 0: for lbm_lidar_misfit (O(N) bytes).  0 on bad arguments. */
size_t lbm_adjoint_workspace_bytes(const lbm_domain *d, const lbm_adjoint_params *p, int ncol, int nh,
                                   int gradient);

/* Run the forward model and evaluate the misfit.
 *   speed, L, theta  inflow parameters (HOST), as lbm_set_inflow_profile
 *   ij, k            HOST int[ncol][2] column positions (x, y) and int[nh] cell heights; every
 *                    sampled cell must be a fluid cell (LBM_EINVAL otherwise, checked on the GPU)
 *   target           DEVICE float[ncol][nh][2] target mean (u, v), or NULL (no misfit)
 *   workspace        DEVICE, 256-byte aligned, ws_bytes >= lbm_adjoint_workspace_bytes(.., 0)
 *   out              DEVICE double[1]: J (not written when target is NULL); may be NULL
 *   mean             DEVICE double[ncol][nh][4] mean (u, v, w, rho), or NULL
 * Synchronises the stream once (sample check) before the steps; the rest is asynchronous. */
lbm_status lbm_lidar_misfit(lbm_domain *d, const lbm_adjoint_params *p, const float *speed, int L,
                            float theta, const int *ij, int ncol, const int *k, int nh,
                            const float *target, void *workspace, size_t ws_bytes, double *out,
                            double *mean);

/* The same forward run, then the reverse sweep.
 *   workspace  ws_bytes >= lbm_adjoint_workspace_bytes(.., 1)
 *   out        DEVICE double[L + 2]: out[0] = J, out[1 + l] = dJ/dspeed[l], out[1 + L] = dJ/dtheta
 * Asynchronous after the sample check; the domain is left at step n_steps of the forward run. */
lbm_status lbm_lidar_misfit_grad(lbm_domain *d, const lbm_adjoint_params *p, const float *speed,
                                 int L, float theta, const int *ij, int ncol, const int *k, int nh,
                                 const float *target, void *workspace, size_t ws_bytes, double *out,
                                 double *mean);

/* ---------------------------------------------------------------------------------------------
 * Batched ensembles: several domains (inflow directions and speeds, lattices of uneven size)
 * advanced together, one kernel launch per time step for all of them.  (The paper runs one case
 * at a time, Sec. 3; an ensemble of inflow conditions is what the assimilation and the wind-rose
 * studies iterate over.)
 *
 * Members keep their own workspaces, profiles and state; every member must use the same storage
 * kind, have no body force, no rotation, no relaxation zones and no synthetic inflow, and have taken
 * steps of the same
 * parity (they then advance in lockstep: lbm_steps_done grows by the same amount on each).  A
 * batched step computes exactly what lbm_step computes on each member.
 * --------------------------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch; /* opaque */

/* Device workspace bytes for a batch of n members (step arguments and block tables, about 1 KB per
 * member); 0 if n is outside [1, 4096]. */
size_t lbm_batch_workspace_bytes(int n);

/* Group n domains.  workspace: DEVICE, 256-byte aligned, ws_bytes >= lbm_batch_workspace_bytes(n),
 * owned by the caller.  stream: cudaStream_t as void* (NULL = default stream; capture needs a
 * non-default one).  LBM_EINVAL for mixed storage kinds, forced or turbulent-inflow members or a
 * member given twice; LBM_ESTATE if the members' step counts differ in parity.  Synchronises the
 * stream once (table upload). */
lbm_status lbm_batch_create(lbm_domain *const *domains, int n, void *workspace, size_t ws_bytes,
                            void *stream, lbm_batch **out);

/* Advance every member by nsteps >= 0 steps (asynchronous on the batch stream). */
lbm_status lbm_batch_step(lbm_batch *b, int nsteps);

/* Record nsteps (even, >= 2) batched steps into a CUDA graph kept by the batch (replaces the
 * previous one).  Nothing runs; the members do not advance. */
lbm_status lbm_batch_capture(lbm_batch *b, int nsteps);

/* Replay the captured graph: every member advances by the captured number of steps.  LBM_ESTATE
 * when nothing is captured or the members are not at the parity of the capture. */
lbm_status lbm_batch_launch(lbm_batch *b);

/* Launch shapes (lbm_batch_shape_count() of them).  Batched kernels with 256-thread blocks
 * compiled for 4 resident blocks per SM, members in the given order, FP32 members with their own
 * cells per thread (as lbm_step), unless stated: 0 = that; 1 = 3 blocks per SM; 2 = largest
 * member first; 3 = 3 blocks per SM, largest first; 4 = one single-domain launch per member and
 * step (no batching); 5 = 128-thread blocks (8 per SM); 6 = 512-thread blocks (2 per SM); 7 =
 * FP32 members one cell per thread; 8 = FP32 members two cells per thread; 9 = persistent grid
 * (as many blocks as fit on the GPU at once, each striding over all members' blocks).  Shapes 5..9
 * need at most 48 members; 7 and 8 apply to FP32 storage only.  The autotuner runs 2 +
 * trial_steps steps of every available shape on the members (they advance by that many steps per
 * shape), times each with CUDA events and keeps the fastest.  trial_steps even, >= 2.  choice (may
 * be NULL) receives the chosen shape, ms_per_step (may be NULL; lbm_batch_shape_count() floats)
 * the ms per step of every shape, -1 for shapes not available to this batch.  Synchronises the
 * stream; drops a captured graph. */
lbm_status lbm_batch_autotune(lbm_batch *b, int trial_steps, int *choice, float *ms_per_step);
int lbm_batch_shape_count(void);

/* Set / read the launch shape (drops a captured graph; LBM_EINVAL for a shape not available). */
lbm_status lbm_batch_set_shape(lbm_batch *b, int shape);
int lbm_batch_shape(const lbm_batch *b);

/* Message of the last failed call on this batch.  Never NULL. */
const char *lbm_batch_last_error(const lbm_batch *b);

/* Release the batch (host memory and its graph); the members and the workspace are untouched. */
void lbm_batch_destroy(lbm_batch *b);

/* Message of the last failed call on this domain ("" if none).  Never NULL. */
const char *lbm_last_error(const lbm_domain *d);

/* Release the handle (host memory only; the caller frees the workspace).  NULL-safe.  The
 * caller must make sure no work of this domain is still running if it reuses the workspace. */
void lbm_destroy(lbm_domain *d);

#ifdef __cplusplus
}
#endif

#endif /* LBM_B300_H */
