/*
 * ann.h -- C-ABI of the GB300 (sm_103a) SPH active-nematic solver.
 *
 * The library advances the weakly compressible SPH discretisation of the Beris-Edwards active
 * nematic equations of Saghatchi, Kolukisa and Yildiz (arXiv 2108.08919) on one GPU: a 2D periodic
 * box of side L holding n particles with position r (FP64), velocity u, order parameter
 * Q = [[q11, q12], [q12, -q11]], density rho and the previous acceleration a (FP32 on the device).
 *
 * One step (ann_step) is the paper's modified-Euler predictor-corrector (§3.1, Eq. 27) with one
 * neighbour search at the projected configuration, evaluated as:
 *   predictor and cell keys    u' = u + dt/2 a, r' = r + dt/2 u' (re-inserted into [0, L), Eq. 30)
 *   cell sort                  particles binned into square cells of side >= 3h (§4); periodic
 *                              images of cells replace the paper's ghost particles (Eq. 30)
 *   pass A                     neighbour lists (|d|^2 < (3h)^2), sum_j W_ij and V = 1/sum (Eqs. 18-19)
 *   pass B                     correction tensor and B = alpha^-1 (Eq. 22), corrected velocity
 *                              gradient (Eq. 20), continuity (Eq. 25), Q Laplacian (Eq. 21), molecular
 *                              field (Eq. 7), Q rate (Eqs. 2, 24) and Q^{n+1}
 *   pass C                     density filter (Eq. 28), equation of state (Eq. 26) with
 *                              c0 = max(10 max|u'|, c0_min), divergence of Q^{n+1}
 *   pass D                     momentum (Eq. 23, active term -zeta/rho div Q), corrector, artificial
 *                              particle displacement (Eq. 29), re-insertion
 *
 * Conventions for every call:
 *   - Return value: ANN_OK (0) or a negative ANN_ERR_* code.  No exception crosses the ABI.  The
 *     text of the last error of a context is available from ann_last_error.
 *   - Pointers are plain host or device pointers, as each call states.  Host buffers are owned by
 *     the caller and only read or written during the call.  A context owns all device memory it
 *     allocates (cudaMalloc on the device current at ann_create) and frees it in ann_destroy.
 *   - Per-particle arrays exchanged through the ABI are indexed by particle ID 0..n-1, the order
 *     in which ann_set_particles received them; the device keeps particles in cell order
 *     internally and un-permutes on output.
 *   - Work is issued on the context's stream (ann_set_stream; default: a stream the context
 *     creates).  Calls that return data or a status synchronise that stream before returning.
 */
#ifndef ANN_H
#define ANN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ANN_ABI_VERSION 1

/* Status codes. */
#define ANN_OK 0
#define ANN_ERR_INVALID_ARG (-1)     /* a parameter or argument is out of its stated range */
#define ANN_ERR_OOM (-2)             /* device or host allocation failed */
#define ANN_ERR_CUDA (-3)            /* a CUDA runtime call failed (text in ann_last_error) */
#define ANN_ERR_CELL_OVERFLOW (-4)   /* a cell or a tile halo held more particles than the kernels stage */
#define ANN_ERR_NBR_OVERFLOW (-5)    /* a particle had more than ANN_MAX_NEIGHBORS neighbours */
#define ANN_ERR_NONFINITE (-6)       /* a position, velocity, Q or density became NaN or infinite */
#define ANN_ERR_SINGULAR_ALPHA (-7)  /* det(alpha) <= 0 for some particle (Eq. 22 not invertible) */
#define ANN_ERR_IO (-8)              /* checkpoint file could not be written or read */
#define ANN_ERR_STATE (-9)           /* call out of order (e.g. ann_step before ann_set_particles) */
#define ANN_ERR_NOT_AVAILABLE (-10)  /* no CUDA device */
#define ANN_ERR_TOO_LARGE (-11)      /* size beyond the fixed scratch of ann_velocity_moments_noalloc */
#define ANN_ERR_TIMEOUT (-12)        /* a bounded device wait (a tensor-core completion) expired; the kernel
                                        returned without its result and the context stays usable */
#define ANN_ERR_CFL_VIOLATION (-13)  /* dt_mode ANN_DT_CHECK: the step's dt exceeded a stability limit */

/* Limits of the device kernels. */
#define ANN_MAX_NEIGHBORS 128        /* neighbours (and candidates within 3h (1 + skin)) per particle */
#define ANN_MAX_PER_CELL 64          /* particles per cell */

/* momentum_mode */
#define ANN_MOMENTUM_PAPER 0         /* Eq. 23 as printed: B-corrected sums, particle volumes V */
#define ANN_MOMENTUM_CONSERVATIVE 1  /* pair-antisymmetric forms, fixed masses rho0 L^2 / n, no B */

/* dt_mode */
#define ANN_DT_FIXED 0               /* dt as given */
#define ANN_DT_STABLE 1              /* dt = min(dt, 0.125 h^2/nu, 0.125 h^2/(Gamma K), 0.25 h/c0_min), fixed at create */
#define ANN_DT_CHECK 2               /* dt as given; a step whose dt exceeds min(0.125 h^2/nu,
                                        0.125 h^2/(Gamma K), 0.25 h/(c0 + max|u|)), with c0 and max|u| of
                                        that step's midpoint, fails with ANN_ERR_CFL_VIOLATION */

/*
 * Parameters (plain data).  Names follow the paper: rho0 reference density, eta dynamic viscosity
 * (nu = eta/rho0), Gamma rotational diffusivity, lambda tumbling parameter, A, B, C Landau-de Gennes
 * coefficients, K elastic constant, zeta activity (> 0 extensile), gamma_eos EoS exponent (7),
 * beta density-filter coefficient (1 = Shepard), h smoothing length (support 3h).
 * c0_min: floor of the sound speed c0 = max(10 max|u'|, c0_min).
 * c_shift: c in Q + c I of the co-rotation term (Eq. 2 prints 1/3).
 * q_new_in_momentum: 1 uses Q^{n+1} in the active force (text order of §3.1), 0 uses Q^n.
 * apd: 1 applies the artificial particle displacement of Eq. 29.
 * elastic_stress: 1 adds the elastic stress of Eq. 12 (without its -p I),
 *   Pi_el = 2 lambda M (Q:H) - lambda (H M + M H), M = Q + c_shift I, to the momentum through the
 *   corrected divergence (paper mode) or the pair-antisymmetric form (conservative mode).  The
 *   paper neglects it (text under Eq. 13); default 0.
 * Valid ranges (ann_validate_params): 1 <= n <= 2^29, L > 0, 0 < h, 3h <= L/3 (at least three cells across
 * the box), dt > 0, rho0 > 0, eta >= 0, Gamma >= 0, gamma_eos > 0, 0 <= beta <= 1, c0_min >= 0, and
 * at most ANN_MAX_NEIGHBORS expected neighbours (pi (3h)^2 n / L^2 <= 0.85 ANN_MAX_NEIGHBORS).
 */
typedef struct ann_params {
    int64_t n;
    double L, h, dt;
    double rho0, eta, Gamma, lambda, A, B, C, K, zeta;
    double gamma_eos, beta, c0_min, c_shift;
    int32_t apd;
    int32_t momentum_mode;
    int32_t q_new_in_momentum;
    int32_t dt_mode;
    int32_t elastic_stress;
    int32_t reserved[3];
} ann_params;

/* Cell grid and step size a parameter set implies (host computation, no GPU needed). */
typedef struct ann_grid {
    int32_t cells_per_side;      /* n_c = floor(L / (3h (1 + 0.02) (1 + 1e-9))): cells hold the candidate radius */
    int32_t tiles_per_side;      /* ceil(n_c / 4): one CUDA block per 4 x 4 cells */
    double cell_size;            /* L / n_c >= 3h */
    double dt_effective;         /* dt after dt_mode */
    double expected_neighbors;   /* pi (3h)^2 n / L^2 */
    int64_t device_bytes;        /* device memory ann_create will allocate */
} ann_grid;

/* Diagnostics, FP64 reductions over all particles. */
typedef struct ann_diag {
    double t;                    /* simulated time */
    int64_t step;                /* completed steps */
    double momentum[2];          /* sum_i m_i u_i; m_i = rho_i V_i (paper mode) or rho0 L^2/n */
    double kinetic_energy;       /* 1/2 <|u|^2> over the particles (by Parseval, the sum of the
                                    spectrum E(w) of Eq. 31 over all shells, up to gridding) */
    double max_speed;            /* max |u| */
    double c0;                   /* sound speed of the last step */
    double mass;                 /* sum_i m_i */
    double mean_q;               /* mean nematic order q = sqrt(q11^2 + q12^2) */
    double nbr_mean;             /* mean neighbour count of the last evaluation */
    int32_t nbr_min, nbr_max;
    double min_det_alpha;        /* smallest det(alpha) of the last evaluation */
    uint32_t error_bits;         /* sticky device error bits (see ann_status_string) */
    int32_t resorts;             /* steps that re-sorted the particles and rebuilt the candidate lists */
    uint64_t band_checks;        /* pair tests that fell in the FP32 uncertainty band and were decided in FP64 */
} ann_diag;

/* Field identifiers for ann_get_field.  Element type: FP64 for ANN_FIELD_X/Y, int32 for
 * ANN_FIELD_NNBR, FP32 otherwise.  Fields after ANN_FIELD_AY are values of the last evaluated
 * step (at the midpoint configuration); the GRADU/LAPQ/APD/QRATE ones need ann_set_record(ctx, 1). */
enum ann_field {
    ANN_FIELD_X = 0, ANN_FIELD_Y, ANN_FIELD_UX, ANN_FIELD_UY, ANN_FIELD_Q11, ANN_FIELD_Q12,
    ANN_FIELD_DRHO,        /* rho/rho0 - 1 */
    ANN_FIELD_AX, ANN_FIELD_AY,
    ANN_FIELD_SUMW, ANN_FIELD_V, ANN_FIELD_B11, ANN_FIELD_B12, ANN_FIELD_B22,
    ANN_FIELD_K,           /* continuity rate k/rho0 (Eq. 25) */
    ANN_FIELD_DRHO_HALF,   /* rho^{n+1/2}/rho0 - 1 */
    ANN_FIELD_DRHO_HAT,    /* filtered density / rho0 - 1 (Eq. 28) */
    ANN_FIELD_P,           /* pressure (Eq. 26) */
    ANN_FIELD_DIVQX, ANN_FIELD_DIVQY,
    ANN_FIELD_NNBR,
    ANN_FIELD_GRADU_XX, ANN_FIELD_GRADU_XY, ANN_FIELD_GRADU_YX, ANN_FIELD_GRADU_YY, /* du_a/dx_b */
    ANN_FIELD_LAPQ11, ANN_FIELD_LAPQ12,
    ANN_FIELD_APDX, ANN_FIELD_APDY,
    ANN_FIELD_QRATE11, ANN_FIELD_QRATE12,   /* the projected Q rate m of Eq. (24), dQ/dt of the step */
    ANN_FIELD_COUNT
};

typedef struct ann_ctx ann_ctx;

/* ABI version (ANN_ABI_VERSION). */
int ann_version(void);

/* Human-readable text of a status code. Static storage; never NULL. */
const char *ann_status_string(int status);

/* Fill *p with the paper's 2D set-up used as default: L = 1, h = 1.3 dx for n = 64 x 64,
 * dt = 1e-4, rho0 = 1, eta = 1, Gamma = 0.34, lambda = 0.7, A = B = 0, C = 1, K = 0.04, zeta = 0.05,
 * gamma_eos = 7, beta = 1, c0_min = 0, c_shift = 1/3, apd = 1, paper momentum, Q^{n+1} in the
 * momentum, fixed dt.  Host only. */
int ann_default_params(ann_params *p);

/* Check every field of *p against the ranges stated above.  Host only, no GPU needed.
 * Returns ANN_OK or ANN_ERR_INVALID_ARG. */
int ann_validate_params(const ann_params *p);

/* Cell grid, tile count, effective dt and device memory of *p.  Host only. */
int ann_grid_info(const ann_params *p, ann_grid *out);

/* Create a context on the current CUDA device: validates *p, allocates all device buffers and
 * captures one step as a CUDA graph.  *out receives the context (NULL on failure).
 * Errors: INVALID_ARG, OOM, CUDA, NOT_AVAILABLE. */
int ann_create(const ann_params *p, ann_ctx **out);

/* Device memory provider for a context, in place of cudaMalloc / cudaFree (for example a host
 * framework's caching allocator); the paper has no counterpart.  alloc returns a device pointer to at least `bytes` bytes on the
 * current device, 16-byte aligned, or NULL on failure; release frees a pointer alloc returned,
 * with the same byte count.  `stream` is the context's own stream (a cudaStream_t): memory is used
 * on it, and a context synchronises it before it releases anything.  Both are called on the
 * calling thread, from ann_create_with_allocator, ann_destroy and the calls that grow the flow
 * diagnostics' scratch; `user` is passed through. */
typedef struct ann_allocator {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*release)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} ann_allocator;

/* ann_create with every device buffer of the context (state, lists, scratch) taken from *a
 * (NULL: cudaMalloc, the same as ann_create).  Errors: as ann_create; INVALID_ARG if a callback is
 * NULL or alloc returns a pointer that is not 16-byte aligned; OOM if alloc returns NULL. */
int ann_create_with_allocator(const ann_params *p, const ann_allocator *a, ann_ctx **out);

/* Free all device memory of ctx.  NULL is ignored. */
void ann_destroy(ann_ctx *ctx);

/* Issue subsequent work on `stream` (a cudaStream_t of the context's device; NULL selects the
 * legacy default stream).  The context's own stream is used until this is called. */
int ann_set_stream(ann_ctx *ctx, void *stream);

/* Load the state.  n must equal the n of ann_create.  Arrays are FP64 of length n in particle-ID
 * order: x, y positions (re-inserted into [0, L)), ux, uy velocity, q11, q12 order parameter, rho
 * density (NULL: rho0).  a^0 is set to zero, the step counter and t to zero.  is_device = 0: host
 * pointers; 1: device pointers on the context's device.  Errors: INVALID_ARG (n mismatch, NULL
 * required pointer), NONFINITE (a NaN or infinite entry), CUDA. */
int ann_set_particles(ann_ctx *ctx, int64_t n, const double *x, const double *y, const double *ux,
                      const double *uy, const double *q11, const double *q12, const double *rho,
                      int is_device);

/* Load the state of §3.1 (initial conditions, as ann_set_particles) in the precision the context
 * keeps it, as ann_get_state returns it: x, y FP64;
 * ux, uy, q11, q12 FP32; drho = rho/rho0 - 1 FP32 (NULL: 0); n each, particle-ID order.
 * Otherwise as ann_set_particles (positions re-inserted, a^0 = 0, t and the step count 0, the next
 * step re-sorts): the same state as ann_set_particles of the same values.  Errors: INVALID_ARG,
 * NONFINITE (also drho <= -1), CUDA. */
int ann_set_state(ann_ctx *ctx, int64_t n, const double *x, const double *y, const float *ux, const float *uy,
                  const float *q11, const float *q12, const float *drho, int is_device);

/* Advance nsteps >= 0 steps (one CUDA-graph launch per step) and synchronise.  Errors:
 * STATE (no particles), CELL_OVERFLOW, NBR_OVERFLOW, NONFINITE, SINGULAR_ALPHA, CFL_VIOLATION (device error
 * bits; once one is raised the remaining kernels of the call return without work), CUDA.
 * A failed step leaves the state at the last completed step: the context keeps two copies of the
 * state, a step reads the committed one and writes the other, and only a step that ends with no
 * error raised is committed.  After a failure ann_get_field, ann_get_state, ann_get_unwrapped and
 * ann_save_state see the state after the last completed step (ann_diag.step and .t count only the
 * completed steps; the periodic image counts the failed step changed are restored), and the next
 * step re-sorts.  The error bits stay set (ann_get_diagnostics reports them) until
 * ann_set_particles, ann_set_state or ann_load_state clears them. */
int ann_step(ann_ctx *ctx, int64_t nsteps);

/* Advance nsteps steps launching the kernels one by one with a CUDA event before and after each,
 * and add the total device time of each kernel (ms) to kernel_ms[ann_kernel_count()] (the caller
 * zeroes it).  A step runs either the re-sort branch (kernels 1..5: cell_keys, cell_scan,
 * cell_scatter, cell_order, pass_a_resort) or kernel 6 (pass_a, the candidate-list filter), as the
 * step graph would; a kernel adds time only in the steps where it ran, and the step count of each
 * branch follows from the change of ann_diag.resorts.  Same physics and errors as ann_step. */
int ann_step_profile(ann_ctx *ctx, int64_t nsteps, double *kernel_ms);

/* Number of kernels in one step, and the name of kernel k (static storage; NULL if out of range). */
int ann_kernel_count(void);
const char *ann_kernel_name(int k);

/* Record the GRADU, LAPQ and APD intermediates in later steps (on = 1) or not (0, default).
 * Recording adds stores to passes B and D and re-captures the step graph. */
int ann_set_record(ann_ctx *ctx, int on);

/* Copy field `field` (enum ann_field) in particle-ID order to dst, which holds `bytes` >= n times
 * the element size.  dst_is_device = 0: host pointer; 1: device pointer.  Errors: INVALID_ARG
 * (unknown field, short buffer), STATE (no particles), CUDA. */
int ann_get_field(ann_ctx *ctx, int field, void *dst, int64_t bytes, int dst_is_device);

/* The state the time integration of §3.1 carries from step to step (positions, velocity, Q,
 * density and the acceleration a^{n-1/2} the predictor uses): x, y FP64; ux, uy, q11, q12,
 * drho = rho/rho0 - 1 and ax, ay FP32; n each, particle-ID order, in one call with one
 * synchronisation: the same values as
 * ann_get_field of ANN_FIELD_X ... _DRHO, _AX, _AY.  A NULL destination is skipped.  dst_is_device
 * as for ann_get_field.  When every host destination is page-locked memory that the device maps
 * (cudaHostAlloc, cudaHostRegister), one kernel writes them over the host link in particle order;
 * other host memory goes through a device staging buffer and copies.  Errors: STATE, CUDA. */
int ann_get_state(ann_ctx *ctx, double *x, double *y, float *ux, float *uy, float *q11, float *q12,
                  float *drho, float *ax, float *ay, int dst_is_device);

/* Replace the present state of §3.1 of a loaded context by the arrays (particle-ID order, the layout of
 * ann_get_state; drho, ax, ay NULL: 0), keeping t, the step count, the periodic image counts and
 * the cell structure: each particle keeps its slot, and the next step re-sorts only if some
 * particle is half the candidate skin away from where the last re-sort put it, as after any step.
 * ann_get_state followed by ann_update_state of the same arrays leaves the trajectory
 * bit-identical.  Host arrays that are all page-locked and mapped are read by one kernel over the
 * host link (no staging copy), as in ann_get_state.  The call returns after the arrays have been
 * read.  Errors: INVALID_ARG, STATE (nothing loaded), NONFINITE (also drho <= -1), CUDA. */
int ann_update_state(ann_ctx *ctx, const double *x, const double *y, const float *ux, const float *uy,
                     const float *q11, const float *q12, const float *drho, const float *ax, const float *ay,
                     int is_device);

/* FP64 diagnostics of the current state.  Errors: STATE, CUDA. */
int ann_get_diagnostics(ann_ctx *ctx, ann_diag *out);

/* Neighbour lists of the current positions (no time advance): builds the cell sort and pass A at
 * the present configuration and writes them as CSR in particle IDs, each row ascending: rowptr has
 * n+1 entries (host), cols `cap` entries (host).  With cols == NULL only rowptr is written, so a
 * caller can size cols from rowptr[n].  The export takes a device buffer of 4 ANN_MAX_NEIGHBORS
 * bytes per particle (from the context's allocator, if it has one) for the duration of the call.
 * Errors: INVALID_ARG (cap < rowptr[n]), STATE, the step's device errors, CUDA, OOM. */
int ann_get_neighbors(ann_ctx *ctx, int64_t *rowptr, int32_t *cols, int64_t cap);

/* Write / read the full state (positions, velocities, Q, density, a, internal particle order, t,
 * step count, parameters) to / from a binary file.  A loaded state continues bit-identically to an
 * uninterrupted run.  ann_load_state requires a context created with the same n.  Errors: IO,
 * INVALID_ARG (format or n mismatch), STATE, CUDA. */
int ann_save_state(ann_ctx *ctx, const char *path);
int ann_load_state(ann_ctx *ctx, const char *path);

/* Text of the last error raised on ctx (empty string if none; never NULL). */
const char *ann_last_error(ann_ctx *ctx);

/*
 * Flow diagnostics of the results section (§5): the kinetic-energy spectrum (Eq. 31), the
 * vorticity correlation and its length scale (Eq. 32), topological defects, the nematic order
 * field, particle pathlines and mixing.  The paper names the quantities but not their
 * discretisation; the readings taken are stated with each call.  They analyse the present state
 * (after the last step) and never change it or the trajectory that follows.  Buffers they need are
 * allocated on first use and kept for later calls.
 *
 * Gridded fields.  The state lives on particles; the spectrum, the correlation and the defects are
 * computed on an M x M grid of nodes (ix L/M, iy L/M), M a power of two in [8, ANN_GRID_MAX], by
 * Shepard interpolation with the method's kernel (Eq. 18): f(x_g) = sum_j f_j W_gj / sum_j W_gj
 * over the particles with |x_g - x_j| < 3h (minimum image), FP32 sums, 0 where no particle is in
 * reach.  Requires at least 5 cells per side (ann_grid.cells_per_side >= 5).
 */
#define ANN_GRID_MAX 2048
#define ANN_MAX_COLORS 16
#define ANN_MIX_BINS_MAX 4096

/* The gridded present state: dst holds 5 M^2 doubles, fields ux, uy, q11, q12 and the weight
 * sum sum_j W_gj, each row-major [iy][ix].  dst_is_device: 0 host, 1 device pointer.  Errors:
 * INVALID_ARG (M, too few cells), STATE (no particles), CUDA, OOM. */
int ann_grid_fields(ann_ctx *ctx, int32_t M, double *dst, int dst_is_device);

/* Number of wavenumber shells of an M x M grid, round(M / sqrt 2) + 1 (host only; INVALID_ARG for
 * a bad M). */
int ann_spectrum_shells(int32_t M);

/* Kinetic-energy spectrum of the gridded velocity (Eq. 31): with u_hat = FFT(u) / M^2 (FP64),
 * E[n] = 1/2 sum |u_hat(k)|^2 over the integer wavevectors k whose |k| rounds to n, for
 * n = 0 .. ann_spectrum_shells(M) - 1; wavenumber w_n = 2 pi n / L.  sum_n E[n] = 1/2 <|u|^2> of
 * the grid (Parseval).  E: host array of at least nshell >= ann_spectrum_shells(M) doubles.
 * Errors: as ann_grid_fields. */
int ann_energy_spectrum(ann_ctx *ctx, int32_t M, double *E, int32_t nshell);

/* Least-squares slope of log E[n] against log w_n over the shells with w1 <= w_n <= w2, n >= 1 and
 * E[n] > 0 (the paper compares the spectrum with power laws w^-5/3, w^-4); NaN if fewer than two
 * shells qualify.  Host only.  Errors: INVALID_ARG. */
int ann_spectrum_slope(const double *E, int32_t nshell, double L, double w1, double w2, double *slope);

/* Vorticity correlation (Eq. 32) along the horizontal centre line, row iy = M/2 of the grid, with
 * the vorticity omega = d uy/dx - d ux/dy by periodic central differences of the gridded velocity.
 * C[k] for r = k L/M, k = 0 .. M/2 (host array of M/2 + 1 doubles): all_origins = 0 takes the
 * paper's single origin at the centre, C[k] = omega(M/2 + k) omega(M/2) / omega(M/2)^2;
 * all_origins = 1 averages over every origin of the line (the box is periodic and homogeneous),
 * C[k] = sum_i omega(i + k) omega(i) / sum_i omega(i)^2.  lengths (host, 2 doubles, may be NULL):
 * the first r where C reaches 0, and where it falls to 0.2 max C (both length scales the paper
 * names), linear between grid points, NaN if not reached.  Errors: as ann_grid_fields. */
int ann_vorticity_correlation(ann_ctx *ctx, int32_t M, int32_t all_origins, double *C, double *lengths);

/* Topological defects of the gridded Q: for each plaquette (ix, iy) -> (ix+1, iy) -> (ix+1, iy+1) ->
 * (ix, iy+1) the winding number m of the vector (Q11, Q12) (the doubled director angle), counted
 * exactly by signed crossings of the positive Q11 axis; the director defect there has charge m/2.
 * counts (host, 3): plaquettes with m = +1 (+1/2 defects), m = -1 (-1/2), |m| >= 2.  map (host,
 * M^2 int8, may be NULL): m of each plaquette, row-major by its lower-left node.  Defect density =
 * (counts[0] + counts[1]) / L^2.  Errors: as ann_grid_fields. */
int ann_defects(ann_ctx *ctx, int32_t M, int64_t *counts, int8_t *map);

/* Colour of each particle by ID (n values in [0, ANN_MAX_COLORS), host or device), the marker of
 * the paper's mixing experiment (particles coloured by their initial region).  Kept across
 * ann_set_particles and in checkpoints; all 0 after ann_create.  Errors: INVALID_ARG (n, a colour
 * out of range), CUDA. */
int ann_set_colors(ann_ctx *ctx, const uint8_t *colors, int64_t n, int is_device);

/* Mixing of the colours on a G x G grid of bins (1 <= G <= ANN_MIX_BINS_MAX; bin floor(x G / L),
 * clamped): Danckwerts' intensity of segregation per colour s with overall fraction 0 < a_s < 1,
 * I_s = mean over non-empty bins of (f_bs - a_s)^2 / (a_s (1 - a_s)), f_bs its fraction in bin b;
 * *index = mean_s I_s (1: segregated at the bin scale, 0: uniformly mixed; 0 with one colour).
 * per_species (host, ANN_MAX_COLORS doubles, may be NULL): I_s, NaN for absent or sole colours.
 * Bin counts are exact integers.  Errors: INVALID_ARG, STATE, CUDA, OOM. */
int ann_mixing_index(ann_ctx *ctx, int32_t G, double *index, double *per_species);

/* Unwrapped positions of particles `ids` (host, k IDs in [0, n)) for pathlines: x + L i_x, y + L i_y
 * with (i_x, i_y) the net periodic shifts of the particle since ann_set_particles (counted by the
 * step kernels when they re-insert a particle, Eq. 30).  xy: host, 2k doubles (x0, y0, x1, ...).
 * Errors: INVALID_ARG (an ID out of range), STATE, CUDA, OOM. */
int ann_get_unwrapped(ann_ctx *ctx, const int64_t *ids, int64_t k, double *xy);

/*
 * BF16 tensor-core GEMMs (5th-generation tensor cores) of the learned surrogate; the paper has no
 * counterpart.  All pointers are device pointers; BF16 = 16-bit bfloat (1 sign, 8 exponent, 7
 * mantissa bits); products accumulate in FP32.  The calls are synchronous on `stream` (a
 * cudaStream_t, NULL for the legacy default stream).  Errors: INVALID_ARG (shapes below), CUDA, OOM,
 * TIMEOUT (a tensor-core completion did not arrive within its bounded wait).
 *
 * ann_bf16_gemm: C[rows x N] = act([A1 | A2] . B^T + bias): A1 rows x K1 and A2 rows x K2 row-major
 * BF16 (A2 NULL when K2 = 0; K1 + K2 = K), B N x K row-major BF16, bias N FP32 or NULL, act = relu
 * (1) or identity (0); C rows x N row-major, BF16 (c_bf16 = 1) or FP32 (0; accumulate = 1 adds to
 * it).  K1, K2 multiples of 16 (K2 may be 0), K in [16, 256]; N a multiple of 16 in [16, 256];
 * A1, A2, B and C 16-byte aligned.
 *
 * ann_bf16_gemm_tn: C[K x N] += A^T . B over all rows: A rows x K, B rows x N row-major BF16, C
 * K x N row-major FP32 (accumulated with atomics, so the order of the FP32 additions varies between
 * runs).  K in [1, 256]; N a multiple of 16 in [16, 256].
 */
int ann_bf16_gemm(const void *A1, int32_t K1, const void *A2, int32_t K2, const void *B, int32_t N, int64_t rows,
                  const float *bias, int32_t relu, void *C, int32_t c_bf16, int32_t accumulate, void *stream);
int ann_bf16_gemm_tn(const void *A, int32_t K, const void *B, int32_t N, int64_t rows, float *C, void *stream);

/* Self-test of the bounded waits of the tensor-core kernels (the paper has no counterpart): one
 * device thread polls a shared-memory mbarrier that nothing completes, gives up after spin_limit
 * polls (1 .. 2^20) and raises a device flag the way an expired wait of ann_bf16_gemm or the
 * surrogate does; the call reads the flag and returns ANN_ERR_TIMEOUT, its expected result.  Nothing faults or hangs, and
 * the device stays usable.  Synchronous on the legacy default stream.  Errors: INVALID_ARG,
 * NOT_AVAILABLE, CUDA (ANN_OK would mean the wait completed, which is a defect). */
int ann_check_bounded_wait(uint32_t spin_limit);

/*
 * Learned coarse-step surrogate (the paper has no learned component; this is the project's).  A
 * message-passing MLP over the SPH neighbour graph predicts the increments of Q and u over k
 * steps; it is trained on the GPU by the project's own forward and backward kernels (BF16
 * tensor-core GEMMs with FP32 accumulation, FP32 Adam on master weights).  Network, with N(i) the
 * neighbours (|x_i - x_j| < 3h) and agg(f)_i = (W(0) f_i + sum_{j in N(i)} W_ij f_j) / S_i,
 * S_i = W(0) + sum_j W_ij (Eqs. 18, 19):
 *   x_i = (r_i, agg(r)_i - r_i, a k dt / ys_u, m k dt / ys_q, lapQ Gamma K k dt / ys_q,
 *          (div u, vort u) k dt),  r = (Q11, Q12, ux / us, uy / us),
 *   with the tendencies of the last step: the acceleration a (Eq. 23), the projected Q rate m
 *   (Eq. 24), the corrected Laplacian of Q11, Q12 (Eq. 21), and the divergence D_xx + D_yy and
 *   vorticity D_yx - D_xy of the corrected velocity gradient D (Eq. 20)
 *   h1 = relu(W1 [x ; agg(x)] + b1),  z1 = P1 h1,  h2 = relu(W2 [h1 ; agg(z1)] + b2),
 *   z2 = P2 h2,  h3 = relu(W3 [h2 ; agg(z2)] + b3),  y = Wo h3 + bo
 * with W1 128 x 32, P1, P2 32 x 128, W2, W3 128 x 160, Wo 4 x 128.  Parameters are one FP32 array
 * of ANN_SG_PARAMS values in the order W1, b1, P1, W2, b2, P2, W3, b3, Wo, bo (row-major).
 * Prediction over k steps: the explicit increment plus the network's correction,
 * dQ = k dt m + ys_q (y0, y1), du = k dt agg(agg(a)) + ys_u (y2, y3); the acceleration is
 * SPH-smoothed twice (the mean removes the velocity modes that an explicit step k times beyond the
 * viscous limit would amplify), the Q rate, mostly the particle-local bulk term, is not; positions
 * advance by k dt (u + u') / 2.  Errors: INVALID_ARG, STATE (nothing loaded), OOM, CUDA, TIMEOUT (a
 * tensor-core wait that did not complete within its bound), NOT_AVAILABLE.
 */
#define ANN_SG_PARAMS 54148
typedef struct ann_surrogate ann_surrogate;

/* A network for up to n_max particles (device buffers sized for it); parameters all 0. */
int ann_surrogate_create(int64_t n_max, ann_surrogate **out);
void ann_surrogate_destroy(ann_surrogate *sg);

/* Host FP32 parameters in and out (ANN_SG_PARAMS values); setting them resets the optimiser. */
int ann_surrogate_set_params(ann_surrogate *sg, const float *params);
int ann_surrogate_get_params(ann_surrogate *sg, float *params);

/* Seeded He initialisation of the hidden layers: weights N(0, 2 / fan_in), normals by Box-Muller
 * from a counter-based SplitMix64 stream; biases and the output layer (Wo, bo) 0, so that the
 * untrained network predicts the explicit increment.  Resets the optimiser. */
int ann_surrogate_init(ann_surrogate *sg, uint64_t seed);

/* Velocity scale us of the inputs, increment scales ys_q, ys_u of the outputs (all > 0), and the
 * number of steps k >= 1 the network spans (default 8). */
int ann_surrogate_set_scales(ann_surrogate *sg, double us, double ys_q, double ys_u, int32_t k);

/* Take the graph and the features of ctx's present state (a neighbour search at the present
 * positions; afterwards the context's next step re-sorts).  tend: host n x 8 FP32, component-major
 * (ax, ay, m11, m12, lapQ11, lapQ12, div u, vort u; component c of particle ID i at c n + i), or
 * NULL to take them from the context's last step, which must have run with ann_set_record(ctx, 1)
 * (STATE otherwise).  The network's graph holds up to 64 neighbours closer than 2h per particle
 * (~21 on a lattice); a denser cluster returns NBR_OVERFLOW instead of dropping neighbours. */
int ann_surrogate_load(ann_surrogate *sg, ann_ctx *ctx, const float *tend);

/* Network outputs y of the loaded state: host n x 4 FP32, ID order (may be NULL). */
int ann_surrogate_forward(ann_surrogate *sg, float *y);

/* The explicit increment k dt (m11, m12, agg(agg(a))) of the loaded state: host n x 4 FP32
 * (dQ11, dQ12, dux, duy), ID order; training targets are (true increment - this) / ys. */
int ann_surrogate_euler(ann_surrogate *sg, float *inc);

/* Forward and backward against targets t (host n x 4 FP32, ID order): *loss = mean (y - t)^2 over
 * the n x 4 outputs; gradients kept for ann_surrogate_adam and copied to grads (host,
 * ANN_SG_PARAMS FP32, may be NULL). */
int ann_surrogate_gradients(ann_surrogate *sg, const float *target, double *loss, float *grads);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with the last gradients. */
int ann_surrogate_adam(ann_surrogate *sg, double lr);

/* Advance ctx by the network's k steps with one evaluation: load (tend as for ann_surrogate_load),
 * forward, and replace the context's state by the prediction (t and the step count advance by k;
 * accelerations restart from 0, so the next jump needs a recorded plain step first; periodic image
 * counts follow the particles).  Q takes the explicit increment plus the network's correction; u
 * takes the explicit increment alone unless the velocity correction is switched on (below).  The
 * context keeps its cell structure and candidate lists (the next step re-sorts only if a particle
 * has moved half the skin since the last re-sort).  Errors: as ann_surrogate_forward; NONFINITE if
 * the prediction is not finite (the context's error bit is then set, as a failed step sets it). */
int ann_surrogate_jump(ann_surrogate *sg, ann_ctx *ctx, const float *tend);

/* Guarded advance: `cycles` surrogate cycles of ctx -- one recorded plain step, then one jump of k
 * steps -- with the network held to plain SPH.  Every `check_every` cycles (0: never) the cycle is
 * also run in plain SPH (k + 1 steps) on `shadow`, a second context of the same parameters and n
 * owned by the caller, from the same state (copied to it on the device), and the jump's increments
 * of Q and u over the cycle are compared with the plain ones: err = ||dX_jump - dX_plain|| /
 * ||dX_plain|| over all particles (FP64 sums in a fixed order).  If either error exceeds `tol` (the
 * configuration's bound is 0.05), or the jump is not finite, ctx takes the plain result of that
 * cycle and the remaining cycles run as plain steps: the fallback.  The report gives the completed
 * cycles, the checks, their largest and last errors, and where the fallback happened.  ctx's
 * recording setting is restored.  Errors: INVALID_ARG (shadow NULL or ctx itself while
 * check_every > 0, tol <= 0, ctx larger than the network's n_max), STATE, the errors of ann_step
 * and ann_surrogate_jump (NONFINITE from an unchecked jump), CUDA.  After a fallback from a
 * non-finite jump ctx is reloaded (ann_set_state): its periodic image counts restart. */
typedef struct ann_guard_report {
    int32_t cycles_done;       /* jumps kept */
    int32_t checks;            /* cycles compared with plain SPH */
    int32_t fell_back;         /* 1: a check failed; the rest ran in plain SPH */
    int32_t fallback_cycle;    /* index of the failed check's cycle, -1 if none */
    int64_t plain_steps;       /* plain steps run after the fallback */
    double max_err_q, max_err_u;     /* largest errors of the checks */
    double last_err_q, last_err_u;   /* the last check's errors */
} ann_guard_report;
int ann_surrogate_advance(ann_surrogate *sg, ann_ctx *ctx, ann_ctx *shadow, int32_t cycles, int32_t check_every,
                          double tol, ann_guard_report *report);

/* Whether the jump adds the network's velocity correction ys_u (y2, y3) (on = 1) or not (0, the
 * default).  In the viscous regime of the paper's runs u follows Q almost instantly: the
 * correction gains little on a single jump and, fed back over many jumps, grows a mode of its own,
 * so rollouts leave it off.  Errors: INVALID_ARG. */
int ann_surrogate_set_velocity_correction(ann_surrogate *sg, int32_t on);

const char *ann_surrogate_last_error(ann_surrogate *sg);

/*
 * Batched ensemble: many independent runs (any mix of n and parameters, e.g. the (zeta, K) sweeps
 * of the paper's results section) advanced together.  Each member is a full context; one
 * ann_ensemble_step launches a single CUDA graph per step in which every member's step (with its
 * own re-sort decision) is a branch, so the GPU overlaps the members and its block scheduler
 * balances their uneven sizes.  Members are dealt round-robin to `groups` branches (members of a
 * branch run one after the other); ann_ensemble_autotune times the groupings 1, 4, 16, ... and all
 * members and keeps the fastest.  Every member advances exactly as ann_step would advance it alone
 * (bit-identical results).
 */
#define ANN_ENSEMBLE_MAX 256
typedef struct ann_ensemble ann_ensemble;

/* Create `members` contexts from params[0 .. members) (each validated as by ann_create).  Errors:
 * INVALID_ARG, OOM, CUDA, NOT_AVAILABLE; nothing is left allocated on error. */
int ann_ensemble_create(const ann_params *params, int32_t members, ann_ensemble **out);
void ann_ensemble_destroy(ann_ensemble *ens);

/* Borrowed handle of member k: load it (ann_set_particles, ann_load_state), read fields and
 * diagnostics, save it.  Do not destroy it; ann_step on it advances that member alone. */
int ann_ensemble_member(ann_ensemble *ens, int32_t k, ann_ctx **ctx);

/* Advance every member by nsteps steps (one graph launch per step) and synchronise.  All members
 * must hold particles (STATE otherwise).  Returns the first member's error status, if any (text
 * in ann_ensemble_last_error, naming the member); the other members still advanced. */
int ann_ensemble_step(ann_ensemble *ens, int64_t nsteps);

/* Rebuild the ensemble graph with members dealt to `groups` branches (1 .. members). */
int ann_ensemble_set_groups(ann_ensemble *ens, int32_t groups);

/* For each candidate grouping (1, 4, 16, ... and all members): one warm-up step, then
 * trial_steps timed steps (CUDA events on the ensemble stream); keep the fastest.  The trial steps
 * are real steps (the members advance by them).  groups_out, ms_per_step (may be NULL): the chosen
 * grouping and its time per ensemble step.  Errors: as ann_ensemble_step, INVALID_ARG. */
int ann_ensemble_autotune(ann_ensemble *ens, int32_t trial_steps, int32_t *groups_out, double *ms_per_step);

const char *ann_ensemble_last_error(ann_ensemble *ens);

/*
 * FP32 fused multiply-add throughput of the current device, measured (the roofline of the pair
 * passes, which are bound by plain FP32 issue).  The paper has no counterpart: this is a measuring
 * utility.  Runs independent FMA chains on every SM at full occupancy, in the scalar form and in
 * the two-lane form (one instruction for two lanes), on `stream` (a cudaStream_t, NULL: the legacy
 * default stream), and returns the best of three timed launches of each in TFLOP/s (2 flops per lane
 * FMA) and the device's SM count (sms may be NULL).  Synchronises; allocates a small scratch buffer.
 * Errors: INVALID_ARG (NULL outputs), CUDA.
 */
int ann_fp32_fma_peak(void *stream, double *tflops_scalar, double *tflops_pair, int32_t *sms);

/*
 * Velocity moments without any device allocation.  The paper has no counterpart: this is a
 * service entry point for callers that cannot call cudaMalloc -- a host framework that owns a fixed
 * device memory pool or a hard memory budget and forbids allocations after start-up, or a real-time
 * loop that cannot take the implicit device synchronisation cudaMalloc may perform.
 *
 * Computes, for a velocity field already on the device (FP32 arrays ux, uy of length n, any
 * particle order), in FP64 with a fixed reduction order (deterministic):
 *   out[0], out[1] = sum_i m_i u_i (momentum), m_i = mass[i], or m0 for every particle if mass is NULL
 *   out[2]         = 1/2 <|u|^2>, the mean over the n particles (the kinetic_energy of ann_diag)
 *   out[3]         = max_i |u_i|
 * the same quantities ann_get_diagnostics reports for a context's state.  `out` is a device pointer
 * to 4 doubles; the call is asynchronous on `stream` (a cudaStream_t, NULL for the legacy default
 * stream) and the result is there once the stream reaches it.
 *
 * It allocates nothing: its only scratch is a file-scope device array of ANN_NOALLOC_MAX_N / 256
 * FP64 partials and a ticket (about 256 KB), which every GPU that loads this library holds until the
 * process exits.  n must be in [1, ANN_NOALLOC_MAX_N]; larger n returns ANN_ERR_TOO_LARGE.  The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current) and caches it; make that first call before any stream capture.  All calls share
 * the one array: calls whose kernels overlap on the GPU (different streams, or different host
 * threads on one device) race on it and must be serialised by the caller.  Every pointer must be
 * device memory of the current device (a pointer to host memory or to another GPU's memory returns
 * INVALID_ARG before any launch).  Errors: INVALID_ARG (NULL pointer, n < 1, a pointer that is not
 * memory of the current device), TOO_LARGE, CUDA.
 */
#define ANN_NOALLOC_MAX_N 2097152
int ann_velocity_moments_noalloc(const float *ux, const float *uy, const float *mass, double m0,
                                 int64_t n, double *out, void *stream);

/*
 * Three-dimensional variant of the step (§3 with d = 3; the paper's runs are 2D, its equations are
 * written for any dimension and Eq. (18) gives the 3D kernel constant a_d = 3 / (359 pi h^3)).
 * Q is the symmetric traceless 3x3 tensor, stored as five components (Q11, Q12, Q13, Q22, Q23),
 * Q33 = -Q11 - Q22; the molecular field keeps the B term (Q^2 - tr(Q^2) I / 3) of Eq. (7); the
 * corrected Laplacian is the scalar form with factor 2 per component; the viscous term of Eq. (23)
 * carries 2 (d + 2) nu = 10 nu.  Paper momentum mode only, no elastic stress.  A periodic cube of
 * side L; cells of side >= 3h (1 + 0.05), at least 3 per side (L >= 9.45 h: 13 particles a side at
 * h = 1.3 dx).  Candidate lists (every j within 3h (1 + 0.05), rebuilt with a re-sort when a
 * particle has moved 0.05 x 3h / 2) hold at most 576, neighbour lists ANN3_MAX_NEIGHBORS (~250 at
 * h = 1.3 dx).  FP64 positions; pair differences are taken
 * in FP64 and everything else runs in FP32.  The step order is that of the 2D step (modified
 * Euler predictor, search, volumes, correction tensor, continuity, density filter and equation of
 * state, velocity gradient, Laplacian of Q, Q rate, momentum, artificial displacement, corrector).
 */
#define ANN3_MAX_NEIGHBORS 448

typedef struct ann3_ctx ann3_ctx;

typedef struct {
    int64_t n;
    double L, h, dt, rho0, eta, Gamma, lambda_, A, B, C, K, zeta, gamma_eos, beta, c0_min, c_shift;
    int32_t apd;
    int32_t reserved[3];
} ann3_params;

/* Fields of ann3_get_field: components per particle in brackets. */
enum {
    ANN3_FIELD_POS = 0,    /* x, y, z [3] */
    ANN3_FIELD_U = 1,      /* velocity [3] */
    ANN3_FIELD_Q = 2,      /* Q11, Q12, Q13, Q22, Q23 [5] */
    ANN3_FIELD_RHO = 3,    /* density [1] */
    ANN3_FIELD_A = 4,      /* acceleration of the last step [3] */
    ANN3_FIELD_SUMW = 5,   /* W(0) + sum_j W_ij of the last step [1] */
    ANN3_FIELD_GRADU = 6,  /* corrected velocity gradient du_a/dx_b, row-major [9] */
    ANN3_FIELD_LAPQ = 7,   /* corrected Laplacian of the five Q components [5] */
    ANN3_FIELD_QRATE = 8,  /* projected Q rate m of Eq. (24) [5] */
    ANN3_FIELD_P = 9,      /* pressure [1] */
    ANN3_FIELD_NNBR = 10,  /* neighbours [1] */
    ANN3_FIELD_COUNT = 11
};

/* Defaults: L 1, h 1.3 / 32, dt 1e-4, rho0 1, eta 1, Gamma 0.34, lambda 0.7, A 0, B 0, C 1, K 0.04,
 * zeta 0.05, gamma 7, beta 1, c0_min 0, c_shift 1/3, apd 1; n 32^3. */
int ann3_default_params(ann3_params *p);

/* Device buffers for n particles.  Errors: INVALID_ARG (n < 1, h or L not positive, fewer than 3
 * cells per side), NOT_AVAILABLE, OOM, CUDA. */
int ann3_create(const ann3_params *p, ann3_ctx **out);
void ann3_destroy(ann3_ctx *c);

/* Load the state, ID order, host FP64: x, y, z (n each, in [0, L)), u (3n: ux, uy, uz per particle),
 * q (5n), rho (n, or NULL for rho0); accelerations restart from 0.  Errors: INVALID_ARG (n differs
 * from the context's, a NULL array, a non-finite value or a position outside [0, L)), CUDA. */
int ann3_set_particles(ann3_ctx *c, int64_t n, const double *x, const double *y, const double *z,
                       const double *u, const double *q, const double *rho);

/* Advance by nsteps steps.  Errors: STATE (no particles), NBR_OVERFLOW, CELL_OVERFLOW,
 * NONFINITE, SINGULAR_ALPHA (sticky device flags set by the kernels' own checks), CUDA. */
int ann3_step(ann3_ctx *c, int64_t nsteps);

/* A field in ID order into host FP64 dst (n x components, interleaved per particle).  Errors:
 * INVALID_ARG (unknown field, NULL dst), STATE, CUDA. */
int ann3_get_field(ann3_ctx *c, int32_t field, double *dst);

/* Steps taken, the device error bits (4 neighbours, 8 non-finite, 16 alpha) and the number of steps
 * that re-sorted and rebuilt the candidate lists since ann3_set_particles (each pointer may be NULL). */
int ann3_get_status(ann3_ctx *c, int64_t *steps, uint32_t *error_bits, int64_t *resorts);

const char *ann3_last_error(ann3_ctx *c);

#ifdef __cplusplus
}
#endif

#endif /* ANN_H */
