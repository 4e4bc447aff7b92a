/*
 * gpweno.h -- C ABI of the GB300 (sm_103a) GP-WENO finite-difference library
 * for the compressible Euler equations.
 *
 * The library evaluates, per face and per Runge-Kutta stage, the conservative
 * flux divergence of the GP-WENO FD-Prim scheme of Reyes, Lee, Graziani and
 * Tzeferacos (arXiv:1808.04960) and fuses it with the SSP-RK3 stage update:
 *
 *   - Riemann states at every face by GP-WENO interpolation of characteristic
 *     variables (Sections 3.2-3.3; the stepwise algorithm of Section 4, step 2),
 *     with the Roe-averaged eigenvectors of the two cells sharing the face;
 *   - local Lax-Friedrichs face flux on those states (Eq. riemann_prob);
 *   - the high-order correction with alpha = -1/24, beta = 3/640
 *     (Eqs. numFlux_cor, FD-ders);
 *   - the flux difference (Eq. disc_fd) and the SSP-RK3 stage combination
 *     (Section 2, step 5; Shu-Osher form).
 *
 * Conventions for every entry point:
 *   - No exception or C++ type crosses this boundary; every function returns
 *     a gpweno_status.  gpweno_last_error() gives a thread-local message for
 *     the last non-OK status raised on the calling thread.
 *   - State arrays are caller-owned DEVICE buffers in structure-of-arrays
 *     layout [nc][nz][ny][nx] (x fastest), interior cells only (no ghost
 *     cells: boundary conditions are applied when tiles are loaded),
 *     nc = ndim + 2 components (rho, rho*u_1, ..., rho*u_ndim, E), element
 *     type float (GPWENO_F32) or double (GPWENO_F64) as chosen at plan
 *     creation.  Buffers must be 16-byte aligned.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Launches are asynchronous; errors of earlier launches surface at the
 *     next call or at gpweno_flags().  Step functions allocate nothing and do
 *     not synchronise.
 *   - A plan owns its weight tables and a small device workspace (flags,
 *     wavespeed maxima); it is not thread-safe to use one plan from two
 *     streams at once.
 */
#ifndef GPWENO_H
#define GPWENO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GPWENO_OK = 0,
    GPWENO_ERR_ARG = 1,          /* invalid argument (message says which) */
    GPWENO_ERR_PRECOMPUTE = 2,   /* GP tables ill-conditioned even in double-double */
    GPWENO_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    GPWENO_ERR_NONPHYSICAL = 4,  /* rho <= 0, p <= 0 or NaN met by a kernel */
    GPWENO_ERR_TIMEOUT = 5       /* reserved: bounded device wait gave up */
} gpweno_status;

typedef enum { GPWENO_F32 = 0, GPWENO_F64 = 1 } gpweno_dtype;
/* Boundary conditions per side of a dimension.  GPWENO_BC_EXTERNAL: the ghost
 * layers of that side are supplied by the caller in a halo buffer (see
 * gpweno_set_halo): the side is a cut between the subdomains of one grid that
 * is split into slabs along its slowest dimension, one slab per rank (the
 * paper's solver is parallelized over cores, Section 5, and its vortex timings
 * of Section 6.2 ran on four).
 * Allowed on the slowest dimension only (x in 1D, y in 2D, z in 3D), which
 * then needs at least R+3 cells. */
typedef enum { GPWENO_BC_PERIODIC = 0, GPWENO_BC_OUTFLOW = 1, GPWENO_BC_EXTERNAL = 2 } gpweno_bc;

typedef struct gpweno_plan_s *gpweno_plan;   /* opaque, owned by the library */

/* Grid description.  ndim in {1,2,3}; n[d] cells and spacing dx[d] for
 * d < ndim (x, y, z order); bc_lo/bc_hi per dimension (gpweno_bc).  Periodic
 * must be set on both sides of a dimension or on neither. */
typedef struct {
    int ndim;
    int n[3];
    double dx[3];
    int bc_lo[3];
    int bc_hi[3];
} gpweno_dims;

/* Options (NULL = defaults).
 *   sigma_over_dx  length hyperparameter of the smoothness-indicator kernel
 *                  (Section 3.4; default 3.0).  Must be > 1.
 *   eps, p         WENO-JS constants of Eq. weights (default 1e-36 and 2; p in {1,2}).
 *   dtype          GPWENO_F32 (bulk arithmetic in FP32, tables rounded from
 *                  double-double) or GPWENO_F64.
 *   cfl            if > 0, gpweno_rk3_step with a dt_dev pointer also writes
 *                  the next step's dt = cfl / sum_d max(|u_d|+c)/dx_d of the
 *                  new state into *dt_dev (fused into the last stage).
 *   flux_form      face flux of Eq. riemann_prob on the GP-WENO states:
 *                  0 = local Lax-Friedrichs (default), 1 = HLLC with Einfeldt
 *                  wave speeds from the Roe average (the paper's default
 *                  solver, Section 7), 2 = HLL with the same speeds (the
 *                  solver of the paper's Mach-3 wind-tunnel test, Section 7).
 *   beta_mean      0 = zero-mean GP smoothness indicators, beta on f_m (the
 *                  paper's choice, Eq. gp-smooth); 1 = non-zero mean, beta on
 *                  f_m - f_i with f_i the centre value of the stencil (the
 *                  variant of Sections 3.3 and 7.1).
 *   candidates     0 = GP candidate predictions (Eq. candidate_interp);
 *                  1 = polynomial (Lagrange) candidates and their linear
 *                  weights with the GP smoothness indicators (the paper's
 *                  WENO-GP hybrid).
 *   scheme         0 = FD-Prim (default): GP-WENO Riemann states at faces,
 *                  face flux, high-order correction (Eqs. riemann_prob,
 *                  numFlux_cor).  1 = FD-Flux (Section 2): the point fluxes are
 *                  read as cell averages of the function whose face values are
 *                  the numerical fluxes (Eqs. prim_F, design); they are split by
 *                  local Lax-Friedrichs, F+- = (F +- alpha U)/2 with alpha the
 *                  largest |u_n| + c over the face's 2R+2 stencil cells, projected
 *                  on the characteristic fields of the conservative Jacobian at
 *                  the Roe average, and reconstructed with GP weights conditioned
 *                  on cell averages; no correction.  Requires flux_form = 0.
 *   ao             1 = GP-AO (Appendix A) in place of GP-WENO for the Riemann
 *                  states: R = 2 gives AO(2,3), R = 3 the recursive AO(3,2,3);
 *                  the high-order GP prediction (Eq. q-intrp) hybridised with
 *                  the GP-CWENO combination of the three 3-point stencils
 *                  (Eqs. cweno_stencil, nonlin-AO, CWENO-lin, GP-AO,
 *                  recursive-weights, AO-recursive), beta of each stencil the
 *                  data-fit term (1/2) f^T K_N(sigma)^-1 f of Eq. log-like
 *                  divided by its value on constant data, 1^T K_N^-1 1, so that
 *                  stencils of different size N agree on smooth data.
 *                  Requires scheme = 0 and candidates = 0.
 *   ao_gamma_hi, ao_gamma_lo
 *                  gamma_HI and gamma_LO of Eq. CWENO-lin, in (0,1)
 *                  (default 0.85 each). */
typedef struct {
    double sigma_over_dx;
    double eps;
    int p;
    int dtype;
    double cfl;
    int flux_form;
    int beta_mean;
    int candidates;
    int scheme;
    int ao;
    double ao_gamma_hi;
    double ao_gamma_lo;
} gpweno_opts;

void gpweno_default_opts(gpweno_opts *opts);

/* Build a plan: GP radius R in {1,2,3} (stencil 2R+1 points, R+1 sub-stencils
 * of R+1 points, Eq. sub-stencil), length hyperparameter l/dx (Eqs. se, kmat,
 * kstar; must satisfy l/dx >= 1), grid `dims`, ratio of specific heats
 * `gamma_gas` (> 1).  The GP weights w_m (Eq. candidate_interp), linear
 * weights gamma_m (Eq. gamm-system, least squares), and the smoothness
 * factors P_h = v_h / sqrt(lambda_h) of K_m(sigma) (Eq. beta-eigen) are
 * computed in double-double arithmetic on the host (Section 4, step 1),
 * rounded to the plan's dtype and kept with the plan.  Allocates a few
 * hundred bytes of device memory on the current device; the plan must be
 * used on that device.  Returns GPWENO_ERR_PRECOMPUTE if the covariance
 * system is too ill-conditioned for double-double. */
gpweno_status gpweno_plan_create(gpweno_plan *out, int R, double ell_over_dx, const gpweno_dims *dims,
                                 double gamma_gas, const gpweno_opts *opts);
gpweno_status gpweno_plan_destroy(gpweno_plan plan);

/* Copy the plan's tables (double precision, before rounding to the plan's
 * dtype) to host arrays; any pointer may be NULL.  All refer to the
 * prediction point x* = x_i + dx/2 (left state of face i+1/2):
 *   w_m   (R+1)*(R+1): w_m[m*(R+1)+j] = weight of point j of sub-stencil m
 *         (sub-stencil m covers cells i-R+m .. i+m), Eq. candidate_interp;
 *   gam   R+1 linear weights (Eqs. gamm-system, M-mat);
 *   P     (R+1)*(R+1): P[h*(R+1)+j] = v_h[j] / sqrt(lambda_h), eigenpairs of
 *         K_m(sigma) ascending (Eq. beta-eigen);
 *   w_big 2R+1 GP weights on the full stencil (Eq. q-intrp). */
gpweno_status gpweno_plan_tables(gpweno_plan plan, double *w_m, double *gam, double *P, double *w_big);

/* Host-only: the double-double GP tables of gpweno_plan_create without a
 * plan or a device (for checking the precompute on machines without a GPU).
 * `candidates` and `scheme` as in gpweno_opts (scheme 1: reconstruction weights).
 * Left-state tables as in gpweno_plan_tables; w_m_r, gam_r are the tables
 * of the right state of face i+1/2 (x* = x_{i+1} - dx/2, stencil of cell
 * i+1).  Any output pointer may be NULL.  Returns GPWENO_ERR_ARG or
 * GPWENO_ERR_PRECOMPUTE as gpweno_plan_create would. */
gpweno_status gpweno_gp_tables(int R, double ell_over_dx, double sigma_over_dx, int candidates, int scheme,
                               double *w_m, double *gam, double *P, double *w_big, double *w_m_r, double *gam_r);

/* dUdt = L(U): the right-hand side of Eq. disc_fd with the corrected fluxes
 * of Eq. numFlux_cor.  U, dUdt: device state arrays (see conventions);
 * they must not overlap. */
gpweno_status gpweno_rhs(gpweno_plan plan, const void *U, void *dUdt, void *stream);

/* One SSP-RK3 step in place on U (three fused stage launches; plans with an
 * external side step with gpweno_rk3_stage instead, GPWENO_ERR_ARG here):
 *   U1 = U + dt L(U);  U2 = 3/4 U + 1/4 (U1 + dt L(U1));  U <- 1/3 U + 2/3 (U2 + dt L(U2)),
 * carried in the equivalent increment form D1 = dt L(U), D2 = 1/4 (D1 + dt L(U+D1)),
 * U <- U + 2/3 (D2 + dt L(U+D2)), whose final sum is compensated (TwoSum): the
 * rounding remainder of each step's update is kept and added to the next one, so
 * FP32 state rounding does not accumulate over long runs.
 * scratch: caller-owned device buffer of 4 state sizes: [0] increment D, [1] U+D1,
 * [2] U+D2 (all three overwritten every step), [3] the compensation remainder,
 * carried from step to step -- it must be ZERO whenever U is (re)initialised and
 * left untouched between steps of one run.
 * dt_dev: NULL to use `dt`; otherwise a device double holding dt, read by
 * the kernels (graph-capturable), and, when the plan's cfl > 0, overwritten
 * after the step with the CFL time step of the new state. */
gpweno_status gpweno_rk3_step(gpweno_plan plan, void *U, void *scratch, double dt, void *dt_dev, void *stream);

/* Allocation-free SSP-RK3 step (the paper has no counterpart: this is a
 * service for callers that may not allocate device memory, e.g. code whose
 * host application owns all device memory through its own pool or caching
 * allocator, or a plug-in handed only the state buffer).  Same kernels as
 * gpweno_rk3_step with dt_dev = NULL, but the three intermediate stage
 * buffers live in a 16 MiB array of device memory that is part of the
 * library image, so the call allocates nothing; no compensation remainder
 * is carried between calls (each call's final sum is rounded once).
 *   - Grids whose three stage copies (each rounded up to 256 bytes) exceed
 *     16 MiB are rejected with GPWENO_ERR_ARG: at most 349,520 cells for
 *     FP32 2D (e.g. 591 x 591), 174,760 for FP64 2D.
 *   - Every GPU that loads the library holds the 16 MiB until exit.
 *   - All calls on a device share the one array and the previous call's
 *     contents stay in it (nothing in it needs to start at zero); calls whose
 *     kernels overlap on the GPU (other streams, other host threads) race.
 *   - The first call on a device looks up the array's device address with
 *     that device current, and so does the first call after the device's
 *     context was torn down and re-created (cudaDeviceReset); make such a
 *     first call before any stream capture.
 *   - gpweno_last_launch_count() afterwards gives this call's launches (3).
 * U: device state buffer (input and output), dt > 0, stream as elsewhere. */
gpweno_status gpweno_rk3_step_noalloc(gpweno_plan plan, void *U, double dt, void *stream);

/* *dt_dev (device double) = cfl / sum_d max over cells of (|u_d| + c)/dx_d. */
gpweno_status gpweno_cfl_dt(gpweno_plan plan, const void *U, double cfl, void *dt_dev, void *stream);

/* ---- Slab decomposition of one grid over several ranks ---------------------
 * One SSP-RK3 step of a slab whose plan has GPWENO_BC_EXTERNAL sides is three
 * calls of gpweno_rk3_stage, and before each the G = R+3 boundary layers of
 * that stage's input state are exchanged with the neighbouring slabs
 * (Eq. disc_fd with the corrected flux of Eq. numFlux_cor reaches G cells):
 *   for k in 0, 1, 2:
 *       gpweno_halo_pack(plan, stage_input(k), send_lo, send_hi, stream);
 *       send send_lo to the lower neighbour and send_hi to the upper one; receive
 *       the lower neighbour's send_hi into recv_lo and the upper one's send_lo
 *       into recv_hi (the caller's transport, e.g. NCCL send/recv);
 *       gpweno_rk3_stage(plan, k, U, scratch, dt, dt_dev, stream);
 * with stage_input(0) = U, stage_input(1) = scratch + 1 state, stage_input(2) =
 * scratch + 2 states (the scratch layout of gpweno_rk3_step), and recv_lo /
 * recv_hi registered once with gpweno_set_halo.  A CFL time step common to all
 * ranks takes one max-reduction of three numbers per step (gpweno_rate_export,
 * then gpweno_dt_from_rates).  Halo layout: [nc][G][layer], G layers of
 * `layer` cells (nx*ny in 3D, nx in 2D, 1 in 1D) in increasing order of the
 * slab coordinate: recv_lo holds the G cells just below the slab, recv_hi the G
 * cells just above it. */

/* Register the device halo buffers the kernels read for the plan's external
 * sides (each nc*G*layer elements of the plan's dtype, 16-byte aligned, owned
 * by the caller and alive while the plan steps); a side that is not external
 * ignores its pointer (may be NULL).  GPWENO_ERR_ARG if an external side gets
 * NULL or the plan has no external side. */
gpweno_status gpweno_set_halo(gpweno_plan plan, const void *recv_lo, const void *recv_hi);

/* Copy the first G and the last G layers of `state` (a device state of the
 * plan's shape; it may be a stage buffer inside the scratch, so only element
 * alignment is required) along the slowest dimension into send_lo and send_hi
 * (halo layout, either may be NULL).  One kernel launch on `stream`.  The
 * slowest dimension must have at least G cells. */
gpweno_status gpweno_halo_pack(gpweno_plan plan, const void *state, void *send_lo, void *send_hi, void *stream);

/* Stage k (0, 1, 2) of gpweno_rk3_step on the same buffers (U, 4-state scratch,
 * dt / dt_dev), one fused launch (two in 3D).  Stage 2 with dt_dev and a plan
 * cfl > 0 accumulates the maxima of (|u_d|+c)/dx_d of the new state in the
 * plan's rate buffer but does not compute the next dt (see gpweno_rate_export).
 * External sides read the registered halo buffers, which must hold stage k's
 * input layers of the neighbours when the launch runs. */
gpweno_status gpweno_rk3_stage(gpweno_plan plan, int stage, void *U, void *scratch, double dt, void *dt_dev,
                               void *stream);

/* Accumulate the maxima of (|u_d|+c)/dx_d over the cells of U in the plan's
 * rate buffer (for a common initial time step across ranks). */
gpweno_status gpweno_rates(gpweno_plan plan, const void *U, void *stream);

/* Copy the plan's three rate maxima (x, y, z; as the bit patterns of
 * non-negative doubles, which order like the doubles, so an unsigned 64-bit
 * max-reduction across ranks is the max of the rates) to the device buffer
 * `rates` (3 x uint64) and clear the plan's buffer.  One launch. */
gpweno_status gpweno_rate_export(gpweno_plan plan, void *rates, void *stream);

/* *dt_dev = cfl / sum_d rates[d] with rates as written by gpweno_rate_export
 * (typically after a max-reduction across ranks).  One launch. */
gpweno_status gpweno_dt_from_rates(gpweno_plan plan, const void *rates, double cfl, void *dt_dev, void *stream);

/* Host-only: the double-double GP-AO tables of a plan with ao = 1 (for
 * checking the precompute without a device).  w_hi: 2 x (2R+1) weights of the
 * full stencil, left (x* = +1/2) then right (x* = -1/2); w_lo: 2 x (2R-1)
 * weights of S_{R-1} (R = 3 only); w3: 2 x 3 x 3 weights of the 3-point
 * stencils of Eq. cweno_stencil; P_hi, P_lo, P_3: the N x N factors
 * v_h / sqrt(lambda_h) of K_N(sigma) (lambda ascending) for N = 2R+1, 2R-1, 3.
 * Any pointer may be NULL.  Errors as gpweno_plan_create (R must be 2 or 3). */
gpweno_status gpweno_ao_tables(int R, double ell_over_dx, double sigma_over_dx, double *w_hi, double *w_lo,
                               double *w3, double *P_hi, double *P_lo, double *P_3);

/* Read and clear the plan's sticky flag word (synchronises the device).
 * Bit 0 (*nonphysical & 1) is set if any kernel since the last read met
 * rho <= 0, p <= 0 or a NaN.  In the bounds-checked test build of the library
 * (compiled with -DGPWENO_CHECKED) bits 1-11 record a shared-memory or global
 * access outside its array, by access site, which that build skipped instead
 * of making; the default build never sets them.  Returns GPWENO_ERR_CUDA if an
 * earlier launch failed. */
gpweno_status gpweno_flags(gpweno_plan plan, int *nonphysical);

/* Batched 2D stepping (same per-face scheme as gpweno_rk3_step): one
 * launch per RK stage serves n independent 2D plans of possibly
 * different grid size, R, l/dx, sigma, face flux, candidates and boundary
 * conditions (all plans must share dtype and device and use beta_mean = 0,
 * scheme = 0 and ao = 0, else GPWENO_ERR_ARG; at most 12 distinct table sets
 * per radius).  The host cuts every
 * instance into strips and row segments and hands each CTA a contiguous run of
 * segments of equal estimated cost (by default 8 CTAs per resident CTA slot,
 * so that the hardware scheduler evens out the estimate's misses).  The batch
 * refers to the member plans,
 * which must outlive it.  tune_cache: NULL, or the path of a text file of
 * lines "<signature hex> <block 128|256> <ctas per SM>" (written by
 * paper_1808_04960_gb300/autotune.py); a line whose signature matches this
 * batch overrides the built-in block-size choice; a line may add three more
 * fields "<strip width cap (0 = as the block allows)> <fewest rows of a segment
 * that does not end its strip> <CTA shares per resident slot (1..16)>" (the
 * tile shapes the autotuner searches).  Allocates its schedule and descriptor
 * arrays on the device. */
gpweno_status gpweno_plan_batch(gpweno_plan *out_batch, const gpweno_plan *plans, int n, const char *tune_cache);

/* One SSP-RK3 step of every instance of a batch plan, in place:
 * U[k] is instance k's state and scratch[k] its 4-state-size scratch (same
 * layout and zero-initialised compensation as gpweno_rk3_step); dt_dev:
 * device array of n doubles (per-instance time steps).  Three kernel
 * launches in total; when the buffer pointers differ from the previous call,
 * the first launch is preceded by one host-to-device copy of the instance
 * descriptors (and a synchronisation of `stream`), so keep them fixed when
 * capturing the step in a CUDA graph. */
gpweno_status gpweno_batch_rk3_step(gpweno_plan batch, void *const *U, void *const *scratch, const void *dt_dev,
                                    void *stream);

/* Schedule of a batch plan (for tuning and reports): block size, CTAs per SM
 * assumed, CTAs per launch, number of segments, instance-list signature. */
int gpweno_batch_info(gpweno_plan batch, int *block, int *ctas_per_sm, int *grid, int *segments,
                      unsigned long long *signature);

/* Schedule of the last 2D stage launch of a (non-batch, 2D) plan: strip width
 * (columns), number of strips, CTAs launched, and the resident CTAs per SM of
 * the kernel build used (FP32 takes a three-CTA build on small grids, four
 * CTAs otherwise; FP64 one).  All zero before the first launch.  Returns
 * GPWENO_ERR_ARG for batch plans and 1D or 3D plans. */
int gpweno_plan_schedule(gpweno_plan plan, int *strip_width, int *strips, int *grid, int *ctas_per_sm);

/* Tile shapes of a batch plan's schedule: the widest strip (columns), the
 * fewest rows of a segment that does not finish its strip, and CTA shares per
 * resident CTA slot. */
int gpweno_batch_tiles(gpweno_plan batch, int *strip_width_cap, int *min_rows, int *ctas_per_slot);

/* Number of kernel launches the last step function issued (for launch accounting). */
int gpweno_last_launch_count(void);

const char *gpweno_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GPWENO_H */
