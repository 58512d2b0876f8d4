/*
 * gg.h -- C ABI of the GB300 (sm_103a) library for the explicit
 * finite-volume time step of the anisotropic, heterogeneous
 * Gatenby-Gawlinski system (Mascia, Pera, Simeoni, arXiv 2006.01748).
 *
 *   eq. (1)   U_t = U(1-U) - delta U W
 *             V_t = rho V(1-V) + D div[(1-U) grad V]
 *             W_t = c (V-W) + div(A grad W)
 *   eq. (2)   A = [[a11, a12], [a12, a22]] per cell, built here as
 *             A = R(theta) diag(lambda1, lambda2) R(theta)^T,
 *             R = [[cos, -sin], [sin, cos]]
 *   eq. (3)   explicit Euler on cell-centred unknowns, one fixed dt
 *   Table 1   five-point tumour stencil, face mobility 1 - (U_P + U_nb)/2
 *   Table 2   nine-point acid stencil (face fluxes, a12 cross terms)
 *   Section 2 zero-flux (Neumann) boundary: no flux through boundary faces,
 *             tangential differences at the boundary use mirror ghosts
 *
 * Paper symbols: delta = d, rho = r, D = alpha, c = c (acid rate); the
 * tensor entries a, b, c of Table 2 are a11, a12, a22 here.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Status: every int-returning call returns GG_OK (0) or a negative
 *   GG_ERR_* code; no exception or exit() crosses the ABI.
 *   gg_last_error(sim) gives a text for the last failure on that object.
 * - Layout of host field arrays: nx*ny values, row-major with x fastest,
 *   element (i, j) at index j*nx + i, i along x in [0, nx), j along y.
 *   Cell (i, j) is centred at ((i + 1/2) dx, (j + 1/2) dy), dx = lx/nx,
 *   dy = ly/ny.
 * - Ownership: the caller owns every pointer it passes; inputs are copied
 *   before the call returns (host) or before the work it enqueues reads
 *   them (device).  The library owns all device memory of a gg_sim /
 *   gg_batch and frees it in gg_destroy / gg_batch_destroy.
 * - Streams: work is enqueued on the cudaStream_t given at creation
 *   (NULL = legacy default stream).  Calls marked "synchronizes" wait for
 *   that stream before they return; the others are asynchronous.
 * - One device: a gg_sim lives on the device that was current when it was
 *   created; make that device current before every later call.
 */
#ifndef GG_H
#define GG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define GG_OK             0
#define GG_ERR_ARG       -1  /* null pointer, bad size or flag, non-finite input */
#define GG_ERR_NOT_SPD   -2  /* some lambda1/lambda2 <= 0: A not positive definite (eq. 2) */
#define GG_ERR_CFL       -3  /* explicit dt above the stable bound */
#define GG_ERR_OOM       -4  /* device allocation failed */
#define GG_ERR_CUDA      -5  /* a CUDA call failed (text in gg_last_error) */
#define GG_ERR_NONFINITE -6  /* the state holds NaN or Inf */
#define GG_ERR_TIMEOUT   -7  /* a bounded device-side wait gave up */
#define GG_ERR_STATE     -8  /* call not valid in the object's current state */

/* ---- precision of the state and the stencil arithmetic ---- */
#define GG_FP64_PLAIN  0  /* double state and arithmetic, one thread per cell */
#define GG_FP32        1  /* float state and arithmetic */
#define GG_FP32_KAHAN  2  /* float arithmetic, Kahan-compensated float state */

/* ---- fields for gg_read / gg_write ---- */
#define GG_FIELD_U       0
#define GG_FIELD_V       1
#define GG_FIELD_W       2
#define GG_FIELD_COMP_U  3  /* Kahan compensation terms (GG_FP32_KAHAN only) */
#define GG_FIELD_COMP_V  4
#define GG_FIELD_COMP_W  5
/* read only: the entries a11, a12, a22 of eq. (2) per cell (for FP32
 * simulations computed in FP64 on read from theta, lambda1, lambda2 and
 * rounded to the destination type) */
#define GG_FIELD_A11     6
#define GG_FIELD_A12     7
#define GG_FIELD_A22     8
/* read only, FP32 simulations only: the coefficients the FP32 kernels read,
 * built once in FP64 and rounded to float (Table 2's weights):
 *   FACE_X(i,j) = (a11(i,j) + a11(i+1,j)) / (2 dx^2), 0 on the last column;
 *   FACE_Y(i,j) = (a22(i,j) + a22(i,j+1)) / (2 dy^2), 0 on the last row;
 *   CROSS(i,j)  = a12(i,j) / (4 dx dy). */
#define GG_FIELD_FACE_X  9
#define GG_FIELD_FACE_Y  10
#define GG_FIELD_CROSS   11

/* ---- gg_params.flags ---- */
#define GG_FLAG_NO_REACTION     1  /* drop U(1-U) - delta U W, rho V(1-V), c(V-W) */
#define GG_FLAG_ALLOW_UNSTABLE  2  /* accept an explicit dt above the stable bound */

typedef struct {
    int32_t nx, ny;   /* cells along x and y, >= 1 */
    double lx, ly;    /* domain [0,lx] x [0,ly]; 0 means 1 (the unit square of Section 2) */
} gg_grid;

typedef struct {
    double delta;          /* aggression rate d of eq. (1), >= 0 */
    double rho;            /* tumour growth rate r, >= 0 */
    double D;              /* tumour diffusion constant alpha, >= 0 */
    double c;              /* acid production/reabsorption rate c, >= 0 */
    double cfl;            /* fraction of dt_max used when dt == 0; 0 means 0.9 */
    double dt;             /* 0: dt = cfl * dt_max; > 0: this dt (checked against dt_max) */
    int32_t precision;     /* GG_FP64_PLAIN, GG_FP32 or GG_FP32_KAHAN */
    int32_t flags;         /* GG_FLAG_* */
    int32_t steps_per_pass;/* time steps per pass over HBM (temporal blocking), 0 = tuned */
    int32_t adapt_every;   /* 0: fixed dt (below); n >= 1: adaptive Delta t_k recomputed
                              on the device every n steps (below); dt must then be 0 */
} gg_params;

/* Stable-step rule (Section 2 recomputes dt for stability without giving a
 * formula; this library's reading):
 *   dt_max = 1 / ( 2 Lambda (1/dx^2 + 1/dy^2) + c + rho + 1 + delta ),
 *   Lambda = max( max over cells of lambda_max(A), D ).
 * It keeps every diagonal coefficient of eq. (3) non-negative and is below
 * h^2 / (4 Lambda) on a square grid.
 *
 * Adaptive step (adapt_every = n >= 1; Section 2's Delta t_k recomputed from
 * the state): at every step k = 0, n, 2n, ... counted from gg_create,
 *   Delta t_k = cfl / max( c + 2 Lambda_A (1/dx^2 + 1/dy^2),
 *                          max over cells of U + delta W - 1,
 *                          max over cells of D S - rho (1 - V) ),
 *   S = sum over the cell's interior faces f of (1 - (U_P + U_nb)/2) / h_f^2,
 *   Lambda_A = max over cells of lambda_max(A),
 * the largest step keeping the coefficient of each unknown's own old value in
 * eq. (3) at least 1 - cfl (the reaction parts are left out with
 * GG_FLAG_NO_REACTION).  It is reduced from the state on the device and read
 * there by the step kernels: no host round trip.  The per-cell terms are
 * evaluated in the state's precision. */

typedef struct {
    double mass[3];      /* dx dy sum of U, V, W (finite values only) */
    double min[3];       /* minima of U, V, W */
    double max[3];       /* maxima of U, V, W */
    int64_t nonfinite;   /* NaN/Inf values over the three fields */
    double tumour_area;  /* dx dy #{V > 1/2} */
    double gap_area;     /* dx dy #{U < gap_eps and V < gap_eps}: interstitial gap of Section 2 */
    double gap_eps;      /* threshold used (input of gg_diagnostics_eps, 0.01 by default) */
} gg_diag;

/* Fronts and the interstitial gap of Section 2 along the four axis rays from
 * one cell (gg_front_rays).  Index d = 0 east (+x), 1 west, 2 north (+y),
 * 3 south; ray d holds the cells k = 0 .. L-1 at k cells from the centre
 * cell (k = 0 is the centre cell itself), h = dx on the east / west rays and
 * dy on the others, distances measured from the centre of cell k = 0. */
typedef struct {
    double front[4];   /* (kT + 1/2) h, kT the farthest cell with V > v_front; 0 if none */
    double edge[4];    /* (kH - 1/2) h, kH the first cell beyond kT with U > u_edge; L if none */
    double gap[4];     /* h times the cells k, kT < k < kH, with U < eps and V < eps */
    double mass_v[4];  /* h sum_k V_k along the ray */
    double mass_u[4];  /* h sum_k U_k along the ray */
} gg_front;

typedef struct gg_sim gg_sim;

/* Create a simulation of eq. (3) on one grid.
 *   theta, lambda1, lambda2: host, nx*ny doubles each; per-cell principal
 *     direction and eigenvalues of A (eq. 2); lambda > 0 required.
 *   u0, v0, w0: host, nx*ny doubles each: initial state at t = 0.
 *   cuda_stream: cudaStream_t to enqueue on (NULL = default stream).
 *   *out receives the new object (NULL on failure).
 * Validates sizes, rates and flags (GG_ERR_ARG), finiteness of all six
 * arrays (GG_ERR_ARG), lambda > 0 (GG_ERR_NOT_SPD) and an explicit dt
 * against dt_max (GG_ERR_CFL unless GG_FLAG_ALLOW_UNSTABLE).  Builds
 * a11, a12, a22 on the device, fixes dt, picks the launch plan.
 * Synchronizes. */
int gg_create(const gg_grid* grid, const gg_params* params,
              const double* theta, const double* lambda1, const double* lambda2,
              const double* u0, const double* v0, const double* w0,
              void* cuda_stream, gg_sim** out);

/* Advance nsteps >= 0 explicit Euler steps of eq. (3) with the fixed dt.
 * Asynchronous: returns once the kernels are enqueued (launch errors are
 * reported as GG_ERR_CUDA). */
int gg_step(gg_sim* sim, int64_t nsteps);

/* Copy one field (GG_FIELD_*) of the current state to dst, nx*ny values in
 * the host layout above.  dst_on_device: 0 host pointer, 1 device pointer.
 * dst_fp64: 1 writes doubles, 0 writes floats.  Synchronizes. */
int gg_read(gg_sim* sim, int32_t field, void* dst, int32_t dst_on_device, int32_t dst_fp64);

/* Overwrite one state field (U, V, W or a compensation field) from src
 * (same conventions as gg_read); used to resume from a checkpoint.
 * Writing U, V or W of a GG_FP32_KAHAN simulation does not touch its
 * compensation terms.  Synchronizes. */
int gg_write(gg_sim* sim, int32_t field, const void* src, int32_t src_on_device, int32_t src_fp64);

/* FP64 diagnostics of the current state: integrals, extrema, non-finite
 * count, tumour and gap areas (gap threshold 0.01).  Synchronizes.
 * Returns GG_ERR_NONFINITE (with *out filled) if the state holds NaN/Inf. */
int gg_diagnostics(gg_sim* sim, gg_diag* out);

/* Same as gg_diagnostics with an explicit gap threshold eps > 0. */
int gg_diagnostics_eps(gg_sim* sim, double eps, gg_diag* out);

/* Front diagnostics of the current state along the four axis rays from cell
 * (i0, j0), 0 <= i0 < nx, 0 <= j0 < ny (normally the centre of the initial
 * tumour): tumour front, healthy-tissue edge, interstitial-gap width and the
 * ray integrals of V and U (gg_front above; thresholds v_front, u_edge, gap
 * threshold eps > 0; 0.5, 0.5 and 0.01 match gg_diagnostics).  *out is a
 * host struct.  Returns GG_OK, GG_ERR_ARG (NULL pointer, centre outside the
 * grid, non-finite threshold, eps <= 0) or GG_ERR_CUDA.  Synchronizes. */
int gg_front_rays(gg_sim* sim, int32_t i0, int32_t j0, double v_front, double u_edge, double eps,
                  gg_front* out);

/* Space-averaged front speed along each ray (the LeVeque-Yee formula): takes
 * gg_front_rays into *before, advances nsteps >= 1 steps (gg_step), takes it
 * into *after, and writes
 *   speed[d] = (after->mass_v[d] - before->mass_v[d]) / (nsteps dt (1 - 0)),
 * the rate of change of the ray integral of V over the jump of V across the
 * front (V = 1 behind it in both invasion regimes of Section 2, V = 0 ahead).
 * before, after: host structs; speed: host, 4 doubles.  Same arguments and
 * status codes as gg_front_rays (GG_ERR_ARG also for nsteps < 1); the
 * simulation is left nsteps steps further.  Synchronizes. */
int gg_front_speed(gg_sim* sim, int32_t i0, int32_t j0, int64_t nsteps, double v_front, double u_edge,
                   double eps, gg_front* before, gg_front* after, double* speed);

/* Discrete adjoint of nsteps steps of eq. (3) starting from the current
 * state X^0 (the transpose of the Jacobian of each step, applied in reverse
 * order; dt is held fixed and not differentiated).
 *   dLdu_N, dLdv_N, dLdw_N: device, nx*ny floats (host layout) holding
 *     dL/d(U,V,W) at step nsteps; NULL means zero.
 *   g_theta, g_lambda1, g_lambda2: device, nx*ny floats: dL/d(theta,
 *     lambda1, lambda2) (chain rule through eq. (2)); may be NULL.
 *   g_u0, g_v0, g_w0: device, nx*ny floats: dL/d(U,V,W) at step 0; may be NULL.
 *   g_scalars: host, 4 doubles: dL/d(delta, rho, D, c); may be NULL.
 *   checkpoint_every: steps between checkpoints (0 = about sqrt(nsteps)).
 * The forward pass stores a checkpoint (the state, with its Kahan terms
 * where the segment is recomputed later) at the start of every segment of
 * checkpoint_every steps; within a segment only the
 * states at even steps are stored, and the reverse pass over a pair of steps
 * rebuilds the state between two stored ones from the earlier (without its
 * Kahan term: it differs from the forward's by its last rounding at most).
 * The stored states of the last segments, as many as fit in 85 % of (this
 * workspace's kept-state buffer + the free device memory), are kept from the
 * forward pass; the others are recomputed from their checkpoints segment by
 * segment (sqrt(N) checkpointing).  The workspace
 * (checkpoints, recompute stash, kept states, adjoint fields) is allocated by
 * the first call, reused by later calls and freed by gg_adjoint_release or
 * gg_destroy.  On return the simulation holds the state at step nsteps, as
 * after gg_step(sim, nsteps).  Not available for GG_FP64_PLAIN
 * (GG_ERR_STATE).  Synchronizes. */
int gg_adjoint(gg_sim* sim, int64_t nsteps,
               const float* dLdu_N, const float* dLdv_N, const float* dLdw_N,
               float* g_theta, float* g_lambda1, float* g_lambda2,
               float* g_u0, float* g_v0, float* g_w0,
               double* g_scalars, int64_t checkpoint_every);

/* Frees the adjoint workspace of sim (a no-op when it has none); the next
 * gg_adjoint allocates it again.  The simulation's state is untouched.
 * Returns GG_OK, or GG_ERR_ARG for a NULL sim.  Synchronizes the device. */
int gg_adjoint_release(gg_sim* sim);

/* Diagnostics without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- code
 * inside a framework whose memory pool owns the device and forbids
 * allocations it does not track, or a time-critical loop that cannot pay for
 * the implicit device-wide synchronisation of cudaMalloc/cudaFree.  It runs
 * the same reduction kernels as gg_diagnostics_eps, on fields the caller
 * already holds:
 *   u, v, w: device, ny rows of `pitch` elements (float, or double when
 *     fp64 != 0), row j starting at element j*pitch, the first nx used (the
 *     padding columns are never read);
 *   dx, dy > 0: cell sizes; eps > 0: gap threshold; *out: host result.
 * Its scratch (608 partial records + 1 result record of 16 doubles, 77,952
 * bytes) is a fixed array in the library's device memory, present on every
 * device that loads the library until the process exits.  Limits: nx, ny >= 1,
 * pitch >= nx and nx*ny <= 2^31 cells; anything else returns GG_ERR_ARG
 * before any device work.  The first call on a device looks up the device
 * address of the scratch array (one cudaGetSymbolAddress, no allocation).
 * All calls share the one array, and every record a call reads is written by
 * that same call, so nothing needs clearing between calls; calls whose work
 * overlaps on the GPU (other streams, other host threads) race on the array
 * and must be serialised by the caller.  The result is copied to the host
 * and cuda_stream is synchronized before the call returns.  Returns GG_OK,
 * GG_ERR_NONFINITE (with *out filled), GG_ERR_ARG or GG_ERR_CUDA (a failed
 * launch or copy of this call; an error left pending by an earlier call is
 * neither reported nor cleared). */
int gg_diagnostics_noalloc(const void* u, const void* v, const void* w, int32_t fp64,
                           int32_t nx, int32_t ny, int32_t pitch, double dx, double dy,
                           double eps, void* cuda_stream, gg_diag* out);

/* Autotuner of the FP32 step: times trial_steps steps (0 means 48) of every
 * candidate launch plan -- the warp-register wavefront with T = 1..4 steps
 * per pass and chunk heights 16..256 rows, the shared-memory wavefront with
 * T in {1, 2, 4, 8} -- on this simulation, keeps the fastest and restores the
 * state it advanced (every plan computes the same bits).  gg_create runs it
 * by itself, once per (nx, ny, precision) and process, when
 * steps_per_pass == 0 and nx*ny >= 2^18.  chosen (may be NULL) receives
 * {T, kernel kind (as gg_plan_info), strip width, chunk height}; the
 * candidates also include the paired-column warp wavefront (kind 3) with
 * T = 1..4 and the same chunk heights.
 * A no-op for GG_FP64_PLAIN.  Synchronizes. */
int gg_autotune(gg_sim* sim, int64_t trial_steps, int32_t* chosen);

/* Choose the launch plan of the FP32 step explicitly: kind 1 = warp-register
 * wavefront (one column per lane, T = 1..4), kind 3 = paired-column warp
 * wavefront (two columns per lane, 64-column strips, T = 1..4), kind 0 =
 * shared-memory wavefront (T = 1..8); strip = output columns per CTA strip
 * (kind 0 only, 0 = default), chunk = rows per chunk (0 = default).  Every
 * plan computes the same bits.
 * GG_ERR_ARG for values out of range, GG_ERR_STATE for GG_FP64_PLAIN. */
int gg_set_plan(gg_sim* sim, int32_t kind, int32_t T, int32_t strip, int32_t chunk);

/* Launch plan in use: info[0..3] = kernel (1 warp-register wavefront,
 * 3 paired-column warp wavefront, 0 shared-memory wavefront, 2 plain FP64),
 * steps per pass T, strip width (written columns), chunk height. */
int gg_plan_info(const gg_sim* sim, int32_t* info);

double gg_dt(const gg_sim* sim);              /* dt of the next step (0 if sim is NULL);
                                                 with the adaptive step it is read from
                                                 the device (synchronizes) */
double gg_time(const gg_sim* sim);            /* simulated time advanced since gg_create:
                                                 steps * dt, or with the adaptive step the
                                                 sum of the Delta t_k taken (synchronizes);
                                                 0 if sim is NULL */
double gg_dt_max(const gg_sim* sim);          /* stable bound dt_max */
int64_t gg_step_count(const gg_sim* sim);     /* steps taken so far */
int32_t gg_steps_per_pass(const gg_sim* sim); /* temporal blocking depth in use */
const char* gg_last_error(const gg_sim* sim); /* text of the last failure ("" if none) */
const char* gg_error_string(int32_t status);  /* static text of a status code */

/* Release the simulation and its device memory (NULL is a no-op).
 * Synchronizes. */
int gg_destroy(gg_sim* sim);

/* ---- ensembles: many independent grids advanced by one persistent launch ---- */

typedef struct gg_batch gg_batch;

/* Create n >= 1 independent simulations, advanced together.
 *   grids[k], params[k]: grid and rates of instance k (precision must be
 *     GG_FP32 or GG_FP32_KAHAN and equal for all instances).
 *   fields: 6*n host pointers, fields[6k + m] = theta, lambda1, lambda2,
 *     u0, v0, w0 of instance k for m = 0..5 (nx*ny doubles each).
 * Validation as in gg_create, per instance.  Synchronizes. */
int gg_batch_create(int32_t n, const gg_grid* grids, const gg_params* params,
                    const double* const* fields, void* cuda_stream, gg_batch** out);

/* Advance every instance nsteps steps with its own dt, in one persistent,
 * cooperative kernel launch that loops over (instance, tile) work items and
 * separates steps by a grid barrier; the launch is captured in a CUDA graph
 * the first time a given nsteps is used and replayed afterwards.  A barrier
 * wait that exceeds its iteration limit sets a device error word and the
 * call returns GG_ERR_TIMEOUT (checked at the next synchronizing call).
 * Asynchronous. */
int gg_batch_step(gg_batch* b, int64_t nsteps);

/* Read field of instance inst (same conventions as gg_read).  Synchronizes;
 * returns GG_ERR_TIMEOUT if a barrier wait of an earlier step gave up. */
int gg_batch_read(gg_batch* b, int32_t inst, int32_t field, void* dst,
                  int32_t dst_on_device, int32_t dst_fp64);

/* Diagnostics of instance inst.  Synchronizes. */
int gg_batch_diagnostics(gg_batch* b, int32_t inst, gg_diag* out);

/* Autotuner of the ensemble launch: times trial_steps steps (>= 1; 0 means
 * 8) of every candidate -- the launch mode (the persistent cooperative
 * kernel with a grid barrier between passes, one launch of one warp per
 * one-column tile per pass, or one launch of one warp per paired-column
 * tile per pass), steps per pass T in {1, 2, 3, 4} and chunk height by in
 * {32, 64, 128, 256} rows (by >= 4T + 8) of the warp tiles, whose strips are
 * 32 - 2T columns wide (one column per lane) or 60 / 56 of 64 (two columns
 * per lane) -- on the batch itself, keeps the fastest, and restores the
 * state it advanced.  chosen (may be NULL) receives {T, strip width, by,
 * threads per CTA (128: persistent mode, 32: a per-pass mode)}; the mode
 * itself is info[7] of gg_batch_launch_info.  Synchronizes. */
int gg_batch_autotune(gg_batch* b, int64_t trial_steps, int32_t* chosen);

/* Sets the ensemble launch plan directly: passes_mode 0 runs the persistent
 * cooperative kernel, 1 one launch per pass (one warp per one-column tile,
 * no grid barrier; a step of at most 4096 passes is captured into one CUDA
 * graph, a longer one is launched directly), 2 the same with the
 * paired-column tiles; T in 1..4 steps per pass; chunk > 0 rows per tile
 * (0 means 64).  Every plan computes the same bits.  Returns GG_OK,
 * GG_ERR_ARG or GG_ERR_OOM / GG_ERR_CUDA.  Synchronizes. */
int gg_batch_set_plan(gg_batch* b, int32_t passes_mode, int32_t T, int32_t chunk);

/* Testing hook for the bounded barrier wait: sets the per-wait time limit
 * (0 < seconds <= 60; 2 s by default) and, with extra_arrivals = 1, makes
 * the grid barrier expect one CTA more than the launch has, so that every
 * wait runs into its limit, sets the device error word and returns (the
 * next synchronizing call reports GG_ERR_TIMEOUT).  extra_arrivals = 0
 * restores normal operation. */
int gg_batch_set_barrier_timeout(gg_batch* b, double seconds, int32_t extra_arrivals);

int32_t gg_batch_steps_per_pass(const gg_batch* b);

/* Launch description of the last gg_batch_step: info[0..7] = steps per pass
 * T, strip width bx, chunk height by, threads per CTA, CTAs of the grid
 * (persistent mode: the persistent grid; passes mode: one per tile), work
 * items (tiles) per pass, 1 if the launch ran as a replayed CUDA graph (0 if
 * it was launched directly), and the mode of the plan (0 persistent, 1 one
 * launch per pass with one-column tiles, 2 with paired-column tiles).
 * info must hold 8 int32. */
int gg_batch_launch_info(const gg_batch* b, int32_t* info);
double gg_batch_dt(const gg_batch* b, int32_t inst);
const char* gg_batch_last_error(const gg_batch* b);
int gg_batch_destroy(gg_batch* b);

/* Arithmetic-rate probe (no counterpart in the paper: it measures the
 * denominators of the ALU rooflines the kernels are reported against).
 * kind 0: FP64 fused multiply-add, 1: FP32 fused multiply-add, 2: packed
 * FP32 pairs (two FMAs per instruction).  Launches `waves` whole waves of
 * 256-thread CTAs (the SM count times the CTAs an SM holds), each thread
 * running 8 independent FMA chains for `iters` iterations, once to warm up
 * and once timed with CUDA events on cuda_stream; *flops_per_s = 2 flops per
 * FMA over the timed launch.  Limits: 1 <= iters <= 2^32, 1 <= waves <= 64;
 * GG_ERR_ARG outside them or for a NULL result, GG_ERR_CUDA on a failed
 * launch or query.  Allocates nothing; synchronizes cuda_stream. */
int gg_probe_fma_rate(int32_t kind, int64_t iters, int32_t waves, void* cuda_stream, double* flops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* GG_H */
