/*
 * fdetd.h - C ABI of the GB300-native exact exponential field solver for
 * cylindrical (azimuthal-mode) particle-in-cell simulations, and of the
 * exponential laser-envelope propagator.
 *
 * Method: "High-order exponential solver method for particle-in-cell simulations
 * in cylindrical geometry" (Majorosi, Hafz, Lecz).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Units c = 1, lengths in laser wavelengths (Sec. 1, normalised units).
 * - Complex azimuthal modes: F(rho, theta, z) = Re sum_m F_m(rho, z) exp(-i m theta),
 *   the complex form of the real (2m, 2m+1) pairs of Sec. 2.1 (Eq. maxwellAM_dtheta).
 * - Radial grids (Eqs. spatialAM_grid, spatialAM_gridR), k = 0..Nr-1:
 *   primary rho_k = (k + 1/2) dr, staggered rho_(-),k = k dr (k = 0 is the axis).
 * - Yee placement (Table tab:spatialAM_boundary): Er, Btheta, Bz on the staggered
 *   radial grid; Etheta, Ez, Br on the primary grid; Ez, Br, Btheta sit at
 *   z = (i - 1/2) dz, the others at z = i dz.  z is periodic with period Nz dz.
 * - Field array of one call: [nmodes][6][Nz][Nr] interleaved complex, components
 *   in the order (Er, Etheta, Ez, Br, Btheta, Bz), r fastest.  complex128 for
 *   FDETD_PREC_FP64, complex64 for every other precision.  Slot k = 0 of Er,
 *   Btheta, Bz is the axis: it is ignored on input and holds the axis value on
 *   output (Sec. 2.4: extrapolated with the order-2N_D coefficients where the
 *   field is constant on the axis - Bz for m = 0, Er and Btheta for m = 1 - and 0
 *   elsewhere).
 * - Current array: [nmodes][3][Nz][Nr] (Jr, Jtheta, Jz) on the Yee locations of
 *   (Er, Etheta, Ez), same complex type as the fields; Jr slot 0 is ignored.
 * - All device pointers must be 16-byte aligned.  A call never frees or keeps a
 *   caller pointer.  `stream` is a cudaStream_t (NULL = legacy default stream).
 *
 * Error handling: every call returns FDETD_OK (0) or one of the FDETD_ERR_*
 * codes; fdetd_last_error() copies a one-line message of the calling thread's
 * last failure.  Argument errors are detected before any work is enqueued.
 * Kernel launches are asynchronous; device-side failures surface at the next
 * synchronising call as FDETD_ERR_CUDA.
 */
#ifndef FDETD_H_
#define FDETD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FDETD_OK = 0,
  FDETD_ERR_ARG = 1,         /* invalid argument (sizes, order, null pointer, misalignment) */
  FDETD_ERR_OOM = 2,         /* device or host allocation failed */
  FDETD_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  FDETD_ERR_EIG = 4,         /* radial eigen-decomposition failed (complex or singular spectrum) */
  FDETD_ERR_UNSUPPORTED = 5, /* valid request the library does not implement (e.g. Nz not a power of 2) */
  FDETD_ERR_TIMEOUT = 6      /* a kernel's bounded pipeline wait expired; it stopped early and freed its resources */
};

/* Arithmetic of the radial transforms (and storage type of the fields). */
enum {
  FDETD_PREC_FP64 = 0,   /* complex128 fields; FP64 everywhere */
  FDETD_PREC_FP32 = 1,   /* complex64 fields; FP32 CUDA-core radial transforms */
  FDETD_PREC_BF16X3 = 2, /* complex64 fields; tcgen05 BF16 2-piece split, 3 products, FP32 accumulate */
  FDETD_PREC_BF16X6 = 3  /* complex64 fields; tcgen05 BF16 3-piece split, 6 products, FP32 accumulate */
};

typedef struct fdetd_plan_s* fdetd_plan_t;
typedef struct fdetd_batch_s* fdetd_batch_t;
typedef struct envelope_plan_s* envelope_plan_t;
typedef struct fdetd_taylor_s* fdetd_taylor_t;

/*
 * fdetd_plan - build the exact exponential step of modes m = 0..M.
 *
 * Defines exp(dt H_m) of the discrete operator of Sec. 2.5 (Eqs.
 * spatialAM_maxwell_Er ... _Bz): staggered finite differences of order `order`
 * (even, 2..32) in z and rho (Eq. spatial_derivativeSt), the parity-dependent
 * axis extensions of Eqs. spatialAM_derivativeS/A, the B_z axis value of
 * Sec. 2.4, taps beyond the outer radius dropped (Sec. 2.2), periodic z.
 * Nz = 64 k in 64..8192 with no prime factor above 7 (FDETD_ERR_UNSUPPORTED otherwise; FP64 takes
 * every power of two and other lengths while the five columns of a family fit in shared memory, about
 * 2500), Nr >= order/2 + 2, M >= 0.  Powers of two whose three field columns do not fit in shared
 * memory (FP64 at 8192) run the z transform in its column-split form: three launches (every column
 * forward in place, the update of every (kz, j) point, every field column back), bitwise the results
 * of the single-pass form; flags & FDETD_FLAG_SPECTRAL_COLUMNS selects that form at any power of two
 * (FDETD_ERR_UNSUPPORTED for other lengths).
 * The radial eigen-decompositions, the omega table and the phase factors are
 * computed in FP64 on the host; device tables are allocated here and owned by
 * the plan.  Blocking; not stream-ordered.
 */
#define FDETD_FLAG_SPECTRAL_COLUMNS 1ull
/* flags & FDETD_FLAG_J_ON_PRIMARY: fdetd_step takes J_rho deposited on the primary radial grid
 * (rho_k = (k + 1/2) dr, like J_theta) and applies the downstagger S_rho^(-, mA) of Eq.
 * spatialAM_staggerS (the J_rho stagger of Eq. spatialAM_filter_Jr, z filter the identity) into a
 * plan-owned copy before the steps of each call: one more launch per call, J itself is not
 * modified; the plan holds a second current-sized device buffer.  fdetd_batch_add refuses such a
 * plan with a current (a batch takes J on the Yee locations; fdetd_current_correct gives them). */
#define FDETD_FLAG_J_ON_PRIMARY 2ull
int fdetd_plan(fdetd_plan_t* out, int Nz, int Nr, int M, int order, double dz, double dr, double dt,
               int precision, uint64_t flags);

/* As fdetd_plan for an explicit list of mode numbers (each 0..64), e.g. {1}. */
int fdetd_plan_modes(fdetd_plan_t* out, int Nz, int Nr, const int* modes, int nmodes, int order,
                     double dz, double dr, double dt, int precision, uint64_t flags);

/*
 * fdetd_step - advance the fields in place by `nsteps` midpoint exponential steps
 * (Eq. maxwellAM_solution2, with the dt factor of the current integral of
 * Eq. maxwellAM_solution):
 *     Psi <- exp(dt H) Psi - dt exp(dt H / 2) J.
 * fields: device, in/out, layout above.  J: device or NULL (J = 0), constant over
 * the nsteps steps and re-consumed in real space every step.  nsteps >= 0.
 * Every step is one real-space round trip: radial projection, z-transform, exact
 * per-(kz, j) rotation with the current term, inverse z-transform, radial
 * back-projection.  Asynchronous on `stream`; uses the plan's scratch buffers,
 * so calls on one plan must not overlap.
 */
int fdetd_step(fdetd_plan_t plan, void* fields, const void* J, int nsteps, void* stream);

/*
 * fdetd_destagger - move the field modes from the Yee grid to the primary grids z_i = i dz,
 * rho_k = (k + 1/2) dr (Sec. 3 field interpolation, Eqs. shapesAM_destagger_E, _B, _Bth), with
 * the upstaggering Lagrange interpolation S^(+) of Eq. spatialAM_staggerS at the plan's order:
 *     E_rho -> S_rho^(+, mA) E_rho,  E_z -> S_z^(+) E_z,  B_rho -> S_z^(+) B_rho,
 *     B_z -> S_rho^(+, mS) B_z,  B_theta -> S_rho^(+, mA) S_z^(+) B_theta,  E_theta copied.
 * z is periodic; radially the axis slot 0 of E_rho, B_theta, B_z must hold the axis value (as
 * fdetd_step writes it), nodes below the axis are mirror images with the symmetric or
 * antisymmetric extension of Eqs. spatialAM_derivativeS/A, nodes past the outer edge are dropped.
 * fields: device, layout and precision of fdetd_step (read only); out: device, same layout, all
 * six fields on the primary grids; must not overlap fields.  Asynchronous on `stream`.
 */
int fdetd_destagger(fdetd_plan_t plan, const void* fields, void* out, void* stream);

/*
 * fdetd_current_correct - the current pipeline in front of fdetd_step (Sec. 2.5 Eqs.
 * spatialAM_filter_Jr/_Jz with the z filters taken as the identity; the planar current correction
 * of Sec. 3, Eqs. shapesAM_currentRHS2m ... shapesAM_currentJth, in the complex mode convention of
 * the field step):
 *     J_rho <- S_rho^(-, mA) J_rho                      (primary -> staggered radial grid)
 *     delta = rho_xy - Div^+ J_rho - (i sigma m / rho) J_theta
 *     [L_rho^(mS) - m^2 rho^-2] phi = delta            (per mode and z row, banded LU)
 *     J_rho += D^- phi,  J_theta += (i sigma m / rho) phi,  J_z unchanged.
 * J: device [modes][3][Nz][Nr] deposited on the primary grids (J_rho, J_theta at (z_i, rho_k), J_z
 * at (z_i - dz/2, rho_k)); rho_xy: device [modes][Nz][Nr], the planar density differential at
 * (z_i, rho_k); both in the plan's complex type.  J_out: device, same layout as J, the corrected
 * current on the Yee locations fdetd_step takes; must not overlap J or rho_xy.  The first call
 * builds the banded operators and LU factors on the host in FP64 and uploads them (FDETD_ERR_EIG if
 * a pivot vanishes); no other device memory is allocated.  Divergence, solve and gradient run in
 * FP64 on FP64 plans and in double-float arithmetic (~46-bit significand) on FP32 plans; the
 * downstagger runs in the data type.  One launch, asynchronous on `stream`.
 * fdetd_current_host_bands (host only): Div^+ and D^- bands [Nr][order+1], LU factors lo [Nr][order/2]
 * and up [Nr][order/2+1] of one mode, from which the device tables are built (layout in
 * csrc/plan_host.cpp).
 */
int fdetd_current_correct(fdetd_plan_t plan, const void* J, const void* rho_xy, void* J_out, void* stream);
int fdetd_current_host_bands(int Nr, int order, double dr, int m, double* divp, double* dm, double* lo, double* up);

/* End-to-end variant with HOST arrays (same layouts): copies fields (and J) to the
 * device, runs fdetd_step, copies the fields back; synchronises `stream`. */
int fdetd_step_host(fdetd_plan_t plan, void* host_fields, const void* host_J, int nsteps, void* stream);

/*
 * fdetd_plan_status - synchronise `stream` and report device-side failures of earlier
 * steps on this plan: FDETD_ERR_CUDA for a CUDA error, FDETD_ERR_TIMEOUT if a
 * tensor-core kernel's bounded mbarrier wait expired (the kernel then skipped its
 * remaining work, drained its own MMAs and released its tensor memory; the output
 * of that step is undefined).  Clears the recorded timeout.
 */
int fdetd_plan_status(fdetd_plan_t plan, void* stream);
/* The same report under the name of the stream-status call: synchronise `stream`, return the plan's
 * device-side failure (FDETD_ERR_TIMEOUT / FDETD_ERR_CUDA) or FDETD_OK. */
int fdetd_stream_status(fdetd_plan_t plan, void* stream);

/*
 * fdetd_plan_set_wait_limit - polls before a bounded mbarrier wait of this plan's
 * tensor-core kernels gives up (polls < 0 restores the default of 2^26; 0 makes every
 * wait give up at once).  A limit of 0 drives the timeout path on a healthy pipeline:
 * the next fdetd_step's kernels stop at their first wait, drain what they issued,
 * release their tensor memory and return, and fdetd_plan_status reports
 * FDETD_ERR_TIMEOUT; the device context stays usable.  FDETD_ERR_UNSUPPORTED for the
 * CUDA-core precisions (they have no pipeline waits).  Takes effect at the next step.
 */
int fdetd_plan_set_wait_limit(fdetd_plan_t plan, long long polls);

/* Bytes of device memory the plan holds (tables + scratch). */
size_t fdetd_plan_device_bytes(fdetd_plan_t plan);

/* Number of kernels one fdetd_step step launches. */
int fdetd_plan_launches_per_step(fdetd_plan_t plan);

/*
 * Per-kernel timing (instrumentation).  While profiling is on, fdetd_step records a
 * CUDA event pair around each of its three kernel stages on the launch stream:
 * 0 = radial projection, 1 = spectral (z transforms + rotation), 2 = radial
 * back-projection.  fdetd_plan_kernel_times synchronises on the recorded events and
 * returns the accumulated milliseconds and launch counts per stage (arrays of 3).
 * Turning profiling on or off resets the accumulators.
 */
int fdetd_plan_set_profiling(fdetd_plan_t plan, int on);
int fdetd_plan_kernel_times(fdetd_plan_t plan, double* ms, long* calls);

/*
 * fdetd_plan_pipeline_waits - pipeline accounting, counted while profiling is on
 * (fdetd_plan_set_profiling(plan, 1) zeroes the counters).  out: 24 unsigned 64-bit SM clock-cycle
 * sums over all CTAs and launches.  out[0..7] the projection and out[8..15] the back-projection
 * (tensor-core plans): [0] CTA residency seen by the MMA-issuing thread, [1] MMA issuer waiting for a
 * stage's A operand (projection: the converted field pieces), [2] waiting for its B operand
 * (back-projection: both operands), [3] waiting for a free TMEM accumulator, [4] producer waiting for
 * a free stage, [5] converters waiting for the staged FP32 tile, [6] converters busy, [7] epilogue
 * busy (TMEM to global).  out[16..23] the spectral kernel specialised on Nz (FP32 data, Nz = 2^k <=
 * 4096): [16] block residency, [17] column loads and first forward stage, [18] other forward stages,
 * [19] last forward stage + update + first inverse stage, [20] other inverse stages, [21] output
 * stage, [22] blocks counted.  Slots a plan's kernels lack stay 0.  Synchronous (device-to-host
 * copy).  fdetd_batch_pipeline_waits reports the tensor-core slots for a batch captured with
 * profiling on (sum over its groups and graph replays; its spectral slots stay 0).
 */
int fdetd_plan_pipeline_waits(fdetd_plan_t plan, unsigned long long* out);

int fdetd_plan_destroy(fdetd_plan_t plan);

/*
 * Tile shapes and schedules of the tensor-core radial transforms (no counterpart in the
 * paper; they change speed, not results: every configuration sums each output over K in
 * the same order, so outputs are bitwise identical).
 *
 * cfg[4] = {N tile of the projection (128 or 256), N tile of the back-projection (128 or
 * 256; 128 for BF16X6; Nz must be a multiple of half of it), tile order of the projection,
 * tile order of the back-projection (0: longest tiles first, round-robin over the persistent
 * CTAs; 1: the same in snake order)}.
 *
 * fdetd_plan_autotune times every valid configuration on the caller's device arrays (fields,
 * J: as for fdetd_step; only read - the back-projection candidates write into a temporary
 * array) on `stream`, keeps the fastest in the plan, and writes the two best times (ms per
 * launch: projection, back-projection) to ms[2] if ms is not NULL.  Blocking (synchronises
 * the stream); allocates a temporary array of the fields' size.  A no-op for the FP64 and
 * FP32 precisions.  fdetd_plan_tile_config reads the plan's configuration and
 * fdetd_plan_set_tile_config sets it (FDETD_ERR_ARG if invalid or not a tensor-core plan).
 */
int fdetd_plan_autotune(fdetd_plan_t plan, const void* fields, const void* J, void* stream, double* ms);
int fdetd_plan_tile_config(fdetd_plan_t plan, int* cfg);
int fdetd_plan_set_tile_config(fdetd_plan_t plan, const int* cfg);

/*
 * fdetd_probe_mma_rounding - diagnostic with no counterpart in the paper: runs one small
 * tcgen05 kind::f16 MMA test on hand-picked bf16 operands (one MMA on K = 0..15, then `reps`
 * (0..64) accumulating MMAs on K = 16..31) and writes 12 rows x 2 columns of FP32 results to
 * host_out[24] (row-major).  The rows are listed at the top of csrc/k_probe.cu; they show the
 * rounding of the tensor core's FP32 accumulation, which the split-BF16 kernels are designed
 * around.  Synchronises `stream`; allocates and frees small device buffers.  Returns
 * FDETD_ERR_UNSUPPORTED on a GPU other than sm_103, FDETD_ERR_TIMEOUT if its bounded wait
 * expired.
 */
int fdetd_probe_mma_rounding(float* host_out, int reps, void* stream);

/*
 * The paper's own time stepper (Sec. 2.5 summary, Eq. maxwellAM_solution2): both exponentials of the
 * midpoint step replaced by N-term Taylor polynomials of the real-space operator H, applied by
 * banded stencils (no radial transform):
 *     Psi <- T_N(h H)^S Psi - dt T_N(h' H)^S' J_state,   T_N(A) = sum_{n<=N} A^n / n!,
 * h = dt / S, h' = (dt / 2) / S', S' = max(1, S / 2), J_state = (J_rho, J_theta, J_z, 0, 0, 0).
 * H is the operator of fdetd_plan (same stencils, axis treatment and periodic z); the result is the
 * exact step only up to the Taylor truncation, and it is stable only for dt small enough that
 * h |H| lies in the Taylor polynomial's stability region.
 *
 * fdetd_taylor_plan: taylor_order N in 2..32, substeps S in 1..1024; modes as for
 * fdetd_plan_modes; FP32 (complex64 fields, same layout as fdetd_step).  Allocates five field-sized
 * work arrays.  fdetd_taylor_step advances `fields` (device) in place by nsteps steps on `stream`;
 * J (device, [modes][3][Nz][Nr]) or NULL is constant over the call (its source term is computed once
 * per call).  The axis slots of E_rho, B_theta, B_z are written from the interior values at the end
 * of the call (Sec. 2.4).  Errors: FDETD_ERR_ARG, FDETD_ERR_OOM, FDETD_ERR_CUDA (fdetd_last_error).
 * fdetd_taylor_launches_per_step = N S term kernels (plus one axis kernel per call).
 * fdetd_taylor_host_bands (host only): the four banded radial operators [4][Nr][order+1] and the axis
 * weights [2][order/2] of mode m, as the kernels use them (layout in csrc/plan_host.cpp).
 */
int fdetd_taylor_plan(fdetd_taylor_t* out, int Nz, int Nr, const int* modes, int nmodes, int order, double dz,
                      double dr, double dt, int taylor_order, int substeps);
int fdetd_taylor_step(fdetd_taylor_t plan, void* fields, const void* J, int nsteps, void* stream);
int fdetd_taylor_launches_per_step(fdetd_taylor_t plan);
int fdetd_taylor_destroy(fdetd_taylor_t plan);
int fdetd_taylor_host_bands(int Nr, int order, double dr, int m, double* bands, double* axis);



/*
 * Batches of uneven instances advanced by one CUDA graph (no counterpart in the paper).
 *
 * fdetd_batch_add registers an instance (a plan with its own device fields and optional J;
 * each plan at most once per batch because its scratch buffers are private to it) and writes
 * its index to *index (may be NULL).
 * fdetd_batch_capture groups the tensor-core instances by precision (up to 64 per group),
 * chooses each group's tile configuration (autotuned on the registered arrays, which it
 * only reads, unless fdetd_batch_set_autotune(batch, 0)), and records `nsteps` steps into
 * one CUDA graph: per step one persistent grouped projection launch and one grouped
 * back-projection launch per group, covering every (instance, mode, z tile, output tile) of
 * the group, with each instance's spectral kernel on its own graph branch in between;
 * instances on the CUDA-core precisions run their own step sequence on concurrent
 * branches.  Blocking before the capture (tile tables, tuning); fdetd_batch_launch replays
 * the graph on `stream`.  Re-capture after adding instances.  The registered pointers must
 * stay valid while the graph is launched.
 * fdetd_batch_group_info(batch, g, info[7], ms[2]) reports group g after a capture: info =
 * {N tile of the projection, N tile of the back-projection, projection tile order,
 * back-projection tile order, instances, projection tiles, back-projection tiles}, ms = the
 * tuned times per launch (0 when not tuned); returns the number of groups (0 if none; info
 * is left untouched when g is out of range), or -FDETD_ERR_ARG for a NULL batch or info.
 *
 * Stage timing: fdetd_batch_set_profiling(batch, 1) before fdetd_batch_capture records CUDA
 * events into the graph around each captured step's grouped projections, the join of the
 * spectral branches and the grouped back-projections (setting it drops the captured graph).
 * After a replay has completed (the caller synchronizes), fdetd_batch_collect_stage_times
 * adds that replay's three stage times to running sums, which fdetd_batch_stage_times copies
 * to ms[3] (projection, spectral, back-projection, milliseconds) with the number of steps
 * summed in *steps (may be NULL).
 *
 * fdetd_batch_step_host(batch, host_fields, host_J, nlaunch, stream): the batch with host
 * buffers.  host_fields[k] / host_J[k] are instance k's fields and current in host memory, in
 * the layouts of fdetd_step (pinned memory gives asynchronous copies); host_J may be NULL when
 * no instance was added with a current.  Copies every instance's inputs to the registered device
 * buffers, advances every instance by nlaunch times the captured steps, copies the fields back into
 * host_fields, and synchronizes `stream` before returning.  FDETD_ERR_ARG for a missing graph or
 * buffer.  Copies and compute overlap: the instances are split into up to
 * fdetd_batch_set_host_pipeline(batch, parts) contiguous parts of about equal bytes (default 16; 1
 * gives the serial form: all copies in, the main graph, all copies out), each with a one-step graph
 * of its own (built at the first call with the main capture's tile shapes; results bitwise equal to
 * the main graph's); part p's inputs are copied in on an internal stream, its graph runs on `stream`
 * once they have landed, and its fields are copied out on a second internal stream while the next
 * part computes.  The batch's graphs share the plans' scratch: do not run them concurrently.
 */
int fdetd_batch_create(fdetd_batch_t* out);
int fdetd_batch_add(fdetd_batch_t batch, fdetd_plan_t plan, void* fields, const void* J, int* index);
int fdetd_batch_set_autotune(fdetd_batch_t batch, int on);
int fdetd_batch_capture(fdetd_batch_t batch, int nsteps, void* stream);
int fdetd_batch_group_info(fdetd_batch_t batch, int group, int* info, double* ms);
int fdetd_batch_launch(fdetd_batch_t batch, void* stream);
int fdetd_batch_set_profiling(fdetd_batch_t batch, int on);
int fdetd_batch_collect_stage_times(fdetd_batch_t batch);
int fdetd_batch_pipeline_waits(fdetd_batch_t batch, unsigned long long* out);
int fdetd_batch_stage_times(fdetd_batch_t batch, double* ms, long* steps);
int fdetd_batch_set_host_pipeline(fdetd_batch_t batch, int parts);
/* Host only: the split the host-buffer step uses.  n items of bytes[k] into at most `parts` contiguous
 * parts: part p closes at the first item where the running size reaches (p + 1) / P of the total, P =
 * min(parts, n), the last part takes the rest.  part_of[k] = part of item k; returns the number of
 * parts, or -FDETD_ERR_ARG. */
int fdetd_host_split_parts(const size_t* bytes, int n, int parts, int* part_of);
int fdetd_batch_step_host(fdetd_batch_t batch, void* const* host_fields, const void* const* host_J, int nlaunch,
                          void* stream);
int fdetd_batch_destroy(fdetd_batch_t batch);

/*
 * Continuous-batching request server (no counterpart in the paper).
 *
 * fdetd_server_create(out, hbm_budget_bytes, chunk_steps, plan_threads, flags) starts a server
 * with one scheduler thread and plan_threads plan-builder threads on the calling thread's current
 * device.  A submitted request is admitted first-come first-served as soon as its device
 * footprint (fdetd_request_device_bytes) fits the budget next to the requests already admitted
 * (later requests never overtake a waiting one); a request larger than the whole budget is
 * refused at submission with FDETD_ERR_OOM.  Admitted requests get their plan built on a builder
 * thread and their state copied to the device, then stay resident until they finish.  All ready
 * field requests advance together as the instances of one batch (fdetd_batch_*: one CUDA graph per
 * step with grouped tensor-core launches), re-captured whenever a request joins or leaves and
 * replayed in chunks of at most chunk_steps steps, never past the end of the shortest request;
 * envelope requests advance chunk by chunk on their own streams, overlapping with the field
 * batch.  A finished request's result is copied to its host `out` buffer and its device memory
 * returned to the budget.  flags: FDETD_SERVER_DRY_RUN makes no CUDA call at all (plans are
 * only checked on the host, a chunk takes 0.1 ms of host time per step, no result is written):
 * the scheduling can then be exercised on machines without a GPU.
 *
 * fdetd_server_submit(server, request, &ticket): the request is copied (its modes array too);
 * the host buffers it points to (fields or the envelope state, J, chi, out) must stay valid
 * until the ticket is done or failed.  Field request: fields/out = [nmodes][6][Nz][Nr] in the
 * layout and complex type of fdetd_step, J = [nmodes][3][Nz][Nr] or NULL.  Envelope request:
 * fields/out = [2][Nz][Nr] complex64 (a, a~), chi = [Nz][Nr] float.  out may be NULL (no copy
 * back) or equal to fields.
 * fdetd_server_poll(server, ticket, &state, &latency_s): state = FDETD_TICKET_*; latency_s =
 * completion - submission time in seconds once done (else -1); returns the request's error
 * code (with its message in fdetd_last_error) for a failed request.
 * fdetd_server_wait(server, ticket, timeout_s, &latency_s): blocks until the ticket is done or
 * failed, or FDETD_ERR_TIMEOUT after timeout_s.
 * fdetd_server_ticket_times(server, ticket, times[3]): submission, admission and completion
 * times (seconds on a monotonic clock; 0 where not reached yet).
 * fdetd_server_stats(server, &stats): budget, bytes in use and their peak, request counts,
 * graph re-captures, scheduling rounds, served cell*mode*steps.
 * fdetd_server_cancel_queued(server, &n): requests still waiting for admission end as failed
 * ("cancelled before admission"); admitted ones run to completion; n = how many (may be NULL).
 * fdetd_server_destroy(server): stops accepting requests, finishes every request already
 * submitted, then joins the threads and frees everything.
 */
enum { FDETD_REQUEST_FIELD = 0, FDETD_REQUEST_ENVELOPE = 1 };
enum {
  FDETD_TICKET_QUEUED = 0,   /* waiting for budget */
  FDETD_TICKET_ADMITTED = 1, /* budget reserved, plan under construction */
  FDETD_TICKET_RUNNING = 2,  /* resident on the device */
  FDETD_TICKET_DONE = 3,
  FDETD_TICKET_FAILED = 4
};
#define FDETD_SERVER_DRY_RUN 1ull

typedef struct {
  int kind;                 /* FDETD_REQUEST_FIELD or FDETD_REQUEST_ENVELOPE */
  int Nz, Nr;
  int nmodes;               /* field: number of modes in `modes` */
  const int* modes;         /* field: the azimuthal modes */
  int order;                /* finite-difference order */
  int precision;            /* field: FDETD_PREC_* */
  int taylor_order;         /* envelope: N_T */
  int steps;                /* time steps to advance */
  double dz, dr, dt, k0;    /* k0: envelope carrier wave number */
  const void* fields;       /* host input state */
  const void* J;            /* field: host current or NULL */
  const float* chi;         /* envelope: host susceptibility */
  void* out;                /* host result buffer or NULL */
} fdetd_request;

typedef struct {
  size_t budget_bytes, used_bytes, peak_bytes;
  size_t queued, building, running;
  uint64_t completed, failed, recaptures, rounds;
  double served_cell_steps;
} fdetd_server_stats_t;

typedef struct fdetd_server_s* fdetd_server_t;

size_t fdetd_request_device_bytes(const fdetd_request* request);
int fdetd_server_create(fdetd_server_t* out, size_t hbm_budget_bytes, int chunk_steps, int plan_threads,
                        uint64_t flags);
int fdetd_server_submit(fdetd_server_t server, const fdetd_request* request, uint64_t* ticket);
int fdetd_server_poll(fdetd_server_t server, uint64_t ticket, int* state, double* latency_s);
int fdetd_server_wait(fdetd_server_t server, uint64_t ticket, double timeout_s, double* latency_s);
int fdetd_server_ticket_times(fdetd_server_t server, uint64_t ticket, double* times);
int fdetd_server_stats(fdetd_server_t server, fdetd_server_stats_t* stats);
int fdetd_server_cancel_queued(fdetd_server_t server, uint64_t* cancelled);
int fdetd_server_destroy(fdetd_server_t server);

/*
 * fdetd_host_tables - host-only (no GPU needed) export of the FP64 plan tables of
 * one mode, for inspection and CPU tests.  Any output pointer may be NULL.
 * PE, PB, QE, QB: (3 Nr)^2 row-major each.  Rows/cols of PE (cols) and QE (rows)
 * are the field blocks (Er, tau Etheta, Ez), of PB (cols) and QB (rows) the blocks
 * (Btheta, tau Br, tau Bz), tau = -i; the other index runs over the coefficient
 * blocks (e, a, tau c) / (b, tau d, tau f).  lam, mu: Nr each; tm_live, te_live: Nr
 * bytes; kappa2: Nz; sp, sm: 2 Nz (re, im) - the DFT symbols of D_z^(+), D_z^(-).
 */
int fdetd_host_tables(int Nz, int Nr, int m, int order, double dz, double dr, double dt, double* PE,
                      double* PB, double* QE, double* QB, double* lam, double* mu, uint8_t* tm_live,
                      uint8_t* te_live, double* kappa2, double* sp, double* sm);

/*
 * fdetd_plan_cache_set_limit / fdetd_plan_cache_stats - the process-wide cache of per-mode radial
 * tables.  A mode's radial eigenbases and projection matrices (Sec. 2.5 operator, Sec. 2.4 axis rule)
 * depend on (Nr, order, dr, m) only, so every plan construction (fdetd_plan, fdetd_plan_modes, the
 * server's builders, fdetd_host_tables) looks them up there first and skips the eigen-decompositions on
 * a hit; the tables are bitwise the same either way.  The cache lives in host memory, is thread-safe
 * and evicts least recently used entries above `bytes` (default 4 GiB; 0 empties and disables it; an
 * entry is 4 (3 Nr)^2 doubles, about 75 MB at Nr = 512).  Stats: bytes held, the limit, entries, and
 * the hit and miss counts since the process started; any pointer may be NULL.  Both return FDETD_OK.
 */
int fdetd_plan_cache_set_limit(size_t bytes);
/* Computes the tables of `modes` for a radial grid (Nr, order, dr) into the cache unless they are there
 * (a server precomputing the grids it expects); host only, thread-safe.  FDETD_ERR_ARG for invalid
 * arguments, FDETD_ERR_EIG if an eigen-decomposition fails. */
int fdetd_plan_cache_warm(int Nr, int order, double dr, const int* modes, int nmodes);
int fdetd_plan_cache_stats(size_t* bytes, size_t* limit, int* entries, uint64_t* hits, uint64_t* misses);

/* Host only: builds the host tables of a multi-mode plan (the modes' radial eigenbases in parallel, as a plan
 * does) and writes per mode the left-to-right sums of PE, PB, QE, QB, lambda and mu to digest[6 i .. 6 i + 5],
 * for checking the parallel build against single-mode fdetd_host_tables.  FDETD_ERR_ARG / FDETD_ERR_EIG as
 * fdetd_plan. */
int fdetd_host_plan_digest(int Nz, int Nr, const int* modes, int nmodes, int order, double dz, double dr, double dt,
                           double* digest);

/* Host-only: staggered (kind 0), centred first (1), centred second (2, e0 first) derivative
 * coefficients of `order`, or axis coefficients (3, N = order/2); returns the count written. */
int fdetd_host_coeffs(int kind, int order, double* out);

/*
 * fdetd_host_spectral_order - host-only: the order in which the spectral kernel stores its per-kz
 * tables (phase records and z symbols).  Its in-place z transform (decimation in frequency with the
 * stage radices of fdetd_host_spectral_radices) leaves kz in mixed-radix digit-reversed order; the
 * record of output position b * RL + r (RL the last stage's radix) sits at table index
 * r * (Nz / RL) + b.  kz: Nz ints, kz[i] = the kz index of table entry i.  precision: FDETD_PREC_*.
 * FDETD_ERR_ARG unless Nz >= 2 has no prime factor above 7 and kz is non-null.
 *
 * fdetd_host_spectral_radices - host-only: the stage radices of the z transform, first to last, in
 * rad[0..15]: for Nz = 2^a the leftover factor 2^(a mod 3) (FP64: 2^(a mod 2)) first when it is not 1,
 * then radix 8 (FP64: 4); for other 7-smooth Nz the factors 7, 5, 3 first, then the power-of-two part
 * the same way.  Returns the number of stages, 0 when Nz has a prime factor above 7, -FDETD_ERR_ARG for
 * a null rad or Nz < 2.
 */
int fdetd_host_spectral_order(int Nz, int precision, int* kz);
int fdetd_host_spectral_radices(int Nz, int precision, int* rad);

/*
 * envelope_plan - exponential laser-envelope propagator of Sec. 4.2, mode m = 0:
 *     da/dt = a~,  da~/dt = (L_rho + L_z - chi) a + 2 i k0 D_z^(C) a + 2 i k0 a~
 * (complex form of Eq. spatialAM_envelope_H; L_rho = D^2_rho + rho^-1 D^(C)_rho with
 * the symmetric axis mirror, Eq. spatialAM_laplaceR; centred differences of order
 * `order` (even, 2..16); periodic z; primary radial grid).  One step applies the
 * truncated Taylor series sum_{n <= taylor_order} (dt H_a)^n / n!
 * (Eq. laserA_envelope_solution), taylor_order 1..16.  Nz >= 2*order, Nr >= order/2+1.
 */
int envelope_plan(envelope_plan_t* out, int Nz, int Nr, int order, int taylor_order, double dz, double dr,
                  double dt, double k0);

/*
 * envelope_step - advance psi_a = (a, a~) in place by nsteps Taylor steps.
 * a: device [2][Nz][Nr] complex64 (a then a~).  chi: device [Nz][Nr] float32,
 * frozen over the call (the mid-step value of Sec. 4.2).  Asynchronous on
 * `stream`; uses the plan's scratch, so calls on one plan must not overlap.
 * One launch per Taylor term.
 *
 * envelope_step_fused - the same step with every Taylor term in one launch (order 8,
 * taylor_order 4, Nz a multiple of 32; FDETD_ERR_UNSUPPORTED otherwise): each tile
 * chains its terms in shared memory, recomputing a halo of N_T order/2 cells; the
 * state alternates between `a` and a plan buffer and ends in `a` (one device copy
 * when nsteps is odd).  Per cell it does the arithmetic of envelope_step, so both
 * give identical bits.  It saves the term-by-term DRAM round trips when the state
 * does not stay in L2 between the term launches, at the cost of the halo work.
 */
int envelope_step(envelope_plan_t plan, void* a, const float* chi, int nsteps, void* stream);
int envelope_step_fused(envelope_plan_t plan, void* a, const float* chi, int nsteps, void* stream);

/*
 * envelope_step_static - the envelope step for callers that cannot allocate device memory
 * (no counterpart in the paper; same mathematics and layouts as envelope_step).
 *
 * Who needs it: applications whose device memory is entirely pre-reserved by their own pool
 * or arena, plugins whose host framework owns every allocation, and latency-critical loops
 * that cannot afford the implicit synchronisation of an allocation.  It takes no plan and
 * allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 *
 * a: device [2][Nz][Nr] complex64 (a, a~), advanced in place; chi: device [Nz][Nr] float32.
 * order (even, 2..32), taylor_order (1..16), dz, dr, dt, k0 as in envelope_plan.
 * Limit: Nz * Nr <= 1048576 (2^20 cells); larger grids return FDETD_ERR_ARG.
 * Scratch: one file-scope device array of 4 * 2^20 complex64 values (32 MiB), held by every
 * GPU that loads the library until the process exits.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress, with the device current) and caches it;
 * make that first call before any stream capture.  All calls share the array and each call
 * overwrites it before reading it (no state carries over, nothing needs clearing), so calls
 * whose kernels overlap on the GPU - on different streams, or on one device from several
 * threads without ordering - race on it and must be serialised by the caller.
 * Asynchronous on `stream`; returns FDETD_OK, FDETD_ERR_ARG or FDETD_ERR_CUDA (this entry
 * point does not set fdetd_last_error).
 */
int envelope_step_static(void* a, const float* chi, int Nz, int Nr, int order, int taylor_order, double dz,
                         double dr, double dt, double k0, int nsteps, void* stream);

/* Number of kernels one envelope step launches. */
size_t envelope_plan_device_bytes(envelope_plan_t plan);  /* device bytes the plan holds */
int envelope_plan_launches_per_step(envelope_plan_t plan);

/*
 * envelope_step_absorbing - the envelope step with the scalar absorbing layer of the appendix
 * (Eqs. absorbingA_Adt, absorbingA_waveA with h = 1, absorbingA_solution2): per step
 *     (a, a~) <- exp(-sigma dt / 4) T_N(dt H_a[chi + sigma^2]) exp(-sigma dt / 4) (a, a~),
 * the damping pointwise on both components and the absorbing term sigma^2 merged into the
 * susceptibility.  sigma: device, [Nz][Nr] float32, >= 0 (zero outside the layers); other
 * arguments as envelope_step.  sigma = 0 gives envelope_step exactly.
 */
int envelope_step_absorbing(envelope_plan_t plan, void* a, const float* chi, const float* sigma, int nsteps,
                            void* stream);


int envelope_plan_destroy(envelope_plan_t plan);

/* Copies the calling thread's last error message (NUL-terminated, truncated to len). */
int fdetd_last_error(char* buf, size_t len);

#ifdef __cplusplus
}
#endif
#endif /* FDETD_H_ */
