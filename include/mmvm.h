/*
 * mmvm.h - C ABI of the GB300 multi-moment vortex method (MMVM) library.
 *
 * The library evaluates and integrates the moment ODE of Uminsky, Wayne &
 * Barbaro, "A multi-moment vortex method for 2D viscous fluids"
 * (arXiv:1010.2475):
 *
 *   omega(x,t) = sum_j sum_{|k|<=M} M^j[k1,k2](t) D^k phi_00(x - x^j(t); lambda(t))
 *       (eq:vorticity_decomposition, eq:moment_expansion_def_tw0)
 *   phi_00(x; lambda) = exp(-|x|^2/lambda^2) / (pi lambda^2),
 *   lambda(t)^2 = lambda_0^2 + 4 nu t                        (eq:phi00)
 *   dM^j_k/dt = A + B + C                                  (eq:Final_CrossCoef)
 *   dx^j/dt from eq:xjdot_Final (the self pair excluded, eq:xjdot)
 *
 * Conventions shared by every entry point:
 *  - n particles, truncation order M (k1 + k2 <= M), K = (M+1)(M+2)/2.
 *  - Positions x: n x 2 float64, row-major (x^j_1, x^j_2).
 *  - Moments: n x K float64, row-major; moment (k1,k2) of particle j sits at
 *    column q(k1+k2) + k2 with q(s) = s(s+1)/2 (grouped by total order, then by
 *    k2).  Column 0 is the circulation M^j[0,0], which must be nonzero for
 *    every particle (eq:mass).
 *  - The separation between particles is s_{j,j'} = x^j - x^{j'} (eq:xjdotA).
 *  - All particles share one core size lambda (the sqrt(2) lambda kernel of
 *    eq:Fullint needs equal cores); viscosity enters only through lambda(t).
 *  - Host pointers are read or written synchronously before the call
 *    returns.  "Device" pointers are CUDA global-memory pointers on the
 *    context's device; such calls are ordered on the context's stream and
 *    return before the GPU work ends (use mmvm_synchronize).
 *  - Return value: 0 (MMVM_OK), a positive value (MMVM_PENDING) or a negative
 *    error code below; mmvm_last_error() gives a message for the calling
 *    thread's last failure.
 *  - A context is not thread-safe: one thread at a time per context.
 */
#ifndef MMVM_H_
#define MMVM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MMVM_OK 0
#define MMVM_PENDING 1
#define MMVM_E_INVALID_ARG (-1)       /* null pointer, bad size, bad enum       */
#define MMVM_E_ZERO_CIRCULATION (-2)  /* some M^j[0,0] == 0 (eq:mass)           */
#define MMVM_E_UNSUPPORTED (-3)       /* order above the compiled limit         */
#define MMVM_E_OOM (-4)               /* device allocation failed / over budget */
/* A served request whose footprint exceeds the server's whole HBM budget is
 * refused at admission with this same code (mmvm_submit).                   */
#define MMVM_E_ADMISSION MMVM_E_OOM
#define MMVM_E_NUMERIC (-5)           /* non-finite value in the state          */
#define MMVM_E_TIMEOUT (-6)           /* a bounded device wait ran out          */
#define MMVM_E_DEVICE (-7)            /* CUDA runtime error                     */

/* Arithmetic of the pair interaction (the all-pairs part of A, B and C).
 * Coefficient tables, the state, RK4, the centroid and circulation sums and
 * the per-particle finish are FP64 in every mode.                           */
#define MMVM_FP64 0        /* pair jets and contractions in FP64              */
#define MMVM_MIXED_FP32 1  /* pair jets and contractions in FP32, sums of
                              source tiles carried as FP32 (hi, lo) pairs     */

/* Largest order of the all-pairs kernels (jets of order 3M).  Single
 * particles (n == 1) accept any order up to MMVM_MAX_ORDER_SINGLE.          */
#define MMVM_MAX_ORDER_PAIRS 8
#define MMVM_MAX_ORDER_SINGLE 64

/* mmvm_config.flags bits.  In MMVM_MIXED_FP32 mode the particles are put in
 * spatial (Morton) order every step and tile pairs whose bounding boxes are
 * far enough apart that the Gaussian part of the pair jet is below FP32
 * rounding take the point-vortex jet (far field); this flag turns that off
 * (every pair takes the full jet).  MMVM_FP64 never uses the far field.     */
#define MMVM_FLAG_NO_FAR_FIELD 1u
/* Single particle: evaluate the self term by the separable route (the
 * coefficient sums of eq:FinalSingleI/II taken one index at a time, no
 * (k, l, beta) table); always used above order 16, this flag forces it at
 * any order (n must then be 1).                                            */
#define MMVM_FLAG_SEPARABLE_SELF 2u

typedef struct mmvm_config {
  int32_t order;        /* truncation order M >= 0                            */
  int32_t precision;    /* MMVM_FP64 or MMVM_MIXED_FP32                       */
  double lambda0;       /* core size lambda_0 > 0 at t = 0 (eq:phi00)        */
  double nu;            /* kinematic viscosity >= 0 (Re = Gamma_ref / nu)     */
  int32_t device;       /* CUDA device ordinal                                */
  uint32_t flags;       /* MMVM_FLAG_* bits, other bits must be 0             */
} mmvm_config;

typedef struct mmvm_ctx mmvm_ctx;

/* Create a context on cfg->device for one instance of the problem of
 * Section 2 of the paper: particles of order M sharing the core lambda(t)
 * with lambda(0) = lambda0 and viscosity nu (eq:phi00; the particle centres
 * and moments come with mmvm_set_state).  *out receives the handle; the
 * caller destroys it with mmvm_destroy.  Errors: INVALID_ARG, UNSUPPORTED,
 * DEVICE.                                                                    */
int mmvm_create(const mmvm_config* cfg, mmvm_ctx** out);

/* Release every device buffer of the context.  NULL is ignored.             */
void mmvm_destroy(mmvm_ctx* ctx);

/* Load a state from HOST memory: n particles, x (n x 2), moments (n x K),
 * time t.  The library copies the data into device memory it owns (buffers
 * grow as needed).  Errors: INVALID_ARG (n < 1, null pointers),
 * ZERO_CIRCULATION, NUMERIC (NaN/Inf), UNSUPPORTED (n > 1 with
 * order > MMVM_MAX_ORDER_PAIRS), OOM, DEVICE.                               */
int mmvm_set_state(mmvm_ctx* ctx, int64_t n, const double* x, const double* moments,
                   double t);

/* Same, from DEVICE pointers: copied device-to-device on the context stream,
 * and the call waits for the copy, so the caller may reuse its buffers when
 * it returns.  The zero-circulation and finiteness checks are not made.     */
int mmvm_set_state_device(mmvm_ctx* ctx, int64_t n, const double* d_x,
                          const double* d_moments, double t);

/* Copy the current state to HOST memory (x: n x 2, moments: n x K, *t).
 * Any of the three pointers may be NULL to skip it.  Synchronises.          */
int mmvm_get_state(mmvm_ctx* ctx, double* x, double* moments, double* t);

/* Copy the current state to DEVICE memory (asynchronous on the stream).      */
int mmvm_get_state_device(mmvm_ctx* ctx, double* d_x, double* d_moments);

/* Right-hand side at the current state (eq:Final_CrossCoef, eq:xjdot_Final):
 * dxdt (n x 2) and dMdt (n x K) written to HOST memory.  Synchronises.      */
int mmvm_rhs(mmvm_ctx* ctx, double* dxdt, double* dMdt);

/* Right-hand side written to DEVICE memory (asynchronous on the stream).     */
int mmvm_rhs_device(mmvm_ctx* ctx, double* d_dxdt, double* d_dMdt);

/* Advance the state by nsteps classic RK4 steps of size dt, lambda evaluated
 * at the stage times (eq:phi00), each stage one right-hand side of
 * eq:Final_CrossCoef / eq:xjdot_Final.  Classic RK4 is not from the paper:
 * it is the fixed-step integrator of the benchmark configurations; the
 * paper integrates with an adaptive embedded pair (Section 4.3), which is
 * mmvm_integrate.  Asynchronous on the context stream (the steps are
 * replayed from a CUDA graph); mmvm_get_state or mmvm_synchronize waits.     */
int mmvm_step(mmvm_ctx* ctx, double dt, int64_t nsteps);

/* Use this CUDA stream (a cudaStream_t, NULL = the context's own stream).    */
int mmvm_set_stream(mmvm_ctx* ctx, void* stream);

/* Wait for the context's queued work; reports asynchronous device errors.    */
int mmvm_synchronize(mmvm_ctx* ctx);

/* Number of particles, order, moments per particle of the loaded state.      */
int64_t mmvm_num_particles(const mmvm_ctx* ctx);
int32_t mmvm_num_moments(int32_t order);

/* Kernel launches issued by this context since creation (for accounting).   */
int64_t mmvm_launch_count(const mmvm_ctx* ctx);

/* Kernel timing.  mmvm_enable_timing(ctx, 1) makes every later right-hand
 * side (also inside mmvm_step, whose steps are then launched directly rather
 * than replayed from the graph) record CUDA events around its all-pairs
 * launch on the context stream.  mmvm_pair_time(ctx, &ms, &count) waits for
 * the stream and returns the summed device time (ms) and number of all-pairs
 * launches since the previous call; only the launches of the last right-hand
 * side or step are kept, so call it after each one.                         */
int mmvm_enable_timing(mmvm_ctx* ctx, int on);
int mmvm_pair_time(mmvm_ctx* ctx, double* ms, int64_t* count);

/* The same time split by kernel for the list form (the all-pairs variants
 * with mmvm_pair_config out[6] > 0): ms[0] the list build and the tree,
 * ms[1] the far-field kernel, ms[2 ..] each near kernel; summed over the
 * right-hand sides that mmvm_pair_time has read since the previous call of
 * this function (*count of them), *nparts = 2 + near kernels (0 for the
 * direct form).  ms must hold max_parts values.                             */
int mmvm_pair_time_parts(mmvm_ctx* ctx, double* ms, int32_t max_parts, int32_t* nparts,
                         int64_t* count);

/* All-pairs kernel configuration in use for the loaded state, out[0..7]:
 *  [0] variant index: 0 .. nv-1 the direct form (source tiles shared by the
 *      target groups of a CTA), nv .. nv+nl-1 the interaction-list form
 *      (MMVM_MIXED_FP32 with the far field only: near lists per target
 *      group, near pairs with all warps of a CTA on one target group, a
 *      separate far-field kernel);
 *  [1] kernels per evaluation (order slices or column parts; the list form
 *      counts its list build and far kernel too);
 *  [2] targets per CTA (list form: threads per CTA of its first near kernel);
 *  [3] CTAs per SM;  [4] sources between CTA barriers (0: none);
 *  [5] source chunks (list form: list segments per target group);
 *  [6] 1 for the list form, else 0;  [7] source ranges of its far kernel.
 * The variant is chosen by timing the compiled variants for the first state
 * of each size class (environment: MMVM_PAIR_VARIANT=<v> forces one,
 * MMVM_AUTOTUNE=0 keeps variant 0).  out must hold 8 values.              */
int mmvm_pair_config(const mmvm_ctx* ctx, int32_t* out);

/* Compiled all-pairs variants of (order, precision): *direct variants of the
 * direct form (numbers 0 .. *direct-1) and *list variants of the list form
 * (numbers *direct .. *direct + *list - 1; MMVM_MIXED_FP32 with the far field
 * only, else 0).  Host-only.  Errors: INVALID_ARG.                          */
int mmvm_pair_variant_counts(int32_t order, int32_t precision, int32_t* direct, int32_t* list);

/* Cumulative counts of ordered pairs the all-pairs kernel evaluated since the
 * context was created, by path: full jet (near) and point-vortex jet (far,
 * MMVM_MIXED_FP32 only, source by source or through tile expansions).  The
 * self pair and the tuning launches are not counted.  Waits for the context
 * stream.                                                                   */
int mmvm_pair_counts(mmvm_ctx* ctx, int64_t* near_pairs, int64_t* far_pairs);

/* The same work in detail, out[4]: near pairs, far pairs evaluated source by
 * source, tile expansions evaluated (one per target and far tile summed
 * about the tile centre), pairs those expansions covered.                   */
int mmvm_pair_work(mmvm_ctx* ctx, int64_t* out);

/* Right-hand side without any device allocation.  The paper has no
 * counterpart: this is a variant of mmvm_rhs_device for callers that cannot
 * call cudaMalloc (an application that owns all device memory through its own
 * pool or budget, a latency-critical path on which cudaMalloc/cudaFree would
 * synchronise the device, a plugin whose host forbids allocation at run time).
 *
 * Computes dx/dt and dM/dt of the state (d_x: n x 2, d_moments: n x K, both
 * device memory, row-major FP64, column order as mmvm_set_state) at time t,
 * with the order, precision, lambda0 and nu of *cfg (cfg->device and
 * cfg->flags are ignored: the current device is used and the far field is
 * off), into the caller's device buffers d_dxdt (n x 2) and d_dMdt (n x K).
 * stream: a cudaStream_t (NULL: the legacy default stream); the call is
 * asynchronous on it, except that the first call on a device, and the first
 * call after a change of order, upload the coefficient tables and wait for
 * them (that call also waits for the whole device when it replaces the tables
 * of another order); make such calls before any stream capture.
 *
 * All scratch lives in one fixed array of 12 MiB (12,583,168 bytes) of
 * device memory per GPU that loads the library, held until the process exits.  Limits: 1 <= n <=
 * 4096 and order <= 8, else MMVM_E_UNSUPPORTED with a message; nothing is
 * allocated (no cudaMalloc, cudaFree or allocating library call).  Every call
 * shares that array, so calls whose work overlaps on the GPU (different
 * streams or host threads) race; serialise them.  Errors: MMVM_E_INVALID_ARG
 * (null pointer, bad precision, lambda0 <= 0, nu < 0, non-finite t),
 * MMVM_E_DEVICE (CUDA error).  Inputs are not scanned for non-finite values
 * or zero circulation.                                                      */
int mmvm_rhs_noalloc(const mmvm_config* cfg, int64_t n, double t, const double* d_x,
                     const double* d_moments, double* d_dxdt, double* d_dMdt, void* stream);

/* Adaptive integration of the loaded state from the context's current time
 * to t_end (>= it) with the Dormand-Prince 5(4) pair (the paper integrates
 * with an adaptive embedded Runge-Kutta pair at tolerance 1e-8): stage
 * derivatives through the same RHS as mmvm_rhs, first same as last; a step
 * is kept when max_i |err_i| / (atol + rtol max(|y_i|, |y5_i|)) <= 1 over
 * y = (x, M); the next step size is h min(5, max(0.2, 0.9 err^(-1/5))) (at
 * most h after a rejection); the last step lands on t_end.  h0: the first
 * step size.  *accepted, *rejected (nullable): the step counts.  Waits for
 * the context stream after every step (the host decides).  Errors:
 * MMVM_E_INVALID_ARG, MMVM_E_NUMERIC (non-finite error estimate),
 * MMVM_E_TIMEOUT (max_steps attempts before t_end; the state is kept at the
 * last accepted step), MMVM_E_DEVICE.                                        */
int mmvm_integrate(mmvm_ctx* ctx, double t_end, double h0, double rtol, double atol,
                   int64_t max_steps, int64_t* accepted, int64_t* rejected);

/* Diagnostics of the context's current state (eq:vorticity_decomposition):
 * the vorticity omega(p) = sum_j sum_k M^j_k D^k phi_00(p - x^j; lambda(t))
 * at npts host points pts (npts x 2, row-major) into the host array omega
 * (npts), FP64 on the device; orders up to 64.  Waits for the context
 * stream.  Errors: MMVM_E_INVALID_ARG (null pointer, no state), MMVM_E_UNSUPPORTED
 * (order above 64), MMVM_E_DEVICE.                                           */
int mmvm_vorticity(mmvm_ctx* ctx, int64_t npts, const double* pts, double* omega);

/* Nonaxisymmetric enstrophy (eq:nonaxi_enstrophy) about the centre (cx, cy):
 * E = int (omega - <omega>_theta)^2 dx over the disk of radius r_max, with
 * <omega>_theta the mean over each circle about the centre; quadrature: nr
 * Gauss-Legendre nodes in r (weight r dr) times ntheta equispaced angles
 * (the trapezoid rule, spectrally accurate for the periodic integrand).
 * The vorticity and the per-ring sums run on the device.  1 <= nr <= 4096,
 * 4 <= ntheta <= 65536.  Errors as mmvm_vorticity.                          */
int mmvm_nonaxi_enstrophy(mmvm_ctx* ctx, double cx, double cy, double r_max, int32_t nr,
                          int32_t ntheta, double* E);

/* Measured fused-multiply-add peak of a device, in flop/s (2 flops per FMA):
 * a full-occupancy grid of independent FMA chains, about 50 ms, timed with
 * CUDA events on a stream of its own.  precision selects the FP64 or the
 * FP32 pipe.  A calibration of the hardware for roofline fractions, not part
 * of the method.  Returns MMVM_E_DEVICE on a CUDA error.                     */
int mmvm_alu_peak(int32_t device, int32_t precision, double* flops_per_s);

/* ------------------------------------------------------------------------
 * Serving: many independent simulations (different n, order, lambda0, nu,
 * dt, step counts) on one GPU at once, with continuous batching.
 *
 * A server owns one worker thread.  Submitted requests wait in a FIFO queue
 * and are admitted while their device footprint (mmvm_request_footprint)
 * fits the HBM budget; admitted simulations keep their state on the device.
 * Simulations of one order and size class form a batch that advances one
 * RK4 step per tick (a graph-captured tick: a persistent all-pairs launch
 * over every member, batched records and finish); batches tick
 * independently on their own streams, members join and leave between ticks,
 * and a simulation leaves at the end of the tick in which it completes
 * nsteps.  The result of a request does not depend on the other requests
 * (its work split and spatial order depend on its own state only).  FP32
 * servers use the far field unless flags holds MMVM_FLAG_NO_FAR_FIELD.
 * Orders up to 16 (a single particle above that: the context API).
 * Submit, poll and stats are thread-safe.
 * ---------------------------------------------------------------------- */
typedef struct mmvm_server mmvm_server;

typedef struct {
  int32_t device;            /* CUDA device ordinal                          */
  int32_t precision;         /* MMVM_FP64 or MMVM_MIXED_FP32, every request  */
  uint64_t hbm_budget_bytes; /* admission budget; 0: half the free device
                                memory at creation                          */
  int32_t max_active;        /* most simulations admitted at once; 0: 256    */
  uint32_t flags;            /* 0 or MMVM_FLAG_NO_FAR_FIELD                  */
} mmvm_server_config;

/* One simulation: the state of eq:vorticity_decomposition at t0 (layouts as
 * mmvm_set_state: x n x 2, moments n x K with K = (order+1)(order+2)/2; both
 * copied by mmvm_submit), the core lambda(t)^2 = lambda0^2 + 4 nu t, and
 * nsteps classic RK4 steps of size dt.                                      */
typedef struct {
  int32_t order;
  double lambda0;
  double nu;
  double t0;
  double dt;
  int64_t nsteps;
  int64_t n;
  const double* x;
  const double* moments;
} mmvm_request;

typedef struct {
  int32_t status;     /* MMVM_OK, MMVM_PENDING or the request's error       */
  int32_t order;
  int64_t n;
  int64_t steps_done;
  double t;           /* time of the state (t0 + steps_done dt)             */
  double queue_ms;    /* submit -> admitted (so far, while queued)          */
  double latency_ms;  /* submit -> result ready (so far, while pending)     */
} mmvm_result;

typedef struct {
  int64_t submitted, completed, failed, queued, active;
  int64_t ticks;             /* batch ticks (one RK4 step of a batch)        */
  int64_t max_batch;         /* most simulations in one batch tick           */
  int64_t max_active;        /* most simulations admitted at once            */
  double pair_interactions;  /* sum over ticks of 4 sum_i n_i^2              */
  double busy_ms;            /* host wall time with a tick on the GPU        */
  uint64_t footprint_bytes;  /* admitted footprint now                       */
  uint64_t peak_footprint_bytes;
  uint64_t budget_bytes;
} mmvm_server_counters;

/* Create a server on cfg->device (starts its worker thread).  Errors:
 * MMVM_E_INVALID_ARG, MMVM_E_DEVICE.                                         */
int mmvm_server_create(const mmvm_server_config* cfg, mmvm_server** out);
/* Stop the worker (after the tick in flight), free everything; requests not
 * yet polled are dropped.                                                   */
void mmvm_server_destroy(mmvm_server* srv);
/* Queue a request; *ticket identifies it for mmvm_poll.  Validates like
 * mmvm_create + mmvm_set_state (MMVM_E_INVALID_ARG, MMVM_E_UNSUPPORTED,
 * MMVM_E_NUMERIC, MMVM_E_ZERO_CIRCULATION) and rejects a request whose
 * footprint exceeds the whole budget (MMVM_E_OOM).                          */
int mmvm_submit(mmvm_server* srv, const mmvm_request* req, uint64_t* ticket);
/* MMVM_PENDING while queued or running (res, if given, shows the progress);
 * when done, copies the final state into x_out (n x 2) and moments_out
 * (n x K) if they are non-null, fills res, forgets the ticket and returns
 * MMVM_OK or the request's error (MMVM_E_NUMERIC if the state became
 * non-finite, MMVM_E_OOM / MMVM_E_DEVICE from the device).  Unknown ticket:
 * MMVM_E_INVALID_ARG.                                                       */
int mmvm_poll(mmvm_server* srv, uint64_t ticket, double* x_out, double* moments_out,
              mmvm_result* res);
/* Counters of the server (see mmvm_server_counters).                           */
int mmvm_server_stats(mmvm_server* srv, mmvm_server_counters* out);
/* Device bytes a request of (order, precision, n) holds while admitted:
 * FP64 state (6 n (2+K) doubles: step start, stage, RK4 sum), source records,
 * partial sums, work lists.  Host-only.                                     */
int mmvm_request_footprint(int32_t order, int32_t precision, int64_t n, uint64_t* bytes);

/* Message for the calling thread's last error ("" if none).                 */
const char* mmvm_last_error(void);
/* The same message under the name of the boundary's error-text call.        */
const char* mmvm_last_error_string(void);

#ifdef __cplusplus
}
#endif
#endif /* MMVM_H_ */
