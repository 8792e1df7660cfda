/*
 * zm.h -- C ABI of the GB300 Z-Model velocity library (libzm.so).
 *
 * The library evaluates the hot path of the Z-Model Rayleigh-Taylor interface solver that
 * Beatnik (arXiv:2406.05490) exercises, on one GPU:
 *   - the surface-derivative stencils, two nodes deep, with periodic or free-edge ghosts
 *     (paper Sec. 3.1, SurfaceMesh and BoundaryCondition);
 *   - the exact all-pairs desingularised Birkhoff-Rott velocity (Sec. 2 BRSolver and
 *     Sec. 3.2.1 ExactBRSolver, the "high order" model);
 *   - the FFT Riesz-transform velocity (Sec. 2, the "low order" model);
 *   - the vorticity derivative and third-order Runge-Kutta time integration, three derivative
 *     evaluations per step (Sec. 3.1 ZModel and TimeIntegrator).
 *
 * Equations (the paper names these ingredients but prints no formulas; this is the reading
 * the library implements).  Mesh n1 x n2, parameter alpha = (i dx1, j dx2), dx_l = L_l / n_l,
 * node p = i*n2 + j.  Per node z = (z1, z2, z3) and w = (w1, w2).
 *     a_l = D_l z (4th-order central), h_kl = a_k . a_l, det = h11 h22 - h12^2,
 *     N = a1 x a2 / |a1 x a2|,  gamma = w1 a2 - w2 a1,
 *     high order:  u_i = -(dx1 dx2 / 4 pi) sum_j (z_i - z_j) x gamma_j / (|z_i - z_j|^2 + delta^2)^(3/2)
 *     low order:   u = -1/2 (R1 w1 + R2 w2) N,   R_l^(k) = -i k_l / |k|  (0 at k = 0, Nyquist)
 *     medium order: dz/dt = the high-order u, while Phi takes the low-order u (Sec. 2: couples
 *                  the FFT and far-field solvers; Sec. 6: FFTs for the change in vorticity)
 *     Phi = g z3 + 1/8 (h22 w1^2 - 2 h12 w1 w2 + h11 w2^2) / det + 1/2 |u|^2
 *     dz/dt = u,    dw_l/dt = -2 A D_l Phi + mu (D_1^2 + D_2^2) w_l
 *     SSP-RK3: y1 = y + dt L(y); y2 = 3/4 y + 1/4 (y1 + dt L(y1)); y' = 1/3 y + 2/3 (y2 + dt L(y2)).
 *
 * Layout of every field array: FP64, component-major, z[c * N + p] (c = 0..2), w[c * N + p]
 * (c = 0..1), u[c * N + p], wdot[c * N + p], with N = n1 * n2.
 *
 * Pointers: every array argument may be host memory or device memory of the context's GPU;
 * the library tells them apart with cudaPointerGetAttributes.  Caller pointers are borrowed
 * for the duration of the call only.  With host pointers a call completes before it returns;
 * with device pointers it is asynchronous on the context's stream (see zm_set_stream).
 *
 * Errors: every int-returning call returns ZM_OK (0) or a negative ZM_ERR_* code;
 * zm_last_error() returns a per-thread message describing the most recent failure.
 * Threading: calls on one context are not re-entrant; distinct contexts may be used from
 * distinct threads and streams concurrently.
 */
#ifndef ZM_H
#define ZM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define ZM_OK 0
#define ZM_ERR_INVALID (-1)      /* bad argument (null pointer, size, parameter range)       */
#define ZM_ERR_NOMEM (-2)        /* device or host allocation failed                          */
#define ZM_ERR_CUDA (-3)         /* a CUDA runtime call or kernel launch failed               */
#define ZM_ERR_TIMEOUT (-4)      /* a bounded device-side wait gave up (status word set)      */
#define ZM_ERR_UNSUPPORTED (-5)  /* valid but not supported: low/medium order on a free-edge
                                    mesh, FFT side of another form than R 2^a              */
#define ZM_ERR_NONFINITE (-6)    /* the state became NaN/Inf (checked by zm_check_finite)    */
#define ZM_ERR_BUSY (-7)         /* resource budget exhausted (serving admission)            */

/* model order (paper Sec. 3.1, ZModel order tag) and precision flag OR'ed into it */
#define ZM_ORDER_LOW 0
#define ZM_ORDER_MEDIUM 1
#define ZM_ORDER_HIGH 2
#define ZM_PREC_FP64 0x000
#define ZM_PREC_FP32C 0x100 /* BR pair terms in FP32 (hi/lo positions near, tile-local
                               coordinates far), per-tile FP32 partials, exact 64-bit fixed-point
                               accumulation across tiles (finer than FP64); all else FP64 */
#define ZM_PREC_DF64 0x200  /* low order only: every stencil, FFT and RK3 operation in
                               double-word arithmetic (pairs of FP32 numbers, ~48-bit significand,
                               FP32 exponent range) instead of FP64 instructions; the resident
                               state is held as FP32 pairs with z1, z2 relative to the mesh
                               coordinates and converted at zm_set_state / zm_get_state /
                               zm_velocity.  Not in the paper: an implementation choice for GPUs
                               whose FP64 rate is far below their FP32 rate */

typedef struct {
    int32_t n1, n2;   /* nodes along alpha1 (slow index i) and alpha2 (fast index j), >= 5 */
    double L1, L2;    /* parameter-domain lengths (> 0); dx_l = L_l / n_l                 */
    int32_t periodic; /* 1: periodic ghosts, z1/z2 shifted by L1/L2 across the seam;
                         0: free edges, two ghost nodes by linear extrapolation            */
} zm_mesh;

typedef struct zm_ctx zm_ctx;

/* Create a context for one interface on the current CUDA device.  Allocates all device state
 * and workspace (owned by the context until zm_destroy).  delta > 0 is the Birkhoff-Rott core
 * size (high order); mu >= 0 the artificial viscosity; `order` is ZM_ORDER_* | ZM_PREC_*.
 * Low and medium order (periodic FFT solver, Sec. 2 and 3.1) take sides L = R 2^a with a >= 3,
 * R odd in 1 .. 19 and L <= 8192 (the paper's 4864 = 19 x 2^8 among them); ZM_PREC_DF64 takes
 * the same sides except powers of two above 4096.
 * Returns ZM_ERR_UNSUPPORTED for low or medium order on a free-edge mesh or on other sides,
 * and for ZM_PREC_DF64 with medium or high order; ZM_ERR_INVALID for ZM_PREC_FP32C combined
 * with ZM_PREC_DF64. */
int zm_create(const zm_mesh *mesh, double atwood, double g, double mu, double delta, int order,
              zm_ctx **out);

/* Use `cuda_stream` (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream; NULL for
 * the legacy default stream) for all later work of this context. */
int zm_set_stream(zm_ctx *ctx, void *cuda_stream);

/* Copy a state (z: 3N doubles, w: 2N doubles) into the context's resident state. */
int zm_set_state(zm_ctx *ctx, const double *z, const double *w);

/* Copy the resident state out (either pointer may be NULL to skip it). */
int zm_get_state(zm_ctx *ctx, double *z, double *w);

/* One derivative evaluation L(z, w) = (u, wdot) without advancing the state (one ZModel call,
 * paper Sec. 3.1).  z, w: input state, or both NULL to use the resident state.
 * u: 3N velocity output (dz/dt).  wdot: 2N vorticity derivative output, may be NULL. */
int zm_velocity(zm_ctx *ctx, const double *z, const double *w, double *u, double *wdot);

/* Advance the resident state by nsteps SSP-RK3 steps of size dt (three derivative evaluations
 * per step, paper Sec. 3.1 TimeIntegrator).  Asynchronous on the context's stream. */
int zm_step(zm_ctx *ctx, double dt, int nsteps);

/* Cutoff Birkhoff-Rott sum (paper Sec. 3.2.2, CutoffBRSolver): from now on sum only over the
 * sources within `cutoff` of each target (0 = all sources, the exact sum).  A pair is in iff
 * |r|^2 <= cutoff^2 with r formed from FP32 hi/lo positions and |r|^2 rounded to FP32.  FP32C
 * contexts (high or medium order); ZM_ERR_UNSUPPORTED otherwise. */
int zm_set_cutoff(zm_ctx *ctx, double cutoff);

/* Autotune the work decomposition of an FP32C high-order context (see zm_batch_autotune; the
 * resident state is used, so set it first).  Other contexts have nothing to tune: *chosen = 0. */
int zm_autotune(zm_ctx *ctx, const char *cache_path, int32_t *chosen);

/* Autotune the tile shapes and the work decomposition of an FP32C high-order context together
 * (see zm_batch_autotune_tiles).  Unlike zm_autotune, the choice can change results within the
 * FP32C bound.  Other contexts: *tp1 = *tp2 = *chunk = 0. */
int zm_autotune_tiles(zm_ctx *ctx, const char *cache_path, int32_t *tp1, int32_t *tp2, int32_t *chunk);

/* Set (get) the tile shape of an FP32C high- or medium-order context: the mesh patch of 256
 * nodes a target or source tile covers, (tp1, tp2) one of (16,16), (8,32), (32,8), (4,64),
 * (64,4) (see zm_batch_set_tile_shape).  Results change within the FP32C bound.  Returns
 * ZM_ERR_INVALID for another shape, ZM_ERR_UNSUPPORTED for other contexts. */
int zm_set_tile_shape(zm_ctx *ctx, int32_t tp1, int32_t tp2);

/* Far path of an FP32C high- or medium-order context's all-pairs sum (see
 * zm_batch_set_far_path): ZM_FAR_CUDA (default) or ZM_FAR_TENSOR.  ZM_ERR_INVALID for another
 * value, ZM_ERR_UNSUPPORTED for other contexts. */
int zm_set_far_path(zm_ctx *ctx, int32_t path);
int zm_get_far_path(zm_ctx *ctx, int32_t *path);
int zm_get_tile_shape(zm_ctx *ctx, int32_t *tp1, int32_t *tp2);

/* Wait for the context's stream; reports ZM_ERR_TIMEOUT / ZM_ERR_CUDA raised by its kernels. */
int zm_sync(zm_ctx *ctx);

/* Free the context and all device memory it owns (synchronises its stream first). */
void zm_destroy(zm_ctx *ctx);

/* Static description of a status code, and the calling thread's last detailed message. */
const char *zm_error_string(int code);
const char *zm_last_error(void);

/* ---- instrumentation ------------------------------------------------------------------- */

/* Kernel classes timed by the optional per-context CUDA-event profiler. */
#define ZM_K_GEOMETRY 0 /* ghost fill + tangents + normal + sheet-strength records          */
#define ZM_K_BR 1       /* all-pairs Birkhoff-Rott sum                                      */
#define ZM_K_REDUCE 2   /* split-source reduction + Phi                                     */
#define ZM_K_VORT 3     /* grad Phi, Laplacian, vorticity derivative, RK3 combine           */
#define ZM_K_FFT 4      /* Riesz-transform FFT passes                                       */
#define ZM_K_COUNT 5

typedef struct {
    double ms[ZM_K_COUNT];        /* summed CUDA-event time per kernel class               */
    int64_t launches[ZM_K_COUNT]; /* launches per kernel class                             */
    int64_t pairs;                /* Birkhoff-Rott pair interactions evaluated (N^2 each)  */
} zm_profile;

/* Turn event timing around every launch on (1) or off (0); turning it on clears counters.
 * Counting launches and pairs is always on. */
int zm_set_profiling(zm_ctx *ctx, int on);
/* Synchronises the stream and reports counters accumulated since the last reset. */
int zm_get_profile(zm_ctx *ctx, zm_profile *out);
int zm_reset_profile(zm_ctx *ctx);

/* Check the resident state for NaN/Inf: returns ZM_OK or ZM_ERR_NONFINITE (synchronous). */
int zm_check_finite(zm_ctx *ctx);

/* Measure a CUDA-core throughput of the current GPU with CUDA events (the roofline denominator
 * of the Birkhoff-Rott kernels; the paper has no counterpart).  kind 0: FP32 FMA flop/s (FMA =
 * 2 flops), 1: FP64 FMA flop/s, 2: MUFU rsqrt operations/s, 3: packed FP32x2 FMA flop/s
 * (fma.rn.f32x2), 4: packed and scalar FP32 FMAs interleaved, flop/s.  Synchronous; allocates
 * 64 bytes. */
int zm_measure_peak(int kind, double *ops_per_s);

/* Exercise the bounded device-side wait that every mbarrier wait in the library uses (the paper
 * has no counterpart): one CTA polls an mbarrier phase up to max_polls times (1 <= max_polls <=
 * 2^34).  arrive = 0: nothing ever arrives, so the wait gives up, the kernel sets the timeout bit
 * of its status word and returns, and this call returns ZM_ERR_TIMEOUT -- the same path a stuck
 * copy would take inside the Birkhoff-Rott kernels, without a hang or a fault; arrive = 1: one
 * thread arrives first and the call returns ZM_OK.  *elapsed_ms (may be NULL) receives the
 * kernel's duration.  Synchronous on the legacy default stream; allocates one int. */
int zm_wait_selftest(int64_t max_polls, int32_t arrive, double *elapsed_ms);

/* The poll limit of the library's bounded waits (the kernels give up after this many polls). */
int64_t zm_wait_poll_limit(void);

/* 1 when this library is the checked build (libzm_checked.so, compiled with ZM_CHECKS=1), else 0.
 * In the checked build every kernel tests the indices it computes (neighbour wraps, tile and
 * record numbers, transposed writes, shared-memory positions) before the access; an index
 * outside its array is counted and the access skipped, so the kernel neither faults nor traps.
 * Compute-sanitizer is not needed for this; the default build has no such tests. */
int zm_checked_build(void);

/* Index violations the checked build has counted since the last clear, over all kernels:
 * *hits (required) the count, *first_index and *source_line (may be NULL) the first offending
 * index and the source line of its test.  clear != 0 resets the count.  Synchronises the device.
 * Returns ZM_OK (with *hits = 0 in the default build), or ZM_ERR_CUDA. */
int zm_bounds_status(uint32_t *hits, int64_t *first_index, int32_t *source_line, int32_t clear);

/* ---- batches of interfaces (high order, FP32C) ------------------------------------------- */

/* Many independent interfaces of uneven mesh sizes advanced together: each RK3 stage runs four
 * launches over the whole batch (geometry, one persistent all-pairs launch over a shared work
 * list, the fixed-point finish, the vorticity/RK3 pass) and a whole step is replayed from a
 * CUDA graph.  Per-interface results are bitwise independent of the other interfaces in the
 * batch and of scheduling (exact fixed-point accumulation), and equal to those of zm_create
 * with ZM_ORDER_HIGH | ZM_PREC_FP32C.  The paper has no batched form: it runs one interface
 * over many ranks (Sec. 3). */
typedef struct zm_batch zm_batch;

/* count interfaces; meshes[k], atwood[k] and delta[k] (> 0) per interface, g and mu shared.
 * Sides >= 5, n1 * n2 <= 2^24 each.  Allocates all device state (owned until destroy). */
int zm_batch_create(int32_t count, const zm_mesh *meshes, const double *atwood, double g,
                    double mu, const double *delta, zm_batch **out);
int zm_batch_set_stream(zm_batch *b, void *cuda_stream);
/* State of interface `index` in or out (host or device pointers, layout as for zm_set_state). */
int zm_batch_set_state(zm_batch *b, int32_t index, const double *z, const double *w);
int zm_batch_get_state(zm_batch *b, int32_t index, double *z, double *w);
/* One derivative evaluation of every interface at its resident state (asynchronous); then
 * zm_batch_get_velocity copies interface `index`'s u (3N) and dw/dt (2N; either may be NULL). */
int zm_batch_velocity(zm_batch *b);
int zm_batch_get_velocity(zm_batch *b, int32_t index, double *u, double *wdot);
/* nsteps SSP-RK3 steps of every interface (asynchronous; one graph launch per step). */
int zm_batch_step(zm_batch *b, double dt, int32_t nsteps);
int zm_batch_sync(zm_batch *b);
/* Tuning: source tiles per all-pairs work item (0 = default by size); results do not change. */
int zm_batch_set_chunk(zm_batch *b, int32_t chunk);
/* Autotuner: times work-item sizes 1, 2, 4, ... 32 source tiles on the resident states (one
 * full derivative evaluation each, twice, CUDA events), keeps the fastest and returns it in
 * *chosen (and its time per evaluation in *best_ms, or -1 if the choice came from a cache).
 * Choices are remembered per (GPU model, SM count, occupancy, size buckets) for the process
 * and, if cache_path is not NULL, appended to / read from that text file.  Results do not
 * depend on the choice (exact fixed-point accumulation); synchronous. */
int zm_batch_autotune(zm_batch *b, const char *cache_path, int32_t *chosen, float *best_ms);
/* Tile shape of the all-pairs sum: every interface is cut into tiles of tp1 x tp2 mesh nodes
 * (256 each; (16,16) by default, or (8,32), (32,8), (4,64), (64,4)) that serve both as target
 * tiles and as source tiles.  Elongated tiles are more compact in space when the two mesh
 * spacings differ, so fewer tile pairs need the near (exact-difference) path.  Changing the
 * shape rebuilds the source records and the plan; results change within the FP32C bound (tile
 * centres and the near/far split move), not bit for bit.  Synchronous. */
int zm_batch_set_tile_shape(zm_batch *b, int32_t tp1, int32_t tp2);
/* How the all-pairs sum treats far tile pairs (bounding spheres at least 1.25 x the sum of
 * their radii apart; near pairs always take the CUDA cores with exact FP32 hi/lo differences).
 * Both evaluate the pair terms in tile-local coordinates, sum_j K_ij (s_j x g_j) - t_i x
 * sum_j K_ij g_j with K_ij = (|s_j - t_i|^2 + delta^2)^(-3/2):
 *   ZM_FAR_CUDA (default)  everything on the CUDA cores (packed FP32x2 instructions);
 *   ZM_FAR_TENSOR          |s_j - t_i|^2 + delta^2 = |t_i|^2 + Y_ij with the Gram part Y (targets
 *                          x 4 times 4 x sources) on the tensor cores (TF32 operands split into
 *                          a TF32 part and a TF32 rest, two MMAs per 128 targets x 32 sources),
 *                          the rest on the CUDA cores.  Correct within the FP32C bound (the
 *                          same error as ZM_FAR_CUDA) but about 1.15x slower on GB300: the
 *                          hand-off and packing work it adds outweighs the arithmetic it
 *                          removes.
 * Results change within the FP32C bound, not bit for bit.  Rebuilds the plan; synchronous.
 * ZM_ERR_INVALID for another value. */
#define ZM_FAR_TENSOR 0
#define ZM_FAR_CUDA 1
int zm_batch_set_far_path(zm_batch *b, int32_t path);
int zm_batch_get_far_path(zm_batch *b, int32_t *path);
int zm_batch_get_tile_shape(zm_batch *b, int32_t *tp1, int32_t *tp2);
/* Autotuner for tiles: times each candidate tile shape at the default work-item size, then the
 * work-item sizes 1 .. 32 for the fastest shape (one evaluation each, twice, CUDA events), keeps
 * the fastest pair, and remembers it like zm_batch_autotune (key suffix "|tiles"; the cache
 * stores shape index * 1000 + work-item size).  Returns the shape and the work-item size, and
 * the time per evaluation in *best_ms (-1 if the choice came from the memo or the cache). */
int zm_batch_autotune_tiles(zm_batch *b, const char *cache_path, int32_t *tp1, int32_t *tp2, int32_t *chunk,
                            float *best_ms);
/* Cutoff sum (see zm_set_cutoff) for interface `index`, or all interfaces if index = -1. */
int zm_batch_set_cutoff(zm_batch *b, int32_t index, double cutoff);
/* Totals: mesh points, pair interactions per evaluation, work items, persistent CTAs. */
int zm_batch_info(zm_batch *b, int64_t *points, int64_t *pairs_per_eval, int64_t *work_items,
                  int32_t *ctas);
int zm_batch_set_profiling(zm_batch *b, int on);
int zm_batch_get_profile(zm_batch *b, zm_profile *out);
void zm_batch_destroy(zm_batch *b);

/* ---- serving: continuous batching of solve requests ------------------------------------- */

/* A worker thread owned by the server admits submitted requests as slots (max_slots) and
 * device memory (mem_budget_bytes, counted per request from its mesh size) free up, keeps every
 * admitted interface's state resident, advances resident interfaces by one RK3 step per
 * iteration (the batched FP32C path, all of them in one set of launches) and retires finished
 * ones between iterations, so requests arriving while others run join the next iteration.  A
 * request's result does not depend on the others (bitwise).  Which requests are admitted and
 * advanced follows the scheduling policy (zm_server_set_policy; default ZM_SERVE_ALL).  The
 * paper has no serving form. */
#define ZM_REQ_QUEUED 0
#define ZM_REQ_RUNNING 1
#define ZM_REQ_DONE 2
#define ZM_REQ_FAILED 3

typedef struct zm_server zm_server;

typedef struct {
    int64_t iterations;    /* loop iterations that ran on the GPU                              */
    int64_t steps;         /* batched RK3 steps                                                */
    int64_t pairs;         /* Birkhoff-Rott pair interactions evaluated                        */
    int64_t completed, failed, queued, running, peak_running;
    int64_t bytes_in_use, peak_bytes; /* device bytes held by admitted requests              */
    double busy_s;         /* wall time spent in GPU iterations                               */
} zm_server_stats;

/* Start a server on the current device (its own stream and worker thread). */
int zm_server_create(size_t mem_budget_bytes, int32_t max_slots, double g, double mu,
                     zm_server **out);
/* Queue a solve: mesh, Atwood number, core size delta > 0, step dt, nsteps SSP-RK3 steps, and
 * the initial state (host pointers, copied before return).  *id receives the request id.
 * ZM_ERR_BUSY if the request alone exceeds the memory budget. */
int zm_server_submit(zm_server *s, const zm_mesh *mesh, double atwood, double delta, double dt,
                     int32_t nsteps, const double *z, const double *w, int64_t *id);
/* Device bytes one request of this mesh holds while admitted (what the budget counts). */
int zm_server_request_bytes(const zm_mesh *mesh, size_t *bytes);
/* Current state of a request (ZM_REQ_*). */
int zm_server_poll(zm_server *s, int64_t id, int32_t *state);
/* Block until the request finished (timeout_s < 0: no limit); returns its status, or
 * ZM_ERR_TIMEOUT if the host-side wait ran out. */
int zm_server_wait(zm_server *s, int64_t id, double timeout_s);
/* Copy a finished request's final state (host pointers, may be NULL), its latency from submit
 * to completion and its queueing time from submit to admission (seconds), and release the
 * request.  Returns the request's status (ZM_ERR_NONFINITE if its state blew up). */
int zm_server_result(zm_server *s, int64_t id, double *z, double *w, double *latency_s,
                     double *queue_s);
/* Cancel a request: a queued one fails at once, a running one leaves at the next iteration. */
int zm_server_cancel(zm_server *s, int64_t id);
int zm_server_get_stats(zm_server *s, zm_server_stats *out);

/* Scheduling policy, changeable at any time (applies from the next iteration):
 * ZM_SERVE_ALL   admission first come, first served (the head of the queue waits until it
 *                fits); every resident interface advances one step per iteration.
 *                pairs_per_iteration is ignored.
 * ZM_SERVE_SRPT  shortest remaining work first: queued requests are admitted least total work
 *                (pair interactions) first wherever they fit; each iteration advances the
 *                resident interfaces with the least remaining work first, adding them while the
 *                iteration's pair interactions stay within pairs_per_iteration (<= 0: no cap;
 *                always at least one interface).  Small requests overtake large ones, which
 *                bounds their latency under overload; under endless overload the largest
 *                requests can starve.
 * Results do not depend on the policy (bitwise).  ZM_ERR_INVALID for an unknown policy. */
#define ZM_SERVE_ALL 0
#define ZM_SERVE_SRPT 1
int zm_server_set_policy(zm_server *s, int32_t policy, int64_t pairs_per_iteration);
/* Stop the worker and free everything (requests still queued or running are dropped). */
void zm_server_destroy(zm_server *s);

/* ---- Birkhoff-Rott sum without allocation ------------------------------------------------ */

/* The paper has no counterpart: this entry point exists for callers that cannot allocate GPU
 * memory -- a host application that reserves all device memory at start-up and forbids later
 * allocations, or code that must not pay the device-wide synchronisation that cudaMalloc and
 * cudaFree imply.  It computes the FP64 all-pairs sum of zm_velocity's high-order path on
 * caller-prepared inputs and allocates nothing: no cudaMalloc, cudaFree or allocating library
 * call.  Its workspace (tile-major source records, split partial sums, a status word; 9 MiB in
 * all) is one static device array inside libzm.so, held by every GPU that loads the library
 * until the process exits.
 *
 *   u_i = sum_j (z_j - z_i) x gamma_j / (|z_j - z_i|^2 + delta^2)^(3/2),  i, j < n
 *
 * n      number of points, 1 <= n <= 65536 (the workspace limit); larger n -> ZM_ERR_INVALID.
 * z      device, 3n doubles, component-major positions (z1[0..n), z2[0..n), z3[0..n)).
 * gamma  device, 3n doubles, component-major scaled sheet strengths; for a mesh these are
 *        (dx1 dx2 / 4 pi)(w1 a2 - w2 a1), which makes u the high-order velocity.
 * delta  core size, > 0.
 * u      device, 3n doubles, output.
 * status optional device int32: set to ZM_OK, or ZM_ERR_TIMEOUT if a bounded device-side wait
 *        gave up, when the work completes.  May be NULL.
 * cuda_stream  the cudaStream_t to run on (NULL: legacy default stream).
 * Asynchronous on cuda_stream; returns ZM_ERR_INVALID for bad sizes, null or host pointers.
 * The first call on each device looks up the workspace's device address (cudaGetSymbolAddress
 * with that device current) and caches it; make that first call before any stream capture.
 * All calls in the process share the one workspace: it keeps the last call's contents, every
 * call rewrites what it reads before reading it, and calls whose work overlaps on the GPU
 * (different streams, or different host threads without ordering) race on it. */
int zm_br_velocity_noalloc(int32_t n, const double *z, const double *gamma, double delta,
                           double *u, int32_t *status, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* ZM_H */
