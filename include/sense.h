/*
 * sense.h -- C ABI of libsense.so, a CUDA (sm_103a) implementation of
 * multi-coil Cartesian SENSE reconstruction.
 *
 * Method: arXiv 1807.11830 (OpenCLIPER), Sec. IV-A, Eq. 1,
 *     M = sum_i S_i^* F^{-1}(Y_i),
 * is the coil-combining adjoint E^H of the encoding operator
 *     E x = { M_f F2 (S_c . x_f) }_{f,c}
 * when every k-space line is sampled.  The library provides E, E^H, the
 * normal operator E^H E and conjugate-gradient SENSE (CG on E^H E x = E^H y),
 * plus root-sum-of-squares (Sec. IV-B).
 *
 * Conventions shared by every entry point:
 *   - F is the unitary DFT, exp(-2 pi i jk/n)/sqrt(n) forward, its conjugate
 *     inverse (Eq. 1 writes F^{-1} with no scale); DC at index 0 (no shift).
 *   - Row index y (slow, "ny") is the phase-encode direction and is masked by
 *     line; x (fast, "nx") is the fully sampled readout.
 *   - Layouts, row-major, complex interleaved (re, im):
 *       image x, out, x_out     [frames][ny][nx]        sense_c32
 *       sensitivities S         [coils][ny][nx]         storage type
 *       k-space y               [frames][coils][lines][nx]  storage type
 *       lines                   [frames][lines] int32, each row strictly
 *                               increasing inside [0, ny)
 *     "storage type" is sense_c32 for SENSE_STORE_C64 and a pair of
 *     bfloat16 (re, im; 4 bytes) for SENSE_STORE_BF16.  All frames of one
 *     plan share the same S.
 *   - Every array argument is a DEVICE pointer on the plan's device, owned by
 *     the caller, 16-byte aligned; the library never frees caller memory.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = legacy default stream).  Argument errors are reported
 *     synchronously by the return value.  Invalid line indices are detected
 *     by the kernels, which skip the offending line and raise a device flag
 *     that sense_plan_check() reports as SENSE_EDEVICE.
 *   - A plan is not thread-safe: calls on one plan must be serialised by the
 *     caller (they share the plan's workspace).
 *   - On any non-OK return, sense_last_error() holds a message for the
 *     calling thread.
 */
#ifndef SENSE_H
#define SENSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { float re, im; } sense_c32;

typedef enum {
  SENSE_OK = 0,
  SENSE_EINVAL = 1,             /* null/unaligned pointer, bad shape or argument */
  SENSE_EUNSUPPORTED_SIZE = 2,  /* ny or nx has no compiled transform (see sense_size_supported) */
  SENSE_ENOMEM = 3,             /* device allocation failed */
  SENSE_ECUDA = 4,              /* a CUDA runtime call failed */
  SENSE_ETIMEOUT = 5,           /* a bounded device-side wait gave up */
  SENSE_ENUMERIC = 6,           /* non-finite CG values: NaN or Inf in a request's y or S (sense_queue_wait) */
  SENSE_EQUEUE_FULL = 7,        /* request queue cannot admit more work */
  SENSE_ENOTFOUND = 8,          /* unknown request id */
  SENSE_EDEVICE = 9             /* a kernel flagged invalid input (bad line index/order) */
} sense_status;

typedef enum { SENSE_STORE_C64 = 0, SENSE_STORE_BF16 = 1 } sense_storage;

/* Problem shape of one plan: ny x nx images, `coils` maps, `frames` images
 * sharing them, `lines` sampled phase-encode rows per frame.
 *
 * `centred` selects the k-space convention (the paper fixes none):
 *   0  DC at index 0 along both axes, image origin at pixel (0, 0): every
 *      transform is the unitary DFT exp(-2 pi i jk/n) / sqrt(n);
 *   1  DC at index n/2 and the image centre at pixel n/2 along both axes:
 *      every transform is the centred unitary DFT
 *      exp(-2 pi i (k - n/2)(j - n/2)/n) / sqrt(n) (fftshift . F . ifftshift),
 *      and `lines` index that centred k-space.
 * Every supported length is even, where the centred DFT equals
 * (-1)^(n/2) D F D with D = diag((-1)^i); the library applies those signs at
 * the kernels' loads and stores, and CG iterates in the sign-modulated image
 * space (the same scalars, residuals and iteration counts), mapping x back at
 * the end. */
typedef struct {
  int ny, nx, coils, frames, lines;
  int storage; /* sense_storage of S and y */
  int centred; /* 0 or 1, see above */
} sense_shape;

/* Per-frame CG outcome written by sense_cg_solve. */
typedef enum {
  SENSE_CG_CONVERGED = 1, /* relative residual reached rel_tol, or became exactly 0 */
  SENSE_CG_MAXITER = 2,   /* max_iter iterations applied */
  SENSE_CG_BREAKDOWN = 3  /* Re<p, E^H E p> was not > 0; x holds the last good iterate */
} sense_cg_outcome;

typedef struct sense_plan sense_plan;

/* 1 if n is a supported transform length for ny or nx, else 0. */
int sense_size_supported(int n);

/* Create a plan for `shape` on CUDA device `device`: validates the shape,
 * uploads FP64-derived twiddle tables and allocates the plan's workspace
 * (compacted k-space intermediate, CG vectors, FP64 partial sums).  The plan
 * owns all of it.  Returns SENSE_EUNSUPPORTED_SIZE for untransformable ny/nx,
 * SENSE_ENOMEM if the workspace does not fit. */
sense_status sense_plan_create(const sense_shape* shape, int device, sense_plan** out);

/* Release everything the plan owns.  Waits for the plan's outstanding work. */
sense_status sense_plan_destroy(sense_plan* plan);

/* Device memory the plan holds, in bytes. */
size_t sense_plan_workspace_bytes(const sense_plan* plan);

/* Encoding operator E (Eq. 1's forward model):
 *   y[f][c][l][:] = (F2 (S_c . x_f))[lines[f][l]][:]
 * x: [frames][ny][nx] c32; S, y: storage type.  In BF16 storage the result is
 * rounded to bfloat16 (round-to-nearest-even) when stored. */
sense_status sense_forward(sense_plan* plan, const sense_c32* x, const void* S, const int32_t* lines, void* y,
                           void* stream);

/* Adjoint E^H (Eq. 1 with zero-filled missing lines):
 *   x_f = sum_c conj(S_c) . F2^H (Z_f y_{f,c}),  Z_f scattering line l to row lines[f][l].
 * With lines = all rows this is exactly Eq. 1 of the paper. */
sense_status sense_adjoint(sense_plan* plan, const void* y, const void* S, const int32_t* lines, sense_c32* x,
                           void* stream);

/* Allocation-free adjoint (the paper has no counterpart; this is a deployment
 * variant of sense_adjoint).  Some callers cannot allocate device memory --
 * plugins inside a host application that owns all device memory through its
 * own pool, processes whose device memory budget is fixed up front, and
 * latency-critical loops that must stay out of the CUDA allocator (cudaMalloc
 * and cudaFree can synchronise the device) -- so they cannot create a plan.
 * This call computes the same x = E^H y as sense_adjoint for `shape` without a
 * plan and without allocating: the row-pass intermediate lives in a fixed
 * file-scope device array of 2^21 complex values (16 MiB) that every GPU
 * which loads the library holds until the process exits, next to twiddle
 * tables for every supported length.  The caller still passes y, S, lines and
 * x (device pointers, layouts as above).
 *   - frames*coils*lines*nx must not exceed 2^21; larger shapes return
 *     SENSE_EINVAL with a message (use sense_adjoint with a plan instead).
 *   - The first call on each device does a one-time set-up with that device
 *     current (symbol addresses and a synchronous upload of the twiddle
 *     tables); make that first call before any stream capture.
 *   - Every call shares the one array and leaves its contents behind: calls
 *     that overlap on the GPU (different streams, or different host threads)
 *     race on it and must be serialised by the caller.
 *   - Line-index errors are skipped by the kernels but not reported, and
 *     neither is a bounded wait of the row pass that gives up (never
 *     expected; the block then stores nothing): there is no plan to hold the
 *     device flag.  Pass valid lines. */
sense_status sense_adjoint_noalloc(const sense_shape* shape, const void* y, const void* S, const int32_t* lines,
                                   sense_c32* x, void* stream);

/* Normal operator out = E^H E x, per frame: the composition of the encoding
 * operator whose adjoint, with every line sampled, is Eq. 1 (Sec. IV-A) with
 * that adjoint.  The paper applies Eq. 1 once and has no normal operator; it
 * is the product every CG iteration needs.  Computed column-wise: because the
 * mask acts on rows only and F_x is unitary, E^H E = sum_c S_c^H F_y^H M_f F_y S_c,
 * so no x-direction transform is needed.  `out` must not alias `x`. */
sense_status sense_normal(sense_plan* plan, const sense_c32* x, const void* S, const int32_t* lines,
                          sense_c32* out, void* stream);

/* CG-SENSE.  The paper reconstructs by Eq. 1 alone (Sec. IV-A), which is the
 * least-squares solution only when every line is sampled and sum_c |S_c|^2 = 1;
 * with undersampled k-space the same encoding model is inverted iteratively
 * by conjugate gradients on its normal equations.  The paper fixes no
 * iteration; the library's choices (per-frame scalars, FP64 inner products,
 * the stopping rules below, breakdown handling) are stated here in full.
 * Hestenes-Stiefel conjugate gradients on (E^H E) x = E^H y, run
 * independently per frame from x0 = 0 with FP64 inner products:
 *   r0 = p0 = E^H y;  per iteration  q = E^H E p,  alpha = <r,r>/Re<p,q>,
 *   x += alpha p,  r -= alpha q,  beta = <r',r'>/<r,r>,  p = r' + beta p.
 * A frame stops when <r,r> becomes 0, when rel_tol > 0 and
 * sqrt(<r,r>/<r0,r0>) <= rel_tol, after max_iter iterations, or on breakdown
 * (Re<p,q> not > 0).  Outputs (device arrays, any may be NULL except x_out):
 *   x_out [frames][ny][nx];  iters_out [frames] iterations applied;
 *   rel_resid_out [frames] sqrt(<r,r>/<r0,r0>) at exit (0 if y_f == 0);
 *   outcome_out [frames] a sense_cg_outcome.
 * The iteration loop runs on the device without host synchronisation; with
 * rel_tol > 0 the host polls a device counter of live frames every few
 * iterations to stop early.  x_out must not alias y or S. */
/* (With sense_plan_set_lambda the system solved is (E^H E + lambda I) x = E^H y.) */
sense_status sense_cg_solve(sense_plan* plan, const void* y, const void* S, const int32_t* lines, int max_iter,
                            double rel_tol, sense_c32* x_out, int32_t* iters_out, double* rel_resid_out,
                            int32_t* outcome_out, void* stream);

/* CG-SENSE with every input and output in HOST memory: the same solve as
 * sense_cg_solve (same stopping rules), for callers that do not manage device
 * memory.  On `stream` the call copies y, S and lines to
 * device buffers the plan owns (allocated on the first call and kept for the
 * plan's life), runs the solve, copies x and the per-frame outputs back, and
 * synchronises `stream` before returning; the return value then also reports
 * errors the kernels flagged (as sense_plan_check does).  Page-locked host
 * buffers make the copies asynchronous DMA transfers; pageable memory works
 * but is staged by the driver.  iters_host, rel_resid_host and outcome_host
 * may be NULL.  Layouts and storage types are those of sense_cg_solve. */
sense_status sense_cg_solve_host(sense_plan* plan, const void* y_host, const void* S_host, const int32_t* lines_host,
                                 int max_iter, double rel_tol, sense_c32* x_host, int32_t* iters_host,
                                 double* rel_resid_host, int32_t* outcome_host, void* stream);

/* ---- Uneven batching ----
 * (No counterpart in the paper: a deployment layer that runs many
 * independent sense_cg_solve problems together; each instance's result is
 * its own solve's.) 
 * A batch holds many independent CG-SENSE problems ("instances") of
 * different ny x nx, coil count, frame count and line count.  Instances are
 * grouped by (ny, nx, storage) into size classes; every CG iteration of every
 * frame of a class runs in one persistent launch (see
 * sense_plan_set_cg_mode), and the whole solve -- CG start of each instance,
 * one persistent launch per class, per-instance outputs -- is captured once
 * per argument set into a CUDA graph and replayed.  Each frame's iterates
 * depend only on its own data and its class's kernel variant, so an instance
 * gives the same result alone (a plan with the same variant and persistent
 * mode) as inside the batch. */
typedef struct sense_batch sense_batch;

/* Per-instance arguments of a batch solve (device pointers; layouts and
 * alignment as for sense_cg_solve; the outputs other than x_out may be NULL). */
typedef struct {
  const void* y;
  const void* S;
  const int32_t* lines;
  sense_c32* x_out;
  int32_t* iters_out;
  double* rel_resid_out;
  int32_t* outcome_out;
} sense_batch_io;

/* Create a batch of `count` instances on `device`: one plan per instance
 * (workspace, CG state) plus per-class scheduling state. */
sense_status sense_batch_create(const sense_shape* shapes, int count, int device, sense_batch** out);
sense_status sense_batch_destroy(sense_batch* batch);
size_t sense_batch_workspace_bytes(const sense_batch* batch);
/* Number of size classes (persistent launches per solve). */
int sense_batch_classes(const sense_batch* batch);
/* Pick each class's normal-operator kernel variant by timing it on the
 * class member with the most frames (see sense_plan_autotune). */
sense_status sense_batch_autotune(sense_batch* batch, const sense_batch_io* io, void* stream);
/* Tikhonov weight of instance `instance`'s CG (see sense_plan_set_lambda). */
sense_status sense_batch_set_lambda(sense_batch* batch, int instance, double lambda);
/* Temporal weight of instance `instance` (see sense_plan_set_temporal). */
sense_status sense_batch_set_temporal(sense_batch* batch, int instance, double lambda_t);
/* Use kernel variant `variant` for every class of row count `ny`. */
sense_status sense_batch_set_variant(sense_batch* batch, int ny, int variant);
/* CG-SENSE on every instance (io[i] for instance i), same stopping rules as
 * sense_cg_solve, asynchronously on `stream`. */
sense_status sense_batch_cg_solve(sense_batch* batch, const sense_batch_io* io, int max_iter, double rel_tol,
                                  void* stream);
/* Synchronise `stream` and report device-flagged errors of any instance. */
sense_status sense_batch_check(sense_batch* batch, void* stream);

/* ---- Serving: request queue with continuous batching ----
 * (No counterpart in the paper: a serving layer over the same CG-SENSE solve;
 * a request's result equals the problem solved alone, see below.) 
 * A scheduler thread admits submitted reconstructions in arrival order while
 * the HBM budget and the live-request limit allow, keeps their k-space, maps
 * and CG state on the device, and advances every live request by one CG
 * iteration per tick (iters_per_tick of them): one persistent launch per size
 * class runs the iterations of every live frame of that class, whatever
 * iteration each frame is at.  A request retires when all its frames have stopped (the stopping
 * rules of sense_cg_solve) or after max_iter ticks; its image is copied to a
 * pinned host buffer and its device memory released.  Requests that arrive
 * while others run join at the next tick.  Each size class uses one kernel
 * variant (autotuned on the first request of the class), so a request's
 * result equals the same problem solved alone by a plan with that variant
 * in persistent mode. */
typedef struct sense_queue sense_queue;

typedef struct {
  size_t hbm_budget_bytes; /* device bytes requests may hold; 0 = free memory at creation minus 1 GiB */
  int max_live;            /* most requests admitted at once; 0 = no limit */
  int autotune;            /* 1: autotune each size class on its first request; 0: variant 0 */
  int iters_per_tick;      /* CG iterations per tick; each frame still stops at its own max_iter /
                              tolerance inside the tick, new requests join between ticks.  0: adaptive --
                              while requests wait for admission, as many as fit in about 4 ms at the
                              last tick's time per iteration (1 to 10); otherwise 10, stretched up to 80
                              (the largest remaining budget of the live requests) */
  size_t staging_reserve_bytes; /* page-locked host staging allocated at creation (0: none); the
                                   staging arena grows on demand beyond it */
  size_t max_live_work;    /* 0 = no limit.  Otherwise admit while the live requests' work, the sum of
                              frames x coils x ny x nx, stays at or below this (a request is admitted
                              alone whatever its size) */
  double admit_waves;      /* saturation-aware admission: requests are admitted in arrival order while
                              the live requests' normal-operator work per CG iteration -- for each live
                              request, frames x column tiles of its size class's kernel variant, divided
                              by the blocks that variant keeps resident on the device -- is below this
                              many waves (the request that crosses it is admitted; a lone request always
                              is).  Under overload the oldest requests then have the GPU to themselves
                              while later ones wait, instead of every admitted request sharing each tick
                              and all finishing near the end of the backlog.  0: the default, 12 waves;
                              negative: no such limit (admission by budget and max_live only) */
} sense_queue_cfg;

typedef enum {
  SENSE_REQ_PENDING = 0, SENSE_REQ_RUNNING = 1, SENSE_REQ_DONE = 2, SENSE_REQ_CANCELLED = 3,
  SENSE_REQ_FAILED = 4
} sense_req_state;

typedef struct {
  uint64_t submitted, admitted, completed, cancelled, failed, refused;
  uint64_t ticks;
  double p50_ms, p99_ms, mean_ms, max_ms; /* submit -> result ready, completed requests */
  size_t hbm_in_use, hbm_budget;
  int live, pending;
  size_t staging_reserved; /* host staging the queue holds (page-locked chunks of 256 MiB or more) */
  size_t staging_in_use;   /* of which held by requests: inputs until uploaded, outputs until waited for */
} sense_queue_stats;

/* cfg may be NULL (all fields 0).  (Scheduler tests create queues with
 * host-only test hooks through sense_queue_create_with_hooks, declared in
 * sense_testing.h.)  When the environment variable
 * SENSE_QUEUE_LOG names a file, the queue appends one JSON line per request
 * that leaves it (completed, failed or cancelled): id, shape, state, status,
 * submit_ms / admit_ms / first_tick_ms / done_ms (milliseconds since the
 * queue was created; first_tick_ms is the end of the request's first tick),
 * latency_ms, ticks, max_iter, and for completed requests the largest
 * per-frame iteration count and relative residual (null if not finite). */
sense_status sense_queue_create(int device, const sense_queue_cfg* cfg, sense_queue** out);
/* Copies the inputs (host memory, layouts of sense_cg_solve) into pinned
 * staging before returning, large inputs with several threads; the caller's
 * buffers are free on return.  Staging comes from an arena of page-locked
 * chunks that is reused across requests of any shape, so after warm-up a
 * submit allocates nothing.  A request's latency is timed from the start of
 * this call.  A request that could never fit the budget is refused with
 * SENSE_EQUEUE_FULL. */
sense_status sense_queue_submit(sense_queue* q, const sense_shape* shape, const void* y_host, const void* S_host,
                                const int32_t* lines_host, int max_iter, double rel_tol, uint64_t* req_id);
/* Non-blocking state of a request; iters = ticks applied so far. */
sense_status sense_queue_poll(sense_queue* q, uint64_t req_id, int* state, int* iters);
/* Block until the request has finished (or timeout_s > 0 elapsed:
 * SENSE_ETIMEOUT), then copy its image [frames][ny][nx] and, if non-NULL,
 * per-frame iterations / relative residuals / outcomes to host memory and
 * forget the request.  SENSE_ENOTFOUND for unknown ids, SENSE_EINVAL for a
 * cancelled request, SENSE_ENOMEM or SENSE_ECUDA for a request that failed
 * (admission or device work; sense_last_error says which).  SENSE_ENUMERIC
 * when a frame stopped in breakdown with a non-finite residual -- its input
 * held NaN or Inf; the outputs are still copied, and that frame's image is
 * its last finite iterate (zero when b = E^H y itself is not finite). */
sense_status sense_queue_wait(sense_queue* q, uint64_t req_id, sense_c32* x_host, int32_t* iters_host,
                              double* resid_host, int32_t* outcome_host, double timeout_s);
/* Cancel a pending or running request (it stops at the next tick boundary). */
sense_status sense_queue_cancel(sense_queue* q, uint64_t req_id);
sense_status sense_queue_stats_get(sense_queue* q, sense_queue_stats* out);
/* Kernel variant the queue uses for a size class (-1 if none yet). */
int sense_queue_variant(sense_queue* q, int ny, int nx, int storage);
/* Fix the kernel variant of a size class (ny, nx, storage) before its first
 * request is admitted -- e.g. one sense_plan_autotune chose in persistent
 * mode on a representative shape -- instead of variant 0 or tuning on the
 * first request.  SENSE_EINVAL if the class already runs another variant or
 * the variant does not exist for ny. */
sense_status sense_queue_set_variant(sense_queue* q, int ny, int nx, int storage, int variant);
/* Stop the scheduler (running requests are cancelled) and free everything. */
sense_status sense_queue_destroy(sense_queue* q);

/* Root sum of squares (Sec. IV-B): out[f][i] = sqrt(sum_c |F2^H(Z_f y_{f,c})[i]|^2),
 * out: [frames][ny][nx] float. S is not used. */
sense_status sense_rss(sense_plan* plan, const void* y, const int32_t* lines, float* out, void* stream);

/* Convert `count` complex64 values to the bfloat16-pair storage format with
 * round-to-nearest-even (for preparing S and y of a BF16 plan). */
sense_status sense_c32_to_bf16(const sense_c32* in, void* out, size_t count, void* stream);

/* How sense_cg_solve runs its iterations.
 *   1 (default): one persistent launch runs every iteration of every frame.
 *     Blocks take work items (a normal-operator column tile or an update
 *     chunk of one frame and iteration) from a global ticket counter in a
 *     fixed order; an item waits only for the previous phase of its own
 *     frame, so frames pipeline and no kernel boundary separates phases.
 *   0: two kernels per iteration (normal operator, update), captured once
 *     per argument set into a CUDA graph and replayed.
 *   2: the same two kernels per iteration launched directly, no graph (the
 *     plain per-instance loop that batching and serving are measured
 *     against).
 * Both give the same iterates up to rounding of the inner products' partial
 * sums (the per-tile and per-chunk partitions differ). */
sense_status sense_plan_set_cg_mode(sense_plan* plan, int mode);

/* How E, E^H, the CG start and root-sum-of-squares run their two passes (the
 * x-direction transforms of the sampled rows, and the y-direction transforms
 * with the maps, line mask and coil sum):
 *   2: both passes in ONE persistent launch for square images whose
 *     length has a TMA column pass (below): row tiles and column tiles of
 *     the frames are handed out in a frame-staggered order, a column tile
 *     waits (bounded) for its frame's row tiles, and the row-transformed
 *     intermediate of only a couple of frames is live at a time, so it stays
 *     in L2 and one frame's row work overlaps another frame's column work.
 *     Measured slower than mode 1 at every shape tried (the column work is
 *     bound by its instruction stream, not by the intermediate's traffic, and
 *     the dynamic schedule adds waits), so it is not the default;
 *   1 (default): two launches, the column pass a persistent kernel that loops over
 *     (frame, 8-column tile) items and stages each coil's map tile and
 *     k-space tile in shared memory by TMA one coil ahead, for every length
 *     from 64 up whose 8-column tile fills whole warps;
 *   0: two launches, the column pass per-tile kernels (one block per
 *     frame and column tile, tiles loaded through registers).
 * Shapes a mode does not cover fall back to the next lower one.  All give the
 * same results up to the rounding order of the coil sums. */
sense_status sense_plan_set_column_pass(sense_plan* plan, int staged);

/* Kernel variants.  Each transform length has one or more compiled variants
 * of the normal-operator kernel (threads per column, columns per block,
 * radix schedule, register cap).  A plan starts with variant 0.
 * sense_plan_set_variant selects one (SENSE_EINVAL if it does not exist for
 * the plan's ny); sense_plan_variant reports the current one. */
sense_status sense_plan_set_variant(sense_plan* plan, int variant);
int sense_plan_variant(const sense_plan* plan);

/* Tikhonov regularisation of this plan's CG solves: sense_cg_solve then
 * solves (E^H E + lambda I) x = E^H y per frame, the same Hestenes-Stiefel
 * iteration with q = E^H E p + lambda p (the paper's method is lambda = 0,
 * the default).  lambda must be finite, >= 0 and representable in FP32
 * (the kernels use it in FP32), else SENSE_EINVAL.  sense_normal is not
 * affected.  Synchronises the device when lambda changes (captured CG
 * graphs are rebuilt). */
sense_status sense_plan_set_lambda(sense_plan* plan, double lambda);

/* Temporal regularisation of this plan's CG over its frames, treated as a
 * cyclic (cine) series: with lambda_t > 0, sense_cg_solve runs ONE CG over
 * all frames on (E^H E + lambda I + lambda_t L) x = E^H y, L the cyclic
 * second difference across frames ((L x)_f = 2 x_f - x_{f-1} - x_{f+1},
 * frame indices modulo F): the normal equations of ||E x - y||^2 +
 * lambda ||x||^2 + lambda_t sum_f ||x_f - x_{f-1}||^2.  The scalars, the
 * stopping test (on the residual of the whole series) and the per-frame
 * outputs (iterations, residual, outcome: equal for every frame) are the
 * series'.  It runs in the persistent CG kernel whatever the CG mode.
 * lambda_t = 0 (the default) keeps the frames independent.  lambda_t must be
 * finite, >= 0 and FP32-representable, else SENSE_EINVAL. */
sense_status sense_plan_set_temporal(sense_plan* plan, double lambda_t);

/* Autotuner: time every variant of the normal-operator kernel on this plan's
 * shape with the caller's S and lines (device pointers), keep the fastest and
 * return it in *variant_out.  What is timed follows the plan's CG mode: in
 * persistent mode (the default) a 10-iteration CG solve with a constant
 * k-space right-hand side, in temporary device buffers the call allocates and
 * frees; in the graph and direct modes one normal-operator launch, with the
 * plan's own CG vectors as scratch.  ms_out (may be NULL) receives the mean
 * milliseconds per timed unit of each variant (kernel variants that do not
 * exist get -1); it must hold 4 values.  Results are cached per (device,
 * shape, storage, timed mode) for the process, and appended to the file named
 * by the environment variable SENSE_AUTOTUNE_CACHE when set (read back on
 * first use).  A cached shape is not re-timed.  Synchronises `stream`;
 * device-flagged errors are reported as by sense_plan_check. */
sense_status sense_plan_autotune(sense_plan* plan, const void* S, const int32_t* lines, int* variant_out,
                                 double* ms_out, void* stream);

/* Synchronise `stream` and report errors the kernels flagged since the last
 * check (SENSE_EDEVICE for bad lines, SENSE_ETIMEOUT for a bounded wait that
 * gave up).  Clears the flags. */
sense_status sense_plan_check(sense_plan* plan, void* stream);

/* Kernel phases timed by the plan's event timers. */
typedef enum {
  SENSE_PHASE_ROWS_FWD = 0, /* E, x-direction pass */
  SENSE_PHASE_ROWS_INV = 1, /* E^H, x-direction pass */
  SENSE_PHASE_FWD_COL = 2,  /* E, y-direction pass with S and the line mask */
  SENSE_PHASE_ADJ_COL = 3,  /* E^H, y-direction pass with conj(S) and the coil sum (also CG start, RSS) */
  SENSE_PHASE_NORMAL = 4,   /* E^H E (sense_normal) */
  SENSE_PHASE_CG_NORMAL = 5,/* E^H E inside CG, with the p update and Re<p,q> */
  SENSE_PHASE_CG_UPDATE = 6,/* CG x/r update with <r,r> */
  SENSE_PHASE_CG_PERSISTENT = 7, /* all CG iterations in one persistent launch */
  SENSE_PHASE_MAPS_TRANSPOSE = 8, /* S -> S^T for kernel variants with lane-major tiles */
  SENSE_PHASE_CG_FINISH = 9,      /* per-frame CG outputs (iterations, residual, outcome) */
  SENSE_PHASE_FWD_FUSED = 10,     /* E, both passes in one launch */
  SENSE_PHASE_ADJ_FUSED = 11,     /* E^H (also CG start, RSS), both passes in one launch */
  SENSE_PHASE_COUNT = 12
} sense_phase;

/* Turn the plan's kernel timers on (1) or off (0); either way the totals
 * are reset.  While on, every launch of the plan is bracketed by a pair of
 * CUDA events recorded on the launching stream, and sense_cg_solve launches
 * its iterations directly instead of replaying a CUDA graph.  Timing is a
 * diagnostic mode: it adds event records between kernels. */
sense_status sense_plan_set_timing(sense_plan* plan, int on);

/* Wait for the timed launches and return, for `phase`, the summed kernel
 * time in milliseconds and the number of launches since timing was turned
 * on.  Either output may be NULL. */
sense_status sense_plan_phase_time(sense_plan* plan, int phase, double* ms_total, long* launches);

/* Self-test of the device-side bounded wait used by the persistent CG
 * kernel: one thread polls a device flag that nothing sets, at most
 * max_spins times (>= 64 ns apart; max_spins in [1, 2^20]), then gives up.
 * Returns SENSE_ETIMEOUT when the wait gave up as designed (the expected
 * outcome), anything else on failure.  The device stays usable. */
sense_status sense_selftest_wait(int device, long max_spins);

/* FP32 throughput of device `device`, measured (diagnostic; the paper has no
 * counterpart): a launch covering every SM at full occupancy runs independent
 * chains of fused multiply-adds, and the best of five timed launches gives
 * *tflops_out = 2 x FMAs / time in TFLOP/s.  This is the measured peak that
 * the transform-bound kernels' ALU roofline is stated against.  Synchronous;
 * takes a few milliseconds; allocates 4 bytes per launched block. */
sense_status sense_fp32_peak(int device, double* tflops_out);

/* Message describing the last non-OK status returned on this thread. */
const char* sense_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SENSE_H */
