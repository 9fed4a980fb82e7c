/*
 * evr.h -- C ABI of the GB300 event-camera intensity-reconstruction library.
 *
 * Method: Reinbacher, Graber, Pock, "Real-Time Intensity-Image Reconstruction for
 * Event Cameras Using Manifold Regularisation", BMVC 2016 (arXiv:1607.06283).
 * A stream of events e^n = (x^n, y^n, theta^n, t^n) (Sec. 3) is integrated packet
 * by packet into the surface of active events t(x,y) (Sec. 3.1) and the data image
 * f (Eq. intensity_update); each packet then runs warm-started primal-dual
 * iterations (Eq. cont_iterates, Eq. update_rules) minimising the generalised
 * Kullback-Leibler data term plus total variation on the event manifold (Eq. 5).
 *
 * Conventions
 *  - Every function returns EVR_OK (0) or a negative EVR_ERR_* code, except
 *    evr_destroy and evr_strerror.
 *  - Images are W x H, row-major, index y*W + x with x the column (0 <= x < W) and
 *    y the row.  Host buffers passed in or out are dense (no padding).
 *  - The library owns all device state.  Input arrays belong to the caller and may
 *    be reused as soon as the call returns (host pointers) or as soon as the work
 *    queued on the handle's CUDA stream has consumed them (device pointers).
 *  - Work is queued on the handle's CUDA stream (its own stream unless
 *    evr_set_cuda_stream chose another).  Calls that return data to the host
 *    synchronise that stream.
 *  - A handle is not thread-safe; distinct handles are independent.
 *  - All computation runs in CUDA kernels for sm_103a; there is no CPU fallback.
 */
#ifndef EVR_H
#define EVR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define EVR_OK 0
#define EVR_ERR_INVALID_ARG (-1)   /* null pointer, bad size, bad parameter */
#define EVR_ERR_OUT_OF_RANGE (-2)  /* an event with x >= W or y >= H */
#define EVR_ERR_BAD_POLARITY (-3)  /* an event with polarity 0 (Sec. 3: theta in {-1, 1}) */
#define EVR_ERR_NONMONOTONIC (-4)  /* a timestamp below its predecessor or the stream clock
                                      (Sec. 3: timestamps increase; equal ones are accepted) */
#define EVR_ERR_OOM (-5)           /* device or pinned host allocation failed */
#define EVR_ERR_CUDA (-6)          /* a CUDA runtime call failed */
#define EVR_ERR_TIMEOUT (-7)       /* reserved: a bounded device-side wait expired */
#define EVR_ERR_NOT_SUPPORTED (-8) /* no usable sm_103a device, or option not built */

/* t_init_us value meaning "never-fired pixels take the first pushed timestamp". */
#define EVR_T_INIT_FIRST INT64_MIN

/* Solver variants (evr_params.solver). */
#define EVR_SOLVER_AUTO 0      /* pick the solver configuration with the autotuner: at
                                  the first solve every candidate is timed once on the
                                  sensor and the six fastest three more times (state
                                  saved and restored); the up to three closest then take
                                  turns on the next nine solves, timed with CUDA events,
                                  and the fastest is kept (evr_solver_settled) */
#define EVR_SOLVER_UNFUSED 1   /* two kernels per iteration (primal step, dual step) */
#define EVR_SOLVER_TILED 2     /* temporally blocked tiles, several iterations per launch */

/* Model and solver parameters.  evr_default_params fills the defaults listed. */
typedef struct {
  float lambda;       /* data weight lambda of Eq. 5; default 90 */
  float delta_pos;    /* Delta+: log step of a positive event (Sec. 3); default 0.15 */
  float delta_neg;    /* Delta-: log step of a negative event (Sec. 3); default 0.15 */
  float u_min;        /* box of Eq. data_term; default exp(-3) */
  float u_max;        /* default exp(3) */
  float u_init;       /* u^0 (unknown in the paper, Sec. 3); default 1 */
  float tau;          /* primal step (Sec. 3.2, tau sigma ||L_g||^2 <= 1 with ||L_g||^2 <=
                         8 + 4 sqrt 2); default (8 + 4 sqrt 2)^-1/2 */
  float sigma;        /* dual step; default (8 + 4 sqrt 2)^-1/2 */
  float time_scale;   /* manifold height per microsecond of time since the last event;
                         default 1e-3 (milliseconds) */
  int64_t t_max_us;   /* clamp of the time since the last event; <= 0 disables;
                         default 100000 */
  int64_t t_init_us;  /* timestamp of never-fired pixels; default EVR_T_INIT_FIRST */
  int data_mode;      /* 0: f = previous image stepped at event pixels (default);
                         1: f persists between packets, stepped at event pixels */
  int manifold;       /* 1: t from the events (default); 0: t = const (Sec. 4.2) */
  int solver;         /* EVR_SOLVER_*; default EVR_SOLVER_AUTO */
  int tile_config;    /* solver configuration index (0 = let the autotuner choose) */
  int storage;        /* format of the dual variable p (between launches) and of the
                         over-relaxed ubar (shared memory): 0 FP32 (default), 1 FP16,
                         2 BF16; arithmetic stays FP32 and both are rounded to the format
                         every iteration.  16-bit formats need the multi-launch tiled
                         solver (not the unfused or persistent ones). */
  int data_term;      /* 0: generalised KL with box [u_min, u_max] (Eq. data_term, default);
                         1: L2 data term of Eq. 7 (ROF on the manifold, no box) */
  int tvl1_iters;     /* iterations of anisotropic TV-L1 denoising of the time surface
                         before the metric (Sec. 4, "a few iterations"); 0 = off (default).
                         Single streams only (evr_batch_create rejects it). */
  float tvl1_lambda;  /* data weight of that denoising; default 1 (removes isolated
                         one-pixel outliers, whose anisotropic TV is 4x their height) */
} evr_params;

typedef struct evr_stream evr_stream; /* opaque handle */

/* Fill *out with the defaults above.  Errors: EVR_ERR_INVALID_ARG if out is NULL. */
int evr_default_params(evr_params* out);

/* Create a stream for a W x H sensor (1 <= W, H <= 65536) on the current CUDA
 * device and allocate its device state: u = u_init, p = 0, no events.
 * Errors: EVR_ERR_INVALID_ARG (null pointers, bad size, lambda <= 0, Delta <= 0,
 * u_min <= 0, u_min >= u_max, u_init outside [u_min, u_max], tau or sigma <= 0,
 * tau sigma (8 + 4 sqrt 2) > 1 + 1e-6, time_scale < 0, bad mode or solver),
 * EVR_ERR_NOT_SUPPORTED (no sm_103a device), EVR_ERR_OOM, EVR_ERR_CUDA.
 * On error *out is set to NULL. */
int evr_create(int W, int H, const evr_params* params, evr_stream** out);

/* Release the device state (synchronises the handle's stream).  NULL is a no-op. */
void evr_destroy(evr_stream* s);

/* Stream selector for evr_set_cuda_stream: the library's own non-blocking stream,
 * which every handle uses until another stream is chosen. */
#define EVR_OWN_STREAM ((void*)(intptr_t)-1)

/* Queue the handle's work on an existing cudaStream_t.  NULL (0) is the legacy
 * default stream (the stream PyTorch calls its default stream); EVR_OWN_STREAM
 * returns to the library's own stream.  Work already queued is waited for first.
 * The library does not take ownership. */
int evr_set_cuda_stream(evr_stream* s, void* cuda_stream);

/* Integrate one packet of n events (Sec. 3 and 3.1): for each event
 * t_last(x,y) = max(t_last(x,y), t), n+(x,y) or n-(x,y) += 1, clock = max(clock, t).
 * Host arrays, structure of arrays: x[n], y[n] (uint16), t_us[n] (int64,
 * microseconds, non-decreasing and not below the stream clock), pol[n] (int8,
 * > 0 positive, < 0 negative, 0 invalid).  The whole packet is validated before any
 * state changes; a rejected packet changes nothing and the code is that of its
 * first invalid event (checked in the order range, polarity, time).  The host
 * checks what it can at once and returns the code; the device repeats the full
 * check.  n = 0 is a no-op.  The arrays are copied before the call returns. */
int evr_push_events(evr_stream* s, const uint16_t* x, const uint16_t* y, const int64_t* t_us,
                    const int8_t* pol, size_t n);

/* As evr_push_events, with device pointers; validation runs on the device only, and
 * a rejection is reported by the next call that synchronises (evr_synchronize,
 * evr_get_image, evr_get_state, evr_gap).  The arrays must stay valid until the
 * queued work has run. */
int evr_push_events_device(evr_stream* s, const uint16_t* x, const uint16_t* y,
                           const int64_t* t_us, const int8_t* pol, size_t n);

/* Solve the current packet: time surface t = time_scale * min(clock - t_last, t_max)
 * (Sec. 3.1), metric (Eq. 2, Eq. 3), data image f (Eq. intensity_update, one factor
 * c1 = exp(Delta+) or c2 = exp(-Delta-) per event, compounded), reset of the event
 * counts, then `iters` primal-dual iterations (Eq. cont_iterates with Eq.
 * update_rules) warm-started from the previous (u, p).  Asynchronous.
 * Errors: EVR_ERR_INVALID_ARG (iters < 0), EVR_ERR_CUDA. */
int evr_solve(evr_stream* s, int iters);

/* Push and solve in one call: the same as evr_push_events_device(s, x, y, t_us, pol, n)
 * followed by evr_solve(s, iters), with the same results.  Once the solver is settled
 * (after the autotuner and its refinement, multi-launch solvers, packets of at most 32768
 * events) the push, the packet's front launches and its iteration kernels run as one
 * CUDA graph, the prologue starting as a programmatic dependent of the push; otherwise
 * the two calls are made.  Asynchronous; errors as the two calls. */
int evr_step_device(evr_stream* s, const uint16_t* x, const uint16_t* y, const int64_t* t_us,
                    const int8_t* pol, size_t n, int iters);

/* The same with host arrays: evr_push_events followed by evr_solve, with the same checks
 * and results.  The packet is packed into one of the handle's pinned staging slots and
 * copied, on a library-owned copy stream, into that slot's device buffer while the
 * earlier packets still solve; the packet's graph (push, front launches, iteration
 * kernels) waits for the copy on the handle's stream.  The arrays may be reused when the
 * call returns.  Errors: as evr_push_events (nothing is queued on a rejected packet or
 * EVR_ERR_OOM), EVR_ERR_CUDA. */
int evr_step(evr_stream* s, const uint16_t* x, const uint16_t* y, const int64_t* t_us,
             const int8_t* pol, size_t n, int iters);

/* Copy the current image u (W*H floats, row-major) to host memory; synchronises.
 * len is the capacity of out_host in floats and must be >= W*H.  Returns the first
 * pending device-side rejection, if any, else EVR_OK. */
int evr_get_image(evr_stream* s, float* out_host, size_t len);

/* Copy the current image into device memory out_dev (W*H floats, dense row-major);
 * asynchronous, on the handle's stream. */
int evr_get_image_device(evr_stream* s, float* out_dev, size_t len);

/* Asynchronous readback of the current image (real-time pipelines: the caller can queue
 * the next packet while this one is solved and copied).  Queues the copy of u (W*H
 * floats, row-major, as evr_get_image) into out_host and returns at once with a ticket
 * (> 0) in *ticket: on the handle's CUDA stream, in order with the solves, u is copied
 * into one of three library-owned device staging images; the copy to the host then
 * runs on a library-owned stream, overlapping the next packets' kernels, and completes
 * at evr_wait_image(ticket) (not at a synchronisation of the handle's stream).  out_host must stay valid and unread
 * until evr_wait_image(ticket) has returned; page-locked memory (cudaHostAlloc, pinned
 * tensors) keeps the copy asynchronous, pageable memory makes the CUDA runtime wait for
 * it here.  At most 16 readbacks are in flight: the 17th waits for the oldest.  Errors:
 * EVR_ERR_INVALID_ARG (null pointer, len < W*H), EVR_ERR_OOM, EVR_ERR_CUDA. */
int evr_get_image_async(evr_stream* s, float* out_host, size_t len, uint64_t* ticket);

/* Wait until the readback `ticket` (and all work queued before it) has completed.
 * Returns EVR_OK, or, when a device-side rejection was pending at that point, that
 * code after clearing it as evr_synchronize does (a rejected packet left the state
 * unchanged; the image is valid).  EVR_ERR_INVALID_ARG for a ticket not issued. */
int evr_wait_image(evr_stream* s, uint64_t ticket);

/* State planes for tests and checkpoints (dense row-major, W*H elements). */
#define EVR_STATE_U 0       /* float */
#define EVR_STATE_P1 1      /* float, dual variable p, component 1 */
#define EVR_STATE_P2 2      /* float */
#define EVR_STATE_P3 3      /* float */
#define EVR_STATE_F 4       /* float, data image of the last solve */
#define EVR_STATE_TLAST 5   /* int64, never-fired pixels report t_init */
#define EVR_STATE_NPOS 6    /* int32, positive events since the last solve */
#define EVR_STATE_NNEG 7    /* int32 */
#define EVR_STATE_CLOCK 8   /* int64[1], latest timestamp */
#define EVR_STATE_TINIT 9   /* int64[1], timestamp of never-fired pixels (0 if unset) */
#define EVR_STATE_SQRTG 10  /* float, sqrt(G) of the last solve */
#define EVR_STATE_TX 11     /* float, L_x t of the last solve (Eq. 3) */
#define EVR_STATE_TY 12     /* float, L_y t of the last solve */

/* Copy a state plane to host memory (bytes = its exact size); synchronises.
 * Returns the first pending device-side rejection, if any. */
int evr_get_state(evr_stream* s, int which, void* out_host, size_t bytes);

/* Overwrite a state plane from host memory, with the layout evr_get_state returns:
 * u, p1, p2, p3, f (float), t_last (int64; a never-fired pixel may hold t_init), n+, n-
 * (int32), clock and t_init (int64[1]; writing t_init marks it as set).  With the
 * values read from another stream after at least one event, this restores a
 * checkpoint: the restored stream continues bit-identically.  The metric planes are
 * recomputed by every solve and cannot be written.  Synchronises. */
int evr_set_state(evr_stream* s, int which, const void* in_host, size_t bytes);

/* Primal energy of Eq. 5 and the dual value of the saddle form (Eq.
 * primal_dual_energy) of the current (u, p) under the last solve's metric and f,
 * reduced on the device in FP64 (fixed reduction order: deterministic).  The gap
 * primal - dual >= 0 is the convergence check.  Synchronises. */
int evr_gap(evr_stream* s, double* primal, double* dual);

/* Largest image (W*H pixels) that evr_gap_static accepts. */
#define EVR_GAP_STATIC_MAX_PIXELS 4194304

/* The FP64 primal energy and dual value of evr_gap, computed from caller-provided
 * device planes without allocating any device memory.  The paper has no counterpart:
 * it exists for callers that may not allocate once they are running -- a real-time
 * loop that cannot afford cudaMalloc's implicit device synchronisation, or a host
 * application that owns all device memory through its own pool.
 *   u, p1, p2, p3, f, tx, ty: device planes of H rows of `pitch` FP32 values (pitch >= W,
 *     row-major, x the column), as read back from a stream (u, p, f, L_x t, L_y t);
 *     each must hold at least pitch*H floats;
 *   lambda, u_min, u_max: the model's parameters;
 *   data_term: 0 the generalised KL term with the box [u_min, u_max] (Eq. 5), 1 the L2
 *     term of Eq. 7 (no box; u_min, u_max still validated, otherwise unused) -- the
 *     value of evr_params.data_term of the stream the planes come from;
 *   out_dev: device memory for 2 doubles, receives {primal, dual};
 *   cuda_stream: cudaStream_t to queue on (NULL: the legacy default stream).
 * Asynchronous.  The reduction's scratch is one fixed 24 KiB device array inside the
 * library (held by every GPU that loads it until the process exits) and shared by
 * all calls: each call overwrites the partials it uses before reading them, and calls
 * whose work overlaps on the GPU race on it.  The first call on a device looks up
 * the array's address and caches it; make that first call before any stream
 * capture.  A device reset (cudaDeviceReset) invalidates the cached address: do not
 * call the entry point on a device after resetting it.  Errors: EVR_ERR_INVALID_ARG
 * (null pointer, W or H <= 0, pitch < W, W*H > EVR_GAP_STATIC_MAX_PIXELS, lambda <= 0,
 * bad box, data_term not 0 or 1), EVR_ERR_CUDA. */
int evr_gap_static(const float* u, const float* p1, const float* p2, const float* p3,
                   const float* f, const float* tx, const float* ty, int W, int H, int pitch,
                   float lambda, float u_min, float u_max, int data_term, double* out_dev,
                   void* cuda_stream);

/* ---- measurement support (the paper has no counterpart) ----
 * Measured bandwidth of one memory level of this GPU, the denominator of a roofline:
 *   level 0: L2 -- a copy between two 16 MiB device buffers that stay resident in L2,
 *            bytes read + written per second;
 *   level 1: shared memory -- conflict-free 16-byte reads by one 1024-thread CTA per SM,
 *            aggregate over all SMs (a kernel on k SMs is bounded by k / SMs of it).
 * *gbs receives GB/s (1e9 bytes per second), the best of five timed launches (CUDA
 * events on cuda_stream, NULL: the legacy default stream) after one warm-up.
 * Allocates and frees 32 MiB of device memory (level 0) or a few bytes (level 1) and
 * synchronises.  Errors: EVR_ERR_INVALID_ARG (null gbs, unknown level), EVR_ERR_OOM,
 * EVR_ERR_CUDA. */
int evr_measure_peak(int level, double* gbs, void* cuda_stream);

/* ---- batching: many independent streams solved together ----
 * A batch holds n streams of possibly different sizes sharing one evr_params.  A step
 * takes at most one packet per stream (streams with no events in the step are left
 * untouched), validates and integrates every packet (one CTA per stream), then runs
 * the packet prologue and `iters` iterations for every stream that had events, as one
 * CUDA graph over a (stream, tile) work list, cut into groups of streams that fit L2
 * (evr_batch_set_grouping).  Each stream's results are bit-identical to a single stream
 * (evr_create) fed the same packets with the same tile_config; the tiled configuration
 * is autotuned over the whole batch at the first step unless tile_config selects one
 * (multi-launch configurations only).  Per-stream packets above 32768 events are
 * rejected with EVR_ERR_INVALID_ARG. */
typedef struct evr_batch evr_batch; /* opaque handle */

/* Create n streams of sizes W[s] x H[s].  Errors as evr_create; EVR_ERR_NOT_SUPPORTED
 * for the unfused solver or a persistent tile_config. */
int evr_batch_create(int n, const int* W, const int* H, const evr_params* params,
                     evr_batch** out);
void evr_batch_destroy(evr_batch* b);
int evr_batch_set_cuda_stream(evr_batch* b, void* cuda_stream);

/* Order of a step's work (results are bit-identical for every setting).  The streams
 * are cut, in index order, into groups whose pass working set ((u, p) of both buffers
 * and the five constant planes, pitch x H pixels each) stays within budget_bytes (a
 * larger stream is a group of its own); the step graph runs each group's prologue and
 * all its iteration passes before the next group, so that the group's state stays in
 * L2 across its passes; with branches = k (1 to 4) group g runs on graph branch g mod k,
 * k groups side by side.  budget_bytes = 0: one group (every pass over all streams);
 * budget_bytes < 0 (the default): chosen with the tiled configuration by the autotuner
 * at the next step with iterations, from 8 to 64 MB and one to four branches, against
 * one group.  Synchronises the batch's stream.  Errors: EVR_ERR_INVALID_ARG (null
 * handle, branches outside 1..4), EVR_ERR_CUDA. */
int evr_batch_set_grouping(evr_batch* b, long long budget_bytes, int branches);

/* How a step runs once the tiled configuration is chosen.
 *   EVR_BATCH_SCHEDULE_GRAPH: one push launch, then a CUDA graph of launches (per group
 *     of streams the prologue and each iteration pass over the group's (stream, tile)
 *     work list).
 *   EVR_BATCH_SCHEDULE_PERSISTENT: the whole step -- every stream's push, prologue and
 *     iteration passes -- is one persistent launch, captured as a one-node CUDA graph
 *     whose arguments take each step's packets.  The grid holds as many CTAs as are
 *     resident at once; they take (stream, item) work items in list order from a queue
 *     and wait, bounded, until the item's stream has completed the items it depends on
 *     (every tile runs the update rules of Eq. update_rules exactly as the tiled
 *     passes do).  The items of a window of streams whose pass working set fits the
 *     grouping budget (evr_batch_set_grouping; 0: every stream) are listed pass after
 *     pass, so the window's state stays in L2.  Tiles of 32 x 32 and 32 x 48 pixels only
 *     (tile_config 1-5, 28-32, 35-42).  A wait that runs out (0.2 s) ends the launch
 *     and is reported as EVR_ERR_TIMEOUT by evr_batch_synchronize.
 *   EVR_BATCH_SCHEDULE_AUTO (the default): the autotuner times both with the chosen
 *     configuration (and the persistent one over window budgets and its tiles) at the
 *     next step with iterations and keeps the faster.
 * Results are bit-identical under every schedule.  Synchronises the batch's stream.
 * Errors: EVR_ERR_INVALID_ARG (null handle, unknown schedule), EVR_ERR_CUDA. */
#define EVR_BATCH_SCHEDULE_AUTO (-1)
#define EVR_BATCH_SCHEDULE_GRAPH 0
#define EVR_BATCH_SCHEDULE_PERSISTENT 1
int evr_batch_set_schedule(evr_batch* b, int schedule);
/* The schedule steps use now (GRAPH or PERSISTENT; GRAPH before the first tuning). */
int evr_batch_get_schedule(evr_batch* b, int* schedule);

/* One step.  Events of all streams concatenated (structure of arrays, device
 * pointers); stream s owns events [offsets[s], offsets[s+1]) (offsets: device int64
 * array of n+1 entries, offsets[0] = 0, non-decreasing).  Validation is per stream
 * and device-side: a rejected packet changes nothing of its stream and is reported by
 * evr_batch_synchronize.  Asynchronous. */
int evr_batch_step_device(evr_batch* b, const uint16_t* x, const uint16_t* y,
                          const int64_t* t_us, const int8_t* pol, const int64_t* offsets,
                          int iters);

/* As evr_batch_step_device with host arrays (offsets on the host); the events are
 * copied into library-owned pinned memory before the call returns (one of two slots;
 * a slot is reused once its host-to-device copy has completed), then moved to the
 * device with one copy. */
int evr_batch_step(evr_batch* b, const uint16_t* x, const uint16_t* y, const int64_t* t_us,
                   const int8_t* pol, const int64_t* offsets, int iters);

/* Image / state plane of stream s (as evr_get_image / evr_get_state); synchronise. */
int evr_batch_get_image(evr_batch* b, int s, float* out_host, size_t len);
/* All images, stream after stream, each W[s]*H[s] floats row-major; synchronises.
 * len is the capacity of out_host in floats.  A device kernel gathers the images into
 * one buffer (allocated at the first readback), then one copy moves them. */
int evr_batch_get_images(evr_batch* b, float* out_host, size_t len);
/* Asynchronous form, as evr_get_image_async: queues the gather (into one of two
 * library-owned staging buffers, on the batch's stream) and the copy into out_host (on
 * a library-owned stream; page-locked memory for an asynchronous copy) and returns a
 * ticket (> 0); at most 16 in flight.  evr_batch_wait_images(ticket) waits for that copy (EVR_OK,
 * EVR_ERR_CUDA, EVR_ERR_INVALID_ARG for a ticket not issued); rejected packets are
 * reported by evr_batch_synchronize. */
int evr_batch_get_images_async(evr_batch* b, float* out_host, size_t len, uint64_t* ticket);
int evr_batch_wait_images(evr_batch* b, uint64_t ticket);
int evr_batch_get_state(evr_batch* b, int s, int which, void* out_host, size_t bytes);

/* Wait; return the first pending rejection (lowest stream index, written to
 * *stream_out if not NULL, -1 if none) and clear all pending rejections. */
int evr_batch_synchronize(evr_batch* b, int* stream_out);

/* Kernel timing of the steps' graphs (per group the prologue and the iteration passes;
 * the buffer flip), as evr_enable_kernel_timing / evr_kernel_time; launches counts
 * every kernel of the graphs; pixel_iters counts every stream as active in every timed
 * step. */
int evr_batch_enable_kernel_timing(evr_batch* b, int enable);
int evr_batch_kernel_time(evr_batch* b, double* ms, int64_t* launches, int64_t* pixel_iters);
const char* evr_batch_solver_name(evr_batch* b);

/* Self-test of the persistent step's bounded waits: one timing run of the current
 * configuration's passes (reading the live state, writing only the other buffer) in
 * which one work item waits for a count its stream never reaches; its wait runs out,
 * every other CTA leaves at its next item or poll, and the last CTA resets the control
 * words.  Returns the status the launch reported (EVR_ERR_TIMEOUT when detection
 * works) after checking that the control words were reset (EVR_ERR_CUDA if not);
 * EVR_ERR_NOT_SUPPORTED when the batch's tile has no persistent form.  Takes about
 * 0.2 s; synchronises. */
int evr_batch_selftest_persist_timeout(evr_batch* b);

/* ---- differentiation of one packet's solve (no counterpart in the paper's text:
 * the adjoint of its iteration, Eq. cont_iterates with Eq. update_rules) ----
 * The solve is u_K = S(u_0, p_0, f, lambda) with the metric fixed: K unrolled
 * iterations.  The calls below are stateless and allocate nothing: every plane is
 * caller-owned device memory of H rows of `pitch` floats (pitch >= W, x the column).
 * The unrolled calls take n >= 1 independent images of the same W x H at once (one
 * packet solve each, lambda shared): a scalar field is n such planes back to back
 * ((n, H, pitch) contiguous), a dual variable p is 3 such fields back to back
 * ((3, n, H, pitch) contiguous, component stride n*pitch*H).  The images are coupled by
 * nothing: image b's result is bit-identical to a call with n = 1 on image b alone.
 * Images of different sizes cannot share a call (one call per size; a caller may pad
 * smaller images into a larger W x H itself, which changes their border terms).  Where
 * pitch is a multiple of 4 (rows of a multiple of 16 bytes) the reverse pass stages its
 * tape slots in shared memory by tensor copies; otherwise it reads them directly (same
 * results).
 * tx, ty are L_x t, L_y t of the packet (evr_get_state EVR_STATE_TX / EVR_STATE_TY).
 * All work is queued on cuda_stream (NULL: legacy default stream).  Errors:
 * EVR_ERR_INVALID_ARG (null pointer, W or H <= 0, pitch < W, n < 1, n*H > 524280,
 * n*H*pitch >= 2^31, K < 1, every < 1), EVR_ERR_CUDA. */

/* Workspace bytes for evr_unrolled_forward/backward (0 for invalid sizes). */
size_t evr_unrolled_workspace_bytes(int W, int H, int pitch, int n, int K, int every);

/* K iterations from (u0, p0), storing (u, p) checkpoints every `every` iterations in
 * `workspace`; result in u_out, p_out.  The iterations are the solver's tiled FP32 passes
 * (MUFU reciprocal square root and reciprocal, a few ulp); the last checkpoint segment's
 * passes also write that segment's tape (p, v and ubar of every iteration) to the
 * workspace.  evr_unrolled_backward recomputes the other segments with the same
 * arithmetic, so it sees the same states bit for bit for any checkpoint spacing; with
 * every >= K it recomputes nothing (the workspace then holds the whole tape,
 * 5 planes per iteration; with every < K it holds the last segment's tape and a second
 * tape of `every` iterations for the recomputation). */
int evr_unrolled_forward(const float* tx, const float* ty, const float* f, const float* u0,
                         const float* p0, int W, int H, int pitch, int n, float lambda,
                         float tau, float sigma, float u_min, float u_max, int K, int every,
                         void* workspace, float* u_out, float* p_out, void* cuda_stream);

/* Reverse mode after evr_unrolled_forward with the same arguments and workspace:
 * from gu_K = dL/du_K and gp_K = dL/dp_K (NULL means 0), walk the adjoint back one
 * checkpoint segment at a time, last segment first, on tiled passes of a few iterations
 * each.  Each segment but the last (whose tape the forward wrote) is first recomputed
 * from its checkpoint into a second tape area of the workspace (p, v and ubar of every
 * iteration).  The checkpoints and the forward's tape are only read, so the call may be
 * repeated.  Outputs: gu0 = dL/du0 and gp0 =
 * dL/dp0 (either may be NULL), gf = dL/df, and glambda_dev[0] = dL/dlambda summed over
 * the n images (device double: FP32 sums over each reverse tile's pixels per iteration,
 * reduced in FP64 in a fixed order).  Clamped pixels and the projection are
 * differentiated on their active side; 1/|p| and 1/s of the KL root are MUFU reciprocal
 * square roots (a few ulp). */
int evr_unrolled_backward(const float* tx, const float* ty, const float* f, int W, int H,
                          int pitch, int n, float lambda, float tau, float sigma, float u_min,
                          float u_max, int K, int every, void* workspace, const float* gu_K,
                          const float* gp_K, float* gu0, float* gp0, float* gf,
                          double* glambda_dev, void* cuda_stream);

/* Launch accounting of the differentiation calls, for benchmarks (process-wide, not
 * thread-safe).  evr_unrolled_timing_start clears the counters and starts counting every
 * kernel that evr_unrolled_forward/backward and evr_data_image(_backward) launch, and
 * recording a CUDA event pair on the call's stream around each of the first 16384
 * reverse-pass launches (the tiled kernel that walks the adjoint back a few iterations at a
 * time).  evr_unrolled_timing_stop waits for the recorded events and returns their summed
 * device time in ms, the number of recorded reverse-pass launches, their reversed
 * pixel-iterations and pixels x launches (for algorithmic byte counts), and the number of
 * all launches; then it stops.  Errors: EVR_ERR_OOM, EVR_ERR_CUDA, EVR_ERR_INVALID_ARG
 * (null pointer). */
int evr_unrolled_timing_start(void);
int evr_unrolled_timing_stop(double* rev_ms, long long* rev_launches, long long* rev_px_iters,
                             long long* rev_px_launches, long long* launches);

/* Data image f = u_prev exp(Delta+ n+ - Delta- n-) (Eq. intensity_update, one factor
 * per event, compounded) from the packet's event counts. */
int evr_data_image(const float* u_prev, const int32_t* npos, const int32_t* nneg, int W, int H,
                   int pitch, float delta_pos, float delta_neg, float* f_out,
                   void* cuda_stream);

/* Its backward: g_uprev = dL/du_prev (may be NULL) and g_delta_dev[0..1] =
 * (dL/dDelta+, dL/dDelta-) in FP64 from gf = dL/df.  scratch: caller-owned device
 * memory of 2*pitch*H + 1024 doubles. */
int evr_data_image_backward(const float* f, const float* u_prev, const int32_t* npos,
                            const int32_t* nneg, int W, int H, int pitch, float delta_pos,
                            float delta_neg, const float* gf, float* g_uprev, double* scratch,
                            double* g_delta_dev, void* cuda_stream);

/* Wait for the handle's queued work; returns the first pending device-side
 * rejection (then clears it), EVR_ERR_CUDA, or EVR_OK. */
int evr_synchronize(evr_stream* s);

/* Kernel timing with CUDA events on the handle's stream around each solve's device
 * work (enable = 1 starts and clears, 0 stops): the packet's front launches (TV-L1 of
 * the time surface when enabled, the prologue) and its iteration kernels, which a
 * tuned multi-launch solve runs as one graph.  The first solve of a handle runs its
 * front launches and the autotuner before the timed region.  evr_kernel_time
 * synchronises and reports the total milliseconds, the number of kernel launches in
 * the timed regions and the pixel-iterations performed since timing was enabled. */
int evr_enable_kernel_timing(evr_stream* s, int enable);
int evr_kernel_time(evr_stream* s, double* ms, int64_t* launches, int64_t* pixel_iters);

/* Failure-detection self-test of the persistent solver's bounded waits (the paper has
 * no counterpart).  Launches it once over the current state with one CTA that never
 * publishes its progress flag: its neighbours' waits run out, set an abort flag that
 * every other CTA polls, and record EVR_ERR_TIMEOUT; all CTAs return.  The stream's
 * (u, p) are restored and its flags cleared afterwards, so it stays usable.  Returns
 * the status the device reported (EVR_ERR_TIMEOUT when detection works),
 * EVR_ERR_NOT_SUPPORTED when no persistent configuration fits the sensor.  Takes well
 * under a second.  Synchronises. */
int evr_selftest_wait_timeout(evr_stream* s);

/* Self-test of the cluster solver's bounded waits (the paper has no counterpart): runs
 * a few iterations of a cluster configuration (kind 3, at least two CTAs, one that fits
 * the sensor) in which one CTA of every cluster never sends its edges, so its
 * neighbours' waits run out; the state is saved first and restored afterwards.
 * Returns the status the device reported (EVR_ERR_TIMEOUT when detection works),
 * EVR_ERR_NOT_SUPPORTED when no cluster configuration fits the sensor.  Takes well
 * under a second.  Synchronises. */
int evr_selftest_cluster_wait_timeout(evr_stream* s);

/* Self-test of the resident solver's bounded grid-barrier wait (the paper has no
 * counterpart): sets the barrier's arrival count far below any target, then runs two
 * barrier intervals of a resident configuration (kind 5, at least two CTAs, one that fits
 * the sensor): every CTA's first wait runs out, one sets the abort flag the others poll,
 * the status records EVR_ERR_TIMEOUT and all CTAs return.  The state is saved first and
 * restored afterwards and the barrier words are cleared, so the stream stays usable.
 * Returns the status the device reported (EVR_ERR_TIMEOUT when detection works),
 * EVR_ERR_NOT_SUPPORTED when no resident configuration fits the sensor.  Takes well under
 * a second.  Synchronises. */
int evr_selftest_resident_wait_timeout(evr_stream* s);

/* Fault injection for tests (the paper has no counterpart): the n-th library
 * allocation of device or page-locked host memory after this call fails as if memory
 * were exhausted (the calls that make it then return EVR_ERR_OOM or EVR_ERR_CUDA and
 * release what they had allocated); n <= 0 disables.  Returns EVR_OK. */
int evr_test_fail_alloc_after(int n);

/* Description of the solver in use, e.g. "tiled 32x32 R4" or "cluster 4x4 of 32x32 R0";
 * static storage. */
const char* evr_solver_name(evr_stream* s);

/* 1 when the solver configuration is settled (EVR_SOLVER_AUTO: the first solve has tuned
 * and the online refinement over the next solves has decided; fixed configurations:
 * always), 0 while later solves may still change it, EVR_ERR_INVALID_ARG for a null
 * handle. */
int evr_solver_settled(evr_stream* s);

/* Static description of a return code. */
const char* evr_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
