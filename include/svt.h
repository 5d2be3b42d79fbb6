/*
 * svt.h -- C ABI of the GB300 SVT track-fitting library (libsvt.so).
 *
 * The chain follows arXiv:1312.0917, Sec. II and Sec. II-A: unpack the packed
 * input words into roads, form every combination of one hit per silicon layer
 * in each road, run the linearised fixed-point fit p_i = f_i . x_i + q_i and
 * the fit's chi-square, then keep the combinations that pass the chi-square
 * cut and survive the hit-warrior.  Where the paper is silent the library
 * fixes the reading; each one is stated at the call that uses it.
 *
 * Conventions for every call:
 *  - Returns SVT_OK (0) or a negative SVT_E_* code; svt_strerror names it.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls only enqueue work on it unless they say they synchronise.
 *  - Device pointers are plain CUDA device addresses owned by the caller (for
 *    example torch tensors); the library never frees them.  The context owns
 *    its own device scratch, sized once by svt_create from svt_limits.
 *  - One context serves one stream at a time; use one context per concurrent
 *    stream.  Calls on one context are not thread-safe.
 *  - Kernels never trap: errors found on the device are written to a device
 *    status word and returned by the next svt_get_tracks / svt_get_stats.
 */
#ifndef SVT_H
#define SVT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SVT_OK            0
#define SVT_E_INVAL      (-1)  /* bad argument (NULL, misaligned, out of range) */
#define SVT_E_BADWORD    (-2)  /* a word breaks the format or the road grammar */
#define SVT_E_TRUNCATED  (-3)  /* the stream does not end at an event boundary */
#define SVT_E_LIMIT      (-4)  /* > 8 hits on a layer of a road or > 256 roads in an event */
#define SVT_E_CAPACITY   (-5)  /* the batch exceeds the context limits or the caller's buffer */
#define SVT_E_CUDA       (-6)  /* a CUDA runtime call failed */
#define SVT_E_TIMEOUT    (-7)  /* a bounded device-side wait gave up */
#define SVT_E_STATE      (-9)  /* call out of order (no constants, nothing unpacked) */

/* ---- execution modes of svt_fit_events ---------------------------------- */
#define SVT_PLAIN       0  /* one kernel per stage, per-combination results in HBM */
#define SVT_PERSISTENT  1  /* one persistent fused kernel, device work queues */

typedef struct svt_ctx svt_ctx;

/* One constant set (Sec. II: "f_i and q_i are pre-defined constant sets"),
 * looked up per road by s = (wedge * 6 + barrel) * 5 + excluded_layer.
 * F and q give the track parameters, C and k the chi-square components:
 *   x   = (hits of the 4 layers other than the excluded one, ascending layer,
 *          then XFT curvature, then XFT phi)
 *   p_i = floor((sum_j F[i][j] x_j) / 4096) + q[i]
 *   a_k = floor((sum_j C[k][j] x_j) / 4096) + k[k],  chi2 = sum_k a_k^2
 * 96 bytes, no padding. */
typedef struct {
    int16_t F[3][6];
    int32_t q[3];
    int16_t C[3][6];
    int32_t k[3];
} svt_const_set;

/* One surviving combination (a fitted track).  40 bytes. */
typedef struct {
    uint32_t event;   /* event index in the batch (order of EE words) */
    uint16_t road;    /* road index within the event (order of EP words) */
    uint16_t comb;    /* combination: sum_l d_l * S_l, S_0 = 1,
                         S_l = S_{l-1} * n_{l-1}; layer 0 varies fastest */
    int32_t p[3];     /* d0, phi, pT (fixed point) */
    uint32_t pad;     /* zero */
    int64_t chi2;
    uint64_t hits;    /* coordinate on layer l in bits 12l .. 12l+11 */
} svt_track;

/* One unpacked road (svt_get_roads).  100 bytes, no hidden padding. */
typedef struct {
    uint32_t event;          /* event index in the batch */
    uint16_t road;           /* road index within the event */
    int16_t curv, phi;       /* XFT track */
    uint8_t wedge, barrel, excl;
    uint8_t n[5];            /* hits per layer */
    uint8_t pad[2];
    uint16_t coord[5][8];    /* coordinate of hit d on layer l (0 beyond n) */
} svt_road;

/* Capacity of a context (0 in a field = its default). */
typedef struct {
    uint64_t max_words;      /* words per batch            (default 1 << 24, below 1 << 31) */
    uint32_t max_events;     /* events per batch           (default 1 << 16) */
    uint32_t max_roads;      /* roads per batch            (default 1 << 20) */
    uint64_t max_tracks;     /* surviving tracks per batch (default 1 << 22) */
    uint32_t hash_slots;     /* cross-road group table, power of 2 (default 1 << 22); a batch
                                may fill 3/4 of it, each group within 64 slots of its home
                                slot, else SVT_E_CAPACITY */
    uint32_t pad;
    uint64_t max_combinations; /* SVT_PLAIN per-combination buffers (default 1 << 26) */
} svt_limits;

/* Counters of the last batch (svt_get_stats). */
typedef struct {
    uint64_t n_events;        /* complete events */
    uint64_t n_roads;         /* roads of complete events */
    uint64_t n_combinations;  /* sum over roads of prod_l n_l ("fits") */
    uint64_t n_passing;       /* combinations with chi2 <= cut */
    uint64_t n_tracks;        /* survivors of the hit-warrior */
    int32_t status;           /* SVT_OK or the batch's error code */
    uint32_t n_groups;        /* distinct cross-road groups published to the group table */
    uint64_t error_word;      /* word position of the first fault (if any) */
    uint64_t phase_ns[6];     /* SVT_PERSISTENT: device time of each stage, from the
                                 first CTA's view of the grid barriers: word scan,
                                 event scatter, unpack, fit + cut + road-local
                                 warrior, cross-road warrior, output (to the last
                                 CTA's exit); 0 when a stage did not complete, and
                                 for SVT_PLAIN */
} svt_stats;

/* Create a context on `device` (cudaSetDevice is called).  Allocates all
 * device scratch for `lim` (NULL = defaults).  *out = NULL on failure. */
int svt_create(svt_ctx **out, int device, const svt_limits *lim);

/* Free the context and its device memory (synchronises the device). */
void svt_destroy(svt_ctx *ctx);

/* Copy n_sets (must be 360 = 12 wedges x 6 barrels x 5 excluded layers)
 * constant sets from HOST memory to the device and set the chi-square cut:
 * a combination passes iff chi2 <= chi2_cut.  Rejects (SVT_E_INVAL) a set
 * whose values could overflow the exact 32-bit accumulation or the 38-bit
 * chi-square of the track key: per row, sum_j |coef_j| * max|x_j| +
 * 4096 * |offset| must stay below 2^31 (hits <= 4095, curvature and phi
 * <= 32768) and sum_k (bound_k / 4096 + 1)^2 below 2^38.  Enqueued on
 * `stream`; the host copy is done when the call returns. */
int svt_load_constants(svt_ctx *ctx, const svt_const_set *sets, uint32_t n_sets,
                       int64_t chi2_cut, void *stream);

/* Sec. II-A, first function: unpack a batch.  d_words: DEVICE pointer to
 * n_words packed 32-bit words, 4-byte aligned, owned by the caller and left
 * unchanged until the batch's svt_get_tracks returns.
 * Word: bit 31 EE (end of event, only with EP), bit 30 EP (end of road),
 * bits 29..27 type (0..4 hit on that layer, 5 curvature, 6 phi, 7 header),
 * bits 26..0 payload (hit: coordinate in bits 11..0; curvature/phi: int16 in
 * bits 15..0; header: wedge 3..0 (<12), barrel 6..4 (<6), excluded layer 9..7
 * (<5)); unused payload bits must be zero.  A road is header, curvature,
 * phi, hits; <= 8 hits per layer, <= 256 roads per event.  The first word that
 * breaks a rule sets the batch status (SVT_E_BADWORD before SVT_E_LIMIT at
 * the same word); a stream not ending in EE is SVT_E_TRUNCATED.
 * The call binds the batch and schedules the unpack stage: in SVT_PLAIN mode
 * it runs as its own kernels inside svt_fit_events (or svt_get_roads), in
 * SVT_PERSISTENT mode inside the fused kernel.  d_words is device memory or
 * page-locked host memory (cudaHostAlloc / cudaMallocHost / registered),
 * which the kernels then read in place over the CPU-GPU link; pageable host
 * memory -> SVT_E_INVAL.  The caller keeps the words unchanged until the
 * batch's svt_get_tracks returns.  n_words > max_words -> SVT_E_CAPACITY. */
int svt_unpack(svt_ctx *ctx, const uint32_t *d_words, size_t n_words, void *stream);

/* Sec. II, second and third functions, plus the selection: every combination
 * of one hit per layer, the fixed-point fit and chi-square, the cut, and the
 * hit-warrior: among one event's passing combinations, t is dropped iff a
 * passing u with a lower key (chi2, road, comb) shares >= 3 hits with t
 * (equal coordinate on the same layer; all five layers count).  Enqueues the
 * work of `mode` on `stream` and returns (asynchronous). */
int svt_fit_events(svt_ctx *ctx, int mode, void *stream);

/* Synchronise `stream`, then copy the batch's surviving tracks, in
 * (event, road, comb) order, to `out` (host or device memory, capacity `cap`
 * records).  *n_out = number of survivors (also when they do not fit, in
 * which case SVT_E_CAPACITY is returned).  Returns the batch status (a
 * device-detected error is returned here with *n_out = 0).  The status block
 * and as many records as the context's previous batch had are copied in one
 * go (one synchronisation when the count does not grow); when the call
 * returns anything but SVT_OK, the contents of `out` are unspecified. */
int svt_get_tracks(svt_ctx *ctx, svt_track *out, size_t cap, size_t *n_out,
                   void *stream);

/* Have the output stage write the surviving tracks straight into `host`
 * (page-locked host memory, cap records, 8-byte aligned; the caller owns
 * it), over the CPU-GPU link, instead of the context's device buffer;
 * svt_get_tracks with out == host then copies nothing.  A batch with more
 * than cap tracks ends with SVT_E_CAPACITY.  host = NULL returns to the
 * device buffer.  SVT_E_INVAL for pageable or unaligned memory.  Takes effect
 * from the next svt_fit_events (a captured graph is dropped). */
int svt_set_track_output(svt_ctx *ctx, svt_track *host, size_t cap);

/* Synchronise `stream` and return the unpacked roads of complete events in
 * stream order (runs the unpack stage first if it has not run yet).
 * *n_out = road count; SVT_E_CAPACITY if cap is too small. */
int svt_get_roads(svt_ctx *ctx, svt_road *out, size_t cap, size_t *n_out, void *stream);

/* Synchronise `stream` and return the counters and status of the last batch. */
int svt_get_stats(svt_ctx *ctx, svt_stats *out, void *stream);

/* Launch settings of the persistent kernel (autotuning); the tracks do not
 * depend on them (every combination of values below gives the same bytes). */
typedef struct {
    int32_t block;           /* threads per CTA: 128, 256 or 512 (0 = 256) */
    int32_t blocks_per_sm;   /* resident CTAs per SM (0 = the occupancy maximum of that block size) */
    int32_t small_n4;        /* roads with more than this many distinct fits (combinations of the
                              * four fitted layers) take a warp of their own (the box path); the
                              * others are fitted in runs of roads (1 .. 256, 0 = 256) */
    int32_t run_roads;       /* roads per queue claim of those runs: 4, 8 or 16 (0 = 8) */
    int32_t max_ctas;        /* cap on the grid (0 = SMs x blocks_per_sm); the autotuner keeps it */
} svt_launch;

/* Set the launch settings; they take effect from the next svt_fit_events
 * (a captured graph is dropped).  SVT_E_INVAL on a value outside the ranges
 * above. */
int svt_set_launch(svt_ctx *ctx, const svt_launch *cfg);

/* The launch settings in use, with the zeros resolved (*out, HOST). */
int svt_get_launch(svt_ctx *ctx, svt_launch *out);

/* One configuration measured by svt_autotune. */
typedef struct {
    svt_launch cfg;
    float ms;                  /* median device time of one SVT_PERSISTENT batch */
} svt_tune_point;

/* Autotuner of the persistent kernel over the grid of svt_launch values:
 * block size 128 / 256 / 512, resident CTAs per SM from 1 to that size's
 * occupancy maximum, small_n4 = 64 / 128 / 256 and run_roads = 4 / 8 / 16.
 * Each configuration runs the bound batch once to warm up and `reps` times
 * timed with CUDA events on `stream`; the one with the smallest median time
 * is kept (as svt_set_launch would).  Writes up to `cap` measured points to
 * `points` (HOST memory) and their number to *n_points.  Requires constants
 * and a bound batch; synchronises `stream`; SVT_E_CAPACITY if cap > 0 is too
 * small (the best configuration is still applied). */
int svt_autotune(svt_ctx *ctx, int reps, svt_tune_point *points, uint32_t cap, uint32_t *n_points,
                 void *stream);

/* Capture the enqueue of svt_fit_events(ctx, mode) for the bound batch into a
 * CUDA graph and use it for later svt_fit_events calls with the same batch
 * binding (enable = 1); enable = 0 returns to direct launches. */
int svt_use_graph(svt_ctx *ctx, int enable);

/* Test hook: spin limit of device-side waits in microseconds (0 = default of
 * two seconds) and, for the next SVT_PERSISTENT launch only (a direct launch,
 * never a graph), skip_arrival = 1: block 0 leaves before its first grid
 * barrier; 2: block 0 leaves after the fit stage, when the cross-road group
 * table has been filled.  The others' waits run out and the batch ends with
 * SVT_E_TIMEOUT; the next svt_fit_events clears the group table first.
 * 0 = no early exit.  Never faults or hangs the device. */
int svt_debug_wait(svt_ctx *ctx, uint32_t wait_limit_us, int skip_arrival);

/* Number of kernels the last svt_fit_events enqueued (for launch accounting). */
int svt_last_launch_count(svt_ctx *ctx);

const char *svt_strerror(int code);

/* Integer throughput of `device`, the denominator of the fit's roofline (not
 * a step of the chain): every thread of a grid that fills the device runs
 * eight independent chains of one operation, timed with CUDA events (best of
 * five launches after a warm-up).  *imad_per_s: 32-bit multiply-adds
 * (mad.lo.u32) per second; *iadd_per_s: 32-bit adds; *mixed_per_s:
 * multiply-adds and xors alternating (two pipes at once).  HOST pointers.
 * Allocates one word of device memory for the duration of the call;
 * synchronises the device. */
int svt_measure_int_peak(int device, double *imad_per_s, double *iadd_per_s, double *mixed_per_s);

/* ---- the chain without allocation ----------------------------------------
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when a batch arrives (a process whose free
 * device memory is owned by another allocator or fixed at start-up, a
 * trigger path where an allocation's latency or failure is not acceptable).
 *
 * svt_run_static runs SVT_PERSISTENT on one batch over a scratch arena that
 * is a fixed-size __device__ array of the library (under 8 MB per device),
 * not a context: it allocates nothing.  Limits: 131072 words, 1024 events,
 * 8192 roads, and a cross-road group table of 32768 slots (filled to 3/4 at
 * most); SVT_E_CAPACITY beyond any of them (n_words is checked before any
 * work, the others on the device).
 * d_words: the batch on the device (4-byte aligned); sets: the 360 constant
 * sets in HOST memory (same admission rule as svt_load_constants); d_tracks:
 * caller-owned DEVICE buffer of `cap` records (8-byte aligned) that receives
 * the tracks in (event, road, comb) order; *n_out (HOST) = number of tracks.
 * With SVT_E_CAPACITY because the tracks did not fit `cap`, *n_out is their
 * number (larger than cap) and nothing is written; with SVT_E_CAPACITY from
 * an arena limit, *n_out = 0.
 * The call synchronises `stream`, so it must never be called on a stream
 * that is being captured into a graph (SVT_E_INVAL).  Every call looks up the
 * arena on the current device; the first call on a device clears the
 * arena's group table and sets the kernel's shared-memory limit.  There is
 * one arena per device, so calls that overlap in time (threads or streams
 * with work in flight) race on it. */
int svt_run_static(const uint32_t *d_words, size_t n_words, const svt_const_set *sets,
                   uint32_t n_sets, int64_t chi2_cut, svt_track *d_tracks, size_t cap,
                   size_t *n_out, void *stream);

/* ---- serving: continuous batching of independent requests -------------- *
 * Not a step of the paper's chain: it serves the chain to a stream of
 * independent requests (batches of events), the low-latency trigger setting
 * of the paper's data-flow tests (Sec. III, Fig. 1).  A server owns `n_slots`
 * slots; each holds a context sized for one request, a CUDA stream and pinned
 * host staging, with the constants resident.  svt_server_submit admits a
 * request as soon as a slot is free and enqueues its host->device copy, its
 * kernel and the read of its status at once, so requests admitted while
 * others run overlap on the device.  A progress thread of the server fetches
 * each result's tracks once their count is known; results are returned in
 * completion order.  Each request's result is the same as running it alone
 * through svt_unpack / svt_fit_events / svt_get_tracks. */
typedef struct svt_server svt_server;

typedef struct {
    uint32_t n_slots;          /* requests on the device at once; 0 = as many as a quarter of
                                  the free device memory holds, at most 8 */
    uint32_t ctas_per_sm;      /* CTAs per SM of each request's persistent kernel (0 = 1) */
    uint32_t max_ctas;         /* grid cap of each request's kernel (0 = SMs x ctas_per_sm) */
    int32_t mode;              /* SVT_PERSISTENT or SVT_PLAIN (0 is SVT_PLAIN) */
    uint64_t max_words;        /* words per slot (0 = 1 << 20, below 1 << 31) */
    uint32_t max_events;       /* events per slot (0 = max_words / 3 + 1: any stream of max_words) */
    uint32_t max_roads;        /* roads per slot (0 = max_words / 3 + 1) */
    uint64_t max_tracks;       /* tracks per slot (0 = 1 << 20) */
    uint32_t hash_slots;       /* cross-road group table per slot, power of 2 (0 = 1 << 20) */
    uint32_t pad;
    uint64_t max_combinations; /* SVT_PLAIN combination buffers per slot (0 = 1 << 24) */
} svt_server_config;

typedef struct {
    uint64_t request_id;
    int32_t status;            /* the request's SVT_* status */
    uint32_t pad;
    uint64_t n_tracks;         /* surviving tracks (0 unless status is SVT_OK) */
    uint64_t n_events;
    uint64_t n_combinations;
    uint64_t latency_ns;       /* svt_server_submit entry -> tracks in host memory */
} svt_server_result;

/* Create a server on `device` with the constant sets (HOST memory, as for
 * svt_load_constants) and chi-square cut resident in every slot.  config
 * NULL = defaults with SVT_PLAIN; the chosen values are in
 * svt_server_get_config.  Starts the server's progress thread. */
int svt_server_create(svt_server **out, int device, const svt_server_config *config,
                      const svt_const_set *sets, uint32_t n_sets, int64_t chi2_cut);

/* Wait (at most 10 s) for the requests in flight, stop the progress thread and
 * free every slot.  Results not taken are dropped. */
void svt_server_destroy(svt_server *srv);

int svt_server_get_config(svt_server *srv, svt_server_config *out);

/* Admit one request: `words` (HOST memory, n_words, copied before return) is a
 * packed word stream as for svt_unpack.  Blocks until a slot is free; returns
 * the request's id in *request_id.  A request with more words, events (EE
 * words) or roads (EP words) than a slot holds is cut at event boundaries
 * into chunks that fit, admitted one after the other as slots free up; its
 * result (one id) joins the chunks' tracks in stream order with their event
 * indices offset, and its status is that of the first chunk that failed.
 * SVT_E_CAPACITY (nothing admitted) only if one event alone exceeds a slot's
 * max_words or max_roads.  Errors of the request itself (format, limits,
 * capacity, CUDA) are its result's status.  Thread-safe. */
int svt_server_submit(svt_server *srv, const uint32_t *words, size_t n_words, uint64_t *request_id);

/* Next completed request, in completion order: waits up to timeout_us
 * microseconds (< 0: no limit); SVT_E_TIMEOUT if none completed. */
int svt_server_wait(svt_server *srv, int64_t timeout_us, svt_server_result *out);

/* Copy the tracks of a completed request (in (event, road, comb) order) to
 * HOST memory `out` (cap records) and release them.  *n_out = number of
 * tracks; SVT_E_CAPACITY (nothing released) if cap is smaller;
 * SVT_E_STATE if the id is unknown or already taken. */
int svt_server_take(svt_server *srv, uint64_t request_id, svt_track *out, size_t cap, size_t *n_out);

#ifdef __cplusplus
}
#endif
#endif /* SVT_H */
