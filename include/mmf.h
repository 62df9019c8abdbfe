/*
 * mmf.h -- C ABI of the GB300 running maximum-minimum filter library.
 *
 * The operation (Lemire, "Streaming Maximum-Minimum Filter Using No More than
 * Three Comparisons per Element", Section 1): for an array a_0..a_{n-1} and a
 * window width w, output for every window [j, j+w), j = 0..n-w,
 *     max[j] = max_{i in [j, j+w)} a_i      min[j] = min_{i in [j, j+w)} a_i
 * (n-w+1 outputs of each; none when w > n).  Every output is one of the input
 * elements, so results are exact (bit-identical to any correct CPU version)
 * for inputs without NaN.  NaN inputs give unspecified results; -0.0 and +0.0
 * compare equal and either may be returned.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are DEVICE pointers (cudaMalloc / torch CUDA tensors)
 *     on the current CUDA device; h_* are HOST pointers.  The caller owns all
 *     of them; the library never frees caller memory.
 *   - Arrays are contiguous, element type given by mmf_dtype.  Element
 *     pointers must be aligned to their element size.  16-byte alignment of
 *     the start of each array gives the fastest path; any element-aligned
 *     address is accepted.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued asynchronously on it; the call returns before it finishes.
 *   - Errors are returned as mmf_status; no C++ exception crosses the ABI.
 *     mmf_last_error() gives a thread-local message for the last failure.
 *     Failures detected on the device (a bounded wait that ran out) are
 *     recorded in a device status word read by mmf_device_status().
 *   - Sizes and indices are int64_t.
 */
#ifndef MMF_H_
#define MMF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { MMF_F32 = 0, MMF_F64 = 1, MMF_I16 = 2, MMF_U8 = 3 } mmf_dtype;

/* MMF_VALID: windows [j, j+w), n-w+1 outputs (Section 1).
 * MMF_CENTERED_CLIPPED: envelope windows [i-r, i+r] clipped to [0, n), n
 * outputs; the window argument is the radius r >= 0 (the upper/lower
 * envelopes used for time-warping lower bounds, cited in Section 1). */
typedef enum { MMF_VALID = 0, MMF_CENTERED_CLIPPED = 1 } mmf_mode;

typedef enum {
    MMF_OK = 0,
    MMF_EINVAL = 1,    /* bad argument (null pointer, negative size, ...)   */
    MMF_ENOMEM = 2,    /* host or device allocation failed / over budget    */
    MMF_ECUDA = 3,     /* a CUDA runtime call failed                        */
    MMF_EBUSY = 4,     /* serving: admission refused, retry later           */
    MMF_ETIMEOUT = 5,  /* a bounded wait ran out                            */
    MMF_ECLOSED = 6,   /* serving: stream already closed / unknown          */
    MMF_ENOTIMPL = 7,  /* combination not supported                         */
    MMF_EDEVICE = 8    /* the device reported an error in its status word   */
} mmf_status;

/* Kernel choice for the 1D filter.  AUTO consults the dispatch table. */
typedef enum {
    MMF_KERNEL_AUTO = 0,
    MMF_KERNEL_BLOCKSCAN = 1, /* van Herk/Gil-Werman block prefix/suffix scan
                                 (Section 2 related work; Table 1 row 2)    */
    MMF_KERNEL_SLIDE = 2,     /* register slide: naive windows of Table 1
                                 row 1, for small w                         */
    MMF_KERNEL_WEDGE = 3,     /* chunked monotonic wedge, Algorithm 1 of
                                 Section 4 per chunk with a w-1 halo        */
    MMF_KERNEL_FRONT = 4      /* the block scan of windows of a tile or more
                                 (w - 1 >= 2048 for f32, 4096 for i16/u8;
                                 not f64) with every CTA on one advancing
                                 front of output tiles                      */
} mmf_kernel;

/* Largest window handled: (w - 1) / tile <= MMF_MAX_WINDOW_TILES, where the
 * tile is 2048 elements for f32, 1024 for f64 and 4096 for i16 and u8 (so w up
 * to about 2.1 M for f32). */
#define MMF_MAX_WINDOW_TILES 1024

/* ---------------------------------------------------------------- 1D ---- */

/* mmf_filter1d -- running max-min filter of one array (Section 1 definition;
 * MMF_CENTERED_CLIPPED gives the envelope variant).
 *   d_in    n elements of `dtype` (may be NULL when n == 0)
 *   n       number of input elements, >= 0
 *   w_or_r  window width w >= 1 (VALID) or radius r >= 0 (CENTERED_CLIPPED)
 *   d_max   output, n-w+1 (VALID, 0 if w > n) or n (CENTERED_CLIPPED)
 *           elements; NULL skips the max side
 *   d_min   same for the min side; NULL skips it (not both NULL)
 * Outputs must not overlap the input.  Allocates nothing (unless a tuned
 * dispatch entry selects MMF_KERNEL_FRONT, whose small workspace comes from
 * the stream-ordered allocator).
 * Returns MMF_OK without touching memory when there are no outputs (w > n or
 * n == 0; pointers may then be NULL).  Otherwise returns MMF_EINVAL for
 * w < 1, r < 0, n < 0, both outputs NULL, a NULL input, or pointers not
 * aligned to the element size; MMF_ENOTIMPL if w exceeds the window limit. */
mmf_status mmf_filter1d(const void *d_in, int64_t n, int64_t w_or_r, mmf_dtype dtype,
                        mmf_mode mode, void *d_max, void *d_min, void *stream);

/* The same filter on arrays in HOST memory (pinned memory is fastest): the
 * outputs are cut into chunks of `chunk` elements (<= 0: 2^26) whose inputs
 * (the chunk plus its windows' reach) are uploaded, filtered and downloaded
 * through device staging on three internal CUDA streams, so uploads, kernels
 * and downloads of successive chunks overlap; the result equals mmf_filter1d
 * on the whole array.  Work starts after the work already queued on `stream`
 * and `stream` waits for the last download, so synchronising `stream` makes
 * h_max/h_min ready.  The library keeps per-device staging of three chunks
 * (grown on demand; growing it synchronises the device).  Calls are
 * serialised per device. */
mmf_status mmf_filter1d_host(const void *h_in, int64_t n, int64_t w_or_r, mmf_dtype dtype, mmf_mode mode,
                             void *h_max, void *h_min, int64_t chunk, void *stream);

/* Largest window of the chunked-wedge kernel: its per-thread rings (the
 * window of inputs and the deques U and L, Section 4) must fit shared memory. */
#define MMF_WEDGE_MAX_WINDOW 496

/* Same as mmf_filter1d with an explicit kernel choice (for tests and the
 * autotuner).  MMF_KERNEL_SLIDE requires w <= 17 for f32, w <= 9 otherwise;
 * MMF_KERNEL_WEDGE computes
 * MMF_VALID windows with w <= MMF_WEDGE_MAX_WINDOW (MMF_EINVAL /
 * MMF_ENOTIMPL otherwise).  MMF_KERNEL_BLOCKSCAN gives each CTA its own range
 * of outputs.  MMF_KERNEL_FRONT (windows of a tile or more, not f64, else
 * MMF_ENOTIMPL) hands output tiles to CTAs in order from a ticket: each tile
 * is read as the end of some windows and, about w elements later, as the
 * start of others while it is still in L2, and the aggregates of the whole
 * tiles inside a window come from the CTAs that read them (published in a
 * stream-ordered workspace of about 12 bytes per 2048 f32 inputs, taken from
 * and returned to the stream-ordered allocator on `stream`; MMF_ECUDA if that
 * allocation fails).  It runs as a cooperative launch.  The built-in
 * automatic choice does not take it (on the long-stream workload it is
 * slower than the per-range schedule). */
mmf_status mmf_filter1d_ex(const void *d_in, int64_t n, int64_t w_or_r, mmf_dtype dtype,
                           mmf_mode mode, void *d_max, void *d_min, void *stream,
                           mmf_kernel kernel);

/* The dispatch table of MMF_KERNEL_AUTO.  Without an entry, AUTO takes the
 * built-in rule (the register slide for w <= 17 for f32 and w <= 9 for the
 * other types, MMF_KERNEL_BLOCKSCAN otherwise).  An entry for a
 * bucket of (dtype, w, n) replaces it wherever its kernel can take the call
 * (windows: exact up to 32, then powers of two; lengths: powers of four).
 * The table is process-wide and thread-safe.
 *
 * mmf_dispatch_set -- sets the entry of the bucket of (n, w) to `kernel`
 *   (MMF_KERNEL_AUTO removes it).  MMF_EINVAL for bad sizes or kernels.
 * mmf_dispatch_get -- the kernel AUTO takes for valid windows of w over n
 *   elements (the entry, else the built-in rule).
 * mmf_dispatch_autotune -- times every kernel that can take valid windows of
 *   w over the n elements of d_in (writing d_max/d_min, n-w+1 each) on
 *   `stream`, which it synchronises; stores the fastest in the table (and in
 *   $MMF_AUTOTUNE_CACHE, keyed by GPU name, when that is set; later processes
 *   read it back) and writes it to *chosen (may be NULL). */
mmf_status mmf_dispatch_set(mmf_dtype dtype, int64_t n, int64_t w, mmf_kernel kernel);
mmf_status mmf_dispatch_get(mmf_dtype dtype, int64_t n, int64_t w, mmf_kernel *kernel);
mmf_status mmf_dispatch_autotune(const void *d_in, int64_t n, int64_t w, mmf_dtype dtype, void *d_max, void *d_min,
                                 void *stream, mmf_kernel *chosen);

/* Arg-max / arg-min filter (Section 5: the streaming algorithm stores the
 * locations of the extremes, so their positions come at no extra cost):
 * for every valid window [j, j+w), d_argmax[j] / d_argmin[j] is the position
 * in the array (int64) of its maximum / minimum, the leftmost among equal
 * values, and d_max / d_min the values; any output may be NULL (not all).
 * n-w+1 outputs each, any w >= 1, computed by van Herk/Gil-Werman block
 * scans (Section 2) over (value, position) pairs: the suffix of a block is
 * left of the next block's prefix, so keeping the suffix's candidate on equal
 * values keeps the leftmost position.  For w > 2048 the call takes a
 * workspace of per-tile aggregates (about 72 bytes per 2048 inputs for f32)
 * from the stream-ordered allocator and returns it on `stream`.  Pointers:
 * element-aligned values, 8-byte aligned positions.  Errors: MMF_EINVAL for
 * w < 1, n < 0, NULL or misaligned buffers; MMF_ENOMEM / MMF_ECUDA from the
 * workspace allocation or the launches. */
mmf_status mmf_argfilter1d(const void *d_in, int64_t n, int64_t w, mmf_dtype dtype, void *d_max, void *d_min,
                           int64_t *d_argmax, int64_t *d_argmin, void *stream);

/* The same with an explicit kernel: MMF_KERNEL_AUTO or MMF_KERNEL_BLOCKSCAN
 * (the block scans above), or MMF_KERNEL_WEDGE (the chunked monotonic wedge of
 * Algorithm 1 with ties kept in the deques, w <= MMF_WEDGE_MAX_WINDOW, else
 * MMF_ENOTIMPL); other kernels give MMF_ENOTIMPL. */
mmf_status mmf_argfilter1d_ex(const void *d_in, int64_t n, int64_t w, mmf_dtype dtype, void *d_max, void *d_min,
                              int64_t *d_argmax, int64_t *d_argmin, void *stream, mmf_kernel kernel);

/* The window-3 filter by the two-comparison scheme of Section 3 (the
 * proposition after the lower bound): knowing the order of the last two
 * elements from the previous step, two comparisons of the new element (with
 * the newer and with the older of the two) give the window's maximum and
 * minimum and the order of the next pair.  Same outputs as mmf_filter1d with
 * w = 3, MMF_VALID (n-2 each; n < 3 gives none).  Each GPU thread takes 16
 * consecutive outputs and starts its pair with one comparison, so a chunk of
 * c outputs makes 1 + 2c comparisons: ceil((n-2)/16) + 2(n-2) in all, which
 * are ADDED to *d_ncmp when it is not NULL (the caller zeroes it).  Any of
 * d_max, d_min, d_ncmp may be NULL (not all).  Pointers element-aligned,
 * d_ncmp 8-byte aligned; MMF_EINVAL otherwise.  The default kernels take
 * w = 3 in a register slide; this entry point shows the scheme's comparison
 * count on the GPU. */
mmf_status mmf_filter1d_w3(const void *d_in, int64_t n, mmf_dtype dtype, void *d_max, void *d_min,
                           unsigned long long *d_ncmp, void *stream);

/* Number of outputs of one side for (n, w_or_r, mode); -1 if invalid. */
int64_t mmf_output_length(int64_t n, int64_t w_or_r, mmf_mode mode);

/* ---------------------------------------------------------------- 2D ---- */

/* Separable 2D filter (Section 1: the 1D filter on rows, then on columns),
 * valid windows: for each of nimg images of H rows x W columns (row pitch
 * `pitch` >= W elements; image k starts at d_in + k*H*pitch),
 *     max[y][x] = max over rows y..y+wy-1, columns x..x+wx-1   (min likewise)
 * for y = 0..H-wy, x = 0..W-wx.  Outputs are packed: image k, row y starts at
 * d_max + (k*(H-wy+1) + y)*(W-wx+1).  Both windows >= 1; a window of 1 skips
 * that pass.  The row pass writes its two intermediates to `d_work` (16-byte
 * aligned, size from mmf_filter2d_workspace; none needed when wy or wx is 1
 * or when the fused kernel runs).  With work_bytes >= 2 * R * elem_size,
 * R = (nimg*H-1)*pitch + W-wx+1 rounded up to 16, the row pass filters all
 * rows as one series (always so for pitch == W at the queried size); with
 * less, row by row.
 * fuse: 0 row pass then column pass; 1 a fused kernel, no intermediates in
 * memory: for wy, wx <= 31 a tile with its halo in shared memory, rows then
 * columns; otherwise the column pass computing each tile's row maxima and
 * minima in registers (wx <= MMF_FUSED_MAX_WX, else MMF_ENOTIMPL); 2 the
 * register-streaming kernel for u8 and f32 (windows up to 9 x 9) and i16 (up
 * to 9 rows x 5 columns): 4 u8 (2 i16) columns packed per 32-bit register
 * with per-element SIMD max/min, f32 one column per register, no
 * intermediates in memory; needs 4-byte aligned input rows (d_in, the pitch
 * in bytes and the image stride), else MMF_ENOTIMPL; -1 automatic (the
 * streaming kernel where it applies, except f32 rows-only windows wider than
 * 3; the tile kernel when wy, wx <= 12 for f32/f64, <= 15 for u8/i16; else
 * the two passes).  Any other value: MMF_EINVAL.
 * Column windows are limited by the column
 * pass's shared memory: up to about 760 rows for f32, 320 for f64 and 1700 for
 * i16/u8 (MMF_ENOTIMPL beyond). */
#define MMF_FUSED_MAX_WX 64
mmf_status mmf_filter2d_workspace(int64_t nimg, int64_t H, int64_t W, int64_t wy, int64_t wx, mmf_dtype dtype,
                                  int fuse, size_t *bytes);
mmf_status mmf_filter2d_separable(const void *d_in, int64_t nimg, int64_t H, int64_t W, int64_t pitch,
                                  int64_t wy, int64_t wx, mmf_dtype dtype, int fuse, void *d_max, void *d_min,
                                  void *d_work, size_t work_bytes, void *stream);

/* ----------------------------------------------------------- batched ---- */

/* A batch plan describes many independent series in one input buffer (the
 * batching pattern: thousands of series of uneven length and window in one
 * persistent launch, captured in a CUDA graph).  Each series s is filtered as
 * by mmf_filter1d (window h_w[s], clipped to the series length in VALID mode
 * by the caller; radius in CENTERED_CLIPPED mode).  The plan owns device
 * tables (series, work items, ticket counters) and a graph cache; it is not
 * thread-safe.  Outputs follow series by series, at the offsets reported by
 * mmf_batch_plan_out_offsets: each series' outputs start on a 32-byte
 * boundary of the output buffers (whole-sector vector stores), after the
 * previous series' outputs and at most 31 bytes of padding that no call
 * writes. */
typedef struct mmf_batch_plan mmf_batch_plan;

/* h_in_off: element offset of each series in the input buffer (NULL: the
 *           series are packed back to back in order)
 * h_len, h_w: length and window (or radius) of each series
 * Allocates the plan and its device tables; *out receives it. */
mmf_status mmf_batch_plan_create(const int64_t *h_in_off, const int64_t *h_len, const int64_t *h_w,
                                 int64_t nseries, mmf_dtype dtype, mmf_mode mode, mmf_batch_plan **out);

/* Frees the plan (NULL is ignored).  No call may use it afterwards. */
void mmf_batch_plan_destroy(mmf_batch_plan *plan);

/* h_off[nseries+1]: start of each series' outputs in the output buffers
 * (elements); series s has n_out outputs from h_off[s] (VALID: len - w + 1,
 * CENTERED_CLIPPED: len), followed by padding up to h_off[s+1];
 * h_off[nseries] = out_len, the end of the last series' outputs. */
mmf_status mmf_batch_plan_out_offsets(const mmf_batch_plan *plan, int64_t *h_off);

/* Required input / output buffer lengths (elements) and, in n_items[4] (may
 * be NULL), the work items per kernel group (0-2 block scans, 3 slide). */
mmf_status mmf_batch_plan_sizes(const mmf_batch_plan *plan, int64_t *in_len, int64_t *out_len, int64_t *n_items);

/* Tuning knobs of a plan beside the segment lengths: series of at most
 * short_cut elements (0 .. 1024 for 1-4 byte types, 512 for f64; 0: none)
 * take the warp-per-series kernel (one warp per series) instead of
 * block-scan work items (a whole CTA per item); windows of at most slide_max
 * (1: none; at most 17 for f32, 9 otherwise) take the register slide instead
 * of block scans.  MMF_EINVAL outside those ranges. */
mmf_status mmf_batch_plan_set_knobs(mmf_batch_plan *plan, int64_t short_cut, int slide_max);
mmf_status mmf_batch_plan_get_knobs(const mmf_batch_plan *plan, int64_t *short_cut, int *slide_max);

/* Output tiles per work item of one kernel group (tuning knob). */
mmf_status mmf_batch_plan_set_segment(mmf_batch_plan *plan, int group, int seg_tiles);
mmf_status mmf_batch_plan_get_segment(const mmf_batch_plan *plan, int group, int *seg_tiles);

/* Tunes the plan on the given buffers (synchronises the stream): first the
 * short-series cut-off (threads per series), then the slide limit (kernel
 * choice for small windows), each timed over the whole plan, then the
 * segment length of each block-scan group; keeps the fastest of each.  With
 * $MMF_AUTOTUNE_CACHE set, the choices are appended to that file, keyed by
 * GPU name and workload shape, and reused by later plans. */
mmf_status mmf_batch_plan_autotune(mmf_batch_plan *plan, const void *d_in, void *d_max, void *d_min,
                                   void *stream);

/* Filters every series: one ticket reset plus one persistent launch per
 * non-empty kernel group, replayed from a CUDA graph (captured on the first
 * call for this set of buffers).  d_max/d_min: out_len elements each (either
 * may be NULL). */
mmf_status mmf_filter1d_batched(mmf_batch_plan *plan, const void *d_in, void *d_max, void *d_min,
                                void *stream);

/* Lower bound of the dynamic-time-warping distance from a precomputed
 * max-min envelope (the application the paper's Section 1 cites): for a
 * plan in MMF_CENTERED_CLIPPED mode whose series all have n_query elements,
 * with U, L the envelope of radius h_w[s] of series s,
 *     d_lb[s] = sqrt( sum_i (q_i - U_i)^2 [q_i > U_i] + (L_i - q_i)^2 [q_i < L_i] )
 * for the query q = d_query (same dtype, device memory).  It is a lower bound
 * of the time-warping distance of q and series s with warping limited to
 * |i - j| <= r.  The envelope is never written: each tile's envelope feeds
 * the sum directly, so the call reads the series once (about a third of the
 * bytes of the envelope filter followed by a separate reduction).
 * d_lb: nseries doubles (8-byte aligned).  Arithmetic: f32 series in f32
 * with a per-warp sum (relative error below 2e-6 of the bound), f64 in
 * double, i16/u8 exactly in integers; sums over the tiles of one series are
 * added atomically in double.  MMF_EINVAL for a VALID plan or series of
 * another length.  Launches directly on `stream` (no graph). */
mmf_status mmf_lb_keogh_batched(mmf_batch_plan *plan, const void *d_in, const void *d_query, int64_t n_query,
                                double *d_lb, void *stream);

/* The plain form: one mmf_filter1d launch per series on `stream`, same
 * kernels, no graph (the baseline the batched form is compared with). */
mmf_status mmf_filter1d_per_series(const mmf_batch_plan *plan, const void *d_in, void *d_max, void *d_min,
                                   void *stream);

/* ---------------------------------------------------------- serving ---- */

/* A streaming service: many concurrent streams, each filtered with zero
 * stream latency (Section 1: a window's outputs are emitted as soon as its
 * last element has arrived).  Each stream's last w-1 samples and its int64
 * sample count stay on the device, so the outputs of the chunks pushed to a
 * stream are exactly the whole-array filter of their concatenation (VALID
 * windows).  Chunks are admitted FIFO while the device-memory budget allows,
 * at most one chunk per stream in flight, and batched across streams into one
 * launch per kernel group (continuous batching: a chunk that arrives while a
 * batch runs joins a later batch as soon as memory and its stream allow).  The
 * server owns a worker thread, its device budget and a few CUDA streams; all
 * its functions are thread-safe. */
typedef struct mmf_server mmf_server;

typedef struct {
    int64_t chunks;             /* chunks completed (since the last reset) */
    int64_t elements;           /* their input samples */
    int64_t batches;            /* batches launched */
    double p50_ms, p99_ms;      /* push-to-completion latency percentiles */
    double max_ms;
    int64_t queued;             /* chunks waiting for admission now */
    int64_t device_bytes_used;  /* budget in use now */
    double p50_queue_ms, p99_queue_ms;     /* push to admission into a batch */
    double p50_service_ms, p99_service_ms; /* admission to completion */
    double max_hold_ms;         /* longest time the worker held the server
                                   lock while setting up one batch */
} mmf_server_stats_t;

/* device_budget_bytes: one device allocation shared by stream state, chunk
 * staging and outputs (>= 1 MiB); max_batch: chunks per launch. */
mmf_status mmf_server_create(size_t device_budget_bytes, int max_batch, mmf_dtype dtype, mmf_server **out);

/* Stops the worker after the batches already on the GPU, frees everything. */
void mmf_server_destroy(mmf_server *server);

/* Opens a stream with window w >= 1 (state: w-1 samples of the budget;
 * MMF_ENOMEM if the budget is exhausted). */
mmf_status mmf_stream_open(mmf_server *server, int64_t w, uint64_t *stream_id);

/* Queues len samples (HOST pointer; pinned memory is faster) for the stream
 * and returns at once.  *n_out receives the number of outputs of this chunk,
 * max(0, N+len-w+1) - max(0, N-w+1) for N samples pushed before it; they are
 * written to the HOST buffers h_max/h_min (either may be NULL, not both when
 * *n_out > 0).  h_chunk, h_max and h_min must stay valid until the ticket
 * completes.  MMF_ECLOSED for a closed or unknown stream, MMF_ENOMEM for a
 * chunk that can never fit the budget, MMF_EDEVICE after a device failure. */
mmf_status mmf_stream_push(mmf_server *server, uint64_t stream_id, const void *h_chunk, int64_t len, void *h_max,
                           void *h_min, int64_t *n_out, uint64_t *ticket);

/* Waits up to timeout_ms for a ticket (MMF_ETIMEOUT if not done; the ticket
 * stays valid).  A completed ticket is consumed. */
mmf_status mmf_ticket_wait(mmf_server *server, uint64_t ticket, int timeout_ms);

/* Many pushes under one lock, in order: the same as calling mmf_stream_push
 * for i = 0..count-1 with stream_ids[i], h_chunks[i], lens[i], h_max[i] and
 * h_min[i] (h_max or h_min may be NULL arrays: no such outputs), writing
 * n_out[i] (may be NULL) and tickets[i].  Stops at the first failing push and
 * returns its status; *n_done (may be NULL) receives the number queued.  For
 * feed handlers that receive many streams' chunks at once. */
mmf_status mmf_stream_push_batch(mmf_server *server, int64_t count, const uint64_t *stream_ids,
                                 const void *const *h_chunks, const int64_t *lens, void *const *h_max,
                                 void *const *h_min, int64_t *n_out, uint64_t *tickets, int64_t *n_done);

/* Waits for every ticket of the array (consuming each), up to timeout_ms in
 * total.  MMF_ETIMEOUT leaves the tickets not yet reached valid; MMF_EDEVICE
 * if a batch of any of them failed. */
mmf_status mmf_ticket_wait_batch(mmf_server *server, int64_t count, const uint64_t *tickets, int timeout_ms);

/* Refuses further pushes, waits up to timeout_ms for the stream's chunks,
 * frees its state (MMF_ETIMEOUT leaves it closed but not yet freed). */
mmf_status mmf_stream_close(mmf_server *server, uint64_t stream_id, int timeout_ms);

/* Stream state snapshot, a checkpoint of one stream: its window, its 64-bit
 * sample count (streams are unbounded; positions are 64-bit as Section 5
 * recommends for streams) and its last min(count, w-1) samples, which are all
 * that later outputs depend on (each output depends on its window only,
 * Section 1).  Waits up to timeout_ms for the stream's queued and in-flight
 * chunks (MMF_ETIMEOUT otherwise); the caller must not push to the stream
 * during the call.  Layout, little-endian: uint32 magic 0x53464d4d ("MMFS"),
 * uint32 version 1, int32 dtype, int32 0, int64 w, int64 count, int64 halo
 * length h, then h samples of the dtype (oldest first).  *size receives the
 * bytes of the snapshot; with h_buf NULL only the size is reported, else
 * buf_bytes must hold it (MMF_EINVAL). */
#define MMF_SNAPSHOT_MAGIC 0x53464d4du
#define MMF_SNAPSHOT_HEADER_BYTES 40
mmf_status mmf_stream_snapshot(mmf_server *server, uint64_t stream_id, void *h_buf, size_t buf_bytes, size_t *size,
                               int timeout_ms);

/* The same state as the stream's monotonic wedge (Section 4): the samples
 * that can still be a window maximum (strictly above every later sample: the
 * deque U of Algorithm 1) or minimum (strictly below every later one: L).  No
 * other sample can decide a later output (a later, larger and a later,
 * smaller sample lie in every later window that holds it), so this state
 * restores the same outputs; it holds about 2 ln(w) samples on i.i.d. noise
 * and on the order of sqrt(w) on a random walk, where the halo holds w-1
 * (monotone data: one side is the whole window).  Layout: the header as above with version 2
 * (halo length h as before), then int64 nU, int64 nL, then nU entries and nL
 * entries, each an int64 distance back from the count (1..h) followed by the
 * sample.  Same waiting, sizing and errors as mmf_stream_snapshot. */
mmf_status mmf_stream_snapshot_wedge(mmf_server *server, uint64_t stream_id, void *h_buf, size_t buf_bytes,
                                     size_t *size, int timeout_ms);

/* Opens a new stream in the state of a snapshot (from this server or another
 * of the same dtype): its later pushes give exactly the outputs the original
 * stream would have given.  MMF_EINVAL for another dtype, a bad header or a
 * short buffer; MMF_ENOMEM if the budget has no room for its state. */
mmf_status mmf_stream_restore(mmf_server *server, const void *h_buf, size_t buf_bytes, uint64_t *stream_id);

/* Stops (1) or resumes (0) admissions: for tests of stalled service. */
mmf_status mmf_server_pause(mmf_server *server, int paused);

/* Latency percentiles and counters; reset != 0 clears them. */
mmf_status mmf_server_stats(mmf_server *server, int reset, mmf_server_stats_t *out);

/* ------------------------------------------- batched, no allocation ---- */

/* Limits of mmf_filter1d_batched_noalloc. */
#define MMF_NOALLOC_MAX_SERIES 512
#define MMF_NOALLOC_MAX_ITEMS 2048

/* The batched filter for callers that must not allocate device memory: a
 * process that reserved its whole device-memory budget up front (a fixed
 * pool shared by its components), or a latency-bound path on an ordinary
 * host thread where an allocation may block on the driver or fail under
 * memory pressure.  The paper has no counterpart to this entry point; it is
 * an interface convenience.
 *
 * Same results as a batch plan over the same series (inputs packed back to
 * back in d_in, outputs in d_max/d_min in series order at the offsets a plan
 * reports, each series on a 32-byte boundary), but it calls no
 * cudaMalloc/cudaFree: its work tables live in one fixed device array of
 * about 74 KB that every GPU which loads the library keeps until the process
 * exits.  The tables are built in static host memory and passed to the GPU
 * as kernel arguments, so the GPU reads no host memory after the call
 * returns.  At most MMF_NOALLOC_MAX_SERIES series; long series are split into
 * at most MMF_NOALLOC_MAX_ITEMS work items.  Larger requests, and lengths
 * whose sum would overflow 64-bit positions, return MMF_EINVAL.
 *
 * The first call on a device also looks up the array's device address (once
 * per device, with that device current).  Every call reuses the same array
 * and clears its counters itself;
 * calls are serialised on the host, but calls that overlap on the GPU (two
 * unordered streams) race on the array and give wrong results: order them on
 * one stream. */
mmf_status mmf_filter1d_batched_noalloc(const void *d_in, const int64_t *h_len, const int64_t *h_w,
                                        int64_t nseries, mmf_dtype dtype, mmf_mode mode, void *d_max,
                                        void *d_min, void *stream);

/* --------------------------------------------------------- device status */

/* Reads (and, if reset != 0, clears) the device status word that kernels set
 * when a bounded wait runs out (bit 0: pipeline wait timeout; bit 1: a work
 * item of another kernel group; bit 2, range-checked builds only: an index
 * outside the launch's buffers, whose access was skipped).  Synchronises the
 * current device.  Returns MMF_OK and writes the word to *out. */
mmf_status mmf_device_status(uint32_t *out, int reset);

/* Test hook for the device-side timeout path of the block-scan kernels (the
 * 1D, batched, 2D row and serving launches).  With starve_copies != 0, the
 * kernels launched afterwards by this process issue none of their input
 * copies, so every pipeline wait runs out after wait_limit_cycles SM clocks
 * (1000 .. 2e9; about 0.5 ns each): the kernel records bit 0 in the device
 * status word, each warp finishes its current work item without waiting
 * again, and all warps of each CTA leave together at the item's end.  The
 * outputs of such a call are unspecified; nothing faults, nothing is left in
 * flight and the context stays usable.  starve_copies == 0 restores normal
 * operation.  For tests only. */
mmf_status mmf_test_set_wait_fault(int starve_copies, int64_t wait_limit_cycles);

/* Test hook for the range-checked build (MMF_CHECKED, see build.py): with
 * elems > 0, block-scan launches afterwards tell their kernels that at most
 * `elems` input elements may be read, below what they actually read; the
 * checked kernels then skip the copies and loads past that bound and record
 * bit 2 of the device status word (the skipped bytes are still inside the
 * caller's buffer, so nothing outside it is touched either way).  0 restores
 * normal operation.  For tests only. */
mmf_status mmf_test_set_input_clip(int64_t elems);

/* Thread-local, NUL-terminated description of the last failure. */
const char *mmf_last_error(void);

/* Library version string. */
const char *mmf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MMF_H_ */
