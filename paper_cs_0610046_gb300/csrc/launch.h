// Internal host-side interface between the C ABI and the per-dtype kernel
// translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "blockscan.cuh"

namespace mmf {

// NVTX range over the rest of the enclosing scope: each C-ABI call and each
// server batch shows as a named range in a profiler's timeline (NVTX v3 is
// header-only; without an attached tool a range costs a pointer test).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct LaunchCtx {
    int device;
    int sms;
    uint32_t *status;  // device status word
    cudaStream_t stream;
};

// Test hooks of the block-scan kernels (mmf_test_set_wait_fault,
// mmf_test_set_input_clip), applied to every launch's finished parameters.
struct TestHooks {
    uint32_t flags;        // kTestStarveCopies or 0
    long long wait_limit;  // SM clocks; 0: the default bound
    int64_t clip_in;       // > 0: the readable bound the kernels check is at most this many elements
};
TestHooks test_hooks();
inline void apply_test_hooks(BlockScanParams &P) {
    const TestHooks h = test_hooks();
    P.test_flags = h.flags;
    P.wait_limit = h.wait_limit;
    if (h.clip_in > 0 && P.in_elems > h.clip_in) P.in_elems = h.clip_in;
}

// One series, statically split into per-CTA items (no allocation).  With
// allow_slide, small windows (w <= 17 for f32, 9 otherwise) use the register slide
// instead of block scans.
// front: -1 automatic, 0 per-CTA ranges, 1 one advancing front (windows of a
// tile or more, f32/i16/u8; it takes a small stream-ordered workspace of
// published tile aggregates).
template <typename T>
cudaError_t blockscan_1d(const LaunchCtx &ctx, const void *in, const SeriesDesc &sd, void *omax, void *omin,
                         bool allow_slide, int front = -1);

// Whether blockscan_1d takes the advancing front for this series (front as
// above; the automatic choice does not take it).
template <typename T> bool front_applies(const SeriesDesc &sd, int sms, int front);

// The same series description applied to `rows` rows at the given element
// pitches (row pass of the 2D filter); items are generated arithmetically.
template <typename T>
cudaError_t blockscan_rows(const LaunchCtx &ctx, const void *in, const SeriesDesc &sd, int64_t rows,
                           int64_t in_pitch, int64_t out_pitch, void *omax, void *omin);

// Short series (batched plans): at most this many elements take the
// warp-per-series kernel (32 lanes x 32 elements; 16 for 8-byte types).
constexpr int64_t short_max_len(int esz) { return esz == 8 ? 512 : 1024; }

// Warp-per-series launch over the series d_ids[0..count) of the table;
// lb_acc (with lb_query of lb_n elements, every series' length): the envelope
// lower bound instead of outputs (each series' sum is written, not added).
template <typename T>
cudaError_t short_table(const LaunchCtx &ctx, const void *in, int64_t in_elems, void *omax, void *omin,
                        const SeriesDesc *d_series, const int64_t *d_ids, int64_t count, const void *lb_query,
                        double *lb_acc, int64_t lb_n = 0);
// Kernel attributes of the short-series kernel (outside any stream capture).
template <typename T> cudaError_t short_prepare(int device, bool lb, int *per_sm);

// Batched outputs: each series' outputs start on a 32-byte boundary of the
// output buffers (whole-sector vector stores); the start after a run of
// outputs that ends at element `end`.
inline int64_t batch_out_start(int64_t end, int esz) {
    const int64_t a = 32 / esz;
    return (end + a - 1) / a * a;
}

// Table-driven launch (batched plans): items of one block mode, pulled from
// an atomic ticket (or round-robin if d_ticket is null).  grid <= 0: one
// persistent wave.
// in_elems: elements of `in` that may be read (the whole input buffer; copies
// that cross a series end stay inside it).  lb_acc (with lb_query): instead of
// storing outputs, add each series' squared query excursions outside its
// envelope to lb_acc[series].
template <typename T>
cudaError_t blockscan_table(const LaunchCtx &ctx, int mode, const void *in, int64_t in_elems, void *omax,
                            void *omin, const SeriesDesc *d_series, const ItemDesc *d_items, int64_t n_items,
                            int *d_ticket, int grid, const void *lb_query = nullptr, double *lb_acc = nullptr);

// The table launch in its lower-bound form (no outputs; see above).
template <typename T>
cudaError_t blockscan_table_lb(const LaunchCtx &ctx, int mode, const void *in, int64_t in_elems,
                               const SeriesDesc *d_series, const ItemDesc *d_items, int64_t n_items, int *d_ticket,
                               int grid, const void *lb_query, double *lb_acc);

// Chunked monotonic wedge (Algorithm 1 per thread chunk), valid windows,
// w <= MMF_WEDGE_MAX_WINDOW.
template <typename T>
cudaError_t wedge_1d(const LaunchCtx &ctx, const void *in, int64_t n, int64_t w, void *omax, void *omin);
// The same with the locations of the extremes (leftmost among equals), int64.
template <typename T>
cudaError_t wedge_arg_1d(const LaunchCtx &ctx, const void *in, int64_t n, int64_t w, void *omax, void *omin,
                         int64_t *amax, int64_t *amin);
// The window-3 filter in at most two comparisons per element (Section 3);
// ncmp (nullable) accumulates the comparisons made.
template <typename T>
cudaError_t w3_1d(const LaunchCtx &ctx, const void *in, int64_t n, void *omax, void *omin,
                  unsigned long long *ncmp);
// Locations by block scans over (value, position) pairs, any window; windows
// above 2048 take a stream-ordered workspace of per-tile aggregates.
template <typename T>
cudaError_t argscan_1d(const LaunchCtx &ctx, const void *in, int64_t n, int64_t w, void *omax, void *omin,
                       int64_t *amax, int64_t *amin);

// Kernel mode for window w: 3 = register slide (if allowed and w <= 17 for
// f32, 9 otherwise), else
// the block-scan mode 0, 1 or 2.
template <typename T> int block_mode(int64_t w, bool allow_slide);

template <typename T> size_t blockscan_smem_bytes();

// Sets the kernel attributes of one mode on the current device (outside any
// stream capture).
template <typename T> cudaError_t blockscan_prepare(int device, int mode);
int blockscan_tile(int dtype);

}  // namespace mmf
