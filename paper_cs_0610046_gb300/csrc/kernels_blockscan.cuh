// Host launchers of the block-scan kernel, instantiated once per dtype.
#pragma once
#include "launch.h"
#include "short.cuh"

namespace mmf {

template <typename T> size_t blockscan_smem_bytes() { return Geo<T>::smem_bytes; }

template <typename T> constexpr size_t smem_of(int mode) {
    return mode == 3 ? Geo<T>::smem_bytes_slide : Geo<T>::smem_bytes;
}

// Sets the shared-memory attribute once per device and returns the number of
// resident CTAs per SM.
template <typename T, int MODE, bool LB = false, bool FRONT = false>
static cudaError_t prepare_blockscan(int device, int *per_sm) {
    static int occ[64] = {0};
    if (device >= 0 && device < 64 && occ[device] > 0) {
        *per_sm = occ[device];
        return cudaSuccess;
    }
    const size_t smem = smem_of<T>(MODE);
    cudaError_t e = cudaFuncSetAttribute(blockscan_kernel<T, MODE, LB, FRONT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int k = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, blockscan_kernel<T, MODE, LB, FRONT>, Geo<T>::NT, smem);
    if (e != cudaSuccess) return e;
    if (k < 1) k = 1;
    if (device >= 0 && device < 64) occ[device] = k;
    *per_sm = k;
    return cudaSuccess;
}

// Kernel mode for window w: 3 = register slide (w <= 17 for f32, 9 for the
// other types, unless a block scan is forced), else the block-scan mode 0, 1
// or 2.
template <typename T> int block_mode(int64_t w, bool allow_slide) {
    const int64_t s = w - 1;
    if (allow_slide && s <= Geo<T>::SLIDE_S) return 3;
    if (s >= 32 * (int64_t)Geo<T>::V) return 2;
    return s >= Geo<T>::V ? 1 : 0;
}

template <typename T, int MODE, bool LB = false>
static void launch_bs(const BlockScanParams &P, int grid, cudaStream_t st) {
    blockscan_kernel<T, MODE, LB><<<(unsigned)grid, Geo<T>::NT, smem_of<T>(MODE), st>>>(P);
}

template <typename T, bool LB = false>
static cudaError_t prepare_mode(int mode, int device, int *per_sm) {
    switch (mode) {
        case 0: return prepare_blockscan<T, 0, LB>(device, per_sm);
        case 1: return prepare_blockscan<T, 1, LB>(device, per_sm);
        case 2: return prepare_blockscan<T, 2, LB>(device, per_sm);
        default: return prepare_blockscan<T, 3, LB>(device, per_sm);
    }
}

template <typename T, bool LB = false>
static void launch_mode(int mode, const BlockScanParams &P, int grid, cudaStream_t st) {
    switch (mode) {
        case 0: launch_bs<T, 0, LB>(P, grid, st); break;
        case 1: launch_bs<T, 1, LB>(P, grid, st); break;
        case 2: launch_bs<T, 2, LB>(P, grid, st); break;
        default: launch_bs<T, 3, LB>(P, grid, st); break;
    }
}

template <typename T> cudaError_t blockscan_prepare(int device, int mode) {
    int per_sm = 1;
    return prepare_mode<T>(mode, device, &per_sm);
}

template <typename T> bool front_applies(const SeriesDesc &sd, int sms, int front) {
    using G = Geo<T>;
    const int64_t q = (sd.w - 1) / G::T_;
    if (!kCarryRing<T> || q < 1 || front == 0 || block_mode<T>(sd.w, true) != 2) return false;
    const int64_t tiles = (sd.n_out + G::T_ - 1) / G::T_;
    if (tiles + q + 2 >= 0xffffffffLL) return false;  // slot tags are 32-bit tile numbers
    // Only on request (or by a tuned dispatch entry): on the long-stream
    // workload the per-range schedule is still the faster one.
    (void)sms;
    return front == 1;
}

// One advancing front: the persistent grid of G CTAs takes output tiles
// round-robin (CTA b: tiles b, b+G, b+2G, ...) in a cooperative launch, so
// that every CTA is resident while others wait for its aggregates and all
// CTAs move through the series together.  Round t reads tile t+q+G ahead and
// publishes its aggregate for the rounds of the next pass of the grid, to a
// stream-ordered workspace [16 bytes | two tagged words per global tile],
// cleared before the launch and returned after it.
template <typename T>
static cudaError_t blockscan_front(const LaunchCtx &ctx, const void *in, const SeriesDesc &sd, void *omax,
                                   void *omin) {
    using G = Geo<T>;
    int per_sm = 1;
    cudaError_t e = prepare_blockscan<T, 2, false, true>(ctx.device, &per_sm);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (sd.n_out + G::T_ - 1) / G::T_;
    const int64_t q = (sd.w - 1) / G::T_;
    const int64_t nglob = tiles + q + 2;  // global tiles an item may publish
    const size_t bytes = 16 + (size_t)nglob * 16;
    uint8_t *ws = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void **>(&ws), bytes, ctx.stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(ws, 0, bytes, ctx.stream);
    if (e == cudaSuccess) {
        BlockScanParams P{};
        P.in = in;
        P.out_max = omax;
        P.out_min = omin;
        P.one = sd;
        P.seg_outputs = G::T_;
        P.n_items = tiles;
        P.ticket = nullptr;
        P.status = ctx.status;
        P.in_elems = sd.in_off + sd.n;
        P.front_slots = reinterpret_cast<unsigned long long *>(ws + 16);
        const int64_t gmax = (int64_t)(ctx.sms > 0 ? ctx.sms : 1) * per_sm;
        const int grid = (int)(tiles < gmax ? tiles : gmax);
        P.front_ahead = grid;
        P.front_last = tiles + q - 2;  // tile t+q-1 of the last output tile t
        apply_test_hooks(P);
        void *args[] = {(void *)&P};
        e = cudaLaunchCooperativeKernel((const void *)blockscan_kernel<T, 2, false, true>, dim3(grid), dim3(G::NT),
                                        args, smem_of<T>(2), ctx.stream);
    }
    const cudaError_t f = cudaFreeAsync(ws, ctx.stream);
    return e != cudaSuccess ? e : f;
}

template <typename T>
cudaError_t blockscan_1d(const LaunchCtx &ctx, const void *in, const SeriesDesc &sd, void *omax, void *omin,
                         bool allow_slide, int front) {
    using G = Geo<T>;
    if (sd.n_out <= 0) return cudaSuccess;
    const int mode = block_mode<T>(sd.w, allow_slide);
    if constexpr (kCarryRing<T>) {
        if (mode == 2 && front_applies<T>(sd, ctx.sms, front)) return blockscan_front<T>(ctx, in, sd, omax, omin);
    }
    int per_sm = 1;
    cudaError_t e = prepare_mode<T>(mode, ctx.device, &per_sm);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (sd.n_out + G::T_ - 1) / G::T_;
    const int64_t gmax = (int64_t)(ctx.sms > 0 ? ctx.sms : 1) * per_sm;
    const int64_t seg_tiles = (tiles + gmax - 1) / gmax;
    const int64_t n_items = (tiles + seg_tiles - 1) / seg_tiles;
    BlockScanParams P{};
    P.in = in;
    P.out_max = omax;
    P.out_min = omin;
    P.series = nullptr;
    P.items = nullptr;
    P.one = sd;
    P.seg_outputs = seg_tiles * G::T_;
    P.n_items = n_items;
    P.ticket = nullptr;
    P.status = ctx.status;
    P.in_elems = sd.in_off + sd.n;
    apply_test_hooks(P);
    launch_mode<T>(mode, P, (int)n_items, ctx.stream);
    return cudaGetLastError();
}

template <typename T>
cudaError_t blockscan_rows(const LaunchCtx &ctx, const void *in, const SeriesDesc &sd, int64_t rows, int64_t in_pitch,
                           int64_t out_pitch, void *omax, void *omin) {
    using G = Geo<T>;
    if (sd.n_out <= 0 || rows <= 0) return cudaSuccess;
    const int mode = block_mode<T>(sd.w, true);
    int per_sm = 1;
    cudaError_t e = prepare_mode<T>(mode, ctx.device, &per_sm);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (sd.n_out + G::T_ - 1) / G::T_;
    const int64_t seg_tiles = tiles < 64 ? tiles : 64;
    const int64_t row_items = (tiles + seg_tiles - 1) / seg_tiles;
    BlockScanParams P{};
    P.in = in;
    P.out_max = omax;
    P.out_min = omin;
    P.one = sd;
    P.seg_outputs = seg_tiles * G::T_;
    P.row_items = row_items;
    P.in_pitch = in_pitch;
    P.out_pitch = out_pitch;
    P.n_items = rows * row_items;
    P.status = ctx.status;
    P.in_elems = (rows - 1) * in_pitch + sd.in_off + sd.n;
    const int64_t gmax = (int64_t)(ctx.sms > 0 ? ctx.sms : 1) * per_sm;
    apply_test_hooks(P);
    launch_mode<T>(mode, P, (int)(P.n_items < gmax ? P.n_items : gmax), ctx.stream);
    return cudaGetLastError();
}

template <typename T>
cudaError_t blockscan_table(const LaunchCtx &ctx, int mode, const void *in, int64_t in_elems, void *omax,
                            void *omin, const SeriesDesc *d_series, const ItemDesc *d_items, int64_t n_items,
                            int *d_ticket, int grid, const void *lb_query, double *lb_acc) {
    if (n_items <= 0) return cudaSuccess;
    if (lb_acc)  // the lower-bound kernels live in their own translation units
        return blockscan_table_lb<T>(ctx, mode, in, in_elems, d_series, d_items, n_items, d_ticket, grid, lb_query,
                                     lb_acc);
    int per_sm = 1;
    cudaError_t e = prepare_mode<T>(mode, ctx.device, &per_sm);
    if (e != cudaSuccess) return e;
    if (grid <= 0) grid = (ctx.sms > 0 ? ctx.sms : 1) * per_sm;
    BlockScanParams P{};
    P.in = in;
    P.out_max = omax;
    P.out_min = omin;
    P.series = d_series;
    P.items = d_items;
    P.seg_outputs = 0;
    P.n_items = n_items;
    P.ticket = d_ticket;
    P.status = ctx.status;
    P.in_elems = in_elems;
    P.lb_query = lb_query;
    P.lb_acc = lb_acc;
    apply_test_hooks(P);
    launch_mode<T>(mode, P, grid, ctx.stream);
    return cudaGetLastError();
}

}  // namespace mmf

#define MMF_INSTANTIATE_BLOCKSCAN(T)                                                                             \
    template size_t mmf::blockscan_smem_bytes<T>();                                                            \
    template cudaError_t mmf::blockscan_prepare<T>(int, int);                                                  \
    template cudaError_t mmf::blockscan_rows<T>(const LaunchCtx &, const void *, const SeriesDesc &, int64_t,   \
                                                int64_t, int64_t, void *, void *);                            \
    template cudaError_t mmf::blockscan_1d<T>(const LaunchCtx &, const void *, const SeriesDesc &, void *,      \
                                               void *, bool, int);                                              \
    template bool mmf::front_applies<T>(const SeriesDesc &, int, int);                                         \
    template cudaError_t mmf::blockscan_table<T>(const LaunchCtx &, int, const void *, int64_t, void *, void *, \
                                                  const SeriesDesc *, const ItemDesc *, int64_t, int *, int,    \
                                                  const void *, double *);                                      \
    template int mmf::block_mode<T>(int64_t, bool);                                                            \
    template cudaError_t mmf::short_table<T>(const LaunchCtx &, const void *, int64_t, void *, void *,         \
                                              const SeriesDesc *, const int64_t *, int64_t, const void *, double *, \
                                              int64_t);                                                          \
    template cudaError_t mmf::short_prepare<T>(int, bool, int *);
