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
template <typename T, int MODE, bool LB = false> static cudaError_t prepare_blockscan(int device, int *per_sm) {
    static int occ[64] = {0};
    if (device >= 0 && device < 64 && occ[device] > 0) {
        *per_sm = occ[device];
        return cudaSuccess;
    }
    const size_t smem = smem_of<T>(MODE);
    cudaError_t e = cudaFuncSetAttribute(blockscan_kernel<T, MODE, LB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int k = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, blockscan_kernel<T, MODE, LB>, Geo<T>::NT, smem);
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

template <typename T>
cudaError_t blockscan_1d(const LaunchCtx &ctx, const void *in, const SeriesDesc &sd, void *omax, void *omin,
                         bool allow_slide) {
    using G = Geo<T>;
    if (sd.n_out <= 0) return cudaSuccess;
    const int mode = block_mode<T>(sd.w, allow_slide);
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
                                               void *, bool);                                                   \
    template cudaError_t mmf::blockscan_table<T>(const LaunchCtx &, int, const void *, int64_t, void *, void *, \
                                                  const SeriesDesc *, const ItemDesc *, int64_t, int *, int,    \
                                                  const void *, double *);                                      \
    template int mmf::block_mode<T>(int64_t, bool);                                                            \
    template cudaError_t mmf::short_table<T>(const LaunchCtx &, const void *, int64_t, void *, void *,         \
                                              const SeriesDesc *, const int64_t *, int64_t, const void *, double *, \
                                              int64_t);                                                          \
    template cudaError_t mmf::short_prepare<T>(int, bool, int *);
