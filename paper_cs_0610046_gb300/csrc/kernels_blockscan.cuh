// Host launchers of the block-scan kernel, instantiated once per dtype.
#pragma once
#include "launch.h"

namespace mmf {

template <typename T> size_t blockscan_smem_bytes() { return Geo<T>::smem_bytes; }

// Sets the shared-memory attribute once per device and returns the number of
// resident CTAs per SM.
template <typename T> static cudaError_t prepare_blockscan(int device, int *per_sm) {
    static int occ[64] = {0};
    if (device >= 0 && device < 64 && occ[device] > 0) {
        *per_sm = occ[device];
        return cudaSuccess;
    }
    cudaError_t e = cudaFuncSetAttribute(blockscan_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Geo<T>::smem_bytes);
    if (e != cudaSuccess) return e;
    int k = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, blockscan_kernel<T>, kThreads, Geo<T>::smem_bytes);
    if (e != cudaSuccess) return e;
    if (k < 1) k = 1;
    if (device >= 0 && device < 64) occ[device] = k;
    *per_sm = k;
    return cudaSuccess;
}

template <typename T>
cudaError_t blockscan_1d(const LaunchCtx &ctx, const void *in, const SeriesDesc &sd, void *omax, void *omin) {
    using G = Geo<T>;
    if (sd.n_out <= 0) return cudaSuccess;
    int per_sm = 1;
    cudaError_t e = prepare_blockscan<T>(ctx.device, &per_sm);
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
    blockscan_kernel<T><<<(unsigned)n_items, kThreads, G::smem_bytes, ctx.stream>>>(P);
    return cudaGetLastError();
}

template <typename T>
cudaError_t blockscan_table(const LaunchCtx &ctx, const void *in, void *omax, void *omin, const SeriesDesc *d_series,
                            const ItemDesc *d_items, int64_t n_items, int *d_ticket, int grid) {
    using G = Geo<T>;
    if (n_items <= 0) return cudaSuccess;
    int per_sm = 1;
    cudaError_t e = prepare_blockscan<T>(ctx.device, &per_sm);
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
    blockscan_kernel<T><<<(unsigned)grid, kThreads, G::smem_bytes, ctx.stream>>>(P);
    return cudaGetLastError();
}

}  // namespace mmf

#define MMF_INSTANTIATE_BLOCKSCAN(T)                                                                             \
    template size_t mmf::blockscan_smem_bytes<T>();                                                            \
    template cudaError_t mmf::blockscan_1d<T>(const LaunchCtx &, const void *, const SeriesDesc &, void *,      \
                                               void *);                                                         \
    template cudaError_t mmf::blockscan_table<T>(const LaunchCtx &, const void *, void *, void *,              \
                                                  const SeriesDesc *, const ItemDesc *, int64_t, int *, int);
