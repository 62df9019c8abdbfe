// Host launchers of the block-scan kernel, instantiated once per dtype.
#pragma once
#include "launch.h"

namespace mmf {

template <typename T> size_t blockscan_smem_bytes() { return Geo<T>::smem_bytes; }

template <typename T> static cudaError_t prepare_blockscan(int device) {
    static bool done[64] = {false};
    if (device >= 0 && device < 64 && done[device]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(blockscan_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Geo<T>::smem_bytes);
    if (e == cudaSuccess && device >= 0 && device < 64) done[device] = true;
    return e;
}

template <typename T>
cudaError_t blockscan_1d(const LaunchCtx &ctx, const void *in, const SeriesDesc &sd, void *omax, void *omin) {
    using G = Geo<T>;
    if (sd.n_out <= 0) return cudaSuccess;
    cudaError_t e = prepare_blockscan<T>(ctx.device);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (sd.n_out + G::T_ - 1) / G::T_;
    const int64_t gmax = ctx.sms > 0 ? ctx.sms : 1;
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
    cudaError_t e = prepare_blockscan<T>(ctx.device);
    if (e != cudaSuccess) return e;
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
