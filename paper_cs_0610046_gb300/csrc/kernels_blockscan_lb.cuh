// The block-scan table launch in its envelope lower-bound form: the LB
// instantiations of the kernel (outputs feed a per-series sum instead of
// being stored).  Only the k_*_lb.cu units include this header, so the
// storing kernels' units compile none of it.
#pragma once
#include "kernels_blockscan.cuh"

namespace mmf {

template <typename T>
cudaError_t blockscan_table_lb(const LaunchCtx &ctx, int mode, const void *in, int64_t in_elems,
                               const SeriesDesc *d_series, const ItemDesc *d_items, int64_t n_items, int *d_ticket,
                               int grid, const void *lb_query, double *lb_acc) {
    int per_sm = 1;
    cudaError_t e = prepare_mode<T, true>(mode, ctx.device, &per_sm);
    if (e != cudaSuccess) return e;
    if (grid <= 0) grid = (ctx.sms > 0 ? ctx.sms : 1) * per_sm;
    BlockScanParams P{};
    P.in = in;
    P.series = d_series;
    P.items = d_items;
    P.n_items = n_items;
    P.ticket = d_ticket;
    P.status = ctx.status;
    P.in_elems = in_elems;
    P.lb_query = lb_query;
    P.lb_acc = lb_acc;
    apply_test_hooks(P);
    launch_mode<T, true>(mode, P, grid, ctx.stream);
    return cudaGetLastError();
}

}  // namespace mmf

#define MMF_INSTANTIATE_BLOCKSCAN_LB(T)                                                                     \
    template cudaError_t mmf::blockscan_table_lb<T>(const LaunchCtx &, int, const void *, int64_t,          \
                                                     const SeriesDesc *, const ItemDesc *, int64_t, int *, int, \
                                                     const void *, double *);
