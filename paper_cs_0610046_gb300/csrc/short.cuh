// Short series (batched plans): one warp per series of at most 32·E elements,
// no CTA barriers.  The block-scan kernel spends a whole tile and two CTA
// barriers on every item; a series of a thousand elements would fill half a
// tile, so short series take this kernel instead.
//
// Per series, lane l holds elements [l·E, l·E + E) in registers.  With blocks
// of B = the largest power of two <= w (Section 2's van Herk/Gil-Werman
// decomposition with blocks no longer than the window, Table 1), every window
// [lo, hi] spans at most three blocks, so
//     out = op(suffix_B[lo], aggregate of the middle block, prefix_B[hi]),
// and a window inside one block starts at the block's start (prefix_B[hi]) or
// ends at the series' end, past which every element is the identity
// (suffix_B[lo]).  Windows clipped to the series (centred mode) are plain
// [max(lo, 0), min(hi, n-1)].  The block scans are thread-local when B <= E,
// else carried across the B/E lanes of a block by shuffles.  Both scans go to
// a warp-private shared array stored element-major (row = position mod E,
// column = lane), so a warp reading one position per lane touches 32
// consecutive words; each output reads two or three of them.  Max and min are
// done one after the other in the same arrays.
#pragma once
#include <cstdint>

#include "blockscan.cuh"
#include "launch.h"

namespace mmf {

template <typename T> struct ShortGeo {
    using R = typename Elem<T>::R;
    static constexpr int E = sizeof(T) == 8 ? 16 : 32;  // elements per lane
    static constexpr int LGE = E == 32 ? 5 : 4;
    static constexpr int NMAX = 32 * E;                  // longest series
    static constexpr int WARPS = 8;                      // per CTA
    static constexpr int ROW = 33;                       // shared row stride (values)
    static constexpr size_t warp_bytes = 2 * (size_t)E * ROW * sizeof(R);
    static constexpr size_t smem_bytes = WARPS * warp_bytes;
};

struct ShortParams {
    const void *in;
    void *out_max;
    void *out_min;
    const SeriesDesc *series;
    const int64_t *ids;  // series of this launch
    int64_t count;
    int64_t in_elems;    // elements of `in` that may be read
    const void *lb_query;  // envelope lower bound (see BlockScanParams)
    double *lb_acc;
    uint32_t *status;
};

extern __shared__ __align__(16) uint8_t short_smem[];

// This lane's E elements of a series starting at src (elements past n are
// read if they lie inside the buffer and ignored later).
template <typename T>
__device__ __forceinline__ void short_load(const T *src, int n, int lane, const T *buf, int64_t buf_n,
                                           typename Elem<T>::R (&x)[ShortGeo<T>::E]) {
    using G = ShortGeo<T>;
    constexpr int E = G::E;
    constexpr int NWD = E * (int)sizeof(T) / 4;
    const T *p = src + lane * E;
    const uintptr_t a = (uintptr_t)p;
    const int sb = (int)(a & 15);
    const uintptr_t al = a - sb;
    const uintptr_t end = al + (uintptr_t)NWD * 4 + (sb ? 16 : 0);
    if (al >= (uintptr_t)buf && end <= (uintptr_t)(buf + buf_n)) {
        uint32_t wd[NWD + 4];
        const uint4 *q = reinterpret_cast<const uint4 *>(al);
#pragma unroll
        for (int c = 0; c < NWD / 4; ++c) {
            const uint4 v = __ldg(q + c);
            wd[4 * c] = v.x; wd[4 * c + 1] = v.y; wd[4 * c + 2] = v.z; wd[4 * c + 3] = v.w;
        }
        if (sb) {
            const uint4 v = __ldg(q + NWD / 4);
            wd[NWD] = v.x; wd[NWD + 1] = v.y; wd[NWD + 2] = v.z; wd[NWD + 3] = v.w;
            shift_bytes<NWD>(wd, sb);
        }
        ExtractLoop<T, 0, 0, E>::run(wd, x);
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = lane * E + e < n ? Elem<T>::load(__ldg(p + e)) : Elem<T>::lo();
    }
}

template <bool MAX, typename R> __device__ __forceinline__ R sop(R a, R b) { return MAX ? vmax(a, b) : vmin(a, b); }

// One side (max or min) of one series: block scans into the warp's arrays,
// then the outputs of this lane's positions into res.  Positions past the
// series' end in v are set to the side's identity first.
template <typename T, bool MAX>
__device__ __forceinline__ void short_side(typename Elem<T>::R (&v)[ShortGeo<T>::E], int n, int w, int d,
                                           int n_out, int lgB, int lane, typename Elem<T>::R *PA,
                                           typename Elem<T>::R *SA, typename Elem<T>::R (&res)[ShortGeo<T>::E]) {
    using G = ShortGeo<T>;
    using R = typename Elem<T>::R;
    constexpr int E = G::E;
    const R id = MAX ? Elem<T>::lo() : Elem<T>::hi();
    const int B = 1 << lgB;
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (lane * E + e >= n) v[e] = id;
    {
        // Prefix within blocks.
        R pre[E];
        pre[0] = v[0];
#pragma unroll
        for (int e = 1; e < E; ++e) pre[e] = (e & (B - 1)) ? sop<MAX>(pre[e - 1], v[e]) : v[e];
        if (lgB > G::LGE) {
            // A block spans 2^(lgB - LGE) lanes: exclusive carry from the
            // earlier lanes of the block.
            const int seg = 1 << (lgB - G::LGE);
            const int pos = lane & (seg - 1);
            R t = pre[E - 1];
#pragma unroll
            for (int k = 1; k < 32; k <<= 1) {
                const R u = __shfl_up_sync(0xffffffffu, t, k);
                if (k < seg && pos >= k) t = sop<MAX>(t, u);
            }
            const R ex = __shfl_up_sync(0xffffffffu, t, 1);
            if (pos) {
#pragma unroll
                for (int e = 0; e < E; ++e) pre[e] = sop<MAX>(pre[e], ex);
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) PA[e * G::ROW + lane] = pre[e];
    }
    {
        // Suffix within blocks.
        R suf[E];
        suf[E - 1] = v[E - 1];
#pragma unroll
        for (int e = E - 2; e >= 0; --e) suf[e] = ((e + 1) & (B - 1)) ? sop<MAX>(suf[e + 1], v[e]) : v[e];
        if (lgB > G::LGE) {
            const int seg = 1 << (lgB - G::LGE);
            const int pos = (seg - 1) - (lane & (seg - 1));
            R t = suf[0];
#pragma unroll
            for (int k = 1; k < 32; k <<= 1) {
                const R u = __shfl_down_sync(0xffffffffu, t, k);
                if (k < seg && pos >= k) t = sop<MAX>(t, u);
            }
            const R ex = __shfl_down_sync(0xffffffffu, t, 1);
            if (pos) {
#pragma unroll
                for (int e = 0; e < E; ++e) suf[e] = sop<MAX>(suf[e], ex);
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) SA[e * G::ROW + lane] = suf[e];
    }
    __syncwarp();
    // Position p lives at row p mod E, column p / E.
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int o = lane * E + e;
        R r = id;
        if (o < n_out) {
            int lo = o + d;
            int hi = lo + w - 1;
            if (lo < 0) lo = 0;
            if (hi > n - 1) hi = n - 1;
            const int bl = lo >> lgB, bh = hi >> lgB;
            const R P = PA[(hi & (E - 1)) * G::ROW + (hi >> G::LGE)];
            const R S = SA[(lo & (E - 1)) * G::ROW + (lo >> G::LGE)];
            if (bl == bh) {
                r = (lo & (B - 1)) == 0 ? P : S;
            } else {
                r = sop<MAX>(S, P);
                if (bh - bl == 2) {
                    const int m = (bl + 1) << lgB;
                    r = sop<MAX>(r, SA[(m & (E - 1)) * G::ROW + (m >> G::LGE)]);
                }
            }
        }
        res[e] = r;
    }
    __syncwarp();
}

template <typename T>
__device__ __forceinline__ void short_store(T *dst, int lane, int n_out, const typename Elem<T>::R (&r)[ShortGeo<T>::E]) {
    constexpr int E = ShortGeo<T>::E;
    T *p = dst + lane * E;
    if (lane * E + E <= n_out && (((uintptr_t)p) & 15) == 0) {
        uint4 *d4 = reinterpret_cast<uint4 *>(p);
#pragma unroll
        for (int c = 0; c < E * (int)sizeof(T) / 16; ++c)
            __stcs(d4 + c, make_uint4(pack_word<T>(r, 4 * c), pack_word<T>(r, 4 * c + 1), pack_word<T>(r, 4 * c + 2),
                                      pack_word<T>(r, 4 * c + 3)));
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (lane * E + e < n_out) p[e] = Elem<T>::store(r[e]);
    }
}

// One side of the envelope lower bound for this lane's positions: the
// squared excursions of the query above the upper envelope (MAX) or below
// the lower one.  The two never both occur at a position (U >= L), so the
// sides add up to the bound's terms.
template <typename T, bool MAX>
__device__ __forceinline__ typename LbAcc<T>::A short_lb_side(const T *query, int lane, int n_out,
                                                              const typename Elem<T>::R (&r)[ShortGeo<T>::E]) {
    using A = typename LbAcc<T>::A;
    constexpr int E = ShortGeo<T>::E;
    const T *q = query + lane * E;
    A part = A(0);
    if (lane * E + E <= n_out && (((uintptr_t)q) & 15) == 0) {
        T qv[E];
#pragma unroll
        for (int c = 0; c < E * (int)sizeof(T) / 16; ++c)
            reinterpret_cast<uint4 *>(qv)[c] = __ldg(reinterpret_cast<const uint4 *>(q) + c);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const A qi = (A)qv[e];
            const A v = (A)Elem<T>::store(r[e]);
            const A dd = MAX ? (qi > v ? qi - v : A(0)) : (qi < v ? v - qi : A(0));
            part += dd * dd;
        }
        return part;
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if (lane * E + e < n_out) {
            const A qi = (A)__ldg(q + e);
            const A v = (A)Elem<T>::store(r[e]);
            const A dd = MAX ? (qi > v ? qi - v : A(0)) : (qi < v ? v - qi : A(0));
            part += dd * dd;
        }
    }
    return part;
}

// LB: the envelope lower bound instead of stored outputs.
template <typename T, bool LB>
__global__ void __launch_bounds__(ShortGeo<T>::WARPS * 32, 2) short_kernel(const ShortParams P) {
    using G = ShortGeo<T>;
    using R = typename Elem<T>::R;
    constexpr int E = G::E;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    R *PA = reinterpret_cast<R *>(short_smem + wib * G::warp_bytes);
    R *SA = PA + E * G::ROW;
    const T *buf = reinterpret_cast<const T *>(P.in);
    const int64_t nwarps = (int64_t)gridDim.x * G::WARPS;
    for (int64_t k = (int64_t)blockIdx.x * G::WARPS + wib; k < P.count; k += nwarps) {
        const int64_t sid = P.ids[k];
        const SeriesDesc sd = P.series[sid];
        const int n = (int)sd.n, d = (int)sd.d, n_out = (int)sd.n_out;
        const int64_t w = sd.w;
        if (n > G::NMAX || n_out <= 0) {
            if (n > G::NMAX && lane == 0) report_error(P.status, kErrBadItem);
            continue;
        }
        if (k + nwarps < P.count) {
            // Bring this warp's next series towards L2 while this one runs.
            const SeriesDesc nx = P.series[P.ids[k + nwarps]];
            if (lane * E < nx.n) prefetch_l2(buf + nx.in_off + lane * E);
        }
        // Windows longer than twice the longest series act like 2·NMAX
        // (every one of them is clipped to the series): 32-bit positions.
        const int wi = (int)(w < 2 * G::NMAX ? w : 2 * G::NMAX);
        int lgB = 0;
        while ((2 << lgB) <= (wi < G::NMAX ? wi : G::NMAX)) ++lgB;
        // Each side loads the series again (L2-resident): the values of one
        // side need not stay in registers through the other.
        using A = typename LbAcc<T>::A;
        A part = A(0);
        {
            R x[E], r[E];
            short_load<T>(buf + sd.in_off, n, lane, buf, P.in_elems, x);
            short_side<T, true>(x, n, wi, d, n_out, lgB, lane, PA, SA, r);
            if constexpr (LB)
                part += short_lb_side<T, true>(reinterpret_cast<const T *>(P.lb_query), lane, n_out, r);
            else if (P.out_max)
                short_store<T>(reinterpret_cast<T *>(P.out_max) + sd.out_off, lane, n_out, r);
        }
        __syncwarp();  // keeps the next side's loads after this side's stores (register pressure)
        {
            R x[E], r[E];
            short_load<T>(buf + sd.in_off, n, lane, buf, P.in_elems, x);
            short_side<T, false>(x, n, wi, d, n_out, lgB, lane, PA, SA, r);
            if constexpr (LB)
                part += short_lb_side<T, false>(reinterpret_cast<const T *>(P.lb_query), lane, n_out, r);
            else if (P.out_min)
                short_store<T>(reinterpret_cast<T *>(P.out_min) + sd.out_off, lane, n_out, r);
        }
        if constexpr (LB) {
            // This warp owns the series: the sum needs no atomics (the
            // accumulator was cleared before the launch).
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) part += __shfl_xor_sync(0xffffffffu, part, s);
            if (lane == 0) P.lb_acc[sid] = (double)part;
        }
    }
}

// Sets the shared-memory attribute of both variants once per device (outside
// any stream capture) and returns the resident CTAs per SM.
template <typename T> cudaError_t short_prepare(int device, bool lb, int *per_sm) {
    using G = ShortGeo<T>;
    static int occ[2][64] = {};
    int &k = occ[lb][device & 63];
    if (k == 0) {
        cudaError_t e = lb ? cudaFuncSetAttribute(short_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)G::smem_bytes)
                           : cudaFuncSetAttribute(short_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)G::smem_bytes);
        if (e != cudaSuccess) return e;
        e = lb ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, short_kernel<T, true>, G::WARPS * 32, G::smem_bytes)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, short_kernel<T, false>, G::WARPS * 32, G::smem_bytes);
        if (e != cudaSuccess) return e;
        if (k < 1) k = 1;
    }
    *per_sm = k;
    return cudaSuccess;
}

// Launch over d_ids[0..count): one wave of persistent CTAs.
template <typename T>
cudaError_t short_table(const LaunchCtx &ctx, const void *in, int64_t in_elems, void *omax, void *omin,
                        const SeriesDesc *d_series, const int64_t *d_ids, int64_t count, const void *lb_query,
                        double *lb_acc) {
    using G = ShortGeo<T>;
    static_assert(G::NMAX == short_max_len(sizeof(T)), "host and kernel agree on short series");
    if (count <= 0) return cudaSuccess;
    const bool lb = lb_acc != nullptr;
    int k = 1;
    cudaError_t pe = short_prepare<T>(ctx.device, lb, &k);
    if (pe != cudaSuccess) return pe;
    ShortParams P{};
    P.in = in;
    P.out_max = omax;
    P.out_min = omin;
    P.series = d_series;
    P.ids = d_ids;
    P.count = count;
    P.in_elems = in_elems;
    P.lb_query = lb_query;
    P.lb_acc = lb_acc;
    P.status = ctx.status;
    const int64_t need = (count + G::WARPS - 1) / G::WARPS;
    const int64_t wave = (int64_t)(ctx.sms > 0 ? ctx.sms : 1) * k;
    const unsigned grid = (unsigned)(need < wave ? need : wave);
    if (lb)
        short_kernel<T, true><<<grid, G::WARPS * 32, G::smem_bytes, ctx.stream>>>(P);
    else
        short_kernel<T, false><<<grid, G::WARPS * 32, G::smem_bytes, ctx.stream>>>(P);
    return cudaGetLastError();
}

}  // namespace mmf
