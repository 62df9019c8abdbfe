// Arg-max / arg-min filter for any window: van Herk/Gil-Werman block scans
// (Section 2) over (value, position) pairs.
//
// Blocks of w positions start at multiples of w.  The window [j, j+w) of an
// output j = b*w + r is the suffix of block b from j followed by the first r
// positions of block b+1; with y[i] = x[i+w] and the blocks as segments,
//     out[j] = S[j] (+) Q[j],  S = segmented inclusive suffix scan of x,
//                              Q = segmented exclusive prefix scan of y.
// Every position in S's range lies left of every position in Q's range, so
// keeping S on equal values keeps the leftmost position; inside each scan the
// earlier position is kept on ties.  The result is the leftmost extreme of
// the window, the same as a left-to-right scan of the window that replaces
// its candidate only on a strictly larger (smaller) value.
//
// One CTA covers a tile of positions [base, base+len):
//   * w <= kArgTile: whole blocks (len = floor(kArgTile/w)*w), nothing
//     crosses the tile;
//   * w > kArgTile: tile t of block b (positions t*kArgTile.. of the block).
//     The part of S right of the tile and the part of Q left of it are
//     per-tile aggregates scanned within each block (argagg_kernel and
//     argblock_scan_kernel below), read as the CTA's two carries.
// Each thread holds E consecutive positions.  A local sweep in each direction
// gives its summary (the aggregate up to its first / last segment boundary
// and whether it has one), a segmented scan of the summaries across the CTA
// (warp shuffles, then warp totals) gives the carry into the thread, and the
// final sweeps form the outputs, which leave through shared memory in
// coalesced stores.  The max and min sides run one after the other on the
// same staged inputs.
#include <climits>
#include <cstdint>

#include "launch.h"
#include "mmf.h"

namespace mmf {
namespace {

constexpr int kArgThreads = 256, kArgE = 8, kArgTile = kArgThreads * kArgE, kArgWarps = kArgThreads / 32;
// Position codes while scanning: 0..kArgTile-1 an x position of the tile,
// kArgTile + p the y position p, and the carries and the empty aggregate.
constexpr int kCodeSC = -1, kCodeQC = -2, kCodeNone = -3;

template <typename K> struct VI {
    K v;
    int i;
};

// Aggregate of a range for both sides; empty ranges hold the identities and
// position INT64_MAX.
template <typename K> struct Agg {
    K vmax, vmin;
    long long imax, imin;
};

// Identities strictly outside the keys of real values where the key type has
// room (doubles are order-preserving 64-bit keys, 8/16-bit values are ints);
// f32 uses -inf/+inf, which equal values in the data only lose ties (the
// proof is in the sweeps: an identity never beats a real position).
template <typename K> struct KeyLim;
template <> struct KeyLim<float> {
    __device__ static float lo() { return __int_as_float(0xff800000); }
    __device__ static float hi() { return __int_as_float(0x7f800000); }
};
template <> struct KeyLim<long long> {
    __device__ static long long lo() { return LLONG_MIN; }
    __device__ static long long hi() { return LLONG_MAX; }
};
template <> struct KeyLim<int> {
    __device__ static int lo() { return INT_MIN; }
    __device__ static int hi() { return INT_MAX; }
};

template <typename K, bool MAX> struct Side {
    __device__ static K id() { return MAX ? KeyLim<K>::lo() : KeyLim<K>::hi(); }
    __device__ static bool better(K a, K b) { return MAX ? a > b : a < b; }
    // a left of b: b only when strictly better.
    __device__ static VI<K> join(VI<K> a, VI<K> b) { return better(b.v, a.v) ? b : a; }
};

// Shared-memory index with one padding slot per 128 bytes, so E consecutive
// elements per thread spread over the banks.
template <typename K> __device__ __forceinline__ int padk(int p) { return p + p / (128 / (int)sizeof(K)); }
template <typename K> __host__ __device__ constexpr int padded_len() { return kArgTile + kArgTile / (128 / (int)sizeof(K)); }

template <typename T> struct ArgParams {
    const T *x;
    long long n, w, n_out;
    T *omax, *omin;
    long long *amax, *amin;
    long long ntiles;  // tiles per block (w > kArgTile), 0 for whole blocks per CTA
    int len_small;     // positions per CTA for whole blocks
    const Agg<typename Elem<T>::R> *pg, *sg;  // per-tile prefix / suffix aggregates
};

template <typename K> struct ArgScanSmem {
    VI<K> ft[kArgWarps], bt[kArgWarps];
    int ff[kArgWarps], bf[kArgWarps];
};

template <typename K> __device__ __forceinline__ VI<K> shfl_up_vi(VI<K> a, int d) {
    return VI<K>{__shfl_up_sync(0xffffffffu, a.v, d), __shfl_up_sync(0xffffffffu, a.i, d)};
}
template <typename K> __device__ __forceinline__ VI<K> shfl_down_vi(VI<K> a, int d) {
    return VI<K>{__shfl_down_sync(0xffffffffu, a.v, d), __shfl_down_sync(0xffffffffu, a.i, d)};
}

template <typename T, bool MAX>
__device__ __forceinline__ void arg_side(const ArgParams<T> &P, long long base, int len, int xlim, int ylim,
                                         unsigned smask, unsigned emask, const typename Elem<T>::R *xs,
                                         const typename Elem<T>::R *ys, typename Elem<T>::R *vo, long long *io,
                                         VI<typename Elem<T>::R> qc, long long qci, VI<typename Elem<T>::R> sc,
                                         long long sci, ArgScanSmem<typename Elem<T>::R> &sm) {
    using K = typename Elem<T>::R;
    using S = Side<K, MAX>;
    const K ID = S::id();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, p0 = tid * kArgE;
    const VI<K> none{ID, kCodeNone};

    // 1. Summaries: forward over y (Q), backward over x (S).
    VI<K> fs = none, bs = none;
    int ff = 0, bf = 0;
#pragma unroll
    for (int k = 0; k < kArgE; ++k) {
        const int p = p0 + k;
        if ((smask >> k) & 1u) {
            fs = none;
            ff = 1;
        }
        const K y = p < ylim ? ys[padk<K>(p)] : ID;
        if (S::better(y, fs.v)) fs = VI<K>{y, kArgTile + p};
    }
#pragma unroll
    for (int k = kArgE - 1; k >= 0; --k) {
        const int p = p0 + k;
        if ((emask >> k) & 1u) {
            bs = none;
            bf = 1;
        }
        const K x = p < xlim ? xs[padk<K>(p)] : ID;
        if (!S::better(bs.v, x)) bs = VI<K>{x, p};
    }

    // 2. Segmented scans of the summaries: inclusive within the warp...
    VI<K> fi = fs, bi = bs;
    int fif = ff, bif = bf;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const VI<K> l = shfl_up_vi(fi, d);
        const int lf = __shfl_up_sync(0xffffffffu, fif, d);
        if (lane >= d) {
            if (!fif) fi = S::join(l, fi);
            fif |= lf;
        }
        const VI<K> r = shfl_down_vi(bi, d);
        const int rf = __shfl_down_sync(0xffffffffu, bif, d);
        if (lane + d < 32) {
            if (!bif) bi = S::join(bi, r);
            bif |= rf;
        }
    }
    if (lane == 31) {
        sm.ft[warp] = fi;
        sm.ff[warp] = fif;
    }
    if (lane == 0) {
        sm.bt[warp] = bi;
        sm.bf[warp] = bif;
    }
    // ... exclusive within the warp ...
    VI<K> fe = shfl_up_vi(fi, 1), be = shfl_down_vi(bi, 1);
    int fef = __shfl_up_sync(0xffffffffu, fif, 1), bef = __shfl_down_sync(0xffffffffu, bif, 1);
    if (lane == 0) {
        fe = none;
        fef = 0;
    }
    if (lane == 31) {
        be = none;
        bef = 0;
    }
    __syncthreads();
    // ... then across warps, with the tile's carries at the two ends.
    VI<K> cf = qc;
    for (int u = 0; u < warp; ++u) cf = sm.ff[u] ? sm.ft[u] : S::join(cf, sm.ft[u]);
    cf = fef ? fe : S::join(cf, fe);
    VI<K> cb = sc;
    for (int u = kArgWarps - 1; u > warp; --u) cb = sm.bf[u] ? sm.bt[u] : S::join(sm.bt[u], cb);
    cb = bef ? be : S::join(be, cb);

    // 3. Final sweeps: Q forward into registers, then S backward joined with Q.
    K qv[kArgE];
    int qi[kArgE];
    VI<K> acc = cf;
#pragma unroll
    for (int k = 0; k < kArgE; ++k) {
        const int p = p0 + k;
        if ((smask >> k) & 1u) acc = none;
        qv[k] = acc.v;
        qi[k] = acc.i;
        const K y = p < ylim ? ys[padk<K>(p)] : ID;
        if (S::better(y, acc.v)) acc = VI<K>{y, kArgTile + p};
    }
    acc = cb;
#pragma unroll
    for (int k = kArgE - 1; k >= 0; --k) {
        const int p = p0 + k;
        if ((emask >> k) & 1u) acc = none;
        const K x = p < xlim ? xs[padk<K>(p)] : ID;
        if (!S::better(acc.v, x)) acc = VI<K>{x, p};
        const bool useq = S::better(qv[k], acc.v);
        const int c = useq ? qi[k] : acc.i;
        // An output of the tile always has its own x in S, so the empty code
        // never reaches a stored output (the last case only fills the slot).
        const long long g = c >= kArgTile ? base + P.w + (c - kArgTile)
                            : c >= 0      ? base + c
                            : c == kCodeSC ? sci
                            : c == kCodeQC ? qci
                                           : base + p;
        vo[padk<K>(p)] = useq ? qv[k] : acc.v;
        io[padk<long long>(p)] = g;
    }
    __syncthreads();
    T *oval = MAX ? P.omax : P.omin;
    long long *oidx = MAX ? P.amax : P.amin;
    const int nv = (int)min((long long)len, P.n_out - base);
    for (int i = tid; i < nv; i += kArgThreads) {
        if (oval) oval[base + i] = Elem<T>::store(vo[padk<K>(i)]);
        if (oidx) oidx[base + i] = io[padk<long long>(i)];
    }
}

template <typename T>
__global__ void __launch_bounds__(kArgThreads) argscan_kernel(const ArgParams<T> P) {
    using K = typename Elem<T>::R;
    extern __shared__ __align__(16) unsigned char arg_smem[];
    __shared__ ArgScanSmem<K> sm;
    constexpr int PK = padded_len<K>();
    K *xs = reinterpret_cast<K *>(arg_smem);
    K *ys = xs + PK;
    K *vo = ys + PK;
    long long *io = reinterpret_cast<long long *>(vo + PK);

    const int tid = threadIdx.x;
    long long base, r0, b = 0, t = 0;
    int len;
    if (P.ntiles == 0) {
        len = P.len_small;
        base = (long long)blockIdx.x * len;
        r0 = 0;
    } else {
        b = (long long)blockIdx.x / P.ntiles;
        t = (long long)blockIdx.x % P.ntiles;
        r0 = t * kArgTile;
        base = b * P.w + r0;
        len = (int)min((long long)kArgTile, P.w - r0);
    }
    if (base >= P.n_out) return;  // uniform per CTA, before any barrier
    const int xlim = (int)max(0LL, min((long long)len, P.n - base));
    const int ylim = (int)max(0LL, min((long long)len, P.n - base - P.w));

    // Stage x[base..) and y[base..) = x[base+w..) as keys (coalesced loads,
    // all issued before the first shared-memory store).
    T xv[kArgE], yv[kArgE];
#pragma unroll
    for (int k = 0; k < kArgE; ++k) {
        const int i = tid + k * kArgThreads;
        xv[k] = i < xlim ? __ldg(P.x + base + i) : T(0);
        yv[k] = i < ylim ? __ldg(P.x + base + P.w + i) : T(0);
    }
#pragma unroll
    for (int k = 0; k < kArgE; ++k) {
        const int i = tid + k * kArgThreads;
        xs[padk<K>(i)] = Elem<T>::load(xv[k]);
        ys[padk<K>(i)] = Elem<T>::load(yv[k]);
    }

    // Segment starts (phase 0) and ends (phase w-1) among the thread's positions.
    const int p0 = tid * kArgE;
    unsigned smask = 0, emask = 0;
    {
        long long r = P.ntiles == 0 ? (long long)(p0 % (int)P.w) : r0 + p0;
#pragma unroll
        for (int k = 0; k < kArgE; ++k) {
            if (r == 0) smask |= 1u << k;
            if (r == P.w - 1) emask |= 1u << k;
            if (++r == P.w) r = 0;
        }
    }

    // Carries of a tile inside a long block: Q's part left of the tile (the
    // start of block b+1 up to tile t) and S's part right of it (the rest of
    // block b after tile t).
    VI<K> qmx{KeyLim<K>::lo(), kCodeNone}, qmn{KeyLim<K>::hi(), kCodeNone};
    VI<K> smx{KeyLim<K>::lo(), kCodeNone}, smn{KeyLim<K>::hi(), kCodeNone};
    long long qmxi = 0, qmni = 0, smxi = 0, smni = 0;
    if (P.ntiles != 0) {
        if (t > 0) {
            const Agg<K> a = P.pg[(b + 1) * P.ntiles + t - 1];
            qmx = VI<K>{a.vmax, kCodeQC};
            qmn = VI<K>{a.vmin, kCodeQC};
            qmxi = a.imax;
            qmni = a.imin;
        }
        if (t + 1 < P.ntiles) {
            const Agg<K> a = P.sg[b * P.ntiles + t + 1];
            smx = VI<K>{a.vmax, kCodeSC};
            smn = VI<K>{a.vmin, kCodeSC};
            smxi = a.imax;
            smni = a.imin;
        }
    }
    __syncthreads();
    if (P.omax || P.amax)
        arg_side<T, true>(P, base, len, xlim, ylim, smask, emask, xs, ys, vo, io, qmx, qmxi, smx, smxi, sm);
    if (P.omin || P.amin) {
        __syncthreads();  // the staging of the max side has been stored
        arg_side<T, false>(P, base, len, xlim, ylim, smask, emask, xs, ys, vo, io, qmn, qmni, smn, smni, sm);
    }
}

// Both sides of a range, any order of positions: larger (smaller) value,
// then the smaller position.
template <typename K> __device__ __forceinline__ void agg_join(Agg<K> &a, const Agg<K> &b) {
    if (b.vmax > a.vmax || (b.vmax == a.vmax && b.imax < a.imax)) {
        a.vmax = b.vmax;
        a.imax = b.imax;
    }
    if (b.vmin < a.vmin || (b.vmin == a.vmin && b.imin < a.imin)) {
        a.vmin = b.vmin;
        a.imin = b.imin;
    }
}

template <typename K> __device__ __forceinline__ Agg<K> agg_shfl_down(const Agg<K> &a, int d) {
    Agg<K> r;
    r.vmax = __shfl_down_sync(0xffffffffu, a.vmax, d);
    r.vmin = __shfl_down_sync(0xffffffffu, a.vmin, d);
    r.imax = __shfl_down_sync(0xffffffffu, a.imax, d);
    r.imin = __shfl_down_sync(0xffffffffu, a.imin, d);
    return r;
}
template <typename K> __device__ __forceinline__ Agg<K> agg_shfl_up(const Agg<K> &a, int d) {
    Agg<K> r;
    r.vmax = __shfl_up_sync(0xffffffffu, a.vmax, d);
    r.vmin = __shfl_up_sync(0xffffffffu, a.vmin, d);
    r.imax = __shfl_up_sync(0xffffffffu, a.imax, d);
    r.imin = __shfl_up_sync(0xffffffffu, a.imin, d);
    return r;
}

template <typename K> __device__ __forceinline__ Agg<K> agg_empty() {
    return Agg<K>{KeyLim<K>::lo(), KeyLim<K>::hi(), LLONG_MAX, LLONG_MAX};
}

// g[b*ntiles + t] = aggregate of x over tile t of block b (clipped to the
// block and to the array), for blocks 0..nb-1; grid-stride over tiles.
template <typename T>
__global__ void __launch_bounds__(kArgThreads) argagg_kernel(const T *x, long long n, long long w, long long ntiles,
                                                            long long nb, Agg<typename Elem<T>::R> *g) {
    using K = typename Elem<T>::R;
    __shared__ Agg<K> part[kArgWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (long long u = blockIdx.x; u < nb * ntiles; u += gridDim.x) {
        const long long b = u / ntiles, t = u % ntiles;
        const long long lo = b * w + t * kArgTile;
        const long long hi = min(min(lo + kArgTile, (b + 1) * w), n);
        Agg<K> a = agg_empty<K>();
        T v[kArgE];
#pragma unroll
        for (int k = 0; k < kArgE; ++k) {
            const long long i = lo + tid + k * kArgThreads;
            v[k] = i < hi ? __ldg(x + i) : T(0);
        }
#pragma unroll
        for (int k = 0; k < kArgE; ++k) {
            const long long i = lo + tid + k * kArgThreads;
            if (i < hi) {
                const K key = Elem<T>::load(v[k]);
                if (key > a.vmax || a.imax == LLONG_MAX) {
                    a.vmax = key;
                    a.imax = i;
                }
                if (key < a.vmin || a.imin == LLONG_MAX) {
                    a.vmin = key;
                    a.imin = i;
                }
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) agg_join(a, agg_shfl_down(a, d));
        if (lane == 0) part[warp] = a;
        __syncthreads();
        if (tid == 0) {
            for (int q = 1; q < kArgWarps; ++q) agg_join(a, part[q]);
            g[u] = a;
        }
        __syncthreads();
    }
}

// Per block: pg[t] = tiles 0..t joined, sg[t] = tiles t..ntiles-1 joined;
// one warp per block, 32 tiles at a time.
template <typename K>
__global__ void __launch_bounds__(kArgThreads) argblock_scan_kernel(const Agg<K> *g, long long ntiles, long long nb,
                                                                   Agg<K> *pg, Agg<K> *sg) {
    const int lane = threadIdx.x & 31;
    const long long b = (long long)blockIdx.x * kArgWarps + (threadIdx.x >> 5);
    if (b >= nb) return;  // the kernel has no barriers
    const Agg<K> *gb = g + b * ntiles;
    Agg<K> carry = agg_empty<K>();
    for (long long t0 = 0; t0 < ntiles; t0 += 32) {
        const long long t = t0 + lane;
        Agg<K> a = t < ntiles ? gb[t] : agg_empty<K>();
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const Agg<K> l = agg_shfl_up(a, d);
            if (lane >= d) {
                Agg<K> m = l;
                agg_join(m, a);
                a = m;
            }
        }
        Agg<K> m = carry;
        agg_join(m, a);
        if (t < ntiles) pg[b * ntiles + t] = m;
        carry = m;
        carry.vmax = __shfl_sync(0xffffffffu, m.vmax, 31);
        carry.vmin = __shfl_sync(0xffffffffu, m.vmin, 31);
        carry.imax = __shfl_sync(0xffffffffu, m.imax, 31);
        carry.imin = __shfl_sync(0xffffffffu, m.imin, 31);
    }
    carry = agg_empty<K>();
    for (long long t1 = ntiles; t1 > 0; t1 -= 32) {
        const long long t = t1 - 32 + lane;  // lanes below 0 hold nothing
        Agg<K> a = t >= 0 ? gb[t] : agg_empty<K>();
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const Agg<K> r = agg_shfl_down(a, d);
            if (lane + d < 32) agg_join(a, r);
        }
        agg_join(a, carry);
        if (t >= 0) sg[b * ntiles + t] = a;
        carry.vmax = __shfl_sync(0xffffffffu, a.vmax, 0);
        carry.vmin = __shfl_sync(0xffffffffu, a.vmin, 0);
        carry.imax = __shfl_sync(0xffffffffu, a.imax, 0);
        carry.imin = __shfl_sync(0xffffffffu, a.imin, 0);
    }
}

}  // namespace

template <typename T>
cudaError_t argscan_1d(const LaunchCtx &ctx, const void *in, int64_t n, int64_t w, void *omax, void *omin,
                       int64_t *amax, int64_t *amin) {
    using K = typename Elem<T>::R;
    const int64_t n_out = n - w + 1;
    if (n_out <= 0) return cudaSuccess;
    constexpr size_t smem = 3 * (size_t)padded_len<K>() * sizeof(K) + (size_t)padded_len<long long>() * 8;
    static int attr_set[64] = {};
    if (smem > 48 * 1024 && !attr_set[ctx.device & 63]) {
        cudaError_t e = cudaFuncSetAttribute(argscan_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set[ctx.device & 63] = 1;
    }
    ArgParams<T> P{static_cast<const T *>(in), n, w, n_out, static_cast<T *>(omax), static_cast<T *>(omin),
                   reinterpret_cast<long long *>(amax), reinterpret_cast<long long *>(amin), 0, 0, nullptr,
                   nullptr};
    if (w <= kArgTile) {
        P.len_small = (int)((kArgTile / w) * w);
        const int64_t grid = (n_out + P.len_small - 1) / P.len_small;
        argscan_kernel<T><<<(unsigned)grid, kArgThreads, smem, ctx.stream>>>(P);
        return cudaGetLastError();
    }
    const int64_t ntiles = (w + kArgTile - 1) / kArgTile;
    const int64_t nbo = (n_out + w - 1) / w;  // blocks holding outputs
    const int64_t nb = nbo + 1;               // and the block after them (Q)
    const size_t ng = (size_t)(nb * ntiles);
    Agg<K> *ws = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&ws), 3 * ng * sizeof(Agg<K>), ctx.stream);
    if (e != cudaSuccess) return e;
    Agg<K> *g = ws, *pg = ws + ng, *sg = ws + 2 * ng;
    const int64_t sms = ctx.sms > 0 ? ctx.sms : 1;
    const int64_t agg_grid = (int64_t)ng < sms * 8 ? (int64_t)ng : sms * 8;
    argagg_kernel<T><<<(unsigned)agg_grid, kArgThreads, 0, ctx.stream>>>(static_cast<const T *>(in), n, w, ntiles,
                                                                       nb, g);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        argblock_scan_kernel<K><<<(unsigned)((nb + kArgWarps - 1) / kArgWarps), kArgThreads, 0, ctx.stream>>>(
            g, ntiles, nb, pg, sg);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        P.ntiles = ntiles;
        P.pg = pg;
        P.sg = sg;
        argscan_kernel<T><<<(unsigned)(nbo * ntiles), kArgThreads, smem, ctx.stream>>>(P);
        e = cudaGetLastError();
    }
    const cudaError_t ef = cudaFreeAsync(ws, ctx.stream);
    return e != cudaSuccess ? e : ef;
}

template cudaError_t argscan_1d<float>(const LaunchCtx &, const void *, int64_t, int64_t, void *, void *, int64_t *,
                                       int64_t *);
template cudaError_t argscan_1d<double>(const LaunchCtx &, const void *, int64_t, int64_t, void *, void *, int64_t *,
                                        int64_t *);
template cudaError_t argscan_1d<int16_t>(const LaunchCtx &, const void *, int64_t, int64_t, void *, void *,
                                         int64_t *, int64_t *);
template cudaError_t argscan_1d<uint8_t>(const LaunchCtx &, const void *, int64_t, int64_t, void *, void *,
                                         int64_t *, int64_t *);

}  // namespace mmf
