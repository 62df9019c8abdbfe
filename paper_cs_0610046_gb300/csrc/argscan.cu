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
//     crosses the tile; x and y are one staged range [base, base+len+w);
//   * w > kArgTile: tile t of block b (positions t*kArgTile.. of the block).
//     The part of S right of the tile and the part of Q left of it are
//     per-tile aggregates scanned within each block (argagg_kernel and
//     argblock_scan_kernel below), read as the CTA's two carries.
// Each thread holds E consecutive positions and both sides (max, min) at
// once.  One forward sweep forms the local exclusive Q (staged in shared
// memory) and the thread's two summaries (Q from its last segment start, S up
// to its first segment end); a segmented scan of the summaries across the CTA
// (warp shuffles, then warp totals) gives the carries into the thread; one
// backward sweep forms S, completes Q with its carry and joins them.  Outputs
// leave through shared memory in 16-byte stores.
//
// Positions are offsets from base (x: p, y: w+p, carries inside [0, w+len)):
// unsigned 32-bit for w < 2^30, else 64-bit.  f32, i16 and u8 compare as
// float keys (exact for 8- and 16-bit integers), so a NaN marks staged
// positions outside the array: every comparison with it is false, so no sweep
// takes it.  f64 keys are order-preserving 64-bit integers, with explicit
// limits.
#include <climits>
#include <cstdint>

#include "launch.h"
#include "mmf.h"

namespace mmf {
namespace {

// 128 threads x 16 positions: the per-thread costs (summary scans, carries)
// spread over 16 elements; E = 16 keeps a thread's positions inside one
// padding group, so its staged addresses are a base plus constants.
constexpr int kArgThreads = 128, kArgE = 16, kArgTile = kArgThreads * kArgE, kArgWarps = kArgThreads / 32;
constexpr int kArgSpanSmall = kArgTile + 512;

template <typename T> struct AKey;
template <> struct AKey<float> {
    using K = float;
    static constexpr bool kNanPad = true;
    __device__ static K load(float v) { return v; }
    __device__ static float store(K k) { return k; }
};
template <> struct AKey<int16_t> {
    using K = float;
    static constexpr bool kNanPad = true;
    __device__ static K load(int16_t v) { return (float)v; }
    __device__ static int16_t store(K k) { return (int16_t)(int)k; }
};
template <> struct AKey<uint8_t> {
    using K = float;
    static constexpr bool kNanPad = true;
    __device__ static K load(uint8_t v) { return (float)v; }
    __device__ static uint8_t store(K k) { return (uint8_t)(int)k; }
};
template <> struct AKey<double> {
    using K = long long;
    static constexpr bool kNanPad = false;
    __device__ static K load(double v) { return Elem<double>::load(v); }
    __device__ static double store(K k) { return Elem<double>::store(k); }
};

// Identities: -inf/+inf for float keys (which an equal value in the data
// only ties: a tied identity is never preferred to a real position in S, and
// Q is taken only when strictly better than S), the 64-bit limits (outside
// every key of a non-NaN double) for f64.
template <typename K> struct KeyLim;
template <> struct KeyLim<float> {
    __device__ static float lo() { return __int_as_float(0xff800000); }
    __device__ static float hi() { return __int_as_float(0x7f800000); }
    __device__ static float pad() { return __int_as_float(0x7fffffff); }
};
template <> struct KeyLim<long long> {
    __device__ static long long lo() { return LLONG_MIN; }
    __device__ static long long hi() { return LLONG_MAX; }
    __device__ static long long pad() { return 0; }
};

template <typename K, typename P> struct VI {
    K v;
    P i;
};

// Aggregate of a range for both sides (global positions); empty ranges hold
// the identities and position INT64_MAX.
template <typename K> struct Agg {
    K vmax, vmin;
    long long imax, imin;
};

// Shared-memory index with one padding slot per 128 bytes, so E consecutive
// elements per thread spread over the banks.
template <typename K> __device__ __forceinline__ int padk(int p) { return p + p / (128 / (int)sizeof(K)); }
template <typename K> __host__ __device__ constexpr int padded_len(int n) { return n + n / (128 / (int)sizeof(K)); }

// Staged-input slots for a span, padded and kept a multiple of 16 bytes.
template <typename K> __host__ __device__ constexpr int arg_span_slots(int span) {
    return (padded_len<K>(span) + 3) & ~3;
}

template <typename T> struct ArgParams {
    const T *x;
    long long n, w, n_out;
    T *omax, *omin;
    long long *amax, *amin;
    long long ntiles;  // tiles per block (w > kArgTile), 0 for whole blocks per CTA
    int len_small;     // positions per CTA for whole blocks
    const Agg<typename AKey<T>::K> *pg, *sg;  // per-tile prefix / suffix aggregates
    uint32_t *status;  // device status word (range checks of a checked build)
    long long ng;      // aggregates in each of pg and sg
};

template <typename K> __device__ __forceinline__ Agg<K> agg_empty() {
    return Agg<K>{KeyLim<K>::lo(), KeyLim<K>::hi(), LLONG_MAX, LLONG_MAX};
}

template <typename K, typename P> struct ArgScanSmem {
    VI<K, P> qmx[kArgWarps], qmn[kArgWarps], smx[kArgWarps], smn[kArgWarps];
    int qf[kArgWarps], sf[kArgWarps];
};

template <typename K, typename P> __device__ __forceinline__ VI<K, P> shfl_up_vi(VI<K, P> a, int d) {
    return VI<K, P>{__shfl_up_sync(0xffffffffu, a.v, d), __shfl_up_sync(0xffffffffu, a.i, d)};
}
template <typename K, typename P> __device__ __forceinline__ VI<K, P> shfl_down_vi(VI<K, P> a, int d) {
    return VI<K, P>{__shfl_down_sync(0xffffffffu, a.v, d), __shfl_down_sync(0xffffffffu, a.i, d)};
}
// a left of b: b only when strictly better.
template <typename K, typename P> __device__ __forceinline__ VI<K, P> jmax(VI<K, P> a, VI<K, P> b) {
    return b.v > a.v ? b : a;
}
template <typename K, typename P> __device__ __forceinline__ VI<K, P> jmin(VI<K, P> a, VI<K, P> b) {
    return b.v < a.v ? b : a;
}

// status, n_out: range checks of a checked build (outputs hold n_out each).
template <typename T, typename P>
__device__ __forceinline__ void store_side(T *oval, long long *oidx, long long base, int nv,
                                           const typename AKey<T>::K *vs, const P *ps, uint32_t *status,
                                           long long n_out) {
    using A = AKey<T>;
    using K = typename A::K;
    const int tid = threadIdx.x;
    auto ok = [&](const void *p, int nb, const void *b0, int esz) { return in_bytes(status, p, nb, b0, n_out * esz); };
    if (oval) {
        constexpr int VW = 16 / (int)sizeof(T);
        T *o = oval + base;
        const int h = min(nv, (int)(((16 - ((uintptr_t)o & 15)) & 15) / sizeof(T)));
        const int nvec = (nv - h) / VW;
        for (int q = tid; q < nvec; q += kArgThreads) {
            const int j = h + q * VW;
            union {
                uint4 u;
                T e[VW];
            } pk;
#pragma unroll
            for (int e = 0; e < VW; ++e) pk.e[e] = A::store(vs[padk<K>(j + e)]);
            if (ok(o + j, 16, oval, (int)sizeof(T))) *reinterpret_cast<uint4 *>(o + j) = pk.u;
        }
        for (int j = tid; j < h; j += kArgThreads)
            if (ok(o + j, (int)sizeof(T), oval, (int)sizeof(T))) o[j] = A::store(vs[padk<K>(j)]);
        for (int j = h + nvec * VW + tid; j < nv; j += kArgThreads)
            if (ok(o + j, (int)sizeof(T), oval, (int)sizeof(T))) o[j] = A::store(vs[padk<K>(j)]);
    }
    if (oidx) {
        long long *o = oidx + base;
        const int h = min(nv, (int)(((uintptr_t)o >> 3) & 1));
        const int nvec = (nv - h) / 2;
        for (int q = tid; q < nvec; q += kArgThreads) {
            const int j = h + 2 * q;
            longlong2 v;
            v.x = base + (long long)ps[padk<P>(j)];
            v.y = base + (long long)ps[padk<P>(j + 1)];
            if (ok(o + j, 16, oidx, 8)) *reinterpret_cast<longlong2 *>(o + j) = v;
        }
        if (tid == 0 && h && ok(o, 8, oidx, 8)) o[0] = base + (long long)ps[padk<P>(0)];
        const int tail = h + 2 * nvec;
        if (tid == 0 && tail < nv && ok(o + tail, 8, oidx, 8)) o[tail] = base + (long long)ps[padk<P>(tail)];
    }
}

// SPAN: staged input slots, 2 * kArgTile, or kArgSpanSmall for whole blocks
// of w <= kArgSpanSmall - kArgTile (one more CTA per SM).  Compile-time
// offsets keep the staged inputs and the output staging provably apart.
template <typename T, typename P, int SPAN>
__global__ void __launch_bounds__(kArgThreads) argscan_kernel(const ArgParams<T> prm) {
    using A = AKey<T>;
    using K = typename A::K;
    using V = VI<K, P>;
    extern __shared__ __align__(16) unsigned char arg_smem[];
    __shared__ ArgScanSmem<K, P> sm;
    constexpr int PK = padded_len<K>(kArgTile), PP = padded_len<P>(kArgTile);
    K *xs = reinterpret_cast<K *>(arg_smem);  // staged keys: x at p, y at yoff + p
    K *vmx = xs + arg_span_slots<K>(SPAN);
    K *vmn = vmx + PK;
    P *pmx = reinterpret_cast<P *>(vmn + PK);
    P *pmn = pmx + PP;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    long long base, r0, b = 0, t = 0;
    int len, yoff;
    if (prm.ntiles == 0) {
        len = prm.len_small;
        base = (long long)blockIdx.x * len;
        r0 = 0;
        yoff = (int)prm.w;
    } else {
        b = (long long)blockIdx.x / prm.ntiles;
        t = (long long)blockIdx.x % prm.ntiles;
        r0 = t * kArgTile;
        base = b * prm.w + r0;
        len = (int)min((long long)kArgTile, prm.w - r0);
        yoff = kArgTile;
    }
    if (base >= prm.n_out) return;  // uniform per CTA, before any barrier
    const int xlim = (int)max(0LL, min((long long)len, prm.n - base));
    const int ylim = (int)max(0LL, min((long long)len, prm.n - base - prm.w));

    // Stage the inputs (span slots: every x position and y position p <
    // kArgTile; loads issued before the stores).
    {
        K kv[2 * kArgE];
        if (prm.ntiles == 0) {
            const long long lim = min((long long)len + prm.w, prm.n - base);
#pragma unroll
            for (int k = 0; k < 2 * kArgE; ++k) {
                const int i = tid + k * kArgThreads;
                kv[k] = i < lim && in_bytes(prm.status, prm.x + base + i, (int)sizeof(T), prm.x, prm.n * (long long)sizeof(T))
                            ? A::load(__ldg(prm.x + base + i))
                            : KeyLim<K>::pad();
            }
        } else {
#pragma unroll
            for (int k = 0; k < 2 * kArgE; ++k) {
                const int i = tid + k * kArgThreads;
                const int off = k < kArgE ? i : i - kArgTile;
                const int lim = k < kArgE ? xlim : ylim;
                const long long src = k < kArgE ? base : base + prm.w;
                kv[k] = off < lim && in_bytes(prm.status, prm.x + src + off, (int)sizeof(T), prm.x,
                                              prm.n * (long long)sizeof(T))
                            ? A::load(__ldg(prm.x + src + off))
                            : KeyLim<K>::pad();
            }
        }
#pragma unroll
        for (int k = 0; k < 2 * kArgE; ++k)
            if (tid + k * kArgThreads < SPAN) xs[padk<K>(tid + k * kArgThreads)] = kv[k];
    }

    // Segment starts (phase 0) and ends (phase w-1) among the thread's positions.
    const int p0 = tid * kArgE;
    unsigned smask = 0, emask = 0;
    {
        const long long r = prm.ntiles == 0 ? (long long)(p0 % (int)prm.w) : r0 + p0;  // phase of p0
        if (r >= prm.w) {
            // past the last tile of a block: no position of this thread is
            // in the tile, and the tile's last position ends its segment
        } else if (prm.w >= kArgE) {  // at most one start and one end
            const long long ks = r == 0 ? 0 : prm.w - r, ke = prm.w - 1 - r;
            if (ks < kArgE) smask = 1u << ks;
            if (ke < kArgE) emask = 1u << ke;
        } else {
            int q = (int)r;
#pragma unroll
            for (int k = 0; k < kArgE; ++k) {
                if (q == 0) smask |= 1u << k;
                if (q == (int)prm.w - 1) emask |= 1u << k;
                if (++q == (int)prm.w) q = 0;
            }
        }
    }
    const K LO = KeyLim<K>::lo(), HI = KeyLim<K>::hi();
    const V nmx{LO, 0}, nmn{HI, 0};
    const P yrel = (P)prm.w;  // offset of y position 0 from base
    // Without NaN padding (f64), positions outside the array read as the
    // identity of each side.
    // A thread's positions p0..p0+E-1 share one padding group.
    const int sx = padk<K>(p0), sp = padk<P>(p0);
    auto xmx = [&](int k) { return A::kNanPad || p0 + k < xlim ? xs[sx + k] : LO; };
    auto xmn = [&](int k) { return A::kNanPad || p0 + k < xlim ? xs[sx + k] : HI; };
    auto ymx = [&](int p) { return A::kNanPad || p < ylim ? xs[padk<K>(yoff + p)] : LO; };
    auto ymn = [&](int p) { return A::kNanPad || p < ylim ? xs[padk<K>(yoff + p)] : HI; };
    __syncthreads();

    // 1. Forward sweep: local exclusive Q staged; summaries.
    V qmx = nmx, qmn = nmn, smx = nmx, smn = nmn;
    bool done = false;
#pragma unroll
    for (int k = 0; k < kArgE; ++k) {
        const int p = p0 + k;
        if ((smask >> k) & 1u) {
            qmx = nmx;
            qmn = nmn;
        }
        vmx[sx + k] = qmx.v;
        vmn[sx + k] = qmn.v;
        pmx[sp + k] = qmx.i;
        pmn[sp + k] = qmn.i;
        const K ya = ymx(p), yb = ymn(p);
        if (ya > qmx.v) qmx = V{ya, (P)(yrel + p)};
        if (yb < qmn.v) qmn = V{yb, (P)(yrel + p)};
        if (!done) {
            const K xa = xmx(k), xb = xmn(k);
            if (xa > smx.v) smx = V{xa, (P)p};
            if (xb < smn.v) smn = V{xb, (P)p};
            done = (emask >> k) & 1u;
        }
    }
    int qf = smask != 0, sf = emask != 0;

    // 2. Segmented scans of the summaries: inclusive within the warp ...
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const V la = shfl_up_vi(qmx, d), lb = shfl_up_vi(qmn, d);
        const int lf = __shfl_up_sync(0xffffffffu, qf, d);
        if (lane >= d) {
            if (!qf) {
                qmx = jmax(la, qmx);
                qmn = jmin(lb, qmn);
            }
            qf |= lf;
        }
        const V ra = shfl_down_vi(smx, d), rb = shfl_down_vi(smn, d);
        const int rf = __shfl_down_sync(0xffffffffu, sf, d);
        if (lane + d < 32) {
            if (!sf) {
                smx = jmax(smx, ra);
                smn = jmin(smn, rb);
            }
            sf |= rf;
        }
    }
    if (lane == 31) {
        sm.qmx[warp] = qmx;
        sm.qmn[warp] = qmn;
        sm.qf[warp] = qf;
    }
    if (lane == 0) {
        sm.smx[warp] = smx;
        sm.smn[warp] = smn;
        sm.sf[warp] = sf;
    }
    // ... exclusive within the warp ...
    V eqa = shfl_up_vi(qmx, 1), eqb = shfl_up_vi(qmn, 1), esa = shfl_down_vi(smx, 1), esb = shfl_down_vi(smn, 1);
    int eqf = __shfl_up_sync(0xffffffffu, qf, 1), esf = __shfl_down_sync(0xffffffffu, sf, 1);
    if (lane == 0) {
        eqa = nmx;
        eqb = nmn;
        eqf = 0;
    }
    if (lane == 31) {
        esa = nmx;
        esb = nmn;
        esf = 0;
    }
    // ... then across warps, with the tile's carries at the two ends: Q's part
    // left of the tile (block b+1 up to tile t) and S's part right of it (the
    // rest of block b after tile t).
    V cqa = nmx, cqb = nmn, csa = nmx, csb = nmn;
    if (prm.ntiles != 0) {
        if (t > 0) {
            const long long gi = (b + 1) * prm.ntiles + t - 1;
            const Agg<K> a = in_range(prm.status, gi, 0, prm.ng) ? prm.pg[gi] : agg_empty<K>();
            cqa = V{a.vmax, (P)(a.imax - base)};
            cqb = V{a.vmin, (P)(a.imin - base)};
        }
        if (t + 1 < prm.ntiles) {
            const long long gi = b * prm.ntiles + t + 1;
            const Agg<K> a = in_range(prm.status, gi, 0, prm.ng) ? prm.sg[gi] : agg_empty<K>();
            csa = V{a.vmax, (P)(a.imax - base)};
            csb = V{a.vmin, (P)(a.imin - base)};
        }
    }
    __syncthreads();
    for (int u = 0; u < warp; ++u) {
        if (sm.qf[u]) {
            cqa = sm.qmx[u];
            cqb = sm.qmn[u];
        } else {
            cqa = jmax(cqa, sm.qmx[u]);
            cqb = jmin(cqb, sm.qmn[u]);
        }
    }
    if (eqf) {
        cqa = eqa;
        cqb = eqb;
    } else {
        cqa = jmax(cqa, eqa);
        cqb = jmin(cqb, eqb);
    }
    for (int u = kArgWarps - 1; u > warp; --u) {
        if (sm.sf[u]) {
            csa = sm.smx[u];
            csb = sm.smn[u];
        } else {
            csa = jmax(sm.smx[u], csa);
            csb = jmin(sm.smn[u], csb);
        }
    }
    if (esf) {
        csa = esa;
        csb = esb;
    } else {
        csa = jmax(esa, csa);
        csb = jmin(esb, csb);
    }

    // 3. Backward sweep: S with its carry, Q completed with its carry before
    // the thread's first segment start, the join, staged in place.
    const int fs = smask ? __ffs(smask) - 1 : kArgE;
    V sa = csa, sb = csb;
#pragma unroll
    for (int k = kArgE - 1; k >= 0; --k) {
        const int p = p0 + k;
        if ((emask >> k) & 1u) {
            sa = nmx;
            sb = nmn;
        }
        const K xa = xmx(k), xb = xmn(k);
        if (xa >= sa.v) sa = V{xa, (P)p};
        if (xb <= sb.v) sb = V{xb, (P)p};
        V qa{vmx[sx + k], pmx[sp + k]}, qb{vmn[sx + k], pmn[sp + k]};
        if (k < fs) {
            qa = jmax(cqa, qa);
            qb = jmin(cqb, qb);
        }
        const V ra = qa.v > sa.v ? qa : sa, rb = qb.v < sb.v ? qb : sb;
        vmx[sx + k] = ra.v;
        pmx[sp + k] = ra.i;
        vmn[sx + k] = rb.v;
        pmn[sp + k] = rb.i;
    }
    __syncthreads();
    const int nv = (int)min((long long)len, prm.n_out - base);
    store_side<T, P>(prm.omax, prm.amax, base, nv, vmx, pmx, prm.status, prm.n_out);
    store_side<T, P>(prm.omin, prm.amin, base, nv, vmn, pmn, prm.status, prm.n_out);
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
template <typename K> __device__ __forceinline__ Agg<K> agg_bcast(const Agg<K> &a, int lane) {
    Agg<K> r;
    r.vmax = __shfl_sync(0xffffffffu, a.vmax, lane);
    r.vmin = __shfl_sync(0xffffffffu, a.vmin, lane);
    r.imax = __shfl_sync(0xffffffffu, a.imax, lane);
    r.imin = __shfl_sync(0xffffffffu, a.imin, lane);
    return r;
}


// g[b*ntiles + t] = aggregate of x over tile t of block b (clipped to the
// block and to the array), for blocks 0..nb-1: one warp per tile (64
// coalesced loads per lane, 16 in flight), no barriers; warps stride over the
// tiles.
template <typename T>
__global__ void __launch_bounds__(256) argagg_kernel(const T *x, long long n, long long w, long long ntiles,
                                                    long long nb, Agg<typename AKey<T>::K> *g, uint32_t *status) {
    using A = AKey<T>;
    using K = typename A::K;
    constexpr int PER_LANE = kArgTile / 32, BATCH = 16;
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = wid; u < nb * ntiles; u += nwarps) {
        const long long b = u / ntiles, t = u % ntiles;
        const long long lo = b * w + t * kArgTile;
        const int lim = (int)max(0LL, min(min((long long)kArgTile, (b + 1) * w - lo), n - lo));
        const T *xt = x + lo;
        // Per lane: extremes and their offsets in the tile (-1: none yet).
        K vmax = KeyLim<K>::lo(), vmin = KeyLim<K>::hi();
        int omax = -1, omin = -1;
        for (int k0 = 0; k0 < PER_LANE; k0 += BATCH) {
            T v[BATCH];
#pragma unroll
            for (int k = 0; k < BATCH; ++k) {
                const int off = lane + (k0 + k) * 32;
                v[k] = off < lim && in_bytes(status, xt + off, (int)sizeof(T), x, n * (long long)sizeof(T))
                           ? __ldg(xt + off)
                           : T(0);
            }
#pragma unroll
            for (int k = 0; k < BATCH; ++k) {
                const int off = lane + (k0 + k) * 32;
                if (off < lim) {  // a lane's offsets increase: strict keeps the earliest
                    const K key = A::load(v[k]);
                    if (key > vmax || omax < 0) {
                        vmax = key;
                        omax = off;
                    }
                    if (key < vmin || omin < 0) {
                        vmin = key;
                        omin = off;
                    }
                }
            }
        }
        Agg<K> a{vmax, vmin, omax < 0 ? LLONG_MAX : lo + omax, omin < 0 ? LLONG_MAX : lo + omin};
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) agg_join(a, agg_shfl_down(a, d));
        if (lane == 0 && in_range(status, u, 0, nb * ntiles)) g[u] = a;
    }
}

// Per block: pg[t] = tiles 0..t joined, sg[t] = tiles t..ntiles-1 joined;
// one warp per block, 32 tiles at a time.
template <typename K>
__global__ void __launch_bounds__(kArgThreads) argblock_scan_kernel(const Agg<K> *g, long long ntiles, long long nb,
                                                                   Agg<K> *pg, Agg<K> *sg, uint32_t *status) {
    const int lane = threadIdx.x & 31;
    const long long b = (long long)blockIdx.x * kArgWarps + (threadIdx.x >> 5);
    if (b >= nb) return;  // the kernel has no barriers
    const Agg<K> *gb = g + b * ntiles;
    Agg<K> carry = agg_empty<K>();
    for (long long t0 = 0; t0 < ntiles; t0 += 32) {
        const long long t = t0 + lane;
        Agg<K> a = t < ntiles && in_range(status, b * ntiles + t, 0, nb * ntiles) ? gb[t] : agg_empty<K>();
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
        if (t < ntiles && in_range(status, b * ntiles + t, 0, nb * ntiles)) pg[b * ntiles + t] = m;
        carry = agg_bcast(m, 31);
    }
    carry = agg_empty<K>();
    for (long long t1 = ntiles; t1 > 0; t1 -= 32) {
        const long long t = t1 - 32 + lane;  // lanes below 0 hold nothing
        Agg<K> a = t >= 0 && in_range(status, b * ntiles + t, 0, nb * ntiles) ? gb[t] : agg_empty<K>();
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const Agg<K> r = agg_shfl_down(a, d);
            if (lane + d < 32) agg_join(a, r);
        }
        agg_join(a, carry);
        if (t >= 0 && in_range(status, b * ntiles + t, 0, nb * ntiles)) sg[b * ntiles + t] = a;
        carry = agg_bcast(a, 0);
    }
}

template <typename T, typename P, int SPAN> constexpr size_t arg_smem_bytes() {
    using K = typename AKey<T>::K;
    return (size_t)arg_span_slots<K>(SPAN) * sizeof(K) + 2 * (size_t)padded_len<K>(kArgTile) * sizeof(K) +
           2 * (size_t)padded_len<P>(kArgTile) * sizeof(P);
}

template <typename T, typename P, int SPAN>
cudaError_t arg_launch(const LaunchCtx &ctx, const ArgParams<T> &prm, int64_t grid) {
    constexpr size_t smem = arg_smem_bytes<T, P, SPAN>();
    static int attr_set[64] = {};
    if (smem > 48 * 1024 && !attr_set[ctx.device & 63]) {
        cudaError_t e =
            cudaFuncSetAttribute(argscan_kernel<T, P, SPAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set[ctx.device & 63] = 1;
    }
    argscan_kernel<T, P, SPAN><<<(unsigned)grid, kArgThreads, smem, ctx.stream>>>(prm);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t argscan_1d(const LaunchCtx &ctx, const void *in, int64_t n, int64_t w, void *omax, void *omin,
                       int64_t *amax, int64_t *amin) {
    using K = typename AKey<T>::K;
    const int64_t n_out = n - w + 1;
    if (n_out <= 0) return cudaSuccess;
    ArgParams<T> prm{static_cast<const T *>(in), n, w, n_out, static_cast<T *>(omax), static_cast<T *>(omin),
                     reinterpret_cast<long long *>(amax), reinterpret_cast<long long *>(amin), 0, 0, nullptr,
                     nullptr, ctx.status, 0};
    // Offsets from a tile's base stay below w + kArgTile: 32-bit up to 2^30.
    const bool wide = w >= (int64_t(1) << 30);
    if (w <= kArgTile) {
        prm.len_small = (int)((kArgTile / w) * w);
        const int64_t grid = (n_out + prm.len_small - 1) / prm.len_small;
        // Windows up to 512 stage kArgTile + w <= kArgSpanSmall inputs: one
        // more CTA per SM (f32: 5 instead of 4).
        return w <= kArgSpanSmall - kArgTile ? arg_launch<T, unsigned, kArgSpanSmall>(ctx, prm, grid)
                                             : arg_launch<T, unsigned, 2 * kArgTile>(ctx, prm, grid);
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
    const int64_t agg_warps = (int64_t)ng < sms * 64 ? (int64_t)ng : sms * 64;  // 8 CTAs of 8 warps per SM
    argagg_kernel<T><<<(unsigned)((agg_warps + 7) / 8), 256, 0, ctx.stream>>>(static_cast<const T *>(in), n, w,
                                                                             ntiles, nb, g, ctx.status);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        argblock_scan_kernel<K><<<(unsigned)((nb + kArgWarps - 1) / kArgWarps), kArgThreads, 0, ctx.stream>>>(
            g, ntiles, nb, pg, sg, ctx.status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        prm.ntiles = ntiles;
        prm.pg = pg;
        prm.sg = sg;
        prm.ng = (long long)ng;
        e = wide ? arg_launch<T, unsigned long long, 2 * kArgTile>(ctx, prm, nbo * ntiles)
                 : arg_launch<T, unsigned, 2 * kArgTile>(ctx, prm, nbo * ntiles);
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
