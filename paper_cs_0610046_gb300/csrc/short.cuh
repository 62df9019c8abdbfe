// Short series (batched plans): one warp per series of at most 32·E elements,
// no CTA barriers.  The block-scan kernel spends a whole tile and two CTA
// barriers on every item; a series of a thousand elements would fill half a
// tile, so short series take this kernel instead.
//
// Per series, lane l holds elements [l·E, l·E + E) in registers.  Blocks are
// exactly w elements long, from position 0: the decomposition of Section 2's
// van Herk/Gil-Werman algorithm (Table 1), so every full window is the suffix
// of one block and the prefix of the next, one operation per output.  The
// block scans restart at block boundaries inside a lane and are carried
// across lanes by a segmented shuffle scan.  Both scans go to a warp-private
// shared array stored element-major (row = position mod E, column = lane), so
// a warp reading one position per lane touches 32 consecutive words.  Max and
// min are done one after the other in the same arrays.
//
// Windows longer than a lane's E elements (w - 1 >= E) take a second
// decomposition, short_lanes: the blocks are the lanes themselves (Section
// 2's decomposition with blocks shorter than the window, as in the block
// scan's long windows), so the prefix and suffix scans run inside a lane
// without restarts or carries, max and min in one pass over the loaded
// values, and the whole lanes a window spans come from per-lane aggregates
// combined by shuffles.
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
    static constexpr size_t warp_bytes = 3 * (size_t)E * ROW * sizeof(R);  // three [E][ROW] arrays
    static constexpr size_t smem_bytes = WARPS * warp_bytes;
    static constexpr size_t smem_bytes_lb = smem_bytes + (size_t)NMAX * sizeof(T);  // + the query
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
    int32_t lb_n;          // query length (every series has it)
    uint32_t *status;
};

extern __shared__ __align__(16) uint8_t short_smem[];

// This lane's E elements of a series starting at src (elements past n are
// read if they lie inside the buffer and ignored later).
template <typename T>
__device__ __forceinline__ void short_load(const T *src, int n, int lane, const T *buf, int64_t buf_n,
                                           typename Elem<T>::R (&x)[ShortGeo<T>::E], uint32_t *status) {
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
        for (int e = 0; e < E; ++e)
            x[e] = lane * E + e < n && in_range(status, (p + e) - buf, 0, buf_n) ? Elem<T>::load(__ldg(p + e))
                                                                              : Elem<T>::lo();
    }
}

template <bool MAX, typename R> __device__ __forceinline__ R sop(R a, R b) { return MAX ? vmax(a, b) : vmin(a, b); }

// One side (max or min) of one series with blocks of exactly w elements
// from position 0 (van Herk/Gil-Werman's own decomposition): a full window
// [lo, lo+w-1] then spans exactly two blocks (or is one block), so its
// extreme is op(suffix_w[lo], prefix_w[lo+w-1]).  A window clipped at the
// start lies in block 0, which starts at position 0: prefix_w[hi].  A window
// clipped at the end whose start shares a block with the last element:
// suffix_w[lo] (identities follow the series).  Positions past the series'
// end in v are set to the side's identity first.  q0: position lane·E modulo
// w (the lane's offset in its block); u1: position lane·E + E - 1 modulo w.
// The scans hold positions lane·E + e (contiguous per lane); the outputs are
// formed for positions 32k + lane (row k of the series), so every shared read
// is a per-lane base plus a constant and a warp stores whole rows.  res[k]:
// the output at position 32k + lane.
template <typename T, bool MAX>
__device__ __forceinline__ void short_side(typename Elem<T>::R (&v)[ShortGeo<T>::E], int n, int w, int d,
                                           int n_out, int q0, int u1, int lane, typename Elem<T>::R *PA,
                                           typename Elem<T>::R *SA, typename Elem<T>::R (&res)[ShortGeo<T>::E]) {
    using G = ShortGeo<T>;
    using R = typename Elem<T>::R;
    constexpr int E = G::E;
    constexpr int CS = 32 / E;  // columns per row of 32 positions
    const R id = MAX ? Elem<T>::lo() : Elem<T>::hi();
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (lane * E + e >= n) v[e] = id;
    const int fs = q0 == 0 ? 0 : w - q0;  // this lane's first block start (>= E: none)
    const int le = E - 2 - (u1 + 1 == w ? -1 : u1);  // its last block end (< 0: none)
    {
        // Prefix, restarting at every block start.
        R pre[E];
        pre[0] = v[0];
        if (w >= E) {  // at most one start in the lane
#pragma unroll
            for (int e = 1; e < E; ++e) pre[e] = e == fs ? v[e] : sop<MAX>(pre[e - 1], v[e]);
        } else {
            int t = q0;
#pragma unroll
            for (int e = 1; e < E; ++e) {
                t = t + 1 == w ? 0 : t + 1;
                pre[e] = t == 0 ? v[e] : sop<MAX>(pre[e - 1], v[e]);
            }
        }
        // Elements before the lane's first block start continue the block of
        // earlier lanes: segmented scan of (lane total since its last start,
        // lane holds a start) over the lanes.
        R tt = pre[E - 1];
        bool f = fs < E;
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const R a = __shfl_up_sync(0xffffffffu, tt, k);
            const bool fa = __shfl_up_sync(0xffffffffu, (int)f, k) != 0;
            if (lane >= k) {
                if (!f) tt = sop<MAX>(a, tt);
                f = f || fa;
            }
        }
        const R carry = __shfl_up_sync(0xffffffffu, tt, 1);
        if (lane > 0) {
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (e < fs) pre[e] = sop<MAX>(pre[e], carry);
        }
#pragma unroll
        for (int e = 0; e < E; ++e) PA[e * G::ROW + lane] = pre[e];
    }
    {
        // Suffix, restarting at every block end.
        R suf[E];
        suf[E - 1] = v[E - 1];
        if (w >= E) {  // at most one end in the lane
#pragma unroll
            for (int e = E - 2; e >= 0; --e) suf[e] = e == le ? v[e] : sop<MAX>(suf[e + 1], v[e]);
        } else {
            int t = u1;
#pragma unroll
            for (int e = E - 2; e >= 0; --e) {
                t = t == 0 ? w - 1 : t - 1;
                suf[e] = t == w - 1 ? v[e] : sop<MAX>(suf[e + 1], v[e]);
            }
        }
        R tt = suf[0];
        bool f = le >= 0;
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const R a = __shfl_down_sync(0xffffffffu, tt, k);
            const bool fa = __shfl_down_sync(0xffffffffu, (int)f, k) != 0;
            if (lane + k < 32) {
                if (!f) tt = sop<MAX>(tt, a);
                f = f || fa;
            }
        }
        const R carry = __shfl_down_sync(0xffffffffu, tt, 1);
        if (lane < 31) {
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (e > le) suf[e] = sop<MAX>(suf[e], carry);
        }
#pragma unroll
        for (int e = 0; e < E; ++e) SA[e * G::ROW + lane] = suf[e];
    }
    __syncwarp();
    // Position p lives at row p mod E, column p / E; for p = 32k + c the row
    // is c mod E and the column CS·k + c / E, so lo = 32k + (lane + d) and
    // hi = lo + w - 1 read at a per-lane base plus CS·k.
    const int a = lane + d, b = a + w - 1;
    const R *sb = SA + (a & (E - 1)) * G::ROW + (a >> G::LGE);
    const R *pb = PA + (b & (E - 1)) * G::ROW + (b >> G::LGE);
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int r0 = 32 * k;  // first position of row k
        if (r0 + d >= 0 && r0 + 31 + d + w - 1 <= n - 1 && r0 + 31 < n_out) {
            res[k] = sop<MAX>(sb[CS * k], pb[CS * k]);  // no window of the row is clipped
        } else {
            const int o = r0 + lane;
            R r = id;
            if (o < n_out) {
                const int lo = o + d;
                int hi = lo + w - 1;
                if (hi > n - 1) hi = n - 1;
                const R P = PA[(hi & (E - 1)) * G::ROW + (hi >> G::LGE)];
                if (lo <= 0) {
                    r = P;  // clipped at the start: block 0 from position 0
                } else {
                    const R S = SA[(lo & (E - 1)) * G::ROW + (lo >> G::LGE)];
                    r = lo / w == hi / w ? S : sop<MAX>(S, P);
                }
            }
            res[k] = r;
        }
    }
    __syncwarp();
}

template <typename R> __device__ __forceinline__ R shfl_down_or(R v, int lane, int dl, R id) {
    const R t = __shfl_down_sync(0xffffffffu, v, dl);
    return lane + dl < 32 ? t : id;
}

// m1 = op over the aggregates of lanes lane+1 .. lane+q-1, m2 = the same
// through lane+q (lanes past 31 hold identities).  D[k] holds op over lanes
// lane .. lane+2^k-1; a run of L lanes (1 <= L <= 31) is two overlapping runs
// of the largest power of two p <= L, one starting at its first lane and one
// ending at its last; runs of 32 or more lanes reach past lane 31 and are the
// suffix D[5].  q is the same on every lane.
template <bool MAX, typename R>
__device__ __forceinline__ void lane_windows(R a, int lane, int q, R id, R &m1, R &m2) {
    R D[6];
    D[0] = a;
#pragma unroll
    for (int k = 0; k < 5; ++k) D[k + 1] = sop<MAX>(D[k], shfl_down_or(D[k], lane, 1 << k, id));
    auto run = [&](int L) -> R {
        if (L <= 0) return id;
        if (L >= 32) return shfl_down_or(D[5], lane, 1, id);
        const int k = 31 - __clz(L), p = 1 << k;
        R Dk = D[0];
#pragma unroll
        for (int kk = 1; kk < 5; ++kk)
            if (k == kk) Dk = D[kk];
        return sop<MAX>(shfl_down_or(Dk, lane, 1, id), shfl_down_or(Dk, lane, 1 + L - p, id));
    };
    m1 = run(q - 1);
    m2 = run(q);
}

// Inclusive scan of the lane aggregates: op over lanes 0 .. lane.
template <bool MAX, typename R> __device__ __forceinline__ R lane_scan(R a, int lane) {
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        const R t = __shfl_up_sync(0xffffffffu, a, k);
        if (lane >= k) a = sop<MAX>(t, a);
    }
    return a;
}

// Adds the squared excursion of the query outside the envelope at one
// position: above the upper envelope or below the lower one (never both:
// U >= L).
template <typename T>
__device__ __forceinline__ typename LbAcc<T>::A lb_term(T qv, typename Elem<T>::R u, typename Elem<T>::R l,
                                                        typename LbAcc<T>::A part) {
    using A = typename LbAcc<T>::A;
    const A qi = (A)qv, U = (A)Elem<T>::store(u), L = (A)Elem<T>::store(l);
    const A dd = qi > U ? qi - U : (qi < L ? L - qi : A(0));
    return part + dd * dd;
}

// Staging of a warp's next series in shared memory (4- and 8-byte types:
// 128 bytes per lane), issued while the current series still forms its
// outputs: lane l's 16-byte chunk c goes to slot c ^ (l mod 8) of its 128
// bytes, so that the eight lanes of each 16-byte read phase hit eight
// different bank groups.  Bytes past the series' end are zero (its last
// element replaces them after the read).  The copy covers PN's identity
// column, which the reader writes again.
template <typename T> constexpr bool short_stages() { return sizeof(T) >= 4; }

template <typename T>
__device__ __forceinline__ void short_stage(const T *nsrc, int nn, int lane, void *stage) {
    constexpr int CH = ShortGeo<T>::E * (int)sizeof(T) / 16;  // 8 chunks per lane
    static_assert(CH == 8, "128 bytes per lane");
    const char *g = reinterpret_cast<const char *>(nsrc);
    const int total = nn * (int)sizeof(T);
    char *sb = reinterpret_cast<char *>(stage) + lane * CH * 16;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const int off = (lane * CH + c) * 16;
        const int bytes = total - off < 0 ? 0 : (total - off > 16 ? 16 : total - off);
        cp_async16(sb + ((c ^ (lane & (CH - 1))) * 16), bytes ? g + off : g, bytes);
    }
    cp_async_commit();
}

template <typename T>
__device__ __forceinline__ void short_read_staged(const void *stage, int lane,
                                                  typename Elem<T>::R (&x)[ShortGeo<T>::E]) {
    constexpr int E = ShortGeo<T>::E, CH = 8, NWD = E * (int)sizeof(T) / 4;
    cp_async_wait_all();
    const uint4 *sb = reinterpret_cast<const uint4 *>(reinterpret_cast<const char *>(stage) + lane * CH * 16);
    uint32_t wd[NWD];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const uint4 v = sb[c ^ (lane & (CH - 1))];
        wd[4 * c] = v.x;
        wd[4 * c + 1] = v.y;
        wd[4 * c + 2] = v.z;
        wd[4 * c + 3] = v.w;
    }
    ExtractLoop<T, 0, 0, E>::run(wd, x);
    __syncwarp();  // every lane's chunks read before the arrays are written again
}

// One series whose windows are longer than a lane (w - 1 >= E), both sides;
// returns this lane's part of the envelope lower bound (LB) or zero.
// Lane j holds positions [jE, jE + E), the last element repeated past the
// series' end (E-element blocks from position 0; every window reaching past
// the end holds that element already, so neither side changes).  P: prefix
// inside the lane's block, to shared memory (PM, PN: element-major
// [e][lane], column 32 an identity column); S: suffix inside the block (max
// in registers, min in SN).  With s = w - 1 = q*E + rr, the window starting
// at position lo = jE + e ends at hi = lo + s in lane j + q (e < E - rr) or
// j + q + 1, so its extreme is op(S[lo], aggregates of the lanes in between,
// P[hi]); hi past the last lane reads the identity column (the aggregates
// in between then run to lane 31).  Lane j forms the outputs o = lo - d of
// its own positions; outputs whose windows start before position 0 (centred
// windows, d < 0) are op(lanes before hi's lane, P[hi]).  The outputs go
// back through shared memory (max to PM, min in place in SN) so that each
// store instruction writes 32 consecutive outputs.
// staged: the series is already in PN (short_stage by the previous call);
// nsrc (if not null): the warp's next series, nn elements, to stage in PN once
// this one no longer reads it.
// Not inlined: the kernel's other decomposition then keeps its own register
// allocation (inlined together they spill).
template <typename T, bool LB>
__device__ __noinline__ typename LbAcc<T>::A short_lanes(const T *src, const T *buf, int64_t buf_n, uint32_t *status,
                                                         int n, int w, int d, int n_out, int lane,
                                                         typename Elem<T>::R *PM, typename Elem<T>::R *PN,
                                                         typename Elem<T>::R *SN, T *omax, T *omin, const T *qs,
                                                         bool staged, const T *nsrc, int nn) {
    using G = ShortGeo<T>;
    using R = typename Elem<T>::R;
    using A = typename LbAcc<T>::A;
    constexpr int E = G::E, ROW = G::ROW;
    const R lo_id = Elem<T>::lo(), hi_id = Elem<T>::hi();
    A part = A(0);
    R x[E];
    if constexpr (short_stages<T>()) {
        if (staged) {
            short_read_staged<T>(PN, lane, x);
            // The staged copy covered PN's identity column (element e·ROW + 32
            // lies in another lane's slot): write it again.
            if (lane < E) PN[lane * ROW + 32] = hi_id;
        } else {
            short_load<T>(src, n, lane, buf, buf_n, x, status);
        }
    } else {
        short_load<T>(src, n, lane, buf, buf_n, x, status);
    }
    const int base = lane * E;
    if (base + E > n) {
        const R last = Elem<T>::load(__ldg(src + n - 1));
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (base + e >= n) x[e] = last;
    }
    // The max side's suffix stays in registers, the min side's goes to SN
    // (both in registers would not fit beside the loaded values).
    R sm[E];
    R am, an;  // lane aggregates
    {
        R pm = x[0], pn = x[0];
        PM[lane] = pm;
        PN[lane] = pn;
#pragma unroll
        for (int e = 1; e < E; ++e) {
            pm = vmax(pm, x[e]);
            pn = vmin(pn, x[e]);
            PM[e * ROW + lane] = pm;
            PN[e * ROW + lane] = pn;
        }
        am = pm;
        an = pn;
        R sn = x[E - 1];
        sm[E - 1] = sn;
        SN[(E - 1) * ROW + lane] = sn;
#pragma unroll
        for (int e = E - 2; e >= 0; --e) {
            sm[e] = vmax(sm[e + 1], x[e]);
            sn = vmin(sn, x[e]);
            SN[e * ROW + lane] = sn;
        }
    }
    const int s = w - 1, q = s >> G::LGE, rr = s & (E - 1);
    R m1m, m2m, m1n, m2n;
    lane_windows<true>(am, lane, q, lo_id, m1m, m2m);
    lane_windows<false>(an, lane, q, hi_id, m1n, m2n);
    __syncwarp();
    // Outputs of this lane's positions.  Element e reads row (e + rr) mod E
    // of lane j + q + (e >= E - rr); the choice is the same on every lane.
    const int c0 = lane + q < 32 ? lane + q : 32, c1 = lane + q + 1 < 32 ? lane + q + 1 : 32;
    const int i0 = rr * ROW + c0, i1 = (rr - E) * ROW + c1;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const bool far = e >= E - rr;
        const int i = (far ? i1 : i0) + e * ROW;
        sm[e] = vmax(vmax(sm[e], far ? m2m : m1m), PM[i]);
        // SN[e][lane] is this lane's own: the min outputs replace it in place.
        SN[e * ROW + lane] = vmin(vmin(SN[e * ROW + lane], far ? m2n : m1n), PN[i]);
    }
    // Outputs whose windows start before position 0 (d < 0): the window is
    // [0, hi], the lanes before hi's lane K and P[hi] (K = 32 past the end:
    // all lanes and the identity column).
    if (d < 0) {
        const R xm = lane_scan<true>(am, lane), xn = lane_scan<false>(an, lane);
        const int cnt = -d < n_out ? -d : n_out;
        for (int o0 = 0; o0 < cnt; o0 += 32) {
            const int o = o0 + lane, hi = o + d + s;
            const int K = (hi >> G::LGE) < 32 ? hi >> G::LGE : 32;
            const int src_lane = K > 0 ? K - 1 : 0;
            const R tm = __shfl_sync(0xffffffffu, xm, src_lane), tn = __shfl_sync(0xffffffffu, xn, src_lane);
            if (o < cnt) {
                const int i = (hi & (E - 1)) * ROW + K;
                const R rm = vmax(K > 0 ? tm : lo_id, PM[i]), rn = vmin(K > 0 ? tn : hi_id, PN[i]);
                if constexpr (LB) {
                    part = lb_term<T>(qs[o], rm, rn, part);
                } else {
                    if (omax) __stcs(omax + o, Elem<T>::store(rm));
                    if (omin) __stcs(omin + o, Elem<T>::store(rn));
                }
            }
        }
    }
    __syncwarp();  // every read of PM and PN done
    if constexpr (short_stages<T>()) {
        if (nsrc) short_stage<T>(nsrc, nn, lane, PN);  // lands while the outputs leave
    }
#pragma unroll
    for (int e = 0; e < E; ++e) PM[e * ROW + lane] = sm[e];
    __syncwarp();
    // Row k: outputs 32k + lane (max in PM, min in SN), formed by the lane
    // holding their window start lo = o + d: element lo mod E of lane lo / E,
    // index ir + k·32/E (o + 32 keeps lo mod E and moves 32/E lanes on).
    // Outputs before -d came from the clipped windows above.
    constexpr int CS = 32 / E;
    const int t0 = lane + d;
    const int ir = (t0 & (E - 1)) * ROW + (t0 >> G::LGE);
    const int o_lo = d < 0 ? -d : 0;
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int o = 32 * k + lane;
        if (o >= o_lo && o < n_out) {
            const int i = ir + CS * k;
            if constexpr (LB) {
                part = lb_term<T>(qs[o], PM[i], SN[i], part);
            } else {
                if (omax) __stcs(omax + o, Elem<T>::store(PM[i]));
                if (omin) __stcs(omin + o, Elem<T>::store(SN[i]));
            }
        }
    }
    __syncwarp();  // the next series writes PM/PN/SN again
    return part;
}

// Outputs of positions 32k + lane (row k) of one side to dst: every row is
// one coalesced 32-element store.
template <typename T>
__device__ __forceinline__ void short_store_rows(T *dst, int lane, int n_out,
                                                 const typename Elem<T>::R (&r)[ShortGeo<T>::E]) {
#pragma unroll
    for (int k = 0; k < ShortGeo<T>::E; ++k)
        if (32 * k + lane < n_out) __stcs(dst + 32 * k + lane, Elem<T>::store(r[k]));
}

// One side of the envelope lower bound for this lane's positions: the
// squared excursions of the query above the upper envelope (MAX) or below
// the lower one.  The two never both occur at a position (U >= L), so the
// sides add up to the bound's terms.
// query: the CTA's shared copy.
template <typename T, bool MAX>
__device__ __forceinline__ typename LbAcc<T>::A short_lb_side(const T *query, int lane, int n_out,
                                                              const typename Elem<T>::R (&r)[ShortGeo<T>::E]) {
    using A = typename LbAcc<T>::A;
    A part = A(0);
#pragma unroll
    for (int k = 0; k < ShortGeo<T>::E; ++k) {
        const int o = 32 * k + lane;
        if (o < n_out) {
            const A qi = (A)query[o];
            const A v = (A)Elem<T>::store(r[k]);
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
    T *qs = reinterpret_cast<T *>(short_smem + G::smem_bytes);  // LB: the query, once per CTA
    if constexpr (LB) {
        const T *q = reinterpret_cast<const T *>(P.lb_query);
        for (int i = threadIdx.x; i < P.lb_n && i < G::NMAX; i += blockDim.x) qs[i] = __ldg(q + i);
        __syncthreads();
    }
    // Column 32 of PA and SA: identities, read by windows reaching past the
    // last lane (nothing else writes it).
    for (int e = lane; e < E; e += 32) {
        PA[e * G::ROW + 32] = Elem<T>::lo();
        SA[e * G::ROW + 32] = Elem<T>::hi();
    }
    __syncwarp();
    bool staged = false;  // this warp's series k is already in shared memory
    for (int64_t k = (int64_t)blockIdx.x * G::WARPS + wib; k < P.count; k += nwarps) {
        const bool cur_staged = staged;
        staged = false;
        const int64_t sid = P.ids[k];
        const SeriesDesc sd = P.series[sid];
        const int n = (int)sd.n, d = (int)sd.d, n_out = (int)sd.n_out;
        const int64_t w = sd.w;
        if (n > G::NMAX || n_out <= 0) {
            if (n > G::NMAX && lane == 0) report_error(P.status, kErrBadItem);
            continue;
        }
        // The warp's next series: towards L2 now, and into shared memory
        // (4- and 8-byte types, 16-byte aligned starts, windows longer than a
        // lane) once this one, if it takes short_lanes too, no longer needs
        // the staging array.
        const T *nsrc = nullptr;
        int nn = 0;
        if (k + nwarps < P.count) {
            const SeriesDesc nx = P.series[P.ids[k + nwarps]];
            if (lane * E < nx.n) prefetch_l2(buf + nx.in_off + lane * E);
            const int64_t nwi = nx.w < 2 * G::NMAX ? nx.w : 2 * G::NMAX;
            if (short_stages<T>() && nx.n <= G::NMAX && nx.n_out > 0 && nwi > E &&
                (((uintptr_t)(buf + nx.in_off)) & 15) == 0) {
                nsrc = buf + nx.in_off;
                nn = (int)nx.n;
            }
        }
        // Windows longer than twice the longest series act like 2·NMAX
        // (every one of them is clipped to the series): 32-bit positions.
        const int wi = (int)(w < 2 * G::NMAX ? w : 2 * G::NMAX);
        using A = typename LbAcc<T>::A;
        A part = A(0);
        if (wi > E) {
            T *om = P.out_max ? reinterpret_cast<T *>(P.out_max) + sd.out_off : nullptr;
            T *on = P.out_min ? reinterpret_cast<T *>(P.out_min) + sd.out_off : nullptr;
            part = short_lanes<T, LB>(buf + sd.in_off, buf, P.in_elems, P.status, n, wi, d, n_out, lane, PA, SA,
                                      SA + E * G::ROW, om, on, qs, cur_staged, nsrc, nn);
            staged = nsrc != nullptr;
        } else {
            // Blocks of w elements, one side after the other; each side loads
            // the series again (L2-resident): the values of one side need not
            // stay in registers through the other.
            const int q0 = (lane * E) % wi, u1 = (lane * E + E - 1) % wi;
            {
                R x[E], r[E];
                short_load<T>(buf + sd.in_off, n, lane, buf, P.in_elems, x, P.status);
                short_side<T, true>(x, n, wi, d, n_out, q0, u1, lane, PA, SA, r);
                if constexpr (LB)
                    part += short_lb_side<T, true>(qs, lane, n_out, r);
                else if (P.out_max)
                    short_store_rows<T>(reinterpret_cast<T *>(P.out_max) + sd.out_off, lane, n_out, r);
            }
            __syncwarp();  // keeps the next side's loads after this side's stores (register pressure)
            {
                R x[E], r[E];
                short_load<T>(buf + sd.in_off, n, lane, buf, P.in_elems, x, P.status);
                short_side<T, false>(x, n, wi, d, n_out, q0, u1, lane, PA, SA, r);
                if constexpr (LB)
                    part += short_lb_side<T, false>(qs, lane, n_out, r);
                else if (P.out_min)
                    short_store_rows<T>(reinterpret_cast<T *>(P.out_min) + sd.out_off, lane, n_out, r);
            }
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
                                                  (int)G::smem_bytes_lb)
                           : cudaFuncSetAttribute(short_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)G::smem_bytes);
        if (e != cudaSuccess) return e;
        e = lb ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, short_kernel<T, true>, G::WARPS * 32, G::smem_bytes_lb)
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
                        double *lb_acc, int64_t lb_n) {
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
    P.lb_n = (int32_t)(lb_n < G::NMAX ? lb_n : G::NMAX);
    P.status = ctx.status;
    const int64_t need = (count + G::WARPS - 1) / G::WARPS;
    const int64_t wave = (int64_t)(ctx.sms > 0 ? ctx.sms : 1) * k;
    const unsigned grid = (unsigned)(need < wave ? need : wave);
    if (lb)
        short_kernel<T, true><<<grid, G::WARPS * 32, G::smem_bytes_lb, ctx.stream>>>(P);
    else
        short_kernel<T, false><<<grid, G::WARPS * 32, G::smem_bytes, ctx.stream>>>(P);
    return cudaGetLastError();
}

}  // namespace mmf
