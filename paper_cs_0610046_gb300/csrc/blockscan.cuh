// Block prefix/suffix-scan running max-min filter (van Herk / Gil-Werman,
// Section 2 and Table 1 row 2 of Lemire's paper), re-designed as a
// persistent, TMA-fed streaming kernel for sm_103a.
//
// Decomposition.  Let s = w-1 and let blocks of B elements tile the input.
// If B <= s, a window [j, j+s] starts in block b(j) and ends in a later block
// b(k), k = j+s, so
//     max[j] = max( S_B[j], agg(blocks strictly between), P_B[k] )
// where S_B[j] is the maximum from j to the end of its block (a suffix scan)
// and P_B[k] the maximum from the start of k's block to k (a prefix scan).
//   * s <  T (tile): B = 2^floor(log2 s); then b(k) is b(j)+1 or b(j)+2 and at
//     most one block aggregate is needed, read back as P_B at that block's end.
//   * s >= T: B = T (blocks are tiles); k lies q or q+1 tiles after j
//     (s = qT + r), and the tiles between contribute tile aggregates kept in a
//     small ring in shared memory.
// With the output index j as the thread's own index, S_B lives in registers,
// and P_B is read from a 3-tile ring in shared memory at offset s.  Each input
// element is read from HBM once (for s >= T the J-side tile is re-read about
// w elements later, normally from L2) and each output written once.
//
// Work decomposition.  A work item is a contiguous range of output tiles of one
// series.  A CTA owns an item at a time and streams its input tiles in order:
// one producer warp issues 1D bulk TMA copies into a ring of stages
// (mbarrier transaction counts), 8 consumer warps read their 16 contiguous
// elements (64 bytes for f32) per tile, scan, and store.  Items come from a
// static round-robin (1D launches: one per CTA) or an atomic ticket (batched
// plans).  Every wait is bounded; a timeout sets a bit in the device status
// word and the CTA drains its copies and returns.
#pragma once
#include <cstdint>

#include "ptx.cuh"

namespace mmf {

// ------------------------------------------------------------ element types
template <typename T> struct Elem;
template <> struct Elem<float> {
    using R = float;
    static constexpr int V = 16;
    __device__ static R lo() { return __int_as_float(0xff800000); }
    __device__ static R hi() { return __int_as_float(0x7f800000); }
};
template <> struct Elem<double> {
    using R = double;
    static constexpr int V = 8;
    __device__ static R lo() { return __longlong_as_double(0xfff0000000000000ULL); }
    __device__ static R hi() { return __longlong_as_double(0x7ff0000000000000ULL); }
};
template <> struct Elem<int16_t> {
    using R = int;
    static constexpr int V = 16;
    __device__ static R lo() { return -32768; }
    __device__ static R hi() { return 32767; }
};
template <> struct Elem<uint8_t> {
    using R = int;
    static constexpr int V = 16;
    __device__ static R lo() { return 0; }
    __device__ static R hi() { return 255; }
};

__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ int vmax(int a, int b) { return max(a, b); }
__device__ __forceinline__ int vmin(int a, int b) { return min(a, b); }

// Element at compile-time byte offset B of a little-endian word array.
template <typename T> struct WordElem;
template <> struct WordElem<float> {
    template <int B> __device__ static float get(const uint32_t *wd) { return __uint_as_float(wd[B >> 2]); }
};
template <> struct WordElem<double> {
    template <int B> __device__ static double get(const uint32_t *wd) {
        return __hiloint2double((int)wd[(B >> 2) + 1], (int)wd[B >> 2]);
    }
};
template <> struct WordElem<int16_t> {
    template <int B> __device__ static int get(const uint32_t *wd) {
        return (int)(int16_t)(wd[B >> 2] >> ((B & 3) * 8));
    }
};
template <> struct WordElem<uint8_t> {
    template <int B> __device__ static int get(const uint32_t *wd) { return (int)((wd[B >> 2] >> ((B & 3) * 8)) & 0xffu); }
};

template <typename T, int S, int I, int V> struct ExtractLoop {
    __device__ static void run(const uint32_t *wd, typename Elem<T>::R *x) {
        x[I] = WordElem<T>::template get<(S + I) * (int)sizeof(T)>(wd);
        ExtractLoop<T, S, I + 1, V>::run(wd, x);
    }
};
template <typename T, int S, int V> struct ExtractLoop<T, S, V, V> {
    __device__ static void run(const uint32_t *, typename Elem<T>::R *) {}
};

// Dispatch the (warp-uniform) element shift to a compile-time extraction.
template <typename T, int S = 0>
__device__ __forceinline__ void extract_shifted(int s, const uint32_t *wd, typename Elem<T>::R *x) {
    if constexpr (S < 16 / (int)sizeof(T)) {
        if (s == S) {
            ExtractLoop<T, S, 0, Elem<T>::V>::run(wd, x);
            return;
        }
        extract_shifted<T, S + 1>(s, wd, x);
    }
}

template <typename T> __device__ __forceinline__ uint32_t pack_word(const typename Elem<T>::R *x, int w);
template <> __device__ __forceinline__ uint32_t pack_word<float>(const float *x, int w) { return __float_as_uint(x[w]); }
template <> __device__ __forceinline__ uint32_t pack_word<double>(const double *x, int w) {
    return (w & 1) ? (uint32_t)__double2hiint(x[w >> 1]) : (uint32_t)__double2loint(x[w >> 1]);
}
template <> __device__ __forceinline__ uint32_t pack_word<int16_t>(const int *x, int w) {
    return ((uint32_t)(uint16_t)x[2 * w]) | ((uint32_t)(uint16_t)x[2 * w + 1] << 16);
}
template <> __device__ __forceinline__ uint32_t pack_word<uint8_t>(const int *x, int w) {
    return ((uint32_t)(x[4 * w] & 0xff)) | ((uint32_t)(x[4 * w + 1] & 0xff) << 8) |
           ((uint32_t)(x[4 * w + 2] & 0xff) << 16) | ((uint32_t)(x[4 * w + 3] & 0xff) << 24);
}

// ------------------------------------------------------------- parameters
struct SeriesDesc {
    int64_t in_off;   // element offset of the series in the input buffer
    int64_t n;        // input length
    int64_t out_off;  // element offset of its outputs in each output buffer
    int64_t w;        // window length (envelope: 2r+1)
    int64_t d;        // input position of output 0's window start: 0 or -r
    int64_t n_out;    // number of outputs
};

struct ItemDesc {
    int64_t series;
    int64_t o_begin;
    int64_t o_end;
};

struct BlockScanParams {
    const void *in;
    void *out_max;
    void *out_min;
    const SeriesDesc *series;  // table (batched) or nullptr (use `one`)
    const ItemDesc *items;     // table (batched) or nullptr (arithmetic)
    SeriesDesc one;            // the single series of a 1D launch
    int64_t seg_outputs;       // 1D: outputs per item (multiple of the tile)
    int64_t n_items;
    int *ticket;               // nullptr: static round-robin; else atomic ticket
    uint32_t *status;          // device status word
};

constexpr int kConsumerWarps = 8;
constexpr int kNT = kConsumerWarps * 32;
constexpr int kThreads = kNT;  // thread 0 also issues the copies
constexpr int kStages = 4;
constexpr int kQCap = 1024 + 8;     // tile-aggregate ring (>= max tiles per window + 2)

template <typename T> struct Geo {
    static constexpr int V = Elem<T>::V;
    static constexpr int LGV = (V == 16) ? 4 : 3;
    static constexpr int T_ = kNT * V;  // tile, elements
    static constexpr int LGT = (T_ == 4096) ? 12 : 11;
    static constexpr int NCH = V * (int)sizeof(T) / 16;  // 16-byte chunks per thread
    static constexpr int STAGE_BYTES = ((T_ * (int)sizeof(T) + 16 + 127) / 128) * 128;
    static constexpr int RING = 3 * T_;                       // logical ring elements
    static constexpr int RING_PHYS = RING + RING / 16 + 16;   // 1 pad per 16
    static constexpr size_t off_stage = 0;
    static constexpr size_t off_ring_max = off_stage + (size_t)kStages * STAGE_BYTES;
    static constexpr size_t off_ring_min = off_ring_max + ((RING_PHYS * sizeof(T) + 127) / 128) * 128;
    static constexpr size_t off_ta_max = off_ring_min + ((RING_PHYS * sizeof(T) + 127) / 128) * 128;
    static constexpr size_t off_ta_min = off_ta_max + ((kQCap * sizeof(T) + 127) / 128) * 128;
    static constexpr size_t off_misc = off_ta_min + ((kQCap * sizeof(T) + 127) / 128) * 128;
    // misc: wtot[2][2 dir][2 side][8] R, mid[2][2][2] R, full barriers,
    // stage items, producer state
    static constexpr size_t off_wtot = 0;
    static constexpr size_t off_mid = off_wtot + 2 * 2 * 2 * kConsumerWarps * 8;
    static constexpr size_t off_bar = off_mid + 2 * 2 * 2 * 8;
    static constexpr size_t off_sitem = off_bar + kStages * 8;
    static constexpr size_t off_prod = off_sitem + kStages * 8;
    static constexpr size_t misc_bytes = off_prod + 64;
    static constexpr size_t smem_bytes = off_misc + misc_bytes;
};

// Per-item quantities, computed identically by producer and consumers.
template <typename T> struct ItemPlan {
    const T *in;
    T *omax;
    T *omin;
    int64_t n;
    int64_t p0;       // input position of relative position 0 (= o_begin + d)
    int64_t o_begin;
    int64_t o_end;
    int64_t s;        // w - 1
    int q;            // s / T
    int caseB;        // s >= T
    int lgB;          // block size log2
    int NC;           // output tiles in the item
    int ok;
};

template <typename T>
__device__ __forceinline__ ItemPlan<T> make_plan(const BlockScanParams &P, int64_t item) {
    using G = Geo<T>;
    ItemPlan<T> ip;
    SeriesDesc sd;
    int64_t ob, oe;
    if (P.items) {
        ItemDesc it = P.items[item];
        sd = P.series[it.series];
        ob = it.o_begin;
        oe = it.o_end;
    } else {
        sd = P.one;
        ob = item * P.seg_outputs;
        oe = ob + P.seg_outputs;
        if (oe > sd.n_out) oe = sd.n_out;
    }
    ip.in = reinterpret_cast<const T *>(P.in) + sd.in_off;
    ip.omax = P.out_max ? reinterpret_cast<T *>(P.out_max) + sd.out_off : nullptr;
    ip.omin = P.out_min ? reinterpret_cast<T *>(P.out_min) + sd.out_off : nullptr;
    ip.n = sd.n;
    ip.o_begin = ob;
    ip.o_end = oe;
    ip.p0 = ob + sd.d;
    ip.s = sd.w - 1;
    ip.q = (int)(ip.s >> G::LGT);
    ip.caseB = ip.s >= G::T_;
    if (ip.caseB) {
        ip.lgB = G::LGT;
    } else {
        int lg = 0;
        while ((2ll << lg) <= ip.s) ++lg;  // floor(log2 s), s >= 1; s == 0 -> 0
        ip.lgB = lg;
    }
    ip.NC = oe > ob ? (int)((oe - ob + G::T_ - 1) >> G::LGT) : 0;
    ip.ok = (ip.q + 2 <= kQCap) && oe >= ob;
    return ip;
}

// Loads of one item, in order: prologue tiles x = (caseB ? 1 : 0) .. q, then
// per output tile c: K tile c+q+1 and, when caseB, J tile c.
template <typename T> __device__ __forceinline__ int item_loads(const ItemPlan<T> &ip) {
    if (!ip.ok) return 1;  // a rejected item is one empty stage
    int pro = ip.caseB ? ip.q : 1;
    return pro + ip.NC * (ip.caseB ? 2 : 1);
}

struct StageCursor {
    int stage = 0;
    uint32_t phase = 0;
    __device__ __forceinline__ void advance() {
        if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
        }
    }
};

// Byte range of input tile x that the TMA engine copies: the 16-byte aligned
// interior of [p0 + xT, p0 + xT + T) clipped to [0, n).
template <typename T> struct TileCopy {
    uintptr_t g_aligned_base;  // 16B-aligned address that maps to stage byte 0
    uintptr_t src;             // first copied byte
    uint32_t bytes;            // copied bytes (multiple of 16, may be 0)
    int64_t a;                 // first input position of the tile
    int64_t int_lo, int_hi;    // positions fully covered by the copy
};

template <typename T> __device__ __forceinline__ TileCopy<T> tile_copy(const ItemPlan<T> &ip, int x) {
    using G = Geo<T>;
    TileCopy<T> tc;
    tc.a = ip.p0 + (int64_t)x * G::T_;
    const intptr_t base = (intptr_t)ip.in;
    const intptr_t ga = base + tc.a * (intptr_t)sizeof(T);
    tc.g_aligned_base = (uintptr_t)(ga & ~(intptr_t)15);
    int64_t lo = tc.a > 0 ? tc.a : 0;
    int64_t hi = tc.a + G::T_ < ip.n ? tc.a + G::T_ : ip.n;
    tc.bytes = 0;
    tc.src = 0;
    tc.int_lo = tc.int_hi = lo;
    if (hi > lo) {
        intptr_t gb = base + lo * (intptr_t)sizeof(T);
        intptr_t ge = base + hi * (intptr_t)sizeof(T);
        intptr_t gbu = (gb + 15) & ~(intptr_t)15;
        intptr_t geu = ge & ~(intptr_t)15;
        if (geu > gbu) {
            tc.bytes = (uint32_t)(geu - gbu);
            tc.src = (uintptr_t)gbu;
            tc.int_lo = (gbu - base) / (intptr_t)sizeof(T);
            tc.int_hi = (geu - base) / (intptr_t)sizeof(T);
        }
    }
    return tc;
}

// ------------------------------------------------------------------ kernel
// Copy issue state of thread 0, kept in shared memory so that it costs the
// other threads no registers.
struct ProdState {
    int64_t item;     // current item (valid when l < nloads)
    int64_t k;        // static round-robin cursor
    int64_t issued;   // loads issued so far (all items)
    int32_t l;        // next load within the item
    int32_t nloads;   // loads of the item
    int32_t finished; // end marker issued
    int32_t pad;
};

template <typename T>
__device__ __forceinline__ bool next_item(const BlockScanParams &P, ProdState &ps, int64_t &item) {
    if (P.ticket) {
        item = atomicAdd(P.ticket, 1);
    } else {
        item = (int64_t)blockIdx.x + ps.k * gridDim.x;
        ++ps.k;
    }
    return item < P.n_items;
}

// Thread 0 only: issue copies until `consumed + kStages` loads are in flight.
// Stages consumed before the caller's barrier are free, so this never waits.
template <typename T>
__device__ void refill(const BlockScanParams &P, uint8_t *smem, int64_t consumed) {
    using G = Geo<T>;
    uint8_t *misc = smem + G::off_misc;
    uint64_t *full_bar = reinterpret_cast<uint64_t *>(misc + G::off_bar);
    int64_t *stage_item = reinterpret_cast<int64_t *>(misc + G::off_sitem);
    ProdState &ps = *reinterpret_cast<ProdState *>(misc + G::off_prod);
    while (!ps.finished && ps.issued < consumed + kStages) {
        const int stage = (int)(ps.issued % kStages);
        if (ps.l >= ps.nloads) {
            int64_t item;
            if (!next_item<T>(P, ps, item)) {
                stage_item[stage] = -1;  // end marker: an empty phase
                mbar_arrive_expect_tx(&full_bar[stage], 0);
                ps.finished = 1;
                ps.issued++;
                break;
            }
            ItemPlan<T> ip = make_plan<T>(P, item);
            if (!ip.ok) report_error(P.status, kErrBadItem);
            ps.item = item;
            ps.nloads = item_loads(ip);
            ps.l = 0;
        }
        ItemPlan<T> ip = make_plan<T>(P, ps.item);
        stage_item[stage] = ps.l == 0 ? ps.item : -2;
        uint32_t bytes = 0;
        void *dst = nullptr;
        const void *src = nullptr;
        bool keep = false;
        if (ip.ok) {
            int x;
            const int pro = ip.caseB ? ip.q : 1;
            if (ps.l < pro) {
                x = ip.caseB ? 1 + ps.l : 0;
                keep = ip.caseB;
            } else {
                const int r = ps.l - pro;
                const int c = ip.caseB ? r >> 1 : r;
                const bool jload = ip.caseB && (r & 1);
                x = jload ? c : c + ip.q + 1;
                keep = ip.caseB && !jload;  // re-read later as a J tile
            }
            TileCopy<T> tc = tile_copy<T>(ip, x);
            bytes = tc.bytes;
            dst = smem + G::off_stage + (size_t)stage * G::STAGE_BYTES + (tc.src - tc.g_aligned_base);
            src = reinterpret_cast<const void *>(tc.src);
        }
        mbar_arrive_expect_tx(&full_bar[stage], bytes);
        if (bytes) tma_load_1d(dst, src, bytes, &full_bar[stage], keep ? policy_evict_last() : policy_evict_first());
        ps.l++;
        ps.issued++;
    }
}

template <typename T, bool FULL>
struct Consumer {
    using R = typename Elem<T>::R;
    using G = Geo<T>;
    static constexpr int V = G::V;

    const BlockScanParams *P;
    uint8_t *smem;
    T *ring_max, *ring_min, *ta_max, *ta_min;
    R *wtot;  // [2 buf][2 dir][2 side][8 warps]
    R *mid;   // [2 buf][2 which][2 side]
    uint64_t *full_bar;
    uint32_t *status;
    int tid, lane, warp;
    int wbuf = 0;
    int64_t consumed = 0;
    StageCursor cur;
    bool failed = false;

    __device__ __forceinline__ int ring_phys(int idx) const { return idx + (idx >> 4); }

    // Barrier over the CTA; afterwards thread 0 refills the consumed stages.
    __device__ __forceinline__ void sync() {
        named_bar_sync(1, kNT);
        if (tid == 0) refill<T>(*P, smem, consumed);
    }

    // Read input tile x of the item into registers (max-side and min-side
    // copies differ only where positions fall outside [0, n): padding).
    __device__ __forceinline__ bool read_tile(const ItemPlan<T> &ip, int x, R (&xm)[V], R (&xn)[V]) {
        if (!mbar_wait_bounded(&full_bar[cur.stage], cur.phase)) {
            report_error(status, kErrWaitTimeout);
            failed = true;
            return false;
        }
        TileCopy<T> tc = tile_copy<T>(ip, x);
        const uint8_t *sb = smem + G::off_stage + (size_t)cur.stage * G::STAGE_BYTES;
        const int shift_b = (int)((((intptr_t)ip.in + tc.a * (intptr_t)sizeof(T))) & 15);
        uint32_t wd[4 * (G::NCH + 1)];
        const uint4 *p4 = reinterpret_cast<const uint4 *>(sb + (size_t)tid * V * sizeof(T));
#pragma unroll
        for (int c = 0; c < G::NCH; ++c) {
            uint4 v = p4[c];
            wd[4 * c] = v.x; wd[4 * c + 1] = v.y; wd[4 * c + 2] = v.z; wd[4 * c + 3] = v.w;
        }
        if (shift_b) {
            uint4 v = p4[G::NCH];
            wd[4 * G::NCH] = v.x; wd[4 * G::NCH + 1] = v.y; wd[4 * G::NCH + 2] = v.z; wd[4 * G::NCH + 3] = v.w;
        } else {
            wd[4 * G::NCH] = wd[4 * G::NCH + 1] = wd[4 * G::NCH + 2] = wd[4 * G::NCH + 3] = 0;
        }
        R xv[V];
        extract_shifted<T>(shift_b / (int)sizeof(T), wd, xv);
        const int64_t pt = tc.a + (int64_t)tid * V;
        if (pt >= tc.int_lo && pt + V <= tc.int_hi) {
#pragma unroll
            for (int i = 0; i < V; ++i) xm[i] = xn[i] = xv[i];
        } else {
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const int64_t p = pt + i;
                if (p < 0 || p >= ip.n) {
                    xm[i] = Elem<T>::lo();
                    xn[i] = Elem<T>::hi();
                } else if (p < tc.int_lo || p >= tc.int_hi) {
                    R v = (R)ip.in[p];
                    xm[i] = xn[i] = v;
                } else {
                    xm[i] = xn[i] = xv[i];
                }
            }
        }
        cur.advance();
        ++consumed;
        return true;
    }
    // Thread-local part of the block-segmented prefix (dir 0) scan.
    __device__ __forceinline__ void local_prefix(R (&m)[V], R (&n)[V], int lgB) const {
        if constexpr (FULL) {
#pragma unroll
            for (int i = 1; i < V; ++i) { m[i] = vmax(m[i - 1], m[i]); n[i] = vmin(n[i - 1], n[i]); }
        } else {
            const int bmask = (1 << lgB) - 1;
#pragma unroll
            for (int i = 1; i < V; ++i)
                if (i & bmask) { m[i] = vmax(m[i - 1], m[i]); n[i] = vmin(n[i - 1], n[i]); }
        }
    }
    __device__ __forceinline__ void local_suffix(R (&m)[V], R (&n)[V], int lgB) const {
        if constexpr (FULL) {
#pragma unroll
            for (int i = V - 2; i >= 0; --i) { m[i] = vmax(m[i + 1], m[i]); n[i] = vmin(n[i + 1], n[i]); }
        } else {
            const int bmask = (1 << lgB) - 1;
#pragma unroll
            for (int i = V - 2; i >= 0; --i)
                if ((i + 1) & bmask) { m[i] = vmax(m[i + 1], m[i]); n[i] = vmin(n[i + 1], n[i]); }
        }
    }

    // Cross-thread carries for segments of 2^lgS threads (lgS = lgB - LGV > 0).
    // dir 0: exclusive prefix carry from lower threads of the segment;
    // dir 1: exclusive suffix carry from higher threads.  Warp totals are
    // published in wtot[wbuf][dir] for segments spanning several warps.
    __device__ __forceinline__ void warp_carry(int dir, R tm, R tn, int lgS, R &cm, R &cn) {
        const int segl = lgS >= 5 ? 32 : (1 << lgS);
        const int lis = lane & (segl - 1);
        const int pos = dir == 0 ? lis : (segl - 1 - lis);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            if (d >= segl) break;
            R om = dir == 0 ? __shfl_up_sync(0xffffffffu, tm, d) : __shfl_down_sync(0xffffffffu, tm, d);
            R on = dir == 0 ? __shfl_up_sync(0xffffffffu, tn, d) : __shfl_down_sync(0xffffffffu, tn, d);
            if (pos >= d) { tm = vmax(tm, om); tn = vmin(tn, on); }
        }
        R em = dir == 0 ? __shfl_up_sync(0xffffffffu, tm, 1) : __shfl_down_sync(0xffffffffu, tm, 1);
        R en = dir == 0 ? __shfl_up_sync(0xffffffffu, tn, 1) : __shfl_down_sync(0xffffffffu, tn, 1);
        if (pos == 0) { em = Elem<T>::lo(); en = Elem<T>::hi(); }
        cm = em;
        cn = en;
        if (lgS > 5) {
            const bool pub = dir == 0 ? (lane == 31) : (lane == 0);
            if (pub) {
                R *wt = wtot + ((wbuf * 2 + dir) * 2) * kConsumerWarps;
                wt[warp] = tm;
                wt[kConsumerWarps + warp] = tn;
            }
        }
    }
    __device__ __forceinline__ void warp_carry_cross(int dir, int lgS, R &cm, R &cn) const {
        const int segw = 1 << (lgS - 5);
        const int wfirst = warp & ~(segw - 1);
        const R *wt = wtot + ((wbuf * 2 + dir) * 2) * kConsumerWarps;
        if (dir == 0) {
            for (int k = wfirst; k < warp; ++k) { cm = vmax(cm, wt[k]); cn = vmin(cn, wt[kConsumerWarps + k]); }
        } else {
            for (int k = warp + 1; k < wfirst + segw; ++k) { cm = vmax(cm, wt[k]); cn = vmin(cn, wt[kConsumerWarps + k]); }
        }
    }

    // Full block-segmented scans: prefix over (pm, pn) and, if do_suf, suffix
    // over (sm, sn).  One consumer barrier when segments span warps.
    __device__ __forceinline__ void scans(R (&pm)[V], R (&pn)[V], bool do_suf, R (&sm)[V], R (&sn)[V], int lgB) {
        local_prefix(pm, pn, lgB);
        if (do_suf) local_suffix(sm, sn, lgB);
        if (lgB > G::LGV) {
            const int lgS = lgB - G::LGV;
            R pcm, pcn, scm = Elem<T>::lo(), scn = Elem<T>::hi();
            warp_carry(0, pm[V - 1], pn[V - 1], lgS, pcm, pcn);
            if (do_suf) warp_carry(1, sm[0], sn[0], lgS, scm, scn);
            if (lgS > 5) {
                sync();
                warp_carry_cross(0, lgS, pcm, pcn);
                if (do_suf) warp_carry_cross(1, lgS, scm, scn);
                wbuf ^= 1;
            }
#pragma unroll
            for (int i = 0; i < V; ++i) { pm[i] = vmax(pm[i], pcm); pn[i] = vmin(pn[i], pcn); }
            if (do_suf) {
#pragma unroll
                for (int i = 0; i < V; ++i) { sm[i] = vmax(sm[i], scm); sn[i] = vmin(sn[i], scn); }
            }
        }
    }

    __device__ __forceinline__ void ring_write(int x, const R (&pm)[V], const R (&pn)[V]) {
        const int base = (x % 3) * G::T_ + tid * V;
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const int ph = ring_phys(base + i);
            ring_max[ph] = (T)pm[i];
            ring_min[ph] = (T)pn[i];
        }
    }

    __device__ __forceinline__ void run_item(const ItemPlan<T> &ip) {
        R sm[V], sn[V];  // suffix scan of the J tile of the current output tile
        const int q = ip.q;
        // ---------------- prologue
        const int xs = ip.caseB ? 1 : 0;
        for (int x = xs; x <= q; ++x) {
            R pm[V], pn[V];
            if (!read_tile(ip, x, pm, pn)) return;
            if (!ip.caseB) {
#pragma unroll
                for (int i = 0; i < V; ++i) { sm[i] = pm[i]; sn[i] = pn[i]; }
            }
            scans(pm, pn, !ip.caseB, sm, sn, ip.lgB);
            if (x == q) ring_write(x, pm, pn);
            if (ip.caseB && tid == kNT - 1) { ta_max[x % kQCap] = (T)pm[V - 1]; ta_min[x % kQCap] = (T)pn[V - 1]; }
        }
        sync();
        // ---------------- main loop over output tiles
        const int64_t s = ip.s;
        for (int c = 0; c < ip.NC; ++c) {
            if (ip.caseB && warp == 0) {
                // Mid1 = max over tile aggregates c+1 .. c+q-1; Mid2 adds c+q.
                R m1 = Elem<T>::lo(), n1 = Elem<T>::hi();
                for (int x = c + 1 + lane; x <= c + q - 1; x += 32) {
                    m1 = vmax(m1, (R)ta_max[x % kQCap]);
                    n1 = vmin(n1, (R)ta_min[x % kQCap]);
                }
#pragma unroll
                for (int d = 16; d >= 1; d >>= 1) {
                    m1 = vmax(m1, __shfl_xor_sync(0xffffffffu, m1, d));
                    n1 = vmin(n1, __shfl_xor_sync(0xffffffffu, n1, d));
                }
                if (lane == 0) {
                    R *md = mid + (c & 1) * 4;
                    const int xl = (c + q) % kQCap;
                    md[0] = m1;
                    md[1] = n1;
                    md[2] = vmax(m1, (R)ta_max[xl]);
                    md[3] = vmin(n1, (R)ta_min[xl]);
                }
            }
            R pm[V], pn[V], nm[V], nn[V];
            const int xk = c + q + 1;
            if (!read_tile(ip, xk, pm, pn)) return;
            if (!ip.caseB) {
#pragma unroll
                for (int i = 0; i < V; ++i) { nm[i] = pm[i]; nn[i] = pn[i]; }
                scans(pm, pn, true, nm, nn, ip.lgB);
            } else {
                if (!read_tile(ip, c, sm, sn)) return;
                scans(pm, pn, true, sm, sn, ip.lgB);
            }
            ring_write(xk, pm, pn);
            if (ip.caseB && tid == kNT - 1) { ta_max[xk % kQCap] = (T)pm[V - 1]; ta_min[xk % kQCap] = (T)pn[V - 1]; }
            sync();

            // ------------ outputs of tile c
            R om[V], on[V];
            const int64_t jr0 = (int64_t)c * G::T_ + (int64_t)tid * V;  // relative J position of element 0
            const int64_t kr0 = jr0 + s;
            const int ring_len = G::RING;
            int ridx = (int)(kr0 % ring_len);
            if (ip.caseB) {
                const R *md = mid + (c & 1) * 4;
                const R m1 = md[0], n1 = md[1], m2 = md[2], n2 = md[3];
                const int64_t cross = (int64_t)(c + q + 1) * G::T_ - kr0;  // i >= cross -> k in tile c+q+1
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    int r = ridx + i;
                    if (r >= ring_len) r -= ring_len;
                    const int ph = ring_phys(r);
                    const bool far = i >= cross;
                    om[i] = vmax(sm[i], vmax((R)ring_max[ph], far ? m2 : m1));
                    on[i] = vmin(sn[i], vmin((R)ring_min[ph], far ? n2 : n1));
                }
            } else if (FULL) {
                const int lgB = ip.lgB;
                const int64_t bj = jr0 >> lgB;
                const int64_t cross = ((bj + 2) << lgB) - kr0;  // i >= cross -> k in block bj+2
                R mm = Elem<T>::lo(), mn_ = Elem<T>::hi();
                if (cross < V) {
                    int r = (int)((((bj + 2) << lgB) - 1) % ring_len);
                    mm = (R)ring_max[ring_phys(r)];
                    mn_ = (R)ring_min[ring_phys(r)];
                }
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    int r = ridx + i;
                    if (r >= ring_len) r -= ring_len;
                    const int ph = ring_phys(r);
                    const bool far = i >= cross;
                    om[i] = vmax(sm[i], vmax((R)ring_max[ph], far ? mm : Elem<T>::lo()));
                    on[i] = vmin(sn[i], vmin((R)ring_min[ph], far ? mn_ : Elem<T>::hi()));
                }
            } else {
                const int lgB = ip.lgB;
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    int r = ridx + i;
                    if (r >= ring_len) r -= ring_len;
                    const int ph = ring_phys(r);
                    R vm = vmax(sm[i], (R)ring_max[ph]);
                    R vn = vmin(sn[i], (R)ring_min[ph]);
                    const int64_t bj = (jr0 + i) >> lgB, bk = (kr0 + i) >> lgB;
                    if (bk == bj + 2) {
                        int rm = (int)(((bk << lgB) - 1) % ring_len);
                        vm = vmax(vm, (R)ring_max[ring_phys(rm)]);
                        vn = vmin(vn, (R)ring_min[ring_phys(rm)]);
                    }
                    om[i] = vm;
                    on[i] = vn;
                }
            }
            // ------------ store
            const int64_t o0 = ip.o_begin + jr0;
            if (o0 < ip.o_end) {
                const bool full = o0 + V <= ip.o_end;
                if (ip.omax) store(ip.omax + o0, om, full ? V : (int)(ip.o_end - o0));
                if (ip.omin) store(ip.omin + o0, on, full ? V : (int)(ip.o_end - o0));
            }
            if (!ip.caseB) {
#pragma unroll
                for (int i = 0; i < V; ++i) { sm[i] = nm[i]; sn[i] = nn[i]; }
            }
        }
    }

    __device__ __forceinline__ void store(T *dst, const R (&v)[V], int cnt) const {
        if (cnt == V && (((uintptr_t)dst) & 15) == 0) {
            uint4 *d4 = reinterpret_cast<uint4 *>(dst);
#pragma unroll
            for (int c = 0; c < G::NCH; ++c) {
                uint4 u;
                u.x = pack_word<T>(v, 4 * c);
                u.y = pack_word<T>(v, 4 * c + 1);
                u.z = pack_word<T>(v, 4 * c + 2);
                u.w = pack_word<T>(v, 4 * c + 3);
                __stcs(d4 + c, u);
            }
        } else {
#pragma unroll
            for (int i = 0; i < V; ++i)
                if (i < cnt) dst[i] = (T)v[i];
        }
    }
};

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) blockscan_kernel(const BlockScanParams P) {
    using G = Geo<T>;
    using R = typename Elem<T>::R;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t *misc = smem + G::off_misc;
    R *wtot = reinterpret_cast<R *>(misc + G::off_wtot);
    R *mid = reinterpret_cast<R *>(misc + G::off_mid);
    uint64_t *full_bar = reinterpret_cast<uint64_t *>(misc + G::off_bar);
    int64_t *stage_item = reinterpret_cast<int64_t *>(misc + G::off_sitem);

    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&full_bar[s], 1);
        fence_mbar_init();
        ProdState &ps = *reinterpret_cast<ProdState *>(misc + G::off_prod);
        ps.item = -1;
        ps.k = 0;
        ps.issued = 0;
        ps.l = 0;
        ps.nloads = 0;
        ps.finished = 0;
        refill<T>(P, smem, 0);
    }
    __syncthreads();

    Consumer<T, true> cf;
    Consumer<T, false> cg;
    auto setup = [&](auto &cc) {
        cc.P = &P;
        cc.smem = smem;
        cc.ring_max = reinterpret_cast<T *>(smem + G::off_ring_max);
        cc.ring_min = reinterpret_cast<T *>(smem + G::off_ring_min);
        cc.ta_max = reinterpret_cast<T *>(smem + G::off_ta_max);
        cc.ta_min = reinterpret_cast<T *>(smem + G::off_ta_min);
        cc.wtot = wtot;
        cc.mid = mid;
        cc.full_bar = full_bar;
        cc.status = P.status;
        cc.tid = tid;
        cc.lane = tid & 31;
        cc.warp = tid >> 5;
    };
    setup(cf);
    setup(cg);
    StageCursor cur;
    int wbuf = 0;
    int64_t consumed = 0;
    while (true) {
        // The first stage of each item carries its index (-1 marks the end).
        if (!mbar_wait_bounded(&full_bar[cur.stage], cur.phase)) {
            report_error(P.status, kErrWaitTimeout);
            return;
        }
        const int64_t item = stage_item[cur.stage];
        if (item < 0) return;
        ItemPlan<T> ip = make_plan<T>(P, item);
        if (!ip.ok) {
            cur.advance();
            ++consumed;
        } else if (ip.caseB || ip.lgB >= Geo<T>::LGV) {
            cf.cur = cur; cf.wbuf = wbuf; cf.consumed = consumed;
            cf.run_item(ip);
            if (cf.failed) return;
            cur = cf.cur; wbuf = cf.wbuf; consumed = cf.consumed;
        } else {
            cg.cur = cur; cg.wbuf = wbuf; cg.consumed = consumed;
            cg.run_item(ip);
            if (cg.failed) return;
            cur = cg.cur; wbuf = cg.wbuf; consumed = cg.consumed;
        }
        // Item boundary: the ring may be reused and consumed stages refilled.
        named_bar_sync(1, kNT);
        if (tid == 0) refill<T>(P, smem, consumed);
    }
}

}  // namespace mmf
