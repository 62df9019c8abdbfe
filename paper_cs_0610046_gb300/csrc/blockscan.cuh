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
// A tile is NT threads x V consecutive elements per thread (f32: 128 x 16).
// Block modes, by s (the register slide, mode 3, takes w <= 17 for f32 and
// w <= 9 for the other types instead):
//   0  s < V:       B = 2^floor(log2 s), blocks inside one thread;
//   1  s < 32V:     B = 2^floor(log2 s), blocks of 2..16 lanes;
//   2  s >= 32V:    B = 32V, one block per warp slice.
// With B = 2^floor(log2 s) (modes 0, 1), k's block is b(j)+1 or b(j)+2, so at
// most one whole block lies between.  Every thread scans its own V elements
// (a local prefix for the K role, a local suffix for the J role); the parts
// of the window outside the two local scans (lane carries inside j's and k's
// blocks, the whole blocks between) are per-thread constants, so each output
// is one three-operand max (and min).  Local prefixes go to a 3-tile ring of
// (max, min) pairs in shared memory and are read back at offset s.  For
// s >= T (case B, mode 2 only) whole tiles lie between: their aggregates
// are kept by warp 0 as a sliding two-stack queue (TileQueue) inside a ring
// of tile aggregates, and the J tile is read a second time, about w elements
// after its read as a K tile.  Otherwise each input element is read from
// global memory once, and each output is written once.
//
// Work decomposition.  A work item is a contiguous range of output tiles of
// one series.  A CTA owns one item at a time and streams its input tiles in
// order.  Each warp reads only its own slice (32V elements) of every tile,
// so each warp has its own ring of kStages stages fed by 1D bulk copies that
// its lane 0 issues (one mbarrier per warp and stage), refilling a stage as
// soon as the warp has read it.  One CTA barrier per tile orders the prefix
// ring and the block aggregates between warps.  Items come from a static
// round-robin (1D launches) or an atomic ticket (batched plans).  Every wait
// is bounded; a timeout sets a bit in the device status word and the CTA
// returns.
#pragma once
#include <cstdint>

#include "ptx.cuh"

namespace mmf {

// ------------------------------------------------------------ element types
// V: elements per thread per tile; PS: log2 of the ring padding period (one
// padding pair every 2^PS pairs keeps strided ring accesses conflict-free).
template <typename T> struct Elem;
template <> struct Elem<float> {
    using R = float;
    using Pair = float2;
    static constexpr int V = 16, PS = 4, NW = 4;
    __device__ static R lo() { return __int_as_float(0xff800000); }
    __device__ static R hi() { return __int_as_float(0x7f800000); }
    __device__ static Pair pair(R m, R n) { return make_float2(m, n); }
    __device__ static R pmax(Pair p) { return p.x; }
    __device__ static R pmin(Pair p) { return p.y; }
    __device__ static R load(float x) { return x; }
    __device__ static float store(R x) { return x; }
};
// Doubles are compared as order-preserving 64-bit integer keys (sign bit kept,
// magnitude bits flipped for negatives): for non-NaN values the integer order
// is the floating-point order, and GB300's integer pipes are far faster than
// its FP64 pipe.  Keys are converted back on store, so results are exact.
template <> struct Elem<double> {
    using R = long long;
    using Pair = longlong2;
    static constexpr int V = 4, PS = 3, NW = 8;
    __device__ static R key(long long b) { return b ^ ((b >> 63) & 0x7fffffffffffffffLL); }
    __device__ static R lo() { return key((long long)0xfff0000000000000ULL); }  // -inf
    __device__ static R hi() { return key(0x7ff0000000000000LL); }              // +inf
    __device__ static Pair pair(R m, R n) { return make_longlong2(m, n); }
    __device__ static R pmax(Pair p) { return p.x; }
    __device__ static R pmin(Pair p) { return p.y; }
    __device__ static R load(double x) { return key(__double_as_longlong(x)); }
    __device__ static double store(R k) { return __longlong_as_double(key(k)); }
};
template <> struct Elem<int16_t> {
    using R = int;
    using Pair = short2;
    static constexpr int V = 16, PS = 4, NW = 8;
    __device__ static R lo() { return -32768; }
    __device__ static R hi() { return 32767; }
    __device__ static Pair pair(R m, R n) { return make_short2((short)m, (short)n); }
    __device__ static R pmax(Pair p) { return p.x; }
    __device__ static R pmin(Pair p) { return p.y; }
    __device__ static R load(int16_t x) { return x; }
    __device__ static int16_t store(R x) { return (int16_t)x; }
};
template <> struct Elem<uint8_t> {
    using R = int;
    using Pair = uchar2;
    static constexpr int V = 16, PS = 4, NW = 8;
    __device__ static R lo() { return 0; }
    __device__ static R hi() { return 255; }
    __device__ static Pair pair(R m, R n) { return make_uchar2((unsigned char)m, (unsigned char)n); }
    __device__ static R pmax(Pair p) { return p.x; }
    __device__ static R pmin(Pair p) { return p.y; }
    __device__ static R load(uint8_t x) { return x; }
    __device__ static uint8_t store(R x) { return (uint8_t)x; }
};

// Arithmetic of the envelope lower bound per element type: f32 in float
// (rounding bounded in the design notes), f64 in double, the integer types
// exactly in 64-bit integers.
template <typename T> struct LbAcc { using A = float; };
template <> struct LbAcc<double> { using A = double; };
template <> struct LbAcc<int16_t> { using A = long long; };
template <> struct LbAcc<uint8_t> { using A = long long; };

__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ long long vmax(long long a, long long b) { return a > b ? a : b; }
__device__ __forceinline__ long long vmin(long long a, long long b) { return a < b ? a : b; }
__device__ __forceinline__ int vmax(int a, int b) { return max(a, b); }
__device__ __forceinline__ int vmin(int a, int b) { return min(a, b); }
// Three-operand forms: one instruction for f32 on sm_100-family GPUs.
__device__ __forceinline__ float vmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float vmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
template <typename X> __device__ __forceinline__ X vmax3(X a, X b, X c) { return vmax(vmax(a, b), c); }
template <typename X> __device__ __forceinline__ X vmin3(X a, X b, X c) { return vmin(vmin(a, b), c); }

// Element at compile-time byte offset B of a little-endian word array.
template <typename T> struct WordElem;
template <> struct WordElem<float> {
    template <int B> __device__ static float get(const uint32_t *wd) { return __uint_as_float(wd[B >> 2]); }
};
template <> struct WordElem<double> {
    template <int B> __device__ static long long get(const uint32_t *wd) {
        return Elem<double>::key((long long)(((unsigned long long)wd[(B >> 2) + 1] << 32) | wd[B >> 2]));
    }
};
template <> struct WordElem<int16_t> {
    template <int B> __device__ static int get(const uint32_t *wd) {
        return (int)(int16_t)(wd[B >> 2] >> ((B & 3) * 8));
    }
};
template <> struct WordElem<uint8_t> {
    template <int B> __device__ static int get(const uint32_t *wd) {
        return (int)((wd[B >> 2] >> ((B & 3) * 8)) & 0xffu);
    }
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

// Moves a little-endian byte sequence of N + 4 words down by sb bytes
// (0 <= sb < 16, the same for the whole warp): afterwards word k holds bytes
// [4k + sb, 4k + sb + 4) of the original sequence, for k < N.  A two-stage
// barrel shift by whole words, then a funnel shift for the rest.
template <int N>
__device__ __forceinline__ void shift_bytes(uint32_t (&wd)[N + 4], int sb) {
    const int sw = sb >> 2;
#pragma unroll
    for (int b = 1; b < 4; b <<= 1) {
        if (sw & b) {
#pragma unroll
            for (int k = 0; k + b < N + 4; ++k) wd[k] = wd[k + b];
        }
    }
    const int br = (sb & 3) * 8;
    if (br) {
#pragma unroll
        for (int k = 0; k < N; ++k) wd[k] = __funnelshift_r(wd[k], wd[k + 1], br);
    }
}

template <typename T> __device__ __forceinline__ uint32_t pack_word(const typename Elem<T>::R *x, int w);
template <> __device__ __forceinline__ uint32_t pack_word<float>(const float *x, int w) { return __float_as_uint(x[w]); }
template <> __device__ __forceinline__ uint32_t pack_word<double>(const long long *x, int w) {
    const unsigned long long b = (unsigned long long)Elem<double>::key(x[w >> 1]);
    return (w & 1) ? (uint32_t)(b >> 32) : (uint32_t)b;
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
    SeriesDesc one;            // the single series of a 1D launch (or every row)
    int64_t seg_outputs;       // 1D: outputs per item (multiple of the tile)
    int64_t n_items;
    int64_t row_items;         // > 0: rows mode, `one` repeated per row, row_items items a row
    int64_t in_pitch;          // rows mode: element stride between rows (input)
    int64_t out_pitch;         // rows mode: element stride between rows (outputs)
    int *ticket;               // nullptr: static round-robin; else atomic ticket
    uint32_t *status;          // device status word
    int64_t in_elems;          // elements of `in` that may be read (copies past a series end stay inside)
    // Envelope lower bound (batched, centred windows): when lb_acc is set, no
    // outputs are stored; each output i of series s instead adds the squared
    // excursion of lb_query[i] outside [min, max] to lb_acc[s].
    const void *lb_query;
    double *lb_acc;
    // Bound of every pipeline wait in SM clocks (0: kWaitLimitCycles), and
    // test flags (kTestStarveCopies: issue no input copies, so that every
    // wait runs out; for tests of the timeout path only).
    long long wait_limit;
    uint32_t test_flags;
    uint32_t pad_;
    // One advancing front (1D series, windows of a tile or more; see
    // run_front_item): work item i is output tile i, CTA b of the grid of G
    // takes items b, b+G, b+2G, ...; the aggregates of the whole tiles inside
    // the windows come from front_slots (two tagged words per global tile,
    // see front_put), published G items earlier by the item that read the
    // tile ahead (front_ahead = G), or at the start for the first G+q tiles.
    // front_last: the last global tile whose aggregate any item takes.
    // nullptr: items read those tiles themselves.
    unsigned long long *front_slots;
    int64_t front_last;
    int32_t front_ahead;
    int32_t pad2_;
};
static_assert(sizeof(BlockScanParams) <= 256, "parameters are copied to a 256-byte shared slot");
enum : uint32_t { kTestStarveCopies = 1u };

constexpr int kStages = 4;             // per-warp slice stages (power of two)
constexpr int kQCap = 1024 + 8;        // tile-aggregate ring (>= max tiles per window + 2)
constexpr int kQueue = 16;             // upcoming item ids under dynamic scheduling
constexpr int kMaxItemSpan = 1 << 30;  // relative positions of an item fit in int32

// Dynamic shared memory of the block-scan kernel (layout in Geo<T>).
extern __shared__ __align__(128) uint8_t bs_smem[];

// Copy-issue state of one warp (its lane 0 issues the warp's slice of every
// tile load).  Kept in shared memory so that it costs no registers.
struct WarpIssue {
    uintptr_t src0;  // this warp's slice of tile 0 of the item being issued, rounded down to 16 bytes
    const void *in;  // its series base
    int64_t n, p0;   // its length and the input position of its tile 0
    int32_t fast_lo, fast_hi;  // tiles whose slice lies inside the series (one copy, no checks)
    int32_t fast_smode;        // their copy mode: 0 (aligned) or 1 | shift << 8
    int32_t fast_extra;        // bytes copied past the slice for the shift (0 or 16)
    int32_t seq;     // its sequence number among this CTA's items
    int32_t l;       // next load within it
    int32_t nloads;  // its number of loads; -1 once the sequence has ended
    int32_t q, caseB, ok, NC, klast;
    int32_t issued;  // loads issued so far by this warp
    int32_t linear;  // load l of the item is tile l (every mode but case B)
    int32_t smode[kStages];  // per stage: copy mode | shift << 8, for the readers
};


// Modes 1 and 2 use thread-local scans with lane carries kept per thread (the
// carry ring) for every type but f64, whose larger pairs would leave room for
// only one CTA per SM; f64 applies the lane carries to every element instead.
template <typename T> constexpr bool kCarryRing = sizeof(T) != 8;

template <typename T> struct Geo {
    using Pair = typename Elem<T>::Pair;
    static constexpr int V = Elem<T>::V;
    static constexpr int PS = Elem<T>::PS;
    static constexpr int LGV = V == 16 ? 4 : (V == 8 ? 3 : 2);
    static constexpr int NW = Elem<T>::NW;  // warps per CTA
    static constexpr int NT = NW * 32;      // threads per CTA
    static constexpr int LGNT = NW == 8 ? 8 : 7;
    static constexpr int T_ = NT * V;  // tile, elements
    static constexpr int LGT = LGV + LGNT;
    static constexpr int SLICE = 32 * V;  // elements of a tile read by one warp
    static constexpr int NCH = V * (int)sizeof(T) / 16;  // 16-byte chunks per thread
    // Register-slide halo (elements after the slice, a multiple of 16 bytes)
    // and the largest w-1 the slide takes: 16 for f32 (one more thread's
    // elements), 8 for the others (their 256-thread CTAs leave 128 registers).
    static constexpr int HALO_MAX = sizeof(T) == 4 ? 16 : (8 > 16 / (int)sizeof(T) ? 8 : 16 / (int)sizeof(T));
    static constexpr int SLIDE_S = sizeof(T) == 4 ? 16 : 8;
    // A warp's slice arrives in PIECES copies of PLANES lanes' elements each,
    // placed PSTRIDE bytes apart; each piece holds room for the
    // register-slide halo and a 16-byte shift.  One piece: the bank spread of
    // the readers comes from the order in which lanes read their words
    // (see read_tile).
    static constexpr int PIECES = 1;
    static constexpr int PLANES = 32 / PIECES;
    static constexpr int PIECE = PLANES * V;  // elements
    static constexpr int PSTRIDE0 = (PIECE + HALO_MAX) * (int)sizeof(T) + 16;
    static constexpr int PSTRIDE = (PSTRIDE0 / 16) % 2 ? PSTRIDE0 : PSTRIDE0 + 16;
    static constexpr int SLICE_BYTES = PIECES * PSTRIDE;
    static constexpr int RING = 3 * T_;  // logical ring pairs
    static constexpr int RING_PHYS = RING + (RING >> PS) + 16;
    static constexpr size_t rnd(size_t b) { return (b + 127) / 128 * 128; }
    static constexpr size_t off_misc = 0;
    static constexpr size_t off_kagg = 0;  // [3 ring slots][NW warps] block aggregates of K tiles
    static constexpr size_t off_jagg = off_kagg + 3 * NW * sizeof(Pair);  // [2][NW] of J tiles
    static constexpr size_t off_tb = off_jagg + 2 * NW * sizeof(Pair);  // [2] whole tiles between (case B)
    static constexpr size_t off_bar = rnd(off_tb + 2 * sizeof(Pair));  // [warp][stage]
    static constexpr size_t off_issue = off_bar + NW * kStages * 8;
    static constexpr size_t off_queue = rnd(off_issue + NW * sizeof(WarpIssue));
    static constexpr size_t off_params = rnd(off_queue + kQueue * 8 + 16);
    static constexpr size_t misc_bytes = rnd(off_params + 256);
    static constexpr size_t off_stage = off_misc + misc_bytes;  // [warp][stage] slices
    static constexpr size_t off_ring = off_stage + rnd((size_t)NW * kStages * SLICE_BYTES);
    static constexpr size_t off_ta = off_ring + rnd(RING_PHYS * sizeof(Pair));
    static constexpr size_t off_cr = off_ta + rnd(kQCap * sizeof(Pair));  // [3 tiles][NT] carry records
    // Carry ring (modes 1, 2): per thread block of the last three tiles, the
    // lane carries inside its scan block: e = threads before it (exclusive),
    // g = including its own elements; [2][3 NT] pairs.
    static constexpr size_t smem_bytes = off_cr + (kCarryRing<T> ? rnd(2 * 3 * NT * sizeof(Pair)) : 0);
    // The register slide uses only the misc area and the stages.
    static constexpr size_t smem_bytes_slide = off_ring;
};
// Shared-memory regions (compile-time offsets from the shared window).
template <typename T> struct Smem {
    using G = Geo<T>;
    using Pair = typename Elem<T>::Pair;
    __device__ static uint8_t *slice(int warp, int s) {
        return bs_smem + G::off_stage + (size_t)(warp * kStages + s) * G::SLICE_BYTES;
    }
    // First byte of `lane`'s elements in a slice stage.
    __device__ static const uint8_t *lane_base(const uint8_t *slice, int lane) {
        return slice + (lane / G::PLANES) * G::PSTRIDE + (lane % G::PLANES) * G::V * (int)sizeof(T);
    }
    __device__ static Pair *ring() { return reinterpret_cast<Pair *>(bs_smem + G::off_ring); }
    __device__ static Pair *ta() { return reinterpret_cast<Pair *>(bs_smem + G::off_ta); }
    __device__ static Pair *cre() { return reinterpret_cast<Pair *>(bs_smem + G::off_cr); }
    __device__ static Pair *crg() { return cre() + 3 * G::NT; }
    __device__ static uint8_t *misc() { return bs_smem + G::off_misc; }
    __device__ static Pair *kagg() { return reinterpret_cast<Pair *>(misc() + G::off_kagg); }
    __device__ static Pair *jagg() { return reinterpret_cast<Pair *>(misc() + G::off_jagg); }
    __device__ static Pair *tb() { return reinterpret_cast<Pair *>(misc() + G::off_tb); }
    __device__ static uint64_t *bar(int warp, int s) {
        return reinterpret_cast<uint64_t *>(misc() + G::off_bar) + warp * kStages + s;
    }
    __device__ static WarpIssue *issue(int warp) { return reinterpret_cast<WarpIssue *>(misc() + G::off_issue) + warp; }
    __device__ static int64_t *queue() { return reinterpret_cast<int64_t *>(misc() + G::off_queue); }
    __device__ static const BlockScanParams &params() {
        return *reinterpret_cast<const BlockScanParams *>(misc() + G::off_params);
    }
};

// Per-item quantities, computed identically by thread 0 and the consumers.
template <typename T> struct ItemPlan {
    int64_t series;  // index in the series table (0 without one)
    double *lb_acc;  // envelope lower bound accumulators (null: store outputs)
    const T *in;
    T *omax;
    T *omin;
    int64_t n;
    int64_t p0;  // input position of relative position 0 (= o_begin + d)
    int64_t o_begin;
    int64_t o_end;
    int s;       // w - 1
    int q;       // s / T
    int caseB;   // s >= T
    int lgB;     // block size log2
    int mode;    // 0: B < V, 1: V <= B < 32V, 2: B = 32V (one block per warp); 3: register slide
    int NC;      // output tiles in the item
    int klast;   // 1 if some window of the last output tile reaches K tile NC+q
    int front;   // an item of the advancing front (one output tile, see run_front_item)
    int la;      // its tile read ahead (relative index q + G), 0 if none
    int64_t gt0; // global tile index of the item's tile 0 (advancing front)
    int ok;
};

// `want_mode` >= 0 rejects items of another block mode.
template <typename T>
__device__ __forceinline__ ItemPlan<T> make_plan(const BlockScanParams &P, int64_t item, int want_mode) {
    using G = Geo<T>;
    ItemPlan<T> ip;
    SeriesDesc sd;
    int64_t ob, oe;
    ip.series = 0;
    ip.lb_acc = P.lb_acc;
    if (P.items) {
        ItemDesc it = P.items[item];
        ip.series = it.series;
        sd = P.series[it.series];
        ob = it.o_begin;
        oe = it.o_end;
    } else if (P.row_items > 0) {
        const int64_t row = item / P.row_items;
        const int64_t seg = item - row * P.row_items;
        sd = P.one;
        sd.in_off += row * P.in_pitch;
        sd.out_off += row * P.out_pitch;
        ob = seg * P.seg_outputs;
        oe = ob + P.seg_outputs;
        if (oe > sd.n_out) oe = sd.n_out;
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
    const int64_t s = sd.w - 1;
    ip.s = (int)s;
    ip.q = (int)(s >> G::LGT);
    ip.caseB = s >= G::T_;
    if (s >= (int64_t)32 * G::V) {
        ip.lgB = G::LGV + 5;
        ip.mode = 2;
    } else {
        int lg = 0;
        while ((2ll << lg) <= s) ++lg;  // floor(log2 s) for s >= 1; 0 for s == 0
        ip.lgB = lg;
        ip.mode = lg >= G::LGV ? 1 : 0;
    }
    const int64_t span = oe - ob;
    ip.NC = span > 0 ? (int)((span + G::T_ - 1) >> G::LGT) : 0;
    ip.klast = span > 0 ? (int)((((span - 1) + s) >> G::LGT) >= ip.NC + ip.q) : 0;
    if (want_mode == 3 && s <= G::SLIDE_S) ip.mode = 3;  // register slide: w <= SLIDE_S + 1
    ip.front = 0;  // rounds of the advancing front have their own plans (front_plan)
    ip.la = 0;
    ip.gt0 = ob >> G::LGT;
    ip.ok = (s >= 0) && (ip.q + 2 <= kQCap) && span >= 0 && span + s + 2 * (int64_t)G::T_ <= kMaxItemSpan &&
            (want_mode < 0 || want_mode == ip.mode);
    return ip;
}

// Number of loads of one item (see load_tile for their order).
__device__ __forceinline__ int item_loads(int ok, int caseB, int q, int NC, int mode, int klast) {
    if (!ok) return 1;  // a rejected item is one empty stage
    if (mode == 3) return NC;  // register slide: tile c with its halo
    return (caseB ? q : 1) + NC * (caseB ? 2 : 1) - ((NC > 0 && !klast) ? 1 : 0);
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

// Tile index of load l of an item: prologue tiles (caseB ? 1 : 0) .. q, then
// per output tile c the K tile c+q+1 and, for caseB, the J tile c.
// (The last K tile is skipped when no window reaches it: !klast.)
__device__ __forceinline__ int load_tile(int l, int caseB, int q, bool &keep, int mode, int NC, int klast) {
    if (mode == 3) {
        keep = false;
        return l;
    }
    const int pro = caseB ? q : 1;
    if (l < pro) {
        keep = caseB;
        return caseB ? 1 + l : 0;
    }
    const int r = l - pro;
    if (!caseB) {
        keep = false;
        return r + q + 1;
    }
    if (!klast && r == 2 * (NC - 1)) {  // last iteration: J tile only
        keep = false;
        return NC - 1;
    }
    const int c = r >> 1;
    keep = !(r & 1);  // a K tile is read again later as a J tile
    return (r & 1) ? c : c + q + 1;
}

// How one warp's slice [a, a + SLICE) of a tile reaches shared memory:
//   0 (fast)    aligned and inside the series: one bulk copy of the slice;
//   1 (shifted) inside the series, unaligned: one bulk copy of the 16-byte
//               aligned cover (inside the readable buffer), read back at an
//               element shift;
//   2 (direct)  threads load their elements (the cover would leave the buffer);
//   3 (empty)   wholly outside the series: identities, nothing is read;
//   4 (clipped) partly outside the series, cover inside the buffer: as 1, and
//               the readers put identities at positions outside the series.
struct SliceCopy {
    int mode;
    int shift;       // elements (mode 1)
    uintptr_t src;   // first copied byte
    uint32_t bytes;  // copied bytes
};

// HALO extra elements after the slice are copied too (register slide).
// `buf`, `buf_n`: the readable buffer that holds the series.
template <typename T, int HALO>
__device__ __forceinline__ SliceCopy slice_copy(const T *in, int64_t n, int64_t a, const T *buf, int64_t buf_n) {
    using G = Geo<T>;
    constexpr int LEN = G::SLICE + HALO;  // elements; LEN * sizeof(T) is a multiple of 16
    SliceCopy sc;
    sc.mode = 2;
    sc.shift = 0;
    sc.src = 0;
    sc.bytes = 0;
    if (a >= n || a + LEN <= 0) {
        sc.mode = 3;
        return sc;
    }
    const bool inside = a >= 0 && a + LEN <= n;
    const uintptr_t start = (uintptr_t)in + (uintptr_t)(a * (int64_t)sizeof(T));
    const int sb = (int)(start & 15);
    if (inside && sb == 0) {
        sc.mode = 0;
        sc.src = start;
        sc.bytes = (uint32_t)(LEN * sizeof(T));
        return sc;
    }
    const uintptr_t al = start - sb;
    const uintptr_t end = al + (uintptr_t)LEN * sizeof(T) + 16;
    if (al >= (uintptr_t)buf && end <= (uintptr_t)(buf + buf_n)) {
        sc.mode = inside ? 1 : 4;
        sc.shift = sb / (int)sizeof(T);
        sc.src = al;
        sc.bytes = (uint32_t)(LEN * sizeof(T) + 16);
    }
    return sc;
}

// The CTA's item with sequence number seq (or >= n_items at the end).
template <typename T>
__device__ __forceinline__ int64_t item_of(const BlockScanParams &P, int seq) {
    if (P.ticket) return Smem<T>::queue()[seq & (kQueue - 1)];
    return (int64_t)blockIdx.x + (int64_t)seq * gridDim.x;
}

// Copy a warp's slice (plus HALO elements and `extra` bytes) starting at
// global address src into the pieces of stage `dst`, completing on bar.
template <typename T, int HALO>
__device__ __forceinline__ void copy_pieces(uint8_t *dst, uintptr_t src, uint32_t extra, uint64_t *bar,
                                            uint64_t pol) {
    using G = Geo<T>;
    const uint32_t bytes = (uint32_t)((G::PIECE + HALO) * sizeof(T)) + extra;
    if constexpr (kChecked) {
        // The copied bytes must lie inside the launch's readable buffer; a
        // copy that would leave it is skipped (the stage completes empty).
        const BlockScanParams &P = Smem<T>::params();
        const int64_t off = (int64_t)(src - (uintptr_t)P.in);
        if (!in_range(P.status, off, 0, P.in_elems * (int64_t)sizeof(T) - (int64_t)bytes * G::PIECES + 1)) {
            mbar_arrive_expect_tx(bar, 0);
            return;
        }
    }
    mbar_arrive_expect_tx(bar, bytes * G::PIECES);
#pragma unroll
    for (int g = 0; g < G::PIECES; ++g)
        tma_load_1d(dst + g * G::PSTRIDE, reinterpret_cast<const void *>(src + (uintptr_t)g * G::PIECE * sizeof(T)),
                    bytes, bar, pol);
}

// Advancing front, lane 0 of `warp`: issue this warp's slice of its next
// load.  The CTA's work is one sequence of rounds (output tiles t = b, b+G,
// b+2G, ...), four loads each: K tile t+q, K tile t+q+1, J tile t and the
// tile read ahead, t+q+G (a round reads all four even where a window does
// not reach the second or no item takes the fourth, so that the order is
// fixed).  Tile positions are computed directly: no per-round set-up.
template <typename T>
__device__ __forceinline__ void issue_next_front(int warp) {
    using G = Geo<T>;
    using S = Smem<T>;
    WarpIssue &wi = *S::issue(warp);
    if (wi.l >= wi.nloads) return;  // the end (or a starved test launch: nloads = -1)
    const BlockScanParams &P = S::params();
    const int l = wi.l;
    const int k = l & 3;
    const int64_t t = (int64_t)blockIdx.x + (int64_t)(l >> 2) * gridDim.x;
    const int64_t q = wi.q;
    const int64_t x = t + (k == 0 ? q : (k == 1 ? q + 1 : (k == 2 ? 0 : q + (int64_t)gridDim.x)));
    const int64_t a = P.one.d + x * G::T_ + (int64_t)warp * G::SLICE;
    const T *in = reinterpret_cast<const T *>(P.in) + P.one.in_off;
    const SliceCopy sc =
        slice_copy<T, 0>(in, P.one.n, a, reinterpret_cast<const T *>(P.in), P.in_elems);
    const int stage = wi.issued & (kStages - 1);
    uint64_t *bar = S::bar(warp, stage);
    wi.smode[stage] = sc.mode | (sc.shift << 8);
    if (sc.mode == 2 || sc.mode == 3) {
        mbar_arrive_expect_tx(bar, 0);
    } else {
        fence_proxy_async_smem();
        // The J tile is read for the last time; the others are read again soon.
        copy_pieces<T, 0>(S::slice(warp, stage), sc.src, sc.mode == 0 ? 0u : 16u, bar,
                          k == 2 ? policy_evict_first() : policy_evict_last());
    }
    wi.l = l + 1;
    wi.issued++;
}

// Lane 0 of `warp`: issue this warp's slice of its next load, if any.
template <typename T, int MODE, bool FRONT = false>
__device__ __forceinline__ void issue_next(int warp) {
    if constexpr (FRONT) {
        issue_next_front<T>(warp);
        return;
    }
    using G = Geo<T>;
    using S = Smem<T>;
    constexpr int HALO = MODE == 3 ? G::HALO_MAX : 0;
    constexpr int LEN = G::SLICE + HALO;
    WarpIssue &wi = *S::issue(warp);
    {
        // Steady state: the next tile of a linear item, whole and aligned.
        const int l = wi.l;
        if (l < wi.nloads && wi.linear && l >= wi.fast_lo && l < wi.fast_hi) {
            const int stage = wi.issued & (kStages - 1);
            uint64_t *bar = S::bar(warp, stage);
            wi.smode[stage] = wi.fast_smode;
            fence_proxy_async_smem();
            copy_pieces<T, HALO>(S::slice(warp, stage), wi.src0 + (uintptr_t)l * G::T_ * sizeof(T), wi.fast_extra,
                                 bar, policy_evict_first());
            wi.l = l + 1;
            wi.issued++;
            return;
        }
        // Steady state of case B (see load_tile): per output tile c the K tile
        // c+q+1 (read again later as a J tile: kept in L2) and the J tile c.
        if (l < wi.nloads && wi.ok && wi.caseB && l >= wi.q) {
            const int r = l - wi.q;
            const int c = r >> 1;
            const bool kt = !(r & 1);
            const int x = kt ? c + wi.q + 1 : c;
            if ((wi.klast || r != 2 * (wi.NC - 1)) && x >= wi.fast_lo && x < wi.fast_hi) {
                const int stage = wi.issued & (kStages - 1);
                uint64_t *bar = S::bar(warp, stage);
                wi.smode[stage] = wi.fast_smode;
                fence_proxy_async_smem();
                copy_pieces<T, HALO>(S::slice(warp, stage), wi.src0 + (uintptr_t)x * G::T_ * sizeof(T),
                                     wi.fast_extra, bar, kt ? policy_evict_last() : policy_evict_first());
                wi.l = l + 1;
                wi.issued++;
                return;
            }
        }
    }
    if (wi.nloads < 0) return;
    if (wi.l >= wi.nloads) {
        const BlockScanParams &P = S::params();
        do {
            wi.seq++;
            const int64_t item = item_of<T>(P, wi.seq);
            if (item >= P.n_items || item < 0) {
                wi.nloads = -1;
                return;
            }
            ItemPlan<T> ip = make_plan<T>(P, item, MODE);
            if (!ip.ok && warp == 0) report_error(P.status, kErrBadItem);
            const int64_t a0 = ip.p0 + (int64_t)warp * G::SLICE;
            const uintptr_t src0 = (uintptr_t)(ip.in + a0);
            // Tiles whose slice [a, a + LEN) lies inside the series take one
            // copy without checks: from the slice itself if it is 16-byte
            // aligned, else (the same shift for every tile of the item) from
            // 16 bytes below, with 16 bytes more, which stays inside the
            // series when a >= 16 bytes and a + LEN + 16 bytes <= n.
            const int sb = (int)(src0 & 15);
            const int64_t lead = sb ? 16 / (int)sizeof(T) : 0;
            const int64_t lo_a = lead, hi_a = ip.n - LEN - lead;  // range of a
            int64_t flo = a0 >= lo_a ? 0 : (lo_a - a0 + G::T_ - 1) / G::T_;
            int64_t fhi = hi_a - a0 >= 0 ? (hi_a - a0) / G::T_ + 1 : 0;
            if (fhi < flo) fhi = flo;
            wi.src0 = src0 - sb;
            wi.fast_smode = sb ? 1 | ((sb / (int)sizeof(T)) << 8) : 0;
            wi.fast_extra = sb ? 16 : 0;
            wi.fast_lo = (int)flo;
            wi.fast_hi = (int)(fhi > 0x7fffffff ? 0x7fffffff : fhi);
            wi.in = ip.in;
            wi.n = ip.n;
            wi.p0 = ip.p0;
            wi.q = ip.q;
            wi.caseB = ip.caseB;
            wi.ok = ip.ok;
            wi.NC = ip.NC;
            wi.klast = ip.klast;
            wi.nloads = item_loads(ip.ok, ip.caseB, ip.q, ip.NC, MODE, ip.klast);
            wi.linear = ip.ok && (MODE == 3 || !ip.caseB);
            wi.l = 0;
        } while (wi.l >= wi.nloads);
    }
    const int stage = wi.issued & (kStages - 1);
    uint64_t *bar = S::bar(warp, stage);
    int smode = 2;
    if (wi.ok) {
        bool keep = false;
        const int x = load_tile(wi.l, wi.caseB, wi.q, keep, MODE, wi.NC, wi.klast);
        const uint64_t pol = keep ? policy_evict_last() : policy_evict_first();
        if (x >= wi.fast_lo && x < wi.fast_hi) {
            smode = wi.fast_smode;
            wi.smode[stage] = smode;
            fence_proxy_async_smem();
            copy_pieces<T, HALO>(S::slice(warp, stage), wi.src0 + (uintptr_t)x * G::T_ * sizeof(T), wi.fast_extra,
                                 bar, pol);
        } else {
            const int64_t a = wi.p0 + (int64_t)x * G::T_ + (int64_t)warp * G::SLICE;
            const BlockScanParams &PP = S::params();
            const SliceCopy sc = slice_copy<T, HALO>(reinterpret_cast<const T *>(wi.in), wi.n, a,
                                                     reinterpret_cast<const T *>(PP.in), PP.in_elems);
            smode = sc.mode | (sc.shift << 8);
            wi.smode[stage] = smode;
            if (sc.mode != 2 && sc.mode != 3) {
                fence_proxy_async_smem();
                copy_pieces<T, HALO>(S::slice(warp, stage), sc.src, 16, bar, pol);
            }
        }
    } else {
        wi.smode[stage] = 2;
    }
    if ((smode & 0xff) == 2 || (smode & 0xff) == 3) mbar_arrive_expect_tx(bar, 0);
    wi.l++;
    wi.issued++;
}

// Sliding maximum/minimum of the tile aggregates of tiles [c+1, c+q-1] (case
// B), kept by warp 0 as a two-stack queue inside the tile-aggregate ring:
// slots [fs, fe) hold suffix maxima up to fe-1, slots [fe, be) raw aggregates
// whose running max is (bm, bn).  Each step costs O(1) amortised.  Every
// lane of warp 0 runs it; the rebuild is a warp scan (lane l takes slot
// top - l of each group of 32, newest first), the rest is the same on every
// lane.
template <typename T> struct TileQueue {
    using R = typename Elem<T>::R;
    using Pair = typename Elem<T>::Pair;
    int fs = 1, fe = 1, be = 1;
    R bm = Elem<T>::lo(), bn = Elem<T>::hi();
    __device__ static Pair &ta(int x) { return Smem<T>::ta()[x % kQCap]; }
    __device__ void push(int x) {
        const Pair a = ta(x);
        bm = vmax(bm, Elem<T>::pmax(a));
        bn = vmin(bn, Elem<T>::pmin(a));
        be = x + 1;
    }
    // Drop the oldest tile, add tile x; rebuild the older part (in place, as
    // suffix maxima of what the newer part holds) when it runs empty.
    __device__ void slide(int x) {
        ++fs;
        push(x);
        if (fs >= fe) {
            const int lane = threadIdx.x & 31;
            R cm = Elem<T>::lo(), cn = Elem<T>::hi();  // slots above the group
            for (int top = be - 1; top >= fs; top -= 32) {
                const int xl = top - lane;
                R m = Elem<T>::lo(), n = Elem<T>::hi();
                if (xl >= fs) {
                    const Pair a = ta(xl);
                    m = Elem<T>::pmax(a);
                    n = Elem<T>::pmin(a);
                }
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const R um = __shfl_up_sync(0xffffffffu, m, d), un = __shfl_up_sync(0xffffffffu, n, d);
                    if (lane >= d) {
                        m = vmax(m, um);
                        n = vmin(n, un);
                    }
                }
                m = vmax(m, cm);
                n = vmin(n, cn);
                if (xl >= fs) ta(xl) = Elem<T>::pair(m, n);
                cm = __shfl_sync(0xffffffffu, m, 31);
                cn = __shfl_sync(0xffffffffu, n, 31);
            }
            __syncwarp();
            bm = Elem<T>::lo();
            bn = Elem<T>::hi();
            fe = be;
        }
    }
    __device__ Pair query() const {
        R m = bm, n = bn;
        if (fs < fe) {
            const Pair f = ta(fs);
            m = vmax(m, Elem<T>::pmax(f));
            n = vmin(n, Elem<T>::pmin(f));
        }
        return Elem<T>::pair(m, n);
    }
};

// Published tile aggregates of the advancing front: global tile g owns two
// 64-bit words, (max bits | tag << 32) and (min bits | tag << 32), tag =
// g + 1 (the workspace starts zeroed: no tag).  Each word is stored and
// loaded whole (single-copy atomic), so a reader that finds the tag in both
// words has both values; no fence is needed, and writers of one slot store
// identical words.  Element types whose register form is 32 bits only.
__device__ __forceinline__ uint32_t rbits(float v) { return __float_as_uint(v); }
__device__ __forceinline__ uint32_t rbits(int v) { return (uint32_t)v; }
__device__ __forceinline__ void rfrom(uint32_t b, float &v) { v = __uint_as_float(b); }
__device__ __forceinline__ void rfrom(uint32_t b, int &v) { v = (int)b; }
template <typename T>
__device__ __forceinline__ void front_put(unsigned long long *slot, uint32_t tag, typename Elem<T>::R m,
                                          typename Elem<T>::R n) {
    const unsigned long long a = ((unsigned long long)tag << 32) | rbits(m);
    const unsigned long long b = ((unsigned long long)tag << 32) | rbits(n);
    asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(slot), "l"(a), "l"(b) : "memory");
}
template <typename T>
__device__ __forceinline__ bool front_get(const unsigned long long *slot, uint32_t tag, typename Elem<T>::R &m,
                                          typename Elem<T>::R &n) {
    unsigned long long a, b;
    asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(slot) : "memory");
    if ((uint32_t)(a >> 32) != tag || (uint32_t)(b >> 32) != tag) return false;
    rfrom((uint32_t)a, m);
    rfrom((uint32_t)b, n);
    return true;
}

// ------------------------------------------------------------ consumer side
// Block modes of an item (s = w-1, warp span W = 32V):
//   0: s < V      B = 2^floor(log2 s) < V: blocks inside a thread
//   1: s < W      B = 2^floor(log2 s) in [V, W/2]: blocks of 2..16 lanes
//   2: s >= W     B = W: one block per warp; for s >= T also tile aggregates
// LB: the output stage feeds the envelope lower bound instead of storing
// (a separate instantiation, so the storing kernels carry none of it).
template <typename T, int KMODE, bool LB = false, bool FRONT = false>
struct Consumer {
    using R = typename Elem<T>::R;
    using Pair = typename Elem<T>::Pair;
    using G = Geo<T>;
    using S = Smem<T>;
    static constexpr int V = G::V;
    static constexpr int T_ = G::T_;
    static constexpr int NW = G::NW;

    int tid, lane, warp;
    StageCursor cur;
    bool failed = false;         // a wait of this thread ran out
    long long wait_limit = kWaitLimitCycles;

    // CTA barrier (the P ring and block aggregates are shared by all warps).
    // A warp whose wait ran out still takes every barrier of its work item
    // (it goes on with identities, without waiting or issuing copies), so no
    // warp is ever left waiting for one that left; all warps leave together
    // at the item boundary, whose barrier ORs their failure flags.
    __device__ __forceinline__ void sync() { named_bar_sync(1, G::NT); }

    // Bounded wait of this thread for the warp's current stage.  A thread
    // whose wait has run out waits no more (its failure flag stays set and is
    // reported once in the status word); nothing else depends on whether the
    // lanes of a warp agree, since every lane carries on through the item
    // and the flags meet at the item boundary's OR barrier.
    __device__ __forceinline__ bool wait_stage() {
        if (mbar_try_wait(S::bar(warp, cur.stage), cur.phase)) return true;
        const bool ok = !failed && mbar_wait_bounded(S::bar(warp, cur.stage), cur.phase, wait_limit);
        if (!ok && !failed) {
            report_error(S::params().status, kErrWaitTimeout);
            failed = true;
        }
        return ok;
    }

    // Before leaving after a failure: wait (bounded) for the copies this warp
    // still has in flight, so that none lands after the CTA has exited.
    __device__ __forceinline__ void drain() {
        if (lane == 0) {
            StageCursor c = cur;
            // Loads issued but not read, from the issue count and the cursor
            // (both modulo 2 kStages; at most kStages apart).
            const int outstanding =
                (S::issue(warp)->issued - (int)(cur.phase * kStages + cur.stage)) & (2 * kStages - 1);
            for (int k = 0; k < outstanding && k < kStages; ++k) {
                if (!mbar_wait_bounded(S::bar(warp, c.stage), c.phase, wait_limit)) break;
                c.advance();
            }
        }
        __syncwarp();
    }

    // Identities at this thread's positions of tile x that lie outside the
    // series [0, n) (clipped copies).
    template <int NE>
    __device__ __forceinline__ void clip(const ItemPlan<T> &ip, int x, int, R (&xm)[NE], R (&xn)[NE]) const {
        const int64_t pt = ip.p0 + (int64_t)x * T_ + (int64_t)warp * G::SLICE + (int64_t)lane * V;
        const int64_t lo = -pt, hi = ip.n - pt;  // valid element indices: [lo, hi)
#pragma unroll
        for (int i = 0; i < NE; ++i) {
            if (i < lo || i >= hi) {
                xm[i] = Elem<T>::lo();
                xn[i] = Elem<T>::hi();
            }
        }
    }

    // This lane's first NWD words (16-byte chunks from its element base) of
    // a slice stage.  16-byte reads are served eight lanes at a time; lanes
    // V*sz bytes apart reading the same chunk index would share banks, so
    // each group of NCH chunks (lane+g's elements) is read starting at chunk
    // rot = ((lane+g) / (8/NCH)) mod NCH, which spreads each group of eight
    // lanes over all banks, and a barrel shift restores the order.
    template <int NWD>
    __device__ __forceinline__ void read_words(const uint8_t *sb, uint32_t *wd) const {
        const uint4 *p4 = reinterpret_cast<const uint4 *>(S::lane_base(sb, lane));
        if constexpr ((G::NCH == 2 || G::NCH == 4) && (NWD / 4) % G::NCH == 0) {
            constexpr int NC = G::NCH;
#pragma unroll
            for (int g = 0; g < NWD / 4 / NC; ++g) {
                const int rot = ((lane + g) / (8 / NC)) & (NC - 1);
                uint4 u[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) u[c] = p4[g * NC + ((c + rot) & (NC - 1))];
                // u[c] holds chunk (c + rot) mod NC: rotate right by rot.
#pragma unroll
                for (int b = 1; b < NC; b <<= 1) {
                    if (rot & b) {
                        uint4 t[NC];
#pragma unroll
                        for (int c = 0; c < NC; ++c) t[c] = u[(c - b + NC) & (NC - 1)];
#pragma unroll
                        for (int c = 0; c < NC; ++c) u[c] = t[c];
                    }
                }
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int k = g * NC + c;
                    wd[4 * k] = u[c].x; wd[4 * k + 1] = u[c].y; wd[4 * k + 2] = u[c].z; wd[4 * k + 3] = u[c].w;
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < NWD / 4; ++c) {
                const uint4 v = p4[c];
                wd[4 * c] = v.x; wd[4 * c + 1] = v.y; wd[4 * c + 2] = v.z; wd[4 * c + 3] = v.w;
            }
        }
    }
    // The 16 bytes that follow this lane's first NWD words (inside the stage:
    // shifted copies carry 16 bytes past the slice and its halo).
    __device__ __forceinline__ void read_tail(const uint8_t *sb, int nwd, uint32_t *wd) const {
        static_assert(G::PIECES == 1, "one piece per slice: lane data is contiguous");
        const uint4 v = reinterpret_cast<const uint4 *>(S::lane_base(sb, lane))[nwd / 4];
        wd[0] = v.x; wd[1] = v.y; wd[2] = v.z; wd[3] = v.w;
    }

    // Read this thread's V elements of input tile x of the item from the
    // warp's slice stage, then let lane 0 refill the stage with the warp's
    // next load.  Max-side and min-side copies differ only at positions
    // outside [0, n), which hold identities.
    // After a failed wait the thread reads whatever the stage holds (every
    // read stays inside the stage or the series; leaving the values unset
    // instead would push the arrays to local memory) and the caller carries
    // on through the item, whose outputs are then unspecified.  The refill is
    // issued either way: a copy issued after a failure is an ordinary copy
    // that lands, and the item boundary waits for every copy still in flight
    // before the CTA leaves.
    __device__ __forceinline__ bool read_tile(const ItemPlan<T> &ip, int x, R (&xm)[V], R (&xn)[V]) {
        const bool ok = wait_stage();
        const int smode = S::issue(warp)->smode[cur.stage];
        const int mode = smode & 0xff;
        const uint8_t *sb = S::slice(warp, cur.stage);
        if (mode == 0) {
            uint32_t wd[4 * G::NCH];
            read_words<4 * G::NCH>(sb, wd);
            R xv[V];
            ExtractLoop<T, 0, 0, V>::run(wd, xv);
#pragma unroll
            for (int i = 0; i < V; ++i) xm[i] = xn[i] = xv[i];
        } else if (mode == 1 || mode == 4) {
            // The slice starts smode >> 8 elements (under 16 bytes) into the
            // stage: this lane's words, then the next 16 bytes, shifted.
            uint32_t wd[4 * G::NCH + 4];
            read_words<4 * G::NCH>(sb, wd);
            read_tail(sb, 4 * G::NCH, wd + 4 * G::NCH);
            shift_bytes<4 * G::NCH>(wd, (smode >> 8) * (int)sizeof(T));
            R xv[V];
            ExtractLoop<T, 0, 0, V>::run(wd, xv);
#pragma unroll
            for (int i = 0; i < V; ++i) xm[i] = xn[i] = xv[i];
            if (mode == 4) clip(ip, x, V, xm, xn);
        } else if (mode == 3) {
#pragma unroll
            for (int i = 0; i < V; ++i) {
                xm[i] = Elem<T>::lo();
                xn[i] = Elem<T>::hi();
            }
        } else {
            const int64_t pt = ip.p0 + (int64_t)x * T_ + (int64_t)warp * G::SLICE + (int64_t)lane * V;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const int64_t p = pt + i;
                if (p < 0 || p >= ip.n ||
                    !in_range(S::params().status, (ip.in - reinterpret_cast<const T *>(S::params().in)) + p, 0,
                              S::params().in_elems)) {
                    xm[i] = Elem<T>::lo();
                    xn[i] = Elem<T>::hi();
                } else {
                    xm[i] = xn[i] = Elem<T>::load(ip.in[p]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) issue_next<T, KMODE, FRONT>(warp);
        __syncwarp();
        cur.advance();
        return ok;
    }

    template <int MODE>
    __device__ __forceinline__ void local_prefix(R (&m)[V], R (&n)[V], int lgB) const {
        if constexpr (MODE > 0) {
#pragma unroll
            for (int i = 1; i < V; ++i) { m[i] = vmax(m[i - 1], m[i]); n[i] = vmin(n[i - 1], n[i]); }
        } else {
            const int bmask = (1 << lgB) - 1;
#pragma unroll
            for (int i = 1; i < V; ++i)
                if (i & bmask) { m[i] = vmax(m[i - 1], m[i]); n[i] = vmin(n[i - 1], n[i]); }
        }
    }
    template <int MODE>
    __device__ __forceinline__ void local_suffix(R (&m)[V], R (&n)[V], int lgB) const {
        if constexpr (MODE > 0) {
#pragma unroll
            for (int i = V - 2; i >= 0; --i) { m[i] = vmax(m[i + 1], m[i]); n[i] = vmin(n[i + 1], n[i]); }
        } else {
            const int bmask = (1 << lgB) - 1;
#pragma unroll
            for (int i = V - 2; i >= 0; --i)
                if ((i + 1) & bmask) { m[i] = vmax(m[i + 1], m[i]); n[i] = vmin(n[i + 1], n[i]); }
        }
    }

    // Block-segmented carries across the lanes of a block of 2^lgS lanes
    // (1 <= lgS <= 5): dir 0 applies the exclusive prefix from lower lanes,
    // dir 1 the exclusive suffix from higher lanes.  Returns the inclusive
    // total of the block (valid in the block's last / first lane).
    __device__ __forceinline__ void lane_carry(int dir, R (&m)[V], R (&n)[V], int lgS, R &tot_m, R &tot_n) const {
        const int segl = 1 << lgS;
        const int lis = lane & (segl - 1);
        const int pos = dir == 0 ? lis : (segl - 1 - lis);
        R tm = dir == 0 ? m[V - 1] : m[0];
        R tn = dir == 0 ? n[V - 1] : n[0];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            if (d >= segl) break;
            R om = dir == 0 ? __shfl_up_sync(0xffffffffu, tm, d) : __shfl_down_sync(0xffffffffu, tm, d);
            R on = dir == 0 ? __shfl_up_sync(0xffffffffu, tn, d) : __shfl_down_sync(0xffffffffu, tn, d);
            if (pos >= d) { tm = vmax(tm, om); tn = vmin(tn, on); }
        }
        R em = dir == 0 ? __shfl_up_sync(0xffffffffu, tm, 1) : __shfl_down_sync(0xffffffffu, tm, 1);
        R en = dir == 0 ? __shfl_up_sync(0xffffffffu, tn, 1) : __shfl_down_sync(0xffffffffu, tn, 1);
        if (pos != 0) {
#pragma unroll
            for (int i = 0; i < V; ++i) { m[i] = vmax(m[i], em); n[i] = vmin(n[i], en); }
        }
        tot_m = tm;
        tot_n = tn;
    }

    __device__ __forceinline__ void ring_write(int x, const R (&pm)[V], const R (&pn)[V]) {
        const int base = (x % 3) * T_ + tid * V;
        Pair *r = S::ring() + base + (base >> G::PS);
#pragma unroll
        for (int i = 0; i < V; ++i) r[i] = Elem<T>::pair(pm[i], pn[i]);
    }

    // Ring slot index of relative position p (p >= 0).
    __device__ __forceinline__ int ring_index(int p) const { return ((p >> G::LGT) % 3) * T_ + (p & (T_ - 1)); }
    __device__ __forceinline__ Pair ring_at(int idx) const { return S::ring()[idx + (idx >> G::PS)]; }

    // Tile aggregates c+1 .. c+q-1, reduced across the warp.
    __device__ __forceinline__ void tiles_between(int c, int q, R &m1, R &n1) const {
        m1 = Elem<T>::lo();
        n1 = Elem<T>::hi();
        for (int x = c + 1 + lane; x <= c + q - 1; x += 32) {
            const Pair pr = S::ta()[x % kQCap];
            m1 = vmax(m1, Elem<T>::pmax(pr));
            n1 = vmin(n1, Elem<T>::pmin(pr));
        }
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) {
            m1 = vmax(m1, __shfl_xor_sync(0xffffffffu, m1, d));
            n1 = vmin(n1, __shfl_xor_sync(0xffffffffu, n1, d));
        }
    }

    // Outputs of output tile c: max(S_B[j], blocks between, P_B[j+s]).
    template <int MODE>
    __device__ __forceinline__ void outputs(const ItemPlan<T> &ip, int c, const R (&sm)[V], const R (&sn)[V]) {
        const int lgB = ip.lgB;
        const int jr0 = c * T_ + tid * V;
        const int kr0 = jr0 + ip.s;
        // Ring addresses of kr0 .. kr0+V-1: one padding step and at most one
        // wrap of the 3-tile ring, both at the same 2^PS boundary.
        const int p = ring_index(kr0);
        const int phys = p + (p >> G::PS);
        const int cpad = (1 << G::PS) - (p & ((1 << G::PS) - 1));
        const int hi_base = (p + cpad == G::RING) ? -cpad : phys + 1;
        R om[V], on[V];
        if constexpr (MODE == 2) {
            // Lane array of block aggregates in window order: case A lanes 0..15
            // = warp blocks of tiles c, c+1; case B lanes 0..7 = J tile c,
            // 8..15 = K tile c+q, 16..23 = K tile c+q+1.  Prefix from the block
            // after j's (lane warp+1); for case B the full tiles c+1..c+q-1
            // join every lane from 7 on.
            const int q = ip.q;
            Pair a;
            if (!ip.caseB) {
                a = lane < NW ? S::kagg()[(c % 3) * NW + lane]
                              : (lane < 2 * NW ? S::kagg()[((c + 1) % 3) * NW + lane - NW]
                                               : Elem<T>::pair(Elem<T>::lo(), Elem<T>::hi()));
            } else {
                a = lane < NW ? S::jagg()[(c & 1) * NW + lane]
                              : (lane < 2 * NW ? S::kagg()[((c + q) % 3) * NW + lane - NW]
                                               : (lane < 3 * NW ? S::kagg()[((c + q + 1) % 3) * NW + lane - 2 * NW]
                                                                : Elem<T>::pair(Elem<T>::lo(), Elem<T>::hi())));
            }
            R am = lane > warp ? Elem<T>::pmax(a) : Elem<T>::lo();
            R an = lane > warp ? Elem<T>::pmin(a) : Elem<T>::hi();
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                R um = __shfl_up_sync(0xffffffffu, am, d);
                R un = __shfl_up_sync(0xffffffffu, an, d);
                if (lane >= d) { am = vmax(am, um); an = vmin(an, un); }
            }
            if (ip.caseB) {
                R tm, tn;
                tiles_between(c, q, tm, tn);
                if (lane >= NW - 1) { am = vmax(am, tm); an = vmin(an, tn); }
            }
            // Lane of k0's block; outputs i >= cross have k in the next block.
            const int kb = kr0 >> lgB;
            const int g0 = ip.caseB ? kb - (c + q) * NW + NW : kb - c * NW;
            const int cross = ((kb + 1) << lgB) - kr0;
            const R c0m = __shfl_sync(0xffffffffu, am, g0 - 1), c0n = __shfl_sync(0xffffffffu, an, g0 - 1);
            const R c1m = __shfl_sync(0xffffffffu, am, g0), c1n = __shfl_sync(0xffffffffu, an, g0);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const Pair pr = S::ring()[(i < cpad ? phys : hi_base) + i];
                const bool far = i >= cross;
                om[i] = vmax(vmax(sm[i], far ? c1m : c0m), Elem<T>::pmax(pr));
                on[i] = vmin(vmin(sn[i], far ? c1n : c0n), Elem<T>::pmin(pr));
            }
        } else if constexpr (MODE == 1) {
            const int bj = jr0 >> lgB;
            const int bend = ((bj + 2) << lgB) - 1;  // last position of block bj+1
            const int cross = bend + 1 - kr0;         // i >= cross: k in block bj+2
            R mm = Elem<T>::lo(), mn = Elem<T>::hi();
            if (cross < V) {
                int idx = p + (bend - kr0);
                if (idx < 0) idx += G::RING;
                const Pair pr = ring_at(idx);
                mm = Elem<T>::pmax(pr);
                mn = Elem<T>::pmin(pr);
            }
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const Pair pr = S::ring()[(i < cpad ? phys : hi_base) + i];
                const bool far = i >= cross;
                om[i] = vmax(vmax(sm[i], far ? mm : Elem<T>::lo()), Elem<T>::pmax(pr));
                on[i] = vmin(vmin(sn[i], far ? mn : Elem<T>::hi()), Elem<T>::pmin(pr));
            }
        } else {
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const Pair pr = S::ring()[(i < cpad ? phys : hi_base) + i];
                R vm = vmax(sm[i], Elem<T>::pmax(pr));
                R vn = vmin(sn[i], Elem<T>::pmin(pr));
                const int bj = (jr0 + i) >> lgB, bk = (kr0 + i) >> lgB;
                if (bk == bj + 2) {
                    int idx = p + ((bk << lgB) - 1 - kr0);
                    if (idx < 0) idx += G::RING;
                    if (idx >= G::RING) idx -= G::RING;
                    const Pair pm = ring_at(idx);
                    vm = vmax(vm, Elem<T>::pmax(pm));
                    vn = vmin(vn, Elem<T>::pmin(pm));
                }
                om[i] = vm;
                on[i] = vn;
            }
        }
        store_out(ip, ip.o_begin + jr0, om, on, out_vec(ip));
    }

    // Output alignment of the item (outputs of a thread start V elements
    // apart): 2 = 32-byte, 1 = 16-byte, 0 = neither (same for every thread).
    __device__ __forceinline__ int out_vec(const ItemPlan<T> &ip) const {
        const uintptr_t oa = (ip.omax ? (uintptr_t)(ip.omax + ip.o_begin) : 0) |
                             (ip.omin ? (uintptr_t)(ip.omin + ip.o_begin) : 0);
        return (oa & 31) == 0 ? 2 : ((oa & 15) == 0 ? 1 : 0);
    }

    // Stores this thread's outputs o0 .. o0+V-1 of the item (those before
    // o_end).  Every lane of the warp calls it (vec from out_vec).
    __device__ __forceinline__ void store_out(const ItemPlan<T> &ip, int64_t o0, const R (&om)[V], const R (&on)[V],
                                              int vec) const {
        if constexpr (LB) {
            lb_out(ip, o0, om, on);
            return;
        }
        const bool full = o0 + V <= ip.o_end;
        const bool wfull = __all_sync(0xffffffffu, full);
        if (vec && full) {
            if constexpr (G::NCH % 2 == 0) {
                if (vec == 2) {
                    if (ip.omax) store_v8(ip.omax + o0, om);
                    if (ip.omin) store_v8(ip.omin + o0, on);
                    return;
                }
            }
            if (ip.omax) store_vec(ip.omax + o0, om);
            if (ip.omin) store_vec(ip.omin + o0, on);
        } else if (!vec && wfull) {
            if (ip.omax) store_shifted(ip.omax + o0, om);
            if (ip.omin) store_shifted(ip.omin + o0, on);
        } else if (o0 < ip.o_end) {
            const int cnt = full ? V : (int)(ip.o_end - o0);
            if (ip.omax) store(ip.omax + o0, om, cnt);
            if (ip.omin) store(ip.omin + o0, on, cnt);
        }
    }

    // Envelope lower bound: this thread's outputs o0 .. o0+V-1 (before o_end)
    // are the upper and lower envelope at series positions o0 + i; the
    // squared excursions of the query there are summed over the warp and
    // added to the series' accumulator (one atomic per warp and tile).
    __device__ __forceinline__ void lb_out(const ItemPlan<T> &ip, int64_t o0, const R (&om)[V],
                                           const R (&on)[V]) const {
        using A = typename LbAcc<T>::A;
        const T *q = reinterpret_cast<const T *>(S::params().lb_query) + o0;
        A part = A(0);
        if (o0 + V <= ip.o_end && (((uintptr_t)q) & 15) == 0) {
            // A whole run with an aligned query: 16-byte loads.
            T qv[V];
#pragma unroll
            for (int c = 0; c < V * (int)sizeof(T) / 16; ++c)
                reinterpret_cast<uint4 *>(qv)[c] = __ldg(reinterpret_cast<const uint4 *>(q) + c);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const A qi = (A)qv[i];
                const A u = (A)Elem<T>::store(om[i]), l = (A)Elem<T>::store(on[i]);
                const A d = qi > u ? qi - u : (qi < l ? l - qi : A(0));
                part += d * d;
            }
        } else {
#pragma unroll
            for (int i = 0; i < V; ++i) {
                if (o0 + i < ip.o_end) {
                    const A qi = (A)__ldg(q + i);
                    const A u = (A)Elem<T>::store(om[i]), l = (A)Elem<T>::store(on[i]);
                    const A d = qi > u ? qi - u : (qi < l ? l - qi : A(0));
                    part += d * d;
                }
            }
        }
#pragma unroll
        for (int k = 16; k >= 1; k >>= 1) part += __shfl_xor_sync(0xffffffffu, part, k);
        if (lane == 0 && part != A(0)) atomicAdd(ip.lb_acc + ip.series, (double)part);
    }

    // A whole warp span of outputs (every lane V values at dst, lanes V
    // elements apart) whose start is not 16-byte aligned: the warp moves its
    // values down by d elements (d: from dst to the next 16-byte boundary,
    // the same for every lane), so that each lane stores whole aligned
    // 16-byte chunks; lane 0 stores its first d values singly and lane 31
    // its last A - d (its last chunk would reach into the next warp's span).
    __device__ __forceinline__ void store_shifted(T *dst, const R (&v)[V]) const {
        constexpr int A = 16 / (int)sizeof(T);  // elements per chunk
        constexpr int NWD = 4 * G::NCH;
        const int d = (int)((16 - ((uintptr_t)dst & 15)) & 15) / (int)sizeof(T);
        uint32_t wd[NWD + 4];
#pragma unroll
        for (int k = 0; k < NWD; ++k) wd[k] = pack_word<T>(v, k);
#pragma unroll
        for (int k = 0; k < 4; ++k) wd[NWD + k] = __shfl_down_sync(0xffffffffu, wd[k], 1);
        shift_bytes<NWD>(wd, d * (int)sizeof(T));
        uint4 *p = reinterpret_cast<uint4 *>(dst + d);
#pragma unroll
        for (int c = 0; c < G::NCH; ++c)
            if (c < G::NCH - 1 || lane != 31 || d == 0)
                __stcs(p + c, make_uint4(wd[4 * c], wd[4 * c + 1], wd[4 * c + 2], wd[4 * c + 3]));
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < A - 1; ++i)
                if (i < d) dst[i] = Elem<T>::store(v[i]);
        }
        if (lane == 31 && d) {
#pragma unroll
            for (int i = V - A + 1; i < V; ++i)
                if (i >= V - A + d) dst[i] = Elem<T>::store(v[i]);
        }
    }

    __device__ __forceinline__ void store(T *dst, const R (&v)[V], int cnt) const {
        if constexpr (G::NCH % 2 == 0) {
            if (cnt == V && (((uintptr_t)dst) & 31) == 0) {
                store_v8(dst, v);
                return;
            }
        }
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
                if (i < cnt) dst[i] = Elem<T>::store(v[i]);
        }
    }

    // Tile aggregate of K tile x from its warp-block aggregates (warp `by`),
    // into the aggregate ring.
    __device__ __forceinline__ void publish_tile_aggregate(int x, int by = 0) const {
        if (warp != by) return;
        Pair a = lane < NW ? S::kagg()[(x % 3) * NW + lane] : Elem<T>::pair(Elem<T>::lo(), Elem<T>::hi());
        R m = Elem<T>::pmax(a), n = Elem<T>::pmin(a);
#pragma unroll
        for (int d = NW / 2; d >= 1; d >>= 1) {
            m = vmax(m, __shfl_xor_sync(0xffffffffu, m, d));
            n = vmin(n, __shfl_xor_sync(0xffffffffu, n, d));
        }
        if (lane == 0) S::ta()[x % kQCap] = Elem<T>::pair(m, n);
    }


    // Prefix (and optionally suffix) block scans of one tile's registers.
    // MODE 2 publishes the warp (= block) totals.
    template <int MODE>
    __device__ __forceinline__ void scan_tile(const ItemPlan<T> &ip, R (&pm)[V], R (&pn)[V], bool suf, R (&sm)[V],
                                              R (&sn)[V], int kslot, int jbuf, bool pre = true) {
        const int lgB = ip.lgB;
        if (pre) local_prefix<MODE>(pm, pn, lgB);
        if (suf) local_suffix<MODE>(sm, sn, lgB);
        if constexpr (MODE > 0) {
            const int lgS = lgB - G::LGV;
            if (lgS > 0) {
                R tm, tn;
                if (pre) {
                    lane_carry(0, pm, pn, lgS, tm, tn);
                    if (MODE == 2 && lane == 31) S::kagg()[kslot * NW + warp] = Elem<T>::pair(tm, tn);
                }
                if (suf) {
                    lane_carry(1, sm, sn, lgS, tm, tn);
                    if (MODE == 2 && jbuf >= 0 && lane == 0) S::jagg()[jbuf * NW + warp] = Elem<T>::pair(tm, tn);
                }
            }
        }
    }

    // ------------------------------------- modes 1 and 2: thread-local scans
    // The window [j, j+s] splits into (a) the rest of j's V-element thread
    // block, (b) the later thread blocks of j's scan block, (c) the whole scan
    // blocks in between, (d) the earlier thread blocks of k's scan block and
    // (e) the start of k's thread block up to k = j+s.  (a) and (e) are scans
    // local to one thread; (b) and (d) are one lane carry per thread (f and e
    // below), (c) one aggregate per thread and side of k.  So every output is
    // max(local suffix, per-thread constant, local prefix from the ring).

    // K role: local prefix of the thread's elements; lane carries within the
    // scan block of 2^lgS lanes: e (exclusive) and g (inclusive).
    __device__ __forceinline__ void scan_k(int lgS, const R (&xm)[V], const R (&xn)[V], R (&pm)[V], R (&pn)[V],
                                           R &em, R &en, R &gm, R &gn) const {
        pm[0] = xm[0];
        pn[0] = xn[0];
#pragma unroll
        for (int i = 1; i < V; ++i) { pm[i] = vmax(pm[i - 1], xm[i]); pn[i] = vmin(pn[i - 1], xn[i]); }
        const int segl = 1 << lgS;
        const int pos = lane & (segl - 1);
        R tm = pm[V - 1], tn = pn[V - 1];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            if (d >= segl) break;
            const R um = __shfl_up_sync(0xffffffffu, tm, d);
            const R un = __shfl_up_sync(0xffffffffu, tn, d);
            if (pos >= d) { tm = vmax(tm, um); tn = vmin(tn, un); }
        }
        gm = tm;
        gn = tn;
        const R xm1 = __shfl_up_sync(0xffffffffu, tm, 1);
        const R xn1 = __shfl_up_sync(0xffffffffu, tn, 1);
        em = pos ? xm1 : Elem<T>::lo();
        en = pos ? xn1 : Elem<T>::hi();
    }

    // J role: local suffix; lane carry f (exclusive suffix within the scan
    // block) and h (inclusive: at the block's first lane, the block aggregate).
    __device__ __forceinline__ void scan_j(int lgS, const R (&xm)[V], const R (&xn)[V], R (&sm)[V], R (&sn)[V],
                                           R &fm, R &fn, R &hm, R &hn) const {
        sm[V - 1] = xm[V - 1];
        sn[V - 1] = xn[V - 1];
#pragma unroll
        for (int i = V - 2; i >= 0; --i) { sm[i] = vmax(sm[i + 1], xm[i]); sn[i] = vmin(sn[i + 1], xn[i]); }
        const int segl = 1 << lgS;
        const int pos = (segl - 1) - (lane & (segl - 1));
        R tm = sm[0], tn = sn[0];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            if (d >= segl) break;
            const R um = __shfl_down_sync(0xffffffffu, tm, d);
            const R un = __shfl_down_sync(0xffffffffu, tn, d);
            if (pos >= d) { tm = vmax(tm, um); tn = vmin(tn, un); }
        }
        hm = tm;
        hn = tn;
        const R xm1 = __shfl_down_sync(0xffffffffu, tm, 1);
        const R xn1 = __shfl_down_sync(0xffffffffu, tn, 1);
        fm = pos ? xm1 : Elem<T>::lo();
        fn = pos ? xn1 : Elem<T>::hi();
    }

    // Both roles at once (independent chains interleave): K role on km/kn,
    // J role on jm/jn (the same tile in case A).
    __device__ __forceinline__ void scan_kj(int lgS, const R (&km)[V], const R (&kn)[V], const R (&jm)[V],
                                            const R (&jn)[V], R (&pm)[V], R (&pn)[V], R &em, R &en, R &gm, R &gn,
                                            R (&sm)[V], R (&sn)[V], R &fm, R &fn, R &hm, R &hn) const {
        pm[0] = km[0];
        pn[0] = kn[0];
        sm[V - 1] = jm[V - 1];
        sn[V - 1] = jn[V - 1];
#pragma unroll
        for (int i = 1; i < V; ++i) {
            pm[i] = vmax(pm[i - 1], km[i]);
            pn[i] = vmin(pn[i - 1], kn[i]);
            sm[V - 1 - i] = vmax(sm[V - i], jm[V - 1 - i]);
            sn[V - 1 - i] = vmin(sn[V - i], jn[V - 1 - i]);
        }
        const int segl = 1 << lgS;
        const int posk = lane & (segl - 1), posj = (segl - 1) - posk;
        R am = pm[V - 1], an = pn[V - 1], bm = sm[0], bn = sn[0];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            if (d >= segl) break;
            const R uam = __shfl_up_sync(0xffffffffu, am, d);
            const R uan = __shfl_up_sync(0xffffffffu, an, d);
            const R ubm = __shfl_down_sync(0xffffffffu, bm, d);
            const R ubn = __shfl_down_sync(0xffffffffu, bn, d);
            if (posk >= d) { am = vmax(am, uam); an = vmin(an, uan); }
            if (posj >= d) { bm = vmax(bm, ubm); bn = vmin(bn, ubn); }
        }
        gm = am;
        gn = an;
        hm = bm;
        hn = bn;
        const R xam = __shfl_up_sync(0xffffffffu, am, 1);
        const R xan = __shfl_up_sync(0xffffffffu, an, 1);
        const R xbm = __shfl_down_sync(0xffffffffu, bm, 1);
        const R xbn = __shfl_down_sync(0xffffffffu, bn, 1);
        em = posk ? xam : Elem<T>::lo();
        en = posk ? xan : Elem<T>::hi();
        fm = posj ? xbm : Elem<T>::lo();
        fn = posj ? xbn : Elem<T>::hi();
    }

    // Column of item-relative thread block u in the rings of modes 1 and 2
    // (its tile is one of the last three).
    __device__ __forceinline__ int col_of(int u) const { return ((u >> G::LGNT) % 3) * G::NT + (u & (G::NT - 1)); }

    // K-side bookkeeping of tile x: local prefixes into the P ring, stored
    // element-major (element i of thread block u at row i, column u, so
    // that a warp reading one element of consecutive blocks touches
    // consecutive words), carries into the carry ring, and (mode 2) the
    // warp's block aggregate.
    template <int MODE>
    __device__ __forceinline__ void k_publish(int x, const R (&pm)[V], const R (&pn)[V], R em, R en, R gm, R gn) {
        const int col = (x % 3) * G::NT + tid;
        Pair *r = S::ring() + col;
#pragma unroll
        for (int i = 0; i < V; ++i) r[i * 3 * G::NT] = Elem<T>::pair(pm[i], pn[i]);
        S::cre()[col] = Elem<T>::pair(em, en);
        S::crg()[col] = Elem<T>::pair(gm, gn);
        if (MODE == 2 && lane == 31) S::kagg()[(x % 3) * NW + warp] = Elem<T>::pair(gm, gn);
    }

    // Outputs of output tile c (modes 1, 2): sm/sn the local suffixes of the
    // J tile, fm/fn its lane carry.  vec: the item's outputs start 16-byte
    // aligned (full groups of V are stored as vectors).
    template <int MODE>
    __device__ __forceinline__ void outputs12(const ItemPlan<T> &ip, int c, const R (&sm)[V], const R (&sn)[V], R fm,
                                              R fn, int vec) {
        const int lgB = MODE == 2 ? G::LGV + 5 : ip.lgB;
        const int jr0 = c * T_ + tid * V;
        const int kr0 = jr0 + ip.s;
        // k = kr0 + i lies in thread block tk0 for i < crossT (as its element
        // o + i), else in tk0 + 1 (element o + i - V).
        const int o = kr0 & (V - 1);  // the same for every thread of the item
        const int crossT = o ? V - o : V;
        const int tk0 = kr0 >> G::LGV;
        const int col0 = col_of(tk0), col1 = col_of(tk0 + 1);
        const int base0 = o * 3 * G::NT + col0, base1 = (o - V) * 3 * G::NT + col1;
        const Pair e0 = S::cre()[col0];
        R e1m = Elem<T>::lo(), e1n = Elem<T>::hi();
        if (o) {
            const Pair e1 = S::cre()[col1];
            e1m = Elem<T>::pmax(e1);
            e1n = Elem<T>::pmin(e1);
        }
        const int Bj = jr0 >> lgB;
        const int Bk0 = kr0 >> lgB;
        const int Bk1 = (kr0 + crossT) >> lgB;  // scan block of k for i >= crossT (if any)
        R mid0m, mid0n, mid1m, mid1n;
        if (MODE == 1 || !ip.caseB) {
            // k's scan block is Bj+q2 or Bj+q2+1 (q2 = s >> lgB), the same two
            // for the whole warp: Ma = blocks Bj+1 .. Bj+q2-1, Mb adds Bj+q2.
            // Mode 1 has q2 = 1 (Ma empty); mode 2 case A reads the warp-block
            // aggregates of tiles c and c+1.
            const int q2 = ip.s >> lgB;
            R Mam = Elem<T>::lo(), Man = Elem<T>::hi(), Mbm, Mbn;
            if constexpr (MODE == 1) {
                const Pair gb = S::crg()[col_of(((Bj + 2) << (lgB - G::LGV)) - 1)];
                Mbm = Elem<T>::pmax(gb);
                Mbn = Elem<T>::pmin(gb);
            } else {
                const int s0 = c % 3, s1 = s0 == 2 ? 0 : s0 + 1;
#pragma unroll
                for (int u = 1; u < NW; ++u) {
                    if (u < q2) {
                        const int g = warp + u;  // warp block of tile c (< NW) or c+1
                        const Pair a = S::kagg()[(g < NW ? s0 : s1) * NW + (g & (NW - 1))];
                        Mam = vmax(Mam, Elem<T>::pmax(a));
                        Man = vmin(Man, Elem<T>::pmin(a));
                    }
                }
                const int g = warp + q2;
                const Pair a = S::kagg()[(g < NW ? s0 : s1) * NW + (g & (NW - 1))];
                Mbm = vmax(Mam, Elem<T>::pmax(a));
                Mbn = vmin(Man, Elem<T>::pmin(a));
            }
            const bool a0 = Bk0 == Bj + q2, a1 = Bk1 == Bj + q2;
            mid0m = a0 ? Mam : Mbm;
            mid0n = a0 ? Man : Mbn;
            mid1m = a1 ? Mam : Mbm;
            mid1n = a1 ? Man : Mbn;
        } else {
            // Case B: the warp blocks Bj+1 .. Bj+q2-1 are the rest of tile c
            // (J-tile block aggregates), the whole tiles c+1 .. c+q-1 (one
            // value per output tile, kept by warp 0), and the first warp
            // blocks of K tile c+q (or all of it and the first of c+q+1).
            // Mb adds block Bj+q2.  All of it is the same for the warp.
            const int q = ip.q;
            const int q2 = ip.s >> lgB;
            const Pair tbv = S::tb()[c & 1];
            R Mam = Elem<T>::pmax(tbv), Man = Elem<T>::pmin(tbv), Mbm, Mbn;
#pragma unroll
            for (int w = 1; w < NW; ++w) {
                if (warp + w < NW) {
                    const Pair a = S::jagg()[(c & 1) * NW + warp + w];
                    Mam = vmax(Mam, Elem<T>::pmax(a));
                    Man = vmin(Man, Elem<T>::pmin(a));
                }
            }
            // Last block of the range, in warp blocks from the start of tile c+q.
            const int last = warp + (q2 - q * NW) - 1;  // in [-1, 2NW-2]
            const int s0 = (c + q) % 3, s1 = (c + q + 1) % 3;
#pragma unroll
            for (int g = 0; g < 2 * NW - 1; ++g) {
                if (g <= last) {
                    const Pair a = S::kagg()[(g < NW ? s0 : s1) * NW + (g & (NW - 1))];
                    Mam = vmax(Mam, Elem<T>::pmax(a));
                    Man = vmin(Man, Elem<T>::pmin(a));
                }
            }
            {
                const int g = last + 1;  // block Bj+q2
                const Pair a = S::kagg()[(g < NW ? s0 : s1) * NW + (g & (NW - 1))];
                Mbm = vmax(Mam, Elem<T>::pmax(a));
                Mbn = vmin(Man, Elem<T>::pmin(a));
            }
            const bool a0 = Bk0 == Bj + q2, a1 = Bk1 == Bj + q2;
            mid0m = a0 ? Mam : Mbm;
            mid0n = a0 ? Man : Mbn;
            mid1m = a1 ? Mam : Mbm;
            mid1n = a1 ? Man : Mbn;
        }
        const R c0m = vmax3(fm, mid0m, Elem<T>::pmax(e0)), c0n = vmin3(fn, mid0n, Elem<T>::pmin(e0));
        const R c1m = vmax3(fm, mid1m, e1m), c1n = vmin3(fn, mid1n, e1n);
        R om[V], on[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const Pair pr = S::ring()[(i < crossT ? base0 : base1) + i * 3 * G::NT];
            const bool far = i >= crossT;
            om[i] = vmax3(sm[i], far ? c1m : c0m, Elem<T>::pmax(pr));
            on[i] = vmin3(sn[i], far ? c1n : c0n, Elem<T>::pmin(pr));
        }
        store_out(ip, ip.o_begin + jr0, om, on, vec);
    }

    // 32-byte streaming stores (full sectors): V * sizeof(T) a multiple of 32,
    // dst 32-byte aligned.
    __device__ __forceinline__ void store_v8(T *dst, const R (&v)[V]) const {
#pragma unroll
        for (int c = 0; c < G::NCH / 2; ++c) {
            asm volatile("st.global.cs.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(
                             reinterpret_cast<uint8_t *>(dst) + 32 * c),
                         "r"(pack_word<T>(v, 8 * c)), "r"(pack_word<T>(v, 8 * c + 1)), "r"(pack_word<T>(v, 8 * c + 2)),
                         "r"(pack_word<T>(v, 8 * c + 3)), "r"(pack_word<T>(v, 8 * c + 4)),
                         "r"(pack_word<T>(v, 8 * c + 5)), "r"(pack_word<T>(v, 8 * c + 6)),
                         "r"(pack_word<T>(v, 8 * c + 7))
                         : "memory");
        }
    }

    __device__ __forceinline__ void store_vec(T *dst, const R (&v)[V]) const {
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
    }

    // J-side state of one output tile: local suffixes and lane carry.
    struct JState {
        R sm[V], sn[V];
        R fm, fn;
    };

    // Case A iteration c: read tile c+1 (K role now, J role of the next
    // output tile, into nx), then the outputs of tile c from cur.
    template <int MODE>
    __device__ __forceinline__ bool step_a(const ItemPlan<T> &ip, int c, int lgS, int vec, const JState &cur,
                                           JState &nx) {
        const bool kload = c + 1 < ip.NC || ip.klast;  // else no window reaches tile c+1
        if (kload) {
            R xm[V], xn[V];
            read_tile(ip, c + 1, xm, xn);
            R pm[V], pn[V], em, en, gm, gn, hm, hn;
            scan_kj(lgS, xm, xn, xm, xn, pm, pn, em, en, gm, gn, nx.sm, nx.sn, nx.fm, nx.fn, hm, hn);
            k_publish<MODE>(c + 1, pm, pn, em, en, gm, gn);
        }
        sync();
        outputs12<MODE>(ip, c, cur.sm, cur.sn, cur.fm, cur.fn, vec);
        return true;
    }

    // Advancing front, one round: output tile t (relative tile 0; its K
    // tiles are relative q and q+1).  The whole tiles inside its windows,
    // t+1 .. t+q-1, enter as published aggregates: tile x was read ahead in
    // round x-q-G, a whole round of the grid earlier (or at the start, for
    // x < q+G), so they are normally there when asked for; this round in turn
    // reads tile t+q+G ahead and publishes it.  Warp 0 starts loading the
    // aggregates with the round, so that their latency overlaps its reads.
    // The four stages of the round are always read (see issue_next_front).
    __device__ __forceinline__ void run_front_round(const ItemPlan<T> &ip, int vec) {
        constexpr int MODE = 2;
        constexpr int lgS = 5;
        const BlockScanParams &P = S::params();
        const int q = ip.q;
        // Warp 0, lane l: the published words of tile 1+l (if inside 1..q-1).
        unsigned long long ea = 0, eb = 0;
        if (warp == 0 && 1 + lane <= q - 1) {
            const unsigned long long *slot = P.front_slots + 2 * (ip.gt0 + 1 + lane);
            asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(ea), "=l"(eb) : "l"(slot));
        }
        JState js;
        R hm, hn;
        {
            R xm[V], xn[V];
            read_tile(ip, q, xm, xn);  // K tile q
            R pm[V], pn[V], em, en, gm, gn;
            scan_k(lgS, xm, xn, pm, pn, em, en, gm, gn);
            k_publish<MODE>(q, pm, pn, em, en, gm, gn);
        }
        {
            R km[V], kn[V], jm[V], jn[V];
            read_tile(ip, q + 1, km, kn);  // K tile q+1
            read_tile(ip, 0, jm, jn);      // J tile 0
            if (ip.klast) {                // some window of the tile reaches K tile q+1
                R pm[V], pn[V], em, en, gm, gn;
                scan_kj(lgS, km, kn, jm, jn, pm, pn, em, en, gm, gn, js.sm, js.sn, js.fm, js.fn, hm, hn);
                k_publish<MODE>(q + 1, pm, pn, em, en, gm, gn);
            } else {
                scan_j(lgS, jm, jn, js.sm, js.sn, js.fm, js.fn, hm, hn);
            }
        }
        if (lane == 0) S::jagg()[warp] = Elem<T>::pair(hm, hn);
        {
            // The tile read ahead: its maximum and minimum only.
            R xm[V], xn[V];
            read_tile(ip, q + (int)gridDim.x, xm, xn);
            if (ip.la) {
                R m = xm[0], n = xn[0];
#pragma unroll
                for (int i = 1; i < V; ++i) {
                    m = vmax(m, xm[i]);
                    n = vmin(n, xn[i]);
                }
#pragma unroll
                for (int d = 16; d >= 1; d >>= 1) {
                    m = vmax(m, __shfl_xor_sync(0xffffffffu, m, d));
                    n = vmin(n, __shfl_xor_sync(0xffffffffu, n, d));
                }
                if (lane == 0) S::jagg()[NW + warp] = Elem<T>::pair(m, n);
            }
        }
        if (warp == 0) {
            // Whole tiles 1..q-1: the early words where their tags are there,
            // else (and for tiles past 1+32) bounded waits for them.
            bool ok = !failed;
            R m = Elem<T>::lo(), n = Elem<T>::hi();
            const long long t0 = clock64();
            for (int x = 1 + lane; ok && x <= q - 1; x += 32) {
                const int64_t g = ip.gt0 + x;
                const uint32_t tag = (uint32_t)(g + 1);
                R am, an;
                bool got = false;
                if (x == 1 + lane && (uint32_t)(ea >> 32) == tag && (uint32_t)(eb >> 32) == tag) {
                    rfrom((uint32_t)ea, am);
                    rfrom((uint32_t)eb, an);
                    got = true;
                }
                while (!got && !(got = front_get<T>(P.front_slots + 2 * g, tag, am, an))) {
                    if (clock64() - t0 > wait_limit) {
                        ok = false;
                        break;
                    }
                    __nanosleep(32);
                }
                if (got) {
                    m = vmax(m, am);
                    n = vmin(n, an);
                }
            }
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1) {
                m = vmax(m, __shfl_xor_sync(0xffffffffu, m, d));
                n = vmin(n, __shfl_xor_sync(0xffffffffu, n, d));
            }
            ok = __all_sync(0xffffffffu, ok);
            if (!ok && !failed) {
                if (lane == 0) report_error(P.status, kErrWaitTimeout);
                failed = true;
            }
            if (lane == 0) S::tb()[0] = Elem<T>::pair(m, n);
        }
        sync();
        if (ip.la && warp == 0) {
            Pair a = lane < NW ? S::jagg()[NW + lane] : Elem<T>::pair(Elem<T>::lo(), Elem<T>::hi());
            R m = Elem<T>::pmax(a), n = Elem<T>::pmin(a);
#pragma unroll
            for (int d = NW / 2; d >= 1; d >>= 1) {
                m = vmax(m, __shfl_xor_sync(0xffffffffu, m, d));
                n = vmin(n, __shfl_xor_sync(0xffffffffu, n, d));
            }
            const int64_t g = ip.gt0 + ip.la;
            if (lane == 0) front_put<T>(P.front_slots + 2 * g, (uint32_t)(g + 1), m, n);
        }
        outputs12<MODE>(ip, 0, js.sm, js.sn, js.fm, js.fn, vec);
    }

    template <int MODE>
    __device__ __forceinline__ void run_item12(const ItemPlan<T> &ip) {
        const int q = ip.q;
        // Mode 2 scan blocks span one warp (2^5 lanes): a compile-time width
        // keeps the lane scans free of branches.
        const int lgS = MODE == 2 ? 5 : ip.lgB - G::LGV;
        const int vec = out_vec(ip);
        if (!ip.caseB) {
            // Tile c is the J tile of output tile c and a K tile of c-1 and c.
            // The loop is unrolled by two so that the J states alternate.
            JState ja, jb;
            {
                R xm[V], xn[V];
                read_tile(ip, 0, xm, xn);
                R pm[V], pn[V], em, en, gm, gn, hm, hn;
                scan_kj(lgS, xm, xn, xm, xn, pm, pn, em, en, gm, gn, ja.sm, ja.sn, ja.fm, ja.fn, hm, hn);
                k_publish<MODE>(0, pm, pn, em, en, gm, gn);
            }
            for (int c = 0; c < ip.NC; c += 2) {
                if (!step_a<MODE>(ip, c, lgS, vec, ja, jb)) return;
                if (c + 1 < ip.NC && !step_a<MODE>(ip, c + 1, lgS, vec, jb, ja)) return;
            }
        } else {
            // w - 1 >= T: K tiles c+q, c+q+1; the J tile c is read again.
            for (int x = 1; x <= q; ++x) {
                R xm[V], xn[V];
                read_tile(ip, x, xm, xn);
                R pm[V], pn[V], em, en, gm, gn;
                scan_k(lgS, xm, xn, pm, pn, em, en, gm, gn);
                k_publish<MODE>(x, pm, pn, em, en, gm, gn);
                sync();
                publish_tile_aggregate(x);
            }
            TileQueue<T> tq;  // warp 0: tiles [c+1, c+q-1]
            if (warp == 0) {
                for (int x = 1; x <= q - 1; ++x) tq.push(x);
                const Pair v = tq.query();
                if (lane == 0) S::tb()[0] = v;
            }
            sync();
            for (int c = 0; c < ip.NC; ++c) {
                const int xk = c + q + 1;
                const bool kload = c + 1 < ip.NC || ip.klast;
                JState js;
                R hm, hn;
                if (kload) {
                    R km[V], kn[V], jm[V], jn[V];
                    read_tile(ip, xk, km, kn);  // K tile c+q+1
                    read_tile(ip, c, jm, jn);   // J tile c
                    R pm[V], pn[V], em, en, gm, gn;
                    scan_kj(lgS, km, kn, jm, jn, pm, pn, em, en, gm, gn, js.sm, js.sn, js.fm, js.fn, hm, hn);
                    k_publish<MODE>(xk, pm, pn, em, en, gm, gn);
                } else {
                    R jm[V], jn[V];
                    read_tile(ip, c, jm, jn);
                    scan_j(lgS, jm, jn, js.sm, js.sn, js.fm, js.fn, hm, hn);
                }
                if (lane == 0) S::jagg()[(c & 1) * NW + warp] = Elem<T>::pair(hm, hn);
                sync();
                // The last warp publishes while warp 0 updates the queue: the
                // two jobs follow the barrier side by side, and the next
                // barrier comes between the aggregate and its reader.
                if (kload) publish_tile_aggregate(xk, NW - 1);
                if (warp == 0 && c + 1 < ip.NC) {
                    // The range of output tile c+1: drop tile c+1, add tile c+q
                    // (published in the previous step).
                    if (q >= 2) tq.slide(c + q);
                    const Pair v = tq.query();
                    if (lane == 0) S::tb()[(c + 1) & 1] = v;
                }
                outputs12<MODE>(ip, c, js.sm, js.sn, js.fm, js.fn, vec);
            }
        }
    }

    // ------------------------------------------------------ register slide
    // Read this thread's V elements and the HALO_MAX that follow them.
    __device__ __forceinline__ bool read_tile_ext(const ItemPlan<T> &ip, int x, R (&xm)[V + G::HALO_MAX],
                                                  R (&xn)[V + G::HALO_MAX]) {
        constexpr int NE = V + G::HALO_MAX;
        const bool ok = wait_stage();  // as in read_tile: on failure the values are unspecified
        const int smode = S::issue(warp)->smode[cur.stage];
        const int mode = smode & 0xff;
        const uint8_t *sb = S::slice(warp, cur.stage);
        constexpr int NWE = NE * (int)sizeof(T) / 4;
        if (mode == 0) {
            uint32_t wd[NWE];
            read_words<NWE>(sb, wd);
            R xv[NE];
            ExtractLoop<T, 0, 0, NE>::run(wd, xv);
#pragma unroll
            for (int i = 0; i < NE; ++i) xm[i] = xn[i] = xv[i];
        } else if (mode == 1 || mode == 4) {
            uint32_t wd[NWE + 4];
            read_words<NWE>(sb, wd);
            read_tail(sb, NWE, wd + NWE);
            shift_bytes<NWE>(wd, (smode >> 8) * (int)sizeof(T));
            R xv[NE];
            ExtractLoop<T, 0, 0, NE>::run(wd, xv);
#pragma unroll
            for (int i = 0; i < NE; ++i) xm[i] = xn[i] = xv[i];
            if (mode == 4) clip(ip, x, NE, xm, xn);
        } else if (mode == 3) {
#pragma unroll
            for (int i = 0; i < NE; ++i) {
                xm[i] = Elem<T>::lo();
                xn[i] = Elem<T>::hi();
            }
        } else {
            const int64_t pt = ip.p0 + (int64_t)x * T_ + (int64_t)warp * G::SLICE + (int64_t)lane * V;
#pragma unroll
            for (int i = 0; i < NE; ++i) {
                const int64_t p = pt + i;
                if (p < 0 || p >= ip.n ||
                    !in_range(S::params().status, (ip.in - reinterpret_cast<const T *>(S::params().in)) + p, 0,
                              S::params().in_elems)) {
                    xm[i] = Elem<T>::lo();
                    xn[i] = Elem<T>::hi();
                } else {
                    xm[i] = xn[i] = Elem<T>::load(ip.in[p]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) issue_next<T, KMODE, FRONT>(warp);
        __syncwarp();
        cur.advance();
        return ok;
    }

    // Windows of W elements straight from registers (the naive row of
    // Table 1), shared by pairwise doubling: after the passes a[i] is the
    // max over 2^k consecutive elements, and two such ranges cover a window.
    template <int W>
    __device__ __forceinline__ void run_slide(const ItemPlan<T> &ip) {
        constexpr int NE = V + G::HALO_MAX;
        constexpr int P2 = W >= 16 ? 16 : (W >= 8 ? 8 : (W >= 4 ? 4 : (W >= 2 ? 2 : 1)));
        const int vec = out_vec(ip);
        for (int c = 0; c < ip.NC; ++c) {
            R am[NE], an[NE];
            read_tile_ext(ip, c, am, an);
#pragma unroll
            for (int p = 1; p < P2; p <<= 1) {
#pragma unroll
                for (int i = 0; i + p < NE; ++i) { am[i] = vmax(am[i], am[i + p]); an[i] = vmin(an[i], an[i + p]); }
            }
            R om[V], on[V];
#pragma unroll
            for (int i = 0; i < V; ++i) {
                om[i] = W > P2 ? vmax(am[i], am[i + W - P2]) : am[i];
                on[i] = W > P2 ? vmin(an[i], an[i + W - P2]) : an[i];
            }
            store_out(ip, ip.o_begin + (int64_t)c * T_ + (int64_t)tid * V, om, on, vec);
        }
    }

    __device__ __forceinline__ void run_item_slide(const ItemPlan<T> &ip) {
        switch (ip.s) {
            case 0: run_slide<1>(ip); break;
            case 1: run_slide<2>(ip); break;
            case 2: run_slide<3>(ip); break;
            case 3: run_slide<4>(ip); break;
            case 4: run_slide<5>(ip); break;
            case 5: run_slide<6>(ip); break;
            case 6: run_slide<7>(ip); break;
            case 7: run_slide<8>(ip); break;
            case 8: run_slide<9>(ip); break;
            default:
                if constexpr (G::SLIDE_S >= 16) {
                    switch (ip.s) {
                        case 9: run_slide<10>(ip); break;
                        case 10: run_slide<11>(ip); break;
                        case 11: run_slide<12>(ip); break;
                        case 12: run_slide<13>(ip); break;
                        case 13: run_slide<14>(ip); break;
                        case 14: run_slide<15>(ip); break;
                        case 15: run_slide<16>(ip); break;
                        default: run_slide<17>(ip); break;
                    }
                }
                break;
        }
    }

    template <int MODE>
    __device__ __forceinline__ void run_item(const ItemPlan<T> &ip) {
        const int q = ip.q;
        R Sc_m[V], Sc_n[V];  // case A: suffix scan of input tile c

        // ---------------- prologue: tile 0 (case A) or tiles 1..q (case B)
        if (!ip.caseB) {
            R pm[V], pn[V];
            read_tile(ip, 0, pm, pn);
#pragma unroll
            for (int i = 0; i < V; ++i) { Sc_m[i] = pm[i]; Sc_n[i] = pn[i]; }
            scan_tile<MODE>(ip, pm, pn, true, Sc_m, Sc_n, 0, -1);
            ring_write(0, pm, pn);
        } else {
            for (int x = 1; x <= q; ++x) {
                R pm[V], pn[V];
                read_tile(ip, x, pm, pn);
                scan_tile<MODE>(ip, pm, pn, false, pm, pn, x % 3, -1);
                if (x == q) ring_write(x, pm, pn);
                sync();
                publish_tile_aggregate(x);
            }
        }
        sync();

        // ---------------- main loop over output tiles
        for (int c = 0; c < ip.NC; ++c) {
            R pm[V], pn[V], Sn_m[V], Sn_n[V];
            const int xk = c + q + 1;
            const bool kload = c + 1 < ip.NC || ip.klast;  // else no window reaches K tile xk
            if (!ip.caseB) {
                if (kload) {
                    read_tile(ip, xk, pm, pn);  // K tile c+1 (also J tile of c+1)
#pragma unroll
                    for (int i = 0; i < V; ++i) { Sn_m[i] = pm[i]; Sn_n[i] = pn[i]; }
                    scan_tile<MODE>(ip, pm, pn, true, Sn_m, Sn_n, xk % 3, -1);
                    ring_write(xk, pm, pn);
                }
                sync();
                outputs<MODE>(ip, c, Sc_m, Sc_n);
                if (kload) {
#pragma unroll
                    for (int i = 0; i < V; ++i) { Sc_m[i] = Sn_m[i]; Sc_n[i] = Sn_n[i]; }
                }
            } else {
                if (kload) read_tile(ip, xk, pm, pn);  // K tile c+q+1
                read_tile(ip, c, Sn_m, Sn_n);          // J tile c
                scan_tile<MODE>(ip, pm, pn, true, Sn_m, Sn_n, xk % 3, c & 1, kload);
                if (kload) ring_write(xk, pm, pn);
                sync();
                if (kload) publish_tile_aggregate(xk);
                outputs<MODE>(ip, c, Sn_m, Sn_n);
            }
        }
    }
};

// Advancing front, at the start of the launch: CTA b publishes the
// aggregates of global tiles b, b+G, ... inside [1, q+G) (the tiles no item
// reads ahead), with plain loads; no wait comes before it.
template <typename T>
__device__ __forceinline__ void front_prologue(const BlockScanParams &P, int tid, int lane, int warp) {
    using G = Geo<T>;
    using R = typename Elem<T>::R;
    using Pair = typename Elem<T>::Pair;
    using S = Smem<T>;
    const SeriesDesc &sd = P.one;
    const T *in = reinterpret_cast<const T *>(P.in) + sd.in_off;
    const int64_t end = ((sd.w - 1) >> G::LGT) + P.front_ahead;
    for (int64_t x = blockIdx.x; x < end; x += gridDim.x) {
        if (x == 0) continue;  // no window has tile 0 inside
        R m = Elem<T>::lo(), n = Elem<T>::hi();
        const int64_t base = sd.d + x * G::T_ + (int64_t)tid * G::V;
#pragma unroll
        for (int i = 0; i < G::V; ++i) {
            const int64_t p = base + i;
            if (p >= 0 && p < sd.n) {
                const R v = Elem<T>::load(in[p]);
                m = vmax(m, v);
                n = vmin(n, v);
            }
        }
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) {
            m = vmax(m, __shfl_xor_sync(0xffffffffu, m, d));
            n = vmin(n, __shfl_xor_sync(0xffffffffu, n, d));
        }
        if (lane == 0) S::jagg()[warp] = Elem<T>::pair(m, n);
        named_bar_sync(1, G::NT);
        if (warp == 0) {
            Pair a = lane < G::NW ? S::jagg()[lane] : Elem<T>::pair(Elem<T>::lo(), Elem<T>::hi());
            m = Elem<T>::pmax(a);
            n = Elem<T>::pmin(a);
#pragma unroll
            for (int d = G::NW / 2; d >= 1; d >>= 1) {
                m = vmax(m, __shfl_xor_sync(0xffffffffu, m, d));
                n = vmin(n, __shfl_xor_sync(0xffffffffu, n, d));
            }
            if (lane == 0) front_put<T>(P.front_slots + 2 * x, (uint32_t)(x + 1), m, n);
        }
        named_bar_sync(1, G::NT);
    }
}

// The plan of round t of the advancing front (output tile t alone).
template <typename T>
__device__ __forceinline__ ItemPlan<T> front_plan(const BlockScanParams &P, int64_t t) {
    using G = Geo<T>;
    const SeriesDesc &sd = P.one;
    ItemPlan<T> ip;
    ip.series = 0;
    ip.lb_acc = nullptr;
    ip.in = reinterpret_cast<const T *>(P.in) + sd.in_off;
    ip.omax = P.out_max ? reinterpret_cast<T *>(P.out_max) + sd.out_off : nullptr;
    ip.omin = P.out_min ? reinterpret_cast<T *>(P.out_min) + sd.out_off : nullptr;
    ip.n = sd.n;
    ip.o_begin = t << G::LGT;
    ip.o_end = ip.o_begin + G::T_ < sd.n_out ? ip.o_begin + G::T_ : sd.n_out;
    ip.p0 = ip.o_begin + sd.d;
    ip.s = (int)(sd.w - 1);
    ip.q = ip.s >> G::LGT;
    ip.caseB = 1;
    ip.lgB = G::LGV + 5;
    ip.mode = 2;
    ip.NC = 1;
    ip.klast = (int)(((ip.o_end - ip.o_begin - 1) + ip.s) >> G::LGT) >= 1 + ip.q;
    ip.front = 1;
    ip.gt0 = t;
    ip.la = t + ip.q + gridDim.x <= P.front_last ? ip.q + (int)gridDim.x : 0;
    ip.ok = 1;
    return ip;
}

// One instantiation per block mode keeps each one within 128 registers (two
// CTAs per SM); an item whose mode differs is rejected (kErrBadItem).  FRONT:
// the advancing front of one series (mode 2, windows of a tile or more; a
// cooperative launch), see run_front_round.
template <typename T, int MODE, bool LB = false, bool FRONT = false>
__global__ void __launch_bounds__(Geo<T>::NT, (Geo<T>::NT * Elem<T>::V == 4096 && MODE != 3) ? 1 : 2)
    blockscan_kernel(const BlockScanParams P) {
    using S = Smem<T>;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    int fetched = 0;  // thread 0: dynamic tickets fetched
    if (tid == 0) {
        *reinterpret_cast<BlockScanParams *>(S::misc() + Geo<T>::off_params) = P;
        if (P.ticket) {
            // Items for sequence numbers 0..kStages: enough for every warp's
            // prefetch until the first item boundary (items of one load).  In
            // the advancing front every item has at least two loads, so the
            // prefetch reaches at most two items ahead: three tickets keep
            // the CTA's items close to the front.
            const int nq = P.front_slots ? 3 : kStages + 1;
            for (; fetched < nq; ++fetched) S::queue()[fetched & (kQueue - 1)] = atomicAdd(P.ticket, 1);
        }
    }
    if (lane == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(S::bar(warp, s), 1);
        WarpIssue &wi = *S::issue(warp);
        wi.src0 = 0;
        wi.fast_lo = wi.fast_hi = 0;
        wi.fast_smode = wi.fast_extra = 0;
        wi.in = nullptr;
        wi.n = wi.p0 = 0;
        wi.seq = -1;
        wi.l = wi.nloads = 0;
        wi.q = wi.caseB = wi.ok = wi.NC = wi.klast = 0;
        wi.linear = 0;
        wi.issued = 0;
        for (int s = 0; s < kStages; ++s) wi.smode[s] = 3;  // empty until a copy is issued
        if constexpr (FRONT) {
            // The CTA's rounds, four loads each.
            const int64_t tiles = (P.one.n_out + Geo<T>::T_ - 1) >> Geo<T>::LGT;
            const int64_t rounds = tiles > blockIdx.x ? (tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
            wi.nloads = (int32_t)(4 * rounds);
            wi.q = (int32_t)((P.one.w - 1) >> Geo<T>::LGT);
        }
        // Test hook: a warp whose sequence has ended issues nothing, so every
        // wait of the kernel runs out.
        if (P.test_flags & kTestStarveCopies) wi.nloads = -1;
        fence_mbar_init();
    }
    __syncthreads();
    if (lane == 0)
        for (int s = 0; s < kStages; ++s) issue_next<T, MODE, FRONT>(warp);
    __syncwarp();

    Consumer<T, MODE, LB, FRONT> cs;
    cs.tid = tid;
    cs.lane = lane;
    cs.warp = warp;
    const BlockScanParams &PS = S::params();
    cs.wait_limit = PS.wait_limit > 0 ? PS.wait_limit : kWaitLimitCycles;
    if constexpr (FRONT) {
        static_assert(MODE == 2 && kCarryRing<T> && !LB, "the advancing front is a mode-2 storing kernel");
        front_prologue<T>(P, tid, lane, warp);
        // Round plans from the launch parameters themselves (constant bank).
        const int64_t tiles = (P.one.n_out + Geo<T>::T_ - 1) >> Geo<T>::LGT;
        const int vec = cs.out_vec(front_plan<T>(P, 0));  // the same for every round (whole vectors apart)
        for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
            cs.run_front_round(front_plan<T>(P, t), vec);
            cs.sync();  // the rings are rewritten by the next round
        }
        if (named_bar_sync_or(2, Geo<T>::NT, cs.failed)) cs.drain();
    } else {
    for (int seq = 0;; ++seq) {
        const int64_t item = item_of<T>(PS, seq);
        if (item >= PS.n_items || item < 0) return;
        // The ticket for the prefetch is requested now and stored at the
        // item's end; the next item's table entries are brought to L1 while
        // this item runs (its item entry now, its series entry at the end).
        int tk = 0;
        if (tid == 0 && PS.ticket) tk = atomicAdd(P.ticket, 1);
        const int64_t next = item_of<T>(PS, seq + 1);
        int64_t nser = -1;
        if (PS.items && next < PS.n_items && next >= 0) nser = __ldg(&PS.items[next].series);
        ItemPlan<T> ip = make_plan<T>(PS, item, MODE);
        if (!ip.ok) {
            // A rejected item occupies one empty stage per warp.
            cs.wait_stage();
            __syncwarp();
            if (lane == 0) issue_next<T, MODE>(warp);
            __syncwarp();
            cs.cur.advance();
        } else {
            // After a failed wait every lane still finishes the item, without
            // waiting again (its outputs are then unspecified).
            if constexpr (MODE == 3)
                cs.run_item_slide(ip);
            else if constexpr (MODE == 0 || !kCarryRing<T>)
                cs.template run_item<MODE>(ip);
            else
                cs.template run_item12<MODE>(ip);
        }
        if (nser >= 0) prefetch_l1(PS.series + nser);
        // The item boundary frees the ring and publishes the queue.  Every
        // warp arrives here, failed or not; if any warp failed, all leave
        // together (after their copies in flight have landed).  The barrier
        // itself ORs the flags, so every warp takes the same decision.
        if (tid == 0 && PS.ticket) {
            S::queue()[fetched & (kQueue - 1)] = tk;
            ++fetched;
        }
        if (named_bar_sync_or(2, Geo<T>::NT, cs.failed)) {  // its own id: barrier 1 is only bar.sync
            cs.drain();
            return;
        }
    }
    }
}

}  // namespace mmf
