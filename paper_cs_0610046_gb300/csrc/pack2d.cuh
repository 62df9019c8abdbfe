// Register-streaming separable 2D filter for small windows (Section 1: the
// 1D filter on rows, then on columns), f32 and, packed, 1- and 2-byte
// elements.  The shared-memory
// tile kernel spends an instruction per element on every step; here every
// max/min is one 16x2 SIMD instruction (PTX max/min .s16x2, .u16x2): i16
// words hold 2 neighbouring columns, and a u8 word of 4 columns is held as
// two u16x2 registers, its even and its odd columns (unpacked once after the
// load, packed once before the store; the byte-wise intrinsics expand to long
// instruction sequences on this GPU).  f32 takes one column per thread and
// word (no packing): each lane loads its own word of a row and takes the
// window's next columns from the next lanes by shuffles, so the last wx-1
// lanes of a warp are a halo whose outputs are not stored (its outputs are
// always word-aligned, so no realignment).
//
// One thread per output word (L = 4 / sizeof(T) columns), one warp per 31
// consecutive words of one band of kPkBand output rows (its lane 31 computes
// the next warp's first word as well, for the stores), streaming down the
// band in tiles of 8 rows:
//   row pass: the input words at the thread's columns and the next two
//             (word loads; neighbours hit L1), the window's elements taken
//             as element-shifted words (i16: funnel shifts of the words;
//             u8: the even/odd streams and their 16-bit shifts), combined
//             per element;
//   column pass: per tile of 8 output rows, the row results of rows
//             y .. y+15 (the next tile's are reused by the next step)
//             combined by doubling, the naive windows of Table 1 shared
//             between neighbours, as in the other 2D kernels;
//   stores: output rows are dense (width Wo), so their words are generally
//             not 4-byte aligned; with a = the misalignment of the warp's
//             first word, lanes 0 .. 30 store the aligned word of their
//             bytes [4-a, 4) and the next lane's bytes [0, 4-a) (one
//             shuffle), lane 31 stores nothing, and the first warp of a row
//             also stores its lane 0's bytes [0, 4-a) (the row's start).
//             Only columns below Wo are stored: whole words where all are,
//             element by element otherwise (at the ends of rows).
// Rows past those a band needs and columns at or past W feed only outputs
// that are not stored, so they read as zero.  The input rows must be 4-byte
// aligned (the host checks the pointer, the pitch and the image stride).
#pragma once
#include <cstdint>

#include "pack2d.h"
#include "ptx.cuh"

namespace mmf {

template <typename T> struct Pk;
// i16: one word, 2 columns, signed 16x2 max/min.
template <> struct Pk<int16_t> {
    static constexpr int L = 2;
    struct V {
        uint32_t w;
    };
    __device__ static V mx(V a, V b) {
        V r;
        asm("max.s16x2 %0, %1, %2;" : "=r"(r.w) : "r"(a.w), "r"(b.w));
        return r;
    }
    __device__ static V mn(V a, V b) {
        V r;
        asm("min.s16x2 %0, %1, %2;" : "=r"(r.w) : "r"(a.w), "r"(b.w));
        return r;
    }
    __device__ static uint32_t pack(V v) { return v.w; }
    // Row window of WX elements from each of the word's columns (elements
    // 0 .. 5 of the 12 bytes w0 w1 w2).
    template <int WX, int NW> __device__ static void row(const uint32_t (&w)[NW], V &m, V &n) {
        const uint32_t w0 = w[0], w1 = w[1], w2 = NW > 2 ? w[NW > 2 ? 2 : 0] : 0u;
        m = n = V{w0};
#pragma unroll
        for (int k = 1; k < WX; ++k) {
            // A funnel shift takes its count modulo 32: byte offset 8 is w2.
            const int b = 2 * k;
            const V s{b < 4 ? __funnelshift_r(w0, w1, 8 * b) : (b < 8 ? __funnelshift_r(w1, w2, 8 * (b - 4)) : w2)};
            m = mx(m, s);
            n = mn(n, s);
        }
    }
};
// u8: one word of 4 columns as two u16x2 registers, e = columns (0, 2),
// o = columns (1, 3), each byte zero-extended; unsigned 16x2 max/min.
template <> struct Pk<uint8_t> {
    static constexpr int L = 4;
    struct V {
        uint32_t e, o;
    };
    __device__ static uint32_t mx2(uint32_t a, uint32_t b) {
        uint32_t r;
        asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
        return r;
    }
    __device__ static uint32_t mn2(uint32_t a, uint32_t b) {
        uint32_t r;
        asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
        return r;
    }
    __device__ static V mx(V a, V b) { return V{mx2(a.e, b.e), mx2(a.o, b.o)}; }
    __device__ static V mn(V a, V b) { return V{mn2(a.e, b.e), mn2(a.o, b.o)}; }
    // Bytes (e.lo, o.lo, e.hi, o.hi): columns 0 1 2 3.
    __device__ static uint32_t pack(V v) { return __byte_perm(v.e, v.o, 0x6240); }
    // Row window of WX elements from each of the word's columns (columns
    // 0 .. 11 of w0 w1 w2).  The even stream holds columns 0, 2, .., 10 in
    // 16-bit lanes, the odd stream 1, 3, .., 11; X[m] = lanes m, m+1 of a
    // stream.  The word shifted by k columns is (E[m], O[m]) for k = 2m and
    // (O[m], E[m+1]) for k = 2m+1.
    template <int WX, int NW> __device__ static void row(const uint32_t (&w)[NW], V &m, V &n) {
        const uint32_t w0 = w[0], w1 = w[1], w2 = NW > 2 ? w[NW > 2 ? 2 : 0] : 0u;
        uint32_t E[5], O[5];
        E[0] = __byte_perm(w0, 0u, 0x4240);
        O[0] = __byte_perm(w0, 0u, 0x4341);
        E[2] = __byte_perm(w1, 0u, 0x4240);
        O[2] = __byte_perm(w1, 0u, 0x4341);
        E[4] = __byte_perm(w2, 0u, 0x4240);
        O[4] = __byte_perm(w2, 0u, 0x4341);
        E[1] = __byte_perm(E[0], E[2], 0x5432);
        O[1] = __byte_perm(O[0], O[2], 0x5432);
        E[3] = __byte_perm(E[2], E[4], 0x5432);
        O[3] = __byte_perm(O[2], O[4], 0x5432);
        m = n = V{E[0], O[0]};
#pragma unroll
        for (int k = 1; k < WX; ++k) {
            const V s = (k & 1) ? V{O[k >> 1], E[(k >> 1) + 1]} : V{E[k >> 1], O[k >> 1]};
            m = mx(m, s);
            n = mn(n, s);
        }
    }
};

// f32: one column per word.
template <> struct Pk<float> {
    static constexpr int L = 1;
    struct V {
        float f;
    };
    __device__ static V mx(V a, V b) { return V{fmaxf(a.f, b.f)}; }
    __device__ static V mn(V a, V b) { return V{fminf(a.f, b.f)}; }
    __device__ static uint32_t pack(V v) { return __float_as_uint(v.f); }
    // Row window of WX elements: this lane's word and the next WX-1 lanes'
    // (every lane of the warp calls it; the last WX-1 lanes get values of
    // their own, which only their unstored outputs see).
    template <int WX, int NW> __device__ static void row(const uint32_t (&w)[NW], V &m, V &n) {
        const float x = __uint_as_float(w[0]);
        m = n = V{x};
#pragma unroll
        for (int k = 1; k < WX; ++k) {
            const V s{__shfl_down_sync(0xffffffffu, x, k)};
            m = mx(m, s);
            n = mn(n, s);
        }
    }
};

// A 4-byte input word at p (range-checked in a checked build: 0 outside).
__device__ __forceinline__ uint32_t pk_ld(const Pack2DParams &P, const uint8_t *p) {
    return in_bytes(P.status, p, 4, P.in, P.in_bytes) ? __ldg(reinterpret_cast<const uint32_t *>(p)) : 0u;
}

// Word j of an input row (bytes [4j, 4j+4)), zero past the row's `rb` bytes.
__device__ __forceinline__ uint32_t pk_word(const Pack2DParams &P, const uint8_t *row, int64_t j, int64_t rb) {
    const int64_t b = 4 * j;
    if (b + 4 <= rb) return pk_ld(P, row + b);
    uint32_t w = 0;
    for (int i = 0; i < 4; ++i)
        if (b + i < rb && in_bytes(P.status, row + b + i, 1, P.in, P.in_bytes))
            w |= (uint32_t)__ldg(row + b + i) << (8 * i);
    return w;
}

// Element e (0 .. L-1) of word w to p, if its column is below Wo.
// ob: the output buffer (range checks of a checked build).
template <typename T>
__device__ __forceinline__ void pk_put(const Pack2DParams &P, const uint8_t *ob, uint8_t *p, uint32_t w, int e) {
    if (!in_bytes(P.status, p + e * (int)sizeof(T), (int)sizeof(T), ob, P.out_bytes)) return;
    if constexpr (sizeof(T) == 1)
        p[e] = (uint8_t)(w >> (8 * e));
    else if constexpr (sizeof(T) == 2)
        reinterpret_cast<uint16_t *>(p)[e] = (uint16_t)(w >> (16 * e));
    else
        reinterpret_cast<uint32_t *>(p)[e] = w;
}

// Per-lane store facts, the same for every row of a task: whether the lane
// stores (halo lanes do not), whether it is the row's first lane (it also
// stores the elements before the first aligned word), and rem = the row's
// elements from the lane's first column on (Wo - x0, clamped to [0, 8]).
struct PkLane {
    bool st, head;
    int rem;
};

// Stores output word v of one row at byte address ob (see the header:
// aligned words across lanes; ob mod 4 is the same on every lane).  Every
// lane of the warp calls it (the shuffle).
template <typename T>
__device__ __forceinline__ void pk_store(const Pack2DParams &P, const uint8_t *obuf, uint8_t *ob, uint32_t v,
                                         const PkLane &pl) {
    constexpr int L = Pk<T>::L, SZ = (int)sizeof(T);
    if constexpr (SZ == 4) {  // f32 outputs are always word-aligned: no exchange
        if (pl.st && pl.rem >= 1 && in_bytes(P.status, ob, 4, obuf, P.out_bytes))
            __stcs(reinterpret_cast<uint32_t *>(ob), v);
        return;
    }
    // sh: bytes of this word before the next aligned word (0 when aligned: the
    // funnel shift by 0 is v itself), so no branch on the alignment.
    const int sh = (int)(-(uintptr_t)ob & 3);
    const uint32_t nxt = __shfl_down_sync(0xffffffffu, v, 1);
    if (!pl.st) return;  // halo words: the next warp's
    const int h = sh / SZ;  // elements of this word before the next aligned word
    const uint32_t aw = __funnelshift_r(v, nxt, 8 * sh);
    uint8_t *ap = ob + sh;
    if (h + L <= pl.rem) {
        if (in_bytes(P.status, ap, 4, obuf, P.out_bytes)) __stcs(reinterpret_cast<uint32_t *>(ap), aw);
    } else {
#pragma unroll
        for (int e = 0; e < L; ++e)
            if (h + e < pl.rem) pk_put<T>(P, obuf, ap, aw, e);
    }
    if (pl.head && h > 0) {
#pragma unroll
        for (int e = 0; e < L; ++e)
            if (e < h && e < pl.rem) pk_put<T>(P, obuf, ob, v, e);
    }
}

// One warp task: the band [y0, y1) of output rows at word column j, windows
// WY x WX (compile-time, so that the row loop holds no indirect jump).
template <typename T, int WY, int WX>
__device__ __forceinline__ void pk_band(const Pack2DParams &P, int lane, int64_t j, bool head, int64_t y0, int64_t y1,
                                        const uint8_t *in, uint8_t *omax, uint8_t *omin, int64_t obase) {
    PkLane pl;
    pl.st = lane < pk_chunk<T>(WX);  // halo lanes store nothing
    pl.head = head && lane == 0;
    {
        const int64_t rem = P.Wo - j * Pk<T>::L;
        pl.rem = rem < 0 ? 0 : (rem > 8 ? 8 : (int)rem);
    }
    using V = typename Pk<T>::V;
    constexpr int L = Pk<T>::L, SZ = (int)sizeof(T);
    constexpr int P2 = WY >= 8 ? 8 : (WY >= 4 ? 4 : (WY >= 2 ? 2 : 1));
    // Words read per row: the window's elements from each of the word's
    // columns lie in words j .. j+NW-1.
    // (f32: one word, the rest from the next lanes.)
    constexpr int NW = SZ == 4 ? 1 : (((L + WX - 1) * SZ + 3) / 4 > 2 ? ((L + WX - 1) * SZ + 3) / 4 : 2);
    const int64_t x0 = j * L;                    // first output column of the word
    const int64_t rb = P.W * SZ, pitchb = P.pitch * SZ;
    const bool interior = 4 * (j + NW) <= rb;  // every word read lies inside the row
    // Input rows y0 .. y1 + WY - 2 feed the band's outputs; rows at or past
    // ylim are not needed and read as 0.
    const int64_t ylim = y1 + WY - 1 < P.H ? y1 + WY - 1 : P.H;
    // A tile's words are all loaded before any of its arithmetic, so that
    // their loads are in flight together.
    auto load = [&](int64_t y, uint32_t (&w)[NW], bool check) {
        if (check && y >= ylim) {
#pragma unroll
            for (int k = 0; k < NW; ++k) w[k] = 0u;
            return;
        }
        const uint8_t *rp = in + y * pitchb;
        if (interior) {
            const uint32_t *q = reinterpret_cast<const uint32_t *>(rp) + j;
#pragma unroll
            for (int k = 0; k < NW; ++k) w[k] = pk_ld(P, reinterpret_cast<const uint8_t *>(q + k));
        } else {
#pragma unroll
            for (int k = 0; k < NW; ++k) w[k] = pk_word(P, rp, j + k, rb);
        }
    };
    auto row = [&](const uint32_t (&w)[NW], V &m, V &n) {
        Pk<T>::template row<WX, NW>(w, m, n);
    };
    V cm[kPkRows], cn[kPkRows];  // row results of the current tile
    {
        uint32_t w[kPkRows][NW];
#pragma unroll
        for (int r = 0; r < kPkRows; ++r) load(y0 + r, w[r], true);
#pragma unroll
        for (int r = 0; r < kPkRows; ++r) row(w[r], cm[r], cn[r]);
    }
    for (int64_t y = y0; y < y1; y += kPkRows) {
        // Rows y .. y+7 (current) and y+8 .. y+8+WY-2 (the start of the next
        // tile); the rest of the next tile goes straight to its registers.
        // Tiles whose next rows all lie below ylim skip the row checks.
        V am[2 * kPkRows], an[2 * kPkRows];
        const bool check = y + 2 * kPkRows > ylim;
        uint32_t w[kPkRows][NW];
#pragma unroll
        for (int r = 0; r < kPkRows; ++r) load(y + kPkRows + r, w[r], check);
#pragma unroll
        for (int r = 0; r < kPkRows; ++r) {
            am[r] = cm[r];
            an[r] = cn[r];
            if (r < WY - 1) {
                row(w[r], am[kPkRows + r], an[kPkRows + r]);
                cm[r] = am[kPkRows + r];
                cn[r] = an[kPkRows + r];
            } else {
                row(w[r], cm[r], cn[r]);
                am[kPkRows + r] = an[kPkRows + r] = V{};  // outside these outputs' windows
            }
        }
        // After the passes am[i] covers rows i .. i+P2-1; the window of WY
        // rows from r is the union of am[r] and am[r + WY - P2].
#pragma unroll
        for (int p = 1; p < P2; p <<= 1) {
#pragma unroll
            for (int i = 0; i + p < 2 * kPkRows; ++i) {
                am[i] = Pk<T>::mx(am[i], am[i + p]);
                an[i] = Pk<T>::mn(an[i], an[i + p]);
            }
        }
        const int64_t e0 = (obase + y * P.Wo + x0) * SZ;  // this lane's first output byte of row y
        const int64_t rowb = P.Wo * SZ;
#pragma unroll
        for (int r = 0; r < kPkRows; ++r) {
            if (y + r >= y1) break;  // the same on every lane
            const uint32_t vm = Pk<T>::pack(WY > P2 ? Pk<T>::mx(am[r], am[r + WY - P2]) : am[r]);
            const uint32_t vn = Pk<T>::pack(WY > P2 ? Pk<T>::mn(an[r], an[r + WY - P2]) : an[r]);
            if (omax) pk_store<T>(P, omax, omax + e0 + r * rowb, vm, pl);
            if (omin) pk_store<T>(P, omin, omin + e0 + r * rowb, vn, pl);
        }
    }
}

template <typename T, int WY>
__global__ void __launch_bounds__(kPkThreads, 2) pack2d_kernel(const Pack2DParams P) {
    const int lane = threadIdx.x & 31;
    const int64_t task = (int64_t)blockIdx.x * (kPkThreads / 32) + (threadIdx.x >> 5);
    if (task >= P.tasks) return;  // whole warps only: no shuffle partner leaves
    const int64_t chunk = task % P.nchunks;
    const int64_t rest = task / P.nchunks;
    const int64_t band = rest % P.nbands, img = rest / P.nbands;
    const int64_t j = chunk * pk_chunk<T>(P.wx) + lane;  // word column (input and output; lanes past
                                                         // the chunk: the halo)
    const bool head = chunk == 0;
    const int64_t y0 = band * kPkBand;
    const int64_t y1 = y0 + kPkBand < P.Ho ? y0 + kPkBand : P.Ho;
    const uint8_t *in = reinterpret_cast<const uint8_t *>(P.in) + img * P.img_stride * (int64_t)sizeof(T);
    uint8_t *omax = reinterpret_cast<uint8_t *>(P.out_max);
    uint8_t *omin = reinterpret_cast<uint8_t *>(P.out_min);
    const int64_t obase = img * P.Ho * P.Wo;  // element offset of the image's outputs
    switch (P.wx) {  // once per task
        case 1: pk_band<T, WY, 1>(P, lane, j, head, y0, y1, in, omax, omin, obase); break;
        case 2: pk_band<T, WY, 2>(P, lane, j, head, y0, y1, in, omax, omin, obase); break;
        case 3: pk_band<T, WY, 3>(P, lane, j, head, y0, y1, in, omax, omin, obase); break;
        case 4: pk_band<T, WY, 4>(P, lane, j, head, y0, y1, in, omax, omin, obase); break;
        case 5: pk_band<T, WY, 5>(P, lane, j, head, y0, y1, in, omax, omin, obase); break;
        case 6: if constexpr (pk_max_wx<T>() >= 6) pk_band<T, WY, 6>(P, lane, j, head, y0, y1, in, omax, omin, obase); break;
        case 7: if constexpr (pk_max_wx<T>() >= 7) pk_band<T, WY, 7>(P, lane, j, head, y0, y1, in, omax, omin, obase); break;
        case 8: if constexpr (pk_max_wx<T>() >= 8) pk_band<T, WY, 8>(P, lane, j, head, y0, y1, in, omax, omin, obase); break;
        default: if constexpr (pk_max_wx<T>() >= 9) pk_band<T, WY, 9>(P, lane, j, head, y0, y1, in, omax, omin, obase); break;
    }
}

template <typename T, int WY> cudaError_t pack2d_launch(cudaStream_t stream, const Pack2DParams &P, unsigned grid) {
    pack2d_kernel<T, WY><<<grid, kPkThreads, 0, stream>>>(P);
    return cudaGetLastError();
}

}  // namespace mmf

#define MMF_INSTANTIATE_PACK2D(T, WY) \
    template cudaError_t mmf::pack2d_launch<T, WY>(cudaStream_t, const mmf::Pack2DParams &, unsigned);
