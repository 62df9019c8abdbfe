// Column pass of the separable 2D filter (Section 1: the 2D filter is the 1D
// filter on rows, then on columns).  Each thread streams CPT adjacent columns
// of one image down the rows in tiles of 8 rows, so consecutive threads touch
// consecutive columns (coalesced rows) and no two threads share state: no CTA
// barrier at all.
//
//   wy <= 9  (slide): outputs of rows 8c..8c+7 are the window max over the
//            current and the next 8-row tile held in registers (pairwise
//            doubling, the naive row of Table 1).
//   wy >= 10 (blocks of 8 rows, van Herk / Gil-Werman, Section 2): with
//            s = wy-1 = 8q + r, row j = 8c+i has k = j+s in tile c+q or
//            c+q+1, and max[j] = max(S_c[i], tiles c+1 .. c+q-1 (or c+q),
//            P(k)), where S is the suffix max inside tile c (the J tile, read
//            again from memory), P the prefix max inside k's tile (a 2-slot
//            per-thread ring in shared memory) and the tiles between come from
//            a per-thread ring of tile aggregates.  That range slides by one
//            tile per step; it is kept as a two-stack queue inside the ring:
//            the older part holds suffix maxima (rebuilt in place when it runs
//            empty), the newer part raw aggregates with a running max, so each
//            step costs O(1) amortised whatever wy.
// The max side reads `src_max` and the min side `src_min` (the row-pass
// outputs, or the image itself when the row window is 1).  The fused form
// (FUSED = true) reads the image only: each 8-row tile of row-pass values is
// computed in registers as the maximum and minimum over wx consecutive image
// elements of each row (neighbouring threads read overlapping elements, which
// the L1 cache serves), so no intermediate reaches memory.
#pragma once
#include <cstdint>

#include "blockscan.cuh"

namespace mmf {

struct ColParams {
    const void *src_max;
    const void *src_min;
    void *out_max;
    void *out_min;
    int64_t nimg, H, Wc;          // images, rows, columns of the column pass
    int64_t in_pitch, in_img;     // element strides (row, image) of the sources
    int64_t out_pitch, out_img;   // element strides of the outputs
    int32_t wy;                   // column window
    int32_t wx;                   // fused: row window (the sources are the image)
    int32_t strips;               // column strips per image
    int32_t qcap;                 // tile-aggregate ring entries per thread (>= q+2)
    uint32_t *status;
    int64_t src_elems, out_elems; // readable elements from each source, writable from each output
};

constexpr int kColThreads = 256;
constexpr int kColRows = 8;  // rows per tile

// Columns per thread: 2 for 1- and 2-byte types when widths and pointers
// allow paired accesses (wider coalesced rows), else 1.
template <typename T> constexpr int col_cpt_max() { return sizeof(T) >= 4 ? 1 : 2; }

// Vector of CPT elements of one row (one load / store per row and thread).
template <typename T, int CPT> struct RowVec;
template <typename T> struct RowVec<T, 1> {
    using R = typename Elem<T>::R;
    __device__ static void load(const T *p, R (&v)[1]) { v[0] = Elem<T>::load(__ldg(p)); }
    __device__ static void store(T *p, const R (&v)[1]) { __stcs(p, Elem<T>::store(v[0])); }
};
template <> struct RowVec<uint8_t, 2> {
    using R = int;
    __device__ static void load(const uint8_t *p, R (&v)[2]) {
        const uint32_t u = __ldg(reinterpret_cast<const unsigned short *>(p));
        v[0] = u & 0xff;
        v[1] = (u >> 8) & 0xff;
    }
    __device__ static void store(uint8_t *p, const R (&v)[2]) {
        const unsigned short u = (unsigned short)((v[0] & 0xff) | ((v[1] & 0xff) << 8));
        *reinterpret_cast<unsigned short *>(p) = u;
    }
};
template <> struct RowVec<int16_t, 2> {
    using R = int;
    __device__ static void load(const int16_t *p, R (&v)[2]) {
        const uint32_t u = __ldg(reinterpret_cast<const unsigned int *>(p));
        v[0] = (int16_t)(u & 0xffff);
        v[1] = (int16_t)(u >> 16);
    }
    __device__ static void store(int16_t *p, const R (&v)[2]) {
        const uint32_t u = (uint32_t)(uint16_t)v[0] | ((uint32_t)(uint16_t)v[1] << 16);
        __stcs(reinterpret_cast<unsigned int *>(p), u);
    }
};

template <typename T> struct ColSmem {
    using Pair = typename Elem<T>::Pair;
    // P ring [2 slots][8 rows][CPT][threads] and aggregates [qcap][CPT][threads].
    static size_t bytes(int qcap, int cpt) {
        return (size_t)(2 * kColRows + qcap) * cpt * kColThreads * sizeof(Pair);
    }
};

extern __shared__ __align__(16) uint8_t col_smem[];

// Loads one 8-row tile (rows y..y+7 of this thread's columns) of one source;
// rows outside [0, H) read as the identity `pad`.
// base, elems: the source buffer (range checks of a checked build).
template <typename T, int CPT>
__device__ __forceinline__ void col_tile(const ColParams &P, const T *base, const T *col, int64_t pitch, int64_t y,
                                         int64_t H, typename Elem<T>::R pad,
                                         typename Elem<T>::R (&v)[kColRows][CPT]) {
#pragma unroll
    for (int r = 0; r < kColRows; ++r) {
        if (y + r >= 0 && y + r < H &&
            in_bytes(P.status, col + (y + r) * pitch, CPT * (int)sizeof(T), base, P.src_elems * (int64_t)sizeof(T))) {
            RowVec<T, CPT>::load(col + (y + r) * pitch, v[r]);
        } else {
#pragma unroll
            for (int c = 0; c < CPT; ++c) v[r][c] = pad;
        }
    }
}

// Tile sources: the row-pass intermediates, or the image itself (fused).
template <typename T, int CPT> struct SepSrc {
    using R = typename Elem<T>::R;
    const T *smax, *smin;
    int64_t pitch, H;
    const ColParams *P;
    __device__ __forceinline__ void tile(int64_t y, R (&vm)[kColRows][CPT], R (&vn)[kColRows][CPT]) const {
        col_tile<T, CPT>(*P, reinterpret_cast<const T *>(P->src_max), smax, pitch, y, H, Elem<T>::lo(), vm);
        col_tile<T, CPT>(*P, reinterpret_cast<const T *>(P->src_min), smin, pitch, y, H, Elem<T>::hi(), vn);
    }
};

template <typename T, int CPT> struct FusedSrc {
    using R = typename Elem<T>::R;
    const T *img;  // this thread's first column of the image
    int64_t pitch, H;
    int wx;
    const ColParams *P;
    __device__ __forceinline__ R ld(const T *p) const {
        return in_bytes(P->status, p, (int)sizeof(T), P->src_max, P->src_elems * (int64_t)sizeof(T))
                   ? Elem<T>::load(__ldg(p))
                   : R(0);
    }
    __device__ __forceinline__ void tile(int64_t y, R (&vm)[kColRows][CPT], R (&vn)[kColRows][CPT]) const {
#pragma unroll
        for (int r = 0; r < kColRows; ++r) {
            if (y + r >= 0 && y + r < H) {
                const T *row = img + (y + r) * pitch;
                R m[CPT], n[CPT];
#pragma unroll
                for (int c = 0; c < CPT; ++c) m[c] = n[c] = ld(row + c);
                // Elements c+1 .. c+wx-1 of column c; element j serves
                // every column c with c < j <= c + wx - 1.
#pragma unroll 4
                for (int j = 1; j < wx + CPT - 1; ++j) {
                    const R v = ld(row + j);
#pragma unroll
                    for (int c = 0; c < CPT; ++c)
                        if (j >= c + 1 && j <= c + wx - 1) { m[c] = vmax(m[c], v); n[c] = vmin(n[c], v); }
                }
#pragma unroll
                for (int c = 0; c < CPT; ++c) { vm[r][c] = m[c]; vn[r][c] = n[c]; }
            } else {
#pragma unroll
                for (int c = 0; c < CPT; ++c) { vm[r][c] = Elem<T>::lo(); vn[r][c] = Elem<T>::hi(); }
            }
        }
    }
};

// base: the output buffer (range checks of a checked build).
template <typename T, int CPT>
__device__ __forceinline__ void col_store(const ColParams &P, const void *base, T *col, int64_t pitch, int64_t y,
                                          int64_t Ho, const typename Elem<T>::R (&v)[kColRows][CPT]) {
#pragma unroll
    for (int r = 0; r < kColRows; ++r)
        if (y + r < Ho &&
            in_bytes(P.status, col + (y + r) * pitch, CPT * (int)sizeof(T), base, P.out_elems * (int64_t)sizeof(T)))
            RowVec<T, CPT>::store(col + (y + r) * pitch, v[r]);
}

template <typename T, int CPT, int W, typename Src>
__device__ __forceinline__ void col_slide(const ColParams &P, const Src &src, T *omax, T *omin, int64_t Ho) {
    using R = typename Elem<T>::R;
    constexpr int P2 = W >= 8 ? 8 : (W >= 4 ? 4 : (W >= 2 ? 2 : 1));
    R cm[kColRows][CPT], cn[kColRows][CPT];  // current tile
    src.tile(0, cm, cn);
    for (int64_t y = 0; y < Ho; y += kColRows) {
        R nm[kColRows][CPT], nn[kColRows][CPT];  // next tile
        src.tile(y + kColRows, nm, nn);
        R om[kColRows][CPT], on[kColRows][CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            R am[2 * kColRows], an[2 * kColRows];
#pragma unroll
            for (int r = 0; r < kColRows; ++r) {
                am[r] = cm[r][c]; am[r + kColRows] = nm[r][c];
                an[r] = cn[r][c]; an[r + kColRows] = nn[r][c];
            }
#pragma unroll
            for (int p = 1; p < P2; p <<= 1) {
#pragma unroll
                for (int i = 0; i + p < 2 * kColRows; ++i) { am[i] = vmax(am[i], am[i + p]); an[i] = vmin(an[i], an[i + p]); }
            }
#pragma unroll
            for (int r = 0; r < kColRows; ++r) {
                om[r][c] = W > P2 ? vmax(am[r], am[r + W - P2]) : am[r];
                on[r][c] = W > P2 ? vmin(an[r], an[r + W - P2]) : an[r];
            }
        }
        if (omax) col_store<T, CPT>(P, P.out_max, omax, P.out_pitch, y, Ho, om);
        if (omin) col_store<T, CPT>(P, P.out_min, omin, P.out_pitch, y, Ho, on);
#pragma unroll
        for (int r = 0; r < kColRows; ++r)
#pragma unroll
            for (int c = 0; c < CPT; ++c) { cm[r][c] = nm[r][c]; cn[r][c] = nn[r][c]; }
    }
}

template <typename T, int CPT, typename Src>
__device__ __forceinline__ void col_blocks(const ColParams &P, const Src &src, T *omax, T *omin, int64_t Ho) {
    using R = typename Elem<T>::R;
    using Pair = typename Elem<T>::Pair;
    const int tid = threadIdx.x;
    const int s = P.wy - 1;
    const int q = s >> 3, rr = s & 7;
    const int qcap = P.qcap;
    Pair *ring = reinterpret_cast<Pair *>(col_smem);                      // [2][8][CPT][NT]
    Pair *ta = ring + 2 * kColRows * CPT * kColThreads;                   // [qcap][CPT][NT]
    auto RP = [&](int slot, int r, int c) -> Pair & { return ring[((slot * kColRows + r) * CPT + c) * kColThreads + tid]; };
    auto TA = [&](int x, int c) -> Pair & { return ta[((x % qcap) * CPT + c) * kColThreads + tid]; };

    // Prefix scan inside a tile; P to ring slot, aggregate to the ring of tile aggregates.
    auto k_tile = [&](int x, R (&km)[kColRows][CPT], R (&kn)[kColRows][CPT]) {
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
#pragma unroll
            for (int r = 1; r < kColRows; ++r) {
                km[r][c] = vmax(km[r - 1][c], km[r][c]);
                kn[r][c] = vmin(kn[r - 1][c], kn[r][c]);
            }
#pragma unroll
            for (int r = 0; r < kColRows; ++r) RP(x & 1, r, c) = Elem<T>::pair(km[r][c], kn[r][c]);
            TA(x, c) = Elem<T>::pair(km[kColRows - 1][c], kn[kColRows - 1][c]);
        }
    };

    // Prologue: tiles 1 .. q (P of tile q stays in the ring).
    for (int x = 1; x <= q; ++x) {
        R km[kColRows][CPT], kn[kColRows][CPT];
        src.tile((int64_t)x * kColRows, km, kn);
        k_tile(x, km, kn);
    }
    const int NC = (int)((Ho + kColRows - 1) / kColRows);
    // Prefetched K tile (c+q+1) and J tile (c) of the next iteration.
    R km[kColRows][CPT], kn[kColRows][CPT], jm[kColRows][CPT], jn[kColRows][CPT];
    src.tile((int64_t)(q + 1) * kColRows, km, kn);
    src.tile(0, jm, jn);
    // Two-stack queue over tile aggregates for the range [c+1, c+q-1] (empty
    // when q < 2): ring slots [fs, fe) hold suffix maxima up to fe-1, slots
    // [fe, be) raw aggregates whose running max is (bm, bn).
    int fs = 1, fe = 1, be = 1;
    R bm[CPT], bn[CPT];
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) { bm[cc] = Elem<T>::lo(); bn[cc] = Elem<T>::hi(); }
    auto push = [&](int x) {  // tile x joins the newer part
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
            const Pair a = TA(x, cc);
            bm[cc] = vmax(bm[cc], Elem<T>::pmax(a));
            bn[cc] = vmin(bn[cc], Elem<T>::pmin(a));
        }
        be = x + 1;
    };
    if (q >= 2)
        for (int x = 1; x <= q - 1; ++x) push(x);
    for (int c = 0; c < NC; ++c) {
        if (c > 0 && q >= 2) {
            ++fs;             // tile c leaves the range
            push(c + q - 1);  // tile c+q-1 joins it
            if (fs >= fe) {
                // Older part empty: the newer part becomes suffix maxima in place.
#pragma unroll
                for (int cc = 0; cc < CPT; ++cc) {
                    R m = Elem<T>::lo(), n = Elem<T>::hi();
                    for (int x = be - 1; x >= fs; --x) {
                        Pair &a = TA(x, cc);
                        m = vmax(m, Elem<T>::pmax(a));
                        n = vmin(n, Elem<T>::pmin(a));
                        a = Elem<T>::pair(m, n);
                    }
                    bm[cc] = Elem<T>::lo();
                    bn[cc] = Elem<T>::hi();
                }
                fe = be;
            }
        }
        R cjm[kColRows][CPT], cjn[kColRows][CPT];
#pragma unroll
        for (int r = 0; r < kColRows; ++r)
#pragma unroll
            for (int cc = 0; cc < CPT; ++cc) { cjm[r][cc] = jm[r][cc]; cjn[r][cc] = jn[r][cc]; }
        k_tile(c + q + 1, km, kn);
        if (c + 1 < NC) {  // prefetch the next iteration's tiles
            src.tile((int64_t)(c + q + 2) * kColRows, km, kn);
            src.tile((int64_t)(c + 1) * kColRows, jm, jn);
        }
        R om[kColRows][CPT], on[kColRows][CPT];
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
            // suffix inside the J tile
#pragma unroll
            for (int r = kColRows - 2; r >= 0; --r) {
                cjm[r][cc] = vmax(cjm[r + 1][cc], cjm[r][cc]);
                cjn[r][cc] = vmin(cjn[r + 1][cc], cjn[r][cc]);
            }
            // tiles strictly between: c+1 .. c+q-1 (near), .. c+q (far)
            R m1 = bm[cc], n1 = bn[cc];
            if (fs < fe) {
                const Pair f = TA(fs, cc);
                m1 = vmax(m1, Elem<T>::pmax(f));
                n1 = vmin(n1, Elem<T>::pmin(f));
            }
            const Pair lastp = TA(c + q, cc);
            const R m2 = vmax(m1, Elem<T>::pmax(lastp)), n2 = vmin(n1, Elem<T>::pmin(lastp));
#pragma unroll
            for (int i = 0; i < kColRows; ++i) {
                const int kr = i + rr;  // row of k within tiles c+q, c+q+1
                const bool far = kr >= kColRows;
                const Pair pk = RP((c + q + (far ? 1 : 0)) & 1, kr & 7, cc);
                om[i][cc] = vmax(vmax(cjm[i][cc], far ? m2 : m1), Elem<T>::pmax(pk));
                on[i][cc] = vmin(vmin(cjn[i][cc], far ? n2 : n1), Elem<T>::pmin(pk));
            }
        }
        if (omax) col_store<T, CPT>(P, P.out_max, omax, P.out_pitch, (int64_t)c * kColRows, Ho, om);
        if (omin) col_store<T, CPT>(P, P.out_min, omin, P.out_pitch, (int64_t)c * kColRows, Ho, on);
    }
}

template <typename T, int CPT, typename Src>
__device__ __forceinline__ void col_dispatch(const ColParams &P, const Src &src, T *omax, T *omin, int64_t Ho) {
    switch (P.wy) {
        case 1: col_slide<T, CPT, 1>(P, src, omax, omin, Ho); break;
        case 2: col_slide<T, CPT, 2>(P, src, omax, omin, Ho); break;
        case 3: col_slide<T, CPT, 3>(P, src, omax, omin, Ho); break;
        case 4: col_slide<T, CPT, 4>(P, src, omax, omin, Ho); break;
        case 5: col_slide<T, CPT, 5>(P, src, omax, omin, Ho); break;
        case 6: col_slide<T, CPT, 6>(P, src, omax, omin, Ho); break;
        case 7: col_slide<T, CPT, 7>(P, src, omax, omin, Ho); break;
        case 8: col_slide<T, CPT, 8>(P, src, omax, omin, Ho); break;
        case 9: col_slide<T, CPT, 9>(P, src, omax, omin, Ho); break;
        default: col_blocks<T, CPT>(P, src, omax, omin, Ho); break;
    }
}

template <typename T, int CPT, bool FUSED>
__global__ void __launch_bounds__(kColThreads) colscan_kernel(const ColParams P) {
    const int64_t img = blockIdx.x / P.strips;
    const int64_t strip = blockIdx.x % P.strips;
    const int64_t x = strip * (kColThreads * CPT) + (int64_t)threadIdx.x * CPT;
    const int64_t Ho = P.H - P.wy + 1;
    if (x >= P.Wc || Ho <= 0 || img >= P.nimg) return;  // no barriers below
    T *omax = P.out_max ? reinterpret_cast<T *>(P.out_max) + img * P.out_img + x : nullptr;
    T *omin = P.out_min ? reinterpret_cast<T *>(P.out_min) + img * P.out_img + x : nullptr;
    if constexpr (FUSED) {
        const FusedSrc<T, CPT> src{reinterpret_cast<const T *>(P.src_max) + img * P.in_img + x, P.in_pitch, P.H,
                                   P.wx, &P};
        col_dispatch<T, CPT>(P, src, omax, omin, Ho);
    } else {
        const SepSrc<T, CPT> src{reinterpret_cast<const T *>(P.src_max) + img * P.in_img + x,
                                 reinterpret_cast<const T *>(P.src_min) + img * P.in_img + x, P.in_pitch, P.H, &P};
        col_dispatch<T, CPT>(P, src, omax, omin, Ho);
    }
}

}  // namespace mmf
