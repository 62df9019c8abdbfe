// Fused separable 2D filter for windows up to kTileMaxW x kTileMaxW (Section
// 1: rows, then columns), one output tile of kTR x kTC pixels per CTA.
//
//   1. the input tile with its halo, (kTR + wy - 1) x (kTC + wx - 1) elements,
//      is read once into shared memory (coalesced rows; zeros outside the
//      image, which only reach outputs outside it);
//   2. row pass: each thread takes runs of 8 outputs of one row and computes
//      their window maxima and minima from registers by pairwise doubling (the
//      naive row of Table 1 shared between neighbouring windows); the results
//      go to two shared tiles;
//   3. column pass: each thread takes runs of 8 rows of one column of those
//      tiles, the same doubling, and writes the outputs (consecutive threads,
//      consecutive columns: coalesced rows).
// Nothing but the image and the outputs touches global memory.  The doubling
// depth P2 (the largest power of two <= w) selects a compiled pass; the
// remainder w - P2 selects compile-time offsets (uniform over the CTA).
#pragma once
#include <cstdint>

#include "blockscan.cuh"

namespace mmf {

constexpr int kTileMaxW = 31;  // largest window in either direction
constexpr int kTR = 32;        // output rows per tile
constexpr int kTC = 128;       // output columns per tile
constexpr int kTThreads = 256;
constexpr int kRun = 8;                        // outputs per thread run
constexpr int kRS = kTC + 1;                   // row-pass tile row stride (odd: conflict-free columns)

struct Tile2DParams {
    const void *in;
    void *out_max, *out_min;
    int64_t nimg, H, W, pitch, img_stride;  // input geometry (elements)
    int64_t Ho, Wo;                         // outputs: image k row y at out + (k*Ho + y)*Wo
    int32_t wy, wx;
    int32_t tiles_x, tiles_y;
    int32_t xs;                  // input tile row stride in shared memory (odd)
    int32_t x_bytes, r_bytes;    // shared-memory regions (16-byte multiples)
#ifdef MMF_CHECKED
    uint32_t *status;            // device status word (range checks)
    int64_t in_elems, out_elems; // readable elements from `in`, writable from each output
#endif
};

// Range checks of a checked build.  Its fields exist only there: with them,
// the ordinary build's one-tile kernels ran up to 20 % slower (3 x 3) although
// the checks themselves compile away.
#ifdef MMF_CHECKED
#define MMF_TILE_IN_OK(P, p) in_bytes((P).status, (p), (int)sizeof(T), (P).in, (P).in_elems * (int64_t)sizeof(T))
#define MMF_TILE_OUT_OK(P, base, p) \
    in_bytes((P).status, (p), (int)sizeof(T), (base), (P).out_elems * (int64_t)sizeof(T))
#else
#define MMF_TILE_IN_OK(P, p) true
#define MMF_TILE_OUT_OK(P, base, p) true
#endif

// Shared memory of one tile for windows wy x wx: the input tile and the two
// row-pass tiles, sized for these windows.
template <typename T> struct Tile2DSmem {
    static int xs(int wx) { return (kTC + wx - 1) | 1; }
    static size_t x_bytes(int wy, int wx) { return ((size_t)(kTR + wy - 1) * xs(wx) * sizeof(T) + 15) / 16 * 16; }
    static size_t r_bytes(int wy) { return ((size_t)(kTR + wy - 1) * kRS * sizeof(T) + 15) / 16 * 16; }
    static size_t bytes(int wy, int wx) { return x_bytes(wy, wx) + 2 * r_bytes(wy); }
};

extern __shared__ __align__(16) uint8_t tile2d_smem[];

// Largest power of two <= w (w in [1, 31]).
__host__ __device__ inline int pow2_floor(int w) { return w >= 16 ? 16 : (w >= 8 ? 8 : (w >= 4 ? 4 : (w >= 2 ? 2 : 1))); }

// Window extremes of kRun consecutive positions from the values a[0..NE)
// (max side) and b[0..NE) (min side), window P2 + r (0 <= r < P2): after the
// doubling passes a[i] covers [i, i + P2), and the window [i, i + P2 + r) is
// the union of a[i] and a[i + r].
template <typename R, int P2>
__device__ __forceinline__ void run_windows(R (&a)[kRun + 2 * P2], R (&b)[kRun + 2 * P2], int r, R (&om)[kRun],
                                            R (&on)[kRun]) {
    constexpr int NE = kRun + 2 * P2;
#pragma unroll
    for (int p = 1; p < P2; p <<= 1) {
#pragma unroll
        for (int i = 0; i + p < NE; ++i) { a[i] = vmax(a[i], a[i + p]); b[i] = vmin(b[i], b[i + p]); }
    }
#pragma unroll
    for (int k = 0; k < P2; ++k) {
        if (k == r) {
#pragma unroll
            for (int i = 0; i < kRun; ++i) {
                om[i] = vmax(a[i], a[i + k]);
                on[i] = vmin(b[i], b[i + k]);
            }
        }
    }
}

// Row pass with doubling depth P2: rows_in rows x kTC/kRun runs; consecutive
// threads take consecutive rows (odd row stride: no bank conflicts).
template <typename T, int P2>
__device__ __forceinline__ void tile_rows(const T *X, int xs, T *RM, T *RN, int rows_in, int cols_in, int r) {
    using R = typename Elem<T>::R;
    constexpr int NE = kRun + 2 * P2;
    for (int task = threadIdx.x; task < rows_in * (kTC / kRun); task += kTThreads) {
        const int row = task % rows_in, c0 = (task / rows_in) * kRun;
        R a[NE], b[NE];
#pragma unroll
        for (int i = 0; i < NE; ++i) {
            const int c = c0 + i;
            a[i] = b[i] = Elem<T>::load(c < cols_in ? X[row * xs + c] : T(0));
        }
        R om[kRun], on[kRun];
        run_windows<R, P2>(a, b, r, om, on);
#pragma unroll
        for (int i = 0; i < kRun; ++i) {
            RM[row * kRS + c0 + i] = Elem<T>::store(om[i]);
            RN[row * kRS + c0 + i] = Elem<T>::store(on[i]);
        }
    }
}

// Column pass with doubling depth P2: kTC columns x kTR/kRun runs;
// consecutive threads take consecutive columns (coalesced output rows).
template <typename T, int P2>
__device__ __forceinline__ void tile_cols(const T *RM, const T *RN, int rows_in, int r, const Tile2DParams &P,
                                          T *omax, T *omin, int64_t y0, int64_t x0) {
    using R = typename Elem<T>::R;
    constexpr int NE = kRun + 2 * P2;
    for (int task = threadIdx.x; task < kTC * (kTR / kRun); task += kTThreads) {
        const int c = task % kTC, r0 = (task / kTC) * kRun;
        const int64_t x = x0 + c;
        if (x >= P.Wo || y0 + r0 >= P.Ho) continue;
        R a[NE], b[NE];
#pragma unroll
        for (int i = 0; i < NE; ++i) {
            const int row = r0 + i;
            const bool in = row < rows_in;
            a[i] = Elem<T>::load(in ? RM[row * kRS + c] : T(0));
            b[i] = Elem<T>::load(in ? RN[row * kRS + c] : T(0));
        }
        R om[kRun], on[kRun];
        run_windows<R, P2>(a, b, r, om, on);
#pragma unroll
        for (int i = 0; i < kRun; ++i) {
            const int64_t y = y0 + r0 + i;
            if (y < P.Ho) {
                if (omax && MMF_TILE_OUT_OK(P, P.out_max, omax + y * P.Wo + x))
                    omax[y * P.Wo + x] = Elem<T>::store(om[i]);
                if (omin && MMF_TILE_OUT_OK(P, P.out_min, omin + y * P.Wo + x))
                    omin[y * P.Wo + x] = Elem<T>::store(on[i]);
            }
        }
    }
}

// PMAX: the largest doubling depth of the two windows.  Registers scale with
// it (two runs of kRun + 2 PMAX values), so small windows keep more CTAs per
// SM; 8-byte values take twice the registers.
template <typename T, int PMAX> constexpr int tile_min_blocks() {
    return sizeof(T) == 8 ? (PMAX <= 2 ? 3 : (PMAX <= 8 ? 2 : 1)) : (PMAX <= 2 ? 4 : (PMAX <= 8 ? 3 : 2));
}

template <typename T, int PMAX>
__global__ void __launch_bounds__(kTThreads, (tile_min_blocks<T, PMAX>())) tile2d_kernel(const Tile2DParams P) {
    T *X = reinterpret_cast<T *>(tile2d_smem);
    T *RM = reinterpret_cast<T *>(tile2d_smem + P.x_bytes);
    T *RN = reinterpret_cast<T *>(tile2d_smem + P.x_bytes + P.r_bytes);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t tiles_per_img = (int64_t)P.tiles_x * P.tiles_y;
    const int64_t img = blockIdx.x / tiles_per_img;
    const int64_t t = blockIdx.x % tiles_per_img;
    const int64_t y0 = (t / P.tiles_x) * kTR, x0 = (t % P.tiles_x) * kTC;
    const int wy = P.wy, wx = P.wx, xs = P.xs;
    const int rows_in = kTR + wy - 1, cols_in = kTC + wx - 1;
    const T *src = reinterpret_cast<const T *>(P.in) + img * P.img_stride;

    // 1. Input tile (positions outside the image read as 0: they only feed
    // outputs outside the image, which are not stored).
    for (int r = warp; r < rows_in; r += kTThreads / 32) {
        const int64_t y = y0 + r;
        const T *row = src + y * P.pitch + x0;
        for (int c = lane; c < cols_in; c += 32)
            X[r * xs + c] = (y < P.H && x0 + c < P.W && MMF_TILE_IN_OK(P, row + c)) ? __ldg(row + c) : T(0);
    }
    __syncthreads();

    // 2. Row pass.
    const int px = pow2_floor(wx), py = pow2_floor(wy);
    switch (px) {
        case 1: tile_rows<T, 1>(X, xs, RM, RN, rows_in, cols_in, wx - 1); break;
        case 2: if constexpr (PMAX >= 2) tile_rows<T, 2>(X, xs, RM, RN, rows_in, cols_in, wx - 2); break;
        case 4: if constexpr (PMAX >= 4) tile_rows<T, 4>(X, xs, RM, RN, rows_in, cols_in, wx - 4); break;
        case 8: if constexpr (PMAX >= 8) tile_rows<T, 8>(X, xs, RM, RN, rows_in, cols_in, wx - 8); break;
        default: if constexpr (PMAX >= 16) tile_rows<T, 16>(X, xs, RM, RN, rows_in, cols_in, wx - 16); break;
    }
    __syncthreads();

    // 3. Column pass.
    T *omax = P.out_max ? reinterpret_cast<T *>(P.out_max) + img * P.Ho * P.Wo : nullptr;
    T *omin = P.out_min ? reinterpret_cast<T *>(P.out_min) + img * P.Ho * P.Wo : nullptr;
    switch (py) {
        case 1: tile_cols<T, 1>(RM, RN, rows_in, wy - 1, P, omax, omin, y0, x0); break;
        case 2: if constexpr (PMAX >= 2) tile_cols<T, 2>(RM, RN, rows_in, wy - 2, P, omax, omin, y0, x0); break;
        case 4: if constexpr (PMAX >= 4) tile_cols<T, 4>(RM, RN, rows_in, wy - 4, P, omax, omin, y0, x0); break;
        case 8: if constexpr (PMAX >= 8) tile_cols<T, 8>(RM, RN, rows_in, wy - 8, P, omax, omin, y0, x0); break;
        default: if constexpr (PMAX >= 16) tile_cols<T, 16>(RM, RN, rows_in, wy - 16, P, omax, omin, y0, x0); break;
    }
}

// Persistent form for small windows (doubling depth PMAX, used for f32
// windows up to 3): each thread keeps its share of the next tile's input in
// registers (rows warp + 8i, columns lane + 32j), so the loads of the next
// tile are in flight while this one is filtered; the one-tile kernel above
// waits for its loads with nothing else to do (ncu on f32 3x3: the global-load
// wait was the largest stall).
template <int PMAX> struct TilePf {
    static constexpr int ROWS = kTR + 2 * PMAX - 1;  // rows_in for windows below 2·PMAX
    static constexpr int COLS = kTC + 2 * PMAX - 1;
    static constexpr int RPW = (ROWS + 7) / 8;       // rows per warp (8 warps)
    static constexpr int CPL = (COLS + 31) / 32;     // columns per lane
};

// Image, first output row and first output column of tile `tile`.
__device__ __forceinline__ void tile_origin(const Tile2DParams &P, int64_t tile, int64_t &img, int64_t &y0,
                                            int64_t &x0) {
    const int64_t per_img = (int64_t)P.tiles_x * P.tiles_y;
    img = tile / per_img;
    const int64_t t = tile - img * per_img;
    y0 = (t / P.tiles_x) * kTR;
    x0 = (t % P.tiles_x) * kTC;
}

template <typename T, int PMAX>
__device__ __forceinline__ void tile_pf_load(const Tile2DParams &P, int64_t tile, int rows_in, int cols_in, int warp,
                                             int lane, T (&v)[TilePf<PMAX>::RPW][TilePf<PMAX>::CPL]) {
    int64_t img, y0, x0;
    tile_origin(P, tile, img, y0, x0);
    const T *src = reinterpret_cast<const T *>(P.in) + img * P.img_stride;
#pragma unroll
    for (int i = 0; i < TilePf<PMAX>::RPW; ++i) {
        const int r = warp + 8 * i;
        const int64_t y = y0 + r;
        const T *row = src + y * P.pitch + x0;
#pragma unroll
        for (int j = 0; j < TilePf<PMAX>::CPL; ++j) {
            const int c = lane + 32 * j;
            v[i][j] = (r < rows_in && c < cols_in && y < P.H && x0 + c < P.W && MMF_TILE_IN_OK(P, row + c))
                          ? __ldg(row + c)
                          : T(0);
        }
    }
}

template <typename T, int PMAX>
__global__ void __launch_bounds__(kTThreads, 2) tile2d_pf_kernel(const Tile2DParams P) {
    using F = TilePf<PMAX>;
    T *X = reinterpret_cast<T *>(tile2d_smem);
    T *RM = reinterpret_cast<T *>(tile2d_smem + P.x_bytes);
    T *RN = reinterpret_cast<T *>(tile2d_smem + P.x_bytes + P.r_bytes);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wy = P.wy, wx = P.wx, xs = P.xs;
    const int rows_in = kTR + wy - 1, cols_in = kTC + wx - 1;
    const int64_t total = P.nimg * P.tiles_x * P.tiles_y;
    const int px = pow2_floor(wx), py = pow2_floor(wy);
    T v[F::RPW][F::CPL];
    int64_t tile = blockIdx.x;
    if (tile < total) tile_pf_load<T, PMAX>(P, tile, rows_in, cols_in, warp, lane, v);
    for (; tile < total; tile += gridDim.x) {
#pragma unroll
        for (int i = 0; i < F::RPW; ++i) {
            const int r = warp + 8 * i;
#pragma unroll
            for (int j = 0; j < F::CPL; ++j) {
                const int c = lane + 32 * j;
                if (r < rows_in && c < cols_in) X[r * xs + c] = v[i][j];
            }
        }
        __syncthreads();
        const int64_t next = tile + gridDim.x;
        if (next < total) tile_pf_load<T, PMAX>(P, next, rows_in, cols_in, warp, lane, v);
        switch (px) {
            case 1: tile_rows<T, 1>(X, xs, RM, RN, rows_in, cols_in, wx - 1); break;
            case 2: tile_rows<T, 2>(X, xs, RM, RN, rows_in, cols_in, wx - 2); break;
            default: if constexpr (PMAX >= 4) tile_rows<T, 4>(X, xs, RM, RN, rows_in, cols_in, wx - 4); break;
        }
        __syncthreads();
        int64_t img, y0, x0;
        tile_origin(P, tile, img, y0, x0);
        T *omax = P.out_max ? reinterpret_cast<T *>(P.out_max) + img * P.Ho * P.Wo : nullptr;
        T *omin = P.out_min ? reinterpret_cast<T *>(P.out_min) + img * P.Ho * P.Wo : nullptr;
        switch (py) {
            case 1: tile_cols<T, 1>(RM, RN, rows_in, wy - 1, P, omax, omin, y0, x0); break;
            case 2: tile_cols<T, 2>(RM, RN, rows_in, wy - 2, P, omax, omin, y0, x0); break;
            default: if constexpr (PMAX >= 4) tile_cols<T, 4>(RM, RN, rows_in, wy - 4, P, omax, omin, y0, x0); break;
        }
        __syncthreads();  // X, RM and RN are rewritten for the next tile
    }
}

}  // namespace mmf
