// Separable 2D running max-min filter (Section 1: the 1D filter on rows, then
// on columns), valid windows: out[y][x] = max over rows y..y+wy-1 and columns
// x..x+wx-1.  Row pass: the 1D block-scan kernel over all rows read as one
// series (or row by row when the workspace is too small for the input's
// pitch).  Column pass: colscan_kernel (one thread per column).  The row-pass
// intermediates go to a caller-provided workspace; the fused forms (tile,
// register-streaming, row extremes inside the column pass) need none.
#include <cstring>
#include <type_traits>

#include "colscan.cuh"
#include "pack2d.h"
#include "tile2d.cuh"
#include "launch.h"
#include "mmf.h"

namespace mmf {
mmf_status set_error(mmf_status st, const char *fmt, ...);
mmf_status cuda_error(cudaError_t e, const char *what);
mmf_status get_ctx(void *stream, LaunchCtx *ctx);
int elem_size(mmf_dtype dt);

template <typename T> static int col_qcap(int64_t wy) { return wy >= 10 ? (int)((wy - 1) / 8) + 2 : 0; }

template <typename T> static size_t col_smem_bytes(int64_t wy, int cpt = col_cpt_max<T>()) {
    return ColSmem<T>::bytes(col_qcap<T>(wy), cpt);
}

template <typename T, int CPT, bool FUSED> static cudaError_t col_launch_cpt(const LaunchCtx &ctx, ColParams P) {
    P.strips = (int)((P.Wc + kColThreads * CPT - 1) / (kColThreads * CPT));
    P.qcap = col_qcap<T>(P.wy);
    P.status = ctx.status;
    const size_t smem = col_smem_bytes<T>(P.wy, CPT);
    static size_t set[64] = {0};
    if (smem > set[ctx.device]) {
        cudaError_t e = cudaFuncSetAttribute(colscan_kernel<T, CPT, FUSED>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set[ctx.device] = smem;
    }
    const int64_t grid = P.nimg * P.strips;
    if (grid <= 0) return cudaSuccess;
    colscan_kernel<T, CPT, FUSED><<<(unsigned)grid, kColThreads, smem, ctx.stream>>>(P);
    return cudaGetLastError();
}

// Paired columns when every row start and the width allow it (the fused
// form reads single elements, so only its outputs need pairing).
template <typename T> static cudaError_t col_launch(const LaunchCtx &ctx, const ColParams &P, bool fused) {
    if constexpr (col_cpt_max<T>() == 2) {
        const uintptr_t a = 2 * sizeof(T) - 1;
        const bool out_ok = P.Wc % 2 == 0 && P.out_pitch % 2 == 0 && P.out_img % 2 == 0 &&
                            ((uintptr_t)P.out_max & a) == 0 && ((uintptr_t)P.out_min & a) == 0;
        const bool in_ok = P.in_pitch % 2 == 0 && P.in_img % 2 == 0 && ((uintptr_t)P.src_max & a) == 0 &&
                           ((uintptr_t)P.src_min & a) == 0;
        if (fused && out_ok) return col_launch_cpt<T, 2, true>(ctx, P);
        if (!fused && out_ok && in_ok) return col_launch_cpt<T, 2, false>(ctx, P);
    }
    return fused ? col_launch_cpt<T, 1, true>(ctx, P) : col_launch_cpt<T, 1, false>(ctx, P);
}

// Fused forms: the tile kernel (halo tile in shared memory) for windows up to
// kTileMaxW in both directions, automatically and on request; beyond that, on
// request (fuse = 1, wx <= MMF_FUSED_MAX_WX), the column pass with row
// maxima computed per row in registers.
static bool tile_fits(int64_t wy, int64_t wx) { return wy <= kTileMaxW && wx <= kTileMaxW; }
// The automatic choice takes the tile kernel up to windows of 12 (4- and
// 8-byte elements) or 15 (1- and 2-byte): above that its halo and doubling
// passes cost more than the row pass (one series over all rows) and the
// column pass together (measured on 32-64 images of 4096 x 4096).
static bool use_fused(int64_t wy, int64_t wx, int fuse, int esz) {
    if (wy == 1 || wx == 1) return false;  // a single pass already
    const int64_t auto_max = esz >= 4 ? 12 : 15;
    return fuse == 1 || fuse == 2 || (fuse < 0 && tile_fits(wy, wx) && wy <= auto_max && wx <= auto_max);
}

// The register-streaming kernel (u8, i16 packed; f32; windows up to
// kPkMaxWy x pk_max_wx, input rows 4-byte aligned: pointer, pitch and image
// stride).
template <typename T> constexpr bool pack_type() { return sizeof(T) <= 2 || std::is_same<T, float>::value; }
template <typename T>
static bool pack_applies(const T *in, int64_t H, int64_t pitch, int64_t wy, int64_t wx) {
    if constexpr (!pack_type<T>()) {
        return false;
    } else {
        const int64_t rowb = pitch * (int64_t)sizeof(T);
        return wy <= kPkMaxWy && wx <= pk_max_wx<T>() && ((uintptr_t)in & 3) == 0 && rowb % 4 == 0 &&
               (H * rowb) % 4 == 0;
    }
}

template <typename T>
static cudaError_t pack_launch(const LaunchCtx &ctx, const T *in, int64_t nimg, int64_t H, int64_t W, int64_t pitch,
                               int64_t wy, int64_t wx, T *omax, T *omin) {
    if constexpr (!pack_type<T>()) {
        return cudaErrorInvalidValue;
    } else {
        Pack2DParams P{};
        P.in = in;
        P.out_max = omax;
        P.out_min = omin;
        P.nimg = nimg;
        P.H = H;
        P.W = W;
        P.pitch = pitch;
        P.img_stride = H * pitch;
        P.Ho = H - wy + 1;
        P.Wo = W - wx + 1;
        P.wy = (int)wy;
        P.wx = (int)wx;
        P.status = ctx.status;
        P.in_bytes = ((nimg - 1) * P.img_stride + (H - 1) * pitch + W) * (int64_t)sizeof(T);
        P.out_bytes = nimg * P.Ho * P.Wo * (int64_t)sizeof(T);
        constexpr int L = 4 / (int)sizeof(T);  // columns per 32-bit word
        const int64_t words = (P.Wo + L - 1) / L;
        const int chunk = pk_chunk<T>((int)wx);
        P.nchunks = (int)((words + chunk - 1) / chunk);
        P.nbands = (int)((P.Ho + kPkBand - 1) / kPkBand);
        P.tasks = nimg * P.nbands * P.nchunks;
        const int64_t grid = (P.tasks + kPkThreads / 32 - 1) / (kPkThreads / 32);
        if (grid <= 0) return cudaSuccess;
        if (grid > 0x7fffffff) return cudaErrorInvalidValue;
        switch (wy) {
            case 1: return pack2d_launch<T, 1>(ctx.stream, P, (unsigned)grid);
            case 2: return pack2d_launch<T, 2>(ctx.stream, P, (unsigned)grid);
            case 3: return pack2d_launch<T, 3>(ctx.stream, P, (unsigned)grid);
            case 4: return pack2d_launch<T, 4>(ctx.stream, P, (unsigned)grid);
            case 5: return pack2d_launch<T, 5>(ctx.stream, P, (unsigned)grid);
            case 6: return pack2d_launch<T, 6>(ctx.stream, P, (unsigned)grid);
            case 7: return pack2d_launch<T, 7>(ctx.stream, P, (unsigned)grid);
            case 8: return pack2d_launch<T, 8>(ctx.stream, P, (unsigned)grid);
            default: return pack2d_launch<T, 9>(ctx.stream, P, (unsigned)grid);
        }
    }
}

template <typename T>
static cudaError_t tile_launch(const LaunchCtx &ctx, const T *in, int64_t nimg, int64_t H, int64_t W, int64_t pitch,
                               int64_t wy, int64_t wx, T *omax, T *omin) {
    Tile2DParams P{};
    P.in = in;
    P.out_max = omax;
    P.out_min = omin;
    P.nimg = nimg;
    P.H = H;
    P.W = W;
    P.pitch = pitch;
    P.img_stride = H * pitch;
    P.Ho = H - wy + 1;
    P.Wo = W - wx + 1;
    P.wy = (int)wy;
    P.wx = (int)wx;
    P.tiles_x = (int)((P.Wo + kTC - 1) / kTC);
    P.tiles_y = (int)((P.Ho + kTR - 1) / kTR);
#ifdef MMF_CHECKED
    P.status = ctx.status;
    P.in_elems = (nimg - 1) * P.img_stride + (H - 1) * pitch + W;
    P.out_elems = nimg * P.Ho * P.Wo;
#endif
    const int64_t grid = nimg * P.tiles_x * P.tiles_y;
    if (grid <= 0) return cudaSuccess;
    if (grid > 0x7fffffff) return cudaErrorInvalidValue;
    P.xs = Tile2DSmem<T>::xs((int)wx);
    P.x_bytes = (int)Tile2DSmem<T>::x_bytes((int)wy, (int)wx);
    P.r_bytes = (int)Tile2DSmem<T>::r_bytes((int)wy);
    const size_t smem = Tile2DSmem<T>::bytes((int)wy, (int)wx);
    const int pmax = pow2_floor((int)(wx > wy ? wx : wy));
    auto go = [&](auto kernel, int slot) -> cudaError_t {
        static size_t set[64][5] = {};
        size_t &have = set[ctx.device & 63][slot];
        if (smem > have) {
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            have = smem;
        }
        kernel<<<(unsigned)grid, kTThreads, smem, ctx.stream>>>(P);
        return cudaGetLastError();
    };
    // Windows up to 7 (f32): the persistent form, one wave of CTAs.
    auto go_pf = [&](auto kernel, int slot) -> cudaError_t {
        static size_t set[64][2] = {};
        static int occ[64][2] = {};
        size_t &have = set[ctx.device & 63][slot];
        int &k = occ[ctx.device & 63][slot];
        if (smem > have) {
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            have = smem;
            k = 0;
        }
        if (k == 0) {
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, kernel, kTThreads, smem);
            if (e != cudaSuccess) return e;
            if (k < 1) k = 1;
        }
        const int64_t wave = (int64_t)(ctx.sms > 0 ? ctx.sms : 1) * k;
        kernel<<<(unsigned)(grid < wave ? grid : wave), kTThreads, smem, ctx.stream>>>(P);
        return cudaGetLastError();
    };
    // f32 windows up to 3: the 1-2 byte types are bound by instructions (the
    // one-tile kernel keeps 4 CTAs per SM to the persistent form's 2), f64
    // and the depth-4 form spill.
    if constexpr (sizeof(T) == 4) {
        if (pmax <= 2) return go_pf(tile2d_pf_kernel<T, 2>, 0);
    }
    switch (pmax) {
        case 1:
        case 2: return go(tile2d_kernel<T, 2>, 0);
        case 4: return go(tile2d_kernel<T, 4>, 1);
        case 8: return go(tile2d_kernel<T, 8>, 2);
        default: return go(tile2d_kernel<T, 16>, 3);
    }
}

// Row pitch of the intermediates: Wo rounded up to 16 elements, so every
// row starts 16-byte aligned.
static int64_t mid_pitch(int64_t Wo) { return (Wo + 15) / 16 * 16; }

template <typename T>
static mmf_status filter2d(const LaunchCtx &ctx, const T *in, int64_t nimg, int64_t H, int64_t W, int64_t pitch,
                           int64_t wy, int64_t wx, int fuse, T *omax, T *omin, void *work, size_t work_bytes) {
    const int64_t Ho = H - wy + 1, Wo = W - wx + 1;
    cudaError_t e = cudaSuccess;
    // Automatic: the streaming kernel for u8/i16 wherever it applies, for f32
    // except rows-only windows of more than 3 (the row pass is faster there).
    const bool auto_pack = sizeof(T) <= 2 || (std::is_same<T, float>::value && !(wy == 1 && wx > 3));
    if (fuse == 2 || (fuse < 0 && auto_pack)) {
        if (pack_applies<T>(in, H, pitch, wy, wx)) {
            e = pack_launch<T>(ctx, in, nimg, H, W, pitch, wy, wx, omax, omin);
            return e == cudaSuccess ? MMF_OK : cuda_error(e, "packed 2D kernel");
        }
        if (fuse == 2)
            return set_error(MMF_ENOTIMPL,
                             "the register-streaming 2D kernel takes u8 and f32 (windows up to %d x 9) and i16 "
                             "(up to %d x 5) with 4-byte aligned rows",
                             kPkMaxWy, kPkMaxWy);
    }
    if (wy == 1) {  // rows only, straight into the outputs
        SeriesDesc sd{0, W, 0, wx, 0, Wo};
        e = blockscan_rows<T>(ctx, in, sd, nimg * H, pitch, Wo, omax, omin);
        return e == cudaSuccess ? MMF_OK : cuda_error(e, "row pass");
    }
    ColParams P{};
    P.out_max = omax;
    P.out_min = omin;
    P.nimg = nimg;
    P.H = H;
    P.Wc = Wo;
    P.out_pitch = Wo;
    P.out_img = Ho * Wo;
    P.out_elems = nimg * Ho * Wo;
    P.wy = (int)wy;
    P.wx = (int)wx;
    const bool fused = use_fused(wy, wx, fuse, (int)sizeof(T));
    if (fused && tile_fits(wy, wx)) {
        e = tile_launch<T>(ctx, in, nimg, H, W, pitch, wy, wx, omax, omin);
        return e == cudaSuccess ? MMF_OK : cuda_error(e, "fused 2D tile");
    }
    if (wx == 1 || fused) {  // columns only (or fused), on the image
        P.src_max = in;
        P.src_min = in;
        P.in_pitch = pitch;
        P.in_img = H * pitch;
        P.src_elems = (nimg - 1) * H * pitch + (H - 1) * pitch + W;
    } else {
        // All rows of all images (stacked, `pitch` apart) read as one series
        // of n elements: the window starting at stream position r*pitch + x
        // is row r's window at column x for x < Wo; the others straddle two
        // rows (or a row's padding) and are never read.  One long series
        // keeps the long-stream schedule (a few long items per CTA) where a
        // series per row gives every CTA many items of two or three tiles.
        // Its intermediates have the input's pitch; when the workspace is
        // too small for that (a pitch above the width), rows one by one.
        const int64_t n = (nimg * H - 1) * pitch + W;
        const int64_t span = mid_pitch(n - wx + 1);
        T *rmax = static_cast<T *>(work);
        if (work_bytes / sizeof(T) >= (size_t)(2 * span)) {
            SeriesDesc sd{0, n, 0, wx, 0, n - wx + 1};
            e = blockscan_1d<T>(ctx, in, sd, rmax, rmax + span, true, 0);
            if (e != cudaSuccess) return cuda_error(e, "row pass");
            P.src_max = rmax;
            P.src_min = rmax + span;
            P.in_pitch = pitch;
            P.in_img = H * pitch;
            P.src_elems = span;
        } else {
            const int64_t wp = mid_pitch(Wo);
            T *rmin = rmax + nimg * H * wp;
            SeriesDesc sd{0, W, 0, wx, 0, Wo};
            e = blockscan_rows<T>(ctx, in, sd, nimg * H, pitch, wp, rmax, rmin);
            if (e != cudaSuccess) return cuda_error(e, "row pass");
            P.src_max = rmax;
            P.src_min = rmin;
            P.in_pitch = wp;
            P.in_img = H * wp;
            P.src_elems = nimg * H * wp;
        }
    }
    e = col_launch<T>(ctx, P, fused);
    return e == cudaSuccess ? MMF_OK : cuda_error(e, "column pass");
}

static mmf_status check2d(int64_t nimg, int64_t H, int64_t W, int64_t pitch, int64_t wy, int64_t wx, mmf_dtype dt,
                          int fuse) {
    if (elem_size(dt) == 0) return set_error(MMF_EINVAL, "unknown dtype %d", (int)dt);
    if (nimg < 0 || H < 0 || W < 0 || pitch < W) return set_error(MMF_EINVAL, "bad image geometry");
    if (wy < 1 || wx < 1) return set_error(MMF_EINVAL, "windows must be >= 1");
    if (fuse < -1 || fuse > 2) return set_error(MMF_EINVAL, "fuse must be -1, 0, 1 or 2 (got %d)", fuse);
    // Far beyond what the column pass's shared memory holds; checked first so
    // that the ring size below stays within an int.
    if (wy > (int64_t(1) << 20)) return set_error(MMF_ENOTIMPL, "column window %lld too large", (long long)wy);
    if (fuse == 1 && wy > 1 && wx > MMF_FUSED_MAX_WX)
        return set_error(MMF_ENOTIMPL, "the fused 2D kernel handles row windows up to %d", MMF_FUSED_MAX_WX);
    // Column-pass shared memory: P ring plus the tile-aggregate ring.
    size_t smem = 0;
    switch (dt) {
        case MMF_F32: smem = col_smem_bytes<float>(wy); break;
        case MMF_F64: smem = col_smem_bytes<double>(wy); break;
        case MMF_I16: smem = col_smem_bytes<int16_t>(wy, 1); break;
        case MMF_U8: smem = col_smem_bytes<uint8_t>(wy, 1); break;
    }
    if (smem > 227 * 1024) return set_error(MMF_ENOTIMPL, "column window %lld too large", (long long)wy);
    return MMF_OK;
}

}  // namespace mmf

using namespace mmf;

extern "C" {

mmf_status mmf_filter2d_workspace(int64_t nimg, int64_t H, int64_t W, int64_t wy, int64_t wx, mmf_dtype dtype,
                                  int fuse, size_t *bytes) {
    if (!bytes) return set_error(MMF_EINVAL, "NULL output");
    mmf_status st = check2d(nimg, H, W, W, wy, wx, dtype, fuse);
    if (st != MMF_OK) return st;
    // Two intermediates of nimg*H rows of pitch W rounded up to 16 elements:
    // room for the row pass over dense images as one series (the width
    // covers both that and the row-by-row form's Wo rounded up).
    const int64_t Wo = W - wx + 1;
    *bytes = (wy > 1 && wx > 1 && Wo > 0 && H >= wy && !use_fused(wy, wx, fuse, elem_size(dtype)))
                 ? (size_t)(2 * nimg * H * mid_pitch(W) * elem_size(dtype))
                 : 0;
    return MMF_OK;
}

mmf_status mmf_filter2d_separable(const void *d_in, int64_t nimg, int64_t H, int64_t W, int64_t pitch, int64_t wy,
                                  int64_t wx, mmf_dtype dtype, int fuse, void *d_max, void *d_min, void *d_work,
                                  size_t work_bytes, void *stream) {
    NvtxRange nvtx_range("mmf_filter2d_separable");
    mmf_status st = check2d(nimg, H, W, pitch, wy, wx, dtype, fuse);
    if (st != MMF_OK) return st;
    const int64_t Ho = H - wy + 1, Wo = W - wx + 1;
    if (nimg == 0 || Ho <= 0 || Wo <= 0) return MMF_OK;
    if (!d_in || (!d_max && !d_min)) return set_error(MMF_EINVAL, "NULL buffers");
    size_t need = 0;
    mmf_filter2d_workspace(nimg, H, W, wy, wx, dtype, fuse, &need);
    if (work_bytes < need || (need && !d_work))
        return set_error(MMF_EINVAL, "workspace of %zu bytes needed", need);
    const int esz = elem_size(dtype);
    if (((uintptr_t)d_in % esz) || ((uintptr_t)d_max % esz) || ((uintptr_t)d_min % esz) || ((uintptr_t)d_work % 16))
        return set_error(MMF_EINVAL, "misaligned pointer (workspace needs 16 bytes)");
    LaunchCtx ctx;
    st = get_ctx(stream, &ctx);
    if (st != MMF_OK) return st;
    switch (dtype) {
        case MMF_F32: return filter2d<float>(ctx, (const float *)d_in, nimg, H, W, pitch, wy, wx, fuse, (float *)d_max, (float *)d_min, d_work, work_bytes);
        case MMF_F64: return filter2d<double>(ctx, (const double *)d_in, nimg, H, W, pitch, wy, wx, fuse, (double *)d_max, (double *)d_min, d_work, work_bytes);
        case MMF_I16: return filter2d<int16_t>(ctx, (const int16_t *)d_in, nimg, H, W, pitch, wy, wx, fuse, (int16_t *)d_max, (int16_t *)d_min, d_work, work_bytes);
        case MMF_U8: return filter2d<uint8_t>(ctx, (const uint8_t *)d_in, nimg, H, W, pitch, wy, wx, fuse, (uint8_t *)d_max, (uint8_t *)d_min, d_work, work_bytes);
    }
    return set_error(MMF_EINVAL, "unknown dtype");
}

}  // extern "C"
