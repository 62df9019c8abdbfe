// Parameters and launcher of the packed 2D kernel (pack2d.cuh; its
// instantiations sit in k_pack_*.cu so that they compile in parallel).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace mmf {

constexpr int kPkThreads = 256;
constexpr int kPkBand = 64;  // output rows per warp task
constexpr int kPkRows = 8;   // output rows per step
constexpr int kPkMaxWy = 9;
template <typename T> constexpr int pk_max_wx() { return sizeof(T) == 2 ? 5 : 9; }
// Output words per warp: 31 and a halo word for the packed types (their rows
// are realigned across lanes); for f32, 33 - wx and wx - 1 halo words (the
// row window's next columns come from the next lanes).
template <typename T> __host__ __device__ constexpr int pk_chunk(int wx) { return sizeof(T) == 4 ? 33 - wx : 31; }

struct Pack2DParams {
    const void *in;
    void *out_max, *out_min;
    int64_t nimg, H, W, pitch, img_stride;  // input geometry (elements)
    int64_t Ho, Wo;                         // outputs: image k row y at out + (k*Ho + y)*Wo
    int32_t wy, wx;
    int32_t nchunks;  // chunks of pk_chunk words per output row (a warp each)
    int32_t nbands;   // bands of kPkBand output rows per image
    int64_t tasks;    // nimg * nbands * nchunks warp tasks
    uint32_t *status;                // device status word (range checks of a checked build)
    int64_t in_bytes, out_bytes;     // readable bytes from `in`, writable from each output
};

// Launches pack2d_kernel<T, WY> on `grid` CTAs (explicitly instantiated
// for T in {uint8_t, int16_t, float} and WY in 1 .. kPkMaxWy).
template <typename T, int WY> cudaError_t pack2d_launch(cudaStream_t stream, const Pack2DParams &P, unsigned grid);

}  // namespace mmf
