// The window-3 filter in at most two comparisons per element (the
// proposition that follows the lower bound of Section 3): with the order of
// the last two elements known from the previous step, comparing the new
// element with each of them decides the window's maximum, its minimum and the
// order of the next pair.
//
// Each thread filters 16 consecutive outputs: its 16 inputs come in 16-byte
// loads and the two that follow them from the next lane (the warp's last lane
// loads them itself).  The thread starts its pair with one comparison, then
// takes two per element, so a chunk of c outputs costs 1 + 2c comparisons.
// With a counter, every comparison made is counted and the warp's total added
// to it once.  Misaligned arrays and the ragged end take a scalar path with
// the same comparisons.
#include <cstdint>

#include "launch.h"
#include "mmf.h"

namespace mmf {
namespace {

constexpr int kW3Out = 16;  // outputs per thread

template <typename T>
__device__ __forceinline__ T shfl_down_elem(T v, int d) {
    if constexpr (sizeof(T) == 8) {
        return __longlong_as_double(__shfl_down_sync(0xffffffffu, __double_as_longlong(v), d));
    } else if constexpr (sizeof(T) == 4) {
        return __shfl_down_sync(0xffffffffu, v, d);
    } else {
        return (T)__shfl_down_sync(0xffffffffu, (int)v, d);
    }
}

// One chunk: inputs e[0..cnt+1], outputs cnt; returns the comparisons made.
template <typename T, int N>
__device__ __forceinline__ int w3_chunk(const T (&e)[N], int cnt, typename Elem<T>::R (&hi)[kW3Out],
                                        typename Elem<T>::R (&lo)[kW3Out]) {
    using R = typename Elem<T>::R;
    R k0 = Elem<T>::load(e[0]), k1 = Elem<T>::load(e[1]);
    bool older_greater = k0 > k1;  // order of the last two
    int c = 1;
#pragma unroll
    for (int o = 0; o < kW3Out; ++o) {
        if (o < cnt) {
            const R k2 = Elem<T>::load(e[o + 2]);
            const bool prev_gt = k1 > k2;   // the newest pair
            const bool older_gt = k0 > k2;  // the older element against the new one
            c += 2;
            if (older_greater) {  // k0 > k1: the maximum is k0 or k2, the minimum k1 or k2
                hi[o] = older_gt ? k0 : k2;
                lo[o] = prev_gt ? k2 : k1;
            } else {  // k1 >= k0
                hi[o] = prev_gt ? k1 : k2;
                lo[o] = older_gt ? k2 : k0;
            }
            older_greater = prev_gt;
            k0 = k1;
            k1 = k2;
        }
    }
    return c;
}

template <typename T>
__global__ void __launch_bounds__(256) w3_kernel(const T *__restrict__ a, long long n, T *omax, T *omin,
                                                 unsigned long long *ncmp, int vec, uint32_t *status) {
    using R = typename Elem<T>::R;
    const long long n_out = n - 2;
    // Range checks of a checked build (always true otherwise).
    auto in_ok = [&](const void *p, int nb) { return in_bytes(status, p, nb, a, n * (long long)sizeof(T)); };
    auto out_ok = [&](const T *base, const void *p, int nb) {
        return in_bytes(status, p, nb, base, n_out * (long long)sizeof(T));
    };
    const long long j0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * kW3Out;
    const int lane = threadIdx.x & 31;
    // The warp takes the vector path when all its inputs are in the array.
    const long long warp_end = (j0 - (long long)lane * kW3Out) + 32LL * kW3Out + 2;
    T e[kW3Out + 2];
    int cnt = 0;
    if (vec && warp_end <= n) {
        constexpr int NV = kW3Out * (int)sizeof(T) / 16;
        union {
            uint4 u[NV];
            T v[kW3Out];
        } ld;
        const uint4 *src = reinterpret_cast<const uint4 *>(a + j0);
#pragma unroll
        for (int q = 0; q < NV; ++q) ld.u[q] = in_ok(src + q, 16) ? __ldg(src + q) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int q = 0; q < kW3Out; ++q) e[q] = ld.v[q];
        T h0 = shfl_down_elem(ld.v[0], 1), h1 = shfl_down_elem(ld.v[1], 1);
        if (lane == 31) {
            h0 = in_ok(a + j0 + kW3Out, (int)sizeof(T)) ? a[j0 + kW3Out] : T(0);
            h1 = in_ok(a + j0 + kW3Out + 1, (int)sizeof(T)) ? a[j0 + kW3Out + 1] : T(0);
        }
        e[kW3Out] = h0;
        e[kW3Out + 1] = h1;
        cnt = kW3Out;
    } else if (j0 < n_out) {
        cnt = (int)min((long long)kW3Out, n_out - j0);
#pragma unroll
        for (int q = 0; q < kW3Out + 2; ++q)
            e[q] = q < cnt + 2 && in_ok(a + j0 + q, (int)sizeof(T)) ? a[j0 + q] : T(0);
    }
    int c = 0;
    if (cnt > 0) {
        R hi[kW3Out], lo[kW3Out];
        c = w3_chunk<T>(e, cnt, hi, lo);
        const bool vst = vec && cnt == kW3Out;
        if (omax) {
            if (vst) {
                union {
                    uint4 u[kW3Out * sizeof(T) / 16];
                    T v[kW3Out];
                } st;
#pragma unroll
                for (int q = 0; q < kW3Out; ++q) st.v[q] = Elem<T>::store(hi[q]);
#pragma unroll
                for (int q = 0; q < (int)(kW3Out * sizeof(T) / 16); ++q)
                    if (out_ok(omax, reinterpret_cast<uint4 *>(omax + j0) + q, 16))
                        reinterpret_cast<uint4 *>(omax + j0)[q] = st.u[q];
            } else {
#pragma unroll
                for (int q = 0; q < kW3Out; ++q)
                    if (q < cnt && out_ok(omax, omax + j0 + q, (int)sizeof(T))) omax[j0 + q] = Elem<T>::store(hi[q]);
            }
        }
        if (omin) {
            if (vst) {
                union {
                    uint4 u[kW3Out * sizeof(T) / 16];
                    T v[kW3Out];
                } st;
#pragma unroll
                for (int q = 0; q < kW3Out; ++q) st.v[q] = Elem<T>::store(lo[q]);
#pragma unroll
                for (int q = 0; q < (int)(kW3Out * sizeof(T) / 16); ++q)
                    if (out_ok(omin, reinterpret_cast<uint4 *>(omin + j0) + q, 16))
                        reinterpret_cast<uint4 *>(omin + j0)[q] = st.u[q];
            } else {
#pragma unroll
                for (int q = 0; q < kW3Out; ++q)
                    if (q < cnt && out_ok(omin, omin + j0 + q, (int)sizeof(T))) omin[j0 + q] = Elem<T>::store(lo[q]);
            }
        }
    }
    if (ncmp) {
        unsigned long long s = (unsigned long long)c;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
        if (lane == 0 && s) atomicAdd(ncmp, s);
    }
}

}  // namespace

template <typename T>
cudaError_t w3_1d(const LaunchCtx &ctx, const void *in, int64_t n, void *omax, void *omin,
                  unsigned long long *ncmp) {
    const int64_t n_out = n - 2;
    if (n_out <= 0) return cudaSuccess;
    const int64_t threads = (n_out + kW3Out - 1) / kW3Out;
    const int64_t blocks = (threads + 255) / 256;
    const int vec = ((uintptr_t)in % 16) == 0 && ((uintptr_t)omax % 16) == 0 && ((uintptr_t)omin % 16) == 0;
    w3_kernel<T><<<(unsigned)blocks, 256, 0, ctx.stream>>>(static_cast<const T *>(in), n, static_cast<T *>(omax),
                                                          static_cast<T *>(omin), ncmp, vec, ctx.status);
    return cudaGetLastError();
}

template cudaError_t w3_1d<float>(const LaunchCtx &, const void *, int64_t, void *, void *, unsigned long long *);
template cudaError_t w3_1d<double>(const LaunchCtx &, const void *, int64_t, void *, void *, unsigned long long *);
template cudaError_t w3_1d<int16_t>(const LaunchCtx &, const void *, int64_t, void *, void *, unsigned long long *);
template cudaError_t w3_1d<uint8_t>(const LaunchCtx &, const void *, int64_t, void *, void *, unsigned long long *);

}  // namespace mmf
