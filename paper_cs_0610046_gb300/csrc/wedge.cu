// Chunked monotonic wedge: Algorithm 1 (Section 4) run serially by every
// thread on its own chunk of outputs.
//
// Thread t owns the outputs [j0, j0+C) and the inputs [j0, j0+C+w-1).  It runs
// the algorithm over those inputs as if its stream began at j0: the first w-1
// steps only fill the wedge (each output depends on its own window alone, so
// restarting at j0 is exact), after that every step emits one output.
//
// Per-thread state in shared memory:
//   * a value ring holding the last vcap inputs (vcap >= w+16: the window plus
//     the inputs staged ahead), filled 8 elements at a time by vector loads;
//   * the deques U and L as rings of 16-bit input indices (capacity >= w+1,
//     Proposition 4 bounds size(U)+size(L) by w+1).
// Every ring is interleaved across the CTA's threads (slot s of thread t in
// 4-byte word (s/E)*tpb + t, E elements per word), so a warp touches 32
// distinct banks whichever slots its threads read.  The fronts of U and L are
// also kept in registers, so an output costs no shared-memory read; outputs
// leave in 8-element vector stores.  The while loops are data dependent: on
// noise they iterate about once per element, on monotone runs rarely
// (Propositions 2 and 3 bound the comparisons by 3 and 2 per element).
#include <cstdint>
#include <cstring>
#include <type_traits>

#include "launch.h"
#include "mmf.h"

namespace mmf {

// Ring element type: the comparison key where it has the element's size (f32,
// f64 keys), the raw element otherwise (u8, i16 widen on read).
template <typename T>
using WedgeS = std::conditional_t<sizeof(typename Elem<T>::R) == sizeof(T), typename Elem<T>::R, T>;

template <typename S> struct WRing {
    static constexpr int E = sizeof(S) >= 4 ? 1 : 4 / (int)sizeof(S);
    S *col;      // this thread's column: base + t*E
    int stride;  // elements between consecutive words of one thread: tpb*E
    __device__ S &at(uint32_t s) const { return col[(s / E) * (uint32_t)stride + (s % E)]; }
};

template <typename T> struct WedgeIO {
    using R = typename Elem<T>::R;
    using S = WedgeS<T>;
    static constexpr int WORDS = 8 * (int)sizeof(T) / 4;  // u8 2, i16 4, f32 8, f64 16

    // Eight consecutive inputs as raw little-endian words; past the end of the
    // array the words are zero (they are never consumed).
    __device__ static void load(const T *src, int64_t avail, bool vec, uint32_t (&wd)[WORDS]) {
        if (vec && avail >= 8) {
            if constexpr (WORDS == 2) {
                const uint2 u = __ldg(reinterpret_cast<const uint2 *>(src));
                wd[0] = u.x;
                wd[1] = u.y;
            } else {
#pragma unroll
                for (int q = 0; q < WORDS / 4; ++q) {
                    const uint4 u = __ldg(reinterpret_cast<const uint4 *>(src) + q);
                    wd[4 * q] = u.x;
                    wd[4 * q + 1] = u.y;
                    wd[4 * q + 2] = u.z;
                    wd[4 * q + 3] = u.w;
                }
            }
        } else {
            T v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = k < avail ? src[k] : T(0);
            memcpy(wd, v, sizeof(v));
        }
    }

    // Write the eight inputs of `wd` to ring slots s..s+7 (s a multiple of 8).
    __device__ static void stage(const WRing<S> &V, uint32_t s, const uint32_t (&wd)[WORDS]) {
        if constexpr (WRing<S>::E > 1) {
            uint32_t *col = reinterpret_cast<uint32_t *>(V.col);
            const uint32_t ws = (uint32_t)V.stride / WRing<S>::E;
#pragma unroll
            for (int q = 0; q < WORDS; ++q) col[(s / WRing<S>::E + q) * ws] = wd[q];
        } else if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int k = 0; k < 8; ++k) V.at(s + k) = __uint_as_float(wd[k]);
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const long long b = (long long)(((unsigned long long)wd[2 * k + 1] << 32) | wd[2 * k]);
                V.at(s + k) = Elem<double>::key(b);
            }
        }
    }

    // Store eight outputs (the first `cnt` of them) at dst.
    __device__ static void store(T *dst, int64_t cnt, bool vec, const R (&r)[8]) {
        if (vec && cnt >= 8) {
            T v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = Elem<T>::store(r[k]);
            uint32_t wd[WORDS];
            memcpy(wd, v, sizeof(v));
            if constexpr (WORDS == 2) {
                __stcs(reinterpret_cast<uint2 *>(dst), make_uint2(wd[0], wd[1]));
            } else {
#pragma unroll
                for (int q = 0; q < WORDS / 4; ++q)
                    __stcs(reinterpret_cast<uint4 *>(dst) + q,
                           make_uint4(wd[4 * q], wd[4 * q + 1], wd[4 * q + 2], wd[4 * q + 3]));
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (k < cnt) dst[k] = Elem<T>::store(r[k]);
        }
    }
};

// Eight int64 positions (the first cnt of them) at dst; whole 16-byte pairs
// when dst is 16-byte aligned.
__device__ __forceinline__ void store_index(int64_t *dst, int64_t cnt, const int64_t (&v)[8]) {
    if (cnt >= 8 && (((uintptr_t)dst) & 15) == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) __stcs(reinterpret_cast<longlong2 *>(dst) + k, make_longlong2(v[2 * k], v[2 * k + 1]));
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k < cnt) dst[k] = v[k];
    }
}

template <typename T> struct Wedge {
    using R = typename Elem<T>::R;
    using S = WedgeS<T>;
    WRing<S> V;
    WRing<uint16_t> U, L;
    uint32_t vmask, imask, w;
    uint32_t uh, us, lh, ls;  // head slot and size of U and L
    uint32_t uf, lf;          // low 16 bits of the front indices
    R ufv, lfv, prev;         // front values, a_{i-1}

    __device__ R val(uint32_t idx) const { return (R)V.at(idx & vmask); }

    __device__ void start(R a0) {
        U.at(0) = 0;
        L.at(0) = 0;
        uh = lh = 0;
        us = ls = 1;
        uf = lf = 0;
        ufv = lfv = prev = a0;
    }

    // One iteration of Algorithm 1 for input i >= 1: afterwards the fronts are
    // the maximum and minimum of the window that ends at i.  ARG (locations
    // wanted, leftmost among equal extremes): an input equal to the previous
    // one joins both deques behind it, so equal earlier indices stay in front,
    // and both fronts may leave the window at once.
    template <bool ARG = false>
    __device__ __forceinline__ void step(uint32_t i, R ai) {
        if (ARG && ai == prev) {
            U.at((uh + us) & imask) = (uint16_t)i;
            ++us;
            L.at((lh + ls) & imask) = (uint16_t)i;
            ++ls;
        } else if (ai > prev) {
            --us;  // i-1 is dominated on the U side
            while (us > 0) {
                const uint32_t b = U.at((uh + us - 1) & imask);
                if (!(ai > val(b))) break;
                --us;
            }
            U.at((uh + us) & imask) = (uint16_t)i;
            if (++us == 1) {
                uf = i & 0xffffu;
                ufv = ai;
            }
            L.at((lh + ls) & imask) = (uint16_t)i;
            ++ls;
        } else {
            --ls;
            while (ls > 0) {
                const uint32_t b = L.at((lh + ls - 1) & imask);
                if (!(ai < val(b))) break;
                --ls;
            }
            L.at((lh + ls) & imask) = (uint16_t)i;
            if (++ls == 1) {
                lf = i & 0xffffu;
                lfv = ai;
            }
            U.at((uh + us) & imask) = (uint16_t)i;
            ++us;
        }
        // Without ties at most one front can hold the index that just left
        // the window (every older index is in exactly one deque).
        const uint32_t gone = (i - w) & 0xffffu;
        if (uf == gone) {
            ++uh;
            --us;
            uf = U.at(uh & imask);
            ufv = val(uf);
            if (!ARG) {
                prev = ai;
                return;
            }
        }
        if (lf == gone) {
            ++lh;
            --ls;
            lf = L.at(lh & imask);
            lfv = val(lf);
        }
        prev = ai;
    }
};

// ARG: also the locations of the extremes (leftmost among equals) in amax /
// amin (int64 positions in the array; either may be null).
template <typename T, bool ARG>
__global__ void __launch_bounds__(256) wedge_kernel(const T *__restrict__ a, int64_t n, int32_t w, int64_t chunk,
                                                    int vlog2, int ilog2, int vec_in, int vec_out,
                                                    T *__restrict__ omax, T *__restrict__ omin,
                                                    int64_t *__restrict__ amax, int64_t *__restrict__ amin,
                                                    uint32_t *status) {
    using IO = WedgeIO<T>;
    using R = typename Elem<T>::R;
    using S = WedgeS<T>;
    extern __shared__ __align__(16) unsigned char wedge_smem[];
    const int tpb = blockDim.x, t = threadIdx.x;
    const int64_t n_out = n - w + 1;
    const int64_t j0 = ((int64_t)blockIdx.x * tpb + t) * chunk;
    if (j0 >= n_out) return;  // the kernel has no barriers
    const int64_t cnt = chunk < n_out - j0 ? chunk : n_out - j0;
    const T *x = a + j0;
    // Range checks of a checked build (always true otherwise): k elements of
    // size sz at p inside a buffer of m elements at base.
    auto ok = [&](const void *p, int64_t k, int sz, const void *base, int64_t m) {
        return in_bytes(status, p, (int)(k * sz), base, m * sz);
    };
    if (w == 1) {  // a window of one element is the element itself
        for (int64_t o = 0; o < cnt; ++o) {
            const T v = ok(x + o, 1, (int)sizeof(T), a, n) ? x[o] : T(0);
            if (omax && ok(omax + j0 + o, 1, (int)sizeof(T), omax, n_out)) omax[j0 + o] = v;
            if (omin && ok(omin + j0 + o, 1, (int)sizeof(T), omin, n_out)) omin[j0 + o] = v;
            if (ARG && amax && ok(amax + j0 + o, 1, 8, amax, n_out)) amax[j0 + o] = j0 + o;
            if (ARG && amin && ok(amin + j0 + o, 1, 8, amin, n_out)) amin[j0 + o] = j0 + o;
        }
        return;
    }
    const uint32_t vcap = 1u << vlog2, icap = 1u << ilog2, h = (uint32_t)w - 1;
    const uint32_t span = (uint32_t)cnt + h;
    Wedge<T> q;
    constexpr int EV = WRing<S>::E, EI = WRing<uint16_t>::E;
    S *vbase = reinterpret_cast<S *>(wedge_smem);
    uint16_t *ubase = reinterpret_cast<uint16_t *>(wedge_smem + (size_t)vcap * tpb * sizeof(S));
    uint16_t *lbase = ubase + (size_t)icap * tpb;
    q.V = WRing<S>{vbase + t * EV, tpb * EV};
    q.U = WRing<uint16_t>{ubase + t * EI, tpb * EI};
    q.L = WRing<uint16_t>{lbase + t * EI, tpb * EI};
    q.vmask = vcap - 1;
    q.imask = icap - 1;
    q.w = (uint32_t)w;

    uint32_t staged = 0;
    auto stage = [&]() {
        uint32_t wd[IO::WORDS];
        const int64_t avail = n - j0 - staged;
        if (ok(x + staged, avail < 8 ? avail : 8, (int)sizeof(T), a, n)) {
            IO::load(x + staged, avail, vec_in != 0, wd);
        } else {
#pragma unroll
            for (int k = 0; k < IO::WORDS; ++k) wd[k] = 0u;
        }
        IO::stage(q.V, staged & q.vmask, wd);
        staged += 8;
    };
    stage();
    q.start(q.val(0));
    for (uint32_t i = 1; i < h; ++i) {  // warm-up on the halo: no output yet
        if (i >= staged) stage();
        q.template step<ARG>(i, q.val(i));
    }
    for (uint32_t o = 0; o < (uint32_t)cnt; o += 8) {
        const uint32_t ib = o + h;
        while (staged < ib + 8 && staged < span) stage();
        R om[8], on[8];
        int64_t im[8], in_[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t i = ib + k;
            if (o + k < (uint32_t)cnt) q.template step<ARG>(i, q.val(i));
            om[k] = q.ufv;
            on[k] = q.lfv;
            if (ARG) {
                // The fronts keep the low 16 bits of their indices; each lies
                // within the window, less than 2^16 back.
                im[k] = j0 + (int64_t)(i - ((i - q.uf) & 0xffffu));
                in_[k] = j0 + (int64_t)(i - ((i - q.lf) & 0xffffu));
            }
        }
        const int64_t left = cnt - o;
        const int64_t nst = left < 8 ? left : 8;
        if (omax && ok(omax + j0 + o, nst, (int)sizeof(T), omax, n_out)) IO::store(omax + j0 + o, left, vec_out != 0, om);
        if (omin && ok(omin + j0 + o, nst, (int)sizeof(T), omin, n_out)) IO::store(omin + j0 + o, left, vec_out != 0, on);
        if (ARG) {
            if (amax && ok(amax + j0 + o, nst, 8, amax, n_out)) store_index(amax + j0 + o, left, im);
            if (amin && ok(amin + j0 + o, nst, 8, amin, n_out)) store_index(amin + j0 + o, left, in_);
        }
    }
}

namespace {
int ceil_log2(int64_t v) {
    int lg = 0;
    while ((int64_t(1) << lg) < v) ++lg;
    return lg;
}
}  // namespace

template <typename T, bool ARG>
static cudaError_t wedge_launch(const LaunchCtx &ctx, const void *in, int64_t n, int64_t w, void *omax, void *omin,
                                int64_t *amax, int64_t *amin) {
    using S = WedgeS<T>;
    const int64_t n_out = n - w + 1;
    if (n_out <= 0) return cudaSuccess;
    const int vlog2 = ceil_log2(w + 16), ilog2 = ceil_log2(w + 1 < 8 ? 8 : w + 1);
    const size_t per_thread = ((size_t)1 << vlog2) * sizeof(S) + ((size_t)2 << ilog2) * sizeof(uint16_t);
    // Threads per CTA: a power of two up to 256 within 96 KB of rings (two
    // CTAs per SM), else one warp within 200 KB.
    int tpb = 256;
    while (tpb > 32 && (size_t)tpb * per_thread > 96 * 1024) tpb /= 2;
    const size_t smem = (size_t)tpb * per_thread;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;  // w above the supported maximum
    static int cached_smem[64][4] = {};
    const int slot = sizeof(T) == 1 ? 0 : sizeof(T) == 2 ? 1 : sizeof(T) == 4 ? 2 : 3;
    int &have = cached_smem[ctx.device & 63][slot];
    if ((int)smem > have) {
        cudaError_t e =
            cudaFuncSetAttribute(wedge_kernel<T, ARG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        have = (int)smem;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wedge_kernel<T, ARG>, tpb, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    // One wave of threads, each with at least 8w outputs (the warm-up of w-1
    // steps then costs at most 1/8 more), a multiple of 8.
    const int64_t resident = (int64_t)(ctx.sms > 0 ? ctx.sms : 1) * per_sm * tpb;
    int64_t chunk = (n_out + resident - 1) / resident;
    if (chunk < 8 * w) chunk = 8 * w;
    if (chunk > (int64_t(1) << 30)) chunk = int64_t(1) << 30;
    chunk = (chunk + 7) & ~int64_t(7);
    const int64_t threads = (n_out + chunk - 1) / chunk;
    const int64_t blocks = (threads + tpb - 1) / tpb;
    const size_t align = 8 * sizeof(T) < 16 ? 8 * sizeof(T) : 16;
    const int vec_in = ((uintptr_t)in % align) == 0;
    const int vec_out = ((uintptr_t)omax % align) == 0 && ((uintptr_t)omin % align) == 0;
    wedge_kernel<T, ARG><<<(unsigned)blocks, tpb, smem, ctx.stream>>>(
        static_cast<const T *>(in), n, (int32_t)w, chunk, vlog2, ilog2, vec_in, vec_out, static_cast<T *>(omax),
        static_cast<T *>(omin), amax, amin, ctx.status);
    return cudaGetLastError();
}

template <typename T>
cudaError_t wedge_1d(const LaunchCtx &ctx, const void *in, int64_t n, int64_t w, void *omax, void *omin) {
    return wedge_launch<T, false>(ctx, in, n, w, omax, omin, nullptr, nullptr);
}

template <typename T>
cudaError_t wedge_arg_1d(const LaunchCtx &ctx, const void *in, int64_t n, int64_t w, void *omax, void *omin,
                         int64_t *amax, int64_t *amin) {
    return wedge_launch<T, true>(ctx, in, n, w, omax, omin, amax, amin);
}

template cudaError_t wedge_1d<float>(const LaunchCtx &, const void *, int64_t, int64_t, void *, void *);
template cudaError_t wedge_1d<double>(const LaunchCtx &, const void *, int64_t, int64_t, void *, void *);
template cudaError_t wedge_1d<int16_t>(const LaunchCtx &, const void *, int64_t, int64_t, void *, void *);
template cudaError_t wedge_1d<uint8_t>(const LaunchCtx &, const void *, int64_t, int64_t, void *, void *);
template cudaError_t wedge_arg_1d<float>(const LaunchCtx &, const void *, int64_t, int64_t, void *, void *, int64_t *,
                                         int64_t *);
template cudaError_t wedge_arg_1d<double>(const LaunchCtx &, const void *, int64_t, int64_t, void *, void *, int64_t *,
                                          int64_t *);
template cudaError_t wedge_arg_1d<int16_t>(const LaunchCtx &, const void *, int64_t, int64_t, void *, void *,
                                           int64_t *, int64_t *);
template cudaError_t wedge_arg_1d<uint8_t>(const LaunchCtx &, const void *, int64_t, int64_t, void *, void *,
                                           int64_t *, int64_t *);

}  // namespace mmf
