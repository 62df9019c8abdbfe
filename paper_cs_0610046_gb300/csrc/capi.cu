// C ABI of the library (declared in include/mmf.h): argument checking, dtype
// dispatch, kernel selection and error reporting.  No C++ exception crosses
// this boundary; failures return an mmf_status and set a thread-local message.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "launch.h"
#include "mmf.h"

namespace mmf {

// Device status word (one per device that loads the module).
__device__ uint32_t g_status_word;

static thread_local char g_err[512] = "";

mmf_status set_error(mmf_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

mmf_status cuda_error(cudaError_t e, const char *what) {
    return set_error(MMF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

struct DevCache {
    bool ready = false;
    int sms = 0;
    uint32_t *status = nullptr;
};
static std::mutex g_dev_mu;
static DevCache g_dev[64];

mmf_status get_ctx(void *stream, LaunchCtx *ctx) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(MMF_EINVAL, "device ordinal %d out of range", dev);
    {
        std::lock_guard<std::mutex> lk(g_dev_mu);
        DevCache &dc = g_dev[dev];
        if (!dc.ready) {
            int sms = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute");
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_status_word);
            if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(status)");
            dc.sms = sms;
            dc.status = static_cast<uint32_t *>(p);
            dc.ready = true;
        }
        ctx->device = dev;
        ctx->sms = dc.sms;
        ctx->status = dc.status;
    }
    ctx->stream = static_cast<cudaStream_t>(stream);
    return MMF_OK;
}

int elem_size(mmf_dtype dt) {
    switch (dt) {
        case MMF_F32: return 4;
        case MMF_F64: return 8;
        case MMF_I16: return 2;
        case MMF_U8: return 1;
    }
    return 0;
}

int tile_of(mmf_dtype dt) {
    switch (dt) {
        case MMF_F32: return 2048;
        case MMF_F64: return 1024;
        default: return 4096;
    }
}

// Translate (n, w_or_r, mode) into the kernel's series description.
mmf_status make_series(int64_t n, int64_t w_or_r, mmf_mode mode, mmf_dtype dt, SeriesDesc *sd) {
    if (n < 0) return set_error(MMF_EINVAL, "n = %lld < 0", (long long)n);
    sd->in_off = 0;
    sd->out_off = 0;
    sd->n = n;
    if (mode == MMF_VALID) {
        if (w_or_r < 1) return set_error(MMF_EINVAL, "window w = %lld < 1", (long long)w_or_r);
        sd->w = w_or_r;
        sd->d = 0;
        sd->n_out = n >= w_or_r ? n - w_or_r + 1 : 0;
    } else if (mode == MMF_CENTERED_CLIPPED) {
        if (w_or_r < 0) return set_error(MMF_EINVAL, "radius r = %lld < 0", (long long)w_or_r);
        // A radius of n-1 already covers the whole array from every centre
        // (and an empty array has no windows, so 2r+1 never overflows).
        int64_t r = w_or_r;
        if (r > n - 1) r = n > 0 ? n - 1 : 0;
        sd->w = 2 * r + 1;
        sd->d = -r;
        sd->n_out = n;
    } else {
        return set_error(MMF_EINVAL, "unknown mode %d", (int)mode);
    }
    if (sd->n_out > 0 && (sd->w - 1) / tile_of(dt) > MMF_MAX_WINDOW_TILES)
        return set_error(MMF_ENOTIMPL, "window %lld exceeds the supported maximum", (long long)sd->w);
    return MMF_OK;
}

static std::atomic<uint32_t> g_test_flags{0};
static std::atomic<long long> g_test_wait_limit{0};
static std::atomic<int64_t> g_test_clip_in{0};

TestHooks test_hooks() {
    return TestHooks{g_test_flags.load(std::memory_order_relaxed), g_test_wait_limit.load(std::memory_order_relaxed),
                     g_test_clip_in.load(std::memory_order_relaxed)};
}

mmf_kernel dispatch_lookup(mmf_dtype dt, int64_t n, int64_t w);  // dispatch.cu

template <typename F> mmf_status dispatch_dtype(mmf_dtype dt, F &&f) {
    switch (dt) {
        case MMF_F32: return f(float{});
        case MMF_F64: return f(double{});
        case MMF_I16: return f(int16_t{});
        case MMF_U8: return f(uint8_t{});
    }
    return set_error(MMF_EINVAL, "unknown dtype %d", (int)dt);
}

}  // namespace mmf

using namespace mmf;

extern "C" {

const char *mmf_last_error(void) { return g_err; }

const char *mmf_version(void) { return "mmf-gb300 0.1 (sm_103a)"; }

mmf_status mmf_argfilter1d_ex(const void *d_in, int64_t n, int64_t w, mmf_dtype dtype, void *d_max, void *d_min,
                              int64_t *d_argmax, int64_t *d_argmin, void *stream, mmf_kernel kernel) {
    NvtxRange nvtx_range("mmf_argfilter1d_ex");
    if (elem_size(dtype) == 0) return set_error(MMF_EINVAL, "unknown dtype %d", (int)dtype);
    if (kernel != MMF_KERNEL_AUTO && kernel != MMF_KERNEL_BLOCKSCAN && kernel != MMF_KERNEL_WEDGE)
        return set_error(MMF_ENOTIMPL, "kernel %d does not compute locations", (int)kernel);
    // Any window: the block scans over (value, position) pairs carry long
    // blocks through per-tile aggregates, so the value filter's window limit
    // does not apply here.
    if (n < 0) return set_error(MMF_EINVAL, "n = %lld < 0", (long long)n);
    if (w < 1) return set_error(MMF_EINVAL, "window w = %lld < 1", (long long)w);
    if (kernel == MMF_KERNEL_WEDGE && w > MMF_WEDGE_MAX_WINDOW)
        return set_error(MMF_ENOTIMPL, "the wedge kernel computes locations for windows up to %d",
                         MMF_WEDGE_MAX_WINDOW);
    if (n < w) return MMF_OK;  // no window fits
    if (!d_max && !d_min && !d_argmax && !d_argmin) return set_error(MMF_EINVAL, "every output is NULL");
    if (!d_in) return set_error(MMF_EINVAL, "NULL input with n = %lld", (long long)n);
    const int esz = elem_size(dtype);
    if (((uintptr_t)d_in % esz) || ((uintptr_t)d_max % esz) || ((uintptr_t)d_min % esz) ||
        ((uintptr_t)d_argmax % 8) || ((uintptr_t)d_argmin % 8))
        return set_error(MMF_EINVAL, "misaligned pointer");
    LaunchCtx ctx;
    const mmf_status st = get_ctx(stream, &ctx);
    if (st != MMF_OK) return st;
    return dispatch_dtype(dtype, [&](auto tag) -> mmf_status {
        using T = decltype(tag);
        const cudaError_t e = kernel == MMF_KERNEL_WEDGE
                                  ? wedge_arg_1d<T>(ctx, d_in, n, w, d_max, d_min, d_argmax, d_argmin)
                                  : argscan_1d<T>(ctx, d_in, n, w, d_max, d_min, d_argmax, d_argmin);
        return e == cudaSuccess ? MMF_OK : cuda_error(e, "argfilter launch");
    });
}

mmf_status mmf_argfilter1d(const void *d_in, int64_t n, int64_t w, mmf_dtype dtype, void *d_max, void *d_min,
                           int64_t *d_argmax, int64_t *d_argmin, void *stream) {
    return mmf_argfilter1d_ex(d_in, n, w, dtype, d_max, d_min, d_argmax, d_argmin, stream, MMF_KERNEL_AUTO);
}

mmf_status mmf_filter1d_w3(const void *d_in, int64_t n, mmf_dtype dtype, void *d_max, void *d_min,
                           unsigned long long *d_ncmp, void *stream) {
    NvtxRange nvtx_range("mmf_filter1d_w3");
    const int esz = elem_size(dtype);
    if (esz == 0) return set_error(MMF_EINVAL, "unknown dtype %d", (int)dtype);
    if (n < 0) return set_error(MMF_EINVAL, "n = %lld", (long long)n);
    if (n < 3) return MMF_OK;  // no window of 3
    if (!d_max && !d_min && !d_ncmp) return set_error(MMF_EINVAL, "every output is NULL");
    if (!d_in) return set_error(MMF_EINVAL, "NULL input with n = %lld", (long long)n);
    if (((uintptr_t)d_in % esz) || ((uintptr_t)d_max % esz) || ((uintptr_t)d_min % esz) ||
        ((uintptr_t)d_ncmp % 8))
        return set_error(MMF_EINVAL, "misaligned pointer");
    LaunchCtx ctx;
    mmf_status st = get_ctx(stream, &ctx);
    if (st != MMF_OK) return st;
    return dispatch_dtype(dtype, [&](auto tag) -> mmf_status {
        using T = decltype(tag);
        const cudaError_t e = w3_1d<T>(ctx, d_in, n, d_max, d_min, d_ncmp);
        return e == cudaSuccess ? MMF_OK : cuda_error(e, "w3 launch");
    });
}

int64_t mmf_output_length(int64_t n, int64_t w_or_r, mmf_mode mode) {
    if (n < 0) return -1;
    if (mode == MMF_VALID) return w_or_r < 1 ? -1 : (n >= w_or_r ? n - w_or_r + 1 : 0);
    if (mode == MMF_CENTERED_CLIPPED) return w_or_r < 0 ? -1 : n;
    return -1;
}

mmf_status mmf_filter1d_ex(const void *d_in, int64_t n, int64_t w_or_r, mmf_dtype dtype, mmf_mode mode,
                           void *d_max, void *d_min, void *stream, mmf_kernel kernel) {
    NvtxRange nvtx_range("mmf_filter1d_ex");
    if (elem_size(dtype) == 0) return set_error(MMF_EINVAL, "unknown dtype %d", (int)dtype);
    SeriesDesc sd;
    mmf_status st = make_series(n, w_or_r, mode, dtype, &sd);
    if (st != MMF_OK) return st;
    if (sd.n_out == 0) return MMF_OK;  // nothing to write (empty outputs may be NULL)
    if (!d_max && !d_min) return set_error(MMF_EINVAL, "both outputs are NULL");
    if (!d_in) return set_error(MMF_EINVAL, "NULL input with n = %lld", (long long)n);
    const int esz = elem_size(dtype);
    if (((uintptr_t)d_in % esz) || ((uintptr_t)d_max % esz) || ((uintptr_t)d_min % esz))
        return set_error(MMF_EINVAL, "pointers must be aligned to the element size");
    LaunchCtx ctx;
    st = get_ctx(stream, &ctx);
    if (st != MMF_OK) return st;
    const int slide_max = dtype == MMF_F32 ? 17 : 9;
    if (kernel == MMF_KERNEL_AUTO) {
        // A tuned entry of the dispatch table replaces the built-in rule
        // where its kernel can take this call.
        const mmf_kernel k = dispatch_lookup(dtype, n, sd.w);
        bool ok = false;
        switch (k) {
            case MMF_KERNEL_SLIDE: ok = sd.w <= slide_max; break;
            case MMF_KERNEL_BLOCKSCAN: ok = true; break;
            case MMF_KERNEL_WEDGE: ok = mode == MMF_VALID && sd.w <= MMF_WEDGE_MAX_WINDOW; break;
            case MMF_KERNEL_FRONT:
                ok = dispatch_dtype(dtype, [&](auto tag) -> mmf_status {
                         using T = decltype(tag);
                         return front_applies<T>(sd, ctx.sms, 1) ? MMF_OK : MMF_ENOTIMPL;
                     }) == MMF_OK;
                break;
            default: break;
        }
        if (ok) kernel = k;
    }
    if (kernel == MMF_KERNEL_SLIDE && sd.w > slide_max)
        return set_error(MMF_EINVAL, "the register slide handles windows up to %d (w = %lld)", slide_max,
                         (long long)sd.w);
    if (kernel == MMF_KERNEL_WEDGE) {
        if (mode != MMF_VALID) return set_error(MMF_ENOTIMPL, "the wedge kernel computes valid windows only");
        if (sd.w > MMF_WEDGE_MAX_WINDOW)
            return set_error(MMF_EINVAL, "the wedge kernel handles windows up to %d", MMF_WEDGE_MAX_WINDOW);
        return dispatch_dtype(dtype, [&](auto tag) -> mmf_status {
            using T = decltype(tag);
            cudaError_t e = wedge_1d<T>(ctx, d_in, n, sd.w, d_max, d_min);
            return e == cudaSuccess ? MMF_OK : cuda_error(e, "wedge launch");
        });
    }
    if (kernel != MMF_KERNEL_AUTO && kernel != MMF_KERNEL_BLOCKSCAN && kernel != MMF_KERNEL_SLIDE &&
        kernel != MMF_KERNEL_FRONT)
        return set_error(MMF_ENOTIMPL, "kernel %d not available", (int)kernel);
    const bool allow_slide = kernel != MMF_KERNEL_BLOCKSCAN && kernel != MMF_KERNEL_FRONT;
    const int front = kernel == MMF_KERNEL_FRONT ? 1 : (kernel == MMF_KERNEL_AUTO ? -1 : 0);
    return dispatch_dtype(dtype, [&](auto tag) -> mmf_status {
        using T = decltype(tag);
        if (front == 1 && !front_applies<T>(sd, ctx.sms, 1))
            return set_error(MMF_ENOTIMPL, "the advancing front takes windows of a tile or more, not f64");
        cudaError_t e = blockscan_1d<T>(ctx, d_in, sd, d_max, d_min, allow_slide, front);
        return e == cudaSuccess ? MMF_OK : cuda_error(e, "filter launch");
    });
}

mmf_status mmf_filter1d(const void *d_in, int64_t n, int64_t w_or_r, mmf_dtype dtype, mmf_mode mode, void *d_max,
                        void *d_min, void *stream) {
    return mmf_filter1d_ex(d_in, n, w_or_r, dtype, mode, d_max, d_min, stream, MMF_KERNEL_AUTO);
}

mmf_status mmf_test_set_wait_fault(int starve_copies, int64_t wait_limit_cycles) {
    if (starve_copies) {
        if (wait_limit_cycles < 1000 || wait_limit_cycles > 2000000000LL)
            return set_error(MMF_EINVAL, "wait limit %lld outside [1000, 2e9] clocks", (long long)wait_limit_cycles);
        g_test_wait_limit.store(wait_limit_cycles);
        g_test_flags.store(kTestStarveCopies);
    } else {
        g_test_flags.store(0);
        g_test_wait_limit.store(0);
    }
    return MMF_OK;
}

mmf_status mmf_test_set_input_clip(int64_t elems) {
    if (elems < 0) return set_error(MMF_EINVAL, "negative clip %lld", (long long)elems);
    g_test_clip_in.store(elems);
    return MMF_OK;
}

mmf_status mmf_device_status(uint32_t *out, int reset) {
    if (!out) return set_error(MMF_EINVAL, "NULL output");
    LaunchCtx ctx;
    mmf_status st = get_ctx(nullptr, &ctx);
    if (st != MMF_OK) return st;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_error(e, "cudaDeviceSynchronize");
    uint32_t v = 0;
    e = cudaMemcpy(&v, ctx.status, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "read status");
    if (reset) {
        uint32_t z = 0;
        e = cudaMemcpy(ctx.status, &z, sizeof(z), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_error(e, "reset status");
    }
    *out = v;
    return MMF_OK;
}

}  // extern "C"
