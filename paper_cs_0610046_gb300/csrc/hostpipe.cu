// The 1D filter on arrays in host memory: chunks of outputs are pipelined
// through device staging on three CUDA streams, so the upload of chunk k+1,
// the filter of chunk k and the download of chunk k-1 overlap (the host link
// is full duplex).  Each chunk's input is its outputs' windows: the chunk
// plus w-1 elements (valid windows) or r on each side (centred windows),
// clipped to the array; positions outside the array are the identities of
// the block-scan kernel, so only the true array ends are clipped (each output
// depends on its own window alone, Section 1, so chunking is exact).
#include <algorithm>
#include <cstring>
#include <mutex>

#include "launch.h"
#include "mmf.h"

namespace mmf {
mmf_status set_error(mmf_status st, const char *fmt, ...);
mmf_status cuda_error(cudaError_t e, const char *what);
mmf_status get_ctx(void *stream, LaunchCtx *ctx);
int elem_size(mmf_dtype dt);
mmf_status make_series(int64_t n, int64_t w_or_r, mmf_mode mode, mmf_dtype dt, SeriesDesc *sd);
}  // namespace mmf

using namespace mmf;

namespace {

constexpr int kSlots = 3;

// Per-device pipeline: streams, events and grow-only staging slots (kept
// until the process exits).
struct Pipe {
    std::mutex mu;
    bool ready = false;
    cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
    cudaEvent_t in_done[kSlots] = {}, run_done[kSlots] = {}, out_done[kSlots] = {}, start = nullptr;
    cudaEvent_t last = nullptr;  // the previous call's last download
    char *in[kSlots] = {}, *out_max[kSlots] = {}, *out_min[kSlots] = {};
    size_t in_cap = 0, out_cap = 0;  // bytes per slot
};
Pipe g_pipe[64];

mmf_status pipe_setup(Pipe &p, size_t in_bytes, size_t out_bytes) {
    cudaError_t e = cudaSuccess;
    if (!p.ready) {
        e = cudaStreamCreateWithFlags(&p.s_in, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p.s_run, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p.s_out, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.last, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(p.last, p.s_out);
        for (int k = 0; k < kSlots && e == cudaSuccess; ++k) {
            e = cudaEventCreateWithFlags(&p.in_done[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.run_done[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.out_done[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_error(e, "host pipeline streams");
        p.ready = true;
    }
    if (in_bytes > p.in_cap || out_bytes > p.out_cap) {
        // Previous calls' work has finished (each call ends on its stream and
        // the next one starts after it), so the slots can be replaced.
        cudaDeviceSynchronize();
        for (int k = 0; k < kSlots; ++k) {
            if (in_bytes > p.in_cap) {
                cudaFree(p.in[k]);
                p.in[k] = nullptr;
            }
            if (out_bytes > p.out_cap) {
                cudaFree(p.out_max[k]);
                cudaFree(p.out_min[k]);
                p.out_max[k] = p.out_min[k] = nullptr;
            }
        }
        const size_t ib = std::max(in_bytes, p.in_cap), ob = std::max(out_bytes, p.out_cap);
        p.in_cap = p.out_cap = 0;
        for (int k = 0; k < kSlots && e == cudaSuccess; ++k) {
            if (!p.in[k]) e = cudaMalloc(&p.in[k], ib);
            if (e == cudaSuccess && !p.out_max[k]) e = cudaMalloc(&p.out_max[k], ob);
            if (e == cudaSuccess && !p.out_min[k]) e = cudaMalloc(&p.out_min[k], ob);
        }
        if (e != cudaSuccess) return set_error(MMF_ENOMEM, "host pipeline staging: %s", cudaGetErrorString(e));
        p.in_cap = ib;
        p.out_cap = ob;
    }
    return MMF_OK;
}

template <typename T>
cudaError_t run_chunk(const LaunchCtx &ctx, const void *in, const SeriesDesc &sd, void *omax, void *omin) {
    return blockscan_1d<T>(ctx, in, sd, omax, omin, true);
}

}  // namespace

extern "C" mmf_status mmf_filter1d_host(const void *h_in, int64_t n, int64_t w_or_r, mmf_dtype dtype, mmf_mode mode,
                                        void *h_max, void *h_min, int64_t chunk, void *stream) {
    NvtxRange nvtx_range("mmf_filter1d_host");
    const int esz = elem_size(dtype);
    if (esz == 0) return set_error(MMF_EINVAL, "unknown dtype %d", (int)dtype);
    SeriesDesc whole;
    mmf_status st = make_series(n, w_or_r, mode, dtype, &whole);
    if (st != MMF_OK) return st;
    if (whole.n_out == 0) return MMF_OK;
    if (!h_in || (!h_max && !h_min)) return set_error(MMF_EINVAL, "NULL buffers");
    if (((uintptr_t)h_in % esz) || ((uintptr_t)h_max % esz) || ((uintptr_t)h_min % esz))
        return set_error(MMF_EINVAL, "pointers must be aligned to the element size");
    if (chunk <= 0) chunk = int64_t(1) << 26;
    chunk = std::max<int64_t>(chunk, 4096);
    LaunchCtx ctx;
    st = get_ctx(stream, &ctx);
    if (st != MMF_OK) return st;
    Pipe &p = g_pipe[ctx.device & 63];
    std::lock_guard<std::mutex> lk(p.mu);
    const int64_t w = whole.w, d = whole.d;  // window length, start of output 0's window
    const int64_t cap = std::min(chunk, whole.n_out);
    st = pipe_setup(p, (size_t)(cap + w - 1) * esz, (size_t)cap * esz);
    if (st != MMF_OK) return st;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    // The pipeline starts after the work already on the caller's stream and
    // after the previous call has left the staging slots.
    cudaError_t e = cudaEventRecord(p.start, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p.s_in, p.start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p.s_in, p.last, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p.s_run, p.last, 0);
    const int64_t nchunks = (whole.n_out + chunk - 1) / chunk;
    for (int64_t c = 0; c < nchunks && e == cudaSuccess; ++c) {
        const int k = (int)(c % kSlots);
        const int64_t o0 = c * chunk, o1 = std::min(whole.n_out, o0 + chunk);
        const int64_t lo = std::max<int64_t>(0, o0 + d), hi = std::min<int64_t>(n, o1 - 1 + d + w);
        // Slot k is free once chunk c-kSlots has been filtered (input) and
        // downloaded (outputs).
        if (c >= kSlots) {
            e = cudaStreamWaitEvent(p.s_in, p.run_done[k], 0);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(p.s_run, p.out_done[k], 0);
            if (e != cudaSuccess) break;
        }
        e = cudaMemcpyAsync(p.in[k], static_cast<const char *>(h_in) + lo * esz, (size_t)(hi - lo) * esz,
                            cudaMemcpyHostToDevice, p.s_in);
        if (e == cudaSuccess) e = cudaEventRecord(p.in_done[k], p.s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p.s_run, p.in_done[k], 0);
        if (e != cudaSuccess) break;
        SeriesDesc sd{0, hi - lo, 0, w, (o0 + d) - lo, o1 - o0};
        LaunchCtx rctx = ctx;
        rctx.stream = p.s_run;
        switch (dtype) {
            case MMF_F32: e = run_chunk<float>(rctx, p.in[k], sd, h_max ? p.out_max[k] : nullptr, h_min ? p.out_min[k] : nullptr); break;
            case MMF_F64: e = run_chunk<double>(rctx, p.in[k], sd, h_max ? p.out_max[k] : nullptr, h_min ? p.out_min[k] : nullptr); break;
            case MMF_I16: e = run_chunk<int16_t>(rctx, p.in[k], sd, h_max ? p.out_max[k] : nullptr, h_min ? p.out_min[k] : nullptr); break;
            default: e = run_chunk<uint8_t>(rctx, p.in[k], sd, h_max ? p.out_max[k] : nullptr, h_min ? p.out_min[k] : nullptr); break;
        }
        if (e == cudaSuccess) e = cudaEventRecord(p.run_done[k], p.s_run);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p.s_out, p.run_done[k], 0);
        if (e == cudaSuccess && h_max)
            e = cudaMemcpyAsync(static_cast<char *>(h_max) + o0 * esz, p.out_max[k], (size_t)(o1 - o0) * esz,
                                cudaMemcpyDeviceToHost, p.s_out);
        if (e == cudaSuccess && h_min)
            e = cudaMemcpyAsync(static_cast<char *>(h_min) + o0 * esz, p.out_min[k], (size_t)(o1 - o0) * esz,
                                cudaMemcpyDeviceToHost, p.s_out);
        if (e == cudaSuccess) e = cudaEventRecord(p.out_done[k], p.s_out);
    }
    // The caller's stream completes when the last download does.
    if (e == cudaSuccess) e = cudaEventRecord(p.last, p.s_out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, p.last, 0);
    return e == cudaSuccess ? MMF_OK : cuda_error(e, "host pipeline");
}
