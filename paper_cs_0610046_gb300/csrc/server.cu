// Streaming service: many concurrent streams, each filtered with zero stream
// latency (Section 1: an output is emitted as soon as the last element of its
// window has arrived).  Each stream keeps its last w-1 samples (the halo) and
// its sample count (int64, as the paper advises for streams) on the device, so
// the outputs of a chunk are exactly those of the whole-array filter for the
// windows that end inside the chunk.
//
// Continuous batching: push() queues a chunk and returns a ticket.  A worker
// thread repeatedly admits queued chunks (FIFO, at most one chunk per stream
// in flight, while the device-memory budget allows), and runs each admitted
// batch as: the chunks placed behind their streams' halos, one batched filter
// launch per kernel group over all of them, one halo-update launch, and the
// outputs returned to the caller's host buffers.  Where the GPU can reach
// those host buffers itself (pinned memory, or any host memory on a system
// with pageable-memory access such as NVLink-C2C), a gather kernel reads the
// chunks and a scatter kernel writes the outputs; otherwise one copy per
// chunk and per output side is issued.  Batches
// rotate over a few CUDA streams so that copies and kernels of consecutive
// batches overlap; chunks that arrive while a batch runs join the next batch
// as soon as memory and their stream allow.  Completion is observed through
// events; the release-to-completion latency of every chunk is recorded.
//
// Device memory: the budget is split into a staging pool (halos and chunk
// inputs) and an output pool whose max and min halves mirror each other (a
// chunk's min outputs sit at the same offset in the min half).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "arena.h"
#include "launch.h"
#include "mmf.h"

namespace mmf {
mmf_status set_error(mmf_status st, const char *fmt, ...);
mmf_status cuda_error(cudaError_t e, const char *what);
mmf_status get_ctx(void *stream, LaunchCtx *ctx);
int elem_size(mmf_dtype dt);

// Copies the new halo of each stream of a batch: the last h_new elements of
// its staging block [halo | chunk].  lim: elements of the staging arena at
// base (range checks of a checked build).
template <typename T>
__global__ void halo_update_kernel(const SeriesDesc *series, const int64_t *halo_off, const int64_t *h_new,
                                   T *base, int n, int64_t lim, uint32_t *status) {
    const int i = blockIdx.x;
    if (i >= n) return;
    const SeriesDesc sd = series[i];
    const int64_t h = h_new[i];
    const int64_t s0 = sd.in_off + sd.n - h, d0 = halo_off[i];
    for (int64_t k = threadIdx.x; k < h; k += blockDim.x)
        if (in_range(status, s0 + k, 0, lim) && in_range(status, d0 + k, 0, lim)) base[d0 + k] = base[s0 + k];
}
// Per-chunk copy descriptor of a batch (offsets in elements).
struct ChunkCopy {
    const void *h_in;  // host chunk (device-accessible)
    void *h_max;       // host outputs (device-accessible, may be null)
    void *h_min;
    int64_t len, stage_off, halo_off, halo_len, out_off, n_out;
};

// Builds every staging block [halo | chunk] of a batch: the halo from the
// stream's device state, the chunk straight from host memory (over the
// CPU-GPU link).  blockIdx.y strides over the chunk.
template <typename T>
__global__ void gather_kernel(const ChunkCopy *cc, int n, T *base, int64_t lim, uint32_t *status) {
    const int i = blockIdx.x;
    if (i >= n) return;
    const ChunkCopy c = cc[i];
    T *stage = base + c.stage_off;
    const int64_t tot = c.halo_len + c.len;
    const int64_t stride = (int64_t)gridDim.y * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; k < tot; k += stride) {
        if (!in_range(status, c.stage_off + k, 0, lim)) continue;
        if (k < c.halo_len)
            stage[k] = in_range(status, c.halo_off + k, 0, lim) ? base[c.halo_off + k] : T(0);
        else
            stage[k] = static_cast<const T *>(c.h_in)[k - c.halo_len];  // k - halo_len < len: the chunk
    }
}

// Writes every chunk's outputs straight to its host buffers.
// lim: elements of each output half (range checks of a checked build).
template <typename T>
__global__ void scatter_kernel(const ChunkCopy *cc, int n, const T *omax, const T *omin, int64_t lim,
                               uint32_t *status) {
    const int i = blockIdx.x;
    if (i >= n) return;
    const ChunkCopy c = cc[i];
    const int64_t stride = (int64_t)gridDim.y * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; k < c.n_out; k += stride) {
        if (!in_range(status, c.out_off + k, 0, lim)) continue;
        if (c.h_max) static_cast<T *>(c.h_max)[k] = omax[c.out_off + k];
        if (c.h_min) static_cast<T *>(c.h_min)[k] = omin[c.out_off + k];
    }
}
}  // namespace mmf

using namespace mmf;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    uint64_t stream;
    const void *h_in;
    int64_t len;
    void *h_max, *h_min;
    int64_t n_out;
    bool direct;  // the GPU can read/write these host buffers itself
    Clock::time_point released;  // pushed
    Clock::time_point admitted;  // taken into a batch
};

struct StreamState {
    int64_t w = 0;
    int64_t count = 0;      // samples pushed so far (int64: unbounded streams)
    int64_t halo_off = -1;  // staging-arena block of w-1 elements
    int64_t halo_len = 0;   // min(count, w-1) once the pushes so far are done
    bool in_flight = false;
    bool closed = false;
    int64_t pending = 0;    // queued or in flight
    int64_t queued = 0;     // samples of this stream's chunks still in the queue
};

struct Batch {
    std::vector<Request> reqs;
    std::vector<std::pair<int64_t, size_t>> stage_blocks, out_blocks;
    std::vector<int64_t> halo_after;
    cudaEvent_t done = nullptr;
};

constexpr int kSlots = 3;  // CUDA streams that batches rotate over
constexpr int64_t kTicketDone = 1, kTicketFailed = 2;

}  // namespace

struct mmf_server {
    int device = 0;
    mmf_dtype dtype = MMF_F32;
    int64_t esz = 4;
    int max_batch = 256;
    char *dev_base = nullptr;  // one allocation: staging arena, then output halves
    size_t stage_size = 0, out_half = 0;
    Arena stage, out;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::unordered_map<uint64_t, StreamState> streams;
    std::list<Request> queue;  // admission order; admitted chunks leave from anywhere
    std::deque<Batch> inflight;
    std::unordered_map<uint64_t, int64_t> tickets;  // 0 pending, 1 done, 2 failed
    uint64_t next_stream = 1, next_ticket = 1;
    bool stop = false, paused = false;
    mmf_status failed = MMF_OK;
    std::thread worker;
    cudaStream_t slots[kSlots] = {};
    cudaEvent_t slot_free[kSlots] = {};
    SeriesDesc *d_series[kSlots] = {};
    ItemDesc *d_items[kSlots] = {};
    int64_t *d_halo[kSlots] = {};  // [2][max_batch]: halo offsets, new halo lengths
    int *d_tick[kSlots] = {};
    SeriesDesc *h_series[kSlots] = {};  // pinned staging of the tables
    ItemDesc *h_items[kSlots] = {};
    int64_t *h_halo[kSlots] = {};
    ChunkCopy *d_copy[kSlots] = {};
    ChunkCopy *h_copy[kSlots] = {};
    bool pageable_ok = false;  // the device can access pageable host memory
    uint64_t nbatches = 0;
    std::vector<double> lat_ms, queue_ms, service_ms;  // per chunk: push to completion, push to admission, admission to completion
    double max_hold_ms = 0.0;  // longest stretch the worker held the lock in one batch's set-up
    cudaEvent_t slot_done[kSlots] = {};  // completion of the batch on each slot (reused, never created per batch)
    int64_t done_chunks = 0, done_elems = 0;
};

namespace {

int mode_for(mmf_dtype dt, int64_t w) {
    switch (dt) {
        case MMF_F32: return block_mode<float>(w, true);
        case MMF_F64: return block_mode<double>(w, true);
        case MMF_I16: return block_mode<int16_t>(w, true);
        default: return block_mode<uint8_t>(w, true);
    }
}

cudaError_t launch_group(mmf_server *S, const LaunchCtx &ctx, int g, int slot, const ItemDesc *items, int64_t ni) {
    char *base = S->dev_base;
    char *omax = base + S->stage_size, *omin = omax + S->out_half;
    const int64_t stage_elems = (int64_t)(S->stage_size / S->esz);
    switch (S->dtype) {
        case MMF_F32: return blockscan_table<float>(ctx, g, base, stage_elems, omax, omin, S->d_series[slot], items, ni, S->d_tick[slot] + g, 0);
        case MMF_F64: return blockscan_table<double>(ctx, g, base, stage_elems, omax, omin, S->d_series[slot], items, ni, S->d_tick[slot] + g, 0);
        case MMF_I16: return blockscan_table<int16_t>(ctx, g, base, stage_elems, omax, omin, S->d_series[slot], items, ni, S->d_tick[slot] + g, 0);
        default: return blockscan_table<uint8_t>(ctx, g, base, stage_elems, omax, omin, S->d_series[slot], items, ni, S->d_tick[slot] + g, 0);
    }
}

cudaError_t launch_halo(mmf_server *S, int slot, int n, cudaStream_t st, uint32_t *status) {
    const int64_t *hoff = S->d_halo[slot];
    const int64_t *hnew = hoff + S->max_batch;
    const int64_t lim = (int64_t)S->stage_size / S->esz;
    switch (S->dtype) {
        case MMF_F32: halo_update_kernel<float><<<n, 256, 0, st>>>(S->d_series[slot], hoff, hnew, (float *)S->dev_base, n, lim, status); break;
        case MMF_F64: halo_update_kernel<double><<<n, 256, 0, st>>>(S->d_series[slot], hoff, hnew, (double *)S->dev_base, n, lim, status); break;
        case MMF_I16: halo_update_kernel<int16_t><<<n, 256, 0, st>>>(S->d_series[slot], hoff, hnew, (int16_t *)S->dev_base, n, lim, status); break;
        default: halo_update_kernel<uint8_t><<<n, 256, 0, st>>>(S->d_series[slot], hoff, hnew, (uint8_t *)S->dev_base, n, lim, status); break;
    }
    return cudaGetLastError();
}

// With S->mu held: admit one batch and enqueue its work (the lock is dropped
// around the CUDA calls).  Returns false if nothing could be admitted.
bool run_batch(mmf_server *S, std::unique_lock<std::mutex> &lk) {
    NvtxRange nvtx_range("mmf_server_batch");
    const auto t_lock = Clock::now();
    const int slot = (int)(S->nbatches % kSlots);
    // The slot's pinned tables and device tables are reused: wait for the
    // batch that last used this slot to have finished its uploads.
    if (cudaEventQuery(S->slot_free[slot]) == cudaErrorNotReady) return false;
    Batch b;
    std::vector<int64_t> stage_off, out_off, halo_before;
    const int64_t esz = S->esz;
    for (auto it = S->queue.begin(); it != S->queue.end() && (int)b.reqs.size() < S->max_batch;) {
        StreamState &ss = S->streams[it->stream];
        if (ss.in_flight) {
            ++it;
            continue;
        }
        const int64_t h = ss.halo_len;
        const size_t in_bytes = (size_t)(h + it->len) * esz;
        const size_t out_bytes = (size_t)it->n_out * esz;
        const int64_t ib = S->stage.alloc(in_bytes);
        if (ib < 0) break;  // no room: wait for completions (FIFO admission)
        const int64_t ob = S->out.alloc(out_bytes);
        if (ob < 0) {
            S->stage.release(ib, in_bytes);
            break;
        }
        ss.in_flight = true;
        ss.queued -= it->len;
        b.reqs.push_back(*it);
        b.stage_blocks.push_back({ib, in_bytes});
        b.out_blocks.push_back({ob, out_bytes});
        stage_off.push_back(ib);
        out_off.push_back(ob);
        halo_before.push_back(h);
        // State after this chunk (used by the next chunk of the stream, which
        // cannot be admitted before this one completes).
        ss.count += it->len;
        ss.halo_len = std::min<int64_t>(ss.count, ss.w - 1);
        b.halo_after.push_back(ss.halo_len);
        b.reqs.back().admitted = t_lock;
        it = S->queue.erase(it);
    }
    if (b.reqs.empty()) return false;
    S->nbatches++;
    const int n = (int)b.reqs.size();
    int64_t counts[4] = {0, 0, 0, 0};
    std::vector<int> modes(n);
    std::vector<int64_t> hoffs(n);
    for (int i = 0; i < n; ++i) {
        const Request &r = b.reqs[i];
        const StreamState &ss = S->streams[r.stream];
        SeriesDesc &sd = S->h_series[slot][i];
        sd.in_off = stage_off[i] / esz;
        sd.n = halo_before[i] + r.len;
        sd.out_off = out_off[i] / esz;
        sd.w = ss.w;
        sd.d = 0;
        sd.n_out = r.n_out;
        modes[i] = mode_for(S->dtype, ss.w);
        if (r.n_out > 0) counts[modes[i]]++;  // chunks without outputs only move the halo
        hoffs[i] = ss.halo_off;
        S->h_halo[slot][i] = ss.halo_off / esz;
        S->h_halo[slot][S->max_batch + i] = b.halo_after[i];
    }
    int64_t pos[4], acc = 0;
    for (int g = 0; g < 4; ++g) {
        pos[g] = acc;
        acc += counts[g];
    }
    for (int i = 0; i < n; ++i)
        if (b.reqs[i].n_out > 0) S->h_items[slot][pos[modes[i]]++] = {i, 0, b.reqs[i].n_out};
    S->max_hold_ms = std::max(S->max_hold_ms, std::chrono::duration<double, std::milli>(Clock::now() - t_lock).count());
    lk.unlock();

    cudaStream_t st = S->slots[slot];
    char *base = S->dev_base;
    char *omax = base + S->stage_size, *omin = omax + S->out_half;
    cudaError_t e = cudaSuccess;
    // Copy descriptors: direct chunks go through the gather/scatter kernels,
    // the others through one copy call per buffer.
    int nd = 0;
    int64_t maxlen = 1, maxout = 1;
    for (int i = 0; i < n; ++i) {
        const Request &r = b.reqs[i];
        if (!r.direct) continue;
        ChunkCopy &c = S->h_copy[slot][nd++];
        c.h_in = r.h_in;
        c.h_max = r.h_max;
        c.h_min = r.h_min;
        c.len = r.len;
        c.stage_off = stage_off[i] / esz;
        c.halo_off = hoffs[i] / esz;
        c.halo_len = halo_before[i];
        c.out_off = out_off[i] / esz;
        c.n_out = r.n_out;
        maxlen = std::max(maxlen, halo_before[i] + r.len);
        maxout = std::max(maxout, r.n_out);
    }
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const Request &r = b.reqs[i];
        if (r.direct) continue;
        char *stage = base + stage_off[i];
        if (halo_before[i] > 0)
            e = cudaMemcpyAsync(stage, base + hoffs[i], halo_before[i] * esz, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && r.len > 0)
            e = cudaMemcpyAsync(stage + halo_before[i] * esz, r.h_in, r.len * esz, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess && nd > 0)
        e = cudaMemcpyAsync(S->d_copy[slot], S->h_copy[slot], nd * sizeof(ChunkCopy), cudaMemcpyHostToDevice, st);
    LaunchCtx ctx;
    if (e == cudaSuccess && get_ctx(st, &ctx) != MMF_OK) e = cudaErrorUnknown;
    const int64_t stage_lim = (int64_t)S->stage_size / esz, out_lim = (int64_t)S->out_half / esz;
    if (e == cudaSuccess && nd > 0) {
        const dim3 g(nd, (unsigned)std::min<int64_t>(32, (maxlen + 2047) / 2048));
        switch (S->dtype) {
            case MMF_F32: gather_kernel<float><<<g, 256, 0, st>>>(S->d_copy[slot], nd, (float *)base, stage_lim, ctx.status); break;
            case MMF_F64: gather_kernel<double><<<g, 256, 0, st>>>(S->d_copy[slot], nd, (double *)base, stage_lim, ctx.status); break;
            case MMF_I16: gather_kernel<int16_t><<<g, 256, 0, st>>>(S->d_copy[slot], nd, (int16_t *)base, stage_lim, ctx.status); break;
            default: gather_kernel<uint8_t><<<g, 256, 0, st>>>(S->d_copy[slot], nd, (uint8_t *)base, stage_lim, ctx.status); break;
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->d_series[slot], S->h_series[slot], n * sizeof(SeriesDesc), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->d_items[slot], S->h_items[slot], n * sizeof(ItemDesc), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->d_halo[slot], S->h_halo[slot], 2 * S->max_batch * sizeof(int64_t),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(S->slot_free[slot], st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->d_tick[slot], 0, 4 * sizeof(int), st);
    int64_t first = 0;
    for (int g = 0; g < 4 && e == cudaSuccess; ++g) {
        if (counts[g]) e = launch_group(S, ctx, g, slot, S->d_items[slot] + first, counts[g]);
        first += counts[g];
    }
    if (e == cudaSuccess) e = launch_halo(S, slot, n, st, ctx.status);
    if (e == cudaSuccess && nd > 0) {
        const dim3 g(nd, (unsigned)std::min<int64_t>(32, (maxout + 2047) / 2048));
        switch (S->dtype) {
            case MMF_F32: scatter_kernel<float><<<g, 256, 0, st>>>(S->d_copy[slot], nd, (const float *)omax, (const float *)omin, out_lim, ctx.status); break;
            case MMF_F64: scatter_kernel<double><<<g, 256, 0, st>>>(S->d_copy[slot], nd, (const double *)omax, (const double *)omin, out_lim, ctx.status); break;
            case MMF_I16: scatter_kernel<int16_t><<<g, 256, 0, st>>>(S->d_copy[slot], nd, (const int16_t *)omax, (const int16_t *)omin, out_lim, ctx.status); break;
            default: scatter_kernel<uint8_t><<<g, 256, 0, st>>>(S->d_copy[slot], nd, (const uint8_t *)omax, (const uint8_t *)omin, out_lim, ctx.status); break;
        }
        e = cudaGetLastError();
    }
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const Request &r = b.reqs[i];
        if (r.direct || r.n_out == 0) continue;
        if (r.h_max) e = cudaMemcpyAsync(r.h_max, omax + out_off[i], r.n_out * esz, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && r.h_min)
            e = cudaMemcpyAsync(r.h_min, omin + out_off[i], r.n_out * esz, cudaMemcpyDeviceToHost, st);
    }
    // The slot's completion event: the batch that used this slot before was
    // retired (at most kSlots - 1 batches are in flight when one starts, and
    // batches retire in order), so the event is free to record again.
    b.done = S->slot_done[slot];
    if (e == cudaSuccess) e = cudaEventRecord(b.done, st);
    lk.lock();
    if (e != cudaSuccess) {
        S->failed = MMF_ECUDA;
        set_error(MMF_ECUDA, "serving batch: %s", cudaGetErrorString(e));
    }
    S->inflight.push_back(std::move(b));
    return true;
}

// With S->mu held: retire finished batches in order.
void retire(mmf_server *S) {
    while (!S->inflight.empty()) {
        Batch &b = S->inflight.front();
        cudaError_t q = b.done ? cudaEventQuery(b.done) : cudaErrorUnknown;
        if (q == cudaErrorNotReady) break;
        const auto now = Clock::now();
        for (size_t i = 0; i < b.reqs.size(); ++i) {
            const Request &r = b.reqs[i];
            S->stage.release(b.stage_blocks[i].first, b.stage_blocks[i].second);
            S->out.release(b.out_blocks[i].first, b.out_blocks[i].second);
            auto sit = S->streams.find(r.stream);
            if (sit != S->streams.end()) {
                sit->second.in_flight = false;
                sit->second.pending--;
            }
            S->tickets[r.ticket] = q == cudaSuccess ? kTicketDone : kTicketFailed;
            S->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r.released).count());
            S->queue_ms.push_back(std::chrono::duration<double, std::milli>(r.admitted - r.released).count());
            S->service_ms.push_back(std::chrono::duration<double, std::milli>(now - r.admitted).count());
            S->done_chunks++;
            S->done_elems += r.len;
        }
        if (q != cudaSuccess) S->failed = MMF_ECUDA;
        S->inflight.pop_front();
        S->cv_done.notify_all();
    }
}

void worker_main(mmf_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        retire(S);
        bool launched = false;
        if (!S->paused && !S->queue.empty() && S->inflight.size() < (size_t)kSlots) launched = run_batch(S, lk);
        if (launched) continue;
        if (!S->inflight.empty()) {
            // Poll completions without holding the lock for long.
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        } else {
            S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
    // Drain whatever is still on the GPU before the buffers go away.
    while (!S->inflight.empty()) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(50));
        lk.lock();
        retire(S);
    }
}

}  // namespace

// Pinned (page-locked) host memory is accessible from kernels; so is any host
// memory where the device supports pageable access.
bool device_accessible(const void *p) {
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeManaged || a.type == cudaMemoryTypeDevice;
}

extern "C" {

mmf_status mmf_server_create(size_t device_budget_bytes, int max_batch, mmf_dtype dtype, mmf_server **out) {
    if (!out) return set_error(MMF_EINVAL, "NULL server output");
    *out = nullptr;
    if (elem_size(dtype) == 0) return set_error(MMF_EINVAL, "unknown dtype %d", (int)dtype);
    if (max_batch < 1 || max_batch > 65536) return set_error(MMF_EINVAL, "max_batch out of range");
    if (device_budget_bytes < (1u << 20)) return set_error(MMF_EINVAL, "budget below 1 MiB");
    mmf_server *S = new (std::nothrow) mmf_server();
    if (!S) return set_error(MMF_ENOMEM, "server");
    cudaGetDevice(&S->device);
    S->dtype = dtype;
    S->esz = elem_size(dtype);
    S->max_batch = max_batch;
    // Budget: half for staging (halos + chunk inputs), half for the outputs
    // (two mirrored quarters: max and min).
    S->out_half = (device_budget_bytes / 4) & ~size_t(255);
    S->stage_size = (device_budget_bytes - 2 * S->out_half) & ~size_t(255);
    cudaError_t e = cudaMalloc(&S->dev_base, S->stage_size + 2 * S->out_half);
    for (int k = 0; k < kSlots && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&S->slots[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->slot_free[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->slot_done[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&S->d_series[k], max_batch * sizeof(SeriesDesc));
        if (e == cudaSuccess) e = cudaMalloc(&S->d_items[k], max_batch * sizeof(ItemDesc));
        if (e == cudaSuccess) e = cudaMalloc(&S->d_halo[k], 2 * max_batch * sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMalloc(&S->d_tick[k], 4 * sizeof(int));
        if (e == cudaSuccess) e = cudaMallocHost(&S->h_series[k], max_batch * sizeof(SeriesDesc));
        if (e == cudaSuccess) e = cudaMallocHost(&S->h_items[k], max_batch * sizeof(ItemDesc));
        if (e == cudaSuccess) e = cudaMallocHost(&S->h_halo[k], 2 * max_batch * sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMalloc(&S->d_copy[k], max_batch * sizeof(ChunkCopy));
        if (e == cudaSuccess) e = cudaMallocHost(&S->h_copy[k], max_batch * sizeof(ChunkCopy));
    }
    int pageable = 0;
    if (e == cudaSuccess) cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, S->device);
    S->pageable_ok = pageable != 0;
    if (e != cudaSuccess) {
        set_error(MMF_ENOMEM, "server resources: %s", cudaGetErrorString(e));
        mmf_server_destroy(S);
        return MMF_ENOMEM;
    }
    S->stage.init(S->stage_size);
    S->out.init(S->out_half);
    // Kernel attributes are set here, outside any capture or worker race.
    for (int g = 0; g < 4; ++g) {
        switch (dtype) {
            case MMF_F32: blockscan_prepare<float>(S->device, g); break;
            case MMF_F64: blockscan_prepare<double>(S->device, g); break;
            case MMF_I16: blockscan_prepare<int16_t>(S->device, g); break;
            case MMF_U8: blockscan_prepare<uint8_t>(S->device, g); break;
        }
    }
    // Room for many outstanding tickets and latency samples up front, so that
    // neither rehashes nor regrows under the lock while chunks stream in.
    S->tickets.reserve(1 << 20);
    S->lat_ms.reserve(1 << 20);
    S->queue_ms.reserve(1 << 20);
    S->service_ms.reserve(1 << 20);
    S->worker = std::thread(worker_main, S);
    *out = S;
    return MMF_OK;
}

void mmf_server_destroy(mmf_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->paused = false;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (int k = 0; k < kSlots; ++k) {
        if (S->slots[k]) cudaStreamSynchronize(S->slots[k]);
        if (S->slots[k]) cudaStreamDestroy(S->slots[k]);
        if (S->slot_free[k]) cudaEventDestroy(S->slot_free[k]);
        if (S->slot_done[k]) cudaEventDestroy(S->slot_done[k]);
        if (S->d_series[k]) cudaFree(S->d_series[k]);
        if (S->d_items[k]) cudaFree(S->d_items[k]);
        if (S->d_halo[k]) cudaFree(S->d_halo[k]);
        if (S->d_tick[k]) cudaFree(S->d_tick[k]);
        if (S->h_series[k]) cudaFreeHost(S->h_series[k]);
        if (S->h_items[k]) cudaFreeHost(S->h_items[k]);
        if (S->h_halo[k]) cudaFreeHost(S->h_halo[k]);
        if (S->d_copy[k]) cudaFree(S->d_copy[k]);
        if (S->h_copy[k]) cudaFreeHost(S->h_copy[k]);
    }
    if (S->dev_base) cudaFree(S->dev_base);
    delete S;
}

mmf_status mmf_stream_open(mmf_server *S, int64_t w, uint64_t *stream_id) {
    if (!S || !stream_id) return set_error(MMF_EINVAL, "NULL argument");
    if (w < 1) return set_error(MMF_EINVAL, "window w = %lld < 1", (long long)w);
    // Compared in elements so that (w-1)*esz cannot wrap around.
    if ((uint64_t)(w - 1) > S->stage.size() / (uint64_t)S->esz)
        return set_error(MMF_ENOMEM, "a window of %lld needs a halo larger than the device budget", (long long)w);
    std::lock_guard<std::mutex> lk(S->mu);
    StreamState ss;
    ss.w = w;
    if (w > 1) {
        ss.halo_off = S->stage.alloc((size_t)(w - 1) * S->esz);
        if (ss.halo_off < 0) return set_error(MMF_ENOMEM, "no device memory left for the stream state");
    }
    const uint64_t id = S->next_stream++;
    S->streams[id] = ss;
    *stream_id = id;
    return MMF_OK;
}

}  // extern "C"

namespace {
// With S->mu held: queue one chunk (see mmf_stream_push).
mmf_status push_locked(mmf_server *S, uint64_t stream_id, const void *h_chunk, int64_t len, void *h_max,
                       void *h_min, int64_t *n_out, uint64_t *ticket) {
    if (len < 0 || (len > 0 && !h_chunk)) return set_error(MMF_EINVAL, "bad chunk");
    // Compared in elements before any byte count is formed (no wrap-around).
    if ((uint64_t)len > S->stage.size() / (uint64_t)S->esz)
        return set_error(MMF_ENOMEM, "chunk larger than the device budget allows");
    if (S->failed != MMF_OK) return set_error(MMF_EDEVICE, "the server failed earlier");
    auto it = S->streams.find(stream_id);
    if (it == S->streams.end() || it->second.closed)
        return set_error(MMF_ECLOSED, "stream %llu is not open", (unsigned long long)stream_id);
    StreamState &ss = it->second;
    // Outputs of this chunk: windows that end inside it (zero latency).  The
    // stream's queued chunks come first.
    const int64_t before = ss.count + ss.queued;
    const int64_t done_before = std::max<int64_t>(0, before - ss.w + 1);
    const int64_t done_after = std::max<int64_t>(0, before + len - ss.w + 1);
    const int64_t m = done_after - done_before;
    if (m > 0 && !h_max && !h_min) return set_error(MMF_EINVAL, "both outputs are NULL");
    const size_t in_need = Arena::round((size_t)(std::min<int64_t>(before, ss.w - 1) + len) * S->esz);
    if (in_need > S->stage.size() || Arena::round((size_t)m * S->esz) > S->out.size())
        return set_error(MMF_ENOMEM, "chunk larger than the device budget allows");
    Request r;
    r.direct = S->pageable_ok || (device_accessible(h_chunk) && device_accessible(h_max) && device_accessible(h_min));
    r.ticket = S->next_ticket++;
    r.stream = stream_id;
    r.h_in = h_chunk;
    r.len = len;
    r.h_max = h_max;
    r.h_min = h_min;
    r.n_out = m;
    r.released = Clock::now();
    S->queue.push_back(r);
    S->tickets[r.ticket] = 0;
    ss.pending++;
    ss.queued += len;
    if (n_out) *n_out = m;
    *ticket = r.ticket;
    return MMF_OK;
}
}  // namespace

extern "C" {

mmf_status mmf_stream_push(mmf_server *S, uint64_t stream_id, const void *h_chunk, int64_t len, void *h_max,
                           void *h_min, int64_t *n_out, uint64_t *ticket) {
    NvtxRange nvtx_range("mmf_stream_push");
    if (!S || !ticket) return set_error(MMF_EINVAL, "NULL argument");
    mmf_status st;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        st = push_locked(S, stream_id, h_chunk, len, h_max, h_min, n_out, ticket);
    }
    if (st == MMF_OK) S->cv_work.notify_one();
    return st;
}

mmf_status mmf_stream_push_batch(mmf_server *S, int64_t count, const uint64_t *stream_ids,
                                 const void *const *h_chunks, const int64_t *lens, void *const *h_max,
                                 void *const *h_min, int64_t *n_out, uint64_t *tickets, int64_t *n_done) {
    NvtxRange nvtx_range("mmf_stream_push_batch");
    if (!S || count < 0 || (count > 0 && (!stream_ids || !h_chunks || !lens || !tickets)))
        return set_error(MMF_EINVAL, "NULL argument");
    mmf_status st = MMF_OK;
    int64_t i = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (; i < count; ++i) {
            st = push_locked(S, stream_ids[i], h_chunks[i], lens[i], h_max ? h_max[i] : nullptr,
                             h_min ? h_min[i] : nullptr, n_out ? n_out + i : nullptr, tickets + i);
            if (st != MMF_OK) break;
        }
    }
    if (n_done) *n_done = i;
    if (i > 0) S->cv_work.notify_one();
    return st;
}

mmf_status mmf_ticket_wait(mmf_server *S, uint64_t ticket, int timeout_ms) {
    if (!S) return set_error(MMF_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return set_error(MMF_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (S->tickets[ticket] == 0) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && S->tickets[ticket] == 0)
            return set_error(MMF_ETIMEOUT, "ticket %llu not done after %d ms", (unsigned long long)ticket, timeout_ms);
    }
    const int64_t st = S->tickets[ticket];
    S->tickets.erase(ticket);
    return st == kTicketDone ? MMF_OK : set_error(MMF_EDEVICE, "the batch of ticket %llu failed", (unsigned long long)ticket);
}

mmf_status mmf_ticket_wait_batch(mmf_server *S, int64_t count, const uint64_t *tickets, int timeout_ms) {
    if (!S || count < 0 || (count > 0 && !tickets)) return set_error(MMF_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    bool failed = false;
    for (int64_t i = 0; i < count; ++i) {
        auto it = S->tickets.find(tickets[i]);
        if (it == S->tickets.end()) return set_error(MMF_EINVAL, "unknown ticket %llu", (unsigned long long)tickets[i]);
        while (it->second == 0) {
            if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && it->second == 0)
                return set_error(MMF_ETIMEOUT, "ticket %llu not done after %d ms (%lld of %lld done)",
                                 (unsigned long long)tickets[i], timeout_ms, (long long)i, (long long)count);
        }
        failed |= it->second != kTicketDone;
        S->tickets.erase(it);
    }
    return failed ? set_error(MMF_EDEVICE, "a batch of these tickets failed") : MMF_OK;
}

mmf_status mmf_stream_close(mmf_server *S, uint64_t stream_id, int timeout_ms) {
    if (!S) return set_error(MMF_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->streams.find(stream_id);
    if (it == S->streams.end() || it->second.closed) return set_error(MMF_ECLOSED, "stream %llu is not open", (unsigned long long)stream_id);
    it->second.closed = true;  // no new pushes
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (S->streams[stream_id].pending > 0) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && S->streams[stream_id].pending > 0)
            return set_error(MMF_ETIMEOUT, "stream %llu still has chunks after %d ms", (unsigned long long)stream_id, timeout_ms);
    }
    StreamState ss = S->streams[stream_id];
    if (ss.halo_off >= 0) S->stage.release(ss.halo_off, (size_t)(ss.w - 1) * S->esz);
    S->streams.erase(stream_id);
    return MMF_OK;
}

namespace {
struct SnapshotHeader {
    uint32_t magic;
    uint32_t version;
    int32_t dtype;
    int32_t zero;
    int64_t w;
    int64_t count;
    int64_t halo_len;
};
static_assert(sizeof(SnapshotHeader) == MMF_SNAPSHOT_HEADER_BYTES, "snapshot header layout");
}  // namespace

}  // extern "C"

namespace {
// The halo of a stream: its last h samples as host bytes, after its pending
// chunks complete (snapshot helpers; S->mu held by the caller).
mmf_status snapshot_halo(mmf_server *S, uint64_t stream_id, int timeout_ms, std::unique_lock<std::mutex> &lk,
                         StreamState *out, std::vector<char> *halo) {
    auto it = S->streams.find(stream_id);
    if (it == S->streams.end() || it->second.closed)
        return set_error(MMF_ECLOSED, "stream %llu is not open", (unsigned long long)stream_id);
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (S->streams[stream_id].pending > 0) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && S->streams[stream_id].pending > 0)
            return set_error(MMF_ETIMEOUT, "stream %llu still has chunks after %d ms", (unsigned long long)stream_id,
                             timeout_ms);
    }
    if (S->failed != MMF_OK) return set_error(MMF_EDEVICE, "the server failed earlier");
    *out = S->streams[stream_id];
    halo->assign((size_t)out->halo_len * S->esz, 0);
    if (out->halo_len > 0) {
        cudaSetDevice(S->device);
        cudaError_t e = cudaMemcpy(halo->data(), S->dev_base + out->halo_off, halo->size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_error(e, "snapshot copy");
    }
    return MMF_OK;
}

// Positions (0..h-1) of the samples strictly above (MAX) or below every later
// one, oldest first: the monotonic wedge's deque of that side.
template <typename T, bool MAX> void wedge_side(const T *a, int64_t h, std::vector<int64_t> *out) {
    out->clear();
    for (int64_t k = 0; k < h; ++k) {
        while (!out->empty() && (MAX ? !(a[out->back()] > a[k]) : !(a[out->back()] < a[k]))) out->pop_back();
        out->push_back(k);
    }
}

template <typename T>
void wedge_sides(const char *halo, int64_t h, std::vector<int64_t> *u, std::vector<int64_t> *l) {
    const T *a = reinterpret_cast<const T *>(halo);
    wedge_side<T, true>(a, h, u);
    wedge_side<T, false>(a, h, l);
}

// A halo with the same later outputs as the wedge: samples of U or L keep
// their values, every other one takes the value of the nearest later sample
// of U (within every later window that holds it, and at least as large).
template <typename T>
void halo_from_wedge(const char *entries, int64_t nu, int64_t nl, int64_t h, char *halo) {
    T *a = reinterpret_cast<T *>(halo);
    std::vector<char> set(h, 0);
    std::vector<T> uval(h);
    const size_t rec = 8 + sizeof(T);
    for (int64_t j = 0; j < nu + nl; ++j) {
        int64_t back;
        T v;
        memcpy(&back, entries + j * rec, 8);
        memcpy(&v, entries + j * rec + 8, sizeof(T));
        const int64_t k = h - back;
        a[k] = v;
        set[k] = 1;
        if (j < nu) set[k] = 2;  // in U
    }
    T last = a[h - 1];  // the newest sample is in both deques
    for (int64_t k = h - 1; k >= 0; --k) {
        if (set[k] == 2) last = a[k];
        else if (set[k] == 0) a[k] = last;
    }
}
}  // namespace

extern "C" {

mmf_status mmf_stream_snapshot(mmf_server *S, uint64_t stream_id, void *h_buf, size_t buf_bytes, size_t *size,
                               int timeout_ms) {
    NvtxRange nvtx_range("mmf_stream_snapshot");
    if (!S || !size) return set_error(MMF_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    StreamState ss;
    std::vector<char> halo;
    mmf_status st = snapshot_halo(S, stream_id, timeout_ms, lk, &ss, &halo);
    if (st != MMF_OK) return st;
    const size_t need = sizeof(SnapshotHeader) + halo.size();
    *size = need;
    if (!h_buf) return MMF_OK;
    if (buf_bytes < need) return set_error(MMF_EINVAL, "snapshot needs %zu bytes", need);
    SnapshotHeader hd{MMF_SNAPSHOT_MAGIC, 1u, (int32_t)S->dtype, 0, ss.w, ss.count, ss.halo_len};
    memcpy(h_buf, &hd, sizeof(hd));
    if (!halo.empty()) memcpy(static_cast<char *>(h_buf) + sizeof(hd), halo.data(), halo.size());
    return MMF_OK;
}

mmf_status mmf_stream_snapshot_wedge(mmf_server *S, uint64_t stream_id, void *h_buf, size_t buf_bytes, size_t *size,
                                     int timeout_ms) {
    NvtxRange nvtx_range("mmf_stream_snapshot_wedge");
    if (!S || !size) return set_error(MMF_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    StreamState ss;
    std::vector<char> halo;
    mmf_status st = snapshot_halo(S, stream_id, timeout_ms, lk, &ss, &halo);
    if (st != MMF_OK) return st;
    std::vector<int64_t> u, l;
    switch (S->dtype) {
        case MMF_F32: wedge_sides<float>(halo.data(), ss.halo_len, &u, &l); break;
        case MMF_F64: wedge_sides<double>(halo.data(), ss.halo_len, &u, &l); break;
        case MMF_I16: wedge_sides<int16_t>(halo.data(), ss.halo_len, &u, &l); break;
        default: wedge_sides<uint8_t>(halo.data(), ss.halo_len, &u, &l); break;
    }
    const size_t rec = 8 + (size_t)S->esz;
    const size_t need = sizeof(SnapshotHeader) + 16 + (u.size() + l.size()) * rec;
    *size = need;
    if (!h_buf) return MMF_OK;
    if (buf_bytes < need) return set_error(MMF_EINVAL, "snapshot needs %zu bytes", need);
    char *p = static_cast<char *>(h_buf);
    SnapshotHeader hd{MMF_SNAPSHOT_MAGIC, 2u, (int32_t)S->dtype, 0, ss.w, ss.count, ss.halo_len};
    memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    const int64_t nu = (int64_t)u.size(), nl = (int64_t)l.size();
    memcpy(p, &nu, 8);
    memcpy(p + 8, &nl, 8);
    p += 16;
    for (const auto *side : {&u, &l}) {
        for (int64_t k : *side) {
            const int64_t back = ss.halo_len - k;
            memcpy(p, &back, 8);
            memcpy(p + 8, halo.data() + k * S->esz, S->esz);
            p += rec;
        }
    }
    return MMF_OK;
}

mmf_status mmf_stream_restore(mmf_server *S, const void *h_buf, size_t buf_bytes, uint64_t *stream_id) {
    NvtxRange nvtx_range("mmf_stream_restore");
    if (!S || !h_buf || !stream_id) return set_error(MMF_EINVAL, "NULL argument");
    if (buf_bytes < sizeof(SnapshotHeader)) return set_error(MMF_EINVAL, "snapshot shorter than its header");
    SnapshotHeader hd;
    memcpy(&hd, h_buf, sizeof(hd));
    if (hd.magic != MMF_SNAPSHOT_MAGIC || (hd.version != 1u && hd.version != 2u) || hd.zero != 0)
        return set_error(MMF_EINVAL, "not a stream snapshot");
    if (hd.dtype != (int32_t)S->dtype) return set_error(MMF_EINVAL, "snapshot of another dtype");
    if (hd.w < 1 || hd.count < 0 || hd.halo_len != std::min<int64_t>(hd.count, hd.w - 1))
        return set_error(MMF_EINVAL, "inconsistent snapshot header");
    // The stream's halo must fit the budget (as in mmf_stream_open); checked
    // before any host buffer is sized from the header.
    if ((uint64_t)(hd.w - 1) > S->stage.size() / (uint64_t)S->esz)
        return set_error(MMF_ENOMEM, "a window of %lld needs a halo larger than the device budget",
                         (long long)hd.w);
    const size_t body = buf_bytes - sizeof(hd);  // bytes after the header
    std::vector<char> rebuilt;
    const char *halo_bytes = static_cast<const char *>(h_buf) + sizeof(hd);
    if (hd.version == 2u) {
        // A wedge: rebuild an equivalent halo.
        if (body < 16) return set_error(MMF_EINVAL, "truncated snapshot");
        int64_t nu, nl;
        memcpy(&nu, halo_bytes, 8);
        memcpy(&nl, halo_bytes + 8, 8);
        const size_t rec = 8 + (size_t)S->esz;
        const uint64_t fits = (body - 16) / rec;  // whole records present in the buffer
        if (nu < 0 || nl < 0 || nu > hd.halo_len || nl > hd.halo_len || (hd.halo_len > 0 && (nu < 1 || nl < 1)) ||
            (uint64_t)nu > fits || (uint64_t)nl > fits - (uint64_t)nu)
            return set_error(MMF_EINVAL, "truncated or inconsistent wedge snapshot");
        for (int64_t j = 0; j < nu + nl; ++j) {
            int64_t back;
            memcpy(&back, halo_bytes + 16 + j * rec, 8);
            if (back < 1 || back > hd.halo_len) return set_error(MMF_EINVAL, "wedge entry outside the halo");
        }
        rebuilt.assign((size_t)hd.halo_len * S->esz, 0);
        if (hd.halo_len > 0) {
            switch (S->dtype) {
                case MMF_F32: halo_from_wedge<float>(halo_bytes + 16, nu, nl, hd.halo_len, rebuilt.data()); break;
                case MMF_F64: halo_from_wedge<double>(halo_bytes + 16, nu, nl, hd.halo_len, rebuilt.data()); break;
                case MMF_I16: halo_from_wedge<int16_t>(halo_bytes + 16, nu, nl, hd.halo_len, rebuilt.data()); break;
                default: halo_from_wedge<uint8_t>(halo_bytes + 16, nu, nl, hd.halo_len, rebuilt.data()); break;
            }
        }
        halo_bytes = rebuilt.data();
    } else if ((uint64_t)hd.halo_len > body / (uint64_t)S->esz) {
        return set_error(MMF_EINVAL, "truncated snapshot");
    }
    uint64_t id = 0;
    mmf_status st = mmf_stream_open(S, hd.w, &id);
    if (st != MMF_OK) return st;
    std::lock_guard<std::mutex> lk(S->mu);
    StreamState &ss = S->streams[id];
    if (hd.halo_len > 0) {
        cudaSetDevice(S->device);
        cudaError_t e = cudaMemcpy(S->dev_base + ss.halo_off, halo_bytes, (size_t)hd.halo_len * S->esz,
                                   cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (ss.halo_off >= 0) S->stage.release(ss.halo_off, (size_t)(ss.w - 1) * S->esz);
            S->streams.erase(id);
            return cuda_error(e, "restore copy");
        }
    }
    ss.count = hd.count;
    ss.halo_len = hd.halo_len;
    *stream_id = id;
    return MMF_OK;
}

mmf_status mmf_server_pause(mmf_server *S, int paused) {
    if (!S) return set_error(MMF_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    S->paused = paused != 0;
    S->cv_work.notify_all();
    return MMF_OK;
}

mmf_status mmf_server_stats(mmf_server *S, int reset, mmf_server_stats_t *out) {
    if (!S || !out) return set_error(MMF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto pct = [](std::vector<double> v, double p) {
        std::sort(v.begin(), v.end());
        return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))];
    };
    out->chunks = S->done_chunks;
    out->elements = S->done_elems;
    out->batches = (int64_t)S->nbatches;
    out->p50_ms = pct(S->lat_ms, 0.50);
    out->p99_ms = pct(S->lat_ms, 0.99);
    out->max_ms = pct(S->lat_ms, 1.0);
    out->queued = (int64_t)S->queue.size();
    out->device_bytes_used = (int64_t)(S->stage.used() + 2 * S->out.used());
    out->p50_queue_ms = pct(S->queue_ms, 0.50);
    out->p99_queue_ms = pct(S->queue_ms, 0.99);
    out->p50_service_ms = pct(S->service_ms, 0.50);
    out->p99_service_ms = pct(S->service_ms, 0.99);
    out->max_hold_ms = S->max_hold_ms;
    if (reset) {
        S->lat_ms.clear();
        S->queue_ms.clear();
        S->service_ms.clear();
        S->max_hold_ms = 0.0;
        S->done_chunks = S->done_elems = 0;
        S->nbatches = 0;
    }
    return MMF_OK;
}

}  // extern "C"
