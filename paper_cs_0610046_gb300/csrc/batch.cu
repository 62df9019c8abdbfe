// Batched running max-min filter: thousands of series of uneven length and
// window in one persistent launch per kernel mode, captured in a CUDA graph.
//
// A plan turns the host description of the series into a device table of
// series and work items.  An item is a contiguous range of output tiles of one
// series; long series are split into items of `seg_tiles` tiles so that every
// CTA's share is balanced (items are ordered longest first and pulled from an
// atomic ticket).  Items are grouped by the kernel mode their window needs
// (register slide, block scans with blocks inside a thread, across lanes, or
// one per warp); each group is one persistent launch.  The first call with a
// given set of buffers captures the ticket resets and the launches into a
// graph; later calls replay it.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "launch.h"
#include "mmf.h"

namespace mmf {
mmf_status set_error(mmf_status st, const char *fmt, ...);
mmf_status cuda_error(cudaError_t e, const char *what);
mmf_status get_ctx(void *stream, LaunchCtx *ctx);
int elem_size(mmf_dtype dt);
int tile_of(mmf_dtype dt);
mmf_status make_series(int64_t n, int64_t w_or_r, mmf_mode mode, mmf_dtype dt, SeriesDesc *sd);
}  // namespace mmf

using namespace mmf;

namespace {

constexpr int kModes = 4;  // 0, 1, 2 block scans; 3 register slide

struct Group {
    int mode = 0;
    int seg_tiles = 16;
    std::vector<ItemDesc> items;
    ItemDesc *d_items = nullptr;
};

// Kernel group of a series' window: the register slide for w <= slide_max
// (at most the slide's own limit), else the block-scan mode.
int kernel_mode(mmf_dtype dt, int64_t w, int slide_max) {
    const bool slide = w <= slide_max;
    switch (dt) {
        case MMF_F32: return block_mode<float>(w, slide);
        case MMF_F64: return block_mode<double>(w, slide);
        case MMF_I16: return block_mode<int16_t>(w, slide);
        default: return block_mode<uint8_t>(w, slide);
    }
}

// The register slide's own window limit for the type.
int slide_limit(mmf_dtype dt) { return dt == MMF_F32 ? 17 : 9; }

}  // namespace

struct mmf_batch_plan {
    int device = 0;
    mmf_dtype dtype = MMF_F32;
    mmf_mode mode = MMF_VALID;
    int64_t nseries = 0;
    int64_t in_len = 0;   // elements the input buffer must hold
    int64_t out_len = 0;  // elements each output buffer must hold
    int64_t common_len = -1;  // the length every series has (-1 if they differ)
    std::vector<SeriesDesc> series;
    std::vector<int64_t> out_off;  // nseries + 1
    Group groups[kModes];
    // Tuned knobs beside the segment lengths: series of at most short_cut
    // elements take the warp-per-series kernel (one warp per series instead
    // of block-scan items of a whole CTA; 0: none), and windows of at most
    // slide_max take the register slide (1: none).
    int64_t short_cut = 0;
    int slide_max = 1;
    std::vector<int64_t> short_ids;  // series taken by the warp-per-series kernel
    int64_t *d_short = nullptr;
    cudaStream_t short_branch = nullptr;
    cudaEvent_t short_join = nullptr;
    SeriesDesc *d_series = nullptr;
    int *d_tickets = nullptr;  // one per group
    cudaStream_t cap_stream = nullptr;
    cudaStream_t branch[kModes] = {};   // capture branches: groups run concurrently
    cudaEvent_t fork = nullptr, join[kModes] = {};
    cudaGraphExec_t exec = nullptr;
    const void *g_in = nullptr;
    void *g_max = nullptr, *g_min = nullptr;
    int g_launches = 0;
};

namespace {

bool is_short(const mmf_batch_plan *p, const SeriesDesc &sd) {
    return sd.n_out > 0 && sd.n <= p->short_cut;
}

void free_items(mmf_batch_plan *p) {
    for (auto &g : p->groups) {
        if (g.d_items) cudaFree(g.d_items);
        g.d_items = nullptr;
    }
    if (p->exec) cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
}

// Split the series of one group into items of at most seg_tiles output tiles
// and upload them, longest first.
mmf_status build_items(mmf_batch_plan *p, int gi) {
    Group &g = p->groups[gi];
    g.items.clear();
    const int64_t T = tile_of(p->dtype);
    const int64_t seg = (int64_t)std::max(1, g.seg_tiles) * T;
    for (int64_t s = 0; s < p->nseries; ++s) {
        const SeriesDesc &sd = p->series[s];
        if (sd.n_out <= 0 || is_short(p, sd) || kernel_mode(p->dtype, sd.w, p->slide_max) != g.mode) continue;
        for (int64_t ob = 0; ob < sd.n_out; ob += seg) g.items.push_back({s, ob, std::min(sd.n_out, ob + seg)});
    }
    std::stable_sort(g.items.begin(), g.items.end(), [&](const ItemDesc &a, const ItemDesc &b) {
        const int64_t ca = a.o_end - a.o_begin + p->series[a.series].w;
        const int64_t cb = b.o_end - b.o_begin + p->series[b.series].w;
        return ca > cb;
    });
    if (g.d_items) cudaFree(g.d_items);
    g.d_items = nullptr;
    if (g.items.empty()) return MMF_OK;
    cudaError_t e = cudaMalloc(&g.d_items, g.items.size() * sizeof(ItemDesc));
    if (e != cudaSuccess) return set_error(MMF_ENOMEM, "plan items: %s", cudaGetErrorString(e));
    e = cudaMemcpy(g.d_items, g.items.data(), g.items.size() * sizeof(ItemDesc), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "upload items");
    return MMF_OK;
}

// The short-series list and every group's items for the current knobs.
mmf_status rebuild_all(mmf_batch_plan *p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
    p->short_ids.clear();
    for (int64_t s = 0; s < p->nseries; ++s)
        if (is_short(p, p->series[s])) p->short_ids.push_back(s);
    if (p->d_short) cudaFree(p->d_short);
    p->d_short = nullptr;
    if (!p->short_ids.empty()) {
        cudaError_t e = cudaMalloc(&p->d_short, p->short_ids.size() * sizeof(int64_t));
        if (e != cudaSuccess) return set_error(MMF_ENOMEM, "plan short-series list: %s", cudaGetErrorString(e));
        e = cudaMemcpy(p->d_short, p->short_ids.data(), p->short_ids.size() * sizeof(int64_t),
                       cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_error(e, "upload short-series list");
    }
    for (int gi = 0; gi < kModes; ++gi) {
        mmf_status st = build_items(p, gi);
        if (st != MMF_OK) return st;
    }
    return MMF_OK;
}

mmf_status launch_group(mmf_batch_plan *p, int gi, const LaunchCtx &ctx, const void *in, void *omax, void *omin,
                        bool ticket, const void *lb_query = nullptr, double *lb_acc = nullptr) {
    Group &g = p->groups[gi];
    if (g.items.empty()) return MMF_OK;
    int *tk = ticket ? p->d_tickets + gi : nullptr;
    cudaError_t e = cudaSuccess;
    const int64_t ni = (int64_t)g.items.size();
    switch (p->dtype) {
        case MMF_F32: e = blockscan_table<float>(ctx, g.mode, in, p->in_len, omax, omin, p->d_series, g.d_items, ni, tk, 0, lb_query, lb_acc); break;
        case MMF_F64: e = blockscan_table<double>(ctx, g.mode, in, p->in_len, omax, omin, p->d_series, g.d_items, ni, tk, 0, lb_query, lb_acc); break;
        case MMF_I16: e = blockscan_table<int16_t>(ctx, g.mode, in, p->in_len, omax, omin, p->d_series, g.d_items, ni, tk, 0, lb_query, lb_acc); break;
        case MMF_U8: e = blockscan_table<uint8_t>(ctx, g.mode, in, p->in_len, omax, omin, p->d_series, g.d_items, ni, tk, 0, lb_query, lb_acc); break;
    }
    return e == cudaSuccess ? MMF_OK : cuda_error(e, "batched launch");
}

// Ticket resets on `st`, then one persistent launch per non-empty group, each
// on its own branch stream (fork/join by events) so that a group's tail
// overlaps the next group's work.
mmf_status enqueue_all(mmf_batch_plan *p, cudaStream_t st, const void *in, void *omax, void *omin,
                       const void *lb_query = nullptr, double *lb_acc = nullptr) {
    LaunchCtx ctx;
    mmf_status s = get_ctx(st, &ctx);
    if (s != MMF_OK) return s;
    cudaError_t e = cudaMemsetAsync(p->d_tickets, 0, kModes * sizeof(int), st);
    if (e != cudaSuccess) return cuda_error(e, "reset tickets");
    e = cudaEventRecord(p->fork, st);
    if (e != cudaSuccess) return cuda_error(e, "fork");
    for (int gi = 0; gi < kModes; ++gi) {
        if (p->groups[gi].items.empty()) continue;
        e = cudaStreamWaitEvent(p->branch[gi], p->fork, 0);
        if (e != cudaSuccess) return cuda_error(e, "branch wait");
        LaunchCtx bctx = ctx;
        bctx.stream = p->branch[gi];
        s = launch_group(p, gi, bctx, in, omax, omin, true, lb_query, lb_acc);
        if (s != MMF_OK) return s;
        e = cudaEventRecord(p->join[gi], p->branch[gi]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->join[gi], 0);
        if (e != cudaSuccess) return cuda_error(e, "join");
    }
    if (!p->short_ids.empty()) {
        e = cudaStreamWaitEvent(p->short_branch, p->fork, 0);
        if (e != cudaSuccess) return cuda_error(e, "branch wait");
        LaunchCtx bctx = ctx;
        bctx.stream = p->short_branch;
        const int64_t cnt = (int64_t)p->short_ids.size();
        switch (p->dtype) {
            case MMF_F32: e = short_table<float>(bctx, in, p->in_len, omax, omin, p->d_series, p->d_short, cnt, lb_query, lb_acc, p->common_len); break;
            case MMF_F64: e = short_table<double>(bctx, in, p->in_len, omax, omin, p->d_series, p->d_short, cnt, lb_query, lb_acc, p->common_len); break;
            case MMF_I16: e = short_table<int16_t>(bctx, in, p->in_len, omax, omin, p->d_series, p->d_short, cnt, lb_query, lb_acc, p->common_len); break;
            case MMF_U8: e = short_table<uint8_t>(bctx, in, p->in_len, omax, omin, p->d_series, p->d_short, cnt, lb_query, lb_acc, p->common_len); break;
        }
        if (e != cudaSuccess) return cuda_error(e, "short-series launch");
        e = cudaEventRecord(p->short_join, p->short_branch);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->short_join, 0);
        if (e != cudaSuccess) return cuda_error(e, "join");
    }
    return MMF_OK;
}

mmf_status capture(mmf_batch_plan *p, const void *in, void *omax, void *omin) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
    for (int gi = 0; gi < kModes; ++gi) {
        if (p->groups[gi].items.empty()) continue;
        cudaError_t pe = cudaSuccess;
        switch (p->dtype) {
            case MMF_F32: pe = blockscan_prepare<float>(p->device, gi); break;
            case MMF_F64: pe = blockscan_prepare<double>(p->device, gi); break;
            case MMF_I16: pe = blockscan_prepare<int16_t>(p->device, gi); break;
            case MMF_U8: pe = blockscan_prepare<uint8_t>(p->device, gi); break;
        }
        if (pe != cudaSuccess) return cuda_error(pe, "prepare kernels");
    }
    if (!p->short_ids.empty()) {
        int k = 0;
        cudaError_t pe = cudaSuccess;
        switch (p->dtype) {
            case MMF_F32: pe = short_prepare<float>(p->device, false, &k); break;
            case MMF_F64: pe = short_prepare<double>(p->device, false, &k); break;
            case MMF_I16: pe = short_prepare<int16_t>(p->device, false, &k); break;
            case MMF_U8: pe = short_prepare<uint8_t>(p->device, false, &k); break;
        }
        if (pe != cudaSuccess) return cuda_error(pe, "prepare kernels");
    }
    LaunchCtx warm;
    mmf_status ws = get_ctx(nullptr, &warm);  // device cache filled outside the capture
    if (ws != MMF_OK) return ws;
    cudaError_t e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_error(e, "begin capture");
    mmf_status s = enqueue_all(p, p->cap_stream, in, omax, omin);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(p->cap_stream, &graph);
    if (s != MMF_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return cuda_error(e, "end capture");
    e = cudaGraphInstantiate(&p->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_error(e, "instantiate graph");
    p->g_in = in;
    p->g_max = omax;
    p->g_min = omin;
    return MMF_OK;
}

// Envelope lower bound: accumulators cleared before the launches, square
// roots taken after them.
// (Their index is the loop's, below n: nothing to range-check.)
__global__ void lb_clear_kernel(double *acc, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc[i] = 0.0;
}
__global__ void lb_sqrt_kernel(double *acc, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc[i] = sqrt(acc[i]);
}

// Autotune cache: one line "key value" per entry in $MMF_AUTOTUNE_CACHE (the
// last entry of a key wins).  Keys name the GPU, dtype, mode and the shape.
std::string cache_key_plan(const mmf_batch_plan *p, const char *knob) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, p->device);
    int64_t total = 0;
    for (auto &sd : p->series) total += sd.n;
    int lt = 0;
    while ((1ll << (lt + 1)) <= std::max<int64_t>(1, total)) ++lt;
    char buf[256];
    snprintf(buf, sizeof(buf), "%s|dt%d|m%d|%s|elems2^%d|series%lld", prop.name, (int)p->dtype, (int)p->mode, knob,
             lt, (long long)p->nseries);
    std::string k(buf);
    for (auto &c : k)
        if (c == ' ') c = '_';
    return k;
}

std::string cache_key(const mmf_batch_plan *p, int gi) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, p->device);
    int64_t tiles = 0, wsum = 0;
    for (auto &it : p->groups[gi].items) {
        tiles += (it.o_end - it.o_begin + tile_of(p->dtype) - 1) / tile_of(p->dtype);
        wsum += p->series[it.series].w;
    }
    char buf[256];
    int lt = 0;
    while ((1ll << (lt + 1)) <= std::max<int64_t>(1, tiles)) ++lt;
    snprintf(buf, sizeof(buf), "%s|dt%d|m%d|g%d|tiles2^%d|series%lld", prop.name, (int)p->dtype, (int)p->mode,
             p->groups[gi].mode, lt, (long long)p->nseries);
    std::string k(buf);
    for (auto &c : k)
        if (c == ' ') c = '_';
    return k;
}

int cache_lookup(const std::string &key) {
    const char *path = getenv("MMF_AUTOTUNE_CACHE");
    if (!path) return 0;
    FILE *f = fopen(path, "r");
    if (!f) return 0;
    char k[512];
    int v = 0, found = 0;
    while (fscanf(f, "%511s %d", k, &v) == 2)
        if (key == k) found = v;
    fclose(f);
    return found;
}

void cache_store(const std::string &key, int v) {
    const char *path = getenv("MMF_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d\n", key.c_str(), v);
    fclose(f);
}

}  // namespace

extern "C" {

mmf_status mmf_batch_plan_create(const int64_t *h_in_off, const int64_t *h_len, const int64_t *h_w, int64_t nseries,
                                 mmf_dtype dtype, mmf_mode mode, mmf_batch_plan **out) {
    NvtxRange nvtx_range("mmf_batch_plan_create");
    if (!out) return set_error(MMF_EINVAL, "NULL plan output");
    *out = nullptr;
    if (nseries < 0 || (nseries > 0 && (!h_len || !h_w))) return set_error(MMF_EINVAL, "bad series description");
    if (elem_size(dtype) == 0) return set_error(MMF_EINVAL, "unknown dtype %d", (int)dtype);
    mmf_batch_plan *p = new (std::nothrow) mmf_batch_plan();
    if (!p) return set_error(MMF_ENOMEM, "plan");
    cudaGetDevice(&p->device);
    p->dtype = dtype;
    p->mode = mode;
    p->nseries = nseries;
    p->series.resize(nseries);
    p->out_off.assign(nseries + 1, 0);
    int64_t in_pos = 0, out_pos = 0;
    const int esz = elem_size(dtype);
    for (int64_t s = 0; s < nseries; ++s) {
        SeriesDesc sd;
        mmf_status st = make_series(h_len[s], h_w[s], mode, dtype, &sd);
        if (st != MMF_OK) {
            delete p;
            return st;
        }
        sd.in_off = h_in_off ? h_in_off[s] : in_pos;
        if (sd.in_off < 0) {
            delete p;
            return set_error(MMF_EINVAL, "negative input offset for series %lld", (long long)s);
        }
        in_pos = sd.in_off + sd.n;
        p->in_len = std::max(p->in_len, sd.in_off + sd.n);
        sd.out_off = batch_out_start(out_pos, esz);
        p->out_off[s] = sd.out_off;
        out_pos = sd.out_off + sd.n_out;
        p->series[s] = sd;
    }
    p->out_off[nseries] = out_pos;
    p->out_len = out_pos;
    p->common_len = nseries > 0 ? p->series[0].n : 0;
    for (int64_t s = 1; s < nseries; ++s)
        if (p->series[s].n != p->common_len) p->common_len = -1;
    for (int gi = 0; gi < kModes; ++gi) {
        p->groups[gi].mode = gi;
        p->groups[gi].seg_tiles = gi == 2 ? 32 : 16;
    }
    cudaError_t e = cudaMalloc(&p->d_tickets, kModes * sizeof(int));
    if (e == cudaSuccess && nseries > 0) e = cudaMalloc(&p->d_series, nseries * sizeof(SeriesDesc));
    if (e == cudaSuccess && nseries > 0)
        e = cudaMemcpy(p->d_series, p->series.data(), nseries * sizeof(SeriesDesc), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
    for (int gi = 0; gi < kModes && e == cudaSuccess; ++gi) {
        e = cudaStreamCreateWithFlags(&p->branch[gi], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->join[gi], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->short_branch, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->short_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        mmf_batch_plan_destroy(p);
        return set_error(MMF_ENOMEM, "plan device tables: %s", cudaGetErrorString(e));
    }
    // Knobs: the built-in choice, or a tuned one cached for this shape.
    p->short_cut = short_max_len(esz);
    p->slide_max = slide_limit(dtype);
    {
        const int cs = cache_lookup(cache_key_plan(p, "short"));
        const int cl = cache_lookup(cache_key_plan(p, "slide"));
        if (cs > 0) p->short_cut = std::min<int64_t>(cs - 1, short_max_len(esz));  // stored + 1 (0 = none)
        if (cl > 0) p->slide_max = std::min(cl, slide_limit(dtype));
    }
    mmf_status rs = rebuild_all(p);
    if (rs != MMF_OK) {
        mmf_batch_plan_destroy(p);
        return rs;
    }
    for (int gi = 0; gi < kModes; ++gi) {
        mmf_status st = MMF_OK;
        const int cached = cache_lookup(cache_key(p, gi));
        if (cached > 0 && cached != p->groups[gi].seg_tiles) {
            p->groups[gi].seg_tiles = cached;
            st = build_items(p, gi);
            if (st != MMF_OK) {
                mmf_batch_plan_destroy(p);
                return st;
            }
        }
    }
    *out = p;
    return MMF_OK;
}

void mmf_batch_plan_destroy(mmf_batch_plan *p) {
    if (!p) return;
    free_items(p);
    if (p->d_series) cudaFree(p->d_series);
    if (p->d_tickets) cudaFree(p->d_tickets);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    for (int gi = 0; gi < kModes; ++gi) {
        if (p->branch[gi]) cudaStreamDestroy(p->branch[gi]);
        if (p->join[gi]) cudaEventDestroy(p->join[gi]);
    }
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->d_short) cudaFree(p->d_short);
    if (p->short_branch) cudaStreamDestroy(p->short_branch);
    if (p->short_join) cudaEventDestroy(p->short_join);
    delete p;
}

mmf_status mmf_batch_plan_out_offsets(const mmf_batch_plan *p, int64_t *h_off) {
    if (!p || !h_off) return set_error(MMF_EINVAL, "NULL argument");
    memcpy(h_off, p->out_off.data(), (p->nseries + 1) * sizeof(int64_t));
    return MMF_OK;
}

mmf_status mmf_batch_plan_sizes(const mmf_batch_plan *p, int64_t *in_len, int64_t *out_len, int64_t *n_items) {
    if (!p) return set_error(MMF_EINVAL, "NULL plan");
    if (in_len) *in_len = p->in_len;
    if (out_len) *out_len = p->out_len;
    if (n_items)
        for (int gi = 0; gi < kModes; ++gi) n_items[gi] = (int64_t)p->groups[gi].items.size();
    return MMF_OK;
}

mmf_status mmf_batch_plan_set_segment(mmf_batch_plan *p, int group, int seg_tiles) {
    if (!p || group < 0 || group >= kModes || seg_tiles < 1) return set_error(MMF_EINVAL, "bad segment request");
    p->groups[group].seg_tiles = seg_tiles;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
    return build_items(p, group);
}

mmf_status mmf_filter1d_batched(mmf_batch_plan *p, const void *d_in, void *d_max, void *d_min, void *stream) {
    NvtxRange nvtx_range("mmf_filter1d_batched");
    if (!p) return set_error(MMF_EINVAL, "NULL plan");
    if (p->out_len == 0) return MMF_OK;
    if (!d_in || (!d_max && !d_min)) return set_error(MMF_EINVAL, "NULL buffers");
    const int esz = elem_size(p->dtype);
    if (((uintptr_t)d_in % esz) || ((uintptr_t)d_max % esz) || ((uintptr_t)d_min % esz))
        return set_error(MMF_EINVAL, "pointers must be aligned to the element size");
    if (!p->exec || p->g_in != d_in || p->g_max != d_max || p->g_min != d_min) {
        mmf_status s = capture(p, d_in, d_max, d_min);
        if (s != MMF_OK) return s;
    }
    cudaError_t e = cudaGraphLaunch(p->exec, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MMF_OK : cuda_error(e, "graph launch");
}

mmf_status mmf_lb_keogh_batched(mmf_batch_plan *p, const void *d_in, const void *d_query, int64_t n_query,
                                double *d_lb, void *stream) {
    NvtxRange nvtx_range("mmf_lb_keogh_batched");
    if (!p) return set_error(MMF_EINVAL, "NULL plan");
    if (p->mode != MMF_CENTERED_CLIPPED) return set_error(MMF_EINVAL, "the lower bound needs an envelope plan");
    if (p->nseries == 0) return MMF_OK;
    if (p->common_len < 0 || p->common_len != n_query)
        return set_error(MMF_EINVAL, "every series must be as long as the query (%lld)", (long long)n_query);
    const int esz = elem_size(p->dtype);
    if (!d_lb || (n_query > 0 && (!d_in || !d_query))) return set_error(MMF_EINVAL, "NULL buffers");
    if (((uintptr_t)d_in % esz) || ((uintptr_t)d_query % esz) || ((uintptr_t)d_lb % 8))
        return set_error(MMF_EINVAL, "misaligned pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LaunchCtx ctx;
    mmf_status s = get_ctx(stream, &ctx);
    if (s != MMF_OK) return s;
    const int nb = (int)std::min<int64_t>((p->nseries + 255) / 256, 4 * std::max(1, ctx.sms));
    lb_clear_kernel<<<nb, 256, 0, st>>>(d_lb, p->nseries);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "clear bounds");
    // The lower-bound launches set their kernels' attributes themselves (no
    // graph is captured here).
    s = enqueue_all(p, st, d_in, nullptr, nullptr, d_query, d_lb);
    if (s != MMF_OK) return s;
    lb_sqrt_kernel<<<nb, 256, 0, st>>>(d_lb, p->nseries);
    e = cudaGetLastError();
    return e == cudaSuccess ? MMF_OK : cuda_error(e, "square roots");
}

mmf_status mmf_filter1d_per_series(const mmf_batch_plan *p, const void *d_in, void *d_max, void *d_min,
                                   void *stream) {
    NvtxRange nvtx_range("mmf_filter1d_per_series");
    if (!p) return set_error(MMF_EINVAL, "NULL plan");
    const int esz = elem_size(p->dtype);
    for (int64_t s = 0; s < p->nseries; ++s) {
        const SeriesDesc &sd = p->series[s];
        if (sd.n_out <= 0) continue;
        const int64_t w_or_r = p->mode == MMF_VALID ? sd.w : (sd.w - 1) / 2;
        mmf_status st = mmf_filter1d(static_cast<const char *>(d_in) + sd.in_off * esz, sd.n, w_or_r, p->dtype,
                                     p->mode, d_max ? static_cast<char *>(d_max) + sd.out_off * esz : nullptr,
                                     d_min ? static_cast<char *>(d_min) + sd.out_off * esz : nullptr, stream);
        if (st != MMF_OK) return st;
    }
    return MMF_OK;
}

// Event time of the whole plan (every group and the short series, no graph)
// on `st`: median of three runs after one warm-up run; < 0 on failure.
static float time_plan(mmf_batch_plan *p, cudaStream_t st, const void *d_in, void *d_max, void *d_min,
                       cudaEvent_t e0, cudaEvent_t e1) {
    float t[3];
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, st);
        if (enqueue_all(p, st, d_in, d_max, d_min) != MMF_OK) return -1.f;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) t[rep - 1] = ms;  // the first run warms up
    }
    std::sort(t, t + 3);
    return t[1];
}

mmf_status mmf_batch_plan_autotune(mmf_batch_plan *p, const void *d_in, void *d_max, void *d_min, void *stream) {
    NvtxRange nvtx_range("mmf_batch_plan_autotune");
    if (!p) return set_error(MMF_EINVAL, "NULL plan");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LaunchCtx ctx;
    mmf_status s = get_ctx(stream, &ctx);
    if (s != MMF_OK) return s;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // 1. Threads per short series: one warp per series for series of at most
    //    short_cut elements, else block-scan items of a whole CTA.
    // 2. Kernel choice for small windows: the register slide up to slide_max,
    //    else the block scans.
    // 3. Segment length (output tiles per work item) per block-scan group.
    // Each knob is timed over the whole plan with the others fixed.
    const int64_t smax = short_max_len(elem_size(p->dtype));
    const int64_t short_cands[] = {0, smax / 4, smax / 2, smax};
    const int lmax = slide_limit(p->dtype);
    const int slide_cands[] = {1, 5, 9, 17};
    for (int knob = 0; knob < 2 && s == MMF_OK; ++knob) {
        const int64_t keep_short = p->short_cut;
        const int keep_slide = p->slide_max;
        int64_t best_short = keep_short;
        int best_slide = keep_slide;
        float best_ms = 1e30f;
        for (int c = 0; c < 4; ++c) {
            if (knob == 0) {
                p->short_cut = short_cands[c];
            } else {
                if (slide_cands[c] > lmax) continue;
                p->slide_max = slide_cands[c];
            }
            s = rebuild_all(p);
            if (s != MMF_OK) break;
            const float ms = time_plan(p, st, d_in, d_max, d_min, e0, e1);
            if (ms < 0.f) {
                s = set_error(MMF_ECUDA, "autotune run failed");
                break;
            }
            if (ms < best_ms) {
                best_ms = ms;
                best_short = p->short_cut;
                best_slide = p->slide_max;
            }
        }
        p->short_cut = knob == 0 ? best_short : keep_short;
        p->slide_max = knob == 1 ? best_slide : keep_slide;
        mmf_status s2 = rebuild_all(p);
        if (s == MMF_OK) s = s2;
    }
    if (s == MMF_OK) {
        cache_store(cache_key_plan(p, "short"), (int)p->short_cut + 1);
        cache_store(cache_key_plan(p, "slide"), p->slide_max);
    }
    const int cands[] = {1, 2, 4, 8, 16, 32, 64, 128};
    for (int gi = 0; gi < kModes && s == MMF_OK; ++gi) {
        if (p->groups[gi].items.empty()) continue;
        int best = p->groups[gi].seg_tiles;
        float best_ms = 1e30f;
        for (int c : cands) {
            p->groups[gi].seg_tiles = c;
            s = build_items(p, gi);
            if (s != MMF_OK) break;
            float ms = 0.f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaMemsetAsync(p->d_tickets + gi, 0, sizeof(int), st);
                cudaEventRecord(e0, st);
                s = launch_group(p, gi, ctx, d_in, d_max, d_min, true);
                cudaEventRecord(e1, st);
                if (s != MMF_OK) break;
                cudaEventSynchronize(e1);
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0) ms += t;  // first run warms up
            }
            if (s != MMF_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        p->groups[gi].seg_tiles = best;
        mmf_status s2 = build_items(p, gi);
        if (s == MMF_OK) s = s2;
        if (s != MMF_OK) break;
        cache_store(cache_key(p, gi), best);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
    return s;
}

mmf_status mmf_batch_plan_set_knobs(mmf_batch_plan *p, int64_t short_cut, int slide_max) {
    if (!p) return set_error(MMF_EINVAL, "NULL plan");
    const int64_t smax = short_max_len(elem_size(p->dtype));
    if (short_cut < 0 || short_cut > smax)
        return set_error(MMF_EINVAL, "short-series cut-off %lld outside [0, %lld]", (long long)short_cut,
                         (long long)smax);
    if (slide_max < 1 || slide_max > slide_limit(p->dtype))
        return set_error(MMF_EINVAL, "slide window limit %d outside [1, %d]", slide_max, slide_limit(p->dtype));
    p->short_cut = short_cut;
    p->slide_max = slide_max;
    return rebuild_all(p);
}

mmf_status mmf_batch_plan_get_knobs(const mmf_batch_plan *p, int64_t *short_cut, int *slide_max) {
    if (!p || !short_cut || !slide_max) return set_error(MMF_EINVAL, "NULL argument");
    *short_cut = p->short_cut;
    *slide_max = p->slide_max;
    return MMF_OK;
}

mmf_status mmf_batch_plan_get_segment(const mmf_batch_plan *p, int group, int *seg_tiles) {
    if (!p || !seg_tiles || group < 0 || group >= kModes) return set_error(MMF_EINVAL, "bad arguments");
    *seg_tiles = p->groups[group].seg_tiles;
    return MMF_OK;
}

}  // extern "C"
