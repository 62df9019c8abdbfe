// Batched filter for callers that must not allocate.
//
// Some callers cannot call cudaMalloc: code that runs while other work holds a
// fixed device-memory budget (a serving process that reserved its pool up
// front), real-time or signal-driven paths where an allocation could block or
// fail, and host callbacks where allocation APIs are not allowed.  This entry
// point runs the batched kernel with its work tables (series, work items and
// ticket counters) in a file-scope device array of fixed size instead of
// plan-owned allocations.  The caller still passes the input and output
// buffers.  Each device that loads the library holds this array until the
// process exits.
//
// The array is shared by every call: a call overwrites the tables left by the
// previous one and clears the ticket counters itself.  Calls whose kernels
// overlap on the GPU (from two host threads, or on two streams without
// ordering between them) race on the tables and give wrong results; order
// them on one stream.
#include <cstdint>
#include <cstring>
#include <mutex>

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

constexpr int kGroups = 4;
constexpr int64_t kMaxItems = MMF_NOALLOC_MAX_ITEMS;

struct NoAllocTables {
    int tickets[kGroups];
    int pad[64 - kGroups];
    SeriesDesc series[MMF_NOALLOC_MAX_SERIES];
    ItemDesc items[kMaxItems];
};

// The work tables.  In host code this name is a stand-in, not a device
// address: its address is taken with cudaGetSymbolAddress per device.
static __device__ __align__(256) NoAllocTables g_noalloc;

struct DevAddr {
    bool ready = false;
    NoAllocTables *ptr = nullptr;
};
static DevAddr g_noalloc_addr[64];
static std::mutex g_noalloc_mu;  // guards the per-device set-up above

int mode_of(mmf_dtype dt, int64_t w) {
    switch (dt) {
        case MMF_F32: return block_mode<float>(w, true);
        case MMF_F64: return block_mode<double>(w, true);
        case MMF_I16: return block_mode<int16_t>(w, true);
        default: return block_mode<uint8_t>(w, true);
    }
}

}  // namespace

extern "C" mmf_status mmf_filter1d_batched_noalloc(const void *d_in, const int64_t *h_len, const int64_t *h_w,
                                                   int64_t nseries, mmf_dtype dtype, mmf_mode mode, void *d_max,
                                                   void *d_min, void *stream) {
    if (nseries < 0 || (nseries > 0 && (!h_len || !h_w))) return set_error(MMF_EINVAL, "bad series description");
    if (nseries > MMF_NOALLOC_MAX_SERIES)
        return set_error(MMF_EINVAL, "%lld series exceed the no-allocation limit of %d", (long long)nseries,
                         MMF_NOALLOC_MAX_SERIES);
    const int esz = elem_size(dtype);
    if (esz == 0) return set_error(MMF_EINVAL, "unknown dtype %d", (int)dtype);

    // Series table (inputs packed in order; outputs in order, each series
    // starting on a 32-byte boundary as in a batch plan) and output length.
    SeriesDesc series[MMF_NOALLOC_MAX_SERIES];
    int64_t in_pos = 0, out_pos = 0, tiles = 0;
    const int64_t T = tile_of(dtype);
    for (int64_t s = 0; s < nseries; ++s) {
        SeriesDesc sd;
        mmf_status st = make_series(h_len[s], h_w[s], mode, dtype, &sd);
        if (st != MMF_OK) return st;
        sd.in_off = in_pos;
        sd.out_off = batch_out_start(out_pos, esz);
        in_pos += sd.n;
        out_pos = sd.out_off + sd.n_out;
        tiles += (sd.n_out + T - 1) / T;
        series[s] = sd;
    }
    if (out_pos == 0) return MMF_OK;
    if (!d_in || (!d_max && !d_min)) return set_error(MMF_EINVAL, "NULL buffers");
    if (((uintptr_t)d_in % esz) || ((uintptr_t)d_max % esz) || ((uintptr_t)d_min % esz))
        return set_error(MMF_EINVAL, "pointers must be aligned to the element size");

    // Work items: series split into runs of seg tiles, grouped by kernel mode.
    // seg grows with the total so that the items always fit the table.
    int64_t seg = 16;
    while (tiles / seg + nseries > kMaxItems) seg *= 2;
    ItemDesc items[kMaxItems];
    int64_t group_begin[kGroups + 1];
    int64_t ni = 0;
    for (int g = 0; g < kGroups; ++g) {
        group_begin[g] = ni;
        for (int64_t s = 0; s < nseries; ++s) {
            const SeriesDesc &sd = series[s];
            if (sd.n_out <= 0 || mode_of(dtype, sd.w) != g) continue;
            for (int64_t ob = 0; ob < sd.n_out; ob += seg * T) {
                if (ni >= kMaxItems) return set_error(MMF_EINVAL, "work items exceed the no-allocation limit");
                items[ni++] = {s, ob, ob + seg * T < sd.n_out ? ob + seg * T : sd.n_out};
            }
        }
    }
    group_begin[kGroups] = ni;

    LaunchCtx ctx;
    mmf_status st = get_ctx(stream, &ctx);
    if (st != MMF_OK) return st;
    // Set-up once per device, with that device current: the device address of
    // the table array.  (The first call on a device does this; make it before
    // any stream capture.)  It is done under a lock, so that a thread which
    // finds the set-up done also sees the address (on a weakly ordered CPU a
    // thread could otherwise see the flag before the pointer).
    NoAllocTables *tab = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        DevAddr &da = g_noalloc_addr[ctx.device];
        if (!da.ready) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc);
            if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-allocation tables)");
            da.ptr = static_cast<NoAllocTables *>(p);
            da.ready = true;
        }
        tab = da.ptr;
    }
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(tab->series, series, nseries * sizeof(SeriesDesc), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tab->items, items, ni * sizeof(ItemDesc), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(tab->tickets, 0, sizeof(tab->tickets), cs);
    if (e != cudaSuccess) return cuda_error(e, "upload no-allocation tables");
    for (int g = 0; g < kGroups; ++g) {
        const int64_t n_items = group_begin[g + 1] - group_begin[g];
        if (n_items == 0) continue;
        const ItemDesc *d_items = tab->items + group_begin[g];
        int *tk = tab->tickets + g;
        switch (dtype) {
            case MMF_F32: e = blockscan_table<float>(ctx, g, d_in, in_pos, d_max, d_min, tab->series, d_items, n_items, tk, 0); break;
            case MMF_F64: e = blockscan_table<double>(ctx, g, d_in, in_pos, d_max, d_min, tab->series, d_items, n_items, tk, 0); break;
            case MMF_I16: e = blockscan_table<int16_t>(ctx, g, d_in, in_pos, d_max, d_min, tab->series, d_items, n_items, tk, 0); break;
            case MMF_U8: e = blockscan_table<uint8_t>(ctx, g, d_in, in_pos, d_max, d_min, tab->series, d_items, n_items, tk, 0); break;
        }
        if (e != cudaSuccess) return cuda_error(e, "no-allocation batched launch");
    }
    return MMF_OK;
}
