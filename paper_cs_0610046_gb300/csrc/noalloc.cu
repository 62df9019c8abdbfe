// Batched filter for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: a process that reserved its whole
// device-memory budget up front (a fixed pool shared by its components), or a
// latency-bound path on an ordinary host thread where an allocation could
// block on the driver or fail under memory pressure.  This entry point runs
// the batched kernel with its work tables (series, work items and ticket
// counters) in a file-scope device array of fixed size instead of
// plan-owned allocations.  The caller still passes the input and output
// buffers.  Each device that loads the library holds this array until the
// process exits.
//
// The tables are built on the host in a static staging image and reach the
// device as the arguments of small copy kernels (at most about 30 KB each),
// so no host memory is read by the GPU after the call returns and no large
// array lives on the caller's stack.
//
// The array is shared by every call: a call overwrites the tables left by the
// previous one and clears the ticket counters itself.  Calls whose kernels
// overlap on the GPU (from two host threads, or on two streams without
// ordering between them) race on the tables and give wrong results; order
// them on one stream.
#include <cstddef>
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
constexpr int kMaxDevices = 64;  // the same bound as the library's device cache (get_ctx)

struct NoAllocTables {
    int tickets[kGroups];
    int pad[64 - kGroups];
    SeriesDesc series[MMF_NOALLOC_MAX_SERIES];
    ItemDesc items[kMaxItems];
};
static_assert(offsetof(NoAllocTables, series) == 256, "tables start after the counters");

// The work tables.  In host code this name is a stand-in, not a device
// address: its address is taken with cudaGetSymbolAddress per device.
static __device__ __align__(256) NoAllocTables g_noalloc;

struct DevAddr {
    bool ready = false;
    NoAllocTables *ptr = nullptr;
};
static DevAddr g_noalloc_addr[kMaxDevices];

// Host staging: the image of the tables a call uploads, and the argument
// block of one copy kernel.  Both are static (no stack arrays, no heap) and
// guarded by g_noalloc_mu for the whole call.
constexpr uint32_t kChunk = 30 * 1024;  // payload bytes per copy kernel (kernel arguments <= 32764 bytes)
struct alignas(16) TableChunk {
    uint32_t off;    // byte offset in the device tables (a multiple of 8)
    uint32_t bytes;  // payload bytes, a multiple of 8
    uint32_t pad[2];
    uint8_t data[kChunk];
};
static_assert(sizeof(TableChunk) <= 32764, "one copy kernel's arguments");
static NoAllocTables g_img;
static TableChunk g_chunk;
static std::mutex g_noalloc_mu;

// Copies one chunk of table bytes from the kernel's arguments into the device
// tables (one CTA; the arguments are read in place).
__global__ void noalloc_upload_kernel(const __grid_constant__ TableChunk c, uint8_t *tables, uint32_t *status) {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(c.data);
    uint32_t *dst = reinterpret_cast<uint32_t *>(tables + c.off);
    for (uint32_t i = threadIdx.x; i < c.bytes / 4; i += blockDim.x)
        if (in_bytes(status, dst + i, 4, tables, (int64_t)sizeof(NoAllocTables))) dst[i] = src[i];
}

// Uploads bytes [off, off + bytes) of the staging image on stream cs.
cudaError_t upload(uint8_t *d_tables, uint32_t off, uint32_t bytes, cudaStream_t cs, uint32_t *status) {
    const uint8_t *img = reinterpret_cast<const uint8_t *>(&g_img);
    for (uint32_t done = 0; done < bytes; done += kChunk) {
        const uint32_t b = bytes - done < kChunk ? bytes - done : kChunk;
        g_chunk.off = off + done;
        g_chunk.bytes = (b + 7) & ~7u;
        std::memcpy(g_chunk.data, img + off + done, g_chunk.bytes);
        void *args[] = {&g_chunk, &d_tables, &status};
        // The arguments are copied at launch: g_chunk is free again on return.
        cudaError_t e = cudaLaunchKernel((const void *)noalloc_upload_kernel, dim3(1), dim3(256), args, 0, cs);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

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
    NvtxRange nvtx_range("mmf_filter1d_batched_noalloc");
    if (nseries < 0 || (nseries > 0 && (!h_len || !h_w))) return set_error(MMF_EINVAL, "bad series description");
    if (nseries > MMF_NOALLOC_MAX_SERIES)
        return set_error(MMF_EINVAL, "%lld series exceed the no-allocation limit of %d", (long long)nseries,
                         MMF_NOALLOC_MAX_SERIES);
    const int esz = elem_size(dtype);
    if (esz == 0) return set_error(MMF_EINVAL, "unknown dtype %d", (int)dtype);

    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    // Series table (inputs packed in order; outputs in order, each series
    // starting on a 32-byte boundary as in a batch plan) and output length.
    SeriesDesc *series = g_img.series;
    int64_t in_pos = 0, out_pos = 0, tiles = 0;
    const int64_t T = tile_of(dtype);
    for (int64_t s = 0; s < nseries; ++s) {
        SeriesDesc sd;
        mmf_status st = make_series(h_len[s], h_w[s], mode, dtype, &sd);
        if (st != MMF_OK) return st;
        // Positions stay far below 2^63: the input ends (and the outputs,
        // at most n per series plus 32 bytes of padding) cannot wrap.
        if (sd.n > INT64_MAX / 2 - in_pos || sd.n_out > INT64_MAX / 2 - out_pos - 32)
            return set_error(MMF_EINVAL, "series lengths overflow 64-bit positions");
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
    ItemDesc *items = g_img.items;
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
    std::memset(g_img.tickets, 0, sizeof(g_img.tickets) + sizeof(g_img.pad));

    LaunchCtx ctx;
    mmf_status st = get_ctx(stream, &ctx);  // refuses device ordinals >= kMaxDevices
    if (st != MMF_OK) return st;
    if (ctx.device < 0 || ctx.device >= kMaxDevices)
        return set_error(MMF_EINVAL, "device ordinal %d out of range", ctx.device);
    // Set-up once per device, with that device current: the device address of
    // the table array (the first call on a device does this).  It runs under
    // the call's lock, so a thread that finds the set-up done also sees the
    // address.
    DevAddr &da = g_noalloc_addr[ctx.device];
    if (!da.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-allocation tables)");
        da.ptr = static_cast<NoAllocTables *>(p);
        da.ready = true;
    }
    NoAllocTables *tab = da.ptr;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    uint8_t *d_tab = reinterpret_cast<uint8_t *>(tab);
    // Counters and series (contiguous from the start), then the items.
    cudaError_t e =
        upload(d_tab, 0, (uint32_t)(offsetof(NoAllocTables, series) + nseries * sizeof(SeriesDesc)), cs, ctx.status);
    if (e == cudaSuccess && ni > 0)
        e = upload(d_tab, (uint32_t)offsetof(NoAllocTables, items), (uint32_t)(ni * sizeof(ItemDesc)), cs, ctx.status);
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
