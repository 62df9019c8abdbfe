// The dispatch table of mmf_filter1d's automatic kernel choice, and its
// autotuner.
//
// Without an entry, MMF_KERNEL_AUTO takes the built-in rule: the register
// slide for windows up to 17 (f32) or 9 (other types), the per-range block
// scan otherwise.  An entry, keyed by (dtype, window bucket,
// length bucket), replaces that rule for its bucket; mmf_dispatch_autotune
// times the candidate kernels on the caller's buffers and stores the
// fastest.  Window buckets are exact up to 32 (where the slide's limits and
// the block modes change) and powers of two above; length buckets are powers
// of four.  With $MMF_AUTOTUNE_CACHE set, tuned entries are appended to that
// file (keyed by GPU name) and read back by later processes.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

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

int log2_floor(int64_t v) {
    int l = 0;
    while (v > 1) {
        v >>= 1;
        ++l;
    }
    return l;
}

uint64_t bucket_key(mmf_dtype dt, int64_t n, int64_t w) {
    const uint64_t wb = w <= 32 ? (uint64_t)w : (uint64_t)(32 + log2_floor(w));
    const uint64_t nb = (uint64_t)(log2_floor(n > 0 ? n : 1) / 2);
    return ((uint64_t)dt << 32) | (wb << 8) | nb;
}

std::mutex g_mu;
std::map<uint64_t, int> g_table;
bool g_loaded = false;

std::string gpu_name() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "gpu";
    std::string k(prop.name);
    for (auto &c : k)
        if (c == ' ') c = '_';
    return k;
}

// Reads the tuned entries of this GPU from $MMF_AUTOTUNE_CACHE once (g_mu held).
void load_cache() {
    if (g_loaded) return;
    g_loaded = true;
    const char *path = getenv("MMF_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    const std::string prefix = "dispatch|" + gpu_name() + "|";
    char k[512];
    int v = 0;
    while (fscanf(f, "%511s %d", k, &v) == 2) {
        if (strncmp(k, prefix.c_str(), prefix.size()) != 0) continue;
        unsigned long long key = 0;
        if (sscanf(k + prefix.size(), "%llx", &key) == 1 && v >= 0 && v <= MMF_KERNEL_FRONT) g_table[key] = v;
    }
    fclose(f);
}

void store_cache(uint64_t key, int v) {
    const char *path = getenv("MMF_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "dispatch|%s|%llx %d\n", gpu_name().c_str(), (unsigned long long)key, v);
    fclose(f);
}

// The built-in rule's kernel for a series (never AUTO).
mmf_kernel builtin(mmf_dtype dt, const SeriesDesc &sd, int sms) {
    const int slide_max = dt == MMF_F32 ? 17 : 9;
    if (sd.w <= slide_max) return MMF_KERNEL_SLIDE;
    bool front = false;
    switch (dt) {
        case MMF_F32: front = front_applies<float>(sd, sms, -1); break;
        case MMF_I16: front = front_applies<int16_t>(sd, sms, -1); break;
        case MMF_U8: front = front_applies<uint8_t>(sd, sms, -1); break;
        default: break;
    }
    return front ? MMF_KERNEL_FRONT : MMF_KERNEL_BLOCKSCAN;
}

}  // namespace

namespace mmf {

// The tuned kernel for a call, or MMF_KERNEL_AUTO if the bucket has none.
mmf_kernel dispatch_lookup(mmf_dtype dt, int64_t n, int64_t w) {
    std::lock_guard<std::mutex> lk(g_mu);
    load_cache();
    auto it = g_table.find(bucket_key(dt, n, w));
    return it == g_table.end() ? MMF_KERNEL_AUTO : static_cast<mmf_kernel>(it->second);
}

}  // namespace mmf

extern "C" {

mmf_status mmf_dispatch_set(mmf_dtype dtype, int64_t n, int64_t w, mmf_kernel kernel) {
    if (elem_size(dtype) == 0) return set_error(MMF_EINVAL, "unknown dtype %d", (int)dtype);
    if (n < 0 || w < 1) return set_error(MMF_EINVAL, "bad size n = %lld, w = %lld", (long long)n, (long long)w);
    if (kernel < MMF_KERNEL_AUTO || kernel > MMF_KERNEL_FRONT) return set_error(MMF_EINVAL, "unknown kernel %d", (int)kernel);
    std::lock_guard<std::mutex> lk(g_mu);
    load_cache();
    const uint64_t key = bucket_key(dtype, n, w);
    if (kernel == MMF_KERNEL_AUTO)
        g_table.erase(key);
    else
        g_table[key] = kernel;
    return MMF_OK;
}

mmf_status mmf_dispatch_get(mmf_dtype dtype, int64_t n, int64_t w, mmf_kernel *kernel) {
    if (!kernel) return set_error(MMF_EINVAL, "NULL output");
    SeriesDesc sd;
    mmf_status st = make_series(n, w, MMF_VALID, dtype, &sd);
    if (st != MMF_OK) return st;
    const mmf_kernel k = dispatch_lookup(dtype, n, w);
    if (k != MMF_KERNEL_AUTO) {
        *kernel = k;
        return MMF_OK;
    }
    LaunchCtx ctx;
    st = get_ctx(nullptr, &ctx);
    if (st != MMF_OK) return st;
    *kernel = builtin(dtype, sd, ctx.sms);
    return MMF_OK;
}

mmf_status mmf_dispatch_autotune(const void *d_in, int64_t n, int64_t w, mmf_dtype dtype, void *d_max, void *d_min,
                                 void *stream, mmf_kernel *chosen) {
    NvtxRange nvtx_range("mmf_dispatch_autotune");
    SeriesDesc sd;
    mmf_status st = make_series(n, w, MMF_VALID, dtype, &sd);
    if (st != MMF_OK) return st;
    if (sd.n_out == 0) return set_error(MMF_EINVAL, "no window of %lld fits %lld elements", (long long)w, (long long)n);
    LaunchCtx ctx;
    st = get_ctx(stream, &ctx);
    if (st != MMF_OK) return st;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    const int slide_max = dtype == MMF_F32 ? 17 : 9;
    bool front_ok = false;
    switch (dtype) {
        case MMF_F32: front_ok = front_applies<float>(sd, ctx.sms, 1); break;
        case MMF_I16: front_ok = front_applies<int16_t>(sd, ctx.sms, 1); break;
        case MMF_U8: front_ok = front_applies<uint8_t>(sd, ctx.sms, 1); break;
        default: break;
    }
    const mmf_kernel cands[] = {MMF_KERNEL_SLIDE, MMF_KERNEL_BLOCKSCAN, MMF_KERNEL_FRONT, MMF_KERNEL_WEDGE};
    cudaEvent_t e0, e1;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) return cuda_error(ce, "autotune events");
    mmf_kernel best = MMF_KERNEL_AUTO;
    float best_ms = 1e30f;
    for (mmf_kernel k : cands) {
        if (k == MMF_KERNEL_SLIDE && w > slide_max) continue;
        if (k == MMF_KERNEL_FRONT && !front_ok) continue;
        if (k == MMF_KERNEL_WEDGE && w > MMF_WEDGE_MAX_WINDOW) continue;
        float t[3] = {0.f, 0.f, 0.f};
        for (int rep = 0; rep < 4 && st == MMF_OK; ++rep) {
            cudaEventRecord(e0, cs);
            st = mmf_filter1d_ex(d_in, n, w, dtype, MMF_VALID, d_max, d_min, stream, k);
            cudaEventRecord(e1, cs);
            if (st != MMF_OK) break;
            ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess) {
                st = cuda_error(ce, "autotune run");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) t[rep - 1] = ms;  // the first run warms up
        }
        if (st != MMF_OK) break;
        const float med = t[0] < t[1] ? (t[1] < t[2] ? t[1] : (t[0] < t[2] ? t[2] : t[0]))
                                      : (t[0] < t[2] ? t[0] : (t[1] < t[2] ? t[2] : t[1]));
        if (med < best_ms) {
            best_ms = med;
            best = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MMF_OK) return st;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_cache();
        const uint64_t key = bucket_key(dtype, n, w);
        g_table[key] = best;
        store_cache(key, best);
    }
    if (chosen) *chosen = best;
    return MMF_OK;
}

}  // extern "C"
