// Thin inline-PTX wrappers for sm_100-family features used by the kernels:
// mbarrier transaction barriers, 1D bulk TMA copies (cp.async.bulk) with L2
// cache-policy hints, named barriers and bounded waits.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mmf {

// Device status word: kernels OR error bits into it instead of trapping.
// kErrRange: a checked build (MMF_CHECKED) found an index outside its range
// and skipped the access.
enum : uint32_t { kErrWaitTimeout = 1u, kErrBadItem = 2u, kErrRange = 4u };

#ifdef MMF_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait that may suspend the thread until the phase completes or about
// `hint_ns` nanoseconds have passed (no busy spinning).
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Default bound of a pipeline wait: about 2 s of SM clock.
constexpr long long kWaitLimitCycles = 4000000000LL;

// Wait for the phase with the given parity to complete, giving up after
// roughly `limit_cycles` SM clocks.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  long long limit_cycles = kWaitLimitCycles) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait_sleep(bar, parity, 20000u)) {
        if (clock64() - t0 > limit_cycles) return false;
    }
    return true;
}

// 16-byte asynchronous copy global -> shared (both addresses 16-byte
// aligned); bytes < 16 fills the rest with zeros (0: nothing is read).
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem_dst)), "l"(gsrc), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// L2 eviction-priority policies for cache hints.
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// 1D bulk copy global -> shared, completion signalled on `bar` as bytes.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                            uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bring the line holding p into L1 (no register, no wait).
__device__ __forceinline__ void prefetch_l1(const void *p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Named barrier over `nthreads` threads (a multiple of 32), id 1..15.
__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Named barrier that also ORs a predicate over the participating threads:
// every thread receives the same result, taken at the barrier itself, so a
// decision based on it (leave the work item) is the same for all of them.
__device__ __forceinline__ bool named_bar_sync_or(int id, int nthreads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void report_error(uint32_t *status, uint32_t bits) {
    if (status) atomicOr(status, bits);
}

// Range check of a global or shared index (a stand-in for a memory
// sanitizer): in a checked build (MMF_CHECKED) it records kErrRange and
// returns false when i lies outside [lo, hi), and the caller skips the
// access; otherwise it is always true and costs nothing.
// The same for an access of n bytes at p inside a buffer of len bytes at base.
__device__ __forceinline__ bool in_bytes(uint32_t *status, const void *p, int n, const void *base, int64_t len) {
    if constexpr (!kChecked) {
        return true;
    } else {
        const int64_t off = reinterpret_cast<const char *>(p) - reinterpret_cast<const char *>(base);
        if (off >= 0 && off + n <= len) return true;
        report_error(status, kErrRange);
        return false;
    }
}

__device__ __forceinline__ bool in_range(uint32_t *status, int64_t i, int64_t lo, int64_t hi) {
    if constexpr (!kChecked) {
        return true;
    } else {
        if (i >= lo && i < hi) return true;
        report_error(status, kErrRange);
        return false;
    }
}

}  // namespace mmf
