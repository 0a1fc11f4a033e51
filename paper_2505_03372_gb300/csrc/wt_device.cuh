// Device-side building blocks shared by the construction kernels: relaxed
// global loads/stores, mbarrier + 1-D TMA bulk copies, the bounded decoupled
// look-back over tiles, and the tree lookup of batched work items.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_common.cuh"

namespace wt {

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// try_wait that suspends the thread for up to hint_ns while the phase is open
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}
// Wait for the given phase parity of an mbarrier with at most kSpinCap polls.
// A wait that gives up sets kStTimeout and returns false (the data is then
// not trusted; the status word reports it).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t* status) {
    uint32_t spins = 0;
    while (!mbar_try_wait_hint(bar, parity, 1000u)) {
        if (++spins > kSpinCap) {
            if ((threadIdx.x & 31) == 0) set_status(status, kStTimeout);
            return false;
        }
    }
    return true;
}
// 1-D TMA bulk copy global -> shared, completion signalled on the mbarrier.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// 1-D TMA bulk copy shared -> global in the CTA's bulk group; dst, src
// 16-byte aligned, bytes a multiple of 16.  Shared-memory writes the copy reads
// must be made visible to the async proxy first (fence_proxy_async).
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until at most N committed bulk groups still read shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// wait until every committed bulk group has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Look-back state word of a tile: flag (2 bits) | aggregate (19 bits) | inclusive prefix (43 bits).
constexpr uint64_t kFlagAgg = 1, kFlagIncl = 2;
__device__ __forceinline__ uint64_t lb_pack(uint64_t flag, uint64_t agg, uint64_t incl) {
    return flag | (agg << 2) | (incl << 21);
}
__device__ __forceinline__ uint64_t lb_flag(uint64_t s) { return s & 3u; }
__device__ __forceinline__ uint64_t lb_agg(uint64_t s) { return (s >> 2) & ((1u << 19) - 1); }
__device__ __forceinline__ uint64_t lb_incl(uint64_t s) { return s >> 21; }

// Decoupled look-back over tiles, run by one full warp: publish this tile's
// count of ones (as its inclusive prefix if it is tile 0), walk back over the
// earlier tiles 32 at a time summing aggregates until an inclusive prefix is
// found, then publish this tile's inclusive prefix.  Returns the ones before
// the tile.  Every wait is bounded: after spin_cap polls the warp sets
// kStTimeout in *status, counts the missing predecessor as zero and returns.
__device__ __forceinline__ uint64_t lookback_warp(uint64_t* state, uint64_t tile, uint64_t ones, uint32_t* status,
                                               uint32_t spin_cap) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) st_relaxed_u64(state + tile, tile == 0 ? lb_pack(kFlagIncl, ones, ones) : lb_pack(kFlagAgg, ones, 0));
    uint64_t excl = 0;
    if (tile == 0) return 0;
    int64_t base = (int64_t)tile - 1;
    uint32_t spins = 0;
    bool timed_out = false;
    while (true) {
        const int64_t idx = base - lane;
        uint64_t st = idx >= 0 ? ld_relaxed_u64(state + idx) : lb_pack(kFlagIncl, 0, 0);
        while (__any_sync(0xffffffffu, lb_flag(st) == 0)) {
            if (++spins > spin_cap) {
                timed_out = true;
                if (lb_flag(st) == 0) st = lb_pack(kFlagIncl, 0, 0);
                break;
            }
            __nanosleep(20);
            if (lb_flag(st) == 0) st = ld_relaxed_u64(state + idx);
        }
        const uint32_t im = __ballot_sync(0xffffffffu, lb_flag(st) == kFlagIncl);
        if (im) {
            const int first = __ffs(im) - 1;
            const uint64_t v = lane < first ? lb_agg(st) : (lane == first ? lb_incl(st) : 0);
            excl += warp_sum_u64(v);
            break;
        }
        excl += warp_sum_u64(lb_agg(st));
        base -= 32;
    }
    if (lane == 0) {
        if (timed_out) set_status(status, kStTimeout);
        st_relaxed_u64(state + tile, lb_pack(kFlagIncl, ones, excl + ones));
    }
    return excl;
}

// Last tree whose first work item is <= g (prefix has ntrees + 1 entries, prefix[0] = 0).
__device__ __forceinline__ uint32_t find_tree(const uint64_t* prefix, uint32_t ntrees, uint64_t g) {
    uint32_t lo = 0, hi = ntrees - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace wt
