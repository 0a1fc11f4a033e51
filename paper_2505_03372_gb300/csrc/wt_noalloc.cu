// Rank/select support of a caller-owned bitvector, built without allocating.
//
// Some callers cannot allocate device memory while they run: code inside a
// custom allocator or a memory-pool callback, a real-time loop that must not
// take the driver's allocation lock, or a host framework that owns every byte
// of device memory and hands out only fixed buffers.  This entry point serves
// them.  The caller supplies the input bitvector and every output array; the
// only other memory the kernel uses is a fixed scratch array compiled into the
// library (one 64-bit look-back word per 65536-bit tile plus a tile counter),
// which every GPU that loads the library keeps until the process exits.
//
// The kernel is the counters-and-samples half of the build's level pass: one
// CTA per 65536-bit tile (one L1 block), a block scan of per-word popcounts for
// the L2 counters, a decoupled look-back over tiles for the L1 counter, and the
// select samples found from the word prefixes.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "wt_internal.hpp"

namespace wt {
namespace {

constexpr uint32_t kNaTileBits = 65536;              // one tile = one L1 block
constexpr uint32_t kNaTileWords = kNaTileBits / 64;  // 1024
constexpr uint32_t kNaThreads = 256;                 // 4 words per thread
constexpr uint64_t kNaMaxTiles = 65536;              // => at most 2^32 bits per call
constexpr uint64_t kNaFlagAgg = 1, kNaFlagIncl = 2;

// Shared by every call on a device: kNaMaxTiles look-back words, then the tile counter.
static __device__ __align__(256) uint64_t g_bv_scratch[kNaMaxTiles + 32];

__device__ __forceinline__ uint64_t na_ld(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void na_st(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// flag (2 bits) | tile ones (19 bits) | inclusive prefix (43 bits)
__device__ __forceinline__ uint64_t na_pack(uint64_t f, uint64_t agg, uint64_t incl) { return f | (agg << 2) | (incl << 21); }

__global__ void __launch_bounds__(kNaThreads) bv_support_kernel(const uint64_t* __restrict__ words, uint64_t nbits,
                                                                uint32_t k_log2, uint64_t* __restrict__ l1,
                                                                uint16_t* __restrict__ l2, uint64_t* __restrict__ s0,
                                                                uint64_t* __restrict__ s1, uint64_t s_cap,
                                                                uint64_t ntiles, uint64_t* __restrict__ scratch,
                                                                uint32_t* __restrict__ status,
                                                                uint64_t* __restrict__ total_ones) {
    __shared__ uint32_t s_wpre[kNaTileWords + 1];  // ones before each word of the tile
    __shared__ uint32_t s_wsum[kNaThreads / 32];
    __shared__ uint64_t s_tile, s_E;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint64_t* state = scratch;
    uint32_t* counter = reinterpret_cast<uint32_t*>(scratch + kNaMaxTiles);

    if (tid == 0) s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= ntiles) return;
    const uint64_t t0 = tile * kNaTileBits;
    const uint64_t nw_total = (nbits + 63) / 64;

    // popcounts of this thread's 4 words (bits at or past nbits do not count)
    uint32_t c[4], sum = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const uint64_t wi = tile * kNaTileWords + tid * 4 + k;
        uint64_t x = wi < nw_total ? __ldg(words + wi) : 0ull;
        const uint64_t end = (wi + 1) * 64;
        if (end > nbits && wi < nw_total) x &= (nbits & 63) ? ((1ull << (nbits & 63)) - 1ull) : ~0ull;
        c[k] = __popcll(x);
        sum += c[k];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    uint32_t wbefore = 0, ones = 0;
#pragma unroll
    for (int k = 0; k < kNaThreads / 32; k++) {
        const uint32_t v = s_wsum[k];
        if (k < warp) wbefore += v;
        ones += v;
    }
    uint32_t run = wbefore + inc - sum;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        s_wpre[tid * 4 + k] = run;
        run += c[k];
    }
    if (tid == 0) s_wpre[kNaTileWords] = ones;

    // look-back for the ones before the tile (= this tile's L1 counter)
    if (warp == 0) {
        if (lane == 0) na_st(state + tile, tile == 0 ? na_pack(kNaFlagIncl, ones, ones) : na_pack(kNaFlagAgg, ones, 0));
        uint64_t excl = 0;
        if (tile > 0) {
            int64_t base = (int64_t)tile - 1;
            uint32_t spins = 0;
            while (true) {
                const int64_t idx = base - lane;
                uint64_t st = idx >= 0 ? na_ld(state + idx) : na_pack(kNaFlagIncl, 0, 0);
                while (__any_sync(0xffffffffu, (st & 3u) == 0)) {
                    if (++spins > kSpinCap) {
                        if (lane == 0 && status) atomicOr(status, kStTimeout);
                        if ((st & 3u) == 0) st = na_pack(kNaFlagIncl, 0, 0);
                        break;
                    }
                    __nanosleep(20);
                    if ((st & 3u) == 0) st = na_ld(state + idx);
                }
                const uint32_t im = __ballot_sync(0xffffffffu, (st & 3u) == kNaFlagIncl);
                uint64_t v;
                if (im) {
                    const int first = __ffs(im) - 1;
                    v = lane < first ? ((st >> 2) & ((1u << 19) - 1)) : (lane == first ? (st >> 21) : 0);
                } else {
                    v = (st >> 2) & ((1u << 19) - 1);
                }
#pragma unroll
                for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                excl += v;
                if (im) break;
                base -= 32;
            }
            if (lane == 0) na_st(state + tile, na_pack(kNaFlagIncl, ones, excl + ones));
        }
        if (lane == 0) s_E = excl;
    }
    __syncthreads();
    const uint64_t E = s_E;
    const uint64_t count = nbits - t0 < kNaTileBits ? nbits - t0 : kNaTileBits;
    const uint64_t zeros = count - ones;
    const uint64_t R0 = t0 - E;

    // L1 and L2 counters (the tile is one L1 block, so L2 values are tile-local prefixes)
    if (tid == 0) l1[tile] = E;
    const uint32_t nl2 = (uint32_t)((count + 511) / 512);
    for (uint32_t b = tid; b < nl2; b += kNaThreads) l2[(t0 >> 9) + b] = (uint16_t)s_wpre[b * 8];
    if (tid == 0 && tile == ntiles - 1 && (nbits & 511) == 0) {
        if ((nbits & 65535) == 0) {
            l1[nbits >> 16] = E + ones;
            l2[nbits >> 9] = 0;
        } else {
            l2[nbits >> 9] = (uint16_t)ones;
        }
    }
    if (tid == 0 && tile == 0) {
        s0[0] = 0;
        s1[0] = 0;
    }
    if (tid == 0 && tile == ntiles - 1 && total_ones) *total_ones = E + ones;
    // select samples: position of every K-th one and every K-th zero
    const uint64_t m1lo = (E >> k_log2) + 1, m1hi = (E + ones) >> k_log2;
    const uint64_t m0lo = (R0 >> k_log2) + 1, m0hi = (R0 + zeros) >> k_log2;
    const uint64_t ns1 = m1hi + 1 - m1lo, ns0 = m0hi + 1 - m0lo;
    for (uint64_t idx = tid; idx < ns1 + ns0; idx += kNaThreads) {
        const uint32_t b = idx < ns1;
        const uint64_t m = b ? m1lo + idx : m0lo + (idx - ns1);
        const uint32_t t = (uint32_t)((m << k_log2) - (b ? E : R0));  // 1-based rank within the tile
        int lo = 0, hi = kNaTileWords - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            const uint32_t cb = b ? s_wpre[mid] : (uint32_t)(mid * 64) - s_wpre[mid];
            if (cb < t) lo = mid;
            else hi = mid - 1;
        }
        const uint32_t before = b ? s_wpre[lo] : (uint32_t)(lo * 64) - s_wpre[lo];
        uint64_t x = __ldg(words + tile * kNaTileWords + lo);
        if (!b) x = ~x;
        if (m < s_cap) (b ? s1 : s0)[m] = t0 + (uint64_t)lo * 64 + select_in_word(x, t - before);
    }
}

// The scratch's device address per device, with the identity of the context it
// was looked up in: a device reset makes a new context (a new identity), and the
// next call looks the address up again instead of using a stale one.
std::mutex g_na_mu;
void* g_na_addr[256];
unsigned long long g_na_ctx[256];
bool g_na_ready[256];

typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

// Identity of the current context (0 if the driver cannot tell).
unsigned long long na_context_id() {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (get_cur && get_id && get_cur(&ctx) == 0 && ctx && get_id(ctx, &id) == 0) return id;
    return 0;
}

}  // namespace
}  // namespace wt

using namespace wt;

extern "C" wt_status wt_bitvector_support_static(const uint64_t* d_words, uint64_t nbits, uint32_t sample_k,
                                                 uint64_t* d_l1, uint16_t* d_l2, uint64_t* d_s0, uint64_t* d_s1,
                                                 uint64_t sample_capacity, uint32_t* d_status, uint64_t* d_ones,
                                                 wt_stream stream) {
    if (nbits == 0 || nbits > kNaMaxTiles * (uint64_t)kNaTileBits) return WT_EINVAL;  // beyond the static scratch
    if (sample_k < 256 || sample_k > (1u << 20) || (sample_k & (sample_k - 1))) return WT_EINVAL;
    if (sample_capacity < (nbits / sample_k) + 2) return WT_EINVAL;
    if (!device_ptr_ok(d_words) || !device_ptr_ok(d_l1) || !device_ptr_ok(d_l2) || !device_ptr_ok(d_s0) ||
        !device_ptr_ok(d_s1))
        return WT_EINVAL;
    if (d_status && !device_ptr_ok(d_status)) return WT_EINVAL;
    if (d_ones && !device_ptr_ok(d_ones)) return WT_EINVAL;
    // an error left pending by earlier work on this thread would otherwise be
    // reported as this call's launch error
    if (cudaPeekAtLastError() != cudaSuccess) return WT_ECUDA;

    // device address of the static scratch, looked up once per device with that device current
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return WT_ECUDA;
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        const unsigned long long ctx = na_context_id();
        if (!g_na_ready[dev] || g_na_ctx[dev] != ctx || ctx == 0) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_bv_scratch) != cudaSuccess) {
                g_na_ready[dev] = false;
                return WT_ECUDA;
            }
            g_na_addr[dev] = p;
            g_na_ctx[dev] = ctx;
            g_na_ready[dev] = true;
        }
        scratch = g_na_addr[dev];
    }
    const uint64_t ntiles = (nbits + kNaTileBits - 1) / kNaTileBits;
    uint32_t k_log2 = 0;
    while ((1u << k_log2) < sample_k) k_log2++;
    cudaStream_t s = stream;
    // the look-back words and the tile counter must start at zero (the array keeps the last call's contents)
    if (cudaMemsetAsync(scratch, 0, ntiles * sizeof(uint64_t), s) != cudaSuccess) return WT_ECUDA;
    if (cudaMemsetAsync(static_cast<uint64_t*>(scratch) + kNaMaxTiles, 0, 32 * sizeof(uint64_t), s) != cudaSuccess)
        return WT_ECUDA;
    bv_support_kernel<<<(unsigned)ntiles, kNaThreads, 0, s>>>(d_words, nbits, k_log2, d_l1, d_l2, d_s0, d_s1,
                                                              sample_capacity, ntiles, static_cast<uint64_t*>(scratch),
                                                              d_status, d_ones);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}
