// Construction of the extended level-wise wavelet tree (Section 5.1,
// Algorithm 4) on one GB300.
//
// Pipeline (all on the device, one stream):
//   1. histogram of S with symbol validation (Section 5.1.1: shared-memory
//      sub-histograms, persistent grid), which also counts the level-0 ones of
//      every 16 KiB tile;
//   2. C = exclusive prefix sum of the histogram;
//   3. node table: for every node (depth l, code prefix p) its start C[a],
//      the precomputed rank_0 at the start (Section 5.2.1) and the two
//      partition offsets, derived from C alone (the number of zeros before a
//      node start is the total size of the left children of the earlier nodes
//      of that level);
//   4. one fused pass per level l: read T_l (S for l = 0, re-encoded with the
//      reduced codes on the fly), write the packed bits of level l, its L1/L2
//      rank counters (Section 4.1) and its select samples (Section 4.2), and
//      stably partition T_l by the level bit into T_{l+1} -- the radix-sort step
//      of Algorithm 4 done as a one-bit split per level.  The global prefix of
//      ones each tile needs for the counters and the partition is an exclusive
//      scan of per-tile counts that the pass before gathered while writing T_l
//      (the histogram for level 0), so every level reads T_l once and writes
//      T_{l+1} once.  Batches of trees (wt_batch.cu) find the prefix by a
//      decoupled look-back over tiles instead.
//   The wavelet matrix layout uses the same passes with one node per level.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "wt_internal.hpp"

namespace wt {

// ===========================================================================
// small device utilities
// ===========================================================================

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
// try_wait that suspends the thread for up to 1 us while the phase is open
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(1000u)
        : "memory");
    return ok != 0;
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

// bit i of x -> bit 2i
__device__ __forceinline__ uint64_t spread2(uint32_t x) {
    uint64_t v = x;
    v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
    v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
    v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}
// bit i (i < 16) of x -> bit 4i
__device__ __forceinline__ uint64_t spread4(uint32_t x) {
    uint64_t v = x & 0xFFFFu;
    v = (v | (v << 24)) & 0x000000FF000000FFull;
    v = (v | (v << 12)) & 0x000F000F000F000Full;
    v = (v | (v << 6)) & 0x0303030303030303ull;
    v = (v | (v << 3)) & 0x1111111111111111ull;
    return v;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Tiles of the level passes: 16 KiB of T_l each (1024 16-byte vectors); the
// histogram counts the level-0 ones of every such tile.
constexpr int kTileBytesHist = 16384;
constexpr uint32_t kTileVecLog2 = 10;
static_assert((16u << kTileVecLog2) == (uint32_t)kTileBytesHist, "tile size");

// ===========================================================================
// 1. histogram + validation
// ===========================================================================

// Also counts, per 16 KiB tile of S, the symbols whose level-0 bit is 1 (the
// symbols >= m0, as codes grow with the symbol), so that the level-0 pass knows
// every tile's prefix of ones (tcnt zeroed; null: not counted).
template <typename T>
__global__ void __launch_bounds__(512) hist_kernel(const T* __restrict__ S, uint64_t n, uint32_t sigma, uint32_t sbins,
                                                   uint32_t cstride, uint32_t copies,
                                                   unsigned long long* __restrict__ hist, uint32_t* __restrict__ status,
                                                   uint32_t m0, unsigned long long* __restrict__ tcnt) {
    constexpr uint32_t TE = kTileBytesHist / sizeof(T);  // elements per tile; a tile is 1024 16-byte vectors
    extern __shared__ uint32_t sh[];
    if constexpr (sizeof(T) == 1) {
        // Bytes: all 256 bins, one copy per lane, bin-major (copy k of bin b at
        // b * 32 + k: every lane counts in its own bank).  No test per symbol:
        // a symbol >= sigma shows as a nonzero bin >= sigma at the end.
        for (uint32_t i = threadIdx.x; i < 256 * 32; i += blockDim.x) sh[i] = 0;
        __syncthreads();
        uint32_t* mine = sh + (threadIdx.x & 31);
        const uint64_t nvec = n / 16;
        const uint4* S4 = reinterpret_cast<const uint4*>(S);
        const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
        // bytes >= m0, two at a time in 16-bit lanes: b + 256 - m0 carries into bit 8 exactly when b >= m0
        const uint32_t madd = (256u - (m0 < 256 ? m0 : 0u)) * 0x00010001u;
        const bool tc = tcnt != nullptr && m0 < 256;
        for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec; v += stride) {
            const uint4 x = __ldg(S4 + v);
            const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int k = 0; k < 4; k++)
#pragma unroll
                for (int j = 0; j < 4; j++) atomicAdd(mine + (((w4[k] >> (8 * j)) & 0xffu) << 5), 1u);
            if (tc) {
                // the warp's 32 vectors lie in one tile
                uint32_t c = 0;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const uint32_t e = ((w4[k] & 0x00FF00FFu) + madd) & 0x01000100u;
                    const uint32_t o = (((w4[k] >> 8) & 0x00FF00FFu) + madd) & 0x01000100u;
                    c += __popc(e | (o << 1));
                }
                const uint32_t am = __activemask();
                c = __reduce_add_sync(am, c);
                if ((threadIdx.x & 31) == (uint32_t)(__ffs(am) - 1) && c) atomicAdd(tcnt + (v >> kTileVecLog2), (unsigned long long)c);
            }
        }
        for (uint64_t j = nvec * 16 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
            const uint32_t b = (uint32_t)S[j];
            atomicAdd(mine + (b << 5), 1u);
            if (tc && b >= m0) atomicAdd(tcnt + j / TE, 1ull);
        }
        __syncthreads();
        bool bad = false;
        for (uint32_t b = threadIdx.x; b < 256; b += blockDim.x) {
            uint32_t c = 0;
            for (uint32_t k = 0; k < 32; k++) c += sh[b * 32 + ((k + b) & 31)];
            if (b >= sigma) bad |= c != 0;
            else if (c) atomicAdd(hist + b, (unsigned long long)c);
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kStSymbol);
        return;
    }
    for (uint32_t i = threadIdx.x; i < cstride * copies; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    // copy k of bin b at b * 32 + k (one copy per lane: every lane has its own
    // bank) or at k * cstride + b
    const bool lanes = copies == 32;
    uint32_t* mine = lanes ? sh + (threadIdx.x & 31) : sh + (threadIdx.x % copies) * cstride;
    bool bad = false;
    constexpr int V = 16 / sizeof(T);
    const uint64_t nvec = n / V;
    const uint4* S4 = reinterpret_cast<const uint4*>(S);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    auto add = [&](uint32_t s) {
        if (s >= sigma) bad = true;
        else if (s < sbins) atomicAdd(mine + (lanes ? s * 32 : s), 1u);
        else atomicAdd(hist + s, 1ull);
    };
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec; v += stride) {
        uint4 x = __ldg(S4 + v);
        const T* e = reinterpret_cast<const T*>(&x);
        uint32_t c = 0;
#pragma unroll
        for (int k = 0; k < V; k++) {
            add((uint32_t)e[k]);
            c += (uint32_t)e[k] >= m0;
        }
        if (tcnt != nullptr) {
            const uint32_t am = __activemask();
            c = __reduce_add_sync(am, c);
            if ((threadIdx.x & 31) == (uint32_t)(__ffs(am) - 1) && c) atomicAdd(tcnt + (v >> kTileVecLog2), (unsigned long long)c);
        }
    }
    for (uint64_t j = nvec * V + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        add((uint32_t)S[j]);
        if (tcnt != nullptr && (uint32_t)S[j] >= m0) atomicAdd(tcnt + j / TE, 1ull);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kStSymbol);
    for (uint32_t b = threadIdx.x; b < sbins; b += blockDim.x) {
        uint32_t c = 0;
        for (uint32_t k = 0; k < copies; k++) c += lanes ? sh[b * 32 + k] : sh[k * cstride + b];
        if (c) atomicAdd(hist + b, (unsigned long long)c);
    }
}

// ===========================================================================
// 2. device-wide exclusive scan of uint64 (out has count + 1 entries)
// ===========================================================================

constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;
constexpr int kScanChunk = kScanThreads * kScanPer;

// Exclusive scan of one chunk by one block (out[i] = carry + sum in[0, i));
// returns the chunk total.
__device__ uint64_t block_scan_chunk(const uint64_t* in, uint64_t* out, uint64_t count, uint64_t carry) {
    __shared__ uint64_t wsum[32];
    __shared__ uint64_t s_total;
    uint64_t v[kScanPer];
    const uint64_t base = (uint64_t)threadIdx.x * kScanPer;
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        v[k] = (base + k < count) ? in[base + k] : 0;
        s += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint64_t x = wsum[lane];
        uint64_t y = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t t = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += t;
        }
        wsum[lane] = y - x;
        if (lane == 31) s_total = y;
    }
    __syncthreads();
    uint64_t run = carry + wsum[warp] + (inc - s);
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        if (base + k < count) out[base + k] = run;
        run += v[k];
    }
    const uint64_t tot = s_total;
    __syncthreads();  // wsum and s_total are reused by the next chunk
    return tot;
}

__global__ void __launch_bounds__(kScanThreads) scan_partials_kernel(const uint64_t* in, uint64_t count,
                                                                     uint64_t* partial) {
    const uint64_t base = (uint64_t)blockIdx.x * kScanChunk;
    uint64_t s = 0;
    const uint64_t end = umin64(count, base + kScanChunk);
    for (uint64_t i = base + threadIdx.x; i < end; i += kScanThreads) s += in[i];
    s = warp_sum_u64(s);
    __shared__ uint64_t ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint64_t x = warp_sum_u64(ws[threadIdx.x]);
        if (threadIdx.x == 0) partial[blockIdx.x] = x;
    }
}

// Single block: exclusive scan of in[0, count) into out[0, count], out[count] = total.
__global__ void __launch_bounds__(kScanThreads) scan_single_kernel(const uint64_t* in, uint64_t* out, uint64_t count) {
    uint64_t carry = 0;
    for (uint64_t base = 0; base < count; base += kScanChunk) {
        uint64_t c = umin64((uint64_t)kScanChunk, count - base);
        carry += block_scan_chunk(in + base, out + base, c, carry);
    }
    if (threadIdx.x == 0) out[count] = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint64_t* in, uint64_t* out, uint64_t count,
                                                                  const uint64_t* partial_excl) {
    const uint64_t base = (uint64_t)blockIdx.x * kScanChunk;
    uint64_t c = umin64((uint64_t)kScanChunk, count - base);
    block_scan_chunk(in + base, out + base, c, partial_excl[blockIdx.x]);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[count] = partial_excl[gridDim.x];
}

// tmp must hold ceil(count / kScanChunk) + 1 + ceil(count / kScanChunk) + 1 entries
void device_exclusive_scan(const uint64_t* in, uint64_t* out, uint64_t count, uint64_t* tmp, cudaStream_t s,
                           const char* name) {
    if (count <= (uint64_t)kScanChunk) {
        ProfScope ps(name, s);
        scan_single_kernel<<<1, kScanThreads, 0, s>>>(in, out, count);
        return;
    }
    uint64_t nb = (count + kScanChunk - 1) / kScanChunk;
    uint64_t* part = tmp;
    uint64_t* part_ex = tmp + nb + 1;
    {
        ProfScope ps(name, s);
        scan_partials_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, count, part);
    }
    {
        ProfScope ps(name, s);
        scan_single_kernel<<<1, kScanThreads, 0, s>>>(part, part_ex, nb);
    }
    {
        ProfScope ps(name, s);
        scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, count, part_ex);
    }
}

// ===========================================================================
// 3. node table
// ===========================================================================

// slot = 2^l - 1 + p.  left[slot] = size of the left child (0 for non-nodes).
__global__ void node_start_kernel(const CodeParams cp, const uint64_t* __restrict__ C, NodeEntry* __restrict__ nodes,
                                  uint64_t* __restrict__ left, uint64_t nslots) {
    uint64_t slot = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= nslots) return;
    uint32_t l = 63u - (uint32_t)__clzll((long long)(slot + 1));
    uint64_t p = slot + 1 - (1ull << l);
    uint64_t a = 0;
    uint64_t w = node_info(cp, l, p, a);
    NodeEntry e = {0, 0, 0, 0};
    uint64_t lf = 0;
    if (w >= 2) {
        uint64_t m = node_mid(a, w);
        e.start = C[a];
        lf = C[m] - e.start;
    }
    nodes[slot] = e;
    left[slot] = lf;
}

// excl = exclusive scan of left over all slots (nslots + 1 entries).
// r0(slot) = zeros before the node = sum of left-child sizes of the earlier
// nodes of its level.  Also writes per-level metadata.
__global__ void node_finish_kernel(NodeEntry* __restrict__ nodes, const uint64_t* __restrict__ left,
                                   const uint64_t* __restrict__ excl, uint64_t nslots) {
    uint64_t slot = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= nslots) return;
    uint32_t l = 63u - (uint32_t)__clzll((long long)(slot + 1));
    uint64_t lvl0 = (1ull << l) - 1;
    NodeEntry e = nodes[slot];
    uint64_t r0 = excl[slot] - excl[lvl0];
    e.r0 = r0;
    e.off0 = e.start - r0;
    e.off1 = left[slot] + r0;
    nodes[slot] = e;
}

struct MetaArgs {
    uint64_t s0[kMaxLevels];  // first symbol whose code has length <= l (sigma if none)
};

// meta[2l] = size_l = C[s0_l]; meta[2l+1] = zeros_l = sum of left-child sizes at level l.
__global__ void meta_kernel(const MetaArgs ma, uint32_t L, const uint64_t* __restrict__ C,
                            const uint64_t* __restrict__ excl, uint64_t* __restrict__ meta) {
    uint32_t l = threadIdx.x;
    if (l >= L) return;
    meta[2 * l] = C[ma.s0[l]];
    meta[2 * l + 1] = excl[(2ull << l) - 1] - excl[(1ull << l) - 1];
}

// ===========================================================================
// 4. the fused level pass
// ===========================================================================

constexpr int kTileBytes = kTileBytesHist;
constexpr int kLpThreads = 256;
constexpr int kLpBlocksPerSM = 6;
constexpr uint64_t kFlagAgg = 1, kFlagIncl = 2;

// look-back state word: flag (2 bits) | aggregate (19 bits) | inclusive prefix (43 bits)
__device__ __forceinline__ uint64_t lb_pack(uint64_t flag, uint64_t agg, uint64_t incl) {
    return flag | (agg << 2) | (incl << 21);
}
__device__ __forceinline__ uint64_t lb_flag(uint64_t s) { return s & 3u; }
__device__ __forceinline__ uint64_t lb_agg(uint64_t s) { return (s >> 2) & ((1u << 19) - 1); }
__device__ __forceinline__ uint64_t lb_incl(uint64_t s) { return s >> 21; }


// 32-bit shared-memory addressing for the byte / half / word scatter stores.
// The value is a 32-bit register whose low 8 / 16 bits are stored: no
// truncation instruction per element (the byte stores of one word pass w,
// w >> 8, w >> 16, w >> 24; measured 0.734 -> 0.716 ms per u8 level pass).
__device__ __forceinline__ void sts_b8(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.b8 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void sts_b16(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.b16 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void sts_b32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ uint4 lds_u128(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr)
                 : "memory");
    return v;
}
// Bytes 4q + fs/8 .. 4q + fs/8 + 15 of the 32 bytes x:y (q < 4, fs a multiple of 8 below 32).
__device__ __forceinline__ uint4 shift16(const uint4 x, const uint4 y, uint32_t q, uint32_t fs) {
    const uint32_t w[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
    switch (q) {
        case 0: return make_uint4(__funnelshift_r(w[0], w[1], fs), __funnelshift_r(w[1], w[2], fs),
                                  __funnelshift_r(w[2], w[3], fs), __funnelshift_r(w[3], w[4], fs));
        case 1: return make_uint4(__funnelshift_r(w[1], w[2], fs), __funnelshift_r(w[2], w[3], fs),
                                  __funnelshift_r(w[3], w[4], fs), __funnelshift_r(w[4], w[5], fs));
        case 2: return make_uint4(__funnelshift_r(w[2], w[3], fs), __funnelshift_r(w[3], w[4], fs),
                                  __funnelshift_r(w[4], w[5], fs), __funnelshift_r(w[5], w[6], fs));
        default: return make_uint4(__funnelshift_r(w[3], w[4], fs), __funnelshift_r(w[4], w[5], fs),
                                   __funnelshift_r(w[5], w[6], fs), __funnelshift_r(w[6], w[7], fs));
    }
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// Partition one group (32 lanes x 16 bytes) of a tile into the shared-memory
// image: the lane's element with level bit b goes to slot A1 + (ones before it
// in the lane) if b = 1, else to A0 + (zeros before it in the lane).  Slots of
// two elements travel as a 16-bit pair.  For one-byte symbols
// the in-word ranks come from byte-wise prefix counts of the level bits; with
// ABS the slots are shared-memory addresses already (A0, A1 include out).
template <typename T, bool FULL, bool ABS = false>
__device__ __forceinline__ void scatter_group(const uint32_t out, const uint4 V, uint32_t m, uint32_t A0, uint32_t A1,
                                              uint32_t j0, uint32_t count, uint32_t shift) {
    constexpr int W = sizeof(T);
    constexpr int EPW = 4 / W;
    constexpr uint32_t SC = ABS ? W : 1;  // slot unit: bytes when ABS, elements otherwise
    const uint32_t wv[4] = {V.x, V.y, V.z, V.w};
    const uint32_t A0x2 = A0 * 0x00010001u, A1x2 = A1 * 0x00010001u;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const uint32_t w = wv[i];
        const uint32_t jw = j0 + i * EPW;
        // ones among the lane's earlier words
        const uint32_t ci = (i == 0) ? 0u : __popc(m & ((1u << (i * EPW)) - 1u));
        const uint32_t b1 = A1x2 + ci * (SC * 0x00010001u);                                     // one-slot base, paired
        const uint32_t b0 = (A0x2 + (uint32_t)(i * EPW * SC) * 0x00010001u) - ci * (SC * 0x00010001u);  // zero-slot base
        if (W == 1) {
            // bytes of y: level bits of the word's 4 elements; pre: ones before each element
            const uint32_t y = (w >> shift) & 0x01010101u;
            const uint32_t pre = y * 0x01010100u;
            const uint32_t sel = y * 0xFFu;
            const uint32_t off = (pre & sel) | ((0x03020100u - pre) & ~sel);  // rank among same-bit elements
            const uint32_t s01 = __byte_perm(sel, 0, 0x1100), s23 = __byte_perm(sel, 0, 0x3322);
            const uint32_t I01 = ((b1 & s01) | (b0 & ~s01)) + __byte_perm(off, 0, 0x4140);
            const uint32_t I23 = ((b1 & s23) | (b0 & ~s23)) + __byte_perm(off, 0, 0x4342);
            const uint32_t ob = ABS ? 0u : out;
            if (FULL || jw + 0 < count) sts_b8(ob + (I01 & 0xFFFFu), w);
            if (FULL || jw + 1 < count) sts_b8(ob + (I01 >> 16), w >> 8);
            if (FULL || jw + 2 < count) sts_b8(ob + (I23 & 0xFFFFu), w >> 16);
            if (FULL || jw + 3 < count) sts_b8(ob + (I23 >> 16), w >> 24);
        } else if (W == 2) {
            const uint32_t bb = (m >> (2 * i)) & 3u;
            const uint32_t sel = (bb & 1u ? 0x0000FFFFu : 0u) | (bb & 2u ? 0xFFFF0000u : 0u);
            // second element: ones before it if it is a one, zeros before it otherwise
            const uint32_t off = ((bb ^ (bb >> 1)) & 1u) ? 0u : (SC << 16);
            const uint32_t I = ((b1 & sel) | (b0 & ~sel)) + off;
            if (FULL || jw + 0 < count) sts_b16(ABS ? (I & 0xFFFFu) : out + 2 * (I & 0xFFFFu), w);
            if (FULL || jw + 1 < count) sts_b16(ABS ? (I >> 16) : out + 2 * (I >> 16), w >> 16);
        } else {
            const uint32_t bit = (m >> i) & 1u;
            if (FULL || jw < count) sts_b32(ABS ? ((bit ? b1 : b0) & 0xFFFFu) : out + 4 * ((bit ? b1 : b0) & 0xFFFFu), w);
        }
    }
}

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

// Diagnostic: tile 1 looks back at a tile 0 that never publishes anything.
__global__ void lookback_timeout_kernel(uint64_t* state, uint32_t* status, uint32_t spin_cap, uint64_t* out) {
    const uint64_t excl = lookback_warp(state, 1, 5, status, spin_cap);
    if (threadIdx.x == 0) *out = excl;
}

// One tile of one level pass (the phases below).  Called by every thread of the
// CTA; returns whether the tile's load used the mbarrier (its parity flips).
template <typename T, bool ENCODE, bool FOLD = false>
__device__ __forceinline__ bool level_pass_tile(const LevelPassArgs& a, const uint64_t tile, uint8_t* smem,
                                                uint64_t* mbar_p, uint32_t mphase) {
    constexpr int W = sizeof(T);
    constexpr int VEPL = 16 / W;                // elements per lane per group (one uint4 per lane)
    constexpr int EPW = 4 / W;                  // elements per 32-bit word
    constexpr int TE = kTileBytes / W;          // elements per tile
    constexpr int NG = kTileBytes / 512;        // groups per tile: one group = 32 lanes x 16 bytes
    constexpr int NWARP = kLpThreads / 32;
    constexpr int GPW = NG / NWARP;             // groups per warp in phase 1
    constexpr int GE = 512 / W;                 // elements (= bits) per group
    constexpr int GBYTES = GE / 8;              // bytes of level bits per group
    constexpr int TPL1 = 65536 / TE;            // tiles per L1 block
    constexpr int GPL2 = W;                     // groups per 512-bit L2 block
    constexpr uint32_t EMASK = (W == 4) ? 0xFFFFFFFFu : ((1u << (8 * W)) - 1u);
    constexpr uint32_t LOWB = (W == 1) ? 0x01010101u : (W == 2 ? 0x00010001u : 1u);  // bit 0 of every element
    static_assert(NG % NWARP == 0 && NG <= 64, "tile shape");

    // the partitioned image first: its byte addresses fit in 16 bits (see ABS)
    uint8_t* outb = smem;
    uint8_t* inb = smem + kTileBytes;
    uint4* in4 = reinterpret_cast<uint4*>(inb);
    uint8_t* wbytes = smem + 2 * kTileBytes + 64;                               // level bits of the tile
    uint32_t* rpre = reinterpret_cast<uint32_t*>(wbytes + kTileBytes / 8 / W);  // NG + 1
    T* ctab = reinterpret_cast<T*>(rpre + 64 + 1);                              // code table (ENCODE, small sigma)

    __shared__ uint64_t s_E, s_EL1, s_p;
    __shared__ uint32_t s_single;
    __shared__ uint32_t s_nc[4];  // ones of T_{l+1} written by this tile: per run, in its first / second tile
    __shared__ uint32_t s_wpre[kTileBytes / 8 / W / 8];  // per 64-bit word of level bits: ones before it in its group
    __shared__ uint32_t s_gcnt[64];
    __shared__ uint32_t s_gnext;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t t0 = tile * TE;
    const uint32_t count = (uint32_t)umin64((uint64_t)TE, a.size - t0);
    const bool full = count == (uint32_t)TE;
    const uint32_t bytes = count * W;
    const uint32_t b16 = bytes & ~15u;
    const uint8_t* srcb = reinterpret_cast<const uint8_t*>(a.src) + t0 * W;
    const bool used_mbar = b16 != 0;

    // ---- phase 0: tile -> shared memory (TMA bulk copy + ragged tail) ----
    if (tid == 0 && b16) {
        mbar_expect_tx(mbar_p, b16);
        bulk_g2s(inb, srcb, b16, mbar_p);
    }
    if (tid < 4) s_nc[tid] = 0;
    for (uint32_t i = b16 + tid; i < bytes; i += kLpThreads) inb[i] = srcb[i];
    if (b16 && warp == 0) {  // one warp waits; the barrier hands the tile to all
        uint32_t spins = 0;
        while (!mbar_try_wait(mbar_p, mphase)) {
            if (++spins > kSpinCap) {
                if (lane == 0) set_status(a.status, kStTimeout);
                break;
            }
        }
    }
    __syncthreads();

    // ---- phase 1: level bits of every lane's 16 bytes -> shared memory ----
    const uint32_t shift = a.shift_bit;
#pragma unroll 2  // two groups in flight: 0.707 -> 0.702 ms per u8 pass (no unrolling: 0.707, four: 0.713)
    for (int gg = 0; gg < GPW; gg++) {
        const int g = warp * GPW + gg;
        uint4 V = in4[g * 32 + lane];
        const uint32_t j0 = g * GE + lane * VEPL;
        uint32_t wv[4] = {V.x, V.y, V.z, V.w};
        if (ENCODE && W == 1 && a.swar_codes) {
            // byte symbols, sigma <= 128 with at most three segments: the code
            // of a symbol in segment i is A_i + ((s & (2^e_i - 1)) << sh_i)
            // (closed form of `encode`), four bytes at a time.  Segment i
            // starts at P_i; a byte is in segment i or later iff s + (128 -
            // P_i) sets its bit 7 (s < 128, so no carry leaves a byte; the
            // bytes past a ragged tile's end carry only into higher bytes,
            // which are past the end too).
            const uint32_t L = a.cp.L, r = a.cp.r;
            auto seg = [&](uint32_t x, uint32_t i) {
                const uint32_t e = a.cp.e[i];
                const uint32_t len = (i + 1 == r) ? i + e : i + 1 + e;
                const uint32_t add = ((1u << i) - 1u) << (L - i);
                return ((x & (((1u << e) - 1u) * 0x01010101u)) << (L - len)) + add * 0x01010101u;
            };
            if (r == 2) {
                // two segments, [0, 2^e0) and [2^e0, sigma): the codes are s and
                // 2^e0 + ((s & (2^e1 - 1)) << (e0 - e1)), and bit e0 of s tells
                // the segment (no sum carries out of a byte)
                const uint32_t e0 = a.cp.e[0], e1 = a.cp.e[1];
                const uint32_t bmask = ((1u << e1) - 1u) * 0x01010101u;
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const uint32_t x = wv[i];
                    const uint32_t hi = (x >> e0) & 0x01010101u;
                    const uint32_t m = hi * 0xFFu;
                    const uint32_t c1 = ((x & bmask) << (e0 - e1)) + (hi << e0);
                    wv[i] = (x & ~m) | (c1 & m);
                }
            } else {
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const uint32_t x = wv[i];
                    uint32_t code = seg(x, 0);
#pragma unroll
                    for (uint32_t k = 1; k < 3; k++) {
                        if (k < r) {
                            const uint32_t g = (x + (128u - (uint32_t)a.cp.P[k]) * 0x01010101u) & 0x80808080u;
                            const uint32_t m = (g >> 7) * 0xFFu;
                            code = (code & ~m) | (seg(x, k) & m);
                        }
                    }
                    wv[i] = code;
                }
            }
            in4[g * 32 + lane] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        } else if (ENCODE && W == 1 && a.ctab_n == 256) {
            // byte symbols: a 256-entry table, no bounds tests (entries past
            // sigma and past the tile's end are never used)
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const uint32_t x = wv[i];
                wv[i] = (uint32_t)ctab[x & 0xffu] | ((uint32_t)ctab[(x >> 8) & 0xffu] << 8) |
                        ((uint32_t)ctab[(x >> 16) & 0xffu] << 16) | ((uint32_t)ctab[x >> 24] << 24);
            }
            in4[g * 32 + lane] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        } else if (ENCODE && !a.cp.pow2) {  // a power-of-two alphabet has identity codes
#pragma unroll
            for (int i = 0; i < 4; i++) {
                uint32_t nv = 0;
#pragma unroll
                for (int k = 0; k < EPW; k++) {
                    const uint32_t e = (wv[i] >> (8 * W * k)) & EMASK;
                    uint32_t code = 0;
                    if (j0 + i * EPW + k < count) {
                        if (a.ctab_n) {
                            code = ctab[e < a.ctab_n ? e : 0];
                        } else {
                            uint32_t len;
                            encode(a.cp, e, code, len);
                        }
                    }
                    nv |= (code & EMASK) << (8 * W * k);
                }
                wv[i] = nv;
            }
            in4[g * 32 + lane] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
        uint32_t m = 0;  // bit k = level bit of the lane's element k
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const uint32_t y = (wv[i] >> shift) & LOWB;
            uint32_t b;
            if (W == 1) b = (y * 0x10204080u) >> 28;
            else if (W == 2) b = (y | (y >> 15)) & 3u;
            else b = y;
            m |= b << (i * EPW);
        }
        if (!full) {
            const uint32_t act = j0 < count ? min(count - j0, (uint32_t)VEPL) : 0u;
            m &= act >= 32 ? 0xFFFFFFFFu : ((1u << act) - 1u);
        }
        if (W == 1) {
            reinterpret_cast<uint16_t*>(wbytes + g * GBYTES)[lane] = (uint16_t)m;
        } else if (W == 2) {
            wbytes[g * GBYTES + lane] = (uint8_t)m;
        } else {
            const uint32_t x = m | (__shfl_down_sync(0xffffffffu, m, 1) << 4);
            if ((lane & 1) == 0) wbytes[g * GBYTES + lane / 2] = (uint8_t)x;
        }
        const uint32_t gc = __reduce_add_sync(0xffffffffu, __popc(m));
        if (lane == 0) s_gcnt[g] = gc;
    }
    if (tid == kLpThreads - 32) {
        s_gnext = 0;
        // does the tile lie inside one node of this level?
        if (a.level == 0) {
            s_single = 1;
            s_p = 0;
        } else {
            const T* te = reinterpret_cast<const T*>(inb);
            const uint64_t p0 = (uint64_t)te[0] >> a.pshift;
            const uint64_t p1 = (uint64_t)te[count - 1] >> a.pshift;
            s_single = p0 == p1;
            s_p = p0;
        }
    }
    __syncthreads();

    // ---- phase 2 (every warp, no barrier): exclusive scan of the 64 group counts ----
    // lane l holds the prefixes of groups 2l and 2l+1
    uint32_t rp0, rp1, ones32;
    {
        const uint32_t c0 = 2 * lane < NG ? s_gcnt[2 * lane] : 0u, c1 = 2 * lane + 1 < NG ? s_gcnt[2 * lane + 1] : 0u;
        const uint32_t sum = c0 + c1;
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        rp0 = inc - sum;
        rp1 = rp0 + c0;
        ones32 = __shfl_sync(0xffffffffu, inc, 31);
        if (warp == 1) {
            if (2 * lane < NG) rpre[2 * lane] = rp0;
            if (2 * lane + 1 < NG) rpre[2 * lane + 1] = rp1;
            if (lane == 0) rpre[NG] = ones32;
        }
    }
    const uint32_t Z = count - ones32;  // zeros of the tile

    // ---- phase 3: look-back (warp 0) || level bits to global + partition into shared memory ----
    // The shared-memory image holds the tile's zeros at out[0, Z) and its ones at
    // out[Z, count), each in input order; it does not depend on the look-back.
    T* out = reinterpret_cast<T*>(outb);
    const uint32_t out_s = smem_addr(outb);
    const bool part = FOLD || a.dst != nullptr;  // the image is needed
    if (warp == 0 && a.tile_excl != nullptr) {
        // the ones before every tile are known (counted by the previous pass)
        if (lane == 0) {
            s_E = a.tile_excl[tile];
            s_EL1 = a.tile_excl[tile - tile % TPL1];
        }
    } else if (warp == 0) {
        const uint64_t ones = ones32;
        const uint64_t excl = lookback_warp(a.state, tile, ones, a.status, kSpinCap);
        // ones before the enclosing L1 block
        const uint32_t q = (uint32_t)(tile % TPL1);
        uint64_t sub = 0;
        if (q && lane < (int)q) sub = lb_agg(ld_relaxed_u64(a.state + tile - q + lane));
        sub = warp_sum_u64(sub);
        if (lane == 0) {
            s_E = excl;
            s_EL1 = excl - sub;
        }
    } else {
        const uint32_t tw = tid - 32;
        const uint32_t nw = (count + 63) / 64;
        const uint64_t* wsrc = reinterpret_cast<const uint64_t*>(wbytes);
        uint64_t* wdst = a.words + tile * (TE / 64);
        for (uint32_t i = tw; i < nw; i += kLpThreads - 32) wdst[i] = wsrc[i];
        if (tile == a.ntiles - 1) {
            const uint64_t first_pad = (a.size + 63) / 64;
            for (uint64_t i = first_pad + tw; i < a.words_alloc; i += kLpThreads - 32) a.words[i] = 0;
        }
    }
    if (part && a.tile_excl != nullptr) {
        // every warp partitions its own GPW groups, two at a time: one scan of
        // the lanes' one counts (16-bit halves) serves both groups
        const uint16_t* m16 = reinterpret_cast<const uint16_t*>(wbytes);
        // slots as shared byte addresses: the image sits first in shared
        // memory, so they fit the 16-bit halves of a pair
        const bool abs_ok = out_s + kTileBytes <= 65536u;
#pragma unroll 1
        for (int pr = 0; pr < GPW / 2; pr++) {
            const int g = warp * GPW + 2 * pr;
            uint32_t ma, mb;
            if (W == 1) {
                ma = m16[g * 32 + lane];
                mb = m16[(g + 1) * 32 + lane];
            } else if (W == 2) {
                ma = wbytes[g * GBYTES + lane];
                mb = wbytes[(g + 1) * GBYTES + lane];
            } else {
                ma = (wbytes[g * GBYTES + lane / 2] >> ((lane & 1) * 4)) & 0xFu;
                mb = (wbytes[(g + 1) * GBYTES + lane / 2] >> ((lane & 1) * 4)) & 0xFu;
            }
            const uint32_t c = __popc(ma) | (__popc(mb) << 16);
            uint32_t inc = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            const uint32_t ex = inc - c;
            {
                // the lane that starts a 64-bit word of level bits records the
                // ones before that word in its group (for the sample search)
                constexpr uint32_t LPW = 64 / VEPL;  // lanes per word
                constexpr uint32_t WPG = GE / 64;    // words per group
                if ((lane % LPW) == 0) {
                    s_wpre[g * WPG + lane / LPW] = ex & 0xFFFFu;
                    s_wpre[(g + 1) * WPG + lane / LPW] = ex >> 16;
                }
            }
            const uint32_t ga = __shfl_sync(0xffffffffu, rp0, g >> 1), gb = __shfl_sync(0xffffffffu, rp1, g >> 1);
            const uint32_t oba = ga + (ex & 0xFFFFu), obb = gb + (ex >> 16);
            const uint32_t ja = g * GE + lane * VEPL, jb = ja + GE;
            const uint4 Va = in4[g * 32 + lane], Vb = in4[(g + 1) * 32 + lane];
            if (full && abs_ok) {
                scatter_group<T, true, true>(out_s, Va, ma, out_s + W * (ja - oba), out_s + W * (Z + oba), ja, count, shift);
                scatter_group<T, true, true>(out_s, Vb, mb, out_s + W * (jb - obb), out_s + W * (Z + obb), jb, count, shift);
            } else if (full) {
                scatter_group<T, true>(out_s, Va, ma, ja - oba, Z + oba, ja, count, shift);
                scatter_group<T, true>(out_s, Vb, mb, jb - obb, Z + obb, jb, count, shift);
            } else {
                scatter_group<T, false>(out_s, Va, ma, ja - oba, Z + oba, ja, count, shift);
                scatter_group<T, false>(out_s, Vb, mb, jb - obb, Z + obb, jb, count, shift);
            }
        }
    } else if (part) {
        // groups are handed out dynamically; warp 0 joins once its look-back is done
#pragma unroll 1
        while (true) {
            uint32_t g = 0;
            if (lane == 0) g = atomicAdd(&s_gnext, 1u);
            g = __shfl_sync(0xffffffffu, g, 0);
            if (g >= (uint32_t)NG) break;
            const uint4 V = in4[g * 32 + lane];
            const uint32_t j0 = g * GE + lane * VEPL;
            uint32_t m;
            if (W == 1) m = reinterpret_cast<const uint16_t*>(wbytes + g * GBYTES)[lane];
            else if (W == 2) m = wbytes[g * GBYTES + lane];
            else m = (wbytes[g * GBYTES + lane / 2] >> ((lane & 1) * 4)) & 0xFu;
            // ones before this lane's elements: group prefix + warp exclusive scan
            const uint32_t c = __popc(m);
            uint32_t inc = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            const uint32_t gpre = __shfl_sync(0xffffffffu, (g & 1u) ? rp1 : rp0, g >> 1);
            const uint32_t ob = gpre + inc - c;
            if (full) scatter_group<T, true>(out_s, V, m, j0 - ob, Z + ob, j0, count, shift);
            else scatter_group<T, false>(out_s, V, m, j0 - ob, Z + ob, j0, count, shift);
        }
    }
    __syncthreads();

    const uint64_t E = s_E, EL1 = s_EL1, ones = ones32;
    const uint64_t zeros = Z;
    const uint64_t R0 = t0 - E;  // zeros before the tile

    // ---- phase 4: L1/L2 counters and select samples ----
    {
        const uint32_t nl2 = (count + 511) / 512;
        for (uint32_t b = tid; b < nl2; b += kLpThreads)
            a.l2[(t0 >> 9) + b] = (uint16_t)(E - EL1 + rpre[b * GPL2]);
        if (tid == 0) {
            if (tile % TPL1 == 0) a.l1[t0 >> 16] = E;
            if (tile == a.ntiles - 1) {
                const uint64_t end = t0 + count;
                if ((end & 511) == 0) {
                    if ((end & 65535) == 0) {
                        a.l1[end >> 16] = E + ones;
                        a.l2[end >> 9] = 0;
                    } else {
                        a.l2[end >> 9] = (uint16_t)(E + ones - EL1);
                    }
                }
            }
            if (tile == 0) {
                a.s0[0] = 0;
                a.s1[0] = 0;
            }
        }
        // one 64-bit word of the tile's bits per thread: a sample falls in the word
        // when the count of b-bits crosses a multiple of K there (at most once, K >= 256)
        const uint32_t kl = a.k_log2;
        constexpr uint32_t WPG = GE / 64;  // words per group
        const uint64_t* w64 = reinterpret_cast<const uint64_t*>(wbytes);
        for (uint32_t t = tid; t * 64 < count; t += kLpThreads) {
            const uint64_t x = w64[t];
            const uint32_t g = t / WPG;
            uint32_t pre = rpre[g];  // ones of the tile before word t
            if (part && a.tile_excl != nullptr) {
                pre += s_wpre[t];  // recorded by the partition
            } else {
                for (uint32_t k = g * WPG; k < t; k++) pre += __popcll(w64[k]);
            }
            const uint32_t nv = count - t * 64;
            const uint64_t valid = nv >= 64 ? ~0ull : ((1ull << nv) - 1ull);
            const uint64_t z = ~x & valid;
            const uint32_t c1 = __popcll(x), c0 = __popcll(z);
            // a multiple of K falls in the word iff the count before it, mod K,
            // overflows there (32-bit test; measured 0.716 -> 0.707 ms per u8 pass)
            const uint32_t km = (1u << kl) - 1u;
            const bool x1 = (((uint32_t)E + pre) & km) + c1 > km;
            const bool x0 = (((uint32_t)R0 + t * 64u - pre) & km) + c0 > km;
            const uint64_t g1 = E + pre, g0 = R0 + (uint64_t)t * 64 - pre;  // ones / zeros before the word
            const uint64_t base = t0 + (uint64_t)t * 64;
            if (x1) {
                const uint64_t m = (g1 + c1) >> kl;
                if (m < a.n_s1) a.s1[m] = base + select_in_word(x, (uint32_t)((m << kl) - g1));
            }
            if (x0) {
                const uint64_t m = (g0 + c0) >> kl;
                if (m < a.n_s0) a.s0[m] = base + select_in_word(z, (uint32_t)((m << kl) - g0));
            }
        }
    }

    if (!part) return used_mbar;

    const uint64_t lim = a.size_next;
    // While copying out, count the ones of level l + 1 per tile of T_{l+1}, so
    // that the next pass knows every tile's prefix without a look-back.
    const bool cnt_next = a.next_cnt != nullptr;
    const uint32_t nsh = a.shift_bit - 1;  // bit of level l + 1 (valid when cnt_next)
    auto next_ones = [&](uint32_t x) { return (uint32_t)__popc((x >> nsh) & LOWB); };
    // A node index comes from an element's code prefix, which the build keeps
    // below the level's node count; a tile whose prefix is not (a corrupted
    // T_l) sets WT_EBOUNDS and skips its write-out instead of reading past
    // the node table.
    if (s_single != 0 && s_p >= a.level_nodes) {
        if (tid == 0) set_status(a.status, kStBounds);
        return used_mbar;
    }

    if (FOLD) {
        // ---- phase 5b (the level before the last): level l+1's bits ----
        // The image holds this tile's part of T_{l+1} in order: the zeros go
        // to T_{l+1}[D0, D0 + Z), the ones to T_{l+1}[D1, D1 + ones).  Level
        // l+1's bit of each element goes to the same position of level l+1's
        // bitvector, so T_{l+1} itself is never written or read again.  First
        // the image's level-(l+1) bits, in image order, into the input
        // buffer (free since phase 3).
        uint64_t* b2 = reinterpret_cast<uint64_t*>(inb);
        const uint32_t nunits = (count * W + 15) / 16;  // 16-byte units of the image
        if (W == 4) {
            // two units (8 elements) per byte of bits
            for (uint32_t p = tid; 2 * p < nunits; p += kLpThreads) {
                const uint4 v0 = lds_u128(out_s + 32 * p), v1 = lds_u128(out_s + 32 * p + 16);
                const uint32_t mm = ((v0.x >> nsh) & 1u) | (((v0.y >> nsh) & 1u) << 1) | (((v0.z >> nsh) & 1u) << 2) |
                                    (((v0.w >> nsh) & 1u) << 3) | (((v1.x >> nsh) & 1u) << 4) |
                                    (((v1.y >> nsh) & 1u) << 5) | (((v1.z >> nsh) & 1u) << 6) | (((v1.w >> nsh) & 1u) << 7);
                reinterpret_cast<uint8_t*>(b2)[p] = (uint8_t)mm;
            }
        } else {
            for (uint32_t u = tid; u < nunits; u += kLpThreads) {
                const uint4 v = lds_u128(out_s + 16 * u);
                const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
                uint32_t mm = 0;
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const uint32_t y = (wv[i] >> nsh) & LOWB;
                    mm |= (W == 1 ? (y * 0x10204080u) >> 28 : (y | (y >> 15)) & 3u) << (i * EPW);
                }
                if (W == 1) reinterpret_cast<uint16_t*>(b2)[u] = (uint16_t)mm;
                else reinterpret_cast<uint8_t*>(b2)[u] = (uint8_t)mm;
            }
        }
        __syncthreads();
        uint64_t* w2 = a.words2;
        if (s_single != 0) {
            // Two runs of consecutive bits.  Each 64-bit word of level l+1
            // that a run touches is cut from two words of the image's bits by
            // a funnel shift; a word the run covers whole is stored, a word it
            // shares with another tile's run is OR-ed in (the words start zeroed).
            const NodeEntry* ne = a.nodes + s_p;
            const uint64_t D0 = __ldg(&ne->off0) + R0;
            const uint64_t D1 = __ldg(&ne->off1) + E;
            uint64_t T0r[2] = {0, 0};                   // first tile of T_{l+1} of each run
            uint32_t clo[2] = {0, 0}, chi[2] = {0, 0};  // per run: ones in its first tile / in the next
#pragma unroll
            for (int run = 0; run < 2; run++) {
                const uint64_t P = run ? D1 : D0;
                const uint64_t len64 = run ? ones : zeros;
                const uint32_t sr = run ? Z : 0u;  // the run's first bit in the image's bits
                if (P >= lim || len64 == 0) continue;
                const uint64_t len = umin64(len64, lim - P);
                T0r[run] = P / TE;
                const uint64_t g0 = P >> 6;
                const uint32_t nw = (uint32_t)(((P + len - 1) >> 6) - g0 + 1);
                for (uint32_t k = tid; k < nw; k += kLpThreads) {
                    const uint64_t wb = (g0 + k) * 64;  // level-(l+1) position of the word's bit 0
                    const int64_t sb = (int64_t)sr + (int64_t)wb - (int64_t)P;  // its bit in the image's bits
                    uint64_t bits;
                    if (sb >= 0) {
                        const uint32_t q = (uint32_t)(sb >> 6), r = (uint32_t)(sb & 63);
                        const uint64_t lo = b2[q];
                        bits = r ? (lo >> r) | (b2[q + 1] << (64 - r)) : lo;
                    } else {
                        bits = b2[0] << (uint32_t)(-sb);  // only the run's first word: -sb < 64
                    }
                    const uint32_t jlo = P > wb ? (uint32_t)(P - wb) : 0u;
                    const uint32_t jhi = P + len < wb + 64 ? (uint32_t)(P + len - wb) : 64u;
                    const uint64_t mask = (jhi == 64 ? ~0ull : ((1ull << jhi) - 1ull)) & (~0ull << jlo);
                    bits &= mask;
                    if (mask == ~0ull) w2[g0 + k] = bits;
                    else if (bits) atomicOr(reinterpret_cast<unsigned long long*>(w2 + g0 + k), (unsigned long long)bits);
                    if (cnt_next) {
                        // a 64-bit word never straddles a tile of T_{l+1}
                        const uint32_t c = (uint32_t)__popcll(bits);
                        if (wb / TE == T0r[run]) clo[run] += c;
                        else chi[run] += c;
                    }
                }
            }
            if (cnt_next) {
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const uint32_t c = __reduce_add_sync(0xffffffffu, (k & 1) ? chi[k >> 1] : clo[k >> 1]);
                    if (lane == 0 && c) atomicAdd(&s_nc[k], c);
                }
                __syncthreads();
                if (tid < 4 && s_nc[tid])
                    atomicAdd(a.next_cnt + ((tid >> 1) ? T0r[1] : T0r[0]) + (tid & 1), (unsigned long long)s_nc[tid]);
            }
        } else {
            // several nodes: every element finds its position from its node's offsets
            const uint32_t ps = a.pshift;
            bool bad_node = false;
            for (uint32_t i = tid; i < count; i += kLpThreads) {
                const T x = out[i];
                const bool one = i >= Z;
                const uint64_t nd = (uint64_t)x >> ps;
                bad_node |= nd >= a.level_nodes;
                const uint64_t Dx = nd < a.level_nodes
                                        ? (one ? __ldg(&a.nodes[nd].off1) + E + (i - Z) : __ldg(&a.nodes[nd].off0) + R0 + i)
                                        : lim;
                const uint32_t bit = Dx < lim ? ((uint32_t)x >> nsh) & 1u : 0u;
                if (bit) atomicOr(reinterpret_cast<unsigned long long*>(w2 + (Dx >> 6)), 1ull << (Dx & 63));
                if (cnt_next) {
                    const uint64_t tl = Dx / TE;
                    const uint32_t am = __activemask();
                    const uint32_t grp = __match_any_sync(am, tl);
                    const uint32_t c = __popc(__ballot_sync(am, bit) & grp);
                    if (lane == __ffs(grp) - 1 && c) atomicAdd(a.next_cnt + tl, (unsigned long long)c);
                }
            }
            if (bad_node) set_status(a.status, kStBounds);
        }
        return used_mbar;
    }

    // ---- phase 5: shared-memory image -> T_{l+1} ----
    T* dst = reinterpret_cast<T*>(a.dst);
    if (s_single != 0) {
        // two contiguous runs: zeros to off0 + R0, ones to off1 + E.  Global 4-byte
        // words are assembled from two shared words with a funnel shift.
        const NodeEntry* ne = a.nodes + s_p;
        const uint64_t D0 = __ldg(&ne->off0) + R0;
        const uint64_t D1 = __ldg(&ne->off1) + E;
        uint64_t T0r[2] = {0, 0};  // first tile of T_{l+1} of each run
        uint32_t clo[2] = {0, 0}, chi[2] = {0, 0};  // per run: in its first tile / in the next
#pragma unroll
        for (int run = 0; run < 2; run++) {
            const uint64_t D = run ? D1 : D0;
            uint64_t len64 = run ? ones : zeros;
            const uint32_t so = run ? Z : 0u;
            if (D >= lim || len64 == 0) continue;
            T0r[run] = D / TE;
            const uint64_t bnd = (T0r[run] + 1) * TE - D;  // elements of the run in its first tile
            const uint32_t len = (uint32_t)umin64(len64, lim - D);
            T* dr = dst + D;
            // element counts of the unaligned head, the 16-byte body and the tail
            const uint32_t mis = (uint32_t)(D * W) & 15u;
            const uint32_t head = min(len, mis ? (16u - mis) / W : 0u);
            const uint32_t nb16 = (len - head) * W / 16;
            const uint32_t tail0 = head + nb16 * (16 / W);
            if (tid < head) {
                const T x = out[so + tid];
                dr[tid] = x;
                if (cnt_next) {
                    const uint32_t c = next_ones((uint32_t)x);
                    if (tid < bnd) clo[run] += c;
                    else chi[run] += c;
                }
            }
            uint4* db = reinterpret_cast<uint4*>(dr + head);
            // the shared/global byte shift is the same for the whole run: every
            // global 16-byte unit is cut from two aligned shared 16-byte units
            const uint32_t sb0 = (so + head) * W;  // shared byte of the first body byte
            const uint32_t src0 = out_s + (sb0 & ~15u);
            const uint32_t q = (sb0 >> 2) & 3u, fs = (sb0 & 3u) * 8u;
            for (uint32_t i = tid; i < nb16; i += kLpThreads) {
                const uint4 v = shift16(lds_u128(src0 + 16 * i), lds_u128(src0 + 16 * i + 16), q, fs);
                db[i] = v;
                if (cnt_next) {
                    // a 16-byte unit of T_{l+1} never straddles one of its tiles
                    const uint32_t c = next_ones(v.x) + next_ones(v.y) + next_ones(v.z) + next_ones(v.w);
                    if (head + i * (16 / W) < bnd) clo[run] += c;
                    else chi[run] += c;
                }
            }
            for (uint32_t i = tail0 + tid; i < len; i += kLpThreads) {
                const T x = out[so + i];
                dr[i] = x;
                if (cnt_next) {
                    const uint32_t c = next_ones((uint32_t)x);
                    if (i < bnd) clo[run] += c;
                    else chi[run] += c;
                }
            }
        }
        if (cnt_next) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t c = __reduce_add_sync(0xffffffffu, (k & 1) ? chi[k >> 1] : clo[k >> 1]);
                if (lane == 0 && c) atomicAdd(&s_nc[k], c);
            }
            __syncthreads();
            if (tid < 4 && s_nc[tid])
                atomicAdd(a.next_cnt + ((tid >> 1) ? T0r[1] : T0r[0]) + (tid & 1), (unsigned long long)s_nc[tid]);
        }
    } else {
        // several nodes: every element finds its node's offsets from its own code
        const uint32_t ps = a.pshift;
        // ones of level l + 1 per tile of T_{l+1}: one atomic per tile per warp
        auto count_multi = [&](const T x, uint64_t Dx) {
            const uint32_t bit = Dx < lim ? ((uint32_t)x >> nsh) & 1u : 0u;
            const uint64_t tl = Dx / TE;
            const uint32_t am = __activemask();
            const uint32_t grp = __match_any_sync(am, tl);
            const uint32_t c = __popc(__ballot_sync(am, bit) & grp);
            if (lane == __ffs(grp) - 1 && c) atomicAdd(a.next_cnt + tl, (unsigned long long)c);
        };
        bool bad_node = false;
        for (uint32_t i = tid; i < zeros; i += kLpThreads) {
            const T x = out[i];
            const uint64_t nd = (uint64_t)x >> ps;
            bad_node |= nd >= a.level_nodes;
            const uint64_t Dx = nd < a.level_nodes ? __ldg(&a.nodes[nd].off0) + R0 + i : lim;
            if (Dx < lim) dst[Dx] = x;
            if (cnt_next) count_multi(x, Dx);
        }
        for (uint32_t i = tid; i < ones; i += kLpThreads) {
            const T x = out[Z + i];
            const uint64_t nd = (uint64_t)x >> ps;
            bad_node |= nd >= a.level_nodes;
            const uint64_t Dx = nd < a.level_nodes ? __ldg(&a.nodes[nd].off1) + E + i : lim;
            if (Dx < lim) dst[Dx] = x;
            if (cnt_next) count_multi(x, Dx);
        }
        if (bad_node) set_status(a.status, kStBounds);
    }
    return used_mbar;
}

// Single tree: one CTA per tile, tiles taken in order from a counter.  FOLD:
// the level before the last, which also writes the last level's bits.
template <typename T, bool ENCODE, bool FOLD>
__global__ void __launch_bounds__(kLpThreads, kLpBlocksPerSM)
    level_pass_kernel(const __grid_constant__ LevelPassArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint64_t s_tile;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_tile = atomicAdd(a.counter, 1u);
        mbar_init(&mbar, 1);
        mbar_fence_init();
    }
    if (ENCODE && a.ctab_n) {
        constexpr int W = sizeof(T);
        T* ctab = reinterpret_cast<T*>(smem + 2 * kTileBytes + 64 + kTileBytes / 8 / W + (64 + 1) * 4);
        for (uint32_t s = tid; s < a.ctab_n; s += kLpThreads) {
            uint32_t code = 0, len;
            if (s < a.cp.sigma) encode(a.cp, s, code, len);
            ctab[s] = (T)code;
        }
    }
    __syncthreads();
    if (s_tile >= a.ntiles) return;
    level_pass_tile<T, ENCODE, FOLD>(a, s_tile, smem, &mbar, 0);
}

// Many trees: a persistent grid walks the concatenation of every tree's tiles
// (tile_prefix[i] = tiles of trees before i), so each tree's tiles are taken in
// order and its look-back only waits on running CTAs.  Codes are computed
// arithmetically (no shared code table).
template <typename T, bool ENCODE>
__global__ void __launch_bounds__(kLpThreads, kLpBlocksPerSM)
    level_pass_batched_kernel(const LevelPassArgs* __restrict__ args, const uint64_t* __restrict__ tile_prefix,
                              uint32_t ntrees, unsigned long long* __restrict__ counter) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint64_t s_g;
    __shared__ uint32_t s_tree;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&mbar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    const uint64_t total = tile_prefix[ntrees];
    const uint32_t lane = tid & 31;
    uint32_t phase = 0;
    for (;;) {
        if (tid < 32) {
            // warp 0 takes the next tile and finds its tree: the last tree whose
            // first tile is <= g, by a 32-ary search (one ballot per round).
            // Invariant: tile_prefix[lo] <= g < tile_prefix[hi].
            uint64_t g = 0;
            if (lane == 0) g = atomicAdd(counter, 1ull);
            g = __shfl_sync(0xffffffffu, g, 0);
            if (lane == 0) s_g = g;
            if (g < total) {
                uint32_t lo = 0, hi = ntrees;
                while (hi - lo > 1) {
                    const uint32_t step = (hi - lo + 31) / 32;
                    const uint32_t idx = lo + lane * step;
                    const bool le = idx < hi && tile_prefix[idx] <= g;
                    const uint32_t m = __ballot_sync(0xffffffffu, le);  // lane 0 (idx = lo) is always set
                    lo += (31u - __clz(m)) * step;
                    hi = hi < lo + step ? hi : lo + step;
                }
                if (lane == 0) s_tree = lo;
            }
        }
        __syncthreads();
        const uint64_t g = s_g;
        if (g >= total) break;
        const uint32_t tr = s_tree;
        if (level_pass_tile<T, ENCODE>(args[tr], g - tile_prefix[tr], smem, &mbar, phase)) phase ^= 1u;
        __syncthreads();
    }
}

constexpr uint32_t kCodeTableBytes = 8192;

// dynamic shared memory: input tile, image, level bits, group prefixes, and the
// code table of level 0 (ctab_n codes, 0 when codes are computed)
// The last level's counters and samples when the pass before wrote its bits
// (phase 5b): one CTA per tile of T_{l+1} (kTileBytes / W bits, one 64-bit
// word per thread), the ones before each tile from the scan of the counts
// phase 5b gathered.  The same quantities as phase 4 of a level pass.
template <int W>
__global__ void __launch_bounds__(kLpThreads) level_support_kernel(const __grid_constant__ LevelPassArgs a) {
    constexpr uint32_t TE = kTileBytes / W;  // bits per tile
    constexpr uint32_t TPL1 = 65536 / TE;    // tiles per L1 block
    static_assert(TE / 64 <= (uint32_t)kLpThreads, "one word per thread");
    __shared__ uint32_t s_wsum[kLpThreads / 32];
    const uint64_t tile = blockIdx.x;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t t0 = tile * TE;
    const uint32_t count = (uint32_t)umin64(TE, a.size - t0);
    const uint32_t nw = (count + 63) / 64;
    const uint64_t E = a.tile_excl[tile], EL1 = a.tile_excl[tile - tile % TPL1];
    const uint64_t R0 = t0 - E;  // zeros before the tile
    const uint64_t x = tid < nw ? a.words[t0 / 64 + tid] : 0ull;
    const uint32_t c1 = (uint32_t)__popcll(x);
    uint32_t inc = c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= (uint32_t)o) inc += t;
    }
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    uint32_t before = 0, ones = 0;
#pragma unroll
    for (uint32_t w = 0; w < kLpThreads / 32; w++) {
        const uint32_t v = s_wsum[w];
        before += w < warp ? v : 0u;
        ones += v;
    }
    const uint32_t pre = before + inc - c1;  // ones of the tile before word tid
    if (tid < nw && (tid & 7) == 0) a.l2[(t0 >> 9) + tid / 8] = (uint16_t)(E - EL1 + pre);
    if (tid == 0) {
        if (tile % TPL1 == 0) a.l1[t0 >> 16] = E;
        if (tile == a.ntiles - 1) {
            const uint64_t end = t0 + count;
            if ((end & 511) == 0) {
                if ((end & 65535) == 0) {
                    a.l1[end >> 16] = E + ones;
                    a.l2[end >> 9] = 0;
                } else {
                    a.l2[end >> 9] = (uint16_t)(E + ones - EL1);
                }
            }
        }
        if (tile == 0) {
            a.s0[0] = 0;
            a.s1[0] = 0;
        }
    }
    if (tid < nw) {
        const uint32_t kl = a.k_log2;
        const uint32_t nv = count - tid * 64;
        const uint64_t valid = nv >= 64 ? ~0ull : ((1ull << nv) - 1ull);
        const uint64_t z = ~x & valid;
        const uint32_t c0 = (uint32_t)__popcll(z);
        const uint32_t km = (1u << kl) - 1u;
        const bool x1 = (((uint32_t)E + pre) & km) + c1 > km;
        const bool x0 = (((uint32_t)R0 + tid * 64u - pre) & km) + c0 > km;
        const uint64_t g1 = E + pre, g0 = R0 + (uint64_t)tid * 64 - pre;  // ones / zeros before the word
        const uint64_t base = t0 + (uint64_t)tid * 64;
        if (x1) {
            const uint64_t m = (g1 + c1) >> kl;
            if (m < a.n_s1) a.s1[m] = base + select_in_word(x, (uint32_t)((m << kl) - g1));
        }
        if (x0) {
            const uint64_t m = (g0 + c0) >> kl;
            if (m < a.n_s0) a.s0[m] = base + select_in_word(z, (uint32_t)((m << kl) - g0));
        }
    }
}

template <typename T>
static size_t level_pass_smem(uint32_t ctab_n) {
    constexpr int W = sizeof(T);
    return 2 * kTileBytes + 64 + kTileBytes / 8 / W + (64 + 1) * 4 + ((ctab_n * W + 15) & ~15u);
}

template <typename T, bool ENC, bool FOLD>
static cudaError_t launch_level_pass(const LevelPassArgs& a, cudaStream_t s) {
    static bool configured = false;
    const size_t sm = level_pass_smem<T>(ENC ? a.ctab_n : 0);
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(level_pass_kernel<T, ENC, FOLD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)level_pass_smem<T>(ENC ? kCodeTableBytes / sizeof(T) : 0));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    ProfScope ps(sizeof(T) == 1 ? "level_pass_u8" : (sizeof(T) == 2 ? "level_pass_u16" : "level_pass_u32"), s);
    level_pass_kernel<T, ENC, FOLD><<<(unsigned)a.ntiles, kLpThreads, sm, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_lp(const LevelPassArgs& a, bool enc, bool fold, cudaStream_t s) {
    if (fold) return enc ? launch_level_pass<T, true, true>(a, s) : launch_level_pass<T, false, true>(a, s);
    return enc ? launch_level_pass<T, true, false>(a, s) : launch_level_pass<T, false, false>(a, s);
}

template <int W>
static cudaError_t launch_level_support(const LevelPassArgs& a, cudaStream_t s) {
    ProfScope ps(W == 1 ? "level_pass_u8" : (W == 2 ? "level_pass_u16" : "level_pass_u32"), s);
    level_support_kernel<W><<<(unsigned)a.ntiles, kLpThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_hist(const void* S, uint64_t n, uint32_t sigma, unsigned long long* hist, uint32_t* status,
                               uint32_t m0, unsigned long long* tcnt, cudaStream_t s) {
    // Sub-histograms in shared memory.  Up to 512 bins, one per lane, bin-major
    // (every lane counts in its own bank, so a warp's atomics never conflict);
    // else as many copies as fit, their stride 1 mod 32 words.
    const uint32_t budget = 64 * 1024;  // bytes of shared memory for sub-histograms
    const uint32_t sbins = std::min<uint32_t>(sigma, budget / 4 - 1);
    uint32_t stride = ((sbins + 31) & ~31u) + 1;
    uint32_t copies = std::max<uint32_t>(1, std::min<uint32_t>(31, budget / (4 * stride)));
    if (sbins * 32 * 4 <= budget) {
        copies = 32;
        stride = sbins;
    }
    size_t sm = sizeof(T) == 1 ? 256 * 32 * 4 : (size_t)stride * copies * 4;
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(hist_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        configured = true;
    }
    int blocks = sm_count() * 3;
    ProfScope ps("histogram", s);
    hist_kernel<T><<<blocks, 512, sm, s>>>(reinterpret_cast<const T*>(S), n, sigma, sbins, stride, copies, hist, status,
                                           m0, tcnt);
    return cudaGetLastError();
}

// ===========================================================================
// host orchestration
// ===========================================================================

static uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// Wavelet matrix: the zeros of every level from C (symbols whose bit L-1-l is 0
// form runs [k 2^(b+1), k 2^(b+1) + 2^b) of the alphabet), one block per level;
// meta as for the tree (size n, zeros) and a one-entry "node" per level whose
// partition offsets send the zeros to [0, Z_l) and the ones to [Z_l, n).
__global__ void __launch_bounds__(256) matrix_meta_kernel(const uint64_t* __restrict__ C, uint32_t sigma, uint32_t L,
                                                          uint64_t n, uint64_t* __restrict__ meta,
                                                          NodeEntry* __restrict__ mnodes) {
    const uint32_t l = blockIdx.x, b = L - 1 - l;
    const uint64_t run = 1ull << b, period = run << 1;
    uint64_t z = 0;
    for (uint64_t k = threadIdx.x; k * period < sigma; k += blockDim.x) {
        const uint64_t a = k * period;
        z += C[umin64(sigma, a + run)] - C[a];
    }
    __shared__ uint64_t ws[8];
    z = warp_sum_u64(z);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = z;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t zz = 0;
        for (int k = 0; k < 8; k++) zz += ws[k];
        meta[2 * l] = n;
        meta[2 * l + 1] = zz;
        NodeEntry e = {0, 0, 0, zz};
        mnodes[l] = e;
    }
}

wt_status build_tree(const void* d_symbols, uint64_t n, uint32_t sigma, uint32_t w, uint32_t sample_k, cudaStream_t s,
                     wt_tree_s* t, uint32_t layout, const void* h_src, cudaStream_t cs) {
    const bool matrix = layout == WT_LAYOUT_MATRIX;
    CodeParams cp = make_code_params(sigma);
    if (matrix) {  // plain L-bit codes: encode gives code = symbol, length L
        cp.pow2 = true;
        cp.r = 1;
        cp.e[0] = cp.L;
        cp.P[0] = 0;
        cp.P[1] = 1ull << cp.L;
    }
    const uint32_t L = cp.L;
    t->desc.layout = layout;
    uint32_t k_log2 = 0;
    while ((1u << k_log2) < sample_k) k_log2++;

    t->desc.cp = cp;
    t->desc.n = n;
    t->desc.k_log2 = k_log2;
    t->symbol_bytes = w;
    t->sample_k = sample_k;

    // ---- header memory: status, C, node table, meta ----
    const uint64_t nslots = matrix ? L : (L ? ((1ull << L) - 1) : 0);  // the matrix: one entry per level
    size_t off_status = 0;
    size_t off_C = 256;
    size_t off_nodes = align_up(off_C + (sigma + 1ull) * 8, 256);
    size_t hdr = align_up(off_nodes + std::max<uint64_t>(nslots, 1) * sizeof(NodeEntry), 256);
    const wt_allocator* A = tree_alloc(t);
    WT_CUDA_TRY(dev_alloc(&t->hdr_mem, hdr, s, A));
    t->hdr_bytes = hdr;
    uint8_t* H = reinterpret_cast<uint8_t*>(t->hdr_mem);
    t->desc.status = reinterpret_cast<uint32_t*>(H + off_status);
    uint64_t* C = reinterpret_cast<uint64_t*>(H + off_C);
    NodeEntry* nodes = reinterpret_cast<NodeEntry*>(H + off_nodes);
    t->desc.C = C;
    t->desc.nodes = nodes;

    // ---- scratch for steps 1-3 ----
    const uint64_t scan_n = std::max<uint64_t>(sigma, nslots);
    const uint64_t scan_tmp = 2 * ((scan_n + kScanChunk - 1) / kScanChunk + 2);
    size_t s_hist = 0;
    size_t s_left = align_up(s_hist + (uint64_t)sigma * 8, 256);
    size_t s_excl = align_up(s_left + std::max<uint64_t>(nslots, 1) * 8, 256);
    size_t s_tmp = align_up(s_excl + (nslots + 1) * 8, 256);
    size_t s_meta = align_up(s_tmp + scan_tmp * 8, 256);
    // ones of level 0 per 16 KiB tile of S, counted by the histogram
    const uint64_t tiles0 = (n * w + kTileBytes - 1) / kTileBytes;
    size_t s_tcnt = align_up(s_meta + 2 * kMaxLevels * 8, 256);
    size_t s_end = align_up(s_tcnt + std::max<uint64_t>(tiles0, 1) * 8, 256);
    void* scratch = nullptr;
    WT_CUDA_TRY(dev_alloc(&scratch, s_end, s, A));
    uint8_t* X = reinterpret_cast<uint8_t*>(scratch);
    uint64_t* hist = reinterpret_cast<uint64_t*>(X + s_hist);
    uint64_t* left = reinterpret_cast<uint64_t*>(X + s_left);
    uint64_t* excl = reinterpret_cast<uint64_t*>(X + s_excl);
    uint64_t* tmp = reinterpret_cast<uint64_t*>(X + s_tmp);
    uint64_t* meta = reinterpret_cast<uint64_t*>(X + s_meta);
    unsigned long long* tcnt0 = reinterpret_cast<unsigned long long*>(X + s_tcnt);
    // m0: the first symbol whose code starts with a 1 (codes grow with the symbol)
    uint32_t m0 = sigma;
    if (L) {
        uint32_t lo = 0, hi = sigma;
        while (lo < hi) {
            const uint32_t mid = lo + (hi - lo) / 2;
            uint32_t code, len;
            encode(cp, mid, code, len);
            if ((code >> (L - 1)) & 1u) hi = mid;
            else lo = mid + 1;
        }
        m0 = lo;
    }

    WT_CUDA_TRY(cudaMemsetAsync(t->hdr_mem, 0, hdr, s));
    WT_CUDA_TRY(cudaMemsetAsync(hist, 0, (uint64_t)sigma * 8, s));
    WT_CUDA_TRY(cudaMemsetAsync(tcnt0, 0, std::max<uint64_t>(tiles0, 1) * 8, s));

    // 1. histogram (with a host source: chunk by chunk as the chunks arrive, the
    // copy of chunk k+1 on a copy stream overlapping the histogram of chunk k)
    if (n) {
        unsigned long long* hh = (unsigned long long*)hist;
        auto hist_part = [&](uint64_t off, uint64_t len) {
            const void* src = static_cast<const uint8_t*>(d_symbols) + off * w;
            unsigned long long* tc = L ? tcnt0 + off * w / kTileBytes : nullptr;  // off is a whole number of tiles
            return w == 1   ? launch_hist<uint8_t>(src, len, sigma, hh, t->desc.status, m0, tc, s)
                   : w == 2 ? launch_hist<uint16_t>(src, len, sigma, hh, t->desc.status, m0, tc, s)
                            : launch_hist<uint32_t>(src, len, sigma, hh, t->desc.status, m0, tc, s);
        };
        cudaError_t e = cudaSuccess;
        if (h_src) {
            const uint64_t chunk = (64ull << 20) / w;  // 64 MiB: a whole number of 16 KiB tiles
            for (uint64_t off = 0; off < n && e == cudaSuccess; off += chunk) {
                const uint64_t len = std::min(chunk, n - off);
                cudaEvent_t ev = nullptr;
                e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(static_cast<uint8_t*>(const_cast<void*>(d_symbols)) + off * w,
                                        static_cast<const uint8_t*>(h_src) + off * w, len * w,
                                        cudaMemcpyHostToDevice, cs);
                if (e == cudaSuccess) e = cudaEventRecord(ev, cs);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
                if (ev) cudaEventDestroy(ev);
                if (e == cudaSuccess) e = hist_part(off, len);
            }
        } else {
            e = hist_part(0, n);
        }
        if (e != cudaSuccess) { dev_free(scratch, s, A); return WT_ECUDA; }
    }
    // 2. C
    device_exclusive_scan(hist, C, sigma, tmp, s);
    // 3. nodes + meta
    if (L && matrix) {
        ProfScope ps("meta", s);
        matrix_meta_kernel<<<L, 256, 0, s>>>(C, sigma, L, n, meta, nodes);
    } else if (L) {
        {
            ProfScope ps("node_start", s);
            node_start_kernel<<<(unsigned)((nslots + 255) / 256), 256, 0, s>>>(cp, C, nodes, left, nslots);
        }
        device_exclusive_scan(left, excl, nslots, tmp, s);
        {
            ProfScope ps("node_finish", s);
            node_finish_kernel<<<(unsigned)((nslots + 255) / 256), 256, 0, s>>>(nodes, left, excl, nslots);
        }
        MetaArgs ma;
        for (uint32_t l = 0; l < L; l++) {
            // first segment whose code length is <= l (lengths never increase with the symbol)
            uint64_t s0 = sigma;
            for (uint32_t i = 0; i < cp.r; i++) {
                uint32_t len = (i + 1 < cp.r || cp.pow2) ? (cp.pow2 ? cp.L : i + 1 + cp.e[i]) : (cp.r - 1 + cp.e[i]);
                if (len <= l) { s0 = cp.P[i]; break; }
            }
            ma.s0[l] = s0;
        }
        ProfScope ps("meta", s);
        meta_kernel<<<1, 32, 0, s>>>(ma, L, C, excl, meta);
    }
    WT_CUDA_TRY(cudaGetLastError());
    uint64_t hmeta[2 * kMaxLevels] = {0};
    uint32_t hstatus = 0;
    if (L) WT_CUDA_TRY(cudaMemcpyAsync(hmeta, meta, 2 * L * 8, cudaMemcpyDeviceToHost, s));
    WT_CUDA_TRY(cudaMemcpyAsync(&hstatus, t->desc.status, 4, cudaMemcpyDeviceToHost, s));
    WT_CUDA_TRY(cudaStreamSynchronize(s));
    if (hstatus & kStSymbol) {
        dev_free(scratch, s, A);
        return WT_ESYMBOL;
    }

    // ---- level memory ----
    struct Lay { size_t words, l1, l2, s0, s1; uint64_t walloc; };
    std::vector<Lay> lay(L);
    size_t off = 0;
    for (uint32_t l = 0; l < L; l++) {
        const uint64_t size = hmeta[2 * l], zeros = hmeta[2 * l + 1], ones = size - zeros;
        t->level_size[l] = size;
        t->level_ones[l] = ones;
        Lay& y = lay[l];
        y.walloc = align_up((size + 63) / 64 + 16, 16);
        y.words = off;
        off = align_up(off + y.walloc * 8, 256);
        y.l1 = off;
        off = align_up(off + (size / kL1Bits + 1) * 8, 256);
        y.l2 = off;
        off = align_up(off + (size / kL2Bits + 1) * 2, 256);
        y.s0 = off;
        off = align_up(off + ((zeros >> k_log2) + 1) * 8, 256);
        y.s1 = off;
        off = align_up(off + ((ones >> k_log2) + 1) * 8, 256);
    }
    t->lvl_bytes = std::max<size_t>(off, 256);
    if (dev_alloc(&t->lvl_mem, t->lvl_bytes, s, A) != cudaSuccess) {
        dev_free(scratch, s, A);
        return WT_ENOMEM;
    }
    uint8_t* M = reinterpret_cast<uint8_t*>(t->lvl_mem);
    for (uint32_t l = 0; l < L; l++) {
        LevelDesc& d = t->desc.lv[l];
        d.words = reinterpret_cast<uint64_t*>(M + lay[l].words);
        d.l1 = reinterpret_cast<uint64_t*>(M + lay[l].l1);
        d.l2 = reinterpret_cast<uint16_t*>(M + lay[l].l2);
        d.s0 = reinterpret_cast<uint64_t*>(M + lay[l].s0);
        d.s1 = reinterpret_cast<uint64_t*>(M + lay[l].s1);
        d.size = t->level_size[l];
        d.ones = t->level_ones[l];
        d.status = t->desc.status;
    }

    // ---- level passes ----
    if (L && n) {
        const uint64_t te = kTileBytes / w;
        const uint64_t max_tiles = (n + te - 1) / te;
        const uint64_t tbytes = align_up(n * w, 256);
        const size_t b_state = align_up(max_tiles * 8, 256);
        // per-tile ones of the next level (two, alternating), their exclusive scan, scan scratch
        const size_t b_cnt = b_state, b_excl = align_up((max_tiles + 1) * 8, 256);
        const size_t b_stmp = align_up(2 * ((max_tiles + kScanChunk - 1) / kScanChunk + 2) * 8, 256);
        void* work = nullptr;
        const size_t work_bytes = 2 * tbytes + b_state + 256 + 2 * b_cnt + b_excl + b_stmp;
        if (dev_alloc(&work, work_bytes, s, A) != cudaSuccess) {
            dev_free(scratch, s, A);
            return WT_ENOMEM;
        }
        uint8_t* Wm = reinterpret_cast<uint8_t*>(work);
        void* buf[2] = {Wm, Wm + tbytes};
        uint64_t* state = reinterpret_cast<uint64_t*>(Wm + 2 * tbytes);
        uint32_t* counters = reinterpret_cast<uint32_t*>(Wm + 2 * tbytes + b_state);
        unsigned long long* ncnt[2];
        ncnt[0] = reinterpret_cast<unsigned long long*>(Wm + 2 * tbytes + b_state + 256);
        ncnt[1] = reinterpret_cast<unsigned long long*>(Wm + 2 * tbytes + b_state + 256 + b_cnt);
        uint64_t* texcl = reinterpret_cast<uint64_t*>(Wm + 2 * tbytes + b_state + 256 + 2 * b_cnt);
        uint64_t* stmp = reinterpret_cast<uint64_t*>(Wm + 2 * tbytes + b_state + 256 + 2 * b_cnt + b_excl);
        WT_CUDA_TRY(cudaMemsetAsync(counters, 0, 256, s));
        // texcl holds the tile prefixes of the current level; level 0's come from the histogram
        device_exclusive_scan(reinterpret_cast<const uint64_t*>(tcnt0), texcl, tiles0, stmp, s, "tile_scan");
        bool have_excl = true;
        for (uint32_t l = 0; l < L; l++) {
            const uint64_t size = t->level_size[l];
            if (size == 0) continue;
            LevelPassArgs a;
            memset(&a, 0, sizeof(a));
            // The level before the last also writes the last level's bits
            // (phase 5b) instead of T_{L-1}; a small kernel then adds that
            // level's counters and samples.  Only where its nodes average 16
            // tiles or more: a tile that spans nodes sets its bits one atomic
            // at a time (on σ = 2^20 or 65536 trees that made the build
            // slower, 13.18 -> 13.43 and 21.49 -> 21.93 ms).
            const uint64_t nodes_l = matrix ? 1ull : (1ull << l);
            const bool fold = l + 2 == L && t->level_size[l + 1] > 0 && have_excl &&
                              nodes_l * te * 16 <= size;
            a.src = l == 0 ? d_symbols : buf[(l - 1) & 1];
            a.dst = (l + 1 < L && !fold) ? buf[l & 1] : nullptr;
            a.size = size;
            a.size_next = (l + 1 < L) ? t->level_size[l + 1] : 0;
            a.ntiles = (size + te - 1) / te;
            a.words_alloc = lay[l].walloc;
            a.words = reinterpret_cast<uint64_t*>(M + lay[l].words);
            a.l1 = reinterpret_cast<uint64_t*>(M + lay[l].l1);
            a.l2 = reinterpret_cast<uint16_t*>(M + lay[l].l2);
            a.s0 = reinterpret_cast<uint64_t*>(M + lay[l].s0);
            a.s1 = reinterpret_cast<uint64_t*>(M + lay[l].s1);
            a.n_s0 = ((size - t->level_ones[l]) >> k_log2) + 1;
            a.n_s1 = (t->level_ones[l] >> k_log2) + 1;
            a.nodes = matrix ? nodes + l : nodes + ((1ull << l) - 1);
            a.state = state;
            a.counter = counters + l;
            a.status = t->desc.status;
            a.level = l;
            a.shift_bit = L - 1 - l;
            a.pshift = matrix ? 32 : L - l;  // the matrix: every tile lies in the level's one node
            a.level_nodes = matrix ? 1 : (1ull << l);
            a.k_log2 = k_log2;
            a.cp = cp;
            // level 0 re-encodes bytes of a small alphabet with few segments
            // arithmetically (measured faster than the code table), others
            // through a code table in shared memory when it fits
            a.swar_codes = (w == 1 && !cp.pow2 && sigma <= 128 && cp.r <= 3) ? 1u : 0u;
            a.ctab_n = a.swar_codes ? 0u : w == 1 ? 256u : ((uint64_t)sigma * w <= kCodeTableBytes) ? sigma : 0;
            // Tile prefixes: from the counts the previous pass gathered, else by look-back.
            if (have_excl) a.tile_excl = texcl;
            else WT_CUDA_TRY(cudaMemsetAsync(state, 0, a.ntiles * 8, s));
            const uint64_t ntiles_next = (a.size_next + te - 1) / te;
            if ((a.dst != nullptr || fold) && ntiles_next) {
                a.next_cnt = ncnt[l & 1];
                WT_CUDA_TRY(cudaMemsetAsync(a.next_cnt, 0, ntiles_next * 8, s));
            }
            if (fold) {
                a.words2 = reinterpret_cast<uint64_t*>(M + lay[l + 1].words);
                WT_CUDA_TRY(cudaMemsetAsync(a.words2, 0, lay[l + 1].walloc * 8, s));
            }
            const bool enc = (l == 0) && !cp.pow2;
            cudaError_t e;
            if (w == 1) e = launch_lp<uint8_t>(a, enc, fold, s);
            else if (w == 2) e = launch_lp<uint16_t>(a, enc, fold, s);
            else e = launch_lp<uint32_t>(a, enc, fold, s);
            if (e != cudaSuccess) {
                dev_free(work, s, A);
                dev_free(scratch, s, A);
                return WT_ECUDA;
            }
            have_excl = a.next_cnt != nullptr;
            if (have_excl)
                device_exclusive_scan(reinterpret_cast<const uint64_t*>(a.next_cnt), texcl, ntiles_next, stmp, s,
                                      "tile_scan");
            if (fold) {
                // the last level: counters and samples from its bits
                const uint32_t ll = l + 1;
                const uint64_t sz = t->level_size[ll];
                LevelPassArgs b;
                memset(&b, 0, sizeof(b));
                b.size = sz;
                b.ntiles = ntiles_next;
                b.words = reinterpret_cast<uint64_t*>(M + lay[ll].words);
                b.l1 = reinterpret_cast<uint64_t*>(M + lay[ll].l1);
                b.l2 = reinterpret_cast<uint16_t*>(M + lay[ll].l2);
                b.s0 = reinterpret_cast<uint64_t*>(M + lay[ll].s0);
                b.s1 = reinterpret_cast<uint64_t*>(M + lay[ll].s1);
                b.n_s0 = ((sz - t->level_ones[ll]) >> k_log2) + 1;
                b.n_s1 = (t->level_ones[ll] >> k_log2) + 1;
                b.tile_excl = texcl;
                b.status = t->desc.status;
                b.k_log2 = k_log2;
                const cudaError_t e2 = w == 1   ? launch_level_support<1>(b, s)
                                       : w == 2 ? launch_level_support<2>(b, s)
                                                : launch_level_support<4>(b, s);
                if (e2 != cudaSuccess) {
                    dev_free(work, s, A);
                    dev_free(scratch, s, A);
                    return WT_ECUDA;
                }
                break;
            }
        }
        dev_free(work, s, A);
    } else {
        // empty levels still need their first counter / sample entries
        for (uint32_t l = 0; l < L; l++) {
            WT_CUDA_TRY(cudaMemsetAsync(M + lay[l].words, 0, lay[l].walloc * 8, s));
            WT_CUDA_TRY(cudaMemsetAsync(M + lay[l].l1, 0, 8, s));
            WT_CUDA_TRY(cudaMemsetAsync(M + lay[l].l2, 0, 2, s));
            WT_CUDA_TRY(cudaMemsetAsync(M + lay[l].s0, 0, 8, s));
            WT_CUDA_TRY(cudaMemsetAsync(M + lay[l].s1, 0, 8, s));
        }
    }
    dev_free(scratch, s, A);
    return WT_OK;
}

// ===========================================================================
// batches of trees: the same pipeline for many trees, with no host round trip
// (every size the host would read back is computed on the device), so the
// whole sequence can be captured in one CUDA graph
// ===========================================================================

uint64_t batch_tile_elems(uint32_t w) { return (uint64_t)kTileBytes / w; }

__device__ __forceinline__ uint32_t find_tree(const uint64_t* prefix, uint32_t ntrees, uint64_t g) {
    uint32_t lo = 0, hi = ntrees - 1;  // last tree whose first item is <= g
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One CTA per chunk of one tree's symbols (batch_chunk(sigma) of them).  The
// counts go to 32-bit bins in shared memory, kBatchSmemBins at a time: an
// alphabet of up to that many bins takes one pass over the chunk, a larger
// one takes one pass per window of bins (the chunk is re-read from L2), and
// every nonzero bin is added once per window to the tree's histogram.
template <typename T>
__global__ void __launch_bounds__(512) batch_hist_kernel(const BatchTreeInfo* __restrict__ info,
                                                         const uint64_t* __restrict__ chunk_prefix, uint32_t ntrees) {
    extern __shared__ uint32_t sh[];  // kBatchSmemBins
    __shared__ uint32_t s_tree;
    const uint64_t g = blockIdx.x;
    if (threadIdx.x == 0) s_tree = find_tree(chunk_prefix, ntrees, g);
    __syncthreads();
    const BatchTreeInfo& ti = info[s_tree];
    const uint32_t sigma = ti.sigma;
    const uint64_t chunk = batch_chunk(sigma);
    const uint64_t c0 = (g - chunk_prefix[s_tree]) * chunk;
    const uint64_t c1 = umin64(ti.n, c0 + chunk);
    const T* S = reinterpret_cast<const T*>(ti.sym);
    unsigned long long* hist = reinterpret_cast<unsigned long long*>(ti.hist);
    constexpr uint32_t V = 16 / sizeof(T);
    // c0 is a multiple of the chunk, so S + c0 is 16-byte aligned like S
    const uint64_t nvec = (c1 - c0) / V;
    const uint4* S4 = reinterpret_cast<const uint4*>(S + c0);
    bool bad = false;
    for (uint32_t base = 0; base < sigma; base += kBatchSmemBins) {
        const uint32_t nb = sigma - base < kBatchSmemBins ? sigma - base : kBatchSmemBins;
        for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0;
        __syncthreads();
        for (uint64_t v = threadIdx.x; v < nvec; v += blockDim.x) {
            const uint4 x = __ldg(S4 + v);
            const T* e = reinterpret_cast<const T*>(&x);
#pragma unroll
            for (uint32_t k = 0; k < V; k++) {
                const uint32_t s = (uint32_t)e[k];
                if (s >= sigma) bad = true;
                else if (s - base < nb) atomicAdd(sh + (s - base), 1u);
            }
        }
        for (uint64_t j = c0 + nvec * V + threadIdx.x; j < c1; j += blockDim.x) {
            const uint32_t s = (uint32_t)S[j];
            if (s >= sigma) bad = true;
            else if (s - base < nb) atomicAdd(sh + (s - base), 1u);
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x)
            if (sh[i]) atomicAdd(hist + base + i, (unsigned long long)sh[i]);
        __syncthreads();
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(ti.status, kStSymbol);
}

// one CTA per tree: C = exclusive scan of the histogram
__global__ void __launch_bounds__(kScanThreads) batch_C_kernel(const BatchTreeInfo* __restrict__ info) {
    const BatchTreeInfo& ti = info[blockIdx.x];
    uint64_t carry = 0;
    for (uint64_t base = 0; base < ti.sigma; base += kScanChunk) {
        const uint64_t c = umin64((uint64_t)kScanChunk, ti.sigma - base);
        carry += block_scan_chunk(ti.hist + base, ti.C + base, c, carry);
    }
    if (threadIdx.x == 0) ti.C[ti.sigma] = carry;
}

// one thread per node slot of every tree
__global__ void batch_node_start_kernel(const BatchTreeInfo* __restrict__ info, const TreeDesc* __restrict__ desc,
                                        const uint64_t* __restrict__ slot_prefix, uint32_t ntrees, uint64_t total) {
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const uint32_t tr = find_tree(slot_prefix, ntrees, g);
    const BatchTreeInfo& ti = info[tr];
    const uint64_t slot = g - slot_prefix[tr];
    const uint32_t l = 63u - (uint32_t)__clzll((long long)(slot + 1));
    const uint64_t p = slot + 1 - (1ull << l);
    uint64_t a = 0;
    const uint64_t wd = node_info(desc[tr].cp, l, p, a);
    NodeEntry e = {0, 0, 0, 0};
    uint64_t lf = 0;
    if (wd >= 2) {
        e.start = ti.C[a];
        lf = ti.C[node_mid(a, wd)] - e.start;
    }
    ti.nodes[slot] = e;
    ti.left[slot] = lf;
}

// one CTA per tree: exclusive scan of the left-child sizes over the tree's slots
__global__ void __launch_bounds__(kScanThreads) batch_left_scan_kernel(const BatchTreeInfo* __restrict__ info) {
    const BatchTreeInfo& ti = info[blockIdx.x];
    uint64_t carry = 0;
    for (uint64_t base = 0; base < ti.nslots; base += kScanChunk) {
        const uint64_t c = umin64((uint64_t)kScanChunk, ti.nslots - base);
        carry += block_scan_chunk(ti.left + base, ti.excl + base, c, carry);
    }
    if (threadIdx.x == 0) ti.excl[ti.nslots] = carry;
}

__global__ void batch_node_finish_kernel(const BatchTreeInfo* __restrict__ info,
                                         const uint64_t* __restrict__ slot_prefix, uint32_t ntrees, uint64_t total) {
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const uint32_t tr = find_tree(slot_prefix, ntrees, g);
    const BatchTreeInfo& ti = info[tr];
    const uint64_t slot = g - slot_prefix[tr];
    const uint32_t l = 63u - (uint32_t)__clzll((long long)(slot + 1));
    NodeEntry e = ti.nodes[slot];
    const uint64_t r0 = ti.excl[slot] - ti.excl[(1ull << l) - 1];
    e.r0 = r0;
    e.off0 = e.start - r0;
    e.off1 = ti.left[slot] + r0;
    ti.nodes[slot] = e;
}

// one thread per (tree, level): level sizes and ones into the tree descriptors
// and the level-pass arguments; tiles per level
__global__ void batch_meta_kernel(const BatchTreeInfo* __restrict__ info, TreeDesc* __restrict__ desc,
                                  LevelPassArgs* __restrict__ lpa, uint64_t* __restrict__ tiles, uint32_t ntrees,
                                  uint32_t maxL, uint64_t te, uint32_t kl) {
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (uint64_t)ntrees * maxL) return;
    const uint32_t tr = (uint32_t)(g % ntrees), l = (uint32_t)(g / ntrees);
    const BatchTreeInfo& ti = info[tr];
    LevelPassArgs& a = lpa[(uint64_t)l * ntrees + tr];
    if (l >= ti.L || ti.n == 0) {
        a.ntiles = 0;
        tiles[(uint64_t)l * ntrees + tr] = 0;
        if (l < ti.L) {
            desc[tr].lv[l].size = 0;
            desc[tr].lv[l].ones = 0;
        }
        return;
    }
    const uint64_t size = ti.C[ti.s0[l]];
    const uint64_t zeros = ti.excl[(2ull << l) - 1] - ti.excl[(1ull << l) - 1];
    const uint64_t ones = size - zeros;
    desc[tr].lv[l].size = size;
    desc[tr].lv[l].ones = ones;
    a.size = size;
    a.size_next = (l + 1 < ti.L) ? ti.C[ti.s0[l + 1]] : 0;
    a.ntiles = (size + te - 1) / te;
    a.n_s0 = (zeros >> kl) + 1;
    a.n_s1 = (ones >> kl) + 1;
    tiles[(uint64_t)l * ntrees + tr] = a.ntiles;
}

// one CTA per level: exclusive scan of the trees' tile counts
__global__ void __launch_bounds__(kScanThreads) batch_tile_scan_kernel(const uint64_t* __restrict__ tiles,
                                                                       uint64_t* __restrict__ prefix,
                                                                       uint32_t ntrees) {
    const uint64_t* in = tiles + (uint64_t)blockIdx.x * ntrees;
    uint64_t* out = prefix + (uint64_t)blockIdx.x * (ntrees + 1);
    uint64_t carry = 0;
    for (uint64_t base = 0; base < ntrees; base += kScanChunk) {
        const uint64_t c = umin64((uint64_t)kScanChunk, ntrees - base);
        carry += block_scan_chunk(in + base, out + base, c, carry);
    }
    if (threadIdx.x == 0) out[ntrees] = carry;
}

template <typename T, bool ENC>
static cudaError_t launch_level_pass_batched(const BatchDev& b, uint32_t l, cudaStream_t s) {
    static bool configured = false;
    const size_t sm = level_pass_smem<T>(0);
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(level_pass_batched_kernel<T, ENC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int grid = sm_count() * (int)((b.lp_ctas >= 1 && b.lp_ctas <= (uint32_t)kLpBlocksPerSM) ? b.lp_ctas
                                                                                                 : kLpBlocksPerSM);
    level_pass_batched_kernel<T, ENC><<<grid, kLpThreads, sm, s>>>(b.lpa + (uint64_t)l * b.ntrees,
                                                                   b.tile_prefix + (uint64_t)l * (b.ntrees + 1),
                                                                   b.ntrees, b.counters + l);
    return cudaGetLastError();
}

wt_status enqueue_batch_build(const BatchDev& b, cudaStream_t s, uint32_t* kernels) {
    uint32_t nk = 0;
    WT_CUDA_TRY(cudaMemsetAsync(b.hist_pool, 0, b.hist_bytes, s));
    WT_CUDA_TRY(cudaMemsetAsync(b.status_pool, 0, (size_t)b.ntrees * 4, s));
    WT_CUDA_TRY(cudaMemsetAsync(b.counters, 0, (size_t)b.maxL * 8, s));
    if (b.total_chunks) {
        nk++;
        const size_t hsm = (size_t)kBatchSmemBins * 4;
        static bool hcfg = false;
        if (!hcfg) {
            cudaFuncSetAttribute(batch_hist_kernel<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
            cudaFuncSetAttribute(batch_hist_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
            cudaFuncSetAttribute(batch_hist_kernel<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
            hcfg = true;
        }
        if (b.w == 1) batch_hist_kernel<uint8_t><<<(unsigned)b.total_chunks, 512, hsm, s>>>(b.info, b.chunk_prefix, b.ntrees);
        else if (b.w == 2) batch_hist_kernel<uint16_t><<<(unsigned)b.total_chunks, 512, hsm, s>>>(b.info, b.chunk_prefix, b.ntrees);
        else batch_hist_kernel<uint32_t><<<(unsigned)b.total_chunks, 512, hsm, s>>>(b.info, b.chunk_prefix, b.ntrees);
    }
    batch_C_kernel<<<b.ntrees, kScanThreads, 0, s>>>(b.info);
    nk++;
    if (b.total_slots) {
        nk += 3;
        batch_node_start_kernel<<<(unsigned)((b.total_slots + 255) / 256), 256, 0, s>>>(b.info, b.desc, b.slot_prefix,
                                                                                       b.ntrees, b.total_slots);
        batch_left_scan_kernel<<<b.ntrees, kScanThreads, 0, s>>>(b.info);
        batch_node_finish_kernel<<<(unsigned)((b.total_slots + 255) / 256), 256, 0, s>>>(b.info, b.slot_prefix,
                                                                                        b.ntrees, b.total_slots);
    }
    if (b.maxL) {
        const uint64_t te = batch_tile_elems(b.w);
        const uint64_t nm = (uint64_t)b.ntrees * b.maxL;
        nk += 2;
        batch_meta_kernel<<<(unsigned)((nm + 255) / 256), 256, 0, s>>>(b.info, b.desc, b.lpa, b.tiles, b.ntrees, b.maxL,
                                                                       te, b.k_log2);
        batch_tile_scan_kernel<<<b.maxL, kScanThreads, 0, s>>>(b.tiles, b.tile_prefix, b.ntrees);
    }
    WT_CUDA_TRY(cudaGetLastError());
    for (uint32_t l = 0; l < b.maxL; l++) {
        WT_CUDA_TRY(cudaMemsetAsync(b.state_pool, 0, b.state_bytes, s));
        cudaError_t e;
        const bool enc = l == 0;
        if (b.w == 1) e = enc ? launch_level_pass_batched<uint8_t, true>(b, l, s) : launch_level_pass_batched<uint8_t, false>(b, l, s);
        else if (b.w == 2) e = enc ? launch_level_pass_batched<uint16_t, true>(b, l, s) : launch_level_pass_batched<uint16_t, false>(b, l, s);
        else e = enc ? launch_level_pass_batched<uint32_t, true>(b, l, s) : launch_level_pass_batched<uint32_t, false>(b, l, s);
        if (e != cudaSuccess) return WT_ECUDA;
        nk++;
    }
    if (kernels) *kernels = nk;
    return WT_OK;
}

}  // namespace wt

extern "C" wt_status wt_selftest_lookback_timeout(uint32_t spin_cap, wt_stream stream) {
    using namespace wt;
    if (spin_cap == 0 || spin_cap > kSpinCap) return WT_EINVAL;
    void* mem = nullptr;
    if (cudaMalloc(&mem, 256) != cudaSuccess) return WT_ENOMEM;
    uint64_t* state = static_cast<uint64_t*>(mem);
    uint32_t* status = reinterpret_cast<uint32_t*>(state + 4);
    uint64_t* out = state + 8;
    wt_status r = WT_ECUDA;
    if (cudaMemsetAsync(mem, 0, 256, stream) == cudaSuccess) {
        lookback_timeout_kernel<<<1, 32, 0, stream>>>(state, status, spin_cap, out);
        uint32_t st = 0;
        if (cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(stream) == cudaSuccess &&
            cudaMemcpy(&st, status, 4, cudaMemcpyDeviceToHost) == cudaSuccess)
            r = (st & kStTimeout) ? WT_ETIMEOUT : WT_OK;
    }
    cudaFree(mem);
    return r;
}
