// Construction of the extended level-wise wavelet tree (Section 5.1,
// Algorithm 4) on one GB300.
//
// Pipeline (all on the device, one stream):
//   1. histogram of S with symbol validation (Section 5.1.1: shared-memory
//      sub-histograms, persistent grid);
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
//      ones that the counters and the partition need comes from a decoupled
//      look-back over tiles, so every level reads T_l once and writes T_{l+1}
//      once.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "wt_device.cuh"
#include "wt_internal.hpp"

namespace wt {

// ===========================================================================
// 1. histogram + validation
// ===========================================================================

template <typename T>
__global__ void __launch_bounds__(512) hist_kernel(const T* __restrict__ S, uint64_t n, uint32_t sigma, uint32_t sbins,
                                                   uint32_t copies, unsigned long long* __restrict__ hist,
                                                   uint32_t* __restrict__ status) {
    extern __shared__ uint32_t sh[];
    for (uint32_t i = threadIdx.x; i < sbins * copies; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    uint32_t* mine = sh + (threadIdx.x % copies) * sbins;
    bool bad = false;
    constexpr int V = 16 / sizeof(T);
    const uint64_t nvec = n / V;
    const uint4* S4 = reinterpret_cast<const uint4*>(S);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    auto add = [&](uint32_t s) {
        if (s >= sigma) bad = true;
        else if (s < sbins) atomicAdd(mine + s, 1u);
        else atomicAdd(hist + s, 1ull);
    };
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec; v += stride) {
        uint4 x = __ldg(S4 + v);
        const T* e = reinterpret_cast<const T*>(&x);
#pragma unroll
        for (int k = 0; k < V; k++) add((uint32_t)e[k]);
    }
    for (uint64_t j = nvec * V + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) add((uint32_t)S[j]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kStSymbol);
    for (uint32_t b = threadIdx.x; b < sbins; b += blockDim.x) {
        uint32_t c = 0;
        for (uint32_t k = 0; k < copies; k++) c += sh[k * sbins + b];
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
static void device_exclusive_scan(const uint64_t* in, uint64_t* out, uint64_t count, uint64_t* tmp, cudaStream_t s) {
    if (count <= (uint64_t)kScanChunk * 4) {
        ProfScope ps("scan_single", s);
        scan_single_kernel<<<1, kScanThreads, 0, s>>>(in, out, count);
        return;
    }
    uint64_t nb = (count + kScanChunk - 1) / kScanChunk;
    uint64_t* part = tmp;
    uint64_t* part_ex = tmp + nb + 1;
    {
        ProfScope ps("scan_partials", s);
        scan_partials_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, count, part);
    }
    {
        ProfScope ps("scan_single", s);
        scan_single_kernel<<<1, kScanThreads, 0, s>>>(part, part_ex, nb);
    }
    {
        ProfScope ps("scan_apply", s);
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
// 4. level passes: wt_level.cu (bit planes); the bounded look-back's self-test
// ===========================================================================

// Diagnostic: tile 1 looks back at a tile 0 that never publishes anything.
__global__ void lookback_timeout_kernel(uint64_t* state, uint32_t* status, uint32_t spin_cap, uint64_t* out) {
    const uint64_t excl = lookback_warp(state, 1, 5, status, spin_cap);
    if (threadIdx.x == 0) *out = excl;
}

template <typename T>
static cudaError_t launch_hist(const void* S, uint64_t n, uint32_t sigma, unsigned long long* hist, uint32_t* status,
                               cudaStream_t s) {
    const uint32_t budget = 64 * 1024;  // bytes of shared memory for sub-histograms
    uint32_t sbins = std::min<uint32_t>(sigma, budget / 4);
    uint32_t copies = std::max<uint32_t>(1, std::min<uint32_t>(16, budget / (4 * std::max<uint32_t>(sbins, 1))));
    size_t sm = (size_t)sbins * copies * 4;
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(hist_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        configured = true;
    }
    int blocks = sm_count() * 3;
    ProfScope ps("histogram", s);
    hist_kernel<T><<<blocks, 512, sm, s>>>(reinterpret_cast<const T*>(S), n, sigma, sbins, copies, hist, status);
    return cudaGetLastError();
}

// ===========================================================================
// host orchestration
// ===========================================================================

static uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

wt_status build_tree(const void* d_symbols, uint64_t n, uint32_t sigma, uint32_t w, uint32_t sample_k, cudaStream_t s,
                     wt_tree_s* t) {
    const CodeParams cp = make_code_params(sigma);
    const uint32_t L = cp.L;
    uint32_t k_log2 = 0;
    while ((1u << k_log2) < sample_k) k_log2++;

    t->desc.cp = cp;
    t->desc.n = n;
    t->desc.k_log2 = k_log2;
    t->symbol_bytes = w;
    t->sample_k = sample_k;

    // ---- header memory: status, C, node table, meta ----
    const uint64_t nslots = L ? ((1ull << L) - 1) : 0;
    size_t off_status = 0;
    size_t off_C = 256;
    size_t off_nodes = align_up(off_C + (sigma + 1ull) * 8, 256);
    size_t hdr = align_up(off_nodes + std::max<uint64_t>(nslots, 1) * sizeof(NodeEntry), 256);
    WT_CUDA_TRY(dev_alloc(&t->hdr_mem, hdr, s));
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
    size_t s_end = align_up(s_meta + 2 * kMaxLevels * 8, 256);
    void* scratch = nullptr;
    WT_CUDA_TRY(dev_alloc(&scratch, s_end, s));
    uint8_t* X = reinterpret_cast<uint8_t*>(scratch);
    uint64_t* hist = reinterpret_cast<uint64_t*>(X + s_hist);
    uint64_t* left = reinterpret_cast<uint64_t*>(X + s_left);
    uint64_t* excl = reinterpret_cast<uint64_t*>(X + s_excl);
    uint64_t* tmp = reinterpret_cast<uint64_t*>(X + s_tmp);
    uint64_t* meta = reinterpret_cast<uint64_t*>(X + s_meta);

    WT_CUDA_TRY(cudaMemsetAsync(t->hdr_mem, 0, hdr, s));
    WT_CUDA_TRY(cudaMemsetAsync(hist, 0, (uint64_t)sigma * 8, s));

    // 1. histogram
    if (n) {
        cudaError_t e = w == 1 ? launch_hist<uint8_t>(d_symbols, n, sigma, (unsigned long long*)hist, t->desc.status, s)
                        : w == 2 ? launch_hist<uint16_t>(d_symbols, n, sigma, (unsigned long long*)hist, t->desc.status, s)
                                 : launch_hist<uint32_t>(d_symbols, n, sigma, (unsigned long long*)hist, t->desc.status, s);
        if (e != cudaSuccess) { dev_free(scratch, s); return WT_ECUDA; }
    }
    // 2. C
    device_exclusive_scan(hist, C, sigma, tmp, s);
    // 3. nodes + meta
    if (L) {
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
        dev_free(scratch, s);
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
    if (dev_alloc(&t->lvl_mem, t->lvl_bytes, s) != cudaSuccess) {
        dev_free(scratch, s);
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
    }

    // ---- level kernels over bit planes (wt_level.cu) ----
    if (L && n) {
        const uint64_t ps = plane_stride(n);
        const uint64_t set_words = (uint64_t)(L - 1) * ps;  // planes 1..L-1 of T_0, the most any level has
        const uint64_t ntile = level_tiles(n);
        const uint64_t w0 = 2 * lay[0].walloc;               // 32-bit words of B_0
        const uint64_t nchunks = transpose_chunks(w0);
        size_t o = 0;
        auto take = [&](size_t bytes) {
            const size_t r = o;
            o = align_up(o + std::max<size_t>(bytes, 8), 256);
            return r;
        };
        const size_t o_set0 = take(set_words * 4);
        const size_t o_set1 = take(L > 2 ? set_words * 4 : 0);
        const size_t o_count = take(ntile * 4);
        const size_t o_prefix = take(ntile * 8);
        const size_t o_first = take(ntile * 4);
        const size_t o_la = take(L * sizeof(LevelArgs));
        const size_t o_ta = take(sizeof(TransposeArgs));
        const size_t o_tp = take((L + 1) * 2 * 8);  // tile prefixes {0, tiles} per level + transpose
        const size_t o_cnt = take(L * 8);
        void* work = nullptr;
        if (dev_alloc(&work, o, s) != cudaSuccess) {
            dev_free(scratch, s);
            return WT_ENOMEM;
        }
        uint8_t* Wm = reinterpret_cast<uint8_t*>(work);
        uint32_t* set[2] = {reinterpret_cast<uint32_t*>(Wm + o_set0), reinterpret_cast<uint32_t*>(Wm + o_set1)};
        uint32_t* count = reinterpret_cast<uint32_t*>(Wm + o_count);
        LevelArgs* d_la = reinterpret_cast<LevelArgs*>(Wm + o_la);
        TransposeArgs* d_ta = reinterpret_cast<TransposeArgs*>(Wm + o_ta);
        uint64_t* d_tp = reinterpret_cast<uint64_t*>(Wm + o_tp);
        unsigned long long* d_cnt = reinterpret_cast<unsigned long long*>(Wm + o_cnt);

        std::vector<LevelArgs> la(L);
        std::vector<uint64_t> tp(2 * (L + 1), 0);  // pairs {0, tiles}
        for (uint32_t l = 0; l < L; l++) {
            LevelArgs& a = la[l];
            memset(&a, 0, sizeof(a));
            const bool last = l + 1 == L;
            a.bits = reinterpret_cast<const uint32_t*>(M + lay[l].words);
            a.in = set[l & 1];
            a.out0 = last ? nullptr : reinterpret_cast<uint32_t*>(M + lay[l + 1].words);
            a.out = set[(l + 1) & 1];
            a.pstride = ps;
            a.size = t->level_size[l];
            a.size_next = last ? 0 : t->level_size[l + 1];
            a.l1 = reinterpret_cast<uint64_t*>(M + lay[l].l1);
            a.l2 = reinterpret_cast<uint16_t*>(M + lay[l].l2);
            a.s0 = reinterpret_cast<uint64_t*>(M + lay[l].s0);
            a.s1 = reinterpret_cast<uint64_t*>(M + lay[l].s1);
            a.n_s0 = ((a.size - t->level_ones[l]) >> k_log2) + 1;
            a.n_s1 = (t->level_ones[l] >> k_log2) + 1;
            a.nodes = nodes + ((1ull << l) - 1);
            a.nnodes = internal_nodes(cp, l);
            a.count = count;
            a.prefix = reinterpret_cast<uint64_t*>(Wm + o_prefix);
            a.next_count = count;
            a.first_node = reinterpret_cast<uint32_t*>(Wm + o_first);
            a.status = t->desc.status;
            a.R = L - l;
            a.k_log2 = k_log2;
            tp[2 * l + 1] = level_tiles(a.size);
        }
        tp[2 * L + 1] = nchunks;
        TransposeArgs ta;
        memset(&ta, 0, sizeof(ta));
        ta.sym = d_symbols;
        ta.n = n;
        ta.bits0 = reinterpret_cast<uint32_t*>(M + lay[0].words);
        ta.bits0_words = w0;
        ta.planes = set[0];
        ta.pstride = ps;
        ta.count = count;
        ta.sigma = sigma;
        ta.L = L;
        ta.pow2 = cp.pow2;
        WT_CUDA_TRY(cudaMemcpyAsync(d_la, la.data(), L * sizeof(LevelArgs), cudaMemcpyHostToDevice, s));
        WT_CUDA_TRY(cudaMemcpyAsync(d_ta, &ta, sizeof(ta), cudaMemcpyHostToDevice, s));
        WT_CUDA_TRY(cudaMemcpyAsync(d_tp, tp.data(), tp.size() * 8, cudaMemcpyHostToDevice, s));
        WT_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, L * 8, s));
        // outputs are ORed into where two runs share a word: they start at zero
        WT_CUDA_TRY(cudaMemsetAsync(t->lvl_mem, 0, t->lvl_bytes, s));
        if (L > 2) WT_CUDA_TRY(cudaMemsetAsync(set[1], 0, set_words * 4, s));
        WT_CUDA_TRY(cudaMemsetAsync(count, 0, ntile * 4, s));
        wt_status st = launch_transpose(d_ta, d_tp + 2 * L, 1, nchunks, w, s);
        for (uint32_t l = 0; l < L && st == WT_OK; l++) {
            if (t->level_size[l] == 0) continue;
            st = launch_count_scan(d_la + l, 1, s);
            if (st == WT_OK && l + 1 < L && cudaMemsetAsync(count, 0, ntile * 4, s) != cudaSuccess) st = WT_ECUDA;
            if (st == WT_OK && l + 1 < L && la[l].nnodes > 1)
                st = launch_first_node(d_la + l, d_tp + 2 * l, 1, tp[2 * l + 1], s);
            if (st == WT_OK) st = launch_level(d_la + l, d_tp + 2 * l, 1, tp[2 * l + 1], s);
        }
        dev_free(work, s);
        if (st != WT_OK) {
            dev_free(scratch, s);
            return st;
        }
    }
    // empty levels (no code reaches them) still need zero words and first counter / sample entries
    for (uint32_t l = 0; l < L; l++) {
        if (n == 0 || t->level_size[l] == 0) {
            WT_CUDA_TRY(cudaMemsetAsync(M + lay[l].words, 0, lay[l].walloc * 8, s));
            WT_CUDA_TRY(cudaMemsetAsync(M + lay[l].l1, 0, 8, s));
            WT_CUDA_TRY(cudaMemsetAsync(M + lay[l].l2, 0, 2, s));
            WT_CUDA_TRY(cudaMemsetAsync(M + lay[l].s0, 0, 8, s));
            WT_CUDA_TRY(cudaMemsetAsync(M + lay[l].s1, 0, 8, s));
        }
    }
    dev_free(scratch, s);
    return WT_OK;
}

// ===========================================================================
// batches of trees: the same pipeline for many trees, with no host round trip
// (every size the host would read back is computed on the device), so the
// whole sequence can be captured in one CUDA graph
// ===========================================================================

constexpr uint32_t kBatchSmemBins = 4096;

// one CTA per chunk of kBatchChunk symbols of one tree
template <typename T>
__global__ void __launch_bounds__(512) batch_hist_kernel(const BatchTreeInfo* __restrict__ info,
                                                         const uint64_t* __restrict__ chunk_prefix, uint32_t ntrees) {
    __shared__ uint32_t sh[kBatchSmemBins];
    __shared__ uint32_t s_tree;
    const uint64_t g = blockIdx.x;
    if (threadIdx.x == 0) s_tree = find_tree(chunk_prefix, ntrees, g);
    __syncthreads();
    const BatchTreeInfo& ti = info[s_tree];
    const uint64_t c0 = (g - chunk_prefix[s_tree]) * kBatchChunk;
    const uint64_t c1 = umin64(ti.n, c0 + kBatchChunk);
    const uint32_t sigma = ti.sigma;
    const bool small = sigma <= kBatchSmemBins;
    if (small)
        for (uint32_t i = threadIdx.x; i < sigma; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const T* S = reinterpret_cast<const T*>(ti.sym);
    unsigned long long* hist = reinterpret_cast<unsigned long long*>(ti.hist);
    bool bad = false;
    for (uint64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
        const uint32_t v = (uint32_t)S[j];
        if (v >= sigma) bad = true;
        else if (small) atomicAdd(sh + v, 1u);
        else atomicAdd(hist + v, 1ull);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(ti.status, kStSymbol);
    if (small)
        for (uint32_t i = threadIdx.x; i < sigma; i += blockDim.x)
            if (sh[i]) atomicAdd(hist + i, (unsigned long long)sh[i]);
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
// and the level arguments; tiles per level
__global__ void batch_meta_kernel(const BatchTreeInfo* __restrict__ info, TreeDesc* __restrict__ desc,
                                  LevelArgs* __restrict__ la, uint64_t* __restrict__ tiles, uint32_t ntrees,
                                  uint32_t maxL, uint32_t kl) {
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (uint64_t)ntrees * maxL) return;
    const uint32_t tr = (uint32_t)(g % ntrees), l = (uint32_t)(g / ntrees);
    const BatchTreeInfo& ti = info[tr];
    uint64_t* rt = tiles + (uint64_t)l * ntrees + tr;
    if (l >= ti.L || ti.n == 0) {
        *rt = 0;
        if (l < ti.L) {
            desc[tr].lv[l].size = 0;
            desc[tr].lv[l].ones = 0;
        }
        return;
    }
    LevelArgs& a = la[(uint64_t)l * ntrees + tr];
    const uint64_t size = ti.C[ti.s0[l]];
    const uint64_t zeros = ti.excl[(2ull << l) - 1] - ti.excl[(1ull << l) - 1];
    const uint64_t ones = size - zeros;
    desc[tr].lv[l].size = size;
    desc[tr].lv[l].ones = ones;
    a.size = size;
    a.size_next = (l + 1 < ti.L) ? ti.C[ti.s0[l + 1]] : 0;
    a.n_s0 = (zeros >> kl) + 1;
    a.n_s1 = (ones >> kl) + 1;
    *rt = level_tiles(size);
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

wt_status enqueue_batch_build(const BatchDev& b, cudaStream_t s, uint32_t* kernels) {
    uint32_t nk = 0;
    WT_CUDA_TRY(cudaMemsetAsync(b.hist_pool, 0, b.hist_bytes, s));
    WT_CUDA_TRY(cudaMemsetAsync(b.status_pool, 0, (size_t)b.ntrees * 4, s));
    WT_CUDA_TRY(cudaMemsetAsync(b.counters, 0, (size_t)(b.maxL ? b.maxL : 1) * 8, s));
    // level outputs are ORed into where two runs share a word: they start at zero
    WT_CUDA_TRY(cudaMemsetAsync(b.words_pool, 0, b.words_bytes, s));
    WT_CUDA_TRY(cudaMemsetAsync(b.count_pool, 0, b.count_bytes, s));
    if (b.total_chunks) {
        nk++;
        if (b.w == 1) batch_hist_kernel<uint8_t><<<(unsigned)b.total_chunks, 512, 0, s>>>(b.info, b.chunk_prefix, b.ntrees);
        else if (b.w == 2) batch_hist_kernel<uint16_t><<<(unsigned)b.total_chunks, 512, 0, s>>>(b.info, b.chunk_prefix, b.ntrees);
        else batch_hist_kernel<uint32_t><<<(unsigned)b.total_chunks, 512, 0, s>>>(b.info, b.chunk_prefix, b.ntrees);
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
        const uint64_t nm = (uint64_t)b.ntrees * b.maxL;
        nk += 2;
        batch_meta_kernel<<<(unsigned)((nm + 255) / 256), 256, 0, s>>>(b.info, b.desc, b.la, b.tiles, b.ntrees, b.maxL,
                                                                       b.k_log2);
        batch_tile_scan_kernel<<<b.maxL, kScanThreads, 0, s>>>(b.tiles, b.tile_prefix, b.ntrees);
    }
    WT_CUDA_TRY(cudaGetLastError());
    if (b.maxL && b.total_tr_chunks) {
        if (launch_transpose(b.ta, b.tr_prefix, b.ntrees, b.total_tr_chunks, b.w, s) != WT_OK) return WT_ECUDA;
        nk++;
    }
    for (uint32_t l = 0; l < b.maxL; l++) {
        const LevelArgs* la = b.la + (uint64_t)l * b.ntrees;
        if (launch_count_scan(la, b.ntrees, s) != WT_OK) return WT_ECUDA;
        WT_CUDA_TRY(cudaMemsetAsync(b.count_pool, 0, b.count_bytes, s));
        if (launch_first_node(la, b.tile_prefix + (uint64_t)l * (b.ntrees + 1), b.ntrees, b.max_tiles, s) != WT_OK)
            return WT_ECUDA;
        if (launch_level(la, b.tile_prefix + (uint64_t)l * (b.ntrees + 1), b.ntrees, b.max_tiles, s) != WT_OK)
            return WT_ECUDA;
        nk += 3;
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
