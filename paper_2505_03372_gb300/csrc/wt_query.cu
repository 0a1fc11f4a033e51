// Batched access / rank / select queries (Sections 5.2-5.4, Algorithms 5-8).
//
// One thread walks one query through the levels (the paper's best setting,
// one thread per query with 64-bit word loads, Sections 5.2.1 and 5.4.1), in
// a persistent grid-stride loop.  Per level a walk reads one node-table entry
// (node start and the precomputed rank at that start, Section 5.2.1), the L1
// and L2 counters and at most one 64-byte block of bit words.  The node
// identity is the prefix of the symbol's reduced code, so rank and select know
// the next level's node before the current binary rank finishes and issue its
// table load early.
//
// Query order.  Queries in random order touch one random 64-byte block per
// level in a tree far larger than L2.  A large batch on a large tree is first
// grouped by where its walk goes -- access by position, rank by (code prefix
// of c, position), select by (code prefix of c, rank j) -- with a counting sort
// over 4096 buckets; the walks then run in that order and write each answer to
// the query's own slot.  The queries in flight at any moment then cover a few
// megabytes of every level, which L2 holds, instead of the whole tree.  Answers
// are the same in either order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_internal.hpp"
#include "wt_walk.cuh"

namespace wt {

constexpr int kQThreads = 256;

// ---------------------------------------------------------------------------
// walks (ORD: inputs in bucket order, answer k goes to out[idx[k]])
// ---------------------------------------------------------------------------

template <bool ORD>
__global__ void __launch_bounds__(kQThreads) access_kernel(const __grid_constant__ TreeDesc t,
                                                           const uint64_t* __restrict__ qi,
                                                           const uint32_t* __restrict__ idx,
                                                           uint32_t* __restrict__ out, uint64_t q, uint32_t slots) {
    extern __shared__ ulonglong2 s_nodes[];
    const NodeCache nc = load_node_cache(t, s_nodes, slots);
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < q; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = __ldg(qi + k);
        const bool bad = i >= t.n;
        out[ORD ? __ldg(idx + k) : k] = bad ? UINT32_MAX : do_access(t, nc, i);
        flag_query_error(t, bad);
    }
}

template <bool ORD>
__global__ void __launch_bounds__(kQThreads) rank_kernel(const __grid_constant__ TreeDesc t,
                                                         const uint32_t* __restrict__ qc,
                                                         const uint64_t* __restrict__ qi,
                                                         const uint32_t* __restrict__ idx,
                                                         uint64_t* __restrict__ out, uint64_t q, uint32_t slots) {
    extern __shared__ ulonglong2 s_nodes[];
    const NodeCache nc = load_node_cache(t, s_nodes, slots);
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < q; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = __ldg(qc + k);
        const uint64_t i = __ldg(qi + k);
        const bool bad = c >= t.cp.sigma || i > t.n;
        out[ORD ? __ldg(idx + k) : k] = bad ? UINT64_MAX : do_rank(t, nc, c, i);
        flag_query_error(t, bad);
    }
}

template <bool ORD>
__global__ void __launch_bounds__(kQThreads) select_kernel(const __grid_constant__ TreeDesc t,
                                                           const uint32_t* __restrict__ qc,
                                                           const uint64_t* __restrict__ qj,
                                                           const uint32_t* __restrict__ idx,
                                                           uint64_t* __restrict__ out, uint64_t q, uint32_t slots) {
    extern __shared__ ulonglong2 s_nodes[];
    const NodeCache nc = load_node_cache(t, s_nodes, slots);
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < q; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = __ldg(qc + k);
        const uint64_t j = __ldg(qj + k);
        const bool bad = !select_valid(t, c, j);
        out[ORD ? __ldg(idx + k) : k] = bad ? UINT64_MAX : do_select(t, nc, c, j);
        flag_query_error(t, bad);
    }
}

template <bool ORD>
__global__ void __launch_bounds__(kQThreads) mixed_kernel(const __grid_constant__ TreeDesc t,
                                                          const uint8_t* __restrict__ kind,
                                                          const uint32_t* __restrict__ qc,
                                                          const uint64_t* __restrict__ qa,
                                                          const uint32_t* __restrict__ idx,
                                                          uint64_t* __restrict__ out, uint64_t q, uint32_t slots) {
    extern __shared__ ulonglong2 s_nodes[];
    const NodeCache nc = load_node_cache(t, s_nodes, slots);
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < q; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t kd = __ldg(kind + k);
        const uint64_t x = __ldg(qa + k);
        uint64_t r = UINT64_MAX;
        bool bad;
        if (kd == 0) {
            bad = x >= t.n;
            if (!bad) r = do_access(t, nc, x);
        } else if (kd == 1) {
            const uint32_t c = __ldg(qc + k);
            bad = c >= t.cp.sigma || x > t.n;
            if (!bad) r = do_rank(t, nc, c, x);
        } else if (kd == 2) {
            const uint32_t c = __ldg(qc + k);
            bad = !select_valid(t, c, x);
            if (!bad) r = do_select(t, nc, c, x);
        } else {
            bad = true;
        }
        out[ORD ? __ldg(idx + k) : k] = r;
        flag_query_error(t, bad);
    }
}

// ---------------------------------------------------------------------------
// query order: counting sort over kBuckets buckets in chunks of kChunk queries
// ---------------------------------------------------------------------------

constexpr uint32_t kBucketBits = 12;
constexpr uint32_t kBuckets = 1u << kBucketBits;
constexpr uint32_t kOrdThreads = 1024;
constexpr uint32_t kOrdPer = 32;
constexpr uint64_t kChunk = (uint64_t)kOrdThreads * kOrdPer;  // queries per CTA
constexpr uint64_t kOrderMinQueries = 1ull << 16;
constexpr size_t kOrderMinTreeBytes = (size_t)64 << 20;

struct OrderKey {
    uint32_t lgn;    // ceil(lg n): positions and ranks above 2^lgn fall in the last bucket
    uint32_t kind;   // 0 access, 1 rank, 2 select, 3 mixed (kind per query)
};

// nbits-bit key of a query: access by position; rank and select by the top bits
// of c's code, then by the top bits of i or j.
__device__ __forceinline__ uint32_t sub_key(const TreeDesc& t, uint32_t lgn, uint32_t kd, uint32_t c, uint64_t x,
                                            uint32_t nbits) {
    const uint32_t L = t.cp.L;
    uint32_t pre = 0, cb = 0;
    if (kd != 0) {
        cb = L < nbits ? L : nbits;
        uint32_t code = 0, len;
        if (c < t.cp.sigma) encode(t.cp, c, code, len);
        pre = cb ? code >> (L - cb) : 0u;
    }
    const uint32_t xb = nbits - cb;
    const uint32_t sh = lgn > xb ? lgn - xb : 0u;
    const uint64_t xs = x >> sh;
    const uint32_t xm = (uint32_t)umin64(xs, (1ull << xb) - 1);
    return (pre << xb) | xm;
}
__device__ __forceinline__ uint32_t query_key(const TreeDesc& t, const OrderKey& ok, const uint8_t* kind,
                                              const uint32_t* qc, const uint64_t* qa, uint64_t k) {
    if (ok.kind < 3) return sub_key(t, ok.lgn, ok.kind, qc ? __ldg(qc + k) : 0u, __ldg(qa + k), kBucketBits);
    const uint32_t kd = umin64(__ldg(kind + k), 3);
    const uint32_t c = kd == 0 ? 0u : __ldg(qc + k);
    return (kd << (kBucketBits - 2)) | sub_key(t, ok.lgn, kd == 3 ? 0u : kd, c, __ldg(qa + k), kBucketBits - 2);
}

// per chunk and bucket: queries of the chunk in the bucket; hist[bucket * nchunks + chunk]
__global__ void __launch_bounds__(kOrdThreads) order_hist_kernel(const __grid_constant__ TreeDesc t, OrderKey ok,
                                                                 const uint8_t* __restrict__ kind,
                                                                 const uint32_t* __restrict__ qc,
                                                                 const uint64_t* __restrict__ qa, uint64_t q,
                                                                 uint64_t* __restrict__ hist, uint64_t nchunks) {
    __shared__ uint32_t h[kBuckets];
    for (uint32_t b = threadIdx.x; b < kBuckets; b += kOrdThreads) h[b] = 0;
    __syncthreads();
    const uint64_t c0 = (uint64_t)blockIdx.x * kChunk, c1 = umin64(q, c0 + kChunk);
    for (uint64_t k = c0 + threadIdx.x; k < c1; k += kOrdThreads) atomicAdd(h + query_key(t, ok, kind, qc, qa, k), 1u);
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < kBuckets; b += kOrdThreads) hist[(uint64_t)b * nchunks + blockIdx.x] = h[b];
}

// place every query of the chunk at its bucket's next slot
__global__ void __launch_bounds__(kOrdThreads) order_scatter_kernel(
    const __grid_constant__ TreeDesc t, OrderKey ok, const uint8_t* __restrict__ kind, const uint32_t* __restrict__ qc,
    const uint64_t* __restrict__ qa, uint64_t q, const uint64_t* __restrict__ offs, uint64_t nchunks,
    uint8_t* __restrict__ skind, uint32_t* __restrict__ sc, uint64_t* __restrict__ sa, uint32_t* __restrict__ sidx) {
    __shared__ uint32_t h[kBuckets];  // next slot of each bucket within this chunk's range
    for (uint32_t b = threadIdx.x; b < kBuckets; b += kOrdThreads) h[b] = 0;
    __syncthreads();
    const uint64_t c0 = (uint64_t)blockIdx.x * kChunk, c1 = umin64(q, c0 + kChunk);
    for (uint64_t k = c0 + threadIdx.x; k < c1; k += kOrdThreads) {
        const uint32_t b = query_key(t, ok, kind, qc, qa, k);
        const uint64_t slot = offs[(uint64_t)b * nchunks + blockIdx.x] + atomicAdd(h + b, 1u);
        sa[slot] = __ldg(qa + k);
        sidx[slot] = (uint32_t)k;
        if (qc) sc[slot] = __ldg(qc + k);
        if (kind) skind[slot] = __ldg(kind + k);
    }
}

struct Ordered {
    void* mem = nullptr;
    uint8_t* kind = nullptr;
    uint32_t* c = nullptr;
    uint64_t* a = nullptr;
    uint32_t* idx = nullptr;
};

static bool use_order(const wt_tree_s* t, uint64_t q) {
    return q >= kOrderMinQueries && q < (1ull << 32) && t->lvl_bytes >= kOrderMinTreeBytes && t->desc.cp.L > 0;
}

// Sort the queries into bucket order (fills o; o.mem must be freed by the caller).
static wt_status order_queries(const wt_tree_s* t, uint32_t kindsel, const uint8_t* d_kind, const uint32_t* d_c,
                               const uint64_t* d_a, uint64_t q, cudaStream_t s, Ordered& o) {
    OrderKey ok;
    ok.lgn = 0;
    while ((1ull << ok.lgn) < t->desc.n) ok.lgn++;
    ok.kind = kindsel;
    const uint64_t nchunks = (q + kChunk - 1) / kChunk;
    const uint64_t nh = (uint64_t)kBuckets * nchunks;
    const uint64_t ntmp = 2 * ((nh + 8191) / 8192 + 2);
    auto al = [](uint64_t x) { return (x + 255) & ~255ull; };
    const uint64_t o_hist = 0, o_offs = al(nh * 8), o_tmp = o_offs + al((nh + 1) * 8), o_a = o_tmp + al(ntmp * 8);
    const uint64_t o_idx = o_a + al(q * 8), o_c = o_idx + al(q * 4), o_k = o_c + al(d_c ? q * 4 : 8);
    const uint64_t total = o_k + al(d_kind ? q : 8);
    if (dev_alloc(&o.mem, total, s) != cudaSuccess) return WT_ENOMEM;
    uint8_t* M = static_cast<uint8_t*>(o.mem);
    uint64_t* hist = reinterpret_cast<uint64_t*>(M + o_hist);
    uint64_t* offs = reinterpret_cast<uint64_t*>(M + o_offs);
    o.a = reinterpret_cast<uint64_t*>(M + o_a);
    o.idx = reinterpret_cast<uint32_t*>(M + o_idx);
    o.c = d_c ? reinterpret_cast<uint32_t*>(M + o_c) : nullptr;
    o.kind = d_kind ? reinterpret_cast<uint8_t*>(M + o_k) : nullptr;
    {
        ProfScope ps("order_hist", s);
        order_hist_kernel<<<(unsigned)nchunks, kOrdThreads, 0, s>>>(t->desc, ok, d_kind, d_c, d_a, q, hist, nchunks);
    }
    device_exclusive_scan(hist, offs, nh, reinterpret_cast<uint64_t*>(M + o_tmp), s, "order_scan");
    {
        ProfScope ps("order_scatter", s);
        order_scatter_kernel<<<(unsigned)nchunks, kOrdThreads, 0, s>>>(t->desc, ok, d_kind, d_c, d_a, q, offs, nchunks,
                                                                         o.kind, o.c, o.a, o.idx);
    }
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------

constexpr uint32_t kNodeCacheSlots = 2048;  // levels 0..10: 32 KB of {start, r0}

static uint32_t cache_slots(const wt_tree_s* t) {
    const uint32_t L = t->desc.cp.L;
    const uint64_t nslots = L ? (1ull << L) - 1 : 0;
    return (uint32_t)(nslots < kNodeCacheSlots ? nslots : kNodeCacheSlots);
}

template <typename K>
static int grid_for(K kernel, uint64_t q, size_t smem) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kQThreads, smem);
    if (per_sm <= 0) per_sm = 1;
    uint64_t need = (q + kQThreads - 1) / kQThreads;
    uint64_t full = (uint64_t)per_sm * sm_count();
    return (int)(need < full ? need : full);
}

// launch a walk kernel with the node cache of the tree's top levels
#define WALK_LAUNCH(kernel, t, q, s, ...)                                                             \
    do {                                                                                              \
        const uint32_t slots_ = cache_slots(t);                                                       \
        const size_t sm_ = (size_t)slots_ * sizeof(ulonglong2);                                       \
        kernel<<<grid_for(kernel, q, sm_), kQThreads, sm_, s>>>(t->desc, __VA_ARGS__, q, slots_);     \
    } while (0)

wt_status launch_access(const wt_tree_s* t, const uint64_t* d_i, uint32_t* d_out, uint64_t q, cudaStream_t s) {
    if (!q) return WT_OK;
    if (use_order(t, q)) {
        Ordered o;
        wt_status st = order_queries(t, 0, nullptr, nullptr, d_i, q, s, o);
        if (st == WT_OK) {
            ProfScope ps("access", s);
            WALK_LAUNCH(access_kernel<true>, t, q, s, o.a, o.idx, d_out);
            if (cudaGetLastError() != cudaSuccess) st = WT_ECUDA;
        }
        if (o.mem) dev_free(o.mem, s);
        return st;
    }
    ProfScope ps("access", s);
    WALK_LAUNCH(access_kernel<false>, t, q, s, d_i, nullptr, d_out);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

wt_status launch_rank(const wt_tree_s* t, const uint32_t* d_c, const uint64_t* d_i, uint64_t* d_out, uint64_t q,
                      cudaStream_t s) {
    if (!q) return WT_OK;
    if (use_order(t, q)) {
        Ordered o;
        wt_status st = order_queries(t, 1, nullptr, d_c, d_i, q, s, o);
        if (st == WT_OK) {
            ProfScope ps("rank", s);
            WALK_LAUNCH(rank_kernel<true>, t, q, s, o.c, o.a, o.idx, d_out);
            if (cudaGetLastError() != cudaSuccess) st = WT_ECUDA;
        }
        if (o.mem) dev_free(o.mem, s);
        return st;
    }
    ProfScope ps("rank", s);
    WALK_LAUNCH(rank_kernel<false>, t, q, s, d_c, d_i, nullptr, d_out);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

wt_status launch_select(const wt_tree_s* t, const uint32_t* d_c, const uint64_t* d_j, uint64_t* d_out, uint64_t q,
                        cudaStream_t s) {
    if (!q) return WT_OK;
    if (use_order(t, q)) {
        Ordered o;
        wt_status st = order_queries(t, 2, nullptr, d_c, d_j, q, s, o);
        if (st == WT_OK) {
            ProfScope ps("select", s);
            WALK_LAUNCH(select_kernel<true>, t, q, s, o.c, o.a, o.idx, d_out);
            if (cudaGetLastError() != cudaSuccess) st = WT_ECUDA;
        }
        if (o.mem) dev_free(o.mem, s);
        return st;
    }
    ProfScope ps("select", s);
    WALK_LAUNCH(select_kernel<false>, t, q, s, d_c, d_j, nullptr, d_out);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

wt_status launch_mixed(const wt_tree_s* t, const uint8_t* d_kind, const uint32_t* d_c, const uint64_t* d_arg,
                       uint64_t* d_out, uint64_t q, cudaStream_t s) {
    if (!q) return WT_OK;
    if (use_order(t, q)) {
        Ordered o;
        wt_status st = order_queries(t, 3, d_kind, d_c, d_arg, q, s, o);
        if (st == WT_OK) {
            ProfScope ps("mixed", s);
            WALK_LAUNCH(mixed_kernel<true>, t, q, s, o.kind, o.c, o.a, o.idx, d_out);
            if (cudaGetLastError() != cudaSuccess) st = WT_ECUDA;
        }
        if (o.mem) dev_free(o.mem, s);
        return st;
    }
    ProfScope ps("mixed", s);
    WALK_LAUNCH(mixed_kernel<false>, t, q, s, d_kind, d_c, d_arg, nullptr, d_out);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

}  // namespace wt
