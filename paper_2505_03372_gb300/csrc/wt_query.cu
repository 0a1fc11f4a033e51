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
// sorted by where its walks go -- access and rank by the position i, select by
// the expected position of the j-th c, 16-bit keys (kind-major for mixed
// batches) in two stable counting passes of 8 bits; the walks then run in that
// order and write each answer to the query's own slot.  The queries in flight
// at any moment then cover a few megabytes of every level, which L2 holds,
// instead of the whole tree.  Answers are the same in either order.
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
        out[ORD ? __ldg(idx + k) : k] = bad ? UINT32_MAX : (t.layout ? do_access_m(t, i) : do_access(t, nc, i));
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
        out[ORD ? __ldg(idx + k) : k] = bad ? UINT64_MAX : (t.layout ? do_rank_m(t, c, i) : do_rank(t, nc, c, i));
        flag_query_error(t, bad);
    }
}

// Select walks.  The walk is latency-bound on L1/L2 hits: every level is a
// chain of dependent loads (samples, L1 counter, about seven L2 probes, the
// words).  Shallow trees run one query per thread, compiled for eight CTAs per
// SM (32 registers); deep trees (kPairLevels levels or more) run two queries
// per thread in lockstep (do_select_n<2>, four CTAs per SM, 64 registers),
// which keeps twice the chains in flight per warp and lets the second query of
// a pair (its sorted neighbour) hit the lines the first brought into L1.
// Measured, 10^7 sorted selects: 7 levels 1.09 ms single / 1.20 ms paired;
// 8 levels 1.88 / 1.45; 12 levels 3.84 / 2.47; 16 levels 4.40 / 2.97; 20
// levels 7.08 / 5.14.  The threshold is kPairLevels.  Loading the first L2
// probes together with the L1 counter (one probe, or three for a four-way
// first step) was slower at every depth: the extra registers spill.

template <bool ORD, int NQ>
__global__ void __launch_bounds__(kQThreads, NQ == 1 ? 8 : 4) select_kernel(const __grid_constant__ TreeDesc t,
                                                                          const uint32_t* __restrict__ qc,
                                                                          const uint64_t* __restrict__ qj,
                                                                          const uint32_t* __restrict__ idx,
                                                                          uint64_t* __restrict__ out, uint64_t q,
                                                                          uint32_t slots) {
    extern __shared__ ulonglong2 s_nodes[];
    const NodeCache nc = load_node_cache(t, s_nodes, slots);
    const uint64_t stride = (uint64_t)NQ * gridDim.x * blockDim.x;
    for (uint64_t k0 = (uint64_t)NQ * ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x); k0 < q; k0 += stride) {
        uint32_t c[NQ];
        uint64_t j[NQ], r[NQ];
        bool in[NQ], ok[NQ], bad[NQ];
        bool any_bad = false;
#pragma unroll
        for (int x = 0; x < NQ; x++) {
            in[x] = k0 + x < q;
            c[x] = in[x] ? __ldg(qc + k0 + x) : 0u;
            j[x] = in[x] ? __ldg(qj + k0 + x) : 1ull;
            bad[x] = in[x] && !select_valid(t, c[x], j[x]);
            ok[x] = in[x] && !bad[x];
            any_bad = any_bad || bad[x];
        }
        if (t.layout) {
#pragma unroll
            for (int x = 0; x < NQ; x++) r[x] = ok[x] ? do_select_m(t, c[x], j[x]) : 0ull;
        } else {
            do_select_n<NQ>(t, nc, c, j, ok, r);
        }
#pragma unroll
        for (int x = 0; x < NQ; x++)
            if (in[x]) out[ORD ? __ldg(idx + k0 + x) : k0 + x] = bad[x] ? UINT64_MAX : r[x];
        flag_query_error(t, any_bad);
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
            if (!bad) r = (t.layout ? do_access_m(t, x) : do_access(t, nc, x));
        } else if (kd == 1) {
            const uint32_t c = __ldg(qc + k);
            bad = c >= t.cp.sigma || x > t.n;
            if (!bad) r = (t.layout ? do_rank_m(t, c, x) : do_rank(t, nc, c, x));
        } else if (kd == 2) {
            const uint32_t c = __ldg(qc + k);
            bad = !select_valid(t, c, x);
            if (!bad) r = (t.layout ? do_select_m(t, c, x) : do_select(t, nc, c, x));
        } else {
            bad = true;
        }
        out[ORD ? __ldg(idx + k) : k] = r;
        flag_query_error(t, bad);
    }
}

// ---------------------------------------------------------------------------
// query order: 16-bit keys, sorted by two stable counting passes of 8 bits
// (low byte, then high byte) over chunks of kChunk queries
// ---------------------------------------------------------------------------

constexpr uint32_t kKeyBits = 16;
constexpr uint32_t kOrdBuckets = 256;
constexpr uint32_t kOrdThreads = 512;
constexpr uint32_t kOrdWarps = kOrdThreads / 32;
// 2048 queries per chunk: the scatter writes runs of about 8 queries per
// bucket.  Chunks of 4096 were slower (scatter 0.139 against 0.122 ms per 10^7
// queries), and so were 1024 (more histogram and scan work) and 8192.
constexpr uint32_t kOrdPer = 4;
constexpr uint32_t kChunk = kOrdThreads * kOrdPer;  // queries per CTA; warp w owns [128 w, 128 w + 128)
constexpr uint64_t kOrderMinQueries = 1ull << 16;
constexpr size_t kOrderMinTreeBytes = (size_t)64 << 20;

struct OrderKey {
    uint32_t lgn;   // ceil(lg n)
    uint32_t kind;  // 0 access, 1 rank, 2 select, 3 mixed (kind per query)
};

struct OrdIn {
    const uint8_t* kind;  // mixed batches only
    const uint32_t* c;    // rank, select and mixed
    const uint64_t* a;
    const uint32_t* idx;  // null: the query's own index
};
struct OrdOut {
    uint8_t* kind;
    uint32_t* c;
    uint64_t* a;
    uint32_t* idx;
};

// nbits-bit key of a query: where in the sequence its walk goes.  Access and
// rank by the position i; select by where the j-th c is expected, j / n_c of
// the way through the sequence.  The walks touch the blocks at and below that
// point on every level, so queries close in key share blocks in L1 and L2.
__device__ __forceinline__ uint32_t sub_key(const TreeDesc& t, uint32_t lgn, uint32_t kd, uint32_t c, uint64_t x,
                                            uint32_t nbits) {
    const uint64_t top = (1ull << nbits) - 1;
    if (kd == 2) {
        if (c >= t.cp.sigma || x == 0) return 0u;
        const uint64_t nc = __ldg(t.C + c + 1) - __ldg(t.C + c);
        if (x > nc) return 0u;
        return (uint32_t)umin64(((x - 1) << nbits) / nc, top);
    }
    const uint32_t sh = lgn > nbits ? lgn - nbits : 0u;
    return (uint32_t)umin64(x >> sh, top);
}
// kKeyBits-bit key (kind-major for mixed batches)
__device__ __forceinline__ uint32_t query_key(const TreeDesc& t, const OrderKey& ok, const OrdIn& in, uint64_t k) {
    if (ok.kind < 3) return sub_key(t, ok.lgn, ok.kind, ok.kind == 2 ? __ldg(in.c + k) : 0u, __ldg(in.a + k), kKeyBits);
    const uint32_t kd = umin64(__ldg(in.kind + k), 3);
    const uint32_t c = kd == 2 ? __ldg(in.c + k) : 0u;
    return (kd << (kKeyBits - 2)) | sub_key(t, ok.lgn, kd == 3 ? 0u : kd, c, __ldg(in.a + k), kKeyBits - 2);
}

// per chunk and bucket (byte `shift / 8` of the key): queries of the chunk in
// the bucket; hist[bucket * nchunks + chunk]
__global__ void __launch_bounds__(kOrdThreads) order_hist_kernel(const __grid_constant__ TreeDesc t, OrderKey ok,
                                                                 OrdIn in, uint64_t q, uint32_t shift,
                                                                 uint64_t* __restrict__ hist, uint64_t nchunks) {
    __shared__ uint32_t h[kOrdBuckets];
    for (uint32_t b = threadIdx.x; b < kOrdBuckets; b += kOrdThreads) h[b] = 0;
    __syncthreads();
    const uint64_t c0 = (uint64_t)blockIdx.x * kChunk, c1 = umin64(q, c0 + kChunk);
    for (uint64_t k = c0 + threadIdx.x; k < c1; k += kOrdThreads)
        atomicAdd(h + ((query_key(t, ok, in, k) >> shift) & (kOrdBuckets - 1)), 1u);
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < kOrdBuckets; b += kOrdThreads) hist[(uint64_t)b * nchunks + blockIdx.x] = h[b];
}

// One stable counting pass: the chunk's queries go to their buckets' slots in
// chunk order.  The chunk is first ranked by bucket in shared memory (each warp
// ranks its own 256 queries in order with match masks; per-bucket counts of the
// warps are then prefix-summed), giving the chunk's permutation; the queries
// are then copied out in permuted order (their second read hits L1), so
// consecutive threads write consecutive slots of one bucket's run.
__global__ void __launch_bounds__(kOrdThreads, 4) order_scatter_kernel(const __grid_constant__ TreeDesc t, OrderKey ok,
                                                                       OrdIn in, uint64_t q, uint32_t shift,
                                                                       const uint64_t* __restrict__ offs,
                                                                       uint64_t nchunks, OrdOut out) {
    __shared__ uint16_t wcnt[kOrdWarps][kOrdBuckets];  // per warp and bucket: count, then first rank
    __shared__ uint16_t perm[kChunk];                   // chunk offset of the query at each sorted place
    __shared__ uint8_t pbkt[kChunk];                    // its bucket
    __shared__ uint32_t lbase[kOrdBuckets];             // first sorted place of each bucket
    __shared__ uint64_t gofs[kOrdBuckets];              // global slot minus sorted place, per bucket
    __shared__ uint32_t wsum[kOrdBuckets / 32];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint32_t i = tid; i < kOrdWarps * kOrdBuckets / 2; i += kOrdThreads) reinterpret_cast<uint32_t*>(wcnt)[i] = 0;
    __syncthreads();
    const uint64_t c0 = (uint64_t)blockIdx.x * kChunk;
    const uint32_t cn = (uint32_t)umin64(q - c0, kChunk);
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t kr[kOrdPer];  // bucket, then bucket << 16 | rank among the warp's queries of the bucket
#pragma unroll
    for (uint32_t r = 0; r < kOrdPer; r++) {  // all keys first, so that their loads overlap
        const uint32_t i = warp * (kOrdPer * 32) + r * 32 + lane;
        kr[r] = i < cn ? (query_key(t, ok, in, c0 + i) >> shift) & (kOrdBuckets - 1) : kOrdBuckets;
    }
#pragma unroll
    for (uint32_t r = 0; r < kOrdPer; r++) {
        const uint32_t i = warp * (kOrdPer * 32) + r * 32 + lane;
        const bool valid = i < cn;
        const uint32_t b = kr[r];
        const uint32_t mask = __match_any_sync(0xffffffffu, b);  // lanes past the end match only each other
        const uint32_t bi = valid ? b : 0u;
        const uint32_t old = wcnt[warp][bi];
        __syncwarp();
        if (valid && lane == (uint32_t)(__ffs(mask) - 1)) wcnt[warp][bi] = (uint16_t)(old + __popc(mask));
        __syncwarp();
        kr[r] = (b << 16) | (old + __popc(mask & lt_mask));
    }
    __syncthreads();
    if (tid < kOrdBuckets) {
        // prefix over the warps of this bucket's counts, then over the buckets
        uint32_t run = 0;
#pragma unroll
        for (uint32_t w = 0; w < kOrdWarps; w++) {
            const uint32_t v = wcnt[w][tid];
            wcnt[w][tid] = (uint16_t)run;
            run += v;
        }
        uint32_t x = run;
#pragma unroll
        for (uint32_t d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        lbase[tid] = x - run;  // exclusive within the warp
    }
    __syncthreads();
    if (tid < kOrdBuckets) {
        uint32_t before = 0;
        for (uint32_t w = 0; w < warp; w++) before += wsum[w];
        const uint32_t ex = lbase[tid] + before;
        lbase[tid] = ex;
        gofs[tid] = offs[(uint64_t)tid * nchunks + blockIdx.x] - ex;
    }
    __syncthreads();
#pragma unroll
    for (uint32_t r = 0; r < kOrdPer; r++) {
        const uint32_t i = warp * (kOrdPer * 32) + r * 32 + lane;
        if (i < cn) {
            const uint32_t b = kr[r] >> 16;
            const uint32_t p = lbase[b] + wcnt[warp][b] + (kr[r] & 0xffffu);
            perm[p] = (uint16_t)i;
            pbkt[p] = (uint8_t)b;
        }
    }
    __syncthreads();
#pragma unroll
    for (uint32_t r = 0; r < kOrdPer; r++) {
        const uint32_t p = tid + r * kOrdThreads;
        if (p < cn) {
            const uint64_t k = c0 + perm[p];
            const uint64_t slot = gofs[pbkt[p]] + p;
            out.a[slot] = __ldg(in.a + k);
            out.idx[slot] = in.idx ? __ldg(in.idx + k) : (uint32_t)k;
            if (in.c) out.c[slot] = __ldg(in.c + k);
            if (in.kind) out.kind[slot] = __ldg(in.kind + k);
        }
    }
}

bool use_order(const wt_tree_s* t, uint64_t q) {
    return q >= kOrderMinQueries && q < (1ull << 32) && t->lvl_bytes >= kOrderMinTreeBytes && t->desc.cp.L > 0;
}

// Sort the queries by key (fills o; o.mem must be freed by the caller).
wt_status order_queries(const wt_tree_s* t, uint32_t kindsel, const uint8_t* d_kind, const uint32_t* d_c,
                               const uint64_t* d_a, uint64_t q, cudaStream_t s, Ordered& o) {
    OrderKey ok;
    ok.lgn = 0;
    while ((1ull << ok.lgn) < t->desc.n) ok.lgn++;
    ok.kind = kindsel;
    const uint64_t nchunks = (q + kChunk - 1) / kChunk;
    const uint64_t nh = (uint64_t)kOrdBuckets * nchunks;
    const uint64_t ntmp = 2 * ((nh + 8191) / 8192 + 2);
    auto al = [](uint64_t x) { return (x + 255) & ~255ull; };
    const uint64_t per_copy = al(q * 8) + al(q * 4) + al(d_c ? q * 4 : 8) + al(d_kind ? q : 8);
    const uint64_t o_hist = 0, o_offs = al(nh * 8), o_tmp = o_offs + al((nh + 1) * 8), o_copy = o_tmp + al(ntmp * 8);
    const uint64_t total = o_copy + 2 * per_copy;
    if (dev_alloc(&o.mem, total, s, tree_alloc(t)) != cudaSuccess) return WT_ENOMEM;
    uint8_t* M = static_cast<uint8_t*>(o.mem);
    uint64_t* hist = reinterpret_cast<uint64_t*>(M + o_hist);
    uint64_t* offs = reinterpret_cast<uint64_t*>(M + o_offs);
    OrdOut cp[2];
    for (int i = 0; i < 2; i++) {
        uint8_t* B = M + o_copy + i * per_copy;
        cp[i].a = reinterpret_cast<uint64_t*>(B);
        cp[i].idx = reinterpret_cast<uint32_t*>(B + al(q * 8));
        cp[i].c = d_c ? reinterpret_cast<uint32_t*>(B + al(q * 8) + al(q * 4)) : nullptr;
        cp[i].kind = d_kind ? B + al(q * 8) + al(q * 4) + al(d_c ? q * 4 : 8) : nullptr;
    }
    OrdIn in{d_kind, d_c, d_a, nullptr};
    for (uint32_t pass = 0; pass < 2; pass++) {
        const uint32_t shift = 8 * pass;
        {
            ProfScope ps("order_hist", s);
            order_hist_kernel<<<(unsigned)nchunks, kOrdThreads, 0, s>>>(t->desc, ok, in, q, shift, hist, nchunks);
        }
        device_exclusive_scan(hist, offs, nh, reinterpret_cast<uint64_t*>(M + o_tmp), s, "order_scan");
        {
            ProfScope ps("order_scatter", s);
            order_scatter_kernel<<<(unsigned)nchunks, kOrdThreads, 0, s>>>(t->desc, ok, in, q, shift, offs,
                                                                                      nchunks, cp[pass]);
        }
        in = OrdIn{cp[pass].kind, cp[pass].c, cp[pass].a, cp[pass].idx};
    }
    o.a = cp[1].a;
    o.idx = cp[1].idx;
    o.c = cp[1].c;
    o.kind = cp[1].kind;
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------

// levels 0..7: 4 KB of {start, r0}.  A larger cache takes shared memory from
// L1, where the walks' counters and words hit: 2048 slots (32 KB per CTA) made
// the deep-tree walks up to 2.6x slower.
constexpr uint32_t kNodeCacheSlots = 256;

static uint32_t cache_slots(const wt_tree_s* t) {
    if (t->desc.layout != 0) return 0;  // a wavelet matrix has no node table to cache
    const uint32_t L = t->desc.cp.L;
    const uint64_t nslots = L ? (1ull << L) - 1 : 0;
    return (uint32_t)(nslots < kNodeCacheSlots ? nslots : kNodeCacheSlots);
}

// deep level-wise trees walk their selects two per thread (see select_kernel)
static bool pair_walks(const wt_tree_s* t) { return t->desc.layout == 0 && t->desc.cp.L >= kPairLevels; }

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
        if (o.mem) dev_free(o.mem, s, tree_alloc(t));
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
        if (o.mem) dev_free(o.mem, s, tree_alloc(t));
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
            auto kfn = pair_walks(t) ? select_kernel<true, 2> : select_kernel<true, 1>;
            WALK_LAUNCH(kfn, t, q, s, o.c, o.a, o.idx, d_out);
            if (cudaGetLastError() != cudaSuccess) st = WT_ECUDA;
        }
        if (o.mem) dev_free(o.mem, s, tree_alloc(t));
        return st;
    }
    ProfScope ps("select", s);
    auto kfn = pair_walks(t) ? select_kernel<false, 2> : select_kernel<false, 1>;
    WALK_LAUNCH(kfn, t, q, s, d_c, d_j, nullptr, d_out);
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
        if (o.mem) dev_free(o.mem, s, tree_alloc(t));
        return st;
    }
    ProfScope ps("mixed", s);
    WALK_LAUNCH(mixed_kernel<false>, t, q, s, d_kind, d_c, d_arg, nullptr, d_out);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

// ---------------------------------------------------------------------------
// ordering as a step of its own (wt_order_queries / wt_walk_ordered): the
// batch is sorted (or, below the ordering thresholds, copied) into private
// arrays, so it can run on another stream while the build's level passes run
// ---------------------------------------------------------------------------

wt_status prepare_order(const wt_tree_s* t, uint32_t kind, const uint8_t* d_kind, const uint32_t* d_c,
                        const uint64_t* d_a, uint64_t q, cudaStream_t s, Ordered& o, bool& ord) {
    ord = use_order(t, q);
    const uint32_t* c = kind >= 1 ? d_c : nullptr;
    const uint8_t* k = kind == 3 ? d_kind : nullptr;
    if (ord) return order_queries(t, kind, k, c, d_a, q, s, o);
    auto al = [](uint64_t x) { return (x + 255) & ~255ull; };
    const uint64_t off_c = al(q * 8), off_k = off_c + (c ? al(q * 4) : 0), total = off_k + (k ? al(q) : 0);
    if (dev_alloc(&o.mem, total ? total : 256, s, tree_alloc(t)) != cudaSuccess) return WT_ENOMEM;
    uint8_t* M = static_cast<uint8_t*>(o.mem);
    o.a = reinterpret_cast<uint64_t*>(M);
    o.c = c ? reinterpret_cast<uint32_t*>(M + off_c) : nullptr;
    o.kind = k ? M + off_k : nullptr;
    o.idx = nullptr;
    cudaError_t e = cudaMemcpyAsync(o.a, d_a, q * 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && c) e = cudaMemcpyAsync(o.c, c, q * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && k) e = cudaMemcpyAsync(o.kind, k, q, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? WT_OK : WT_ECUDA;
}

wt_status walk_prepared(const wt_tree_s* t, uint32_t kind, bool ord, const Ordered& o, void* d_out, uint64_t q,
                        cudaStream_t s) {
    if (!q) return WT_OK;
    if (kind == 0) {
        ProfScope ps("access", s);
        auto kfn = ord ? access_kernel<true> : access_kernel<false>;
        WALK_LAUNCH(kfn, t, q, s, o.a, o.idx, static_cast<uint32_t*>(d_out));
    } else if (kind == 1) {
        ProfScope ps("rank", s);
        auto kfn = ord ? rank_kernel<true> : rank_kernel<false>;
        WALK_LAUNCH(kfn, t, q, s, o.c, o.a, o.idx, static_cast<uint64_t*>(d_out));
    } else if (kind == 2) {
        ProfScope ps("select", s);
        const bool pair = pair_walks(t);
        auto kfn = ord ? (pair ? select_kernel<true, 2> : select_kernel<true, 1>)
                       : (pair ? select_kernel<false, 2> : select_kernel<false, 1>);
        WALK_LAUNCH(kfn, t, q, s, o.c, o.a, o.idx, static_cast<uint64_t*>(d_out));
    } else {
        ProfScope ps("mixed", s);
        auto kfn = ord ? mixed_kernel<true> : mixed_kernel<false>;
        WALK_LAUNCH(kfn, t, q, s, o.kind, o.c, o.a, o.idx, static_cast<uint64_t*>(d_out));
    }
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

}  // namespace wt
