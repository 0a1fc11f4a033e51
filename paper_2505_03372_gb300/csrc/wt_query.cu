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
#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_internal.hpp"

namespace wt {

__device__ __forceinline__ ulonglong2 node_sr(const TreeDesc& t, uint32_t l, uint64_t p) {
    // {start, r0} of node (l, p); slots are 32-byte aligned
    return ldg_nc_v2(reinterpret_cast<const uint64_t*>(t.nodes + ((1ull << l) - 1 + p)));
}

// Algorithm 5 with the early stop at nodes of at most two symbols.
__device__ __forceinline__ uint32_t do_access(const TreeDesc& t, uint64_t i) {
    const CodeParams& cp = t.cp;
    if (cp.L == 0) return 0;
    uint64_t p = 0;
    for (uint32_t l = 0; l < cp.L; l++) {
        uint64_t a, width;
        if (cp.pow2) {
            width = 1ull << (cp.L - l);
            a = p << (cp.L - l);
        } else {
            width = node_info(cp, l, p, a);
        }
        if (width == 1) return (uint32_t)a;
        const ulonglong2 ne = node_sr(t, l, p);
        const uint64_t pos = ne.x + i;
        if (width == 2) return (uint32_t)(a + bit_at(t.lv[l], pos));
        uint32_t b;
        const uint64_t r1 = rank1_bit(t.lv[l], pos, b);
        const uint64_t zb = (pos - r1) - ne.y;  // zeros of the node before i
        i = b ? i - zb : zb;
        p = 2 * p + b;
    }
    return UINT32_MAX;  // not reached: every root-to-leaf path ends at a leaf
}

// Algorithm 6: the code of c gives the direction at every level.
__device__ __forceinline__ uint64_t do_rank(const TreeDesc& t, uint32_t c, uint64_t i) {
    const CodeParams& cp = t.cp;
    uint32_t code, len;
    encode(cp, c, code, len);
    ulonglong2 ne = node_sr(t, 0, 0);
    for (uint32_t l = 0; l < len; l++) {
        if (i == 0) return 0;
        const uint32_t b = (code >> (cp.L - 1 - l)) & 1u;
        const uint64_t pos = ne.x + i;
        const uint64_t r0n = ne.y;
        if (l + 1 < len) ne = node_sr(t, l + 1, code >> (cp.L - 1 - l));  // next node, issued early
        const uint64_t r1 = rank1(t.lv[l], pos);
        const uint64_t zb = (pos - r1) - r0n;
        i = b ? i - zb : zb;
    }
    return i;
}

// Algorithms 7 and 8: leaf to root; the node of c at level l is the prefix of
// its code, so getNodeStart becomes a table index.
__device__ __forceinline__ uint64_t do_select(const TreeDesc& t, uint32_t c, uint64_t j) {
    const CodeParams& cp = t.cp;
    uint32_t code, len;
    encode(cp, c, code, len);
    if (len == 0) return j - 1;
    int l = (int)len - 1;
    ulonglong2 ne = node_sr(t, (uint32_t)l, (uint64_t)code >> (cp.L - (uint32_t)l));
    for (; l >= 0; l--) {
        const uint32_t b = (code >> (cp.L - 1 - (uint32_t)l)) & 1u;
        const uint64_t start = ne.x;
        const uint64_t kb = b ? (start - ne.y) : ne.y;  // b-bits before the node
        if (l > 0) ne = node_sr(t, (uint32_t)l - 1, (uint64_t)code >> (cp.L - (uint32_t)l + 1));
        const uint64_t pos = select_b(t.lv[l], b, kb + j, t.k_log2);
        j = pos + 1 - start;
    }
    return j - 1;
}

__device__ __forceinline__ bool select_valid(const TreeDesc& t, uint32_t c, uint64_t j) {
    if (c >= t.cp.sigma || j == 0) return false;
    return j <= __ldg(t.C + c + 1) - __ldg(t.C + c);
}

__device__ __forceinline__ void flag_query_error(const TreeDesc& t, bool bad) {
    if (__any_sync(__activemask(), bad)) {
        if (bad) atomicOr(t.status, kStQuery);
    }
}

constexpr int kQThreads = 256;

__global__ void __launch_bounds__(kQThreads) access_kernel(const __grid_constant__ TreeDesc t,
                                                           const uint64_t* __restrict__ qi, uint32_t* __restrict__ out,
                                                           uint64_t q) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < q; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = __ldg(qi + k);
        const bool bad = i >= t.n;
        out[k] = bad ? UINT32_MAX : do_access(t, i);
        flag_query_error(t, bad);
    }
}

__global__ void __launch_bounds__(kQThreads) rank_kernel(const __grid_constant__ TreeDesc t,
                                                         const uint32_t* __restrict__ qc,
                                                         const uint64_t* __restrict__ qi, uint64_t* __restrict__ out,
                                                         uint64_t q) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < q; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = __ldg(qc + k);
        const uint64_t i = __ldg(qi + k);
        const bool bad = c >= t.cp.sigma || i > t.n;
        out[k] = bad ? UINT64_MAX : do_rank(t, c, i);
        flag_query_error(t, bad);
    }
}

__global__ void __launch_bounds__(kQThreads) select_kernel(const __grid_constant__ TreeDesc t,
                                                           const uint32_t* __restrict__ qc,
                                                           const uint64_t* __restrict__ qj, uint64_t* __restrict__ out,
                                                           uint64_t q) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < q; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = __ldg(qc + k);
        const uint64_t j = __ldg(qj + k);
        const bool bad = !select_valid(t, c, j);
        out[k] = bad ? UINT64_MAX : do_select(t, c, j);
        flag_query_error(t, bad);
    }
}

__global__ void __launch_bounds__(kQThreads) mixed_kernel(const __grid_constant__ TreeDesc t,
                                                          const uint8_t* __restrict__ kind,
                                                          const uint32_t* __restrict__ qc,
                                                          const uint64_t* __restrict__ qa, uint64_t* __restrict__ out,
                                                          uint64_t q) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < q; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t kd = __ldg(kind + k);
        const uint64_t x = __ldg(qa + k);
        uint64_t r = UINT64_MAX;
        bool bad;
        if (kd == 0) {
            bad = x >= t.n;
            if (!bad) r = do_access(t, x);
        } else if (kd == 1) {
            const uint32_t c = __ldg(qc + k);
            bad = c >= t.cp.sigma || x > t.n;
            if (!bad) r = do_rank(t, c, x);
        } else if (kd == 2) {
            const uint32_t c = __ldg(qc + k);
            bad = !select_valid(t, c, x);
            if (!bad) r = do_select(t, c, x);
        } else {
            bad = true;
        }
        out[k] = r;
        flag_query_error(t, bad);
    }
}

template <typename K>
static int grid_for(K kernel, uint64_t q) {
    static int per_sm = 0;
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kQThreads, 0);
        if (per_sm <= 0) per_sm = 1;
    }
    uint64_t need = (q + kQThreads - 1) / kQThreads;
    uint64_t full = (uint64_t)per_sm * sm_count();
    return (int)(need < full ? need : full);
}

wt_status launch_access(const wt_tree_s* t, const uint64_t* d_i, uint32_t* d_out, uint64_t q, cudaStream_t s) {
    if (!q) return WT_OK;
    ProfScope ps("access", s);
    access_kernel<<<grid_for(access_kernel, q), kQThreads, 0, s>>>(t->desc, d_i, d_out, q);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

wt_status launch_rank(const wt_tree_s* t, const uint32_t* d_c, const uint64_t* d_i, uint64_t* d_out, uint64_t q,
                      cudaStream_t s) {
    if (!q) return WT_OK;
    ProfScope ps("rank", s);
    rank_kernel<<<grid_for(rank_kernel, q), kQThreads, 0, s>>>(t->desc, d_c, d_i, d_out, q);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

wt_status launch_select(const wt_tree_s* t, const uint32_t* d_c, const uint64_t* d_j, uint64_t* d_out, uint64_t q,
                        cudaStream_t s) {
    if (!q) return WT_OK;
    ProfScope ps("select", s);
    select_kernel<<<grid_for(select_kernel, q), kQThreads, 0, s>>>(t->desc, d_c, d_j, d_out, q);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

wt_status launch_mixed(const wt_tree_s* t, const uint8_t* d_kind, const uint32_t* d_c, const uint64_t* d_arg,
                       uint64_t* d_out, uint64_t q, cudaStream_t s) {
    if (!q) return WT_OK;
    ProfScope ps("mixed", s);
    mixed_kernel<<<grid_for(mixed_kernel, q), kQThreads, 0, s>>>(t->desc, d_kind, d_c, d_arg, d_out, q);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

}  // namespace wt
