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
#include "wt_walk.cuh"

namespace wt {

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
