// Binary rank (Section 4.1, Algorithm 1) and sampled binary select (Section
// 4.2, Algorithm 2) over a caller-owned bitvector and the support structures
// wt_bitvector_support_static wrote: the same device functions the tree walks
// use on a level, one thread per query.
#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_internal.hpp"

namespace wt {
namespace {

constexpr int kBvThreads = 256;

__global__ void __launch_bounds__(kBvThreads) bv_rank_kernel(const LevelDesc lv, const uint64_t* __restrict__ qi,
                                                             uint64_t* __restrict__ out, uint64_t q,
                                                             uint32_t* __restrict__ status) {
    bool bad_any = false;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < q; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = __ldg(qi + k);
        const bool bad = i > lv.size;
        out[k] = bad ? UINT64_MAX : rank1(lv, i);
        bad_any |= bad;
    }
    if (status && __any_sync(__activemask(), bad_any) && bad_any) atomicOr(status, kStQuery);
}

__global__ void __launch_bounds__(kBvThreads) bv_select_kernel(const LevelDesc lv, uint32_t b, uint32_t k_log2,
                                                               const uint64_t* __restrict__ qj,
                                                               uint64_t* __restrict__ out, uint64_t q,
                                                               uint32_t* __restrict__ status) {
    const uint64_t total = b ? lv.ones : lv.size - lv.ones;
    bool bad_any = false;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < q; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j = __ldg(qj + k);
        const bool bad = j == 0 || j > total;
        out[k] = bad ? UINT64_MAX : select_b(lv, b, j, k_log2);
        bad_any |= bad;
    }
    if (status && __any_sync(__activemask(), bad_any) && bad_any) atomicOr(status, kStQuery);
}

bool bv_dev(const void* p) { return device_ptr_ok(p); }

template <typename K>
int bv_grid(K kernel, uint64_t q) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBvThreads, 0);
    if (per_sm <= 0) per_sm = 1;
    const uint64_t need = (q + kBvThreads - 1) / kBvThreads, full = (uint64_t)per_sm * sm_count();
    return (int)(need < full ? need : full);
}

}  // namespace
}  // namespace wt

using namespace wt;

extern "C" wt_status wt_bitvector_rank(const uint64_t* d_words, uint64_t nbits, const uint64_t* d_l1,
                                       const uint16_t* d_l2, const uint64_t* d_i, uint64_t* d_out, uint64_t q,
                                       uint32_t* d_status, wt_stream stream) {
    if (nbits == 0 || (reinterpret_cast<uintptr_t>(d_words) & 31u)) return WT_EINVAL;
    if (!bv_dev(d_words) || !bv_dev(d_l1) || !bv_dev(d_l2)) return WT_EINVAL;
    if (d_status && !bv_dev(d_status)) return WT_EINVAL;
    if (!q) return WT_OK;
    if (!bv_dev(d_i) || !bv_dev(d_out)) return WT_EINVAL;
    LevelDesc lv = {};
    lv.words = d_words;
    lv.l1 = d_l1;
    lv.l2 = d_l2;
    lv.size = nbits;
    lv.status = d_status;
    ProfScope ps("bv_rank", stream);
    bv_rank_kernel<<<bv_grid(bv_rank_kernel, q), kBvThreads, 0, stream>>>(lv, d_i, d_out, q, d_status);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

extern "C" wt_status wt_bitvector_select(const uint64_t* d_words, uint64_t nbits, uint64_t ones, uint32_t b,
                                         const uint64_t* d_l1, const uint16_t* d_l2, const uint64_t* d_s0,
                                         const uint64_t* d_s1, uint32_t sample_k, const uint64_t* d_j,
                                         uint64_t* d_out, uint64_t q, uint32_t* d_status, wt_stream stream) {
    if (nbits == 0 || b > 1 || ones > nbits || (reinterpret_cast<uintptr_t>(d_words) & 31u)) return WT_EINVAL;
    if (sample_k < 256 || sample_k > (1u << 20) || (sample_k & (sample_k - 1))) return WT_EINVAL;
    if (!bv_dev(d_words) || !bv_dev(d_l1) || !bv_dev(d_l2) || !bv_dev(d_s0) || !bv_dev(d_s1)) return WT_EINVAL;
    if (d_status && !bv_dev(d_status)) return WT_EINVAL;
    if (!q) return WT_OK;
    if (!bv_dev(d_j) || !bv_dev(d_out)) return WT_EINVAL;
    uint32_t k_log2 = 0;
    while ((1u << k_log2) < sample_k) k_log2++;
    LevelDesc lv = {};
    lv.words = d_words;
    lv.l1 = d_l1;
    lv.l2 = d_l2;
    lv.s0 = d_s0;
    lv.s1 = d_s1;
    lv.size = nbits;
    lv.ones = ones;
    lv.status = d_status;
    ProfScope ps(b ? "bv_select1" : "bv_select0", stream);
    bv_select_kernel<<<bv_grid(bv_select_kernel, q), kBvThreads, 0, stream>>>(lv, b, k_log2, d_j, d_out, q,
                                                                              d_status);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}
