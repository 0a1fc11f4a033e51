// Host-side internals of libwt: the tree object, allocation and launch
// accounting.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_common.cuh"

struct wt_tree_s {
    wt::TreeDesc desc;        // device pointers + code parameters, passed to query kernels
    cudaStream_t stream;      // build stream (tree memory is freed on it)
    int device;
    uint32_t symbol_bytes;
    uint32_t sample_k;
    uint64_t level_size[wt::kMaxLevels];
    uint64_t level_ones[wt::kMaxLevels];
    void* hdr_mem;            // C, node table, status
    size_t hdr_bytes;
    void* lvl_mem;            // bit arrays, L1, L2, samples of every level
    size_t lvl_bytes;
    // learned select (wt_train_select): per-segment error bounds, MLP parameters, counters
    wt::LearnedDesc learned;
    void* learned_mem;
    size_t learned_bytes;
    uint64_t magic;
};

constexpr uint64_t kTreeMagic = 0x5754475233303031ull;

namespace wt {

// ---- launch accounting / timing (wt_profile.cu) ----
void prof_before(const char* name, cudaStream_t s);
void prof_after(const char* name, cudaStream_t s);

struct ProfScope {
    const char* n;
    cudaStream_t s;
    ProfScope(const char* name, cudaStream_t st) : n(name), s(st) { prof_before(n, s); }
    ~ProfScope() { prof_after(n, s); }
};

// ---- memory (wt_api.cu) ----
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

// ---- build (wt_build.cu) ----
wt_status build_tree(const void* d_symbols, uint64_t n, uint32_t sigma, uint32_t w, uint32_t sample_k,
                     cudaStream_t s, wt_tree_s* t);

// ---- learned select (wt_learned.cu) ----
wt_status train_select(wt_tree_s* t, uint32_t mode, uint32_t steps, float lr, uint32_t pairs, cudaStream_t s);
wt_status launch_select_learned(const wt_tree_s* t, const uint32_t* d_c, const uint64_t* d_j, uint64_t* d_out,
                                uint64_t q, cudaStream_t s);
void free_learned(wt_tree_s* t, cudaStream_t s);

// ---- queries (wt_query.cu) ----
wt_status launch_access(const wt_tree_s* t, const uint64_t* d_i, uint32_t* d_out, uint64_t q, cudaStream_t s);
wt_status launch_rank(const wt_tree_s* t, const uint32_t* d_c, const uint64_t* d_i, uint64_t* d_out, uint64_t q,
                      cudaStream_t s);
wt_status launch_select(const wt_tree_s* t, const uint32_t* d_c, const uint64_t* d_j, uint64_t* d_out, uint64_t q,
                        cudaStream_t s);
wt_status launch_mixed(const wt_tree_s* t, const uint8_t* d_kind, const uint32_t* d_c, const uint64_t* d_arg,
                       uint64_t* d_out, uint64_t q, cudaStream_t s);

int sm_count();

}  // namespace wt

#define WT_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return (_e == cudaErrorMemoryAllocation ? WT_ENOMEM : WT_ECUDA); \
    } while (0)
