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
    uint32_t is_view;         // a tree of a batch (wt_batch_tree): memory belongs to the batch
    uint32_t has_alloc;       // 1: memory comes from `alloc` (wt_options.allocator), else the device's pool
    wt_allocator alloc;
    uint64_t magic;
};

constexpr uint64_t kTreeMagic = 0x5754475233303031ull;

namespace wt {

// ---- launch accounting / timing (wt_profile.cu) ----
void prof_before(const char* name, cudaStream_t s);
void prof_after(const char* name, cudaStream_t s);
void prof_count(const char* name, uint64_t n);  // count launches without timing them (graph runs)

struct ProfScope {
    const char* n;
    cudaStream_t s;
    ProfScope(const char* name, cudaStream_t st) : n(name), s(st) { prof_before(n, s); }
    ~ProfScope() { prof_after(n, s); }
};

// ---- memory (wt_api.cu) ----
// Device memory comes from the caller's allocator when one is given (null:
// the device's stream-ordered pool).  A failed allocation returns
// cudaErrorMemoryAllocation.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s, const wt_allocator* a = nullptr);
void dev_free(void* p, cudaStream_t s, const wt_allocator* a = nullptr);
inline const wt_allocator* tree_alloc(const wt_tree_s* t) { return t->has_alloc ? &t->alloc : nullptr; }

// True if p is memory a kernel on the current device may dereference: device
// memory of this device, or managed memory.
bool device_ptr_ok(const void* p);

// ---- build (wt_build.cu) ----
// layout: WT_LAYOUT_TREE or WT_LAYOUT_MATRIX.  h_src (optional): host symbols to
// copy into d_symbols (a device buffer of n symbols, allocated on the copy
// stream cs) chunk by chunk on cs during the histogram.
wt_status build_tree(const void* d_symbols, uint64_t n, uint32_t sigma, uint32_t w, uint32_t sample_k,
                     cudaStream_t s, wt_tree_s* t, uint32_t layout = 0, const void* h_src = nullptr,
                     cudaStream_t cs = nullptr);

// out[k] = sum of in[0..k) for k <= count (count + 1 entries); tmp holds
// 2 * (ceil(count / 8192) + 1) entries
void device_exclusive_scan(const uint64_t* in, uint64_t* out, uint64_t count, uint64_t* tmp, cudaStream_t s,
                           const char* name = "scan");

// ---- learned select (wt_learned.cu) ----
wt_status train_select(wt_tree_s* t, uint32_t mode, uint32_t steps, float lr, uint32_t pairs, cudaStream_t s);
wt_status launch_select_learned(const wt_tree_s* t, const uint32_t* d_c, const uint64_t* d_j, uint64_t* d_out,
                                uint64_t q, cudaStream_t s);
void free_learned(wt_tree_s* t, cudaStream_t s);
wt_status export_learned(const wt_tree_s* t, uint32_t level, uint32_t b, bool resid, void* h_dst, uint64_t* count);

// ---- batches of trees (wt_batch.cu, built by wt_build.cu) ----
struct BatchTreeInfo {
    const void* sym;
    uint64_t n;
    uint32_t sigma;
    uint32_t L;
    uint64_t nslots;           // 2^L - 1
    uint64_t* hist;            // sigma
    uint64_t* C;               // sigma + 1
    NodeEntry* nodes;          // nslots (at least 1)
    uint64_t* left;            // nslots
    uint64_t* excl;            // nslots + 1
    uint32_t* status;
    uint64_t s0[kMaxLevels];   // first symbol whose code has length <= l (sigma if none)
};

struct BatchDev {
    uint32_t ntrees, w, maxL, k_log2;
    uint32_t lp_ctas;                // CTAs per SM of the persistent level pass
    uint64_t total_chunks, total_slots;
    BatchTreeInfo* info;
    TreeDesc* desc;
    LevelPassArgs* lpa;              // [maxL][ntrees]
    uint64_t* tiles;                 // [maxL][ntrees]
    uint64_t* tile_prefix;           // [maxL][ntrees + 1]
    unsigned long long* counters;    // [maxL]
    uint64_t* chunk_prefix;          // [ntrees + 1] histogram chunks per tree
    uint64_t* slot_prefix;           // [ntrees + 1] node slots per tree
    uint64_t* hist_pool;
    size_t hist_bytes;
    uint64_t* state_pool;
    size_t state_bytes;
    uint32_t* status_pool;           // [ntrees]
};

constexpr uint64_t kBatchChunk = 65536;  // symbols per histogram work item (small alphabets)
constexpr uint32_t kBatchSmemBins = 16384;  // histogram bins counted in shared memory at once
// Symbols per histogram work item of a tree: alphabets above kBatchSmemBins
// are counted in shared memory one window of bins at a time, over larger
// chunks, so that each bin is flushed to the tree's histogram once per window.
inline __host__ __device__ uint64_t batch_chunk(uint32_t sigma) {
    return sigma > kBatchSmemBins ? (1ull << 20) : kBatchChunk;
}

wt_status enqueue_batch_build(const BatchDev& b, cudaStream_t s, uint32_t* kernels);
uint64_t batch_tile_elems(uint32_t w);

// ---- queries (wt_query.cu) ----
// Large batches are sorted by where their walks go before walking (wt_query.cu):
// the sorted arguments, symbols and kinds and each sorted query's original index;
// mem (one pool allocation) must be freed by the caller on the same stream.
struct Ordered {
    void* mem = nullptr;
    uint8_t* kind = nullptr;
    uint32_t* c = nullptr;
    uint64_t* a = nullptr;
    uint32_t* idx = nullptr;
};
bool use_order(const wt_tree_s* t, uint64_t q);
// the batch sorted by walk key (ord = true), or copied as it is (small batches), into o
wt_status prepare_order(const wt_tree_s* t, uint32_t kind, const uint8_t* d_kind, const uint32_t* d_c,
                        const uint64_t* d_a, uint64_t q, cudaStream_t s, Ordered& o, bool& ord);
// the walk of a prepared batch: answer k of the original order lands in d_out[k]
wt_status walk_prepared(const wt_tree_s* t, uint32_t kind, bool ord, const Ordered& o, void* d_out, uint64_t q,
                        cudaStream_t s);
// kindsel: 0 access, 1 rank, 2 select, 3 mixed (d_kind per query)
wt_status order_queries(const wt_tree_s* t, uint32_t kindsel, const uint8_t* d_kind, const uint32_t* d_c,
                        const uint64_t* d_a, uint64_t q, cudaStream_t s, Ordered& o);

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
