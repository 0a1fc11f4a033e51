// Batches of independent trees built and queried by one CUDA graph launch.
//
// wt_batch_create lays out every tree's memory in one allocation (worst-case
// sizes from n and sigma, so nothing has to be read back), writes the per-tree
// descriptors, and captures into one CUDA graph: the batched histogram, C,
// node tables and level sizes (wt_build.cu), one persistent level-pass kernel
// per level that walks the tiles of all trees, and the registered query batch.
// wt_batch_run launches that graph; no host synchronisation happens inside it.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "wt_internal.hpp"
#include "wt_walk.cuh"

struct wt_batch_s {
    uint64_t magic;
    int device;
    uint32_t ntrees, w, K, query_threads;
    wt::BatchDev dev;
    void* mem;
    size_t mem_bytes;
    std::vector<wt::TreeDesc> h_desc;  // device pointers filled, sizes zero (computed on the device)
    std::vector<uint32_t> L;
    // registered queries
    const uint32_t* q_tree;
    const uint8_t* q_kind;
    const uint32_t* q_c;
    const uint64_t* q_arg;
    uint64_t* q_out;
    uint64_t q;
    // captured graph
    cudaStream_t cap_stream;
    uint32_t has_alloc;  // the one allocation came from `alloc` (wt_batch_options.allocator)
    wt_allocator alloc;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    uint32_t graph_kernels;
};

constexpr uint64_t kBatchMagic = 0x5754424154434831ull;

namespace wt {

constexpr int kBqMaxThreads = 512;
__device__ const NodeCache kNoCache = {nullptr, 0};

__global__ void __launch_bounds__(kBqMaxThreads) batch_query_kernel(const TreeDesc* __restrict__ desc, uint32_t ntrees,
                                                                    const uint32_t* __restrict__ qt,
                                                                    const uint8_t* __restrict__ kind,
                                                                    const uint32_t* __restrict__ qc,
                                                                    const uint64_t* __restrict__ qa,
                                                                    uint64_t* __restrict__ out, uint64_t q) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < q; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t tr = __ldg(qt + k);
        if (tr >= ntrees) {
            out[k] = UINT64_MAX;
            continue;  // no tree to flag: the batch status reports it through tree 0
        }
        const TreeDesc& t = desc[tr];
        const uint32_t kd = __ldg(kind + k);
        const uint64_t x = __ldg(qa + k);
        uint64_t r = UINT64_MAX;
        bool bad;
        if (kd == 0) {
            bad = x >= t.n;
            if (!bad) r = do_access(t, kNoCache, x);
        } else if (kd == 1) {
            const uint32_t c = __ldg(qc + k);
            bad = c >= t.cp.sigma || x > t.n;
            if (!bad) r = do_rank(t, kNoCache, c, x);
        } else if (kd == 2) {
            const uint32_t c = __ldg(qc + k);
            bad = !select_valid(t, c, x);
            if (!bad) r = do_select(t, kNoCache, c, x);
        } else {
            bad = true;
        }
        out[k] = r;
        if (bad) atomicOr(t.status, kStQuery);
    }
}

static uint64_t al(uint64_t x, uint64_t a = 256) { return (x + a - 1) / a * a; }

static bool is_dev(const void* p) { return device_ptr_ok(p); }

static wt_status capture(wt_batch_s* b) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaStream_t s = b->cap_stream;
    WT_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    uint32_t nk = 0;
    wt_status st = enqueue_batch_build(b->dev, s, &nk);
    if (st == WT_OK && b->q) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_query_kernel, (int)b->query_threads, 0);
        if (per_sm <= 0) per_sm = 1;
        const uint64_t need = (b->q + b->query_threads - 1) / b->query_threads;
        const uint64_t full = (uint64_t)per_sm * sm_count();
        batch_query_kernel<<<(unsigned)(need < full ? need : full), b->query_threads, 0, s>>>(
            b->dev.desc, b->ntrees, b->q_tree, b->q_kind, b->q_c, b->q_arg, b->q_out, b->q);
        nk++;
        if (cudaGetLastError() != cudaSuccess) st = WT_ECUDA;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s, &g);
    if (st != WT_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (ec != cudaSuccess) return WT_ECUDA;
    b->graph = g;
    WT_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
    b->graph_kernels = nk;
    return WT_OK;
}

}  // namespace wt

using namespace wt;

static bool batch_ok(const wt_batch_s* b) { return b && b->magic == kBatchMagic; }

static void batch_free(wt_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->mem) {
        if (b->has_alloc) {
            b->alloc.free(b->mem, nullptr, b->alloc.ctx);
        } else {
            cudaFree(b->mem);
        }
    }
    b->magic = 0;
    delete b;
}

extern "C" {

wt_status wt_batch_create(uint32_t ntrees, const void* const* h_symbols, const uint64_t* h_n, const uint32_t* h_sigma,
                          uint32_t symbol_bytes, const wt_batch_options* opt, wt_batch* out) {
    if (!out) return WT_EINVAL;
    *out = nullptr;
    if (ntrees == 0 || ntrees > (1u << 20) || !h_symbols || !h_n || !h_sigma) return WT_EINVAL;
    if (symbol_bytes != 1 && symbol_bytes != 2 && symbol_bytes != 4) return WT_EINVAL;
    const uint32_t K = (opt && opt->sample_k) ? opt->sample_k : 4096u;
    if (K < 256 || K > (1u << 20) || (K & (K - 1))) return WT_EINVAL;
    const uint32_t qthreads = (opt && opt->query_threads) ? opt->query_threads : 256u;
    const wt_allocator* alloc = opt ? opt->allocator : nullptr;
    if (alloc && (!alloc->alloc || !alloc->free)) return WT_EINVAL;
    const uint32_t lp_ctas = (opt && opt->lp_ctas_per_sm) ? opt->lp_ctas_per_sm : 6u;
    if (lp_ctas > 6) return WT_EINVAL;
    if (qthreads != 128 && qthreads != 256 && qthreads != 512) return WT_EINVAL;
    for (uint32_t i = 0; i < ntrees; i++) {
        const uint32_t sg = h_sigma[i];
        if (sg == 0 || sg > (1u << kMaxSigmaLog)) return WT_EINVAL;
        if (symbol_bytes < 4 && (uint64_t)sg > (1ull << (8 * symbol_bytes))) return WT_EINVAL;
        if (h_n[i] >= (1ull << 40)) return WT_EINVAL;
        if (h_n[i]) {
            if (!is_dev(h_symbols[i]) || (reinterpret_cast<uintptr_t>(h_symbols[i]) & 15u)) return WT_EINVAL;
        }
    }
    uint32_t kl = 0;
    while ((1u << kl) < K) kl++;
    const uint32_t w = symbol_bytes;
    const uint64_t te = batch_tile_elems(w);

    wt_batch_s* b = new wt_batch_s();
    b->magic = kBatchMagic;
    cudaGetDevice(&b->device);
    b->ntrees = ntrees;
    b->w = w;
    b->K = K;
    b->query_threads = qthreads;
    b->L.resize(ntrees);
    std::vector<CodeParams> cps(ntrees);
    uint32_t maxL = 0;
    for (uint32_t i = 0; i < ntrees; i++) {
        cps[i] = make_code_params(h_sigma[i]);
        b->L[i] = cps[i].L;
        maxL = cps[i].L > maxL ? cps[i].L : maxL;
    }

    // ---- layout: globals, pools, then one block per tree ----
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) {
        const uint64_t o = off;
        off = al(off + (bytes ? bytes : 8));
        return o;
    };
    const uint64_t o_info = take((uint64_t)ntrees * sizeof(BatchTreeInfo));
    const uint64_t o_desc = take((uint64_t)ntrees * sizeof(TreeDesc));
    const uint64_t o_lpa = take((uint64_t)maxL * ntrees * sizeof(LevelPassArgs));
    const uint64_t o_tiles = take((uint64_t)maxL * ntrees * 8);
    const uint64_t o_tpre = take((uint64_t)maxL * (ntrees + 1) * 8);
    const uint64_t o_cnt = take((uint64_t)(maxL ? maxL : 1) * 8);
    const uint64_t o_cpre = take((uint64_t)(ntrees + 1) * 8);
    const uint64_t o_spre = take((uint64_t)(ntrees + 1) * 8);
    const uint64_t o_status = take((uint64_t)ntrees * 4);
    uint64_t hist_total = 0, state_total = 0;
    for (uint32_t i = 0; i < ntrees; i++) {
        hist_total += al((uint64_t)h_sigma[i] * 8);
        state_total += al(((h_n[i] + te - 1) / te) * 8);
    }
    const uint64_t o_hist = take(hist_total);
    const uint64_t o_state = take(state_total);
    struct TreeOff {
        uint64_t C, nodes, left, excl, tbuf[2];
        std::vector<uint64_t> words, l1, l2, s0, s1, walloc;
    };
    std::vector<TreeOff> to(ntrees);
    for (uint32_t i = 0; i < ntrees; i++) {
        const uint64_t n = h_n[i];
        const uint32_t L = cps[i].L;
        const uint64_t nslots = L ? ((1ull << L) - 1) : 0;
        TreeOff& t = to[i];
        t.C = take(((uint64_t)h_sigma[i] + 1) * 8);
        t.nodes = take((nslots ? nslots : 1) * sizeof(NodeEntry));
        t.left = take((nslots ? nslots : 1) * 8);
        t.excl = take((nslots + 1) * 8);
        t.tbuf[0] = take(L > 1 ? n * w : 0);
        t.tbuf[1] = take(L > 2 ? n * w : 0);
        for (uint32_t l = 0; l < L; l++) {
            const uint64_t wa = al((n + 63) / 64 + 16, 16);
            t.walloc.push_back(wa);
            t.words.push_back(take(wa * 8));
            t.l1.push_back(take((n / kL1Bits + 1) * 8));
            t.l2.push_back(take((n / kL2Bits + 1) * 2));
            t.s0.push_back(take(((n >> kl) + 2) * 8));
            t.s1.push_back(take(((n >> kl) + 2) * 8));
        }
    }
    if (alloc) {
        b->has_alloc = 1;
        b->alloc = *alloc;
        b->mem = alloc->alloc(off, nullptr, alloc->ctx);  // legacy default stream, synchronised below
        if (b->mem && cudaStreamSynchronize(nullptr) != cudaSuccess) {
            batch_free(b);
            return WT_ECUDA;
        }
    } else if (cudaMalloc(&b->mem, off) != cudaSuccess) {
        b->mem = nullptr;
    }
    if (!b->mem) {
        cudaGetLastError();
        delete b;
        return WT_ENOMEM;
    }
    b->mem_bytes = off;
    uint8_t* M = static_cast<uint8_t*>(b->mem);
    if (cudaMemset(M, 0, off) != cudaSuccess) {
        batch_free(b);
        return WT_ECUDA;
    }

    // ---- host-side descriptors ----
    std::vector<BatchTreeInfo> info(ntrees);
    b->h_desc.assign(ntrees, TreeDesc());
    std::vector<LevelPassArgs> lpa((size_t)maxL * ntrees);
    memset(lpa.data(), 0, lpa.size() * sizeof(LevelPassArgs));
    std::vector<uint64_t> cpre(ntrees + 1, 0), spre(ntrees + 1, 0);
    uint64_t hist_off = o_hist, state_off = o_state;
    for (uint32_t i = 0; i < ntrees; i++) {
        const uint64_t n = h_n[i];
        const uint32_t L = cps[i].L;
        const uint64_t nslots = L ? ((1ull << L) - 1) : 0;
        BatchTreeInfo& ti = info[i];
        memset(&ti, 0, sizeof(ti));
        ti.sym = h_symbols[i];
        ti.n = n;
        ti.sigma = h_sigma[i];
        ti.L = L;
        ti.nslots = nslots;
        ti.hist = reinterpret_cast<uint64_t*>(M + hist_off);
        hist_off += al((uint64_t)h_sigma[i] * 8);
        ti.C = reinterpret_cast<uint64_t*>(M + to[i].C);
        ti.nodes = reinterpret_cast<NodeEntry*>(M + to[i].nodes);
        ti.left = reinterpret_cast<uint64_t*>(M + to[i].left);
        ti.excl = reinterpret_cast<uint64_t*>(M + to[i].excl);
        ti.status = reinterpret_cast<uint32_t*>(M + o_status) + i;
        for (uint32_t l = 0; l < L; l++) {
            uint64_t s0 = h_sigma[i];
            for (uint32_t k = 0; k < cps[i].r; k++) {
                const uint32_t len = cps[i].pow2 ? cps[i].L : (k + 1 < cps[i].r ? k + 1 + cps[i].e[k] : cps[i].r - 1 + cps[i].e[k]);
                if (len <= l) {
                    s0 = cps[i].P[k];
                    break;
                }
            }
            ti.s0[l] = s0;
        }
        TreeDesc& d = b->h_desc[i];
        memset(&d, 0, sizeof(d));
        d.cp = cps[i];
        d.n = n;
        d.k_log2 = kl;
        d.nodes = ti.nodes;
        d.C = ti.C;
        d.status = ti.status;
        uint64_t* state = reinterpret_cast<uint64_t*>(M + state_off);
        state_off += al(((n + te - 1) / te) * 8);
        for (uint32_t l = 0; l < L; l++) {
            LevelDesc& v = d.lv[l];
            v.words = reinterpret_cast<uint64_t*>(M + to[i].words[l]);
            v.l1 = reinterpret_cast<uint64_t*>(M + to[i].l1[l]);
            v.l2 = reinterpret_cast<uint16_t*>(M + to[i].l2[l]);
            v.s0 = reinterpret_cast<uint64_t*>(M + to[i].s0[l]);
            v.s1 = reinterpret_cast<uint64_t*>(M + to[i].s1[l]);
            v.status = ti.status;
            LevelPassArgs& a = lpa[(size_t)l * ntrees + i];
            a.src = l == 0 ? h_symbols[i] : static_cast<const void*>(M + to[i].tbuf[(l - 1) & 1]);
            a.dst = (l + 1 < L) ? static_cast<void*>(M + to[i].tbuf[l & 1]) : nullptr;
            a.words_alloc = to[i].walloc[l];
            a.words = const_cast<uint64_t*>(v.words);
            a.l1 = const_cast<uint64_t*>(v.l1);
            a.l2 = const_cast<uint16_t*>(v.l2);
            a.s0 = const_cast<uint64_t*>(v.s0);
            a.s1 = const_cast<uint64_t*>(v.s1);
            a.nodes = ti.nodes + ((1ull << l) - 1);
            a.state = state;
            a.status = ti.status;
            a.level = l;
            a.shift_bit = L - 1 - l;
            a.pshift = L - l;
            a.level_nodes = 1ull << l;
            a.k_log2 = kl;
            a.ctab_n = 0;
            a.cp = cps[i];
        }
        cpre[i + 1] = cpre[i] + (n + batch_chunk(h_sigma[i]) - 1) / batch_chunk(h_sigma[i]);
        spre[i + 1] = spre[i] + nslots;
    }
    BatchDev& bd = b->dev;
    bd.ntrees = ntrees;
    bd.w = w;
    bd.maxL = maxL;
    bd.k_log2 = kl;
    bd.lp_ctas = lp_ctas;
    bd.total_chunks = cpre[ntrees];
    bd.total_slots = spre[ntrees];
    bd.info = reinterpret_cast<BatchTreeInfo*>(M + o_info);
    bd.desc = reinterpret_cast<TreeDesc*>(M + o_desc);
    bd.lpa = reinterpret_cast<LevelPassArgs*>(M + o_lpa);
    bd.tiles = reinterpret_cast<uint64_t*>(M + o_tiles);
    bd.tile_prefix = reinterpret_cast<uint64_t*>(M + o_tpre);
    bd.counters = reinterpret_cast<unsigned long long*>(M + o_cnt);
    bd.chunk_prefix = reinterpret_cast<uint64_t*>(M + o_cpre);
    bd.slot_prefix = reinterpret_cast<uint64_t*>(M + o_spre);
    bd.hist_pool = reinterpret_cast<uint64_t*>(M + o_hist);
    bd.hist_bytes = hist_total;
    bd.state_pool = reinterpret_cast<uint64_t*>(M + o_state);
    bd.state_bytes = state_total;
    bd.status_pool = reinterpret_cast<uint32_t*>(M + o_status);
    bool ok = cudaMemcpy(bd.info, info.data(), ntrees * sizeof(BatchTreeInfo), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(bd.desc, b->h_desc.data(), ntrees * sizeof(TreeDesc), cudaMemcpyHostToDevice) == cudaSuccess &&
              (lpa.empty() || cudaMemcpy(bd.lpa, lpa.data(), lpa.size() * sizeof(LevelPassArgs),
                                         cudaMemcpyHostToDevice) == cudaSuccess) &&
              cudaMemcpy(bd.chunk_prefix, cpre.data(), cpre.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(bd.slot_prefix, spre.data(), spre.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        batch_free(b);
        return WT_ECUDA;
    }
    const wt_status st = capture(b);
    if (st != WT_OK) {
        batch_free(b);
        return st;
    }
    *out = b;
    return WT_OK;
}

wt_status wt_batch_set_queries(wt_batch batch, const uint32_t* d_tree, const uint8_t* d_kind, const uint32_t* d_c,
                               const uint64_t* d_arg, uint64_t* d_out, uint64_t q) {
    if (!batch_ok(batch)) return WT_EINVAL;
    if (q && (!is_dev(d_tree) || !is_dev(d_kind) || !is_dev(d_c) || !is_dev(d_arg) || !is_dev(d_out))) return WT_EINVAL;
    batch->q_tree = d_tree;
    batch->q_kind = d_kind;
    batch->q_c = d_c;
    batch->q_arg = d_arg;
    batch->q_out = d_out;
    batch->q = q;
    return capture(batch);
}

wt_status wt_batch_run(wt_batch batch, wt_stream stream) {
    if (!batch_ok(batch) || !batch->exec) return WT_EINVAL;
    prof_count("batch_graph", batch->graph_kernels);
    return cudaGraphLaunch(batch->exec, stream) == cudaSuccess ? WT_OK : WT_ECUDA;
}

wt_status wt_batch_status_sync(wt_batch batch, wt_stream stream) {
    if (!batch_ok(batch)) return WT_EINVAL;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return WT_ECUDA;
    std::vector<uint32_t> st(batch->ntrees);
    if (cudaMemcpy(st.data(), batch->dev.status_pool, st.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return WT_ECUDA;
    uint32_t bits = 0;
    for (uint32_t v : st) bits |= v;
    if (bits && cudaMemset(batch->dev.status_pool, 0, st.size() * 4) != cudaSuccess) return WT_ECUDA;
    if (bits & kStBounds) return WT_EBOUNDS;
    if (bits & kStTimeout) return WT_ETIMEOUT;
    if (bits & kStSymbol) return WT_ESYMBOL;
    if (bits & kStQuery) return WT_EQUERY;
    return WT_OK;
}

wt_status wt_batch_tree(wt_batch batch, uint32_t index, wt_tree* out) {
    if (!batch_ok(batch) || !out || index >= batch->ntrees) return WT_EINVAL;
    *out = nullptr;
    if (cudaDeviceSynchronize() != cudaSuccess) return WT_ECUDA;
    wt_tree_s* t = new wt_tree_s();
    if (cudaMemcpy(&t->desc, batch->dev.desc + index, sizeof(TreeDesc), cudaMemcpyDeviceToHost) != cudaSuccess) {
        delete t;
        return WT_ECUDA;
    }
    t->stream = nullptr;
    t->device = batch->device;
    t->symbol_bytes = batch->w;
    t->sample_k = batch->K;
    for (uint32_t l = 0; l < t->desc.cp.L; l++) {
        t->level_size[l] = t->desc.lv[l].size;
        t->level_ones[l] = t->desc.lv[l].ones;
    }
    t->is_view = 1;
    t->magic = kTreeMagic;
    *out = t;
    return WT_OK;
}

void wt_batch_destroy(wt_batch batch) {
    if (!batch_ok(batch)) return;
    cudaDeviceSynchronize();
    batch_free(batch);
}

uint64_t wt_batch_bytes(wt_batch batch) { return batch_ok(batch) ? batch->mem_bytes : 0; }

}  // extern "C"
