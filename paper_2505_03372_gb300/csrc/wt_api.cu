// extern "C" entry points of libwt (declared in include/wt.h), device memory
// and launch accounting.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "wt_internal.hpp"

namespace wt {

// ---------------------------------------------------------------------------
// device memory: stream-ordered pool allocations, kept cached in the pool
// ---------------------------------------------------------------------------

static std::once_flag g_pool_once;

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s, const wt_allocator* a) {
    if (bytes == 0) bytes = 256;
    if (a) {
        *p = a->alloc(bytes, s, a->ctx);
        return *p ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    std::call_once(g_pool_once, [] {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;  // keep freed blocks for reuse by later builds
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
    return cudaMallocAsync(p, bytes, s);
}

void dev_free(void* p, cudaStream_t s, const wt_allocator* a) {
    if (!p) return;
    if (a) a->free(p, s, a->ctx);
    else cudaFreeAsync(p, s);
}

bool device_ptr_ok(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // clear the error this query left
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    if (at.type != cudaMemoryTypeDevice) return false;
    int dev = -1;
    return cudaGetDevice(&dev) == cudaSuccess && at.device == dev;
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// ---------------------------------------------------------------------------
// launch accounting and optional event timing
// ---------------------------------------------------------------------------

struct KStat {
    uint64_t launches = 0;
    double ms = 0.0;
};
struct Pending {
    std::string name;
    cudaEvent_t a, b;
};

static std::mutex g_mu;
static std::map<std::string, KStat> g_stats;
static std::vector<Pending> g_pending;
static std::vector<cudaEvent_t> g_free_events;
static std::atomic<uint64_t> g_launches{0};
static std::atomic<int> g_timing{0};
static thread_local cudaEvent_t tl_start = nullptr;

static cudaEvent_t take_event() {
    if (!g_free_events.empty()) {
        cudaEvent_t e = g_free_events.back();
        g_free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_before(const char* name, cudaStream_t s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    std::lock_guard<std::mutex> lk(g_mu);
    g_stats[name].launches++;
    if (g_timing.load()) {
        tl_start = take_event();
        cudaEventRecord(tl_start, s);
    }
}

void prof_count(const char* name, uint64_t n) {
    g_launches.fetch_add(n, std::memory_order_relaxed);
    std::lock_guard<std::mutex> lk(g_mu);
    g_stats[name].launches += n;
}

void prof_after(const char* name, cudaStream_t s) {
    if (!g_timing.load() || !tl_start) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = take_event();
    cudaEventRecord(b, s);
    g_pending.push_back({name, tl_start, b});
    tl_start = nullptr;
}

static void collect_pending() {
    for (auto& p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
            g_stats[p.name].ms += ms;
        g_free_events.push_back(p.a);
        g_free_events.push_back(p.b);
    }
    g_pending.clear();
}

// ---------------------------------------------------------------------------
// argument checks
// ---------------------------------------------------------------------------

static bool is_device_ptr(const void* p) { return device_ptr_ok(p); }

static bool tree_ok(const wt_tree_s* t) { return t && t->magic == kTreeMagic; }

// True if p is host memory (pinned or pageable), not device or managed memory.
static bool is_host_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;  // unknown to CUDA: ordinary pageable memory
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

// The library's copy streams of the current device (host-to-device and
// device-to-host staging of wt_build_host and wt_query_host), created on first
// use and kept for the life of the process.  A device reset destroys them: the
// next call on that device after a reset fails with WT_ECUDA.
struct Staging {
    cudaStream_t h2d, d2h;
};
static bool staging_streams(Staging* out) {
    static std::mutex mu;
    static cudaStream_t st[256][2];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return false;
    std::lock_guard<std::mutex> lk(mu);
    for (int k = 0; k < 2; k++)
        if (!st[dev][k] && cudaStreamCreateWithFlags(&st[dev][k], cudaStreamNonBlocking) != cudaSuccess) {
            st[dev][k] = nullptr;
            return false;
        }
    out->h2d = st[dev][0];
    out->d2h = st[dev][1];
    return true;
}

// `waiter` waits for the work queued on `on` so far (an event; a host
// synchronisation if no event can be made).
static void order_after(cudaStream_t waiter, cudaStream_t on) {
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess && cudaEventRecord(ev, on) == cudaSuccess &&
        cudaStreamWaitEvent(waiter, ev, 0) == cudaSuccess) {
        cudaEventDestroy(ev);
        return;
    }
    if (ev) cudaEventDestroy(ev);
    cudaStreamSynchronize(on);
}

static wt_tree_s* new_tree(cudaStream_t stream, const wt_allocator* alloc) {
    wt_tree_s* t = new wt_tree_s();
    memset(&t->desc, 0, sizeof(t->desc));
    cudaGetDevice(&t->device);
    t->stream = stream;
    t->has_alloc = alloc != nullptr;
    if (alloc) t->alloc = *alloc;
    t->magic = kTreeMagic;
    return t;
}

static void release_tree(wt_tree_s* t) {
    free_learned(t, t->stream);
    dev_free(t->hdr_mem, t->stream, tree_alloc(t));
    dev_free(t->lvl_mem, t->stream, tree_alloc(t));
    t->magic = 0;
    delete t;
}

}  // namespace wt

using namespace wt;

extern "C" {

const char* wt_status_str(wt_status s) {
    switch (s) {
        case WT_OK: return "WT_OK";
        case WT_EINVAL: return "WT_EINVAL: invalid argument";
        case WT_ESYMBOL: return "WT_ESYMBOL: input symbol >= sigma";
        case WT_ENOMEM: return "WT_ENOMEM: device allocation failed";
        case WT_ECUDA: return "WT_ECUDA: CUDA runtime error";
        case WT_EQUERY: return "WT_EQUERY: query argument out of range";
        case WT_ETIMEOUT: return "WT_ETIMEOUT: bounded device wait gave up";
        case WT_EUNSUPPORTED: return "WT_EUNSUPPORTED: operation not available";
        case WT_EBOUNDS: return "WT_EBOUNDS: a query walk's load failed its bounds check (debug library)";
    }
    return "unknown wt_status";
}

wt_status wt_build(const void* d_symbols, uint64_t n, uint32_t sigma, uint32_t symbol_bytes, const wt_options* opt,
                   wt_stream stream, wt_tree* out) {
    if (!out) return WT_EINVAL;
    *out = nullptr;
    if (symbol_bytes != 1 && symbol_bytes != 2 && symbol_bytes != 4) return WT_EINVAL;
    if (sigma == 0 || sigma > (1u << kMaxSigmaLog)) return WT_EINVAL;
    if (symbol_bytes < 4 && (uint64_t)sigma > (1ull << (8 * symbol_bytes))) return WT_EINVAL;
    if (n >= (1ull << 40)) return WT_EINVAL;
    if (n) {
        if (!is_device_ptr(d_symbols)) return WT_EINVAL;
        if (reinterpret_cast<uintptr_t>(d_symbols) & 15u) return WT_EINVAL;
    }
    uint32_t K = (opt && opt->sample_k) ? opt->sample_k : 4096u;
    if (K < 256 || K > (1u << 20) || (K & (K - 1))) return WT_EINVAL;
    const uint32_t layout = opt ? opt->layout : WT_LAYOUT_TREE;
    if (layout != WT_LAYOUT_TREE && layout != WT_LAYOUT_MATRIX) return WT_EINVAL;

    const wt_allocator* alloc = opt ? opt->allocator : nullptr;
    if (alloc && (!alloc->alloc || !alloc->free)) return WT_EINVAL;

    wt_tree_s* t = new_tree(stream, alloc);
    wt_status st = build_tree(d_symbols, n, sigma, symbol_bytes, K, stream, t, layout);
    if (st != WT_OK) {
        release_tree(t);
        return st;
    }
    *out = t;
    return WT_OK;
}

wt_status wt_build_host(const void* h_symbols, uint64_t n, uint32_t sigma, uint32_t symbol_bytes,
                        const wt_options* opt, wt_stream stream, wt_tree* out) {
    if (!out) return WT_EINVAL;
    *out = nullptr;
    if (symbol_bytes != 1 && symbol_bytes != 2 && symbol_bytes != 4) return WT_EINVAL;
    if (sigma == 0 || sigma > (1u << kMaxSigmaLog)) return WT_EINVAL;
    if (symbol_bytes < 4 && (uint64_t)sigma > (1ull << (8 * symbol_bytes))) return WT_EINVAL;
    if (n >= (1ull << 40)) return WT_EINVAL;
    if (n && !is_host_ptr(h_symbols)) return WT_EINVAL;
    uint32_t K = (opt && opt->sample_k) ? opt->sample_k : 4096u;
    if (K < 256 || K > (1u << 20) || (K & (K - 1))) return WT_EINVAL;
    const uint32_t layout = opt ? opt->layout : WT_LAYOUT_TREE;
    if (layout != WT_LAYOUT_TREE && layout != WT_LAYOUT_MATRIX) return WT_EINVAL;
    const wt_allocator* alloc = opt ? opt->allocator : nullptr;
    if (alloc && (!alloc->alloc || !alloc->free)) return WT_EINVAL;
    // The device copy is filled chunk by chunk on the library's copy stream
    // (`stream` waits per chunk).  From the pool it is taken on that copy
    // stream, so the copies need not wait for the work already queued on
    // `stream`; a caller's allocator gets the request on `stream` (the stream
    // it is released on), and the copies then wait for that point.
    Staging sg;
    if (!staging_streams(&sg)) return WT_ECUDA;
    void* d_buf = nullptr;
    if (n && dev_alloc(&d_buf, n * symbol_bytes, alloc ? stream : sg.h2d, alloc) != cudaSuccess) return WT_ENOMEM;
    if (n && alloc) order_after(sg.h2d, stream);
    wt_tree_s* t = new_tree(stream, alloc);
    wt_status st = build_tree(d_buf, n, sigma, symbol_bytes, K, stream, t, layout, h_symbols, sg.h2d);
    if (n) {
        order_after(stream, sg.h2d);     // every chunk copied (also when the build stopped early)
        dev_free(d_buf, stream, alloc);  // after the histogram and the level passes that read it
    }
    if (st != WT_OK) {
        release_tree(t);
        return st;
    }
    *out = t;
    return WT_OK;
}

void wt_destroy(wt_tree tree) {
    if (!tree_ok(tree)) return;
    release_tree(tree);  // a tree of a batch holds no level or header memory of its own
}

wt_status wt_access(wt_tree tree, const uint64_t* d_i, uint32_t* d_out, uint64_t q, wt_stream stream) {
    if (!tree_ok(tree)) return WT_EINVAL;
    if (!q) return WT_OK;
    if (!is_device_ptr(d_i) || !is_device_ptr(d_out)) return WT_EINVAL;
    return launch_access(tree, d_i, d_out, q, stream);
}

wt_status wt_rank(wt_tree tree, const uint32_t* d_c, const uint64_t* d_i, uint64_t* d_out, uint64_t q,
                  wt_stream stream) {
    if (!tree_ok(tree)) return WT_EINVAL;
    if (!q) return WT_OK;
    if (!is_device_ptr(d_c) || !is_device_ptr(d_i) || !is_device_ptr(d_out)) return WT_EINVAL;
    return launch_rank(tree, d_c, d_i, d_out, q, stream);
}

wt_status wt_select(wt_tree tree, const uint32_t* d_c, const uint64_t* d_j, uint64_t* d_out, uint64_t q,
                    wt_stream stream) {
    if (!tree_ok(tree)) return WT_EINVAL;
    if (!q) return WT_OK;
    if (!is_device_ptr(d_c) || !is_device_ptr(d_j) || !is_device_ptr(d_out)) return WT_EINVAL;
    return launch_select(tree, d_c, d_j, d_out, q, stream);
}

wt_status wt_query_mixed(wt_tree tree, const uint8_t* d_kind, const uint32_t* d_c, const uint64_t* d_arg,
                         uint64_t* d_out, uint64_t q, wt_stream stream) {
    if (!tree_ok(tree)) return WT_EINVAL;
    if (!q) return WT_OK;
    if (!is_device_ptr(d_kind) || !is_device_ptr(d_c) || !is_device_ptr(d_arg) || !is_device_ptr(d_out))
        return WT_EINVAL;
    return launch_mixed(tree, d_kind, d_c, d_arg, d_out, q, stream);
}

// ---------------------------------------------------------------------------
// ordering as a step of its own
// ---------------------------------------------------------------------------

constexpr uint64_t kOrderMagic = 0x5754474f52444552ull;

struct wt_order_s {
    uint64_t magic;
    const wt_tree_s* tree;
    uint32_t kind;
    uint64_t q;
    bool ord;             // sorted by walk key (else the batch as it was given)
    Ordered o;
    cudaEvent_t ready;    // recorded on `stream` after the arrays are written
    cudaStream_t stream;  // the order's stream: its memory is taken and returned there
    uint32_t has_alloc;
    wt_allocator alloc;
};

wt_status wt_order_queries(wt_tree tree, uint32_t kind, const uint8_t* d_kind, const uint32_t* d_c,
                           const uint64_t* d_arg, uint64_t q, wt_stream stream, wt_order* out) {
    if (!out) return WT_EINVAL;
    *out = nullptr;
    if (!tree_ok(tree) || kind > 3) return WT_EINVAL;
    if (tree->is_view) return WT_EUNSUPPORTED;
    if (q && (!is_device_ptr(d_arg) || (kind >= 1 && !is_device_ptr(d_c)) || (kind == 3 && !is_device_ptr(d_kind))))
        return WT_EINVAL;
    wt_order_s* od = new wt_order_s();
    od->magic = kOrderMagic;
    od->tree = tree;
    od->kind = kind;
    od->q = q;
    od->stream = stream;
    od->has_alloc = tree->has_alloc;
    od->alloc = tree->alloc;
    wt_status st = q ? prepare_order(tree, kind, d_kind, d_c, d_arg, q, stream, od->o, od->ord) : WT_OK;
    if (st == WT_OK && cudaEventCreateWithFlags(&od->ready, cudaEventDisableTiming) != cudaSuccess) st = WT_ECUDA;
    if (st == WT_OK && cudaEventRecord(od->ready, stream) != cudaSuccess) st = WT_ECUDA;
    if (st != WT_OK) {
        if (od->o.mem) dev_free(od->o.mem, stream, od->has_alloc ? &od->alloc : nullptr);
        if (od->ready) cudaEventDestroy(od->ready);
        delete od;
        return st;
    }
    *out = od;
    return WT_OK;
}

wt_status wt_walk_ordered(wt_tree tree, wt_order order, void* d_out, wt_stream stream) {
    if (!tree_ok(tree) || !order || order->magic != kOrderMagic || order->tree != tree) return WT_EINVAL;
    if (!order->q) return WT_OK;
    if (!is_device_ptr(d_out)) return WT_EINVAL;
    if (cudaStreamWaitEvent(stream, order->ready, 0) != cudaSuccess) return WT_ECUDA;
    return walk_prepared(tree, order->kind, order->ord, order->o, d_out, order->q, stream);
}

wt_status wt_order_destroy(wt_order order, wt_stream stream) {
    if (!order || order->magic != kOrderMagic) return WT_EINVAL;
    wt_status st = WT_OK;
    if (order->o.mem) {
        // the last walk may still read the arrays on `stream`: the order's stream
        // waits for it, then the memory goes back where it was taken
        cudaEvent_t done = nullptr;
        if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(done, stream) != cudaSuccess || cudaStreamWaitEvent(order->stream, done, 0) != cudaSuccess)
            st = WT_ECUDA;
        if (done) cudaEventDestroy(done);
        if (st != WT_OK) cudaStreamSynchronize(stream);  // no event: wait for the walk on the host instead
        dev_free(order->o.mem, order->stream, order->has_alloc ? &order->alloc : nullptr);
    }
    cudaEventDestroy(order->ready);
    order->magic = 0;
    delete order;
    return st;
}

// ---------------------------------------------------------------------------
// host-resident query pipeline
// ---------------------------------------------------------------------------

namespace {

struct HostPipe {
    cudaStream_t h2d = nullptr, d2h = nullptr;  // the library's copy streams of this device
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_walk[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
    bool ok = true;
    HostPipe() {
        Staging sg;
        ok = staging_streams(&sg);
        h2d = sg.h2d;
        d2h = sg.d2h;
        for (int b = 0; b < 2 && ok; b++)
            ok = cudaEventCreateWithFlags(&ev_in[b], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&ev_walk[b], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&ev_out[b], cudaEventDisableTiming) == cudaSuccess;
    }
    ~HostPipe() {  // destruction is deferred by CUDA until the queued work completes
        for (int b = 0; b < 2; b++) {
            if (ev_in[b]) cudaEventDestroy(ev_in[b]);
            if (ev_walk[b]) cudaEventDestroy(ev_walk[b]);
            if (ev_out[b]) cudaEventDestroy(ev_out[b]);
        }
    }
};

}  // namespace

wt_status wt_query_host(wt_tree tree, uint32_t kind, const uint8_t* h_kind, const uint32_t* h_c,
                        const uint64_t* h_arg, void* h_out, uint64_t q, uint64_t chunk, wt_stream stream) {
    if (!tree_ok(tree) || kind > 3) return WT_EINVAL;
    if (!q) return WT_OK;
    const bool need_c = kind != 0, need_kind = kind == 3;
    if (!is_host_ptr(h_arg) || !is_host_ptr(h_out) || (need_c && !is_host_ptr(h_c)) ||
        (need_kind && !is_host_ptr(h_kind)))
        return WT_EINVAL;
    if (!chunk) chunk = std::min<uint64_t>(q, 1ull << 24);
    chunk = std::min(chunk, q);
    const uint64_t nch = (q + chunk - 1) / chunk;
    const size_t osz = kind == 0 ? 4 : 8;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    // per buffer: arguments, symbols, kinds, answers
    const size_t o_c = al(chunk * 8), o_k = o_c + (need_c ? al(chunk * 4) : 0),
                 o_o = o_k + (need_kind ? al(chunk) : 0), per = o_o + al(chunk * osz);
    const int nbuf = nch > 1 ? 2 : 1;
    HostPipe hp;
    if (!hp.ok) return WT_ECUDA;
    // From the pool the buffers are taken on the copy-in stream (no wait for the
    // work queued on `stream`); a caller's allocator gets the request on
    // `stream`, where they are also released, and the copy-in stream waits.
    const wt_allocator* alloc = tree_alloc(tree);
    void* mem = nullptr;
    if (dev_alloc(&mem, per * nbuf, alloc ? stream : hp.h2d, alloc) != cudaSuccess) return WT_ENOMEM;
    if (alloc) order_after(hp.h2d, stream);
    uint8_t* M = static_cast<uint8_t*>(mem);
    cudaStream_t s = stream;
    wt_status st = WT_OK;
    for (uint64_t i = 0; i < nch && st == WT_OK; i++) {
        const int b = (int)(i & 1);
        const uint64_t off = i * chunk, len = std::min(chunk, q - off);
        uint8_t* B = M + b * per;
        uint64_t* d_arg = reinterpret_cast<uint64_t*>(B);
        uint32_t* d_c = need_c ? reinterpret_cast<uint32_t*>(B + o_c) : nullptr;
        uint8_t* d_kind = need_kind ? B + o_k : nullptr;
        void* d_out = B + o_o;
        // copy in (the buffer's previous chunk has been copied out)
        if (i >= 2 && cudaStreamWaitEvent(hp.h2d, hp.ev_out[b], 0) != cudaSuccess) st = WT_ECUDA;
        if (st == WT_OK && cudaMemcpyAsync(d_arg, h_arg + off, len * 8, cudaMemcpyHostToDevice, hp.h2d) != cudaSuccess)
            st = WT_ECUDA;
        if (st == WT_OK && need_c &&
            cudaMemcpyAsync(d_c, h_c + off, len * 4, cudaMemcpyHostToDevice, hp.h2d) != cudaSuccess)
            st = WT_ECUDA;
        if (st == WT_OK && need_kind &&
            cudaMemcpyAsync(d_kind, h_kind + off, len, cudaMemcpyHostToDevice, hp.h2d) != cudaSuccess)
            st = WT_ECUDA;
        if (st == WT_OK && cudaEventRecord(hp.ev_in[b], hp.h2d) != cudaSuccess) st = WT_ECUDA;
        // walk on the caller's stream
        if (st == WT_OK && cudaStreamWaitEvent(s, hp.ev_in[b], 0) != cudaSuccess) st = WT_ECUDA;
        if (st == WT_OK) {
            switch (kind) {
                case 0: st = launch_access(tree, d_arg, static_cast<uint32_t*>(d_out), len, s); break;
                case 1: st = launch_rank(tree, d_c, d_arg, static_cast<uint64_t*>(d_out), len, s); break;
                case 2: st = launch_select(tree, d_c, d_arg, static_cast<uint64_t*>(d_out), len, s); break;
                default: st = launch_mixed(tree, d_kind, d_c, d_arg, static_cast<uint64_t*>(d_out), len, s); break;
            }
        }
        if (st == WT_OK && cudaEventRecord(hp.ev_walk[b], s) != cudaSuccess) st = WT_ECUDA;
        // copy out
        if (st == WT_OK && cudaStreamWaitEvent(hp.d2h, hp.ev_walk[b], 0) != cudaSuccess) st = WT_ECUDA;
        if (st == WT_OK && cudaMemcpyAsync(static_cast<uint8_t*>(h_out) + off * osz, d_out, len * osz,
                                           cudaMemcpyDeviceToHost, hp.d2h) != cudaSuccess)
            st = WT_ECUDA;
        if (st == WT_OK && cudaEventRecord(hp.ev_out[b], hp.d2h) != cudaSuccess) st = WT_ECUDA;
    }
    // The copy-out stream waits for everything queued on the caller's stream
    // (all walks, even after an error), then the caller's stream waits for the
    // last copy-out; the buffers go back to the pool after both.
    cudaEvent_t walked = nullptr, done = nullptr;
    if (cudaEventCreateWithFlags(&walked, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) {
        cudaStreamSynchronize(s);  // no events: order by waiting on the host instead
        cudaStreamSynchronize(hp.d2h);
        cudaStreamSynchronize(hp.h2d);
        dev_free(mem, alloc ? s : hp.d2h, alloc);
        if (walked) cudaEventDestroy(walked);
        return WT_ECUDA;
    }
    cudaEventRecord(walked, s);
    cudaStreamWaitEvent(hp.d2h, walked, 0);
    cudaEventRecord(done, hp.d2h);
    cudaStreamWaitEvent(s, done, 0);
    dev_free(mem, alloc ? s : hp.d2h, alloc);  // after the last copy-out
    cudaEventDestroy(walked);
    cudaEventDestroy(done);
    return st;
}

wt_status wt_status_sync(wt_tree tree, wt_stream stream) {
    if (!tree_ok(tree)) return WT_EINVAL;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return WT_ECUDA;
    uint32_t bits = 0;
    if (cudaMemcpy(&bits, tree->desc.status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return WT_ECUDA;
    if (bits) {
        if (cudaMemset(tree->desc.status, 0, 4) != cudaSuccess) return WT_ECUDA;
    }
    if (bits & kStBounds) return WT_EBOUNDS;
    if (bits & kStTimeout) return WT_ETIMEOUT;
    if (bits & kStSymbol) return WT_ESYMBOL;
    if (bits & kStQuery) return WT_EQUERY;
    return WT_OK;
}

wt_status wt_info(wt_tree tree, wt_info_t* out) {
    if (!tree_ok(tree) || !out) return WT_EINVAL;
    memset(out, 0, sizeof(*out));
    out->n = tree->desc.n;
    out->sigma = tree->desc.cp.sigma;
    out->levels = tree->desc.cp.L;
    out->symbol_bytes = tree->symbol_bytes;
    out->sample_k = tree->sample_k;
    for (uint32_t l = 0; l < tree->desc.cp.L; l++) {
        out->level_size[l] = tree->level_size[l];
        out->level_ones[l] = tree->level_ones[l];
    }
    out->tree_bytes = tree->hdr_bytes + tree->lvl_bytes;
    out->layout = tree->desc.layout;
    return WT_OK;
}

wt_status wt_export(wt_tree tree, uint32_t level, uint32_t what, void* h_dst, uint64_t* count) {
    if (!tree_ok(tree) || !count) return WT_EINVAL;
    const TreeDesc& d = tree->desc;
    const uint32_t L = d.cp.L, sigma = d.cp.sigma;
    const void* src = nullptr;
    size_t esz = 8;
    uint64_t cnt = 0;
    if (what == WT_EXPORT_C) {
        cnt = sigma + 1ull;
        src = d.C;
    } else if (what == WT_EXPORT_CODES || what == WT_EXPORT_LENS) {
        if (d.layout == WT_LAYOUT_MATRIX && what == WT_EXPORT_LENS) return WT_EUNSUPPORTED;
        cnt = sigma;
        *count = cnt;
        if (h_dst) {
            for (uint32_t s = 0; s < sigma; s++) {
                uint32_t code, len;
                encode(d.cp, s, code, len);
                if (what == WT_EXPORT_CODES) reinterpret_cast<uint64_t*>(h_dst)[s] = code;
                else reinterpret_cast<uint8_t*>(h_dst)[s] = (uint8_t)len;
            }
        }
        return WT_OK;
    } else if (what == WT_EXPORT_NODES) {
        if (d.layout == WT_LAYOUT_MATRIX) return WT_EUNSUPPORTED;
        cnt = L ? ((1ull << L) - 1) : 0;
        *count = cnt;
        if (h_dst && cnt) {
            std::vector<NodeEntry> tmp(cnt);
            if (cudaMemcpyAsync(tmp.data(), d.nodes, cnt * sizeof(NodeEntry), cudaMemcpyDeviceToHost, tree->stream) !=
                    cudaSuccess ||
                cudaStreamSynchronize(tree->stream) != cudaSuccess)
                return WT_ECUDA;
            uint64_t* o = reinterpret_cast<uint64_t*>(h_dst);
            for (uint64_t slot = 0; slot < cnt; slot++) {
                uint32_t l = 63u - (uint32_t)__builtin_clzll(slot + 1);
                uint64_t p = slot + 1 - (1ull << l), a = 0;
                uint64_t w = node_info(d.cp, l, p, a);
                const NodeEntry& e = tmp[slot];
                bool valid = w >= 2;
                o[4 * slot + 0] = valid ? e.start : 0;
                o[4 * slot + 1] = valid ? e.r0 : 0;
                o[4 * slot + 2] = valid ? e.off1 - e.r0 + e.start : 0;
                o[4 * slot + 3] = valid ? 1 : 0;
            }
        }
        return WT_OK;
    } else if (what == WT_EXPORT_EPS0 || what == WT_EXPORT_EPS1 || what == WT_EXPORT_MLP ||
               what == WT_EXPORT_RESID0 || what == WT_EXPORT_RESID1) {
        if (level >= L || tree->learned.mode == kLearnNone) return WT_EUNSUPPORTED;
        if (what == WT_EXPORT_MLP) {
            cnt = 2 * kMlpParams;
            src = tree->learned.mlp + 2 * level * kMlpParams;
            esz = 4;
        } else {
            const uint32_t b = (what == WT_EXPORT_EPS1 || what == WT_EXPORT_RESID1) ? 1u : 0u;
            return export_learned(tree, level, b, what == WT_EXPORT_RESID0 || what == WT_EXPORT_RESID1, h_dst, count);
        }
    } else {
        if (level >= L) return WT_EINVAL;
        const LevelDesc& v = d.lv[level];
        const uint64_t size = v.size, ones = v.ones, zeros = size - ones;
        switch (what) {
            case WT_EXPORT_BITS: cnt = (size + 63) / 64; src = v.words; break;
            case WT_EXPORT_L1: cnt = size / kL1Bits + 1; src = v.l1; break;
            case WT_EXPORT_L2: cnt = size / kL2Bits + 1; src = v.l2; esz = 2; break;
            case WT_EXPORT_S0: cnt = (zeros >> d.k_log2) + 1; src = v.s0; break;
            case WT_EXPORT_S1: cnt = (ones >> d.k_log2) + 1; src = v.s1; break;
            default: return WT_EINVAL;
        }
    }
    *count = cnt;
    if (h_dst && cnt) {
        if (cudaMemcpyAsync(h_dst, src, cnt * esz, cudaMemcpyDeviceToHost, tree->stream) != cudaSuccess ||
            cudaStreamSynchronize(tree->stream) != cudaSuccess)
            return WT_ECUDA;
    }
    return WT_OK;
}

void wt_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_timing.store(on ? 1 : 0);
}

void wt_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    collect_pending();
    g_stats.clear();
    g_launches.store(0);
}

uint64_t wt_profile_launches(void) { return g_launches.load(); }

size_t wt_profile_report(char* buf, size_t cap) {
    std::lock_guard<std::mutex> lk(g_mu);
    collect_pending();
    std::string s = "{";
    bool first = true;
    char tmp[256];
    for (auto& kv : g_stats) {
        snprintf(tmp, sizeof(tmp), "%s\"%s\": {\"launches\": %llu, \"ms\": %.6f}", first ? "" : ", ", kv.first.c_str(),
                 (unsigned long long)kv.second.launches, kv.second.ms);
        s += tmp;
        first = false;
    }
    s += "}";
    if (buf && cap) {
        size_t k = s.size() < cap - 1 ? s.size() : cap - 1;
        memcpy(buf, s.data(), k);
        buf[k] = 0;
    }
    return s.size() + 1;
}

}  // extern "C"
