/*
 * libwt — level-wise wavelet tree on one GB300 GPU (sm_103a).
 *
 * C ABI of the library built from paper_2505_03372_gb300/csrc.  All compute
 * runs in hand-written CUDA kernels; there is no CPU fallback.  Section and
 * algorithm numbers refer to M. Franzreb Salgado, "GPU Implementation of the
 * Wavelet Tree", arXiv 2505.03372 (2025).
 *
 * Conventions shared by every entry point
 *  - Pointers named d_* are device pointers (cudaMalloc / cudaMallocAsync /
 *    PyTorch CUDA tensors) of the current device, or managed memory; h_* are
 *    host pointers.  Device memory of another GPU is refused (WT_EINVAL).
 *    The caller owns them; the library never frees or retains them past
 *    the call (or, for asynchronous calls, past the completion of the work
 *    it enqueued on `stream`).
 *  - `stream` is a CUDA stream (the same type as cudaStream_t); NULL means the
 *    legacy default stream.  Work is enqueued on it; calls return before the
 *    GPU finishes unless stated otherwise.
 *  - Host-detectable argument errors (null pointers, bad sizes, a freed
 *    handle) return a status synchronously and enqueue nothing.
 *  - Data-dependent errors (a symbol >= sigma, a query out of range, a
 *    bounded device wait that gave up) are found on the GPU: the affected
 *    output gets a sentinel (UINT32_MAX / UINT64_MAX) and a sticky status word
 *    in the tree records the error; wt_status_sync() reports and clears it.
 *    No kernel traps.
 *  - Positions and counts are 0-based and 64-bit; rank is exclusive
 *    (Section 1 / Section 4, following SDSL): rank_c(i) counts positions < i.
 *  - Symbol arrays and the tree's bit arrays use 1, 2 or 4 bytes per symbol.
 *    Device symbol pointers must be 16-byte aligned (they are read with TMA
 *    bulk copies).  Limits: n < 2^40, 1 <= sigma <= 2^26 and
 *    sigma <= 2^(8*symbol_bytes).
 */
#ifndef WT_H
#define WT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* wt_stream; /* identical to cudaStream_t */
typedef struct wt_tree_s* wt_tree;     /* opaque, owned by libwt, immutable after build */
typedef struct wt_batch_s* wt_batch;   /* opaque: many trees built and queried by one graph launch */
typedef struct wt_order_s* wt_order;   /* opaque: a query batch sorted by walk key (wt_order_queries) */

typedef enum {
    WT_OK = 0,
    WT_EINVAL = 1,      /* bad argument: null pointer, sigma == 0, width not 1/2/4, limits exceeded, misaligned pointer */
    WT_ESYMBOL = 2,     /* some input symbol is >= sigma (found by the build's histogram pass) */
    WT_ENOMEM = 3,      /* device allocation failed */
    WT_ECUDA = 4,       /* a CUDA runtime call failed (launch error, ...) */
    WT_EQUERY = 5,      /* some query argument was out of range; that output holds a sentinel */
    WT_ETIMEOUT = 6,    /* a bounded device-side wait gave up; results of that call are not valid */
    WT_EUNSUPPORTED = 7, /* operation not available for this tree (e.g. no trained select model) */
    WT_EBOUNDS = 8      /* a bounds check failed and the access was skipped; results of that
                           call are not valid.  Query walks check every load in the debug
                           library (libwt_debug.so) only; the build checks its node-table
                           lookups in both libraries */
} wt_status;

/*
 * Device memory supplied by the caller (for example PyTorch's caching
 * allocator), so that the tree and every scratch buffer live in the caller's
 * pool.  Not part of the paper; an interface convention of this library.
 *  alloc(bytes, stream, ctx)  returns device memory of at least `bytes` bytes on
 *        the current device, 256-byte aligned, that work enqueued on `stream`
 *        after the call may use; NULL when it cannot (the call that asked then
 *        returns WT_ENOMEM after releasing what it had allocated).
 *  free(ptr, stream, ctx)  returns a block: the library has enqueued its last use
 *        of it on `stream`, the stream it was allocated on, so it may be handed
 *        out again to work ordered after that point on that stream.
 * Every request is made on the caller's `stream` and every block is
 * released on it, after its last use there.  (So the staging buffers of
 * wt_build_host and wt_query_host are taken on `stream` too, and their copies
 * wait for the work already queued on it; with the default pool those copies
 * overlap that work instead.)
 * The struct is copied; ctx and the functions must stay valid until the last
 * handle built with them is destroyed.  The callbacks run on the calling
 * thread, inside the library call.
 */
typedef struct {
    void* (*alloc)(size_t bytes, wt_stream stream, void* ctx);
    void (*free)(void* ptr, wt_stream stream, void* ctx);
    void* ctx;
} wt_allocator;

/* Build options.  Zero-initialised fields take the default. */
typedef struct {
    uint32_t sample_k; /* select sample interval K: the position of every K-th one and every K-th
                          zero is stored (Section 4.2).  Power of two in [256, 2^20]; default 4096,
                          the value of the paper's wavelet-tree experiments (Section 6.3). */
    uint32_t layout;   /* WT_LAYOUT_TREE (0, default): the level-wise wavelet tree with reduced
                          codes (Sections 5.1-5.4).  WT_LAYOUT_MATRIX (1): the wavelet matrix the
                          paper names as future work (Section 7): plain L-bit codes, every level
                          one stable partition of the whole level by its bit (zeros first); the
                          same queries, answered by walking with the per-level zero counts.
                          wt_train_select / wt_select_learned and WT_EXPORT_NODES / LENS are
                          WT_EUNSUPPORTED on a matrix. */
    const wt_allocator* allocator; /* NULL: the device's stream-ordered pool (cudaMallocAsync).  Else the
                          tree, the build's scratch, the query ordering's scratch, the host pipeline's
                          buffers and the learned-select tables all come from it. */
    uint32_t reserved[4];
} wt_options;

#define WT_LAYOUT_TREE 0u
#define WT_LAYOUT_MATRIX 1u

/* Size of the rank blocks (Section 4.1): L1 blocks of 65536 bits with a 64-bit
 * count of ones before the block; L2 blocks of 512 bits with a 16-bit count of
 * ones from the start of their L1 block.  |L2| = 512 is the value of every
 * experiment in Section 6. */
#define WT_L1_BITS 65536u
#define WT_L2_BITS 512u
#define WT_MAX_LEVELS 26u

/*
 * wt_build — construct the extended level-wise wavelet tree of Section 5
 * (Algorithm 4) with reduced codes (Section 5.1, Algorithm 3) over the
 * sequence S = d_symbols[0..n) drawn from [0, sigma).
 *
 * Level l (0 <= l < L = ceil(lg sigma)) stores bit l (from the top) of the code
 * of every symbol of S stably sorted by its first l code bits, for the symbols
 * whose code is longer than l; bits are packed LSB-first in 64-bit words and
 * each level starts on a 128-byte boundary (Section 4).  The same pass per
 * level writes the L1/L2 rank counters (Section 4.1) and the select samples
 * (Section 4.2), and stably partitions the level's symbols into the next
 * level's order.  The cumulative histogram C and the rank of every node
 * start are stored (the "extended" tree and precomputed node ranks, Section 5
 * and Section 5.2.1).
 *
 *  d_symbols     device, n symbols of symbol_bytes bytes each, 16-byte aligned;
 *                read only, not retained after the call returns.
 *  n             number of symbols, 0 <= n < 2^40.
 *  sigma         alphabet size, symbols must be < sigma.
 *  symbol_bytes  1, 2 or 4.
 *  opt           NULL for defaults.
 *  out           receives the handle (NULL on error).
 *
 * The call synchronises `stream` once (to read back the level sizes, which
 * fix the tree's allocation) and returns with the remaining work enqueued.
 * Returns WT_ESYMBOL, without a tree, if some symbol is >= sigma.
 */
wt_status wt_build(const void* d_symbols, uint64_t n, uint32_t sigma, uint32_t symbol_bytes,
                   const wt_options* opt, wt_stream stream, wt_tree* out);

/* Release all device memory of the tree (stream-ordered on the build stream). */
void wt_destroy(wt_tree tree);

/*
 * wt_build_host — wt_build from symbols in host memory (pinned or pageable),
 * the chunked construction the paper proposes (Section 7): the symbols are
 * copied to the device in 64 MiB chunks on an internal copy stream that does
 * not wait for work already queued on `stream`, and the histogram counts each
 * chunk on `stream` as it arrives, so the copy overlaps earlier work on the
 * stream and the histogram; the level passes then run as in wt_build.  The
 * device copy of the symbols comes from the allocator in opt (or the
 * stream-ordered pool) and is returned after the build; h_symbols must stay valid until the call returns (it
 * synchronises once, as wt_build does).  Arguments and results as wt_build;
 * a device pointer as h_symbols returns WT_EINVAL.
 */
wt_status wt_build_host(const void* h_symbols, uint64_t n, uint32_t sigma, uint32_t symbol_bytes,
                        const wt_options* opt, wt_stream stream, wt_tree* out);

/*
 * wt_access — Algorithm 5: d_out[k] = S[d_i[k]] for k < q.
 *  d_i    device, q positions; a position >= n yields UINT32_MAX and WT_EQUERY.
 *  d_out  device, q symbols (uint32).
 */
wt_status wt_access(wt_tree tree, const uint64_t* d_i, uint32_t* d_out, uint64_t q, wt_stream stream);

/*
 * wt_rank — Algorithm 6: d_out[k] = #{ j < d_i[k] : S[j] = d_c[k] }.
 *  d_c    device, q symbols; d_c[k] >= sigma yields UINT64_MAX and WT_EQUERY.
 *  d_i    device, q positions in [0, n]; larger yields UINT64_MAX and WT_EQUERY.
 *  d_out  device, q counts.
 */
wt_status wt_rank(wt_tree tree, const uint32_t* d_c, const uint64_t* d_i, uint64_t* d_out, uint64_t q,
                  wt_stream stream);

/*
 * wt_select — Algorithms 7 and 8 over the sampled binary select of
 * Algorithm 2: d_out[k] = position of the d_j[k]-th (1-based) occurrence of
 * d_c[k].  d_j[k] outside [1, count(d_c[k])] or d_c[k] >= sigma yields
 * UINT64_MAX and WT_EQUERY.
 */
wt_status wt_select(wt_tree tree, const uint32_t* d_c, const uint64_t* d_j, uint64_t* d_out, uint64_t q,
                    wt_stream stream);

/*
 * wt_query_mixed — one launch over a mixed batch: d_kind[k] = 0 access(d_arg[k]),
 * 1 rank(d_c[k], d_arg[k]), 2 select(d_c[k], d_arg[k]).  Results are widened to
 * uint64 in d_out (access results are symbols).  d_c is ignored for access.
 * Any other kind yields UINT64_MAX and WT_EQUERY.
 */
wt_status wt_query_mixed(wt_tree tree, const uint8_t* d_kind, const uint32_t* d_c, const uint64_t* d_arg,
                         uint64_t* d_out, uint64_t q, wt_stream stream);

/*
 * wt_order_queries / wt_walk_ordered / wt_order_destroy — the query calls
 * above in two steps, so that the first can run on another stream while the
 * build's level passes run (Sections 5.2-5.4: the walks; the ordering is this
 * library's, see wt_access).
 *  wt_order_queries: copy the batch (kind 0 access: d_arg = i; 1 rank: d_c,
 *     d_arg = i; 2 select: d_c, d_arg = j; 3 mixed: d_kind, d_c, d_arg as in
 *     wt_query_mixed) into arrays the order owns, sorted by where each walk
 *     goes when the batch and the tree are large enough (the same rule as
 *     wt_access).  It needs only the tree's header (n, sigma, C), which is
 *     final when wt_build / wt_build_host return, so `stream` may be any
 *     stream of the tree's device.  The input arrays may be reused once
 *     `stream` has passed this call.  *out is null on error.  Trees of a batch
 *     (wt_batch_tree) return WT_EUNSUPPORTED.
 *  wt_walk_ordered: walk an order on `stream` (waiting for the order's
 *     stream), writing answer k of the original batch to d_out[k]: uint32_t
 *     for access, uint64_t otherwise; same answers, sentinels and status as
 *     the one-step calls.  The tree must be the one the order was made for.
 *  wt_order_destroy: release the order after the work queued on `stream`
 *     (the stream of its last walk); the memory returns on the order's own
 *     stream, which must still exist, after it waits for `stream`.
 * Pointers: device memory of the current device.  Errors: WT_EINVAL for a
 * bad tree, order, kind or pointer, WT_ENOMEM, WT_ECUDA.
 */
wt_status wt_order_queries(wt_tree tree, uint32_t kind, const uint8_t* d_kind, const uint32_t* d_c,
                           const uint64_t* d_arg, uint64_t q, wt_stream stream, wt_order* out);
wt_status wt_walk_ordered(wt_tree tree, wt_order order, void* d_out, wt_stream stream);
wt_status wt_order_destroy(wt_order order, wt_stream stream);

/*
 * wt_query_host — the end-to-end query path of Section 6 (queries copied in
 * from the host, answers copied back): the batch is split into chunks of
 * `chunk` queries (0: min(q, 2^24)); chunk i+1 is copied in while chunk i
 * walks and chunk i-1 is copied out, with at most two chunks resident on the
 * device.  Each chunk is answered exactly as wt_access / wt_rank / wt_select /
 * wt_query_mixed would answer it (including the query ordering of large
 * chunks).
 *  kind    0 access, 1 rank, 2 select, 3 mixed (per-query kinds in h_kind).
 *  h_kind  host, q uint8 kinds (kind 3 only; else ignored, may be null).
 *  h_c     host, q symbols (kinds 1-3; ignored for access, may be null).
 *  h_arg   host, q positions i (access, rank) or ranks j (select), uint64.
 *  h_out   host, q answers: uint32 for access, uint64 for kinds 1-3.
 * Host buffers may be pinned (page-locked: the copies are asynchronous) or
 * pageable (the driver stages the copies and may block the calling thread).
 * Device pointers are rejected with WT_EINVAL.  The walks run on `stream`,
 * after the work already queued there (typically the build); the copies run
 * on two internal streams and do not wait for that work, so the first chunk's
 * copy overlaps it.  The call returns once everything is queued; h_out holds
 * the answers after `stream` has been synchronised, and the host buffers must
 * stay valid until then.  Data errors are reported as for the device calls.
 * Device memory: two chunks of arguments and answers, from the tree's allocator
 * (or the stream-ordered pool), returned after the last copy-out.
 */
wt_status wt_query_host(wt_tree tree, uint32_t kind, const uint8_t* h_kind, const uint32_t* h_c,
                        const uint64_t* h_arg, void* h_out, uint64_t q, uint64_t chunk, wt_stream stream);

/* Synchronise `stream`, then return and clear the tree's sticky device status
 * (WT_OK if no data-dependent error happened since the last call). */
wt_status wt_status_sync(wt_tree tree, wt_stream stream);

typedef struct {
    uint64_t n;
    uint32_t sigma;
    uint32_t levels;       /* L = ceil(lg sigma); 0 for sigma == 1 */
    uint32_t symbol_bytes;
    uint32_t sample_k;
    uint64_t level_size[WT_MAX_LEVELS]; /* bits in level l = #symbols whose code is longer than l */
    uint64_t level_ones[WT_MAX_LEVELS];
    uint64_t tree_bytes;   /* device bytes held by the tree */
    uint32_t layout;       /* WT_LAYOUT_TREE or WT_LAYOUT_MATRIX */
    uint32_t reserved;
} wt_info_t;

/* Host-side metadata; no device work. */
wt_status wt_info(wt_tree tree, wt_info_t* out);

/*
 * wt_export — copy logical contents to host memory, for comparison with a
 * reference.  Synchronous (device-to-host copies on the build stream).
 *  what = WT_EXPORT_BITS   level bits, ceil(size/64) uint64 words, tail bits zero
 *         WT_EXPORT_L1     floor(size/65536)+1 uint64: ones in B[0, 65536 k)
 *         WT_EXPORT_L2     floor(size/512)+1 uint16: ones from the start of the
 *                          enclosing L1 block to position 512 m
 *         WT_EXPORT_S0/S1  floor(zeros/K)+1 (ones) uint64: [0] = 0 and [m] =
 *                          position of the (m K)-th zero (one)
 *         WT_EXPORT_C      sigma+1 uint64 cumulative histogram (level ignored)
 *         WT_EXPORT_CODES  sigma uint64 codes left-aligned in L bits
 *         WT_EXPORT_LENS   sigma uint8 code lengths
 *         WT_EXPORT_NODES  (2^L - 1) x 4 uint64 in heap order, slot 2^d - 1 + p
 *                          for the node at depth d with code prefix p:
 *                          {start = C[a], r0 = rank_0(d, start), mid =
 *                          C[a + prevPow2(b - a)], valid}
 *  h_dst  host buffer or NULL; *count receives the element count either way.
 */
enum {
    WT_EXPORT_BITS = 0,
    WT_EXPORT_L1 = 1,
    WT_EXPORT_L2 = 2,
    WT_EXPORT_S0 = 3,
    WT_EXPORT_S1 = 4,
    WT_EXPORT_C = 5,
    WT_EXPORT_CODES = 6,
    WT_EXPORT_LENS = 7,
    WT_EXPORT_NODES = 8,
    WT_EXPORT_EPS0 = 9,   /* learned select: bound of every anchor segment of the zeros, in bits,
                             floor(zeros / (4 K)) + 1 uint32 */
    WT_EXPORT_EPS1 = 10,  /* the same for the ones */
    WT_EXPORT_MLP = 11,   /* learned select: 2 x 97 float MLP parameters of the level (b = 0, then b = 1) */
    WT_EXPORT_RESID0 = 12, /* learned select (PLA): three knot residuals R_1..3 per anchor segment of the
                             zeros, in bits, 3 (floor(zeros / (4 K)) + 1) int32 */
    WT_EXPORT_RESID1 = 13  /* the same for the ones */
};
wt_status wt_export(wt_tree tree, uint32_t level, uint32_t what, void* h_dst, uint64_t* count);

/*
 * Learned select (not in the paper; the workload's "learned select").  For
 * every level and bit value b a model predicts the position of the k-th b-bit.
 * The ranks are cut into anchor segments of 4 K ranks: segment m runs from the
 * (4 m K)-th b-bit to the (4 (m+1) K)-th, whose positions are select samples
 * the build already stores (Section 4.2), or to the virtual (count_b + 1)-th
 * b-bit at the end of the level.  Each segment keeps one 8-byte record: three
 * knot residuals and its error bound (about half the bytes of the select
 * samples).
 *   mode 1 (PLA): piecewise-linear with fitted knots: knot t = 1, 2, 3 sits at
 *          rank k0 + floor(t (k1 - k0) / 4) and position x0 + floor(t (x1 -
 *          x0) / 4) + R_t, the residuals R_t (WT_EXPORT_RESID0/1) fitted on
 *          the GPU by least squares to the positions of the segment's b-bits;
 *          a rank is predicted from its two knots (ka, xa), (kb, xb) as xa +
 *          floor((k - ka) (xb - xa) / (kb - ka)), exact integer arithmetic.
 *   mode 2 (MLP): the fraction u = (k - 4 m K) / (segment length) is mapped to
 *          u + g(u), g a 1 -> 32 -> 1 ReLU network in FP32 per (level, b), trained
 *          on the GPU with Adam on (u, position fraction) pairs drawn from the
 *          built levels (opt->pairs per model, opt->steps steps, learning rate
 *          opt->lr); g starts at 0, the line through the anchors.
 * wt_train_select then evaluates the model at the rank of every b-bit of every
 * level and stores per segment the largest distance between prediction and
 * position, rounded up (WT_EXPORT_EPS0/1).  wt_select_learned answers the same queries as
 * wt_select: per level it searches only the window prediction +- bound; if the
 * counters show the bit is outside the window the level falls back to the
 * sampled select and a counter records it (wt_learned_info).  Results are
 * identical to wt_select.  mode 0 removes the model.  Returns WT_EUNSUPPORTED
 * from wt_select_learned if no model was trained.  wt_train_select allocates
 * (stream-ordered on `stream`) and enqueues its work.
 */
typedef struct {
    uint32_t steps;  /* Adam steps (default 300) */
    uint32_t pairs;  /* training pairs per model, <= 16384 (default 8192) */
    float lr;        /* learning rate (default 0.01) */
    uint32_t reserved[5];
} wt_train_options;

wt_status wt_train_select(wt_tree tree, uint32_t mode, const wt_train_options* opt, wt_stream stream);
wt_status wt_select_learned(wt_tree tree, const uint32_t* d_c, const uint64_t* d_j, uint64_t* d_out, uint64_t q,
                            wt_stream stream);

typedef struct {
    uint32_t mode;
    uint32_t pad;
    uint64_t fallbacks;                     /* level searches that left their window, since training */
    uint64_t model_bytes;                   /* device bytes of the records (residuals, bounds) + parameters */
    double eps_mean[WT_MAX_LEVELS][2];      /* mean per-segment bound, per level and b */
    uint32_t eps_max[WT_MAX_LEVELS][2];
    uint64_t anchor_bytes;                  /* bytes of the select samples that serve as anchors (8 per
                                               segment; stored once, with the tree) */
} wt_learned_info_t;

/* Synchronises the tree's stream; copies bound statistics to the host. */
wt_status wt_learned_info(wt_tree tree, wt_learned_info_t* out);

/*
 * Batches of independent trees (not in the paper; the workload of thousands of
 * small trees).  wt_batch_create lays out ntrees trees in one device
 * allocation — sizes are worst cases from n and sigma, so nothing is read back
 * — and captures into one CUDA graph the whole construction of every tree
 * (the same steps as wt_build, each a kernel over all trees at once: one
 * persistent level-pass kernel per level walks the tiles of every tree) plus
 * the query batch registered with wt_batch_set_queries.  wt_batch_run launches
 * that graph on `stream` (no host synchronisation inside); it may be run again
 * after the caller rewrites the symbol or query buffers in place.
 *
 *  h_symbols  host array of ntrees device pointers (16-byte aligned) to each
 *             tree's symbols; the buffers must stay valid while the batch runs.
 *  h_n, h_sigma  host arrays of sizes and alphabet sizes (limits as wt_build).
 *  opt        sample_k as in wt_options; query_threads 128, 256 or 512 threads
 *             per CTA of the query kernel (default 256); lp_ctas_per_sm the
 *             level pass's persistent grid; NULL for defaults.
 * Queries: d_tree[k] < ntrees selects the tree, then d_kind / d_c / d_arg /
 * d_out as in wt_query_mixed.  A tree index >= ntrees yields UINT64_MAX.
 * wt_batch_status_sync reports the OR of every tree's sticky status.
 * wt_batch_tree returns a handle on one tree of the batch (after a run) for
 * wt_info / wt_export / wt_access / ... ; it shares the batch's memory, must
 * be released with wt_destroy before wt_batch_destroy, and reflects the
 * contents of the last completed run.
 */
typedef struct {
    uint32_t sample_k;
    uint32_t query_threads;
    const wt_allocator* allocator; /* NULL: cudaMalloc; else the batch's one allocation comes from it
                                      (allocated and released on the legacy default stream) */
    uint32_t lp_ctas_per_sm;       /* CTAs per SM of the persistent batched level pass: 1 to 6
                                      (0: 6, the most that fit) */
    uint32_t reserved[3];
} wt_batch_options;

wt_status wt_batch_create(uint32_t ntrees, const void* const* h_symbols, const uint64_t* h_n, const uint32_t* h_sigma,
                          uint32_t symbol_bytes, const wt_batch_options* opt, wt_batch* out);
wt_status wt_batch_set_queries(wt_batch batch, const uint32_t* d_tree, const uint8_t* d_kind, const uint32_t* d_c,
                               const uint64_t* d_arg, uint64_t* d_out, uint64_t q);
wt_status wt_batch_run(wt_batch batch, wt_stream stream);
wt_status wt_batch_status_sync(wt_batch batch, wt_stream stream);
wt_status wt_batch_tree(wt_batch batch, uint32_t index, wt_tree* out);
uint64_t wt_batch_bytes(wt_batch batch);
void wt_batch_destroy(wt_batch batch);

/*
 * wt_mlp_gradient — one evaluation of the MLP's loss and gradient on the GPU,
 * with the same device code the training kernel runs (for checking the
 * backward pass).  Host arrays: h_params 97 floats {w1[32], b1[32], w2[32], b2},
 * h_u / h_t n inputs and targets (n <= 16384); h_grad receives 97 floats,
 * *h_loss the loss mean_i (u_i + g(u_i) - t_i)^2.  Synchronous.
 */
wt_status wt_mlp_gradient(const float* h_params, const float* h_u, const float* h_t, uint32_t n, float* h_grad,
                          float* h_loss);

/*
 * wt_bitvector_support_static — rank/select support of a caller-owned
 * bitvector, computed without allocating any device memory.  The paper has no
 * counterpart to this entry point; it exists for callers that cannot allocate
 * while they run: code that executes inside an allocator or memory-pool
 * callback, latency-critical loops that must not take the driver's allocation
 * path, or host frameworks that own all device memory and pass in fixed
 * buffers.  Everything the caller passes is an input or an output; the only
 * other memory used is a scratch array compiled into libwt (a 64-bit word per
 * 65536-bit tile plus a counter, 512 KiB), which every GPU that loads the
 * library keeps until the process exits.
 *
 * It writes the same counters and samples wt_build stores for a level
 * (wt_export's WT_EXPORT_L1, L2, S0 and S1 contents) for the bitvector
 * d_words[0 .. ceil(nbits/64)) (LSB-first; bits at or past nbits are ignored):
 *  d_l1   floor(nbits/65536) + 1 uint64: ones in B[0, 65536 k)
 *  d_l2   floor(nbits/512) + 1 uint16: ones from the start of the enclosing
 *         65536-bit block to position 512 m
 *  d_s0, d_s1  sample_capacity uint64 each; [0] = 0 and [m] = position of the
 *         (m * sample_k)-th zero / one; entries past the last sample are not written
 *  sample_capacity  at least floor(nbits / sample_k) + 2
 *  d_status  optional device word; WT_ETIMEOUT's bit (1 << WT_ETIMEOUT) is OR-ed
 *         into it if a bounded device wait gave up.
 *  d_ones optional device word; receives the number of ones of the bitvector
 *         (the count wt_bitvector_select takes).
 * Limits: 1 <= nbits <= 2^32 (the size of the static scratch); larger or
 * empty inputs, a sample_k that is not a power of two in [256, 2^20], a too
 * small sample_capacity or a pointer that is not device memory of the current
 * device return WT_EINVAL before any work is enqueued; so does a CUDA error
 * left pending on the calling thread by earlier work (WT_ECUDA).  No
 * cudaMalloc, cudaFree or other allocating call is made.
 * The first call on a device looks up the device address of the static
 * scratch (cudaGetSymbolAddress, with that device current); make that first
 * call before any stream capture.  The address is kept per device together
 * with the identity of the context it belongs to; after a device reset the
 * next call sees a new context and looks the address up again.  Every call on a device shares the scratch,
 * which keeps the last call's contents; each call clears what must start at
 * zero.  Calls whose work overlaps on the GPU (different streams, or a call
 * issued while another is still running) race on the scratch and give wrong
 * results: serialise them.  Work is enqueued on `stream`; the call returns
 * before it finishes.
 */
wt_status wt_bitvector_support_static(const uint64_t* d_words, uint64_t nbits, uint32_t sample_k, uint64_t* d_l1,
                                      uint16_t* d_l2, uint64_t* d_s0, uint64_t* d_s1, uint64_t sample_capacity,
                                      uint32_t* d_status, uint64_t* d_ones, wt_stream stream);

/*
 * wt_bitvector_rank / wt_bitvector_select — binary rank (Section 4.1,
 * Algorithm 1) and sampled binary select (Section 4.2, Algorithm 2) over a
 * caller-owned bitvector whose support structures wt_bitvector_support_static
 * wrote (the same layout as one level of a tree).  One thread per query.
 *  d_words  device, 32-byte aligned, the bits LSB-first; the allocation must hold whole 512-bit
 *           blocks plus one: at least (floor(nbits / 512) + 1) * 8 words (the
 *           walks read 32-byte halves of a block); bits at or past nbits must
 *           be zero.
 *  d_l1, d_l2, d_s0, d_s1, sample_k  as written by wt_bitvector_support_static.
 *  ones     number of ones in the bitvector (select's bound and last sample).
 *  rank:    d_out[k] = ones in B[0, d_i[k]) for d_i[k] <= nbits.
 *  select:  d_out[k] = position of the d_j[k]-th (1-based) bit equal to b
 *           (b = 0 or 1) for 1 <= d_j[k] <= count_b.
 * Out-of-range queries yield UINT64_MAX and OR 1 << WT_EQUERY into *d_status
 * (optional device word).  In the debug library a load outside the arrays'
 * documented lengths is skipped and ORs 1 << WT_EBOUNDS into *d_status (for
 * example, select with samples that point past nbits).  Asynchronous on
 * `stream`.  Host-detectable errors
 * (null or non-device pointers, nbits == 0, b > 1, sample_k not a power of two
 * in [256, 2^20], ones > nbits) return WT_EINVAL before any work is queued.
 */
wt_status wt_bitvector_rank(const uint64_t* d_words, uint64_t nbits, const uint64_t* d_l1, const uint16_t* d_l2,
                            const uint64_t* d_i, uint64_t* d_out, uint64_t q, uint32_t* d_status, wt_stream stream);
wt_status wt_bitvector_select(const uint64_t* d_words, uint64_t nbits, uint64_t ones, uint32_t b,
                              const uint64_t* d_l1, const uint16_t* d_l2, const uint64_t* d_s0,
                              const uint64_t* d_s1, uint32_t sample_k, const uint64_t* d_j, uint64_t* d_out,
                              uint64_t q, uint32_t* d_status, wt_stream stream);

/*
 * wt_alphabet — minimal-alphabet extraction (Section 6.2: a text's symbols
 * mapped to [0, sigma) before the build when sigma is not known): sigma = the
 * number of distinct values in d_symbols; d_out[k] = the rank of d_symbols[k]
 * among those values, in the input's width (d_out == d_symbols is allowed);
 * d_values (optional, device, room for min(n, 2^(8 w)) uint32) receives the
 * distinct values in increasing order, so d_values[d_out[k]] == d_symbols[k].
 * *h_sigma receives sigma; the call synchronises `stream` to read it.
 * Method: a presence bitmap of 2^(8 w) bits, its rank/select support
 * (wt_bitvector_support_static), rank for the mapping, select for d_values.
 * Device memory from the stream-ordered pool: the bitmap and its support
 * (about 32 B, 8 KiB or 560 MiB for w = 1, 2, 4), returned before the call ends.
 *  d_symbols  device, n symbols of symbol_bytes (1, 2 or 4) bytes.
 * n == 0 gives sigma = 0.  Null pointers, a width other than 1, 2, 4 or host
 * memory return WT_EINVAL.
 */
wt_status wt_alphabet(const void* d_symbols, uint64_t n, uint32_t symbol_bytes, void* d_out, uint32_t* d_values,
                      uint32_t* h_sigma, wt_stream stream);

/*
 * wt_selftest_lookback_timeout — diagnostic for the bounded device waits.
 * Runs the build's decoupled look-back for a tile whose predecessor never
 * publishes its count, with at most spin_cap polls (1 <= spin_cap <= 2^22;
 * the build uses 2^22).  The wait gives up, the kernel records WT_ETIMEOUT in
 * a status word and returns normally, so the context stays usable.  Returns
 * WT_ETIMEOUT when that path works (the expected result).  Synchronous.
 */
wt_status wt_selftest_lookback_timeout(uint32_t spin_cap, wt_stream stream);

/* Human-readable name of a status code (static storage). */
const char* wt_status_str(wt_status s);

/*
 * Launch accounting and kernel timing (tracing support; no effect on results).
 *  wt_profile_enable(1) brackets every kernel launch with CUDA events on its
 *  stream; wt_profile_report() synchronises those events and writes a JSON
 *  object {"kernel name": {"launches": L, "ms": T}, ...} into buf (cap bytes,
 *  NUL-terminated, truncated if short) and returns the length needed.
 *  wt_profile_launches() counts every kernel this library launched since load
 *  (or since the last reset), whether or not timing is enabled.
 */
void wt_profile_enable(int on);
void wt_profile_reset(void);
uint64_t wt_profile_launches(void);
size_t wt_profile_report(char* buf, size_t cap);

#ifdef __cplusplus
}
#endif

#endif /* WT_H */
