// Level passes of the construction (Section 5.1, Algorithm 4) over bit-sliced
// sequences.
//
// Algorithm 4 sorts the text by the next code bit at every level (a radix-sort
// step) and reads the level's bits off the sorted sequence.  Here T_l, the
// sequence S stably sorted by the first l code bits, is stored as R = L - l
// bit planes over its positions: plane j holds code bit L-1-(l+j) of every
// element, so plane 0 is the level bitvector B_l itself and the other planes
// are the bits that later levels need.  T_{l+1} is the stable partition of T_l
// by B_l inside every node: the zeros of a node keep their order at
// off0 + rank_0(position), its ones at off1 + rank_1(position) (the node
// table's offsets, Section 5.2.1).  A plane moves under that partition one
// 32-bit word at a time: the word is compressed twice, once under the zeros of
// B_l's word and once under its ones, and the two compressed pieces are
// appended to the tile's zero run and one run.  The compress follows Hacker's
// Delight (2nd ed., Section 7-4): the five shift masks depend only on B_l's
// word, so they are computed once and reused for every plane.  A level thus
// reads R bits and writes R - 1 bits per element, and 32 elements move per
// instruction.
//
// Per level one kernel walks tiles of 16,384 positions.  A tile reads B_l's
// words, writes the level's L1/L2 counters (Section 4.1) and select samples
// (Section 4.2) from the ones before it (an exclusive scan of per-tile counts),
// and moves planes 1..R-1.  Output words covered by one run are stored;
// words shared by two runs are ORed into, so the output planes must start at
// zero: each kernel clears the input planes it consumes, and those buffers hold
// the next level's output.  While it writes B_{l+1} the kernel counts its ones
// per tile of level l+1; a scan of those counts gives the next level's prefixes.
// Tiles are independent of each other: no look-back, no waiting on other CTAs.
// Level 0's planes come from S by a transpose of the codes.  Every kernel walks
// the work items of one or many trees (a batch), so a single tree is a batch
// of one.
#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_device.cuh"
#include "wt_internal.hpp"

namespace wt {

static_assert(sizeof(LevelArgs) % 8 == 0, "level arguments are copied as 64-bit words");

constexpr uint32_t kTileThreads = 512;  // one 32-bit word of every plane per thread
constexpr uint32_t kTileWords = kTile / 32;
constexpr uint32_t kTilesPerL1 = kL1Bits / kTile;
constexpr uint32_t kScanPerThread = 8;
constexpr uint32_t kSlots = 16;         // plane ring: planes of the current and the next tiles
constexpr uint32_t kImgWords = 520;     // one run image: 512 words + alignment and read-ahead
constexpr uint32_t kPairs = 3;          // run-image slots in rotation, each for a pair of planes
constexpr uint32_t kTrThreads = 256;    // transpose: 32 symbols per thread
constexpr uint32_t kTrTable = 1024;     // codes tabulated in shared memory up to this sigma

uint64_t transpose_chunks(uint64_t words32) { return (words32 + kTrThreads - 1) / kTrThreads; }
uint64_t plane_stride(uint64_t n) { return level_tiles(n) * kTileWords; }

// Internal nodes (two or more symbols) of level l.  In prefix order they come
// first: a prefix whose node is a leaf or absent belongs to a code that ended
// at or above level l, and such codes belong to the largest symbols.
uint64_t internal_nodes(const CodeParams& cp, uint32_t l) {
    uint64_t lo = 0, hi = 1ull << l;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        uint64_t a = 0;
        if (node_info(cp, l, mid, a) >= 2) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <bool B>
struct BoolTag {
    static constexpr bool value = B;
};

// ===========================================================================
// bit tools
// ===========================================================================

// One stage of the 32x32 bit-matrix transpose: swap the off-diagonal S x S
// blocks of every pair of rows (k, k + S).
template <int S, uint32_t M>
__device__ __forceinline__ void tr_stage(uint32_t (&A)[32]) {
#pragma unroll
    for (int k = 0; k < 32; k++) {
        if (k & S) continue;
        const uint32_t t = ((A[k] >> S) ^ A[k + S]) & M;
        A[k + S] ^= t;
        A[k] ^= t << S;
    }
}
// Afterwards bit k of A[b] is bit b of the old A[k].
__device__ __forceinline__ void transpose32(uint32_t (&A)[32]) {
    tr_stage<16, 0x0000FFFFu>(A);
    tr_stage<8, 0x00FF00FFu>(A);
    tr_stage<4, 0x0F0F0F0Fu>(A);
    tr_stage<2, 0x33333333u>(A);
    tr_stage<1, 0x55555555u>(A);
}

// Shift masks of compress_left(., m): stage i moves the selected bits left by
// 2^i.  A bit of m moves left by the number of zeros of m above it; stage i
// takes the bits whose remaining distance has bit i set, found as the parity
// of the zeros above them (a suffix XOR).  Moving bits never land on occupied
// positions, so the move is an add: m + v * (2^(2^i) - 1).
__device__ __forceinline__ void compress_masks(uint32_t m, uint32_t (&mv)[5]) {
    uint32_t mk = ~m >> 1;  // zeros of m, seen from the bit below
#pragma unroll
    for (int i = 0; i < 5; i++) {
        uint32_t mp = mk ^ (mk >> 1);  // suffix XOR: parity of the marked bits at or above
        mp ^= mp >> 2;
        mp ^= mp >> 4;
        mp ^= mp >> 8;
        mp ^= mp >> 16;
        const uint32_t v = mp & m;
        mv[i] = v;
        m += v * ((1u << (1 << i)) - 1u);
        mk &= ~mp;
    }
}
// The bits of x under m (x already masked by m), packed towards bit 31 in
// order: one AND and one multiply-add per stage.
__device__ __forceinline__ uint32_t compress_left(uint32_t x, const uint32_t (&mv)[5]) {
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const uint32_t t = x & mv[i];
        x += t * ((1u << (1 << i)) - 1u);
    }
    return x;
}

// Largest node index p < nnodes whose start is <= pos (node 0 starts at 0).
// One warp, 32 probes per round.
__device__ __forceinline__ uint64_t warp_find_node(const NodeEntry* nodes, uint64_t nnodes, uint64_t pos) {
    const uint32_t lane = threadIdx.x & 31;
    uint64_t lo = 0, hi = nnodes;
    while (hi - lo > 1) {
        const uint64_t step = (hi - lo + 31) / 32;
        const uint64_t p = lo + lane * step;
        const bool ok = p < hi && __ldg(&nodes[p].start) <= pos;
        const uint32_t m = __ballot_sync(0xffffffffu, ok);
        const uint32_t last = 31u - __clz(m);
        lo += last * step;
        hi = umin64(hi, lo + step);
    }
    return lo;
}

// ===========================================================================
// level 0: symbols -> bit planes
// ===========================================================================

// Encode and transpose the 32 symbols of one word of B_0: plane j gets code bit
// L-1-j of each.  Returns the ones of B_0's word.
template <typename T>
__device__ __forceinline__ uint32_t transpose_word(const TransposeArgs& a, const CodeParams& cp, bool table,
                                                   const uint32_t* s_code, uint64_t word) {
    const uint64_t n = a.n;
    const uint32_t sigma = cp.sigma, L = cp.L;
    const uint64_t e0 = word * 32;
    constexpr int EPW = 4 / (int)sizeof(T);  // symbols per 32-bit word
    uint32_t A[32];
    const T* S = reinterpret_cast<const T*>(a.sym) + e0;
    const uint32_t cnt = (uint32_t)umin64(32, n - e0);
    if (cnt == 32) {
        // 32 symbols = 2 * sizeof(T) aligned 16-byte loads (S is 16-byte aligned, e0 a multiple of 32)
        const uint4* S4 = reinterpret_cast<const uint4*>(S);
#pragma unroll
        for (int v = 0; v < 2 * (int)sizeof(T); v++) {
            const uint4 q = __ldg(S4 + v);
            const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int k = 0; k < EPW; k++)
                    A[(v * 4 + i) * EPW + k] =
                        sizeof(T) == 4 ? wv[i] : (wv[i] >> (8 * sizeof(T) * k)) & ((1u << (8 * sizeof(T))) - 1u);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 32; k++) {
            A[k] = 0u;
            if ((uint32_t)k < cnt) A[k] = (uint32_t)S[k];
        }
    }
#pragma unroll
    for (int k = 0; k < 32; k++) {
        const uint32_t s = A[k] < sigma ? A[k] : 0u;  // symbols >= sigma are reported by the histogram
        uint32_t code = s;
        if (!cp.pow2) {
            if (table) {
                code = s_code[s];
            } else {
                uint32_t len;
                encode(cp, s, code, len);
            }
        }
        A[k] = (uint32_t)k < cnt ? code : 0u;
    }
    uint32_t b0 = 0;
    if (sizeof(T) == 1) {
        // codes of at most 8 bits: four per word; bit b of the four bytes of a
        // word gathers into a nibble with one multiply (bits 28..31 of the product)
        uint32_t P[8];
#pragma unroll
        for (int i = 0; i < 8; i++) P[i] = A[4 * i] | (A[4 * i + 1] << 8) | (A[4 * i + 2] << 16) | (A[4 * i + 3] << 24);
#pragma unroll
        for (int b = 0; b < 8; b++) {
            if ((uint32_t)b < L) {
                uint32_t acc = 0;
#pragma unroll
                for (int i = 0; i < 8; i++) acc += (((P[i] & (0x01010101u << b)) * (0x10204080u >> b)) >> 28) << (4 * i);
                const uint32_t j = L - 1 - b;  // plane j holds code bit L-1-j
                if (j == 0) b0 = acc;
                else a.planes[(uint64_t)(j - 1) * a.pstride + word] = acc;
            }
        }
    } else {
        transpose32(A);
#pragma unroll
        for (int b = 0; b < 32; b++) {
            if ((uint32_t)b < L) {
                const uint32_t j = L - 1 - b;
                if (j == 0) b0 = A[b];
                else a.planes[(uint64_t)(j - 1) * a.pstride + word] = A[b];
            }
        }
    }
    a.bits0[word] = b0;
    return __popc(b0);
}

// One CTA per 256 words of 32 symbols of one tree; words of B_0 past n are
// written as zeros.  The CTA's words lie in one tile, whose count of ones it
// adds to.
template <typename T>
__global__ void __launch_bounds__(kTrThreads) transpose_kernel(const TransposeArgs* __restrict__ args,
                                                               const uint64_t* __restrict__ chunk_prefix,
                                                               uint32_t ntrees) {
    __shared__ uint32_t s_code[kTrTable];
    __shared__ uint32_t s_tree;
    __shared__ uint32_t s_ones;
    if (threadIdx.x == 0) {
        s_tree = ntrees > 1 ? find_tree(chunk_prefix, ntrees, blockIdx.x) : 0u;
        s_ones = 0;
    }
    __syncthreads();
    const TransposeArgs& a = args[s_tree];
    CodeParams cp;  // encode() reads sigma, L and pow2 only
    cp.sigma = a.sigma;
    cp.L = a.L;
    cp.pow2 = a.pow2;
    const bool table = !cp.pow2 && cp.sigma <= kTrTable;
    if (table) {
        for (uint32_t s = threadIdx.x; s < cp.sigma; s += kTrThreads) {
            uint32_t code, len;
            encode(cp, s, code, len);
            s_code[s] = code;
        }
        __syncthreads();
    }
    const uint64_t word = (blockIdx.x - chunk_prefix[s_tree]) * kTrThreads + threadIdx.x;
    uint32_t ones = 0;
    if (word < a.bits0_words) {
        if (word * 32 < a.n) ones = transpose_word<T>(a, cp, table, s_code, word);
        else a.bits0[word] = 0;
    }
    const uint32_t ws = __reduce_add_sync(0xffffffffu, ones);
    if ((threadIdx.x & 31) == 0 && ws) atomicAdd(&s_ones, ws);
    __syncthreads();
    const uint64_t w0 = (blockIdx.x - chunk_prefix[s_tree]) * kTrThreads;
    if (threadIdx.x == 0 && s_ones) atomicAdd(a.count + (w0 / kTileWords), s_ones);
}

// ===========================================================================
// the level kernel
// ===========================================================================

// Single-node tiles: write-out plan of one run (image aligned with its output
// words: image word wb + i holds output word k0 + i, wb = k0 mod 4).
struct RunPlan {
    uint64_t k0;       // first output word
    uint32_t nw;       // output words (0: nothing to write)
    uint32_t wb;       // image word of output word 0
    uint32_t ta, tb;   // output words [ta, tb) leave by one bulk copy
    uint32_t fmask;    // bits of the first word inside the run
    uint32_t lmask;    // bits of the last word inside the run
    uint64_t tile;     // tile of level l+1 holding the run's first bit
};

// Load cursor (thread 0): issues plane loads in (tile, plane) order, tiles
// blockIdx.x, blockIdx.x + gridDim.x, ..., whenever a ring slot is free.
struct Cursor {
    uint64_t g;          // tile being loaded (global index over the trees' tiles)
    uint32_t tree, j, R, bytes;
    const uint32_t* bits;
    const uint32_t* in;
    uint64_t pstride, w0;  // plane stride, first word of the tile
    uint64_t size, first;  // the tree's level size and first tile
    uint32_t issued;
};
struct TileSmem {
    uint32_t ring[kSlots][kTileWords];     // planes in flight, in (tile, plane) order
    uint32_t img[kPairs][2][2][kImgWords]; // [slot][plane of the pair][zero run, one run]
    uint32_t zero[kTileWords];             // zeros: source of the bulk clears of consumed planes
    uint32_t b[kTileWords];                // B_l words of the tile
    uint32_t pre[kTileWords];              // ones before each word within the tile
    LevelArgs args;                        // the current tile's tree
    RunPlan run[2];                        // single-node tiles: zero run, one run
    uint64_t mbar[kSlots];
    uint64_t t0, E, p0;                    // tile start, ones of B_l before it, its first node
    uint32_t count, O;                     // tile elements, ones
    uint32_t tree;
    Cursor cur;                            // load cursor (thread 0)
    uint32_t ones[4];                      // ones of B_{l+1} per (run, side of a tile boundary)
    uint32_t wsum[kTileThreads / 32];
};

// Append a compressed piece (cnt bits at the top of vl) at image bit off.
__device__ __forceinline__ void place(uint32_t* img, uint32_t off, uint32_t cnt, uint32_t vl) {
    if (cnt == 0) return;
    const uint32_t v = vl >> (32 - cnt);
    const uint32_t wi = off >> 5, sh = off & 31;
    atomicOr(img + wi, v << sh);
    if (sh + cnt > 32) atomicOr(img + wi + 1, __funnelshift_l(v, 0u, sh));
}

// Ones of run bits [x0, x1) inside a piece of c bits (right-aligned in v) at run bit pre.
__device__ __forceinline__ uint32_t ones_in(uint32_t v, uint32_t pre, uint32_t c, uint32_t x0, uint32_t x1) {
    const uint32_t lo = x0 > pre ? x0 - pre : 0u;
    const uint32_t hi = x1 > pre ? (uint32_t)umin64(x1 - pre, c) : 0u;
    if (hi <= lo) return 0;
    const uint32_t m = (hi >= 32 ? 0xffffffffu : (1u << hi) - 1u) & ~((1u << lo) - 1u);
    return __popc(v & m);
}

// Add ones to the tiles of the next level: one atomic per distinct tile of a warp.
__device__ __forceinline__ void count_key(uint32_t* next_count, bool active, uint64_t key, uint32_t ones) {
    const uint64_t k = active ? key : ~0ull;
    const uint32_t grp = __match_any_sync(0xffffffffu, k);
    const uint32_t sum = __reduce_add_sync(grp, active ? ones : 0u);
    if (active && sum && (threadIdx.x & 31) == (uint32_t)(__ffs(grp) - 1)) atomicAdd(next_count + key, sum);
}

// A run of output bits [d, e) (multi-node tiles): shifted out of an image whose
// run bit 0 sits at image bit pos0.
struct Run {
    uint64_t k0;       // first output word
    uint32_t nw;       // output words (0: nothing to write)
    uint32_t wb;       // image word of output word 0's window
    uint32_t sh;       // bit offset of the window in the image words
    uint32_t fmask;    // bits of the first word inside the run
    uint32_t lmask;    // bits of the last word inside the run
};
__device__ __forceinline__ Run make_run(uint64_t d, uint64_t n, uint64_t lim, uint32_t pos0) {
    Run r;
    r.nw = 0;
    r.k0 = 0;
    r.wb = r.sh = 0;
    r.fmask = r.lmask = 0;
    if (n == 0 || d >= lim) return r;
    const uint64_t e = umin64(d + n, lim);
    const uint32_t s = (uint32_t)d & 31u;
    r.k0 = d >> 5;
    r.nw = (uint32_t)(((e - 1) >> 5) - r.k0 + 1);
    const uint32_t p = pos0 - s;  // image position of output word 0's bit 0
    r.wb = p >> 5;
    r.sh = p & 31u;
    r.fmask = ~((1u << s) - 1u);
    r.lmask = (e & 31) ? (1u << (e & 31)) - 1u : 0xffffffffu;
    if (r.nw == 1) r.fmask &= r.lmask;
    return r;
}
// Output word i of a run: a store when the run covers the word, an OR into a
// zero-initialised word shared with another run otherwise.  Returns its ones.
__device__ __forceinline__ uint32_t run_word(const Run& r, uint32_t i, const uint32_t* img, uint32_t* plane) {
    uint32_t v = r.sh ? __funnelshift_r(img[r.wb + i], img[r.wb + i + 1], r.sh) : img[r.wb + i];
    const uint32_t mask = i == 0 ? r.fmask : (i + 1 == r.nw ? r.lmask : 0xffffffffu);
    if (mask == 0xffffffffu) {
        plane[r.k0 + i] = v;
    } else {
        v &= mask;
        atomicOr(plane + r.k0 + i, v);
    }
    return __popc(v);
}
// Plan of a single-node run of n bits at output bit d (image bit d mod 128 of its image).
__device__ __forceinline__ RunPlan plan_run(uint64_t d, uint64_t n, uint64_t lim) {
    RunPlan p;
    const Run r = make_run(d, n, lim, (uint32_t)d & 127u);
    p.k0 = r.k0;
    p.nw = r.nw;
    p.wb = r.wb;
    p.fmask = r.fmask;
    p.lmask = r.lmask;
    // whole words [f, l) and their 16-byte aligned part [ta, tb)
    const uint32_t f = r.fmask == 0xffffffffu ? 0u : 1u;
    const uint32_t l = (r.nw > 0 && (r.nw == 1 ? r.fmask : r.lmask) != 0xffffffffu) ? r.nw - 1 : r.nw;
    uint32_t ta = f + ((4u - (uint32_t)((r.k0 + f) & 3)) & 3u);
    uint32_t tb = l >= 4 ? l - (uint32_t)((r.k0 + l) & 3) : 0u;
    if (ta > r.nw) ta = r.nw;
    if (tb < ta) tb = ta;
    p.ta = ta;
    p.tb = tb;
    p.tile = d / kTile;
    return p;
}
// One of the (at most eight) output words around a run's bulk span, or nothing.
__device__ __forceinline__ void plan_edge_word(const RunPlan& p, uint32_t q, const uint32_t* img, uint32_t* plane) {
    const uint32_t i = q < p.ta ? q : p.tb + (q - p.ta);
    if (i >= p.nw) return;
    uint32_t v = img[p.wb + i];
    const uint32_t mask = i == 0 ? p.fmask : (i + 1 == p.nw ? p.lmask : 0xffffffffu);
    if (mask == 0xffffffffu) plane[p.k0 + i] = v;
    else atomicOr(plane + p.k0 + i, v & mask);
}

// Write plane j's runs from images img0 (zeros) and img1 (ones).  Single-node
// tiles: 16 threads (base..base+15) write the words around two bulk copies;
// several nodes: one warp per node.  Returns nothing; j == 1 also counts ones.
template <bool FIRST>
__device__ __forceinline__ void write_plane(TileSmem& S, const LevelArgs& a, uint32_t j, const uint32_t* img0,
                                            const uint32_t* img1, bool single, uint32_t base) {
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* plane = j == 1 ? a.out0 : a.out + (uint64_t)(j - 2) * a.pstride;
    if (single) {
        if (tid >= base && tid < base + 16) {
            const uint32_t t = tid - base;
            const RunPlan& p = S.run[t >> 3];
            const uint32_t* img = t < 8 ? img0 : img1;
            const uint32_t q = t & 7;
            if (q == 0 && p.tb > p.ta) bulk_s2g(plane + p.k0 + p.ta, img + p.wb + p.ta, 4 * (p.tb - p.ta));
            plan_edge_word(p, q, img, plane);
            if (FIRST && q == 0) {  // this run's ones of B_{l+1}, per tile of level l+1
                const uint32_t k = (t >> 3) * 2;
                if (S.ones[k]) atomicAdd(a.next_count + p.tile, S.ones[k]);
                if (S.ones[k + 1]) atomicAdd(a.next_count + p.tile + 1, S.ones[k + 1]);
            }
        }
        return;
    }
    const uint64_t t0 = S.t0, E = S.E, lim = a.size_next;
    const uint32_t count = S.count, O = S.O, nw = (count + 31) / 32;
    auto ones_before = [&](uint32_t r) -> uint32_t {
        const uint32_t wi = r >> 5;
        if (wi >= nw) return O;
        return S.pre[wi] + __popc(S.b[wi] & ((1u << (r & 31)) - 1u));
    };
    for (uint64_t p = S.p0 + warp; p < a.nnodes; p += kTileThreads / 32) {
        const uint64_t st = __ldg(&a.nodes[p].start);
        if (st >= t0 + count) break;
        const uint64_t en = p + 1 < a.nnodes ? __ldg(&a.nodes[p + 1].start) : a.size;
        const uint32_t q0 = (uint32_t)(umax64(st, t0) - t0), q1 = (uint32_t)(umin64(en, t0 + count) - t0);
        const uint32_t ob0 = ones_before(q0), ob1 = ones_before(q1);
        const uint32_t zs = q0 - ob0, ze = q1 - ob1;
        const Run rz = make_run(__ldg(&a.nodes[p].off0) + (t0 - E) + zs, ze - zs, lim, 32 + zs);
        const Run ro = make_run(__ldg(&a.nodes[p].off1) + E + ob0, ob1 - ob0, lim, 32 + ob0);
        for (uint32_t i0 = 0; i0 < rz.nw + ro.nw; i0 += 32) {
            const uint32_t i = i0 + lane;
            const bool act = i < rz.nw + ro.nw;
            uint32_t ones = 0;
            uint64_t k = 0;
            if (act) {
                if (i < rz.nw) {
                    ones = run_word(rz, i, img0, plane);
                    k = rz.k0 + i;
                } else {
                    ones = run_word(ro, i - rz.nw, img1, plane);
                    k = ro.k0 + (i - rz.nw);
                }
            }
            if (FIRST) count_key(a.next_count, act, k / kTileWords, ones);
        }
    }
}

__device__ __forceinline__ void cursor_tile(Cursor& c, const LevelArgs* args, const uint64_t* tile_prefix,
                                            uint32_t ntrees, uint64_t total) {
    if (c.g >= total) return;
    const uint32_t tr0 = c.tree;
    while (c.tree + 1 < ntrees && tile_prefix[c.tree + 1] <= c.g) c.tree++;
    if (c.tree != tr0 || c.bits == nullptr) {
        const LevelArgs& a = args[c.tree];
        c.R = a.R;
        c.bits = a.bits;
        c.in = a.in;
        c.pstride = a.pstride;
        c.size = a.size;
        c.first = tile_prefix[c.tree];
    }
    const uint64_t t0 = (c.g - c.first) * kTile;
    const uint32_t count = (uint32_t)umin64(kTile, c.size - t0);
    c.w0 = t0 >> 5;
    c.bytes = (((count + 31) / 32) * 4 + 15) & ~15u;
    c.j = 0;
}
__device__ __forceinline__ void cursor_pump(Cursor& c, TileSmem& S, uint32_t released, const LevelArgs* args,
                                            const uint64_t* tile_prefix, uint32_t ntrees, uint64_t total) {
    while (c.g < total && c.issued - released < kSlots) {
        const uint32_t slot = c.issued % kSlots;
        const uint32_t* src = (c.j == 0 ? c.bits : c.in + (uint64_t)(c.j - 1) * c.pstride) + c.w0;
        mbar_expect_tx(&S.mbar[slot], c.bytes);
        bulk_g2s(S.ring[slot], src, c.bytes, &S.mbar[slot]);
        c.issued++;
        if (++c.j == c.R) {
            c.g += gridDim.x;
            cursor_tile(c, args, tile_prefix, ntrees, total);
        }
    }
}

__global__ void __launch_bounds__(kTileThreads, 2) level_kernel(const LevelArgs* __restrict__ args,
                                                                const uint64_t* __restrict__ tile_prefix,
                                                                uint32_t ntrees) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    TileSmem& S = *reinterpret_cast<TileSmem*>(smem_raw);
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // threads that issue bulk copies: clears (0) and run write-outs (32, 40, 64, 72)
    const bool bulk_thread = tid == 0 || tid == 32 || tid == 40 || tid == 64 || tid == 72;
    const uint64_t total = tile_prefix[ntrees];
    Cursor& cur = S.cur;
    if (tid == 0) {
        for (uint32_t i = 0; i < kSlots; i++) mbar_init(&S.mbar[i], 1);
        mbar_fence_init();
        S.tree = 0xffffffffu;
    }
    for (uint32_t i = tid; i < kPairs * 2 * 2 * kImgWords / 4; i += kTileThreads)
        reinterpret_cast<uint4*>(&S.img[0][0][0][0])[i] = make_uint4(0, 0, 0, 0);
    S.zero[tid] = 0;
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
        cur.g = blockIdx.x;
        cur.tree = 0;
        cur.issued = 0;
        cur.bits = nullptr;
        cursor_tile(cur, args, tile_prefix, ntrees, total);
        cursor_pump(cur, S, 0, args, tile_prefix, ntrees, total);
    }
    uint32_t seq = 0;   // planes consumed by this CTA
    uint32_t pair = 0;  // plane pairs processed by this CTA (image slot rotation)
    uint32_t tree = 0;  // this thread's view of the current tile's tree
    for (uint64_t g = blockIdx.x; g < total; g += gridDim.x) {
        while (tree + 1 < ntrees && tile_prefix[tree + 1] <= g) tree++;
        if (tree != S.tree) {  // uniform: copy the tree's arguments (the previous tile is done with them)
            __syncthreads();
            if (tid < sizeof(LevelArgs) / 8)
                reinterpret_cast<uint64_t*>(&S.args)[tid] = reinterpret_cast<const uint64_t*>(args + tree)[tid];
            __syncthreads();
            if (tid == 0) S.tree = tree;
        }
        const LevelArgs& a = S.args;
        const uint32_t R = a.R;
        const uint64_t tile = g - tile_prefix[tree];
        const uint64_t t0 = tile * kTile;
        const uint64_t size = a.size;
        const uint32_t count = (uint32_t)umin64(kTile, size - t0);
        const uint32_t nw = (count + 31) / 32;
        // metadata loads, used after the next barrier
        const uint64_t E = a.prefix[tile];                                   // ones of B_l before the tile
        const uint64_t EL1 = a.prefix[tile & ~(uint64_t)(kTilesPerL1 - 1)];  // ... before its L1 block
        const uint64_t p0 = (R > 1 && a.nnodes > 1) ? umin64(a.first_node[tile], a.nnodes - 1) : 0;

        // ---- plane 0 = B_l (waited by warp 0 before the barrier) ----
        if (warp == 0) mbar_wait(&S.mbar[seq % kSlots], (seq / kSlots) & 1u, a.status);
        __syncthreads();
        if (tid < 4) S.ones[tid] = 0;
        const uint32_t valid = tid < nw ? ((tid == nw - 1 && (count & 31)) ? (1u << (count & 31)) - 1u : 0xffffffffu) : 0u;
        const uint32_t m1 = S.ring[seq % kSlots][tid] & valid, m0 = ~m1 & valid;
        const uint32_t c1 = __popc(m1), c0 = __popc(m0);
        uint32_t inc = c1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= (uint32_t)o) inc += t;
        }
        if (lane == 31) S.wsum[warp] = inc;
        uint32_t mv0[5], mv1[5];
        if (R > 1) {
            compress_masks(m0, mv0);
            compress_masks(m1, mv1);
            if (warp == 0) {  // planes 1 and 2 (the first pair)
                mbar_wait(&S.mbar[(seq + 1) % kSlots], ((seq + 1) / kSlots) & 1u, a.status);
                if (R > 2) mbar_wait(&S.mbar[(seq + 2) % kSlots], ((seq + 2) / kSlots) & 1u, a.status);
            }
        } else if (warp == 0 && g + gridDim.x < total) {  // next tile's plane 0
            mbar_wait(&S.mbar[(seq + 1) % kSlots], ((seq + 1) / kSlots) & 1u, a.status);
        }
        __syncthreads();
        if (tid == 0) cursor_pump(cur, S, seq + 1, args, tile_prefix, ntrees, total);  // plane 0's slot is free
        const uint32_t ws = lane < kTileThreads / 32 ? S.wsum[lane] : 0u;
        const uint32_t before = __reduce_add_sync(0xffffffffu, lane < warp ? ws : 0u);
        const uint32_t O = __reduce_add_sync(0xffffffffu, ws);  // ones of the tile
        const uint32_t pre1 = before + inc - c1;  // ones before this word within the tile
        const uint32_t pre0 = 32 * tid - pre1;    // zeros before it (earlier words are full)

        // ---- level l: L1 / L2 counters and select samples ----
        if ((tid & 15) == 0 && tid < nw) a.l2[(t0 >> 9) + (tid >> 4)] = (uint16_t)(E - EL1 + pre1);
        if (tid == 0) {
            if ((tile & (kTilesPerL1 - 1)) == 0) a.l1[t0 >> 16] = E;
            if (t0 + count == size && (size & 511) == 0) {
                if ((size & 65535) == 0) {
                    a.l1[size >> 16] = E + O;
                    a.l2[size >> 9] = 0;
                } else {
                    a.l2[size >> 9] = (uint16_t)(E + O - EL1);
                }
            }
            if (tile == 0) {
                a.s0[0] = 0;
                a.s1[0] = 0;
            }
        }
        if (tid < nw) {  // at most one sample of each kind per word (K >= 256)
            const uint32_t kl = a.k_log2;
            const uint64_t g1 = E + pre1, g0 = (t0 - E) + pre0;  // ones / zeros before the word
            const uint64_t base = t0 + 32ull * tid;
            if (((g1 + c1) >> kl) != (g1 >> kl)) {
                const uint64_t m = (g1 + c1) >> kl;
                if (m < a.n_s1) a.s1[m] = base + select_in_word(m1, (uint32_t)((m << kl) - g1));
            }
            if (((g0 + c0) >> kl) != (g0 >> kl)) {
                const uint64_t m = (g0 + c0) >> kl;
                if (m < a.n_s0) a.s0[m] = base + select_in_word(m0, (uint32_t)((m << kl) - g0));
            }
        }
        if (R == 1) {
            seq += 1;
            continue;
        }

        // ---- runs of the tile in T_{l+1} ----
        S.b[tid] = m1;
        S.pre[tid] = pre1;
        const uint64_t lim = a.size_next;
        const bool single = p0 + 1 >= a.nnodes || __ldg(&a.nodes[p0 + 1].start) >= t0 + count;
        uint32_t qz, qo;               // image bits of this thread's zero / one piece
        uint32_t thr[4] = {0, 0, 0, 0};  // per run: bits before the next tile of level l+1, bits below size_{l+1}
        if (single) {
            // each run's image is aligned with its output words (image word k0 mod 4
            // holds output word k0), so whole words leave by bulk copy
            const uint64_t d0 = __ldg(&a.nodes[p0].off0) + (t0 - E);
            const uint64_t d1 = __ldg(&a.nodes[p0].off1) + E;
            qz = ((uint32_t)d0 & 127u) + pre0;
            qo = ((uint32_t)d1 & 127u) + pre1;
            if (tid == 0) S.run[0] = plan_run(d0, count - O, lim);
            if (tid == 8) S.run[1] = plan_run(d1, O, lim);
            thr[0] = (uint32_t)umin64(((d0 / kTile) + 1) * kTile - d0, count - O);
            thr[1] = d0 >= lim ? 0u : (uint32_t)umin64(count - O, lim - d0);
            thr[2] = (uint32_t)umin64(((d1 / kTile) + 1) * kTile - d1, O);
            thr[3] = d1 >= lim ? 0u : (uint32_t)umin64(O, lim - d1);
        } else {
            // several nodes: images start at bit 32 and runs are shifted into place
            qz = 32 + pre0;
            qo = 32 + pre1;
            if (tid == 0) {
                S.t0 = t0;
                S.E = E;
                S.p0 = p0;
                S.count = count;
                S.O = O;
            }
        }

        // ---- planes 1..R-1 in pairs (planes of a pair are ready: waited before the last barrier) ----
        if (tid == 0) {
            S.t0 = t0;
            S.count = count;
        }
        auto do_pair = [&](auto first_tag, uint32_t j) {
            constexpr bool FIRST = decltype(first_tag)::value;
            const bool two = j + 1 < R;
            const uint32_t ps = pair % kPairs;
            if (tid == 0) {  // consumed input planes: clear for reuse as outputs
                const uint32_t bytes = (((S.count + 31) / 32) * 4 + 15) & ~15u;
                const uint64_t w0 = S.t0 >> 5;
                bulk_s2g(a.in + (uint64_t)(j - 1) * a.pstride + w0, S.zero, bytes);
                if (two) bulk_s2g(a.in + (uint64_t)j * a.pstride + w0, S.zero, bytes);
            }
            {
                const uint32_t x = S.ring[(seq + j) % kSlots][tid];
                const uint32_t cz = compress_left(x & m0, mv0), co = compress_left(x & m1, mv1);
                place(S.img[ps][0][0], qz, c0, cz);
                place(S.img[ps][0][1], qo, c1, co);
                if (FIRST && single) {
                    // ones of B_{l+1}: per run, before and after the tile boundary of level l+1
                    const uint32_t vz = c0 ? cz >> (32 - c0) : 0u, vo = c1 ? co >> (32 - c1) : 0u;
                    uint32_t n0 = ones_in(vz, pre0, c0, 0, umin64(thr[0], thr[1]));
                    uint32_t n1 = ones_in(vz, pre0, c0, thr[0], thr[1]);
                    uint32_t n2 = ones_in(vo, pre1, c1, 0, umin64(thr[2], thr[3]));
                    uint32_t n3 = ones_in(vo, pre1, c1, thr[2], thr[3]);
                    n0 = __reduce_add_sync(0xffffffffu, n0);
                    n1 = __reduce_add_sync(0xffffffffu, n1);
                    n2 = __reduce_add_sync(0xffffffffu, n2);
                    n3 = __reduce_add_sync(0xffffffffu, n3);
                    if (lane == 0) {
                        if (n0) atomicAdd(&S.ones[0], n0);
                        if (n1) atomicAdd(&S.ones[1], n1);
                        if (n2) atomicAdd(&S.ones[2], n2);
                        if (n3) atomicAdd(&S.ones[3], n3);
                    }
                }
            }
            if (two) {
                const uint32_t x = S.ring[(seq + j + 1) % kSlots][tid];
                place(S.img[ps][1][0], qz, c0, compress_left(x & m0, mv0));
                place(S.img[ps][1][1], qo, c1, compress_left(x & m1, mv1));
            }
            fence_proxy_async();
            if (bulk_thread) bulk_wait_read<0>();  // the previous pair's images have been read
            if (warp == 0) {  // the next pair, or the next tile's plane 0
                const uint32_t n0 = j + 2, n1 = j + 3;
                if (n0 < R) {
                    mbar_wait(&S.mbar[(seq + n0) % kSlots], ((seq + n0) / kSlots) & 1u, a.status);
                    if (n1 < R) mbar_wait(&S.mbar[(seq + n1) % kSlots], ((seq + n1) / kSlots) & 1u, a.status);
                } else if (g + gridDim.x < total) {
                    mbar_wait(&S.mbar[(seq + R) % kSlots], ((seq + R) / kSlots) & 1u, a.status);
                }
            }
            __syncthreads();
            if (tid == 0) cursor_pump(cur, S, seq + j + (two ? 2 : 1), args, tile_prefix, ntrees, total);
            write_plane<FIRST>(S, a, j, S.img[ps][0][0], S.img[ps][0][1], single, 32);
            if (two) write_plane<false>(S, a, j + 1, S.img[ps][1][0], S.img[ps][1][1], single, 64);
            if (bulk_thread) bulk_commit();
            // the slot of the pair before last is free (its reads were waited before the last barrier)
            uint4* z = reinterpret_cast<uint4*>(&S.img[(pair + 2) % kPairs][0][0][0]);
            for (uint32_t i = tid; i < 2 * 2 * kImgWords / 4; i += kTileThreads) z[i] = make_uint4(0, 0, 0, 0);
            pair++;
        };
        do_pair(BoolTag<true>(), 1);
        for (uint32_t j = 3; j < R; j += 2) do_pair(BoolTag<false>(), j);
        seq += R;
    }
    if (bulk_thread) bulk_wait_all();
}

// ===========================================================================
// first node of every tile (levels with several nodes)
// ===========================================================================

// One thread per tile of every tree: the last internal node starting at or
// before the tile's first position (binary search over the node starts).
__global__ void __launch_bounds__(256) first_node_kernel(const LevelArgs* __restrict__ args,
                                                         const uint64_t* __restrict__ tile_prefix, uint32_t ntrees) {
    const uint64_t total = tile_prefix[ntrees];
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t tree = ntrees > 1 ? find_tree(tile_prefix, ntrees, g) : 0u;
        const LevelArgs& a = args[tree];
        if (a.R < 2 || a.nnodes < 2) continue;
        const uint64_t tile = g - tile_prefix[tree];
        const uint64_t t0 = tile * kTile;
        uint64_t lo = 0, hi = a.nnodes - 1;
        while (lo < hi) {
            const uint64_t mid = (lo + hi + 1) >> 1;
            if (__ldg(&a.nodes[mid].start) <= t0) lo = mid;
            else hi = mid - 1;
        }
        a.first_node[tile] = (uint32_t)lo;
    }
}

// ===========================================================================
// prefixes: exclusive scan of per-tile counts, one CTA per tree
// ===========================================================================

__global__ void __launch_bounds__(1024) count_scan_kernel(const LevelArgs* __restrict__ args) {
    __shared__ uint64_t s_w[32];
    __shared__ uint64_t s_carry;
    const LevelArgs& a = args[blockIdx.x];
    const uint64_t n = level_tiles(a.size);
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (uint64_t base = 0; base < n; base += 1024 * kScanPerThread) {
        uint64_t v[kScanPerThread];
        uint64_t sum = 0;
#pragma unroll
        for (uint32_t k = 0; k < kScanPerThread; k++) {
            const uint64_t i = base + (uint64_t)tid * kScanPerThread + k;
            v[k] = i < n ? a.count[i] : 0;
            sum += v[k];
        }
        uint64_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= (uint32_t)o) inc += t;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            uint64_t x = s_w[lane], xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t t = __shfl_up_sync(0xffffffffu, xi, o);
                if (lane >= (uint32_t)o) xi += t;
            }
            s_w[lane] = xi - x;
        }
        __syncthreads();
        uint64_t run = s_carry + s_w[warp] + inc - sum;
#pragma unroll
        for (uint32_t k = 0; k < kScanPerThread; k++) {
            const uint64_t i = base + (uint64_t)tid * kScanPerThread + k;
            if (i < n) a.prefix[i] = run;
            run += v[k];
        }
        __syncthreads();
        if (tid == 1023) s_carry = run;
        __syncthreads();
    }
}

// ===========================================================================
// launchers
// ===========================================================================

wt_status launch_transpose(const TransposeArgs* d_args, const uint64_t* d_chunk_prefix, uint32_t ntrees,
                           uint64_t chunks, uint32_t w, cudaStream_t s) {
    if (!chunks) return WT_OK;
    ProfScope ps("transpose", s);
    if (w == 1) transpose_kernel<uint8_t><<<(unsigned)chunks, kTrThreads, 0, s>>>(d_args, d_chunk_prefix, ntrees);
    else if (w == 2) transpose_kernel<uint16_t><<<(unsigned)chunks, kTrThreads, 0, s>>>(d_args, d_chunk_prefix, ntrees);
    else transpose_kernel<uint32_t><<<(unsigned)chunks, kTrThreads, 0, s>>>(d_args, d_chunk_prefix, ntrees);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

wt_status launch_level(const LevelArgs* d_args, const uint64_t* d_tile_prefix, uint32_t ntrees,
                       uint64_t max_tiles, cudaStream_t s) {
    static int per_sm = 0;
    const size_t sm = sizeof(TileSmem);
    if (!per_sm) {
        if (cudaFuncSetAttribute(level_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
            return WT_ECUDA;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, level_kernel, kTileThreads, sm);
        if (per_sm <= 0) per_sm = 1;
    }
    const uint64_t grid = umin64(max_tiles ? max_tiles : 1, (uint64_t)per_sm * sm_count());
    ProfScope ps("level", s);
    level_kernel<<<(unsigned)grid, kTileThreads, sm, s>>>(d_args, d_tile_prefix, ntrees);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

wt_status launch_first_node(const LevelArgs* d_args, const uint64_t* d_tile_prefix, uint32_t ntrees,
                            uint64_t max_tiles, cudaStream_t s) {
    const uint64_t grid = umin64((max_tiles + 255) / 256 + 1, (uint64_t)sm_count() * 8);
    ProfScope ps("first_node", s);
    first_node_kernel<<<(unsigned)grid, 256, 0, s>>>(d_args, d_tile_prefix, ntrees);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

wt_status launch_count_scan(const LevelArgs* d_args, uint32_t ntrees, cudaStream_t s) {
    if (!ntrees) return WT_OK;
    ProfScope ps("count_scan", s);
    count_scan_kernel<<<ntrees, 1024, 0, s>>>(d_args);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

}  // namespace wt
