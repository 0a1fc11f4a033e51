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
// Per level:
//  * rank pass (B_l only; tiles of 65,536 bits = one L1 block): popcounts, a
//    decoupled look-back for the ones before the tile, the L1/L2 counters
//    (Section 4.1) and select samples (Section 4.2), the ones before every
//    move tile and its first node, and a zero in every output word that two
//    runs share (the move pass ORs into those and stores all others);
//  * move pass (tiles of 16,384 elements, independent of each other):
//    planes 1..R-1 of T_l -> B_{l+1} and planes 1..R-2 of T_{l+1}.
// Level 0's planes come from S by a 32x32 bit-matrix transpose of the codes.
// Every kernel walks the work items of one or many trees (a batch), so a
// single tree is a batch of one.
#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_device.cuh"
#include "wt_internal.hpp"

namespace wt {

constexpr uint32_t kRankThreads = 512;  // four 32-bit words per thread
constexpr uint32_t kRankWords = kRankTile / 32;
constexpr uint32_t kMoveThreads = 512;  // one 32-bit word of every plane per thread
constexpr uint32_t kMoveWords = kMoveTile / 32;
constexpr uint32_t kMovesPerRank = kRankTile / kMoveTile;
constexpr uint32_t kSlots = 8;          // plane ring of the move pass
constexpr uint32_t kImgWords = 520;     // one run image: 512 words + read-ahead
constexpr uint32_t kTrThreads = 256;    // transpose: 32 symbols per thread
constexpr uint32_t kTrTable = 1024;     // codes tabulated in shared memory up to this sigma

uint64_t transpose_chunks(uint64_t words32) { return (words32 + kTrThreads - 1) / kTrThreads; }
uint64_t plane_stride(uint64_t n) { return (n + kMoveTile - 1) / kMoveTile * kMoveWords; }

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

// Shift masks of compress(., m): stage i moves the selected bits right by 2^i.
// A bit of m moves right by the number of zeros of m below it; stage i takes
// the bits whose remaining distance has bit i set, found as the parity of the
// zeros below them (a prefix XOR).
__device__ __forceinline__ void compress_masks(uint32_t m, uint32_t (&mv)[5]) {
    uint32_t mk = ~m << 1;  // zeros of m, seen from the bit above
#pragma unroll
    for (int i = 0; i < 5; i++) {
        uint32_t mp = mk ^ (mk << 1);  // prefix XOR: parity of the marked bits at or below
        mp ^= mp << 2;
        mp ^= mp << 4;
        mp ^= mp << 8;
        mp ^= mp << 16;
        const uint32_t v = mp & m;
        mv[i] = v;
        m = (m ^ v) | (v >> (1 << i));
        mk &= ~mp;
    }
}
// The bits of x under m, packed towards bit 0 in order.
__device__ __forceinline__ uint32_t compress(uint32_t x, uint32_t m, const uint32_t (&mv)[5]) {
    x &= m;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const uint32_t t = x & mv[i];
        x = (x ^ t) | (t >> (1 << i));
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

// One CTA per 256 words of 32 symbols of one tree.  A thread reads its 32
// symbols, encodes them, transposes the 32 codes and writes one word of every
// plane (plane 0 into B_0).  Words of B_0 past n are written as zeros.
template <typename T>
__global__ void __launch_bounds__(kTrThreads) transpose_kernel(const TransposeArgs* __restrict__ args,
                                                               const uint64_t* __restrict__ chunk_prefix,
                                                               uint32_t ntrees) {
    __shared__ uint32_t s_code[kTrTable];
    __shared__ uint32_t s_tree;
    if (threadIdx.x == 0) s_tree = ntrees > 1 ? find_tree(chunk_prefix, ntrees, blockIdx.x) : 0u;
    __syncthreads();
    const TransposeArgs& a = args[s_tree];
    const uint64_t n = a.n;
    const uint32_t sigma = a.sigma, L = a.L;
    CodeParams cp;  // encode() reads sigma, L and pow2 only
    cp.sigma = sigma;
    cp.L = L;
    cp.pow2 = a.pow2;
    const bool table = !cp.pow2 && sigma <= kTrTable;
    if (table) {
        for (uint32_t s = threadIdx.x; s < sigma; s += kTrThreads) {
            uint32_t code, len;
            encode(cp, s, code, len);
            s_code[s] = code;
        }
        __syncthreads();
    }
    const uint64_t word = (blockIdx.x - chunk_prefix[s_tree]) * kTrThreads + threadIdx.x;
    if (word >= a.bits0_words) return;
    const uint64_t e0 = word * 32;
    if (e0 >= n) {
        a.bits0[word] = 0;
        return;
    }
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
    transpose32(A);
#pragma unroll
    for (int b = 0; b < 32; b++) {
        if ((uint32_t)b < L) {
            const uint32_t j = L - 1 - b;  // plane j holds code bit L-1-j
            if (j == 0) a.bits0[word] = A[b];
            else a.planes[(uint64_t)(j - 1) * a.pstride + word] = A[b];
        }
    }
}

// ===========================================================================
// rank pass
// ===========================================================================

// Zero the first and the last word of a run of output bits [d, d + nbits)
// (clipped at lim) when the run covers them only partly; the move pass ORs
// into exactly those words.
__device__ __forceinline__ void zero_run_edges(const LevelArgs& a, uint64_t d, uint64_t nbits) {
    const uint64_t lim = a.size_next;
    if (nbits == 0 || d >= lim) return;
    const uint64_t e = umin64(d + nbits, lim);
    const uint32_t np = a.R - 2;  // output planes besides B_{l+1}
    if (d & 31) {
        const uint64_t w = d >> 5;
        a.out0[w] = 0;
        for (uint32_t j = 0; j < np; j++) a.out[j * a.pstride + w] = 0;
    }
    if (e & 31) {
        const uint64_t w = (e - 1) >> 5;
        a.out0[w] = 0;
        for (uint32_t j = 0; j < np; j++) a.out[j * a.pstride + w] = 0;
    }
}

__global__ void __launch_bounds__(kRankThreads) rank_pass_kernel(const LevelArgs* __restrict__ args,
                                                                 const uint64_t* __restrict__ tile_prefix,
                                                                 uint32_t ntrees, unsigned long long* __restrict__ counter) {
    __shared__ uint32_t s_b[kRankWords];    // B_l words of the tile
    __shared__ uint32_t s_pre[kRankWords];  // ones before each word within the tile
    __shared__ uint32_t s_wsum[kRankThreads / 32];
    __shared__ uint64_t s_g, s_E;
    __shared__ uint32_t s_tree;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t total = tile_prefix[ntrees];
    for (;;) {
        if (tid == 0) {
            const uint64_t g = atomicAdd(counter, 1ull);
            s_g = g;
            if (g < total) s_tree = ntrees > 1 ? find_tree(tile_prefix, ntrees, g) : 0u;
        }
        __syncthreads();
        const uint64_t g = s_g;
        if (g >= total) break;
        const LevelArgs& a = args[s_tree];
        const uint64_t tile = g - tile_prefix[s_tree];
        const uint64_t size = a.size;
        const uint64_t t0 = tile * kRankTile;
        const uint32_t count = (uint32_t)umin64(kRankTile, size - t0);
        const uint32_t nw = (count + 31) / 32;

        // ---- words, popcounts, prefix within the tile ----
        const uint32_t w0 = tid * 4;
        uint32_t w[4];
        const uint32_t* src = a.bits + (t0 >> 5) + w0;
        if (w0 + 4 <= nw) {
            const uint4 q = *reinterpret_cast<const uint4*>(src);
            w[0] = q.x;
            w[1] = q.y;
            w[2] = q.z;
            w[3] = q.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                w[k] = 0u;
                if (w0 + k < nw) w[k] = src[k];
            }
        }
        if (count & 31) {
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (w0 + k == nw - 1) w[k] &= (1u << (count & 31)) - 1u;
        }
        const uint32_t c = __popc(w[0]) + __popc(w[1]) + __popc(w[2]) + __popc(w[3]);
        uint32_t inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= (uint32_t)o) inc += t;
        }
        if (lane == 31) s_wsum[warp] = inc;
        __syncthreads();
        uint32_t before = 0, ones = 0;
#pragma unroll
        for (uint32_t i = 0; i < kRankThreads / 32; i++) {
            const uint32_t v = s_wsum[i];
            before += i < warp ? v : 0u;
            ones += v;
        }
        const uint32_t pre = before + inc - c;  // ones before this thread's first word
        {
            uint32_t p = pre;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                s_b[w0 + k] = w[k];
                s_pre[w0 + k] = p;
                p += __popc(w[k]);
            }
        }
        if (warp == 0) {
            const uint64_t E = lookback_warp(a.state, tile, ones, a.status, kSpinCap);
            if (lane == 0) s_E = E;
        }
        __syncthreads();
        const uint64_t E = s_E;  // ones of B_l before the tile

        // ---- L1 / L2 counters (the tile is one L1 block) ----
        if (tid == 0) a.l1[t0 >> 16] = E;
        if ((tid & 3) == 0 && w0 < nw) a.l2[(t0 >> 9) + tid / 4] = (uint16_t)pre;
        if (tid == 0 && t0 + count == size && (size & 511) == 0) {
            if ((size & 65535) == 0) {
                a.l1[size >> 16] = E + ones;
                a.l2[size >> 9] = 0;
            } else {
                a.l2[size >> 9] = (uint16_t)ones;
            }
        }
        // ---- select samples: at most one of each kind per word (K >= 256) ----
        if (tid == 0 && tile == 0) {
            a.s0[0] = 0;
            a.s1[0] = 0;
        }
        {
            const uint32_t kl = a.k_log2;
            uint32_t p = pre;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t wi = w0 + k;
                if (wi < nw) {
                    const uint32_t x = w[k];
                    const uint32_t valid = (wi == nw - 1 && (count & 31)) ? (1u << (count & 31)) - 1u : 0xffffffffu;
                    const uint32_t z = ~x & valid;
                    const uint32_t c1 = __popc(x), c0 = __popc(z);
                    const uint64_t g1 = E + p;                       // ones before the word
                    const uint64_t g0 = (t0 - E) + 32ull * wi - p;   // zeros before the word
                    const uint64_t base = t0 + 32ull * wi;
                    if (((g1 + c1) >> kl) != (g1 >> kl)) {
                        const uint64_t m = (g1 + c1) >> kl;
                        if (m < a.n_s1) a.s1[m] = base + select_in_word(x, (uint32_t)((m << kl) - g1));
                    }
                    if (((g0 + c0) >> kl) != (g0 >> kl)) {
                        const uint64_t m = (g0 + c0) >> kl;
                        if (m < a.n_s0) a.s0[m] = base + select_in_word(z, (uint32_t)((m << kl) - g0));
                    }
                    p += c1;
                }
            }
        }

        // ---- move tiles: ones before each, its first node, shared output words ----
        if (a.out0 != nullptr && warp < kMovesPerRank) {
            const uint64_t m0 = t0 + (uint64_t)warp * kMoveTile;
            if (m0 < size) {
                const uint64_t mt = tile * kMovesPerRank + warp;
                const uint64_t mend = umin64(m0 + kMoveTile, size);
                const uint64_t Pm = E + s_pre[warp * kMoveWords];  // ones before the move tile
                const uint64_t p0 = a.nnodes > 1 ? warp_find_node(a.nodes, a.nnodes, m0) : 0;
                if (lane == 0) {
                    a.prefix[mt] = Pm;
                    a.first_node[mt] = (uint32_t)p0;
                }
                if (a.size_next > 0) {
                    // ones before position t0 + r of this rank tile, 0 <= r <= count
                    auto ones_before = [&](uint32_t r) -> uint32_t {
                        const uint32_t wi = r >> 5;
                        if (wi >= nw) return ones;
                        return s_pre[wi] + __popc(s_b[wi] & ((1u << (r & 31)) - 1u));
                    };
                    for (uint64_t pb = p0;; pb += 32) {
                        const uint64_t p = pb + lane;
                        bool inside = false;
                        if (p < a.nnodes) {
                            const NodeEntry ne = a.nodes[p];
                            const uint64_t st = ne.start;
                            const uint64_t en = p + 1 < a.nnodes ? __ldg(&a.nodes[p + 1].start) : size;
                            inside = st < mend;
                            const uint64_t q0 = umax64(st, m0), q1 = umin64(en, mend);
                            if (inside && q0 < q1) {
                                const uint32_t ob0 = ones_before((uint32_t)(q0 - t0));
                                const uint32_t ob1 = ones_before((uint32_t)(q1 - t0));
                                const uint64_t r1 = E + ob0, r0 = q0 - r1;
                                zero_run_edges(a, ne.off0 + r0, (q1 - q0) - (ob1 - ob0));
                                zero_run_edges(a, ne.off1 + r1, ob1 - ob0);
                            }
                        }
                        if (!__shfl_sync(0xffffffffu, inside, 31)) break;
                    }
                }
            }
        }
        // ---- B_{l+1} past size_{l+1} stays zero ----
        if (a.out0 != nullptr && t0 + count == size)
            for (uint64_t i = ((a.size_next + 31) >> 5) + tid; i < a.out0_words; i += kRankThreads) a.out0[i] = 0;
        __syncthreads();
    }
}

// ===========================================================================
// move pass
// ===========================================================================

struct MoveSmem {
    uint32_t ring[kSlots][kMoveWords];  // planes in flight
    uint32_t img[3][2][kImgWords];      // zero-run / one-run images, three sets in rotation
    uint32_t b[kMoveWords];             // B_l words of the tile
    uint32_t pre[kMoveWords];           // ones before each word within the tile
    uint64_t mbar[kSlots];
    uint32_t wsum[kMoveThreads / 32];
};

// Append a compressed piece of cnt bits at bit offset off of a run image.
__device__ __forceinline__ void place(uint32_t* img, uint32_t off, uint32_t cnt, uint32_t v) {
    if (cnt == 0) return;
    const uint32_t wi = off >> 5, sh = off & 31;
    atomicOr(img + wi, v << sh);
    if (sh + cnt > 32) atomicOr(img + wi + 1, v >> (32 - sh));
}

// Output word k of a run [d, e) whose bits come from an image starting at
// image bit a0: a store when the run covers the word, an OR otherwise.
__device__ __forceinline__ void copy_word(uint32_t* dst, uint64_t k, uint64_t d, uint64_t e, const uint32_t* img,
                                          uint32_t a0) {
    const uint64_t gb = k << 5;
    const uint32_t lo = gb < d ? (uint32_t)(d - gb) : 0u;
    const uint32_t hi = gb + 32 > e ? (uint32_t)(e - gb) : 32u;
    const int64_t sp = (int64_t)a0 + (int64_t)(gb - d);  // image bit of output bit gb (>= -31)
    const int32_t wi = (int32_t)(sp >> 5);
    const uint32_t sh = (uint32_t)sp & 31u;
    const uint32_t lw = wi >= 0 ? img[wi] : 0u;
    const uint32_t v = __funnelshift_r(lw, img[wi + 1], sh);
    if (lo == 0 && hi == 32) {
        dst[k] = v;
    } else {
        const uint32_t mask = (hi == 32 ? 0xffffffffu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
        atomicOr(dst + k, v & mask);
    }
}

// A run's output words: first word index and count (0 if clipped away).
__device__ __forceinline__ uint64_t run_words(uint64_t d, uint64_t n, uint64_t lim, uint64_t& k0, uint64_t& e) {
    if (n == 0 || d >= lim) return 0;
    e = umin64(d + n, lim);
    k0 = d >> 5;
    return ((e - 1) >> 5) - k0 + 1;
}

__global__ void __launch_bounds__(kMoveThreads, 2) move_pass_kernel(const LevelArgs* __restrict__ args,
                                                                    const uint64_t* __restrict__ tile_prefix,
                                                                    uint32_t ntrees, unsigned long long* __restrict__ counter) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    MoveSmem& S = *reinterpret_cast<MoveSmem*>(smem_raw);
    __shared__ uint64_t s_g;
    __shared__ uint32_t s_tree;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (uint32_t i = 0; i < kSlots; i++) mbar_init(&S.mbar[i], 1);
        mbar_fence_init();
    }
    for (uint32_t i = tid; i < 3 * 2 * kImgWords; i += kMoveThreads) (&S.img[0][0][0])[i] = 0;
    uint32_t seq = 0;  // plane loads issued and consumed so far by this CTA
    const uint64_t total = tile_prefix[ntrees];
    for (;;) {
        if (tid == 0) {
            const uint64_t g = atomicAdd(counter, 1ull);
            s_g = g;
            if (g < total) s_tree = ntrees > 1 ? find_tree(tile_prefix, ntrees, g) : 0u;
        }
        __syncthreads();
        const uint64_t g = s_g;
        if (g >= total) break;
        const LevelArgs& a = args[s_tree];
        const uint64_t tile = g - tile_prefix[s_tree];
        const uint64_t t0 = tile * kMoveTile;
        const uint32_t count = (uint32_t)umin64(kMoveTile, a.size - t0);
        const uint32_t nw = (count + 31) / 32;
        const uint32_t R = a.R;
        const uint32_t bytes = (nw * 4 + 15) & ~15u;
        auto issue = [&](uint32_t j) {
            const uint32_t slot = (seq + j) % kSlots;
            const uint32_t* src = j == 0 ? a.bits + (t0 >> 5) : a.in + (uint64_t)(j - 1) * a.pstride + (t0 >> 5);
            mbar_expect_tx(&S.mbar[slot], bytes);
            bulk_g2s(S.ring[slot], src, bytes, &S.mbar[slot]);
        };
        if (tid == 0)
            for (uint32_t j = 0; j < R && j < kSlots; j++) issue(j);

        // ---- plane 0 = B_l: masks, counts, offsets within the tile ----
        mbar_wait(&S.mbar[seq % kSlots], (seq / kSlots) & 1u, a.status);
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
        const uint64_t E = a.prefix[tile];  // ones of B_l before the tile
        uint32_t mv0[5], mv1[5];
        compress_masks(m0, mv0);
        compress_masks(m1, mv1);
        __syncthreads();
        if (tid == 0 && R > kSlots) issue(kSlots);  // plane 0's slot is free
        uint32_t before = 0, O = 0;
#pragma unroll
        for (uint32_t i = 0; i < kMoveThreads / 32; i++) {
            const uint32_t v = S.wsum[i];
            before += i < warp ? v : 0u;
            O += v;
        }
        const uint32_t pre1 = before + inc - c1;  // ones before this word within the tile
        const uint32_t pre0 = 32 * tid - pre1;    // zeros before it (earlier words are full)
        S.b[tid] = m1;
        S.pre[tid] = pre1;

        // ---- nodes of the tile ----
        const uint64_t lim = a.size_next;
        const uint64_t p0 = a.nnodes > 1 ? umin64(a.first_node[tile], a.nnodes - 1) : 0;
        const bool single = p0 + 1 >= a.nnodes || __ldg(&a.nodes[p0 + 1].start) >= t0 + count;
        uint64_t d0 = 0, d1 = 0, k00 = 0, k01 = 0, e0 = 0, e1 = 0, nw0 = 0, nw1 = 0;
        if (single) {
            const NodeEntry& ne = a.nodes[p0];
            d0 = __ldg(&ne.off0) + (t0 - E);
            d1 = __ldg(&ne.off1) + E;
            nw0 = run_words(d0, count - O, lim, k00, e0);
            nw1 = run_words(d1, O, lim, k01, e1);
        }

        // ---- planes 1..R-1 ----
        for (uint32_t j = 1; j < R; j++) {
            const uint32_t u = seq + j, slot = u % kSlots;
            mbar_wait(&S.mbar[slot], (u / kSlots) & 1u, a.status);
            const uint32_t x = S.ring[slot][tid];
            const uint32_t set = j % 3;
            place(S.img[set][0], pre0, c0, compress(x, m0, mv0));
            place(S.img[set][1], pre1, c1, compress(x, m1, mv1));
            __syncthreads();
            if (tid == 0 && j + kSlots < R) issue(j + kSlots);
            uint32_t* dst = j == 1 ? a.out0 : a.out + (uint64_t)(j - 2) * a.pstride;
            const uint32_t* img0 = S.img[set][0];
            const uint32_t* img1 = S.img[set][1];
            if (single) {
                for (uint64_t i = tid; i < nw0 + nw1; i += kMoveThreads) {
                    if (i < nw0) copy_word(dst, k00 + i, d0, e0, img0, 0);
                    else copy_word(dst, k01 + (i - nw0), d1, e1, img1, 0);
                }
            } else {
                // one warp per node of the tile
                auto ones_before = [&](uint32_t r) -> uint32_t {
                    const uint32_t wi = r >> 5;
                    if (wi >= nw) return O;
                    return S.pre[wi] + __popc(S.b[wi] & ((1u << (r & 31)) - 1u));
                };
                for (uint64_t p = p0 + warp; p < a.nnodes; p += kMoveThreads / 32) {
                    const uint64_t st = __ldg(&a.nodes[p].start);
                    if (st >= t0 + count) break;
                    const uint64_t en = p + 1 < a.nnodes ? __ldg(&a.nodes[p + 1].start) : a.size;
                    const uint32_t r0 = (uint32_t)(umax64(st, t0) - t0), r1 = (uint32_t)(umin64(en, t0 + count) - t0);
                    const uint32_t ob0 = ones_before(r0), ob1 = ones_before(r1);
                    const uint32_t zs = r0 - ob0, ze = r1 - ob1;
                    uint64_t k0, e, kk0, ee;
                    const uint64_t dz = __ldg(&a.nodes[p].off0) + (t0 - E) + zs;
                    const uint64_t dn = __ldg(&a.nodes[p].off1) + E + ob0;
                    const uint64_t nz = run_words(dz, ze - zs, lim, k0, e);
                    const uint64_t no = run_words(dn, ob1 - ob0, lim, kk0, ee);
                    for (uint64_t i = lane; i < nz + no; i += 32) {
                        if (i < nz) copy_word(dst, k0 + i, dz, e, img0, zs);
                        else copy_word(dst, kk0 + (i - nz), dn, ee, img1, ob0);
                    }
                }
            }
            // the set used two planes ago is free (everyone passed this plane's barrier)
            uint32_t* z = &S.img[(j + 2) % 3][0][0];
            for (uint32_t i = tid; i < 2 * kImgWords; i += kMoveThreads) z[i] = 0;
        }
        seq += R;
        __syncthreads();
        if (R > 1) {
            uint32_t* z = &S.img[(R - 1) % 3][0][0];
            for (uint32_t i = tid; i < 2 * kImgWords; i += kMoveThreads) z[i] = 0;
        }
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

wt_status launch_rank_pass(const LevelArgs* d_args, const uint64_t* d_tile_prefix, uint32_t ntrees,
                           unsigned long long* counter, uint64_t max_tiles, cudaStream_t s) {
    static int per_sm = 0;
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rank_pass_kernel, kRankThreads, 0);
        if (per_sm <= 0) per_sm = 1;
    }
    const uint64_t grid = umin64(max_tiles ? max_tiles : 1, (uint64_t)per_sm * sm_count());
    ProfScope ps("rank_pass", s);
    rank_pass_kernel<<<(unsigned)grid, kRankThreads, 0, s>>>(d_args, d_tile_prefix, ntrees, counter);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

wt_status launch_move_pass(const LevelArgs* d_args, const uint64_t* d_tile_prefix, uint32_t ntrees,
                           unsigned long long* counter, uint64_t max_tiles, cudaStream_t s) {
    static int per_sm = 0;
    const size_t sm = sizeof(MoveSmem);
    if (!per_sm) {
        if (cudaFuncSetAttribute(move_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
            return WT_ECUDA;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, move_pass_kernel, kMoveThreads, sm);
        if (per_sm <= 0) per_sm = 1;
    }
    const uint64_t grid = umin64(max_tiles ? max_tiles : 1, (uint64_t)per_sm * sm_count());
    ProfScope ps("move_pass", s);
    move_pass_kernel<<<(unsigned)grid, kMoveThreads, sm, s>>>(d_args, d_tile_prefix, ntrees, counter);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

}  // namespace wt
