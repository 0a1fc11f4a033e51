// Shared definitions of libwt's CUDA sources.
//
// Reduced codes (Section 5.1, Algorithm 3) are not tabulated: they follow in
// closed form from the binary expansion of sigma.  Write
// sigma = 2^e[0] + 2^e[1] + ... + 2^e[r-1] with e[0] > ... > e[r-1] and
// P[i] = 2^e[0] + ... + 2^e[i-1].  The alphabet split of Section 5.1 (a node
// [a,b) sends [a, a+prevPow2(b-a)) left) peels these powers off the right
// spine, so [0, sigma) falls into r segments [P[i], P[i+1]), each a complete
// subtree of depth e[i].  A symbol of segment i < r-1 has the code
// 1^i 0 (e[i] low bits of s) and length i + 1 + e[i]; a symbol of the last
// segment has 1^(r-1) (e[r-1] low bits) and length r - 1 + e[r-1].  For sigma
// a power of two (r = 1) this is the identity code of length L = lg sigma.
// Segment i of a symbol s is found from the highest bit where s and sigma
// differ (sigma has a one there and s a zero).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wt.h"

namespace wt {

constexpr uint32_t kL1Bits = WT_L1_BITS;  // Section 4.1
constexpr uint32_t kL2Bits = WT_L2_BITS;  // Section 6: |L2| = 512
constexpr uint32_t kMaxLevels = WT_MAX_LEVELS;
constexpr uint32_t kMaxSigmaLog = 26;

// sticky device status bits (one per wt_status value)
constexpr uint32_t kStSymbol = 1u << WT_ESYMBOL;
constexpr uint32_t kStQuery = 1u << WT_EQUERY;
constexpr uint32_t kStTimeout = 1u << WT_ETIMEOUT;

// iteration cap of every device-side spin wait
constexpr uint32_t kSpinCap = 1u << 22;

struct CodeParams {
    uint32_t sigma;
    uint32_t L;     // ceil(lg sigma)
    uint32_t r;     // popcount(sigma); 1 for a power of two
    uint32_t pow2;  // sigma is a power of two (identity codes)
    uint32_t e[32]; // exponents of sigma's set bits, descending; e[0] = L for a power of two
    uint64_t P[33]; // P[i] = sum_{k < i} 2^e[k]
};

__host__ __device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

__host__ __device__ inline uint32_t clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __clz(x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}
__host__ __device__ inline uint32_t popc32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __popc(x);
#else
    return __builtin_popcount(x);
#endif
}
__host__ __device__ inline uint32_t popc64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return __popcll(x);
#else
    return __builtin_popcountll(x);
#endif
}

inline CodeParams make_code_params(uint32_t sigma) {
    CodeParams cp = {};
    cp.sigma = sigma;
    uint32_t L = 0;
    while ((1ull << L) < sigma) L++;
    cp.L = L;
    cp.pow2 = (sigma & (sigma - 1)) == 0;
    if (cp.pow2) {
        cp.r = 1;
        cp.e[0] = L;
    } else {
        uint32_t r = 0;
        for (int b = 31; b >= 0; b--)
            if (sigma >> b & 1u) cp.e[r++] = (uint32_t)b;
        cp.r = r;
    }
    cp.P[0] = 0;
    for (uint32_t i = 0; i < cp.r; i++) cp.P[i + 1] = cp.P[i] + (1ull << cp.e[i]);
    return cp;
}

// Code of symbol s (s < sigma), left-aligned in L bits, and its length.
__host__ __device__ inline void encode(const CodeParams& cp, uint32_t s, uint32_t& code, uint32_t& len) {
    if (cp.pow2) {
        code = s;
        len = cp.L;
        return;
    }
    uint32_t d = s ^ cp.sigma;
    uint32_t e = 31u - clz32(d);                   // segment exponent
    uint32_t j = popc32((uint32_t)((uint64_t)cp.sigma >> (e + 1)));  // segment index
    uint32_t low = s & ((1u << e) - 1u);
    uint64_t str;
    if (cp.sigma & ((1u << e) - 1u)) {  // not the last segment: 1^j 0 low
        str = ((((uint64_t)1 << j) - 1) << (e + 1)) | low;
        len = j + 1 + e;
    } else {  // last segment: 1^(r-1) low
        str = ((((uint64_t)1 << j) - 1) << e) | low;
        len = j + e;
    }
    code = (uint32_t)(str << (cp.L - len));
}

// Node at depth l with code prefix p (l bits): first symbol a and width
// (number of symbols below it).  Returns width 0 if no node of the
// (reduced) tree has this prefix.  A width of 1 is a leaf.
__host__ __device__ inline uint64_t node_info(const CodeParams& cp, uint32_t l, uint64_t p, uint64_t& a) {
    uint32_t r = cp.r;
    uint32_t j = 0;  // leading ones of p as an l-bit string
    if (l > 0) {
        uint64_t x = ~(p << (64 - l));
#ifdef __CUDA_ARCH__
        j = (uint32_t)__clzll((long long)x);
#else
        j = x ? (uint32_t)__builtin_clzll(x) : 64u;
#endif
        if (j > l) j = l;
    }
    if (j + 1 >= r) {  // inside the last segment's complete subtree (always for a power of two)
        uint32_t t = l - (r - 1);
        uint32_t er = cp.e[r - 1];
        if (t > er) return 0;
        uint64_t low = p & ((1ull << t) - 1);
        a = cp.P[r - 1] + (low << (er - t));
        return 1ull << (er - t);
    }
    if (j == l) {  // on the right spine above the last segment: [P[l], sigma)
        a = cp.P[l];
        return (uint64_t)cp.sigma - cp.P[l];
    }
    uint32_t t = l - j - 1;  // free bits inside segment j
    uint32_t ek = cp.e[j];
    if (t > ek) return 0;
    uint64_t low = p & ((1ull << t) - 1);
    a = cp.P[j] + (low << (ek - t));
    return 1ull << (ek - t);
}

// Split point of an internal node [a, a+width): a + prevPow2(width).
__host__ __device__ inline uint64_t node_mid(uint64_t a, uint64_t width) {
    uint64_t p = 1;
#ifdef __CUDA_ARCH__
    p = 1ull << (63 - __clzll((long long)(width - 1)));
#else
    while (p * 2 < width) p *= 2;
#endif
    return a + p;
}

// Per-node entry, heap-indexed: slot 2^l - 1 + p for depth l, prefix p.
struct NodeEntry {
    uint64_t start;  // C[a]: first position of the node in level l
    uint64_t r0;     // rank_0(l, start): precomputed node-start rank (Section 5.2.1)
    uint64_t off0;   // start - r0: next-level position of a zero = off0 + rank_0(pos)
    uint64_t off1;   // C[mid] - start + r0: next-level position of a one = off1 + rank_1(pos)
};

struct LevelDesc {
    const uint64_t* words;  // bits, LSB-first, 128-byte aligned
    const uint64_t* l1;     // floor(size/65536) + 1 entries
    const uint16_t* l2;     // floor(size/512) + 1 entries
    const uint64_t* s0;     // floor(zeros/K) + 1 entries, s0[0] = 0
    const uint64_t* s1;     // floor(ones/K) + 1 entries, s1[0] = 0
    uint64_t size;
    uint64_t ones;
    uint32_t* status;  // where a debug build reports a failed bounds check (may be null)
};

// Everything a query kernel needs, passed by value as a __grid_constant__.
struct TreeDesc {
    CodeParams cp;
    uint64_t n;
    uint32_t k_log2;  // select sample interval K = 2^k_log2
    uint32_t layout;  // 0: level-wise tree; 1: wavelet matrix (zeros of level l = lv[l].size - lv[l].ones)
    const NodeEntry* nodes;
    const uint64_t* C;  // sigma + 1
    uint32_t* status;
    LevelDesc lv[kMaxLevels];
};

// Arguments of one level pass over one tree (see wt_build.cu).
struct LevelPassArgs {
    const void* src;   // T_l
    void* dst;         // T_{l+1}, or null at the last level
    uint64_t size;     // size_l
    uint64_t size_next;
    uint64_t ntiles;
    uint64_t words_alloc;
    uint64_t* words;
    uint64_t* l1;
    uint16_t* l2;
    uint64_t* s0;
    uint64_t* s1;
    uint64_t n_s0, n_s1;     // allocated sample entries (writes beyond are dropped)
    const NodeEntry* nodes;  // level-l slice of the node table
    uint64_t* state;         // ntiles look-back words, zeroed (used when tile_excl is null)
    const uint64_t* tile_excl;           // ones of T_l before each tile (ntiles + 1), or null: look-back
    unsigned long long* next_cnt;        // ones of T_{l+1} per tile of T_{l+1}, zeroed; or null
    uint64_t* words2;  // level l+1's words (zeroed) when this pass also writes level l+1's bits
                       // (the level before the last; dst is then null), else null
    uint32_t* counter;       // tile counter, zeroed
    uint32_t* status;
    uint32_t level;
    uint32_t shift_bit;  // L - 1 - l
    uint32_t pshift;     // L - l (prefix = code >> pshift), unused at level 0
    uint32_t k_log2;
    uint64_t level_nodes;  // entries of the level's node-table slice: every element's code prefix is below it
    uint32_t ctab_n;     // level 0 re-encoding: table size (0 = compute codes arithmetically)
    uint32_t swar_codes; // level 0, bytes: codes by per-segment SWAR arithmetic (sigma <= 128, <= 3 segments)
    CodeParams cp;       // used when re-encoding at level 0
};

// Learned select (wt_train_select).  Per level and bit value b the b-bits'
// ranks are cut into anchor segments of kAnchor select samples (kAnchor K
// ranks); segment m runs between the anchors S_b[kAnchor m] and
// S_b[kAnchor (m+1)] (the build's samples, not stored again).  Each segment
// has one 8-byte record: three knot residuals (int16, in units of 2^rsh bits)
// of the fitted piecewise-linear model and the segment's error bound (uint16,
// in units of 2^esh bits): the k-th b-bit lies within the bound of the
// model's prediction for k.
constexpr uint32_t kMlpHidden = 32;
constexpr uint32_t kMlpParams = 3 * kMlpHidden + 1;  // w1[32], b1[32], w2[32], b2
constexpr uint32_t kLearnNone = 0, kLearnPla = 1, kLearnMlp = 2;
constexpr uint32_t kAnchorLog2 = 2;  // kAnchor = 4 samples per anchor segment
constexpr uint32_t kKnots = 3;       // interior knots per anchor segment

struct LearnedDesc {
    uint32_t mode;                       // kLearnNone / kLearnPla (fitted knots) / kLearnMlp
    uint32_t pad;
    const ushort4* rec[kMaxLevels][2];   // (count_b >> (k_log2 + kAnchorLog2)) + 1 records: r1, r2, r3, eps
    uint8_t rsh[kMaxLevels][2];          // residual unit 2^rsh bits
    uint8_t esh[kMaxLevels][2];          // bound unit 2^esh bits
    const float* mlp;                    // [level][b][kMlpParams], mode kLearnMlp only
    unsigned long long* fallbacks;       // queries whose window check failed (answered by sampled select)
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

__device__ __forceinline__ ulonglong2 ldg_nc_v2(const uint64_t* p) {
    ulonglong2 v;
    asm("ld.global.nc.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p));
    return v;
}

// 32 bytes (one sector) in one request; p 32-byte aligned
__device__ __forceinline__ void ldg_nc_v4(const uint64_t* p, uint64_t& a, uint64_t& b, uint64_t& c, uint64_t& d) {
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
}

// Debug builds (compiled with WT_DEBUG_BOUNDS=1: libwt_debug.so) check the
// index of every load a query walk makes against the array's length above
// (words: the 512-bit blocks up to the one holding position size, plus the
// node table's 2^L - 1 slots); a failed check sets WT_EBOUNDS in the status
// word and the load is skipped (its value is taken as 0).  Release builds
// compile the checks out.
#ifndef WT_DEBUG_BOUNDS
#define WT_DEBUG_BOUNDS 0
#endif
constexpr uint32_t kStBounds = 1u << WT_EBOUNDS;

__device__ __forceinline__ bool dbg_in(bool in_range, uint32_t* status) {
#if WT_DEBUG_BOUNDS
    if (!in_range) {
        if (status) atomicOr(status, kStBounds);
        return false;
    }
#endif
    return true;
}
__device__ __forceinline__ uint64_t lv_nl1(const LevelDesc& lv) { return (lv.size >> 16) + 1; }
__device__ __forceinline__ uint64_t lv_nl2(const LevelDesc& lv) { return (lv.size >> 9) + 1; }
__device__ __forceinline__ uint64_t lv_nwords(const LevelDesc& lv) { return ((lv.size >> 9) + 1) * 8; }
__device__ __forceinline__ uint64_t lv_nsamples(const LevelDesc& lv, uint32_t b, uint32_t k_log2) {
    return ((b ? lv.ones : lv.size - lv.ones) >> k_log2) + 1;
}
// checked loads: words[i .. i + 3] as one 32-byte load, and one element
__device__ __forceinline__ void ld_words4(const LevelDesc& lv, uint64_t i, uint64_t& a, uint64_t& b, uint64_t& c,
                                          uint64_t& d) {
    if (dbg_in(i + 3 < lv_nwords(lv), lv.status)) ldg_nc_v4(lv.words + i, a, b, c, d);
    else a = b = c = d = 0;
}
template <typename T>
__device__ __forceinline__ T ld_chk(const T* p, uint64_t i, uint64_t n, uint32_t* status) {
    return dbg_in(i < n, status) ? __ldg(p + i) : T(0);
}

// Binary rank_1 (Algorithm 1 with 64-bit words): ones in B_l[0, pos), and the
// bit at pos (needed by access, returned with the rank as in Section 5.2.1).
// Reads the L1 and L2 counters and the words of pos's 512-bit block up to pos;
// counts the half holding pos by three popcounts and a select, the other half
// (if before pos) by four.
__device__ __forceinline__ uint64_t rank1_bit(const LevelDesc& lv, uint64_t pos, uint32_t& bit) {
    const uint64_t blk = pos >> 9;
    const uint32_t wi = (uint32_t)(pos >> 6) & 7u;
    const uint32_t bi = (uint32_t)pos & 63u;
    const bool second = wi >= 4;  // pos lies in the block's second 32-byte half
    uint64_t a0, a1, a2, a3, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
    ld_words4(lv, blk << 3, a0, a1, a2, a3);  // 64-byte aligned block
    if (second) ld_words4(lv, (blk << 3) + 4, b0, b1, b2, b3);
    const uint64_t r = ld_chk(lv.l1, pos >> 16, lv_nl1(lv), lv.status) + (uint64_t)ld_chk(lv.l2, blk, lv_nl2(lv), lv.status);
    // ones of the first half if pos is past it, then the full words of pos's
    // half before pos's word, then pos's word below bit bi
    const uint32_t first = second ? __popcll(a0) + __popcll(a1) + __popcll(a2) + __popcll(a3) : 0u;
    const uint64_t x0 = second ? b0 : a0, x1 = second ? b1 : a1, x2 = second ? b2 : a2, x3 = second ? b3 : a3;
    const uint32_t q = wi & 3u;
    const uint32_t before = (q > 0 ? (uint32_t)__popcll(x0) : 0u) + (q > 1 ? (uint32_t)__popcll(x1) : 0u) +
                            (q > 2 ? (uint32_t)__popcll(x2) : 0u);
    const uint64_t xq = q == 0 ? x0 : (q == 1 ? x1 : (q == 2 ? x2 : x3));
    bit = (uint32_t)(xq >> bi) & 1u;
    return r + first + before + (uint32_t)__popcll(xq & ((1ull << bi) - 1ull));
}

// rank_1 alone (rank walks, bitvector rank): one masked popcount per word of
// the block, which measured faster than rank1_bit's form when the bit is not
// needed (text rank walk 0.61 against 0.68 ms per 10^7); access, which needs
// the bit, is faster with rank1_bit's (0.70 -> 0.53 ms)
__device__ __forceinline__ uint64_t rank1(const LevelDesc& lv, uint64_t pos) {
    const uint64_t blk = pos >> 9;
    const uint32_t wi = (uint32_t)(pos >> 6) & 7u;
    const uint32_t bi = (uint32_t)pos & 63u;
    uint64_t w[8];
    ld_words4(lv, blk << 3, w[0], w[1], w[2], w[3]);  // 64-byte aligned block
    w[4] = w[5] = w[6] = w[7] = 0;
    if (wi >= 4) ld_words4(lv, (blk << 3) + 4, w[4], w[5], w[6], w[7]);
    const uint64_t r = ld_chk(lv.l1, pos >> 16, lv_nl1(lv), lv.status) + (uint64_t)ld_chk(lv.l2, blk, lv_nl2(lv), lv.status);
    uint32_t c = 0;
#pragma unroll
    for (uint32_t k = 0; k < 8; k++) {
        const uint64_t m = k < wi ? ~0ull : (k == wi ? ((1ull << bi) - 1ull) : 0ull);
        c += __popcll(w[k] & m);
    }
    return r + c;
}

__device__ __forceinline__ uint32_t bit_at(const LevelDesc& lv, uint64_t pos) {
    return (uint32_t)(ld_chk(lv.words, pos >> 6, lv_nwords(lv), lv.status) >> (pos & 63)) & 1u;
}

// Position (0..63) of the k-th (1-based) set bit of x; popc(x) >= k.  Binary
// halving with popcounts, six steps for a 64-bit word (Section 5.4.1).
__device__ __forceinline__ uint32_t select_in_word(uint64_t x, uint32_t k) {
    uint32_t pos = 0;
#pragma unroll
    for (uint32_t wdt = 32; wdt >= 1; wdt >>= 1) {
        uint32_t c = __popcll(x & ((1ull << wdt) - 1ull));
        if (k > c) {
            k -= c;
            x >>= wdt;
            pos += wdt;
        }
    }
    return pos;
}

// Position (0..63) of the k-th (1-based) set bit of x, popc(x) >= k: one split
// of the word into 32-bit halves, then binary halving with 32-bit popcounts.
__device__ __forceinline__ uint32_t select_in_word32(uint64_t x, uint32_t k) {
    uint32_t w = (uint32_t)x;
    const uint32_t pl = __popc(w);
    uint32_t pos = 0;
    if (k > pl) {
        k -= pl;
        w = (uint32_t)(x >> 32);
        pos = 32;
    }
#pragma unroll
    for (uint32_t wdt = 16; wdt >= 1; wdt >>= 1) {
        const uint32_t c = __popc(w & ((1u << wdt) - 1u));
        if (k > c) {
            k -= c;
            w >>= wdt;
            pos += wdt;
        }
    }
    return pos;
}

// Binary select (Algorithm 2): the position of the k-th (1-based) bit equal to
// b in level lv, 1 <= k <= count_b.  The listing is read this way: the sample
// index is floor(k / K), samples[0] = 0 and samples[m] is the position of the
// (m K)-th b-bit; the first L1 block is the floor (not the ceiling) of the
// sample position over 65536; the L2 search stays inside the enclosing L1
// block and below the next sample; the predicate of both searches is "fewer
// than k b-bits before the block"; the word loop starts at the chosen L2
// block's absolute position.
//
// The search runs in stages over a SelB state so that a thread can walk
// several queries in lockstep (their loads of one stage in flight together):
//   selb_range    the two samples around k (or a caller's window) -> position range
//   selb_l1       the L1 block: one load, a scan only if the range crosses an
//                 L1 boundary; the L2 entry at the range start is loaded with it
//   selb_step     one step of the binary search over the L2 entries of the
//                 range, relative to the L1 block (while lo < hi)
//   selb_words    the first 32-byte half of the chosen 512-bit block
//   selb_half     the second half instead, if the bit lies beyond the first
//   selb_finish   word and bit inside the half (select_in_word32)
// Inside an L1 block every quantity fits 32 bits.  The first L2 probe does not
// wait for the L1 counter: the predicate compares with kk = k - (b-bits before
// the L1 block) only after the probe is issued.
// Level-wise trees of at least this many levels walk their selects two
// queries per thread (do_select_n<2>), shallower ones one per thread.
constexpr uint32_t kPairLevels = 8;

struct SelB {
    uint64_t k;               // rank sought (1-based) among the b-bits
    uint64_t lo_pos, hi_pos;  // position range that holds the k-th b-bit
    uint64_t i1, c1;          // L1 block and its counter
    const uint16_t* L2;       // L2 counters of block i1
    uint64_t w0, w1, w2, w3;  // one 32-byte half of the chosen 512-bit block
    uint32_t b, lo, hi;       // bit value; L2 range [lo, hi] inside block i1
    uint32_t kk, c2lo, kw;    // rank inside block i1; L2 counter at lo; rank inside the half
    uint32_t half;            // 0 or 4: which half
    bool ok;                  // the counters agree that the bit is in the range
#if WT_DEBUG_BOUNDS
    uint64_t dbg_nl2;         // L2 entries from block i1's first one to the end
    uint32_t* dbg_status;
#endif
};


// samples S_b[m], S_b[m + 1] around k (m = floor(k / K)); past the last sample
// the range ends at the level's last bit.  on = false leaves a state that the
// later stages walk on position 0 without effect.
__device__ __forceinline__ void selb_range(SelB& s, const LevelDesc& lv, uint32_t b, uint64_t k, uint32_t k_log2,
                                           bool on) {
    const uint64_t* S = b ? lv.s1 : lv.s0;
    const uint64_t total = b ? lv.ones : lv.size - lv.ones;
    const uint64_t m = k >> k_log2;
    s.b = b;
    s.k = k;
    s.ok = true;
    const uint64_t ns = lv_nsamples(lv, b, k_log2);
    s.lo_pos = on ? ld_chk(S, m, ns, lv.status) : 0ull;
    s.hi_pos = on ? ((((m + 1) << k_log2) <= total) ? ld_chk(S, m + 1, ns, lv.status) : lv.size - 1) : 0ull;
}

// a caller's window [lo, hi] instead of the samples (lo <= hi <= size - 1);
// the stages then also check that the k-th b-bit lies inside it (s.ok)
__device__ __forceinline__ void selb_window(SelB& s, uint32_t b, uint64_t k, uint64_t lo, uint64_t hi) {
    s.b = b;
    s.k = k;
    s.ok = true;
    s.lo_pos = lo;
    s.hi_pos = hi;
}

// Precondition: lo_pos <= hi_pos <= size - 1.
__device__ __forceinline__ void selb_l1(SelB& s, const LevelDesc& lv) {
    const uint64_t hi1 = s.hi_pos >> 16;
    s.i1 = s.lo_pos >> 16;
    s.c1 = ld_chk(lv.l1, s.i1, lv_nl1(lv), lv.status);
    s.lo = (uint32_t)(s.lo_pos >> 9) & 127u;
    s.hi = (s.i1 == hi1) ? ((uint32_t)(s.hi_pos >> 9) & 127u) : 127u;
    while (s.i1 < hi1) {  // last L1 block of the range with fewer than k b-bits before it
        const uint64_t c1n = ld_chk(lv.l1, s.i1 + 1, lv_nl1(lv), lv.status);
        if ((s.b ? c1n : ((s.i1 + 1) << 16) - c1n) >= s.k) break;
        s.i1++;
        s.c1 = c1n;
        s.lo = 0;
        s.hi = (s.i1 == hi1) ? ((uint32_t)(s.hi_pos >> 9) & 127u) : 127u;
    }
    s.L2 = lv.l2 + (s.i1 << 7);
    s.c2lo = ld_chk(lv.l2, (s.i1 << 7) + s.lo, lv_nl2(lv), lv.status);
#if WT_DEBUG_BOUNDS
    s.dbg_nl2 = lv_nl2(lv) > (s.i1 << 7) ? lv_nl2(lv) - (s.i1 << 7) : 0;
    s.dbg_status = lv.status;
#endif
}

// b-bits of L1 block i1 before its L2 entry e (e relative to the block)
__device__ __forceinline__ uint32_t selb_l2count(const SelB& s, uint32_t e, uint32_t v) {
    return s.b ? v : (e << 9) - v;
}

// CHECK: a caller's window may miss the bit, so the stages keep s.ok; between
// the samples the bit is always there and the checks are left out.
template <bool CHECK>
__device__ __forceinline__ void selb_rank(SelB& s) {
    const uint64_t before = s.b ? s.c1 : (s.i1 << 16) - s.c1;
    if (CHECK) s.ok = before < s.k;
    s.kk = (uint32_t)(s.k - before);  // 1..65536 when the bit is in block i1
}

__device__ __forceinline__ void selb_step(SelB& s) {
    const uint32_t mid = (s.lo + s.hi + 1) >> 1;
#if WT_DEBUG_BOUNDS
    const uint32_t v = ld_chk(s.L2, mid, s.dbg_nl2, s.dbg_status);
#else
    const uint32_t v = __ldg(s.L2 + mid);
#endif
    if (selb_l2count(s, mid, v) < s.kk) {
        s.lo = mid;
        s.c2lo = v;
    } else {
        s.hi = mid - 1;
    }
}

// rank inside the chosen 512-bit block; its first 32-byte half
template <bool CHECK>
__device__ __forceinline__ void selb_words(SelB& s, const LevelDesc& lv) {
    const uint32_t before = selb_l2count(s, s.lo, s.c2lo);
    if (CHECK) s.ok = s.ok && before < s.kk;
    s.kw = s.kk - before;
    s.half = 0;
    ld_words4(lv, ((s.i1 << 7) + s.lo) << 3, s.w0, s.w1, s.w2, s.w3);
}

// the second half instead, if the bit lies beyond the first
__device__ __forceinline__ void selb_half(SelB& s, const LevelDesc& lv, bool on) {
    const uint64_t fl = s.b ? 0ull : ~0ull;
    const uint32_t h = __popcll(s.w0 ^ fl) + __popcll(s.w1 ^ fl) + __popcll(s.w2 ^ fl) + __popcll(s.w3 ^ fl);
    if (on && h < s.kw) {
        s.kw -= h;
        s.half = 4;
        ld_words4(lv, (((s.i1 << 7) + s.lo) << 3) + 4, s.w0, s.w1, s.w2, s.w3);
    }
}

template <bool CHECK>
__device__ __forceinline__ uint64_t selb_finish(SelB& s) {
    const uint64_t fl = s.b ? 0ull : ~0ull;
    const uint64_t a0 = s.w0 ^ fl, a1 = s.w1 ^ fl, a2 = s.w2 ^ fl, a3 = s.w3 ^ fl;
    const uint32_t p0 = __popcll(a0), p1 = __popcll(a1), p2 = __popcll(a2);
    uint64_t wv = a3;
    uint32_t wj = 3, kw = s.kw;
    if (p0 >= kw) {
        wv = a0;
        wj = 0;
    } else if (p0 + p1 >= kw) {
        wv = a1;
        wj = 1;
        kw -= p0;
    } else if (p0 + p1 + p2 >= kw) {
        wv = a2;
        wj = 2;
        kw -= p0 + p1;
    } else {
        kw -= p0 + p1 + p2;
        if (CHECK) s.ok = s.ok && kw <= (uint32_t)__popcll(a3);
    }
    return ((((s.i1 << 7) + s.lo) << 9) + ((uint64_t)(s.half + wj) << 6)) + select_in_word32(wv, kw);
}

// Searches stay inside the level's arrays: lo <= hi always, hi is at most the
// L2 entry of the range's last position, and a range that crosses an L1
// boundary makes block i1 a full one.
__device__ __forceinline__ uint64_t select_b(const LevelDesc& lv, uint32_t b, uint64_t k, uint32_t k_log2) {
    SelB s;
    selb_range(s, lv, b, k, k_log2, true);
    selb_l1(s, lv);
    selb_rank<false>(s);
    while (s.lo < s.hi) selb_step(s);
    selb_words<false>(s, lv);
    selb_half(s, lv, true);
    return selb_finish<false>(s);
}

__device__ __forceinline__ void set_status(uint32_t* st, uint32_t bits) { atomicOr(st, bits); }

#endif  // __CUDACC__

}  // namespace wt
