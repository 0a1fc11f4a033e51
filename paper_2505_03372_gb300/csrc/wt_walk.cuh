// Level walks of the queries (Sections 5.2-5.4, Algorithms 5-8), shared by the
// single-tree and the batched query kernels.  One thread walks one query.
#pragma once

#include "wt_common.cuh"

namespace wt {

// {start, r0} of the first `slots` node-table slots, copied into shared memory
// by the query kernels (the top levels of the tree: every walk passes them)
struct NodeCache {
    const ulonglong2* s;
    uint32_t slots;
};

__device__ __forceinline__ ulonglong2 node_sr(const TreeDesc& t, const NodeCache& nc, uint32_t l, uint64_t p) {
    // {start, r0} of node (l, p); slots are 32-byte aligned
    const uint64_t slot = (1ull << l) - 1 + p;
    if (slot < nc.slots) return nc.s[slot];
    if (!dbg_in(slot < (1ull << t.cp.L) - 1, t.status)) return make_ulonglong2(0, 0);
    return ldg_nc_v2(reinterpret_cast<const uint64_t*>(t.nodes + slot));
}

// Algorithm 5 with the early stop at nodes of at most two symbols.
__device__ __forceinline__ uint32_t do_access(const TreeDesc& t, const NodeCache& nc, uint64_t i) {
    const CodeParams& cp = t.cp;
    if (cp.L == 0) return 0;
    uint64_t p = 0;
    for (uint32_t l = 0; l < cp.L; l++) {
        uint64_t a, width;
        if (cp.pow2) {
            width = 1ull << (cp.L - l);
            a = p << (cp.L - l);
        } else {
            width = node_info(cp, l, p, a);
        }
        if (width == 1) return (uint32_t)a;
        const ulonglong2 ne = node_sr(t, nc, l, p);
        const uint64_t pos = ne.x + i;
        if (width == 2) return (uint32_t)(a + bit_at(t.lv[l], pos));
        uint32_t b;
        const uint64_t r1 = rank1_bit(t.lv[l], pos, b);
        const uint64_t zb = (pos - r1) - ne.y;  // zeros of the node before i
        i = b ? i - zb : zb;
        p = 2 * p + b;
    }
    return UINT32_MAX;  // not reached: every root-to-leaf path ends at a leaf
}

// Algorithm 6: the code of c gives the direction at every level.
__device__ __forceinline__ uint64_t do_rank(const TreeDesc& t, const NodeCache& nc, uint32_t c, uint64_t i) {
    const CodeParams& cp = t.cp;
    uint32_t code, len;
    encode(cp, c, code, len);
    ulonglong2 ne = node_sr(t, nc, 0, 0);
    for (uint32_t l = 0; l < len; l++) {
        if (i == 0) return 0;
        const uint32_t b = (code >> (cp.L - 1 - l)) & 1u;
        const uint64_t pos = ne.x + i;
        const uint64_t r0n = ne.y;
        if (l + 1 < len) ne = node_sr(t, nc, l + 1, code >> (cp.L - 1 - l));  // next node, issued early
        const uint64_t r1 = rank1(t.lv[l], pos);
        const uint64_t zb = (pos - r1) - r0n;
        i = b ? i - zb : zb;
    }
    return i;
}

// Algorithms 7 and 8: leaf to root; the node of c at level l is the prefix of
// its code, so getNodeStart becomes a table index.  NQ queries walk in
// lockstep, one level at a time from the longest code down: at every stage of
// the binary select (wt_common.cuh, SelB) the loads of all NQ queries are
// issued before any is used, so one thread keeps NQ dependent chains in
// flight.  A query joins at its own leaf level (levels above its code length
// are skipped); act[q] = false walks nothing.
template <int NQ>
__device__ __forceinline__ void do_select_n(const TreeDesc& t, const NodeCache& nc, const uint32_t (&c)[NQ],
                                            const uint64_t (&jin)[NQ], const bool (&act)[NQ], uint64_t (&res)[NQ]) {
    const CodeParams& cp = t.cp;
    uint32_t code[NQ], len[NQ];
    uint64_t j[NQ];
    ulonglong2 ne[NQ];
    int lmax = -1;
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        code[q] = 0;
        len[q] = 0;
        if (act[q]) encode(cp, c[q], code[q], len[q]);
        j[q] = jin[q];
        lmax = max(lmax, (int)len[q] - 1);
        ne[q] = make_ulonglong2(0, 0);
        if (len[q]) ne[q] = node_sr(t, nc, len[q] - 1, (uint64_t)code[q] >> (cp.L - (len[q] - 1)));
    }
    for (int l = lmax; l >= 0; l--) {
        const LevelDesc& lv = t.lv[l];
        bool on[NQ];
        uint64_t start[NQ];
        SelB s[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            // a lone query walks from its own leaf level, so it is on every level of the loop
            on[q] = NQ == 1 || l < (int)len[q];
            const uint32_t b = (code[q] >> (cp.L - 1 - (uint32_t)l)) & 1u;
            start[q] = ne[q].x;
            const uint64_t kb = b ? (start[q] - ne[q].y) : ne[q].y;  // b-bits before the node
            if (on[q] && l > 0) ne[q] = node_sr(t, nc, (uint32_t)l - 1, (uint64_t)code[q] >> (cp.L - (uint32_t)l + 1));
            selb_range(s[q], lv, b, kb + j[q], t.k_log2, on[q]);
        }
#pragma unroll
        for (int q = 0; q < NQ; q++) selb_l1(s[q], lv);
#pragma unroll
        for (int q = 0; q < NQ; q++) selb_rank<false>(s[q]);
        bool more = true;
        while (more) {
            more = false;
#pragma unroll
            for (int q = 0; q < NQ; q++) {
                if (s[q].lo < s[q].hi) selb_step(s[q]);
                more = more || s[q].lo < s[q].hi;
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; q++) selb_words<false>(s[q], lv);
#pragma unroll
        for (int q = 0; q < NQ; q++) selb_half(s[q], lv, on[q]);
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const uint64_t pos = selb_finish<false>(s[q]);
            if (on[q]) j[q] = pos + 1 - start[q];
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; q++) res[q] = j[q] - 1;
}

__device__ __forceinline__ uint64_t do_select(const TreeDesc& t, const NodeCache& nc, uint32_t c, uint64_t j) {
    const uint32_t cc[1] = {c};
    const uint64_t jj[1] = {j};
    const bool act[1] = {true};
    uint64_t r[1];
    do_select_n<1>(t, nc, cc, jj, act, r);
    return r[0];
}

// ---------------------------------------------------------------------------
// Wavelet matrix (layout 1): plain L-bit codes; level l+1 holds level l's
// zeros first (in order) and its ones after them, so a position moves down by
// rank_0, or by Z_l + rank_1 (Z_l = zeros of level l), and up by select.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t do_access_m(const TreeDesc& t, uint64_t i) {
    uint32_t code = 0;
    for (uint32_t l = 0; l < t.cp.L; l++) {
        const LevelDesc& lv = t.lv[l];
        uint32_t b;
        const uint64_t r1 = rank1_bit(lv, i, b);
        code = (code << 1) | b;
        i = b ? (lv.size - lv.ones) + r1 : i - r1;
    }
    return code;
}

// rank_c(i): the range [s, e) of level-l positions above [0, i) of c's run
__device__ __forceinline__ uint64_t do_rank_m(const TreeDesc& t, uint32_t c, uint64_t i) {
    uint64_t s = 0, e = i;
    for (uint32_t l = 0; l < t.cp.L; l++) {
        const LevelDesc& lv = t.lv[l];
        const uint32_t b = (c >> (t.cp.L - 1 - l)) & 1u;
        const uint64_t r1s = rank1(lv, s), r1e = rank1(lv, e);
        if (b) {
            const uint64_t z = lv.size - lv.ones;
            s = z + r1s;
            e = z + r1e;
        } else {
            s -= r1s;
            e -= r1e;
        }
    }
    return e - s;
}

// select_c(j): down to the start of c's run below the last level, then up
__device__ __forceinline__ uint64_t do_select_m(const TreeDesc& t, uint32_t c, uint64_t j) {
    const uint32_t L = t.cp.L;
    uint64_t s = 0;
    for (uint32_t l = 0; l < L; l++) {
        const LevelDesc& lv = t.lv[l];
        const uint32_t b = (c >> (L - 1 - l)) & 1u;
        const uint64_t r1 = rank1(lv, s);
        s = b ? (lv.size - lv.ones) + r1 : s - r1;
    }
    uint64_t p = s + j - 1;
    for (int l = (int)L - 1; l >= 0; l--) {
        const LevelDesc& lv = t.lv[l];
        const uint32_t b = (c >> (L - 1 - (uint32_t)l)) & 1u;
        p = b ? select_b(lv, 1, p - (lv.size - lv.ones) + 1, t.k_log2) : select_b(lv, 0, p + 1, t.k_log2);
    }
    return p;
}

// Copy the first `slots` {start, r0} pairs of the node table into shared memory
// (every thread of the CTA calls this; it ends with a barrier).
__device__ __forceinline__ NodeCache load_node_cache(const TreeDesc& t, ulonglong2* s, uint32_t slots) {
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x)
        s[i] = ldg_nc_v2(reinterpret_cast<const uint64_t*>(t.nodes + i));
    __syncthreads();
    NodeCache nc;
    nc.s = s;
    nc.slots = slots;
    return nc;
}

__device__ __forceinline__ bool select_valid(const TreeDesc& t, uint32_t c, uint64_t j) {
    if (c >= t.cp.sigma || j == 0) return false;
    return j <= __ldg(t.C + c + 1) - __ldg(t.C + c);
}

__device__ __forceinline__ void flag_query_error(const TreeDesc& t, bool bad) {
    if (__any_sync(__activemask(), bad)) {
        if (bad) atomicOr(t.status, kStQuery);
    }
}

}  // namespace wt
