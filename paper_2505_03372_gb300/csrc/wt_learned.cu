// Learned select: a model per (level, bit value b) predicts where the k-th
// b-bit of a level lies, a stored per-segment bound makes the prediction
// exact, and the sampled select of Algorithm 2 is the fallback.
//
// Anchor segments.  The build stores, per level and b, the position S_b[m] of
// the (m K)-th b-bit (Section 4.2).  Every kAnchor-th of those pairs is an
// anchor: anchor segment m holds the ranks k with floor(k / (kAnchor K)) = m
// and runs from (k0, x0) = (m kAnchor K, S_b[kAnchor m]) to (k1, x1) =
// ((m+1) kAnchor K, S_b[kAnchor (m+1)]), the last one to the virtual
// (count_b + 1)-th b-bit at position size_l.  Nothing of the anchors is stored
// again; each segment owns one 8-byte record.
//
// Models.  PLA (fitted knots): knot t = 0..4 sits at rank kappa_t = k0 +
// floor(t (k1 - k0) / 4) and position x0 + floor(t (x1 - x0) / 4) + R_t, the
// residuals R_1..3 fitted on the GPU by least squares to the positions of the
// segment's b-bits (the hat-function basis gives a 3x3 system per segment; R_0
// = R_4 = 0); a rank k is predicted by interpolating between the two knots
// (ka, xa), (kb, xb) around it, xa + floor((k - ka) (xb - xa) / (kb - ka)),
// exact in integers (a shift in every full segment).  Untrained (R = 0) it is
// the line through the anchors.  MLP: the fraction u = (k - k0) / (k1 - k0) is
// mapped to u + g(u), g a 1 -> 32 -> 1 ReLU network in FP32 shared by all
// segments of a (level, b), trained with Adam on the GPU (g starts at 0, the
// line through the anchors).
//
// Bounds.  A scan over every bit of every level evaluates the model at every
// b-bit's rank and keeps the segment's largest |prediction - position|, stored
// rounded up to a unit of 2^esh bits.  The MLP's prediction is a fixed chain of
// correctly rounded operations (__fmaf_rn, __fmul_rn, __fdiv_rn), so the query
// recomputes exactly the value the bound was taken on.
//
// Query.  At each level the window [p - eps, p + eps] replaces the sample range
// of the sampled select: L1 scan, L2 binary search and word scan run inside
// it.  If the counters show that the k-th b-bit is not in the window (which an
// exact bound rules out) the level falls back to the sampled select and a
// counter records it.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "wt_internal.hpp"

namespace wt {

struct Seg {
    uint64_t k0, k1, x0, x1;
};

// anchor segment m of (level, b); kl = log2 K
__device__ __forceinline__ Seg anchor_seg(const LevelDesc& lv, uint32_t b, uint64_t m, uint32_t kl) {
    const uint64_t* S = b ? lv.s1 : lv.s0;
    const uint64_t total = b ? lv.ones : lv.size - lv.ones;
    const uint32_t ka = kl + kAnchorLog2;
    Seg g;
    g.k0 = m << ka;
    const uint64_t ns = lv_nsamples(lv, b, kl);
    g.x0 = ld_chk(S, m << kAnchorLog2, ns, lv.status);
    if (((m + 1) << ka) <= total) {
        g.k1 = (m + 1) << ka;
        g.x1 = ld_chk(S, (m + 1) << kAnchorLog2, ns, lv.status);
    } else {
        g.k1 = total + 1;
        g.x1 = lv.size;
    }
    return g;
}

__device__ __forceinline__ uint64_t knot_rank(const Seg& g, uint32_t t) { return g.k0 + ((t * (g.k1 - g.k0)) >> 2); }

// untrained knot position t: t quarters of the way from x0 to x1
__device__ __forceinline__ uint64_t knot_base(const Seg& g, uint32_t t) { return g.x0 + ((t * (g.x1 - g.x0)) >> 2); }

// xa + floor((k - ka) (xb - xa) / (kb - ka)) for ka <= k < kb, exact in 64-bit
// integers ((k - ka) < 2^14 and xb - xa < 2^48).  Knots of a full segment are
// K = 2^kl ranks apart, so the division is a shift there; only the last
// segment of a (level, b) divides.
__device__ __forceinline__ uint64_t interp(uint64_t ka, uint64_t kb, uint64_t xa, uint64_t xb, uint64_t k,
                                           uint32_t kl) {
    const uint64_t d = kb - ka, prod = (k - ka) * (xb - xa);
    return xa + (d == (1ull << kl) ? (prod >> kl) : prod / d);
}

// Residual of knot t = 1..3 of a record, in bits.
__device__ __forceinline__ int64_t resid(const ushort4 r, uint32_t rsh, uint32_t t) {
    const uint16_t v = t == 1 ? r.x : (t == 2 ? r.y : r.z);
    return (int64_t)(int16_t)v * (int64_t(1) << rsh);
}

// Fitted-knot prediction for rank k of segment g, record rec (residuals in
// units of 2^rsh bits for knots t = 1..3).  Only the residuals of the two
// knots around k are unpacked.
// Knot positions are non-decreasing and inside [x0, x1] (the fit guarantees it).
// The knots are quarters of the segment; the interpolation between the two
// knots around k is exact integer arithmetic.
__device__ __forceinline__ uint64_t predict_knots(const Seg& g, const ushort4 rec, uint32_t rsh, uint64_t k,
                                                  uint32_t kl) {
    if (g.k1 - g.k0 == (4ull << kl)) {
        // a full segment (all but the last of a level and b): knots K ranks
        // apart, so t = (k - k0) / K and the interpolation divides by K; the
        // same integers as the general form below, with shifts for divisions
        const uint32_t off = (uint32_t)(k - g.k0);
        const uint32_t t = off >> kl;
        const uint64_t span = g.x1 - g.x0;
        const uint64_t xa = t == 0 ? g.x0 : (uint64_t)((int64_t)(g.x0 + ((t * span) >> 2)) + resid(rec, rsh, t));
        const uint64_t xb = t == 3 ? g.x1 : (uint64_t)((int64_t)(g.x0 + (((t + 1) * span) >> 2)) + resid(rec, rsh, t + 1));
        const uint64_t dx = xb - xa;
        const uint32_t dk = off & ((1u << kl) - 1u);  // k - ka < K
        const uint64_t prod = dx < (1ull << 32) ? (uint64_t)dk * (uint32_t)dx : (uint64_t)dk * dx;
        return xa + (prod >> kl);
    }
    if (g.k1 - g.k0 < 4) return interp(g.k0, g.k1, g.x0, g.x1, k, kl);
    const uint64_t k1r = knot_rank(g, 1), k2r = knot_rank(g, 2), k3r = knot_rank(g, 3);
    const uint32_t t = (k >= k1r) + (k >= k2r) + (k >= k3r);
    const uint64_t ka = t == 0 ? g.k0 : (t == 1 ? k1r : (t == 2 ? k2r : k3r));
    const uint64_t kb = t == 0 ? k1r : (t == 1 ? k2r : (t == 2 ? k3r : g.k1));
    const uint64_t xa = t == 0 ? g.x0 : (uint64_t)((int64_t)knot_base(g, t) + resid(rec, rsh, t));
    const uint64_t xb = t == 3 ? g.x1 : (uint64_t)((int64_t)knot_base(g, t + 1) + resid(rec, rsh, t + 1));
    return interp(ka, kb, xa, xb, k, kl);
}

// g(u) = b2 + sum_j w2[j] * relu(w1[j] * u + b1[j]); P = {w1[32], b1[32], w2[32], b2}
__device__ __forceinline__ float mlp_g(const float* P, float u) {
    float y = P[3 * kMlpHidden];
#pragma unroll 8
    for (uint32_t j = 0; j < kMlpHidden; j++) {
        const float a = __fmaf_rn(P[j], u, P[kMlpHidden + j]);
        y = __fmaf_rn(P[2 * kMlpHidden + j], fmaxf(a, 0.f), y);
    }
    return y;
}

__device__ __forceinline__ uint64_t predict_mlp(const Seg& g, uint64_t k, const float* P) {
    const float u = __fdiv_rn((float)(k - g.k0), (float)(g.k1 - g.k0));
    float h = __fadd_rn(u, mlp_g(P, u));
    h = fminf(fmaxf(h, 0.f), 1.f);
    const uint64_t span = g.x1 - g.x0;
    uint64_t off = (uint64_t)__fmul_rn((float)span, h);
    return g.x0 + (off < span ? off : span);
}

__device__ __forceinline__ uint64_t predict(uint32_t mode, const Seg& g, const ushort4 rec, uint32_t rsh, uint64_t k,
                                            const float* P, uint32_t kl) {
    return mode == kLearnMlp ? predict_mlp(g, k, P) : predict_knots(g, rec, rsh, k, kl);
}

// ---------------------------------------------------------------------------
// fit: least-squares knot residuals, one warp per anchor segment
// ---------------------------------------------------------------------------

struct FitArgs {
    LevelDesc lv;
    uint32_t b, kl;
    uint64_t nseg;
    float* resid;             // [nseg][3], bits
    unsigned int* maxabs;     // float bits of the largest |residual| of the (level, b)
};

// The warp walks the segment's words 32 at a time; each lane enumerates the
// b-bits of its word with their ranks and accumulates the normal equations of
// the hat-function basis: knot t's function is 1 at kappa_t and falls
// linearly to 0 at the neighbouring knots, so a rank touches at most two.
__global__ void __launch_bounds__(256) fit_knots_kernel(const __grid_constant__ FitArgs a) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t m = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (m >= a.nseg) return;
    const LevelDesc& lv = a.lv;
    const Seg g = anchor_seg(lv, a.b, m, a.kl);
    const uint64_t span = g.k1 - g.k0;
    float* out = a.resid + 3 * m;
    if (span < 4 || g.x1 <= g.x0) {
        if (lane < 3) out[lane] = 0.f;
        return;
    }
    uint64_t kap[5];
#pragma unroll
    for (uint32_t t = 0; t < 5; t++) kap[t] = t == 4 ? g.k1 : knot_rank(g, t);
    // rank of the first b-bit at or after x0: k0 for m >= 1 (the anchor itself), 1 for m = 0
    uint64_t rank = m ? g.k0 : 1;
    float s00 = 0, s11 = 0, s22 = 0, s01 = 0, s12 = 0, y0 = 0, y1 = 0, y2 = 0;
    const uint64_t w0 = g.x0 >> 6, w1 = (g.x1 - 1) >> 6;
    for (uint64_t wb = w0; wb <= w1; wb += 32) {
        const uint64_t w = wb + lane;
        uint64_t x = 0;
        if (w <= w1) {
            x = __ldg(lv.words + w);
            if (!a.b) x = ~x;
            if (w == w0) x &= ~0ull << (g.x0 & 63);
            const uint64_t end = g.x1 < lv.size ? g.x1 : lv.size;  // positions in [x0, min(x1, size))
            if ((w << 6) + 64 > end) {
                const uint64_t keep = end > (w << 6) ? end - (w << 6) : 0;
                x &= keep >= 64 ? ~0ull : ((1ull << keep) - 1ull);
            }
        }
        const uint32_t c = __popcll(x);
        uint32_t inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= (uint32_t)o) inc += v;
        }
        uint64_t k = rank + (inc - c);
        rank += __shfl_sync(0xffffffffu, inc, 31);
        while (x) {
            const uint32_t i = __ffsll((long long)x) - 1;
            x &= x - 1;
            if (k >= g.k1) break;
            const uint64_t pos = (w << 6) + i;
            const uint32_t t = (k >= kap[1]) + (k >= kap[2]) + (k >= kap[3]);
            const float u = (float)(k - kap[t]) / (float)(kap[t + 1] - kap[t]);
            // distance of the position from the untrained model (the knots at quarters of the segment)
            const float xa = (float)(knot_base(g, t) - g.x0), xb = (float)(knot_base(g, t + 1) - g.x0);
            const float d = (float)(pos - g.x0) - (xa + u * (xb - xa));
            const float pa = 1.f - u, pb = u;  // weights of knots t and t + 1
            // knot indices 1..3 map to unknowns 0..2; knots 0 and 4 are the fixed anchors
            if (t == 0) {
                s00 += pb * pb;
                y0 += pb * d;
            } else if (t == 1) {
                s00 += pa * pa;
                s11 += pb * pb;
                s01 += pa * pb;
                y0 += pa * d;
                y1 += pb * d;
            } else if (t == 2) {
                s11 += pa * pa;
                s22 += pb * pb;
                s12 += pa * pb;
                y1 += pa * d;
                y2 += pb * d;
            } else {
                s22 += pa * pa;
                y2 += pa * d;
            }
            k++;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s00 += __shfl_xor_sync(0xffffffffu, s00, o);
        s11 += __shfl_xor_sync(0xffffffffu, s11, o);
        s22 += __shfl_xor_sync(0xffffffffu, s22, o);
        s01 += __shfl_xor_sync(0xffffffffu, s01, o);
        s12 += __shfl_xor_sync(0xffffffffu, s12, o);
        y0 += __shfl_xor_sync(0xffffffffu, y0, o);
        y1 += __shfl_xor_sync(0xffffffffu, y1, o);
        y2 += __shfl_xor_sync(0xffffffffu, y2, o);
    }
    if (lane == 0) {
        // tridiagonal 3x3 solve in FP64 (Thomas); an unknown without data stays 0
        double r[3] = {0, 0, 0};
        const double d0 = s00, d1 = s11, d2 = s22, e01 = s01, e12 = s12;
        const double det = d0 * (d1 * d2 - e12 * e12) - e01 * (e01 * d2);
        if (fabs(det) > 1e-9 * (fabs(d0 * d1 * d2) + 1e-30)) {  // Cramer's rule
            const double c0 = y0, c1 = y1, c2 = y2;
            r[0] = (c0 * (d1 * d2 - e12 * e12) - e01 * (c1 * d2 - e12 * c2)) / det;
            r[1] = (d0 * (c1 * d2 - e12 * c2) - c0 * e01 * d2) / det;
            r[2] = (d0 * (d1 * c2 - c1 * e12) - e01 * e01 * c2 + c0 * e01 * e12) / det;
        }
        float mx = 0.f;
        for (int t = 0; t < 3; t++) {
            const float v = isfinite(r[t]) ? (float)r[t] : 0.f;
            out[t] = v;
            mx = fmaxf(mx, fabsf(v));
        }
        atomicMax(a.maxabs, __float_as_uint(mx));
    }
}

__device__ __forceinline__ uint32_t shift_for(float maxv, float lim) {
    uint32_t sh = 0;
    while (sh < 30 && maxv > lim * (float)(1u << sh)) sh++;
    return sh;
}

// Residuals to int16 units of 2^rsh bits, with the knots kept non-decreasing
// and inside [x0, x1]; a segment where that fails keeps the line (R = 0).
__global__ void __launch_bounds__(256) quantize_knots_kernel(const __grid_constant__ FitArgs a, ushort4* rec,
                                                             const unsigned int* maxabs) {
    const uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= a.nseg) return;
    const uint32_t rsh = shift_for(__uint_as_float(*maxabs), 32767.f);
    const Seg g = anchor_seg(a.lv, a.b, m, a.kl);
    int32_t q[3] = {0, 0, 0};
    if (g.k1 - g.k0 >= 4) {
        int64_t prev = (int64_t)g.x0;
        bool ok = true;
        for (uint32_t t = 1; t <= 3; t++) {
            const int64_t base = (int64_t)knot_base(g, t);
            const float r = a.resid[3 * m + t - 1];
            int64_t v = (int64_t)llrintf(r / (float)(1u << rsh));
            v = v > 32767 ? 32767 : (v < -32767 ? -32767 : v);
            int64_t xi = base + v * (int64_t(1) << rsh);
            if (xi < prev) {  // raise to the previous knot, in whole units
                v = (prev - base + (int64_t(1) << rsh) - 1) >> rsh;
                xi = base + v * (int64_t(1) << rsh);
            }
            if (xi > (int64_t)g.x1) {
                v = ((int64_t)g.x1 - base) >> rsh;
                xi = base + v * (int64_t(1) << rsh);
            }
            if (xi < prev || xi > (int64_t)g.x1 || v > 32767 || v < -32767) ok = false;
            q[t - 1] = (int32_t)v;
            prev = xi;
        }
        if (!ok) q[0] = q[1] = q[2] = 0;
    }
    rec[m] = make_ushort4((uint16_t)(int16_t)q[0], (uint16_t)(int16_t)q[1], (uint16_t)(int16_t)q[2], 0);
}

// ---------------------------------------------------------------------------
// scan: per-segment bounds (and training pairs) over every bit of one level
// ---------------------------------------------------------------------------

struct ScanArgs {
    LevelDesc lv;
    uint32_t kl;
    uint32_t mode;
    const float* P[2];        // model parameters per b (mode kLearnMlp)
    const ushort4* rec[2];    // knot residuals per b (mode kLearnPla)
    uint32_t rsh[2];
    uint32_t* eps[2];         // per segment, zeroed before the scan; null = do not record bounds
    unsigned int* epsmax;     // [2] largest bound of the level per b
    float2* pairs[2];         // training pairs (u, t) per b; null = do not record pairs
    uint32_t* npairs;         // [2]
    uint64_t stride[2];       // record the pair of every stride-th b-bit
    uint32_t cap;
};

__global__ void __launch_bounds__(256) learn_scan_kernel(const __grid_constant__ ScanArgs a) {
    const LevelDesc& lv = a.lv;
    const uint64_t nblk = (lv.size + 511) / 512;
    const uint32_t ka = a.kl + kAnchorLog2;
    for (uint64_t blk = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; blk < nblk;
         blk += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t pos0 = blk << 9;
        const uint64_t ones_before = __ldg(lv.l1 + (pos0 >> 16)) + __ldg(lv.l2 + blk);
#pragma unroll 1
        for (uint32_t b = 0; b < 2; b++) {
            if (!a.eps[b] && !a.pairs[b]) continue;
            uint64_t r = b ? ones_before : pos0 - ones_before;  // b-bits before the block
            uint64_t cur_m = ~0ull;
            uint32_t cur_max = 0;
            Seg g = {0, 1, 0, 0};
            ushort4 rec = make_ushort4(0, 0, 0, 0);  // R = 0: the line through the anchors
            const float* P = a.P[b];
#pragma unroll 1
            for (uint32_t w = 0; w < 8; w++) {
                const uint64_t p = pos0 + 64 * w;
                if (p >= lv.size) break;
                uint64_t x = __ldg(lv.words + (blk << 3) + w);
                if (!b) x = ~x;
                const uint64_t nb = lv.size - p;
                if (nb < 64) x &= (1ull << nb) - 1ull;
                while (x) {
                    const uint32_t i = __ffsll((long long)x) - 1;
                    x &= x - 1;
                    const uint64_t k = ++r;
                    const uint64_t pos = p + i;
                    const uint64_t m = k >> ka;
                    if (m != cur_m) {
                        if (a.eps[b] && cur_m != ~0ull && cur_max) {
                            atomicMax(a.eps[b] + cur_m, cur_max);
                            atomicMax(a.epsmax + b, cur_max);
                        }
                        cur_m = m;
                        cur_max = 0;
                        g = anchor_seg(lv, b, m, a.kl);
                        if (a.mode == kLearnPla && a.rec[b]) rec = a.rec[b][m];
                    }
                    if (a.eps[b]) {
                        const uint64_t pr = predict(a.mode, g, rec, a.rsh[b], k, P, a.kl);
                        const uint64_t e = pr > pos ? pr - pos : pos - pr;
                        const uint32_t e32 = e > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)e;
                        cur_max = e32 > cur_max ? e32 : cur_max;
                    }
                    if (a.pairs[b] && (k % a.stride[b]) == 0 && k != g.k0) {
                        const uint32_t idx = atomicAdd(a.npairs + b, 1u);
                        if (idx < a.cap) {
                            const float u = (float)(k - g.k0) / (float)(g.k1 - g.k0);
                            const float t = (float)((double)(pos - g.x0) / (double)(g.x1 - g.x0));
                            a.pairs[b][idx] = make_float2(u, t);
                        }
                    }
                }
            }
            if (a.eps[b] && cur_m != ~0ull && cur_max) {
                atomicMax(a.eps[b] + cur_m, cur_max);
                atomicMax(a.epsmax + b, cur_max);
            }
        }
    }
}

// Bounds into the records: uint16 units of 2^esh bits, rounded up.
__global__ void __launch_bounds__(256) store_bounds_kernel(ushort4* rec, const uint32_t* eps, uint64_t nseg,
                                                           const unsigned int* epsmax) {
    const uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nseg) return;
    uint32_t esh = 0;
    while (esh < 31 && ((uint64_t)*epsmax + (1ull << esh) - 1) >> esh > 65535) esh++;
    const uint64_t q = ((uint64_t)eps[m] + (1ull << esh) - 1) >> esh;
    ushort4 r = rec[m];
    r.w = (uint16_t)q;
    rec[m] = r;
}

// ---------------------------------------------------------------------------
// MLP training: one CTA per model, lane j of every warp owns hidden unit j
// ---------------------------------------------------------------------------

constexpr int kTrainThreads = 256;
constexpr int kTrainWarps = kTrainThreads / 32;

// Full-batch loss (mean over n of (u + g(u) - t)^2) and gradient with respect
// to P, over data[0, n).  Called by all threads of the CTA; grad (kMlpParams
// floats) and *loss are written to shared memory by the end of the call.
__device__ void mlp_batch_grad(const float* P, const float2* data, uint32_t n, float* part /*[warps][params+1]*/,
                               float* grad, float* loss) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float w1 = P[lane], b1 = P[kMlpHidden + lane], w2 = P[2 * kMlpHidden + lane], b2 = P[3 * kMlpHidden];
    const float inv_n = n ? 1.f / (float)n : 0.f;
    float gw1 = 0.f, gb1 = 0.f, gw2 = 0.f, gb2 = 0.f, l = 0.f;
    for (uint32_t i = warp; i < n; i += kTrainWarps) {
        const float2 d = data[i];
        const float a = fmaf(w1, d.x, b1);
        const float h = fmaxf(a, 0.f);
        float y = w2 * h;
#pragma unroll
        for (int o = 16; o; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
        const float r = d.x + y + b2 - d.y;  // prediction error of this pair
        const float e = 2.f * r * inv_n;     // dLoss/dy
        gw2 += e * h;
        const float de = a > 0.f ? e * w2 : 0.f;
        gw1 += de * d.x;
        gb1 += de;
        gb2 += e;
        l += r * r * inv_n;
    }
    float* pw = part + warp * (kMlpParams + 1);
    pw[lane] = gw1;
    pw[kMlpHidden + lane] = gb1;
    pw[2 * kMlpHidden + lane] = gw2;
    if (lane == 0) {
        pw[3 * kMlpHidden] = gb2;
        pw[kMlpParams] = l;
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t <= kMlpParams; t += blockDim.x) {
        float s = 0.f;
        for (int w = 0; w < kTrainWarps; w++) s += part[w * (kMlpParams + 1) + t];
        if (t < kMlpParams) grad[t] = s;
        else *loss = s;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kTrainThreads) mlp_train_kernel(const float2* __restrict__ pairs,
                                                                  const uint32_t* __restrict__ npairs, uint32_t cap,
                                                                  float* __restrict__ params, uint32_t steps, float lr,
                                                                  float* __restrict__ losses) {
    extern __shared__ float2 data[];
    __shared__ float P[kMlpParams], M1[kMlpParams], M2[kMlpParams], G[kMlpParams];
    __shared__ float part[kTrainWarps * (kMlpParams + 1)];
    __shared__ float loss;
    const uint32_t model = blockIdx.x;
    const uint32_t n = min(npairs[model], cap);
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) data[i] = pairs[(uint64_t)model * cap + i];
    for (uint32_t t = threadIdx.x; t < kMlpParams; t += blockDim.x) {
        P[t] = params[model * kMlpParams + t];
        M1[t] = 0.f;
        M2[t] = 0.f;
    }
    __syncthreads();
    if (n == 0) return;
    const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    float c1 = 1.f, c2 = 1.f;
    for (uint32_t s = 0; s < steps; s++) {
        mlp_batch_grad(P, data, n, part, G, &loss);
        c1 *= beta1;
        c2 *= beta2;
        for (uint32_t t = threadIdx.x; t < kMlpParams; t += blockDim.x) {
            const float g = G[t];
            M1[t] = beta1 * M1[t] + (1.f - beta1) * g;
            M2[t] = beta2 * M2[t] + (1.f - beta2) * g * g;
            const float mh = M1[t] / (1.f - c1), vh = M2[t] / (1.f - c2);
            P[t] -= lr * mh / (sqrtf(vh) + eps);
        }
        __syncthreads();
    }
    mlp_batch_grad(P, data, n, part, G, &loss);
    for (uint32_t t = threadIdx.x; t < kMlpParams; t += blockDim.x) params[model * kMlpParams + t] = P[t];
    if (threadIdx.x == 0 && losses) losses[model] = loss;
}

// one gradient evaluation (no update), for checking the backward pass
__global__ void __launch_bounds__(kTrainThreads) mlp_grad_kernel(const float* __restrict__ params,
                                                                 const float2* __restrict__ pairs, uint32_t n,
                                                                 float* __restrict__ grad_out) {
    extern __shared__ float2 data[];
    __shared__ float P[kMlpParams], G[kMlpParams];
    __shared__ float part[kTrainWarps * (kMlpParams + 1)];
    __shared__ float loss;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) data[i] = pairs[i];
    for (uint32_t t = threadIdx.x; t < kMlpParams; t += blockDim.x) P[t] = params[t];
    __syncthreads();
    mlp_batch_grad(P, data, n, part, G, &loss);
    for (uint32_t t = threadIdx.x; t < kMlpParams; t += blockDim.x) grad_out[t] = G[t];
    if (threadIdx.x == 0) grad_out[kMlpParams] = loss;
}

// ---------------------------------------------------------------------------
// query
// ---------------------------------------------------------------------------

// {start, r0} of node (l, p) from the node table (slots are 32-byte aligned)
__device__ __forceinline__ ulonglong2 node_entry_sr(const TreeDesc& t, uint32_t l, uint64_t p) {
    const uint64_t slot = (1ull << l) - 1 + p;
    if (!dbg_in(slot < (1ull << t.cp.L) - 1, t.status)) return make_ulonglong2(0, 0);
    return ldg_nc_v2(reinterpret_cast<const uint64_t*>(t.nodes + slot));
}

// Learned select of NQ queries in lockstep (see do_select_n): per level the
// node entry (issued a level early), the anchor samples and the segment's
// record, the model's prediction p, then the staged search of the binary
// select (SelB) inside [p - eps, p + eps].  A query whose counters show the
// bit outside its window falls back to the sampled select and is counted.
template <int NQ, uint32_t MODE>
__device__ __forceinline__ void do_select_learned_n(const TreeDesc& t, const LearnedDesc& ld, const float* mlp_s,
                                                    const uint32_t (&c)[NQ], const uint64_t (&jin)[NQ],
                                                    const bool (&act)[NQ], uint64_t (&res)[NQ], uint32_t& fb) {
    const CodeParams& cp = t.cp;
    const uint32_t kl = t.k_log2;
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
        if (len[q]) ne[q] = node_entry_sr(t, len[q] - 1, (uint64_t)code[q] >> (cp.L - (len[q] - 1)));
    }
    for (int l = lmax; l >= 0; l--) {
        const LevelDesc& lv = t.lv[l];
        bool on[NQ];
        uint32_t b[NQ];
        uint64_t start[NQ], k[NQ];
        Seg g[NQ];
        ushort4 r[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            on[q] = NQ == 1 || l < (int)len[q];  // a lone query is on every level of the loop
            b[q] = (code[q] >> (cp.L - 1 - (uint32_t)l)) & 1u;
            start[q] = ne[q].x;
            // rank 1 of level l stands in for a query that is not on this level
            k[q] = on[q] ? (b[q] ? (start[q] - ne[q].y) : ne[q].y) + j[q] : 1ull;
            if (on[q] && l > 0) ne[q] = node_entry_sr(t, (uint32_t)l - 1, (uint64_t)code[q] >> (cp.L - (uint32_t)l + 1));
            const uint64_t m = k[q] >> (kl + kAnchorLog2);
            g[q] = anchor_seg(lv, b[q], m, kl);
            // records: (count_b >> (log2 K + kAnchorLog2)) + 1 per (level, b)
            r[q] = dbg_in(m < (lv_nsamples(lv, b[q], kl + kAnchorLog2)), lv.status) ? ld.rec[l][b[q]][m]
                                                                                   : make_ushort4(0, 0, 0, 0);
        }
        SelB s[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const uint64_t p = predict(MODE, g[q], r[q], ld.rsh[l][b[q]], k[q], mlp_s + (2 * l + b[q]) * kMlpParams, kl);
            const uint64_t e = (uint64_t)r[q].w << ld.esh[l][b[q]];
            const uint64_t hi = umin64(p + e, lv.size - 1);
            const uint64_t lo = umin64(p > e ? p - e : 0ull, hi);  // lo <= hi <= size - 1
            selb_window(s[q], b[q], k[q], lo, hi);
        }
#pragma unroll
        for (int q = 0; q < NQ; q++) selb_l1(s[q], lv);
#pragma unroll
        for (int q = 0; q < NQ; q++) selb_rank<true>(s[q]);
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
        for (int q = 0; q < NQ; q++) selb_words<true>(s[q], lv);
#pragma unroll
        for (int q = 0; q < NQ; q++) selb_half(s[q], lv, on[q]);
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            uint64_t pos = selb_finish<true>(s[q]);
            if (on[q] && !s[q].ok) {
                fb++;
                pos = select_b(lv, b[q], k[q], kl);
            }
            if (on[q]) j[q] = pos + 1 - start[q];
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; q++) res[q] = j[q] - 1;
}

constexpr int kLqThreads = 256;

// ORD: the queries were sorted by walk key; idx[k] is query k's original slot.
// NQ = 2 for deep trees, as for the sampled select.  Bounds: 48 registers for
// one query per thread, 64 for two (a few spilled words cost less than the
// fourth CTA per SM gains: 36.9 -> 35.4 ms for 10^8 PLA selects on a 16-level
// tree).
// MODE (kLearnPla or kLearnMlp) is a template parameter: each model's walk
// carries only its own prediction code, and the fitted-knot walk needs fewer
// registers without the network's.
template <bool ORD, int NQ, uint32_t MODE>
__global__ void __launch_bounds__(kLqThreads, NQ == 1 ? 5 : 4) select_learned_kernel(
    const __grid_constant__ TreeDesc t, const __grid_constant__ LearnedDesc ld, const uint32_t* __restrict__ qc,
    const uint64_t* __restrict__ qj, const uint32_t* __restrict__ idx, uint64_t* __restrict__ out, uint64_t q) {
    extern __shared__ float mlp_s[];
    if (MODE == kLearnMlp) {
        const uint32_t np = 2 * t.cp.L * kMlpParams;
        for (uint32_t i = threadIdx.x; i < np; i += blockDim.x) mlp_s[i] = ld.mlp[i];
        __syncthreads();
    }
    uint32_t fb = 0;
    const uint64_t stride = (uint64_t)NQ * gridDim.x * blockDim.x;
    for (uint64_t k0 = (uint64_t)NQ * ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x); k0 < q; k0 += stride) {
        uint32_t c[NQ];
        uint64_t j[NQ], r[NQ];
        bool in[NQ], ok[NQ], bad[NQ];
        bool any_bad = false;
#pragma unroll
        for (int x = 0; x < NQ; x++) {
            in[x] = k0 + x < q;
            c[x] = in[x] ? __ldg(qc + k0 + x) : 0u;
            j[x] = in[x] ? __ldg(qj + k0 + x) : 1ull;
            bad[x] = in[x] && (c[x] >= t.cp.sigma || j[x] == 0 || j[x] > __ldg(t.C + c[x] + 1) - __ldg(t.C + c[x]));
            ok[x] = in[x] && !bad[x];
            any_bad = any_bad || bad[x];
        }
        do_select_learned_n<NQ, MODE>(t, ld, mlp_s, c, j, ok, r, fb);
#pragma unroll
        for (int x = 0; x < NQ; x++)
            if (in[x]) out[ORD ? __ldg(idx + k0 + x) : k0 + x] = bad[x] ? UINT64_MAX : r[x];
        if (__any_sync(__activemask(), any_bad) && any_bad) atomicOr(t.status, kStQuery);
    }
    if (fb) atomicAdd(ld.fallbacks, (unsigned long long)fb);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static void init_mlp(float* P) {
    // g = 0 at the start (w2 = b2 = 0), hidden kinks spread over u in [0, 1]
    for (uint32_t j = 0; j < kMlpHidden; j++) {
        const float slope = (j & 1) ? -1.f : 1.f;
        const float knot = (j + 0.5f) / kMlpHidden;
        P[j] = slope;
        P[kMlpHidden + j] = -slope * knot;
        P[2 * kMlpHidden + j] = 0.f;
    }
    P[3 * kMlpHidden] = 0.f;
}

void free_learned(wt_tree_s* t, cudaStream_t s) {
    if (t->learned_mem) dev_free(t->learned_mem, s, tree_alloc(t));
    t->learned_mem = nullptr;
    t->learned_bytes = 0;
    memset(&t->learned, 0, sizeof(t->learned));
}

static uint64_t anchor_segments(const wt_tree_s* t, uint32_t l, uint32_t b) {
    const uint64_t cnt = b ? t->level_ones[l] : t->level_size[l] - t->level_ones[l];
    return (cnt >> (t->desc.k_log2 + kAnchorLog2)) + 1;
}

// mode kLearnPla: fit the knots (fit_knots_kernel, quantize_knots_kernel);
// mode kLearnMlp: training pairs from the levels, then Adam.  Both: the bound
// scan over every bit and the bounds into the records.
wt_status train_select(wt_tree_s* t, uint32_t mode, uint32_t steps, float lr, uint32_t pairs_cap, cudaStream_t s) {
    const uint32_t L = t->desc.cp.L, kl = t->desc.k_log2;
    free_learned(t, s);
    if (mode == kLearnNone || L == 0) return WT_OK;
    const wt_allocator* A = tree_alloc(t);
    // model memory: fallback counter | MLP params | records per (level, b)
    std::vector<size_t> roff(2 * L);
    size_t off = 256 + ((2 * L * kMlpParams * 4 + 255) / 256) * 256;
    uint64_t max_seg = 1;
    for (uint32_t l = 0; l < L; l++)
        for (uint32_t b = 0; b < 2; b++) {
            roff[2 * l + b] = off;
            const uint64_t ns = anchor_segments(t, l, b);
            off += (ns * sizeof(ushort4) + 255) / 256 * 256;
            max_seg = ns > max_seg ? ns : max_seg;
        }
    void* mem = nullptr;
    if (dev_alloc(&mem, off, s, A) != cudaSuccess) return WT_ENOMEM;
    t->learned_mem = mem;
    t->learned_bytes = off;
    uint8_t* M = static_cast<uint8_t*>(mem);
    LearnedDesc& ld = t->learned;
    ld.mode = mode;
    ld.fallbacks = reinterpret_cast<unsigned long long*>(M);
    float* mlp = reinterpret_cast<float*>(M + 256);
    ld.mlp = mlp;
    for (uint32_t l = 0; l < L; l++)
        for (uint32_t b = 0; b < 2; b++) ld.rec[l][b] = reinterpret_cast<const ushort4*>(M + roff[2 * l + b]);
    // scratch: per (level, b) maxima | residuals of the largest segment count | bounds | training pairs
    const size_t sc_max = 256, sc_res = sc_max + ((size_t)4 * L * 4 + 255) / 256 * 256;
    const size_t sc_eps = sc_res + (max_seg * 3 * 4 + 255) / 256 * 256;
    const size_t sc_pairs = sc_eps + (2 * max_seg * 4 + 255) / 256 * 256;
    const size_t sc_end = sc_pairs + (mode == kLearnMlp ? (size_t)2 * L * pairs_cap * sizeof(float2) + 2 * L * 4 : 0);
    void* scratch = nullptr;
    if (dev_alloc(&scratch, sc_end, s, A) != cudaSuccess) {
        free_learned(t, s);  // no half-trained model stays behind
        return WT_ENOMEM;
    }
    uint8_t* X = static_cast<uint8_t*>(scratch);
    unsigned int* maxabs = reinterpret_cast<unsigned int*>(X + sc_max);      // [L][2]
    unsigned int* epsmax = maxabs + 2 * L;                                    // [L][2]
    float* resid = reinterpret_cast<float*>(X + sc_res);
    uint32_t* eps = reinterpret_cast<uint32_t*>(X + sc_eps);
    wt_status st = WT_OK;
    auto fail = [&](wt_status e) {
        dev_free(scratch, s, A);
        free_learned(t, s);
        return e;
    };
    if (cudaMemsetAsync(mem, 0, off, s) != cudaSuccess || cudaMemsetAsync(scratch, 0, sc_res, s) != cudaSuccess)
        return fail(WT_ECUDA);
    std::vector<float> hp(2 * L * kMlpParams);
    for (uint32_t i = 0; i < 2 * L; i++) init_mlp(hp.data() + i * kMlpParams);
    if (cudaMemcpyAsync(mlp, hp.data(), hp.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)  // hp is a host temporary
        return fail(WT_ECUDA);
    const int grid = sm_count() * 8;

    if (mode == kLearnPla) {
        for (uint32_t l = 0; l < L && st == WT_OK; l++) {
            if (!t->level_size[l]) continue;
            for (uint32_t b = 0; b < 2; b++) {
                FitArgs fa;
                fa.lv = t->desc.lv[l];
                fa.b = b;
                fa.kl = kl;
                fa.nseg = anchor_segments(t, l, b);
                fa.resid = resid;
                fa.maxabs = maxabs + 2 * l + b;
                {
                    ProfScope ps("learn_fit", s);
                    fit_knots_kernel<<<(unsigned)((fa.nseg * 32 + 255) / 256), 256, 0, s>>>(fa);
                }
                {
                    ProfScope ps("learn_quantize", s);
                    quantize_knots_kernel<<<(unsigned)((fa.nseg + 255) / 256), 256, 0, s>>>(
                        fa, const_cast<ushort4*>(ld.rec[l][b]), fa.maxabs);
                }
            }
        }
    } else {
        // training pairs from the built levels, then Adam on every model at once
        float2* pairs = reinterpret_cast<float2*>(X + sc_pairs);
        uint32_t* npairs = reinterpret_cast<uint32_t*>(X + sc_pairs + (size_t)2 * L * pairs_cap * sizeof(float2));
        if (cudaMemsetAsync(npairs, 0, 2 * L * 4, s) != cudaSuccess) return fail(WT_ECUDA);
        for (uint32_t l = 0; l < L; l++) {
            if (!t->level_size[l]) continue;
            ScanArgs a;
            memset(&a, 0, sizeof(a));
            a.lv = t->desc.lv[l];
            a.kl = kl;
            a.mode = kLearnMlp;
            a.cap = pairs_cap;
            a.npairs = npairs + 2 * l;
            for (uint32_t b = 0; b < 2; b++) {
                const uint64_t cnt = b ? t->level_ones[l] : t->level_size[l] - t->level_ones[l];
                a.pairs[b] = pairs + (size_t)(2 * l + b) * pairs_cap;
                a.stride[b] = cnt > pairs_cap ? (cnt + pairs_cap - 1) / pairs_cap : 1;
            }
            ProfScope ps("learn_pairs", s);
            learn_scan_kernel<<<grid, 256, 0, s>>>(a);
        }
        const size_t sm = (size_t)pairs_cap * sizeof(float2);
        static bool cfg = false;
        if (!cfg) {
            cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
            cfg = true;
        }
        ProfScope ps("mlp_train", s);
        mlp_train_kernel<<<2 * L, kTrainThreads, sm, s>>>(pairs, npairs, pairs_cap, mlp, steps, lr, nullptr);
    }
    std::vector<unsigned int> hmax(4 * L, 0);
    if (cudaMemcpyAsync(hmax.data(), maxabs, 2 * L * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(WT_ECUDA);
    for (uint32_t l = 0; l < L; l++)
        for (uint32_t b = 0; b < 2; b++) {
            float mx;
            memcpy(&mx, &hmax[2 * l + b], 4);
            uint32_t sh = 0;
            while (sh < 30 && mx > 32767.f * (float)(1u << sh)) sh++;
            ld.rsh[l][b] = (uint8_t)(mode == kLearnPla ? sh : 0);
        }
    // bounds: one scan per level over both bit values, then into the records
    for (uint32_t l = 0; l < L; l++) {
        if (!t->level_size[l]) continue;
        const uint64_t ns[2] = {anchor_segments(t, l, 0), anchor_segments(t, l, 1)};
        if (cudaMemsetAsync(eps, 0, (ns[0] + ns[1]) * 4, s) != cudaSuccess) return fail(WT_ECUDA);
        ScanArgs a;
        memset(&a, 0, sizeof(a));
        a.lv = t->desc.lv[l];
        a.kl = kl;
        a.mode = mode;
        a.epsmax = epsmax + 2 * l;
        for (uint32_t b = 0; b < 2; b++) {
            a.P[b] = mlp + (2 * l + b) * kMlpParams;
            a.rec[b] = ld.rec[l][b];
            a.rsh[b] = ld.rsh[l][b];
            a.eps[b] = eps + (b ? ns[0] : 0);
            a.stride[b] = 1;
        }
        {
            ProfScope ps("learn_bounds", s);
            learn_scan_kernel<<<grid, 256, 0, s>>>(a);
        }
        for (uint32_t b = 0; b < 2; b++) {
            ProfScope ps("learn_store", s);
            store_bounds_kernel<<<(unsigned)((ns[b] + 255) / 256), 256, 0, s>>>(const_cast<ushort4*>(ld.rec[l][b]),
                                                                                a.eps[b], ns[b], epsmax + 2 * l + b);
        }
    }
    std::vector<unsigned int> hemax(2 * L, 0);
    if (cudaMemcpyAsync(hemax.data(), epsmax, 2 * L * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(WT_ECUDA);
    for (uint32_t l = 0; l < L; l++)
        for (uint32_t b = 0; b < 2; b++) {
            uint32_t esh = 0;
            while (esh < 31 && (((uint64_t)hemax[2 * l + b] + (1ull << esh) - 1) >> esh) > 65535) esh++;
            ld.esh[l][b] = (uint8_t)esh;
        }
    dev_free(scratch, s, A);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

using LearnedKernel = void (*)(TreeDesc, LearnedDesc, const uint32_t*, const uint64_t*, const uint32_t*, uint64_t*,
                               uint64_t);

static LearnedKernel learned_kernel(bool ord, bool pair, bool mlp) {
    if (ord) {
        if (pair) return mlp ? select_learned_kernel<true, 2, kLearnMlp> : select_learned_kernel<true, 2, kLearnPla>;
        return mlp ? select_learned_kernel<true, 1, kLearnMlp> : select_learned_kernel<true, 1, kLearnPla>;
    }
    if (pair) return mlp ? select_learned_kernel<false, 2, kLearnMlp> : select_learned_kernel<false, 2, kLearnPla>;
    return mlp ? select_learned_kernel<false, 1, kLearnMlp> : select_learned_kernel<false, 1, kLearnPla>;
}

wt_status launch_select_learned(const wt_tree_s* t, const uint32_t* d_c, const uint64_t* d_j, uint64_t* d_out,
                                uint64_t q, cudaStream_t s) {
    if (!q) return WT_OK;
    const bool mlp = t->learned.mode == kLearnMlp;
    const size_t sm = mlp ? (size_t)2 * t->desc.cp.L * kMlpParams * 4 : 0;
    const bool pair = t->desc.cp.L >= kPairLevels;
    static int per_sm[2][2] = {{0, 0}, {0, 0}};
    if (!per_sm[pair][mlp]) {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, learned_kernel(false, pair, mlp), kLqThreads, 20 * 1024);
        per_sm[pair][mlp] = v > 0 ? v : 1;
    }
    uint64_t need = (q + kLqThreads - 1) / kLqThreads, full = (uint64_t)per_sm[pair][mlp] * sm_count();
    const unsigned grid = (unsigned)(need < full ? need : full);
    const char* name = mlp ? "select_learned_mlp" : "select_learned_pla";
    // large batches walk in the same order as the sampled select's
    if (use_order(t, q)) {
        Ordered o;
        wt_status st = order_queries(t, 2, nullptr, d_c, d_j, q, s, o);
        if (st == WT_OK) {
            ProfScope ps(name, s);
            learned_kernel(true, pair, mlp)<<<grid, kLqThreads, sm, s>>>(t->desc, t->learned, o.c, o.a, o.idx, d_out, q);
            if (cudaGetLastError() != cudaSuccess) st = WT_ECUDA;
        }
        if (o.mem) dev_free(o.mem, s, tree_alloc(t));
        return st;
    }
    ProfScope ps(name, s);
    learned_kernel(false, pair, mlp)<<<grid, kLqThreads, sm, s>>>(t->desc, t->learned, d_c, d_j, nullptr, d_out, q);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

}  // namespace wt

using namespace wt;

static bool tree_valid(const wt_tree_s* t) { return t && t->magic == kTreeMagic; }

static bool dev_ptr(const void* p) { return device_ptr_ok(p); }

namespace wt {
// wt_export of the learned model: per anchor segment the bound (uint32 bits)
// or the three knot residuals (int32 bits).  Synchronous.
wt_status export_learned(const wt_tree_s* t, uint32_t level, uint32_t b, bool resid, void* h_dst, uint64_t* count) {
    const uint64_t segs = anchor_segments(t, level, b);
    *count = resid ? 3 * segs : segs;
    if (!h_dst) return WT_OK;
    std::vector<ushort4> r(segs);
    if (cudaStreamSynchronize(t->stream) != cudaSuccess ||
        cudaMemcpy(r.data(), t->learned.rec[level][b], segs * sizeof(ushort4), cudaMemcpyDeviceToHost) != cudaSuccess)
        return WT_ECUDA;
    for (uint64_t m = 0; m < segs; m++) {
        if (resid) {
            int32_t* o = static_cast<int32_t*>(h_dst) + 3 * m;
            const uint32_t sh = t->learned.rsh[level][b];
            o[0] = (int32_t)((int64_t)(int16_t)r[m].x * (int64_t(1) << sh));
            o[1] = (int32_t)((int64_t)(int16_t)r[m].y * (int64_t(1) << sh));
            o[2] = (int32_t)((int64_t)(int16_t)r[m].z * (int64_t(1) << sh));
        } else {
            const uint64_t e = (uint64_t)r[m].w << t->learned.esh[level][b];
            static_cast<uint32_t*>(h_dst)[m] = (uint32_t)(e > 0xFFFFFFFFull ? 0xFFFFFFFFull : e);
        }
    }
    return WT_OK;
}
}  // namespace wt

extern "C" {

wt_status wt_train_select(wt_tree tree, uint32_t mode, const wt_train_options* opt, wt_stream stream) {
    if (!tree_valid(tree) || mode > kLearnMlp) return WT_EINVAL;
    if (tree->desc.layout == WT_LAYOUT_MATRIX) return WT_EUNSUPPORTED;
    const uint32_t steps = (opt && opt->steps) ? opt->steps : 300;
    const float lr = (opt && opt->lr > 0.f) ? opt->lr : 1e-2f;
    const uint32_t pairs = (opt && opt->pairs) ? opt->pairs : 8192;
    if (pairs > 16384 || steps > 100000) return WT_EINVAL;
    return train_select(tree, mode, steps, lr, pairs, stream);
}

wt_status wt_select_learned(wt_tree tree, const uint32_t* d_c, const uint64_t* d_j, uint64_t* d_out, uint64_t q,
                            wt_stream stream) {
    if (!tree_valid(tree)) return WT_EINVAL;
    if (tree->learned.mode == kLearnNone) return tree->desc.cp.L ? WT_EUNSUPPORTED : launch_select(tree, d_c, d_j, d_out, q, stream);
    if (!q) return WT_OK;
    if (!dev_ptr(d_c) || !dev_ptr(d_j) || !dev_ptr(d_out)) return WT_EINVAL;
    return launch_select_learned(tree, d_c, d_j, d_out, q, stream);
}

wt_status wt_learned_info(wt_tree tree, wt_learned_info_t* out) {
    if (!tree_valid(tree) || !out) return WT_EINVAL;
    memset(out, 0, sizeof(*out));
    const LearnedDesc& ld = tree->learned;
    out->mode = ld.mode;
    if (ld.mode == kLearnNone) return WT_OK;
    if (cudaStreamSynchronize(tree->stream) != cudaSuccess) return WT_ECUDA;
    unsigned long long fb = 0;
    if (cudaMemcpy(&fb, ld.fallbacks, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return WT_ECUDA;
    out->fallbacks = fb;
    const uint32_t L = tree->desc.cp.L;
    uint64_t anchors = 0;
    for (uint32_t l = 0; l < L; l++) {
        for (uint32_t b = 0; b < 2; b++) {
            const uint64_t segs = anchor_segments(tree, l, b);
            anchors += segs * 8;
            std::vector<ushort4> r(segs);
            if (cudaMemcpy(r.data(), ld.rec[l][b], segs * sizeof(ushort4), cudaMemcpyDeviceToHost) != cudaSuccess)
                return WT_ECUDA;
            double sum = 0;
            uint64_t mx = 0;
            for (const ushort4& v : r) {
                const uint64_t e = (uint64_t)v.w << ld.esh[l][b];
                sum += (double)e;
                mx = e > mx ? e : mx;
            }
            out->eps_mean[l][b] = segs ? sum / segs : 0.0;
            out->eps_max[l][b] = (uint32_t)(mx > 0xFFFFFFFFull ? 0xFFFFFFFFull : mx);
        }
    }
    out->anchor_bytes = anchors;
    out->model_bytes = tree->learned_bytes;
    return WT_OK;
}

wt_status wt_mlp_gradient(const float* h_params, const float* h_u, const float* h_t, uint32_t n, float* h_grad,
                          float* h_loss) {
    if (!h_params || !h_u || !h_t || !h_grad || n == 0 || n > 16384) return WT_EINVAL;
    std::vector<float2> pairs(n);
    for (uint32_t i = 0; i < n; i++) pairs[i] = make_float2(h_u[i], h_t[i]);
    void* d = nullptr;
    const size_t bytes = n * sizeof(float2) + 2 * kMlpParams * 4 + 256;
    if (cudaMalloc(&d, bytes) != cudaSuccess) return WT_ENOMEM;
    float2* dp = static_cast<float2*>(d);
    float* dpar = reinterpret_cast<float*>(dp + n);
    float* dg = dpar + kMlpParams;
    wt_status st = WT_OK;
    if (cudaMemcpy(dp, pairs.data(), n * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dpar, h_params, kMlpParams * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        st = WT_ECUDA;
    } else {
        cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        {
            ProfScope ps("mlp_grad", 0);
            mlp_grad_kernel<<<1, kTrainThreads, n * sizeof(float2)>>>(dpar, dp, n, dg);
        }
        std::vector<float> g(kMlpParams + 1);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(g.data(), dg, (kMlpParams + 1) * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
            st = WT_ECUDA;
        } else {
            memcpy(h_grad, g.data(), kMlpParams * 4);
            if (h_loss) *h_loss = g[kMlpParams];
        }
    }
    cudaFree(d);
    return st;
}

}  // extern "C"
