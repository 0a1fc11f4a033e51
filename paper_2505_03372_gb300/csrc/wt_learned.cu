// Learned select: a model per (level, bit value b) predicts where the k-th
// b-bit of a level lies, a stored per-segment bound eps makes the prediction
// exact, and the sampled select of Algorithm 2 is the fallback.
//
// Knots.  The build already stores, per level and b, the position S_b[m] of
// the (m*K)-th b-bit (Section 4.2).  Those (rank -> position) pairs are the
// knots of every model: k in segment m = k >> log2(K) lies between
// (k0 = m*K, x0 = S_b[m]) and (k1 = (m+1)*K, x1 = S_b[m+1]); the last segment
// ends at the virtual (count_b + 1)-th b-bit at position size_l.
//
// Models.  PLA: linear interpolation between the knots (the predictor with
// nothing learned).  MLP: the within-segment fraction u = (k - k0) / (k1 - k0)
// is mapped to h = u + g(u), g a 1 -> 32 -> 1 ReLU network in FP32 shared by all
// segments of a (level, b); prediction x0 + floor((x1 - x0) * h).  g is trained
// on the GPU (Adam, full-batch) on pairs (u, (pos - x0) / (x1 - x0)) that the
// scan kernel enumerates from the built levels; it starts at g = 0, i.e. at PLA.
//
// Bounds.  A scan over every bit of every level evaluates the model at every
// b-bit's rank k and keeps eps_b[m] = max |prediction(k) - position(k)| per
// segment.  The prediction is a fixed sequence of correctly rounded operations
// (__fmaf_rn, __fmul_rn, __fdiv_rn), so the query reproduces it exactly.
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

struct Knots {
    uint64_t k0, k1, x0, x1;
};

__device__ __forceinline__ Knots seg_knots(const LevelDesc& lv, uint32_t b, uint64_t m, uint32_t kl) {
    const uint64_t* S = b ? lv.s1 : lv.s0;
    const uint64_t total = b ? lv.ones : lv.size - lv.ones;
    Knots kn;
    kn.k0 = m << kl;
    kn.x0 = __ldg(S + m);
    if (((m + 1) << kl) <= total) {
        kn.k1 = (m + 1) << kl;
        kn.x1 = __ldg(S + m + 1);
    } else {
        kn.k1 = total + 1;
        kn.x1 = lv.size;
    }
    return kn;
}

__device__ __forceinline__ uint64_t predict_pla(const Knots& kn, uint64_t k) {
    return kn.x0 + ((k - kn.k0) * (kn.x1 - kn.x0)) / (kn.k1 - kn.k0);
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

__device__ __forceinline__ uint64_t predict_mlp(const Knots& kn, uint64_t k, const float* P) {
    const float u = __fdiv_rn((float)(k - kn.k0), (float)(kn.k1 - kn.k0));
    float h = __fadd_rn(u, mlp_g(P, u));
    h = fminf(fmaxf(h, 0.f), 1.f);
    const uint64_t span = kn.x1 - kn.x0;
    uint64_t off = (uint64_t)__fmul_rn((float)span, h);
    return kn.x0 + (off < span ? off : span);
}

__device__ __forceinline__ uint64_t predict(uint32_t mode, const Knots& kn, uint64_t k, const float* P) {
    return mode == kLearnMlp ? predict_mlp(kn, k, P) : predict_pla(kn, k);
}

// ---------------------------------------------------------------------------
// scan: per-segment bounds (and training pairs) over every bit of one level
// ---------------------------------------------------------------------------

struct ScanArgs {
    LevelDesc lv;
    uint32_t kl;
    uint32_t mode;
    const float* P[2];        // model parameters per b (mode kLearnMlp)
    uint32_t* eps[2];         // zeroed before the scan; null = do not record bounds
    float2* pairs[2];         // training pairs (u, t) per b; null = do not record pairs
    uint32_t* npairs;         // [2]
    uint64_t stride[2];       // record the pair of every stride-th b-bit
    uint32_t cap;
};

__global__ void __launch_bounds__(256) learn_scan_kernel(const __grid_constant__ ScanArgs a) {
    const LevelDesc& lv = a.lv;
    const uint64_t nblk = (lv.size + 511) / 512;
    for (uint64_t blk = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; blk < nblk;
         blk += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t pos0 = blk << 9;
        const uint64_t ones_before = __ldg(lv.l1 + (pos0 >> 16)) + __ldg(lv.l2 + blk);
#pragma unroll 1
        for (uint32_t b = 0; b < 2; b++) {
            uint64_t r = b ? ones_before : pos0 - ones_before;  // b-bits before the block
            uint64_t cur_m = ~0ull;
            uint32_t cur_max = 0;
            Knots kn = {0, 1, 0, 0};
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
                    const uint64_t m = k >> a.kl;
                    if (m != cur_m) {
                        if (a.eps[b] && cur_m != ~0ull && cur_max) atomicMax(a.eps[b] + cur_m, cur_max);
                        cur_m = m;
                        cur_max = 0;
                        kn = seg_knots(lv, b, m, a.kl);
                    }
                    if (a.eps[b]) {
                        const uint64_t pr = predict(a.mode, kn, k, P);
                        const uint64_t e = pr > pos ? pr - pos : pos - pr;
                        const uint32_t e32 = e > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)e;
                        cur_max = e32 > cur_max ? e32 : cur_max;
                    }
                    if (a.pairs[b] && (k % a.stride[b]) == 0 && k != kn.k0) {
                        const uint32_t idx = atomicAdd(a.npairs + b, 1u);
                        if (idx < a.cap) {
                            const float u = (float)(k - kn.k0) / (float)(kn.k1 - kn.k0);
                            const float t = (float)((double)(pos - kn.x0) / (double)(kn.x1 - kn.x0));
                            a.pairs[b][idx] = make_float2(u, t);
                        }
                    }
                }
            }
            if (a.eps[b] && cur_m != ~0ull && cur_max) atomicMax(a.eps[b] + cur_m, cur_max);
        }
    }
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

// Sampled-select search restricted to the window [lo, hi]; ok = false if the
// counters show the k-th b-bit is not inside it.
__device__ __forceinline__ uint64_t select_b_window(const LevelDesc& lv, uint32_t b, uint64_t k, uint64_t lo,
                                                    uint64_t hi, bool& ok) {
    uint64_t i1 = lo >> 16;
    const uint64_t hi1 = hi >> 16;
    while (i1 < hi1) {
        const uint64_t nx = i1 + 1;
        const uint64_t c1 = __ldg(lv.l1 + nx);
        if ((b ? c1 : (nx << 16) - c1) < k) i1 = nx;
        else break;
    }
    const uint64_t c1 = __ldg(lv.l1 + i1);
    const uint64_t base1 = b ? c1 : (i1 << 16) - c1;
    if (base1 >= k) {
        ok = false;
        return 0;
    }
    uint64_t kk = k - base1;
    uint64_t lo2 = umax64(i1 << 7, lo >> 9);
    uint64_t hi2 = umin64((i1 << 7) + 127, hi >> 9);
    if (lo2 > hi2) lo2 = hi2;
    while (lo2 < hi2) {
        const uint64_t mid = (lo2 + hi2 + 1) >> 1;
        const uint64_t c2 = __ldg(lv.l2 + mid);
        if ((b ? c2 : ((mid << 9) - (i1 << 16)) - c2) < kk) lo2 = mid;
        else hi2 = mid - 1;
    }
    {
        const uint64_t c2 = __ldg(lv.l2 + lo2);
        const uint64_t cb = b ? c2 : ((lo2 << 9) - (i1 << 16)) - c2;
        if (cb >= kk) {
            ok = false;
            return 0;
        }
        kk -= cb;
    }
    // words of the 512-bit block, one 32-byte half at a time
    const uint64_t* wp = lv.words + (lo2 << 3);
    uint32_t kw = (uint32_t)kk;
#pragma unroll 1
    for (uint32_t h = 0; h < 8; h += 4) {
        uint64_t w[4];
        ldg_nc_v4(wp + h, w[0], w[1], w[2], w[3]);
#pragma unroll
        for (uint32_t e = 0; e < 4; e++) {
            const uint64_t a = b ? w[e] : ~w[e];
            const uint32_t p = __popcll(a);
            if (p >= kw) return (lo2 << 9) + ((uint64_t)(h + e) << 6) + select_in_word(a, kw);
            kw -= p;
        }
    }
    ok = false;  // not in this 512-bit block: the window did not hold the bit
    return 0;
}

__device__ __forceinline__ uint64_t select_b_learned(const TreeDesc& t, const LearnedDesc& ld, const float* mlp_s,
                                                     uint32_t l, uint32_t b, uint64_t k, uint32_t& fb) {
    const LevelDesc& lv = t.lv[l];
    const uint64_t m = k >> t.k_log2;
    const Knots kn = seg_knots(lv, b, m, t.k_log2);
    const uint64_t p = predict(ld.mode, kn, k, mlp_s + (2 * l + b) * kMlpParams);
    const uint64_t e = __ldg(ld.eps[l][b] + m);
    const uint64_t lo = p > e ? p - e : 0;
    const uint64_t hi = umin64(p + e, lv.size - 1);
    bool ok = true;
    const uint64_t pos = select_b_window(lv, b, k, lo, hi, ok);
    if (ok) return pos;
    fb++;
    return select_b(lv, b, k, t.k_log2);
}

constexpr int kLqThreads = 256;

// ORD: the queries were sorted by walk key; idx[k] is query k's original slot.
template <bool ORD>
__global__ void __launch_bounds__(kLqThreads) select_learned_kernel(const __grid_constant__ TreeDesc t,
                                                                    const __grid_constant__ LearnedDesc ld,
                                                                    const uint32_t* __restrict__ qc,
                                                                    const uint64_t* __restrict__ qj,
                                                                    const uint32_t* __restrict__ idx,
                                                                    uint64_t* __restrict__ out, uint64_t q) {
    extern __shared__ float mlp_s[];
    if (ld.mode == kLearnMlp) {
        const uint32_t np = 2 * t.cp.L * kMlpParams;
        for (uint32_t i = threadIdx.x; i < np; i += blockDim.x) mlp_s[i] = ld.mlp[i];
        __syncthreads();
    }
    uint32_t fb = 0;
    for (uint64_t kq = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; kq < q; kq += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = __ldg(qc + kq);
        uint64_t j = __ldg(qj + kq);
        bool bad = c >= t.cp.sigma || j == 0;
        if (!bad) bad = j > __ldg(t.C + c + 1) - __ldg(t.C + c);
        uint64_t res = UINT64_MAX;
        if (!bad) {
            uint32_t code, len;
            encode(t.cp, c, code, len);
            for (int l = (int)len - 1; l >= 0; l--) {
                const uint32_t b = (code >> (t.cp.L - 1 - (uint32_t)l)) & 1u;
                const ulonglong2 ne =
                    ldg_nc_v2(reinterpret_cast<const uint64_t*>(t.nodes + ((1ull << l) - 1 + ((uint64_t)code >> (t.cp.L - (uint32_t)l)))));
                const uint64_t kb = b ? (ne.x - ne.y) : ne.y;
                const uint64_t pos = select_b_learned(t, ld, mlp_s, (uint32_t)l, b, kb + j, fb);
                j = pos + 1 - ne.x;
            }
            res = j - 1;
        }
        out[ORD ? __ldg(idx + kq) : kq] = res;
        if (__any_sync(__activemask(), bad) && bad) atomicOr(t.status, kStQuery);
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

wt_status train_select(wt_tree_s* t, uint32_t mode, uint32_t steps, float lr, uint32_t pairs_cap, cudaStream_t s) {
    const uint32_t L = t->desc.cp.L, kl = t->desc.k_log2;
    free_learned(t, s);
    if (mode == kLearnNone || L == 0) return WT_OK;
    // layout: fallback counter | MLP params | eps arrays
    std::vector<size_t> eoff(2 * L);
    size_t off = 256 + ((2 * L * kMlpParams * 4 + 255) / 256) * 256;
    for (uint32_t l = 0; l < L; l++) {
        for (uint32_t b = 0; b < 2; b++) {
            const uint64_t cnt = b ? t->level_ones[l] : t->level_size[l] - t->level_ones[l];
            eoff[2 * l + b] = off;
            off += (((cnt >> kl) + 1) * 4 + 255) / 256 * 256;
        }
    }
    void* mem = nullptr;
    if (dev_alloc(&mem, off, s, tree_alloc(t)) != cudaSuccess) return WT_ENOMEM;
    t->learned_mem = mem;
    t->learned_bytes = off;
    uint8_t* M = static_cast<uint8_t*>(mem);
    WT_CUDA_TRY(cudaMemsetAsync(mem, 0, off, s));
    LearnedDesc& ld = t->learned;
    ld.mode = mode;
    ld.fallbacks = reinterpret_cast<unsigned long long*>(M);
    float* mlp = reinterpret_cast<float*>(M + 256);
    ld.mlp = mlp;
    for (uint32_t l = 0; l < L; l++)
        for (uint32_t b = 0; b < 2; b++) ld.eps[l][b] = reinterpret_cast<uint32_t*>(M + eoff[2 * l + b]);

    const int grid = sm_count() * 8;
    std::vector<float> hp(2 * L * kMlpParams);
    for (uint32_t i = 0; i < 2 * L; i++) init_mlp(hp.data() + i * kMlpParams);
    WT_CUDA_TRY(cudaMemcpyAsync(mlp, hp.data(), hp.size() * 4, cudaMemcpyHostToDevice, s));
    WT_CUDA_TRY(cudaStreamSynchronize(s));  // hp is a host temporary

    if (mode == kLearnMlp) {
        // training pairs from the built levels, then Adam on every model at once
        void* scratch = nullptr;
        const size_t pbytes = (size_t)2 * L * pairs_cap * sizeof(float2);
        if (dev_alloc(&scratch, pbytes + 2 * L * 4 + 256, s, tree_alloc(t)) != cudaSuccess) {
            free_learned(t, s);  // no half-trained model stays behind
            return WT_ENOMEM;
        }
        float2* pairs = static_cast<float2*>(scratch);
        uint32_t* npairs = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(scratch) + pbytes);
        WT_CUDA_TRY(cudaMemsetAsync(npairs, 0, 2 * L * 4, s));
        for (uint32_t l = 0; l < L; l++) {
            if (!t->level_size[l]) continue;
            ScanArgs a;
            memset(&a, 0, sizeof(a));
            a.lv = t->desc.lv[l];
            a.kl = kl;
            a.mode = kLearnPla;
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
        {
            const size_t sm = (size_t)pairs_cap * sizeof(float2);
            static bool cfg = false;
            if (!cfg) {
                cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
                cfg = true;
            }
            ProfScope ps("mlp_train", s);
            mlp_train_kernel<<<2 * L, kTrainThreads, sm, s>>>(pairs, npairs, pairs_cap, mlp, steps, lr, nullptr);
        }
        dev_free(scratch, s, tree_alloc(t));
    }
    for (uint32_t l = 0; l < L; l++) {
        if (!t->level_size[l]) continue;
        ScanArgs a;
        memset(&a, 0, sizeof(a));
        a.lv = t->desc.lv[l];
        a.kl = kl;
        a.mode = mode;
        for (uint32_t b = 0; b < 2; b++) {
            a.P[b] = mlp + (2 * l + b) * kMlpParams;
            a.eps[b] = const_cast<uint32_t*>(ld.eps[l][b]);
            a.stride[b] = 1;
        }
        ProfScope ps("learn_bounds", s);
        learn_scan_kernel<<<grid, 256, 0, s>>>(a);
    }
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

wt_status launch_select_learned(const wt_tree_s* t, const uint32_t* d_c, const uint64_t* d_j, uint64_t* d_out,
                                uint64_t q, cudaStream_t s) {
    if (!q) return WT_OK;
    const size_t sm = t->learned.mode == kLearnMlp ? (size_t)2 * t->desc.cp.L * kMlpParams * 4 : 0;
    static int per_sm = 0;
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_learned_kernel<false>, kLqThreads, 20 * 1024);
        if (per_sm <= 0) per_sm = 1;
    }
    uint64_t need = (q + kLqThreads - 1) / kLqThreads, full = (uint64_t)per_sm * sm_count();
    const unsigned grid = (unsigned)(need < full ? need : full);
    const char* name = t->learned.mode == kLearnMlp ? "select_learned_mlp" : "select_learned_pla";
    // large batches walk in the same order as the sampled select's
    if (use_order(t, q)) {
        Ordered o;
        wt_status st = order_queries(t, 2, nullptr, d_c, d_j, q, s, o);
        if (st == WT_OK) {
            ProfScope ps(name, s);
            select_learned_kernel<true><<<grid, kLqThreads, sm, s>>>(t->desc, t->learned, o.c, o.a, o.idx, d_out, q);
            if (cudaGetLastError() != cudaSuccess) st = WT_ECUDA;
        }
        if (o.mem) dev_free(o.mem, s, tree_alloc(t));
        return st;
    }
    ProfScope ps(name, s);
    select_learned_kernel<false><<<grid, kLqThreads, sm, s>>>(t->desc, t->learned, d_c, d_j, nullptr, d_out, q);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ECUDA;
}

}  // namespace wt

using namespace wt;

static bool tree_valid(const wt_tree_s* t) { return t && t->magic == kTreeMagic; }

static bool dev_ptr(const void* p) { return device_ptr_ok(p); }

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
    const uint32_t L = tree->desc.cp.L, kl = tree->desc.k_log2;
    for (uint32_t l = 0; l < L; l++) {
        for (uint32_t b = 0; b < 2; b++) {
            const uint64_t cnt = b ? tree->level_ones[l] : tree->level_size[l] - tree->level_ones[l];
            const uint64_t segs = (cnt >> kl) + 1;
            std::vector<uint32_t> e(segs);
            if (cudaMemcpy(e.data(), ld.eps[l][b], segs * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return WT_ECUDA;
            double sum = 0;
            uint32_t mx = 0;
            for (uint32_t v : e) {
                sum += v;
                mx = v > mx ? v : mx;
            }
            out->eps_mean[l][b] = segs ? sum / segs : 0.0;
            out->eps_max[l][b] = mx;
        }
    }
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
