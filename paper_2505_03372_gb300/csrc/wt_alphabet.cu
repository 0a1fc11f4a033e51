// Minimal-alphabet extraction: the distinct values of a text, their ranks as
// the new symbols, through a presence bitmap with rank/select support (the same
// binary rank and select a tree level uses, Sections 4.1 and 4.2).
#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_internal.hpp"

extern "C" wt_status wt_bitvector_support_static(const uint64_t* d_words, uint64_t nbits, uint32_t sample_k,
                                                 uint64_t* d_l1, uint16_t* d_l2, uint64_t* d_s0, uint64_t* d_s1,
                                                 uint64_t sample_capacity, uint32_t* d_status, uint64_t* d_ones,
                                                 wt_stream stream);

namespace wt {
namespace {

constexpr int kAlThreads = 512;
constexpr uint32_t kAlSampleK = 4096;

// presence bitmap of the values; byte and 16-bit symbols first mark a
// per-CTA bitmap in shared memory
template <typename T>
__global__ void __launch_bounds__(kAlThreads) presence_kernel(const T* __restrict__ S, uint64_t n,
                                                              unsigned long long* __restrict__ bitmap) {
    constexpr uint32_t kLocalWords = sizeof(T) <= 2 ? (1u << (8 * sizeof(T))) / 64 : 1;
    __shared__ unsigned long long local[kLocalWords];
    if (sizeof(T) <= 2) {
        for (uint32_t i = threadIdx.x; i < kLocalWords; i += blockDim.x) local[i] = 0;
        __syncthreads();
    }
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = (uint32_t)S[k];
        const unsigned long long bit = 1ull << (v & 63);
        if (sizeof(T) <= 2) {
            if (!(local[v >> 6] & bit)) atomicOr(&local[v >> 6], bit);
        } else {
            if (!(*(volatile unsigned long long*)(bitmap + (v >> 6)) & bit)) atomicOr(bitmap + (v >> 6), bit);
        }
    }
    if (sizeof(T) <= 2) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < kLocalWords; i += blockDim.x)
            if (local[i]) atomicOr(bitmap + i, local[i]);
    }
}

// the number of present values: rank_1 at the end of the bitmap
// (S and out may be the same array: each thread reads its symbol before writing it)
template <typename T>
__global__ void __launch_bounds__(kAlThreads) remap_kernel(const LevelDesc lv, const T* S, T* out, uint64_t n) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x)
        out[k] = (T)rank1(lv, (uint64_t)S[k]);
}

__global__ void __launch_bounds__(kAlThreads) values_kernel(const LevelDesc lv, uint32_t* __restrict__ values,
                                                            uint64_t sigma) {
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < sigma;
         c += (uint64_t)gridDim.x * blockDim.x)
        values[c] = (uint32_t)select_b(lv, 1, c + 1, 12);  // kAlSampleK = 2^12
}

bool al_dev(const void* p) { return device_ptr_ok(p); }

template <typename T>
wt_status run_alphabet(const void* d_symbols, uint64_t n, void* d_out, uint32_t* d_values, uint32_t* h_sigma,
                       cudaStream_t s) {
    const uint64_t nbits = 1ull << (8 * sizeof(T));
    auto al = [](uint64_t x) { return (x + 255) & ~255ull; };
    const uint64_t nwords = (nbits / 512 + 1) * 8;  // whole 512-bit blocks plus one
    const uint64_t cap = nbits / kAlSampleK + 2;
    const uint64_t o_l1 = al(nwords * 8), o_l2 = o_l1 + al((nbits / 65536 + 1) * 8),
                   o_s0 = o_l2 + al((nbits / 512 + 1) * 2), o_s1 = o_s0 + al(cap * 8), o_st = o_s1 + al(cap * 8),
                   o_sig = o_st + 256, total = o_sig + 256;
    void* mem = nullptr;
    if (dev_alloc(&mem, total, s) != cudaSuccess) return WT_ENOMEM;
    uint8_t* M = static_cast<uint8_t*>(mem);
    uint64_t* words = reinterpret_cast<uint64_t*>(M);
    LevelDesc lv = {};
    lv.words = words;
    lv.l1 = reinterpret_cast<uint64_t*>(M + o_l1);
    lv.l2 = reinterpret_cast<uint16_t*>(M + o_l2);
    lv.s0 = reinterpret_cast<uint64_t*>(M + o_s0);
    lv.s1 = reinterpret_cast<uint64_t*>(M + o_s1);
    lv.size = nbits;
    uint32_t* status = reinterpret_cast<uint32_t*>(M + o_st);
    lv.status = status;
    wt_status st = WT_OK;
    uint64_t sigma = 0;
    if (cudaMemsetAsync(mem, 0, total, s) != cudaSuccess) st = WT_ECUDA;
    if (st == WT_OK && n) {
        const T* S = static_cast<const T*>(d_symbols);
        const int grid = sm_count() * 2;
        {
            ProfScope ps("alphabet_presence", s);
            presence_kernel<T><<<grid, kAlThreads, 0, s>>>(S, n, reinterpret_cast<unsigned long long*>(words));
        }
        // sigma = the ones of the presence bitmap, counted by the support kernel
        uint64_t* d_sigma = reinterpret_cast<uint64_t*>(M + o_sig);
        st = wt_bitvector_support_static(words, nbits, kAlSampleK, const_cast<uint64_t*>(lv.l1),
                                         const_cast<uint16_t*>(lv.l2), const_cast<uint64_t*>(lv.s0),
                                         const_cast<uint64_t*>(lv.s1), cap, status, d_sigma, s);
        if (st == WT_OK && cudaMemcpyAsync(&sigma, d_sigma, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            st = WT_ECUDA;
        if (st == WT_OK && cudaStreamSynchronize(s) != cudaSuccess) st = WT_ECUDA;
        if (st == WT_OK) {
            lv.ones = sigma;
            ProfScope ps("alphabet_remap", s);
            remap_kernel<T><<<grid * 2, kAlThreads, 0, s>>>(lv, S, static_cast<T*>(d_out), n);
            if (d_values && sigma)
                values_kernel<<<(unsigned)((sigma + kAlThreads - 1) / kAlThreads), kAlThreads, 0, s>>>(lv, d_values,
                                                                                                      sigma);
            if (cudaGetLastError() != cudaSuccess) st = WT_ECUDA;
        }
        uint32_t hst = 0;
        if (st == WT_OK && (cudaMemcpyAsync(&hst, status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                            cudaStreamSynchronize(s) != cudaSuccess))
            st = WT_ECUDA;
        if (st == WT_OK && (hst & kStTimeout)) st = WT_ETIMEOUT;
    }
    dev_free(mem, s);
    if (st == WT_OK) *h_sigma = (uint32_t)sigma;
    return st;
}

}  // namespace
}  // namespace wt

using namespace wt;

extern "C" wt_status wt_alphabet(const void* d_symbols, uint64_t n, uint32_t symbol_bytes, void* d_out,
                                 uint32_t* d_values, uint32_t* h_sigma, wt_stream stream) {
    if (!h_sigma || (symbol_bytes != 1 && symbol_bytes != 2 && symbol_bytes != 4)) return WT_EINVAL;
    if (n && (!al_dev(d_symbols) || !al_dev(d_out))) return WT_EINVAL;
    if (d_values && !al_dev(d_values)) return WT_EINVAL;
    if (!n) {
        *h_sigma = 0;
        return WT_OK;
    }
    switch (symbol_bytes) {
        case 1: return run_alphabet<uint8_t>(d_symbols, n, d_out, d_values, h_sigma, stream);
        case 2: return run_alphabet<uint16_t>(d_symbols, n, d_out, d_values, h_sigma, stream);
        default: return run_alphabet<uint32_t>(d_symbols, n, d_out, d_values, h_sigma, stream);
    }
}
