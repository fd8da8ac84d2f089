// rsort.cu -- sparse per-flow rate statistics: a least-significant-digit radix sort of a
// window's (key << 14 | bucket) log and the lower median of every key from the sorted log.
//
// The median of a key's eligible flows (Sec. III.B.2.1: the median rate from the counts of
// 10 kb/s buckets) needs the whole distribution of its buckets. A histogram per key
// (10,001 buckets) costs 40 KB per key and result slot; for registries of 10^5 sites that
// is 8 GB per slot. The sparse form keeps one 32-bit word per eligible flow instead and
// sorts it once, when the statistics are read: after the sort each key's buckets are one
// ascending run, so its lower median is the run's element ceil(n/2) - 1.
//
// Sort: 8-bit digits, one pass per digit of the significant bits; each pass is a per-CTA
// digit histogram over contiguous tiles, one exclusive scan of the (digit, CTA) counts, and
// a stable scatter (sub-tiles of 256 records in order; ranks within a warp from
// __match_any_sync, warps offset by the counts of the warps before them).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "gnm_internal.cuh"

namespace gnm {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr uint32_t kRsTile = 4096;  // least records per CTA and pass

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint32_t* __restrict__ in, uint32_t n, int shift,
                                                        uint32_t tile, uint32_t* __restrict__ hist, uint32_t G) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t b0 = (uint64_t)blockIdx.x * tile;
    const uint64_t b1 = b0 + tile < n ? b0 + tile : n;
    for (uint64_t i = b0 + threadIdx.x; i < b1; i += kRsThreads) atomicAdd(&h[(__ldg(in + i) >> shift) & 255u], 1u);
    __syncthreads();
    hist[(size_t)threadIdx.x * G + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of len counts in place (one CTA of 1024 threads, contiguous chunks).
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t* a, uint32_t len) {
    __shared__ uint32_t s[1024];
    const uint32_t t = threadIdx.x;
    const uint32_t per = (len + 1023u) / 1024u;
    const uint32_t b0 = min(t * per, len), b1 = min(b0 + per, len);
    uint32_t sum = 0;
    for (uint32_t i = b0; i < b1; ++i) sum += a[i];
    s[t] = sum;
    __syncthreads();
    for (uint32_t off = 1; off < 1024u; off <<= 1) {
        const uint32_t v = t >= off ? s[t - off] : 0u;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    uint32_t run = t ? s[t - 1] : 0u;
    for (uint32_t i = b0; i < b1; ++i) {
        const uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint32_t* __restrict__ in,
                                                           uint32_t* __restrict__ out, uint32_t n, int shift,
                                                           uint32_t tile, const uint32_t* __restrict__ hist,
                                                           uint32_t G) {
    __shared__ uint32_t run[256];             // next output position per digit
    __shared__ uint32_t wcnt[kRsWarps][256];  // per-warp digit counts, then offsets
    const uint32_t t = threadIdx.x, warp = t >> 5, lane = t & 31u;
    run[t] = hist[(size_t)t * G + blockIdx.x];
    const uint64_t b0 = (uint64_t)blockIdx.x * tile;
    const uint64_t b1 = b0 + tile < n ? b0 + tile : n;
    for (uint64_t base = b0; base < b1; base += kRsThreads) {
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) wcnt[w][t] = 0;
        __syncthreads();
        const uint64_t i = base + t;
        const bool valid = i < b1;
        const uint32_t x = valid ? __ldg(in + i) : 0u;
        const uint32_t d = valid ? (x >> shift) & 255u : 256u + lane;  // tail lanes: groups of their own
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == (uint32_t)__popc(peers) - 1u) wcnt[warp][d] = (uint32_t)__popc(peers);
        __syncthreads();
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) {
            const uint32_t c = wcnt[w][t];
            wcnt[w][t] = tot;
            tot += c;
        }
        __syncthreads();
        if (valid) out[run[d] + wcnt[warp][d] + rank] = x;
        __syncthreads();
        run[t] += tot;
    }
}

// Lower median of every key from the sorted log: key k's run is [lb(k << 14), lb((k+1) << 14)).
__device__ __forceinline__ uint32_t lower_bound64(const uint32_t* __restrict__ a, uint32_t n, uint64_t v) {
    uint32_t lo = 0, len = n;
    while (len > 0) {
        const uint32_t half = len >> 1;
        if ((uint64_t)__ldg(a + lo + half) < v) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo;
}

__global__ void k_sparse_median(const uint32_t* __restrict__ sorted, uint32_t n, uint32_t n_keys,
                                uint32_t* __restrict__ med, uint32_t* __restrict__ count) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_keys) return;
    const uint32_t a = lower_bound64(sorted, n, (uint64_t)k << 14);
    const uint32_t b = lower_bound64(sorted, n, (uint64_t)(k + 1) << 14);
    const uint32_t c = b - a;
    count[k] = c;
    med[k] = c ? (__ldg(sorted + a + (c + 1u) / 2u - 1u) & 0x3FFFu) : GNM_NO_MEDIAN;
}

}  // namespace

size_t radix_sort_hist_words(uint32_t n, int sms) {
    const uint32_t G = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(1, ((uint64_t)n + kRsTile - 1) / kRsTile),
                                                    (uint64_t)sms * 4);
    return (size_t)G * 256;
}

cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* tmp, uint32_t n, int bits, uint32_t* hist, int sms,
                           cudaStream_t st, uint32_t** result) {
    *result = keys;
    if (n <= 1) return cudaSuccess;
    const uint32_t G = (uint32_t)(radix_sort_hist_words(n, sms) / 256);
    uint32_t tile = (uint32_t)(((uint64_t)n + G - 1) / G);
    tile = (tile + kRsThreads - 1) / kRsThreads * kRsThreads;
    const uint32_t grid = (uint32_t)(((uint64_t)n + tile - 1) / tile);
    uint32_t* src = keys;
    uint32_t* dst = tmp;
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<<<grid, kRsThreads, 0, st>>>(src, n, shift, tile, hist, grid);
        k_rs_scan<<<1, 1024, 0, st>>>(hist, grid * 256u);
        k_rs_scatter<<<grid, kRsThreads, 0, st>>>(src, dst, n, shift, tile, hist, grid);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        std::swap(src, dst);
    }
    *result = src;
    return cudaSuccess;
}

cudaError_t launch_sparse_median(const uint32_t* sorted, uint32_t n, uint32_t n_keys, uint32_t* med, uint32_t* count,
                                 cudaStream_t st) {
    if (n_keys == 0) return cudaSuccess;
    k_sparse_median<<<(n_keys + 255) / 256, 256, 0, st>>>(sorted, n, n_keys, med, count);
    return cudaGetLastError();
}

}  // namespace gnm
