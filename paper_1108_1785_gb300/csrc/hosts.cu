// hosts.cu -- per-host sums (Sec. III.B.2.1: statistics "for each host in a registered
// site"). After the key kernel of a split launch, every record of a registered site adds
// its six sums to the entry of its (remote host, dir) in its window's host table: open
// addressing with linear probing, entries claimed by a 64-bit compare-and-swap, sums by
// 64-bit atomic adds (integer sums: exact in any order).
#include <cuda_runtime.h>

#include "agg_kernel.cuh"  // (rate_of_sums)
#include "gnm_internal.cuh"

namespace gnm {
namespace {

constexpr uint32_t kHostThreads = 512;

// Mix of a 64-bit host key (finaliser of a 64-bit hash: xor-shift, multiply, xor-shift).
__device__ __forceinline__ uint64_t mix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xFF51AFD7ED558CCDull;
    k ^= k >> 33;
    k *= 0xC4CEB9FE1A85EC53ull;
    k ^= k >> 33;
    return k;
}

__device__ __forceinline__ uint32_t first_win(const WinDesc* w, uint32_t n, uint64_t lo) {
    uint32_t a = 0, b = n;
    while (a < b) {
        const uint32_t m = (a + b) >> 1;
        if (w[m].end > lo) b = m;
        else a = m + 1;
    }
    return a;
}

// Records [blockIdx.x * chunk, +chunk), window segment by window segment.
__global__ void __launch_bounds__(kHostThreads)
    k_host_stats(const __grid_constant__ AggParams p, const uint32_t* __restrict__ keys, uint64_t chunk) {
    const uint64_t lo = min((uint64_t)blockIdx.x * chunk, p.n_total);
    const uint64_t hi = min(lo + chunk, p.n_total);
    const uint32_t nk = 2u * p.n_sites, mask = p.hcap - 1u;
    for (uint32_t w = first_win(p.wins, p.n_wins, lo); w < p.n_wins; ++w) {
        const WinDesc wd = p.wins[w];
        if (wd.begin >= hi) break;
        unsigned long long* tk = p.hkeys + (size_t)wd.slot * p.hcap;
        unsigned long long* tr = p.hrows + (size_t)wd.slot * p.hcap * kNStat;
        const uint64_t e0 = min(wd.end, hi);
        for (uint64_t i = max(wd.begin, lo) + threadIdx.x; i < e0; i += blockDim.x) {
            const uint32_t key = __ldg(keys + i);
            if (key >= nk) continue;  // unmatched classes have no host
            const uint32_t dir = key & 1u;
            const uint32_t remote = dir ? __ldg(p.dst + i) : __ldg(p.src + i);  // outbound: destination
            const unsigned long long hk = ((((unsigned long long)remote) << 1) | dir) + 1ull;
            uint32_t h = (uint32_t)mix64(hk) & mask;
            uint32_t probes = 0;
            bool found = false;
            while (probes <= mask) {
                unsigned long long cur = __ldcg(tk + h);
                if (cur == 0ull) cur = atomicCAS(tk + h, 0ull, hk);
                if (cur == 0ull || cur == hk) {
                    found = true;
                    break;
                }
                h = (h + 1u) & mask;
                ++probes;
            }
            if (!found) {  // the table is full: count the record's host as lost
                atomicAdd(p.hover + wd.slot, 1u);
                continue;
            }
            const uint32_t pk = __ldg(p.pkts + i), oc = __ldg(p.oct + i);
            const uint32_t dur = __ldg(p.last + i) - __ldg(p.first + i);  // modulo 2^32
            const bool ack_ok = (uint64_t)oc >= (uint64_t)p.min_avg * (uint64_t)pk;
            const bool many = pk >= p.min_pkts, longd = dur >= p.min_dur;
            const bool admin_ok = p.admin_rule == GNM_ADMIN_OR ? (many && longd) : (many || longd);
            unsigned long long* r = tr + (size_t)h * kNStat;
            atomicAdd(r + 0, 1ull);
            atomicAdd(r + 1, (unsigned long long)oc);
            atomicAdd(r + 2, (unsigned long long)pk);
            if (dur != 0u && ack_ok && admin_ok) {
                atomicAdd(r + 3, 1ull);
                atomicAdd(r + 4, (unsigned long long)oc);
                atomicAdd(r + 5, (unsigned long long)dur);
            }
        }
    }
}

// Rate of every host entry (as the per-site rate: octets * 8 bits / (ms / 1000), one
// rounding per operation, formed on the integer units; NaN without eligible duration).
__global__ void k_host_rates(const unsigned long long* __restrict__ rows, uint32_t n, double* __restrict__ rate) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += stride)
        rate[h] = dev::rate_of_sums(rows[(size_t)h * kNStat + 4], rows[(size_t)h * kNStat + 5]);
}

}  // namespace

cudaError_t launch_host_rates(const unsigned long long* rows, uint32_t n, double* rate, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const uint32_t blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    (void)cudaGetLastError();
    k_host_rates<<<blocks, 256, 0, st>>>(rows, n, rate);
    return cudaGetLastError();
}

cudaError_t launch_host_stats(const AggParams& p, const uint32_t* keys, int grid, cudaStream_t st) {
    if (p.n_total == 0 || grid <= 0) return cudaSuccess;
    const uint64_t chunk = (p.n_total + grid - 1) / grid;
    (void)cudaGetLastError();
    k_host_stats<<<grid, kHostThreads, 0, st>>>(p, keys, chunk);
    return cudaGetLastError();
}

}  // namespace gnm
