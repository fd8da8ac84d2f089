// kernels_misc.cu -- dispatch of the aggregation variants, and the small kernels around
// it: stand-alone finalisation (rates, flags), flag compaction and batch lookups.
#include "agg_kernel.cuh"

namespace gnm {

cudaError_t launch_aggregate_l2(const AggParams& p, const LaunchShape& s, cudaStream_t st);
cudaError_t launch_aggregate_smem(const AggParams& p, const LaunchShape& s, cudaStream_t st);
cudaError_t launch_aggregate_rmi(const AggParams& p, const LaunchShape& s, cudaStream_t st);
cudaError_t launch_aggregate_staged(const AggParams& p, const LaunchShape& s, cudaStream_t st);
cudaError_t launch_aggregate_radix(const AggParams& p, const LaunchShape& s, cudaStream_t st);
cudaError_t launch_aggregate_keys(const AggParams& p, const LaunchShape& s, cudaStream_t st);
cudaError_t launch_keys_l2(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st);
cudaError_t launch_keys_smem(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st);
cudaError_t launch_keys_rmi(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st);
cudaError_t launch_keys_staged(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st);
cudaError_t launch_keys_radix(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st);
cudaError_t launch_keys_radixblk(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st);
cudaError_t launch_keys_radixblk2(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st);
cudaError_t launch_keys_radixblk2h(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st);
cudaError_t launch_keys_hash24(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st);
cudaError_t launch_aggregate_hash24(const AggParams& p, const LaunchShape& s, cudaStream_t st);

cudaError_t launch_keys(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st) {
    switch (s.lookup) {
        case kLookupSmem: return launch_keys_smem(p, s, keys, st);
        case kLookupRmi: return launch_keys_rmi(p, s, keys, st);
        case kLookupStaged: return launch_keys_staged(p, s, keys, st);
        case kLookupHash24: return launch_keys_hash24(p, s, keys, st);
        case kLookupRadix:
            return s.keys_h16        ? launch_keys_radixblk2h(p, s, keys, st)
                   : s.keys_blk == 2 ? launch_keys_radixblk2(p, s, keys, st)
                   : s.keys_blk == 4 ? launch_keys_radixblk(p, s, keys, st)
                                     : launch_keys_radix(p, s, keys, st);
        default: return launch_keys_l2(p, s, keys, st);
    }
}

cudaError_t launch_aggregate(const AggParams& p, const LaunchShape& s, cudaStream_t st) {
    if (s.split) return launch_aggregate_keys(p, s, st);
    switch (s.lookup) {
        case kLookupSmem: return launch_aggregate_smem(p, s, st);
        case kLookupRmi: return launch_aggregate_rmi(p, s, st);
        case kLookupStaged: return launch_aggregate_staged(p, s, st);
        case kLookupRadix: return launch_aggregate_radix(p, s, st);
        case kLookupHash24: return launch_aggregate_hash24(p, s, st);
        default: return launch_aggregate_l2(p, s, st);
    }
}

size_t aggregate_smem_bytes(int lookup, int table, uint32_t n_ranges, uint32_t keys,
                            uint32_t table_cap, uint32_t n_models, uint32_t radix_bits) {
    size_t a, b;
    return dev::smem_layout(lookup, table, n_ranges, keys, table_cap, n_models, radix_bits, &a, &b);
}

namespace {

__global__ void k_finalize(const __grid_constant__ AggParams p, uint32_t slot) {
    dev::finalize_rows<true>(p, slot, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// blockIdx.y: window of the launch; its keys are spread over blockIdx.x.
constexpr uint32_t kFinKeys = 256;

__global__ void __launch_bounds__(kFinKeys, 4) k_finalize_windows(const __grid_constant__ AggParams p) {
    __shared__ __align__(16) uint64_t stage[kFinKeys * kNStat];  // per warp: 32 keys' stats rows
    const WinDesc wd = p.wins[blockIdx.y];
    const uint32_t* parts =
        p.partials ? p.partials + (size_t)wd.part_base * part_stride_words(p.table_rows) : nullptr;
    const bool in_area = !p.partials || p.part_groups ||
                         chk(p.check_err,
                             ((uint64_t)wd.part_base + wd.n_parts) * part_stride_words(p.table_rows) <= p.partial_cap,
                             kChkPartial, wd.part_base);
    dev::finalize_rows<true>(p, wd.slot, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, parts,
                             p.partials && in_area ? wd.n_parts : 0u, blockIdx.y,
                             stage + (threadIdx.x & ~31u) * kNStat);
}

// One warp per key: the key's eligible flows (the histogram's total) and the bucket where
// the running count first reaches ceil(n/2) -- the bucket of the lower median.
constexpr uint32_t kMedWarps = 8;

__global__ void __launch_bounds__(kMedWarps * 32) k_rate_median(const uint32_t* __restrict__ hist, uint32_t n_keys,
                                                                uint32_t* __restrict__ med,
                                                                uint32_t* __restrict__ count) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t k = blockIdx.x * kMedWarps + (threadIdx.x >> 5);
    if (k >= n_keys) return;  // whole warps leave together
    const uint32_t* h = hist + (size_t)k * kRateBuckets;
    uint32_t total = 0;
    for (uint32_t b = lane; b < kRateBuckets; b += 32u) total += __ldg(h + b);
    total = __reduce_add_sync(0xFFFFFFFFu, total);
    uint32_t m = GNM_NO_MEDIAN;
    if (total) {
        const uint32_t want = (uint32_t)(((uint64_t)total + 1u) / 2u);
        uint32_t base = 0;  // flows in the buckets before this round's 32
        for (uint32_t b0 = 0; b0 < kRateBuckets; b0 += 32u) {
            const uint32_t b = b0 + lane;
            const uint32_t v = b < kRateBuckets ? __ldg(h + b) : 0u;
            uint32_t incl = v;  // inclusive scan over the warp
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
                if ((int)lane >= d) incl += y;
            }
            const unsigned hit = __ballot_sync(0xFFFFFFFFu, base + incl >= want);
            if (hit) {
                m = b0 + (uint32_t)(__ffs(hit) - 1);
                break;
            }
            base += __shfl_sync(0xFFFFFFFFu, incl, 31);
        }
    }
    if (lane == 0) {
        med[k] = m;
        count[k] = total;
    }
}

__global__ void k_warn_runs(const uint32_t* __restrict__ med, uint32_t n_keys, uint32_t below,
                            uint32_t consecutive, uint32_t* __restrict__ run, uint32_t* __restrict__ out,
                            uint32_t* __restrict__ n) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n_keys; k += stride) {
        const uint32_t m = med[k];
        const uint32_t r = (m != GNM_NO_MEDIAN && m < below) ? run[k] + 1u : 0u;
        run[k] = r;
        if (r >= consecutive) out[atomicAdd(n, 1u)] = k;
    }
}

// Keys (site*2+dir) whose eligible flows reach min_flows and whose rate is strictly
// below thr (Sec. III.B.1; Sec. IV.B "less than"); order is restored on the host.
__global__ void k_flag_compact(const double* __restrict__ rate, const uint64_t* __restrict__ stats,
                               uint32_t n_site_keys, double thr, uint32_t min_flows,
                               uint32_t* __restrict__ out, uint32_t* __restrict__ count) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n_site_keys; k += stride) {
        const uint64_t ef = stats[(size_t)k * kNStat + 3];
        if (ef >= (uint64_t)min_flows && rate[k] < thr) out[atomicAdd(count, 1u)] = k;
    }
}

template <int LOOKUP>
__global__ void k_lookup(const __grid_constant__ AggParams p, const uint32_t* __restrict__ addr,
                         uint64_t n, uint32_t* __restrict__ site_out, uint32_t* __restrict__ pos_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t* s_starts = nullptr;
    const float *ra = nullptr, *rb = nullptr;
    const uint32_t *rx0 = nullptr, *reps = nullptr;
    if (LOOKUP == kLookupSmem) {
        uint32_t* st = reinterpret_cast<uint32_t*>(smem_raw);
        for (uint32_t i = threadIdx.x; i < p.n_ranges; i += blockDim.x) st[i] = __ldg(p.starts + i);
        s_starts = st;
    }
    if (LOOKUP == kLookupStaged) {
        uint32_t* st = reinterpret_cast<uint32_t*>(smem_raw);
        for (uint32_t i = threadIdx.x; i < p.n_blocks; i += blockDim.x) st[i] = __ldg(p.sample + i);
        s_starts = st;
    }
    if (LOOKUP == kLookupRadix) {
        uint32_t* d = reinterpret_cast<uint32_t*>(smem_raw);
        const uint32_t nd = 1u << p.radix_bits, sh = 16u - p.radix_bits;
        for (uint32_t i = threadIdx.x; i <= nd; i += blockDim.x) d[i] = __ldg(p.dir16 + ((size_t)i << sh));
        s_starts = d;
    }
    if (LOOKUP == kLookupRmi && !p.rmi.leaves_global) {
        const uint32_t L = p.rmi.n_models;
        float* a = reinterpret_cast<float*>(smem_raw);
        float* b = a + L;
        uint32_t* x0 = reinterpret_cast<uint32_t*>(b + L);
        uint32_t* e = x0 + L;
        for (uint32_t i = threadIdx.x; i < L; i += blockDim.x) {
            a[i] = __ldg(p.rmi.a + i);
            b[i] = __ldg(p.rmi.b + i);
            x0[i] = __ldg(p.rmi.x0 + i);
            e[i] = __ldg(p.rmi.eps + i);
        }
        ra = a; rb = b; rx0 = x0; reps = e;
    }
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t x = __ldg(addr + i);
        uint32_t idx;
        if (LOOKUP == kLookupHash24) {  // the /24 table has sites, not range positions
            uint32_t xs[1] = {x}, st[1];
            dev::hash24_sites<1>(p.h24, p.h24_mask, xs, st);
            if (site_out) site_out[i] = st[0];
            continue;
        }
        if (LOOKUP == kLookupRmi) {
            idx = dev::rmi_lookup(p.rmi, ra, rb, rx0, reps, p.starts, p.n_ranges, x, p.violations);
        } else if (LOOKUP == kLookupRadix) {
            uint32_t xs[1] = {x}, b[1];
            dev::radix_search<1>(s_starts, p.radix_bits, p.starts, xs, b, p.n_ranges, p.check_err);
            idx = b[0];
        } else if (LOOKUP == kLookupStaged) {
            uint32_t xs[1] = {x}, b[1];
            dev::pred_search<1, true>(s_starts, p.n_blocks, xs, b);
            idx = dev::staged_block_pos(p.blocks + 4 * (size_t)b[0], b[0], x, p.n_ranges);
        } else {
            uint32_t xs[1] = {x}, b[1];
            if (LOOKUP == kLookupSmem) dev::pred_search<1, true>(s_starts, p.n_ranges, xs, b);
            else dev::pred_search<1, false>(p.starts, p.n_ranges, xs, b);
            idx = b[0];
        }
        if (pos_out) pos_out[i] = idx;
        if (site_out) site_out[i] = __ldg(p.rsite + idx);
    }
}

}  // namespace

cudaError_t launch_finalize(const AggParams& p, uint32_t slot, cudaStream_t st) {
    const uint32_t blocks = (p.keys + 255) / 256;
    (void)cudaGetLastError();
    k_finalize<<<blocks > 4096 ? 4096 : blocks, 256, 0, st>>>(p, slot);
    return cudaGetLastError();
}

cudaError_t launch_finalize_windows(const AggParams& p, cudaStream_t st) {
    if (p.n_wins == 0) return cudaSuccess;
    // key blocks per window: all of them, up to one wave of resident CTAs over the windows
    // (the threads then loop over their keys, so that the warps of an SM are in different
    // phases -- loads, FP64 rates, stores -- instead of moving through waves in step)
    static int resident[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int res = dev < 64 ? resident[dev] : 0;
    if (res == 0) {
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_finalize_windows, kFinKeys, 0);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        res = std::max(1, per_sm * sms);
        if (dev < 64) resident[dev] = res;
    }
    const uint32_t bx = (p.keys + kFinKeys - 1) / kFinKeys;
    const uint32_t cap = std::max<uint32_t>(1u, (uint32_t)res / p.n_wins);
    (void)cudaGetLastError();
    k_finalize_windows<<<dim3(std::min(bx, cap), p.n_wins), kFinKeys, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_warn_runs(const uint32_t* med, uint32_t n_keys, uint32_t below, uint32_t consecutive,
                             uint32_t* run, uint32_t* out, uint32_t* n, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(n, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess || n_keys == 0) return e;
    const uint32_t blocks = std::min<uint32_t>((n_keys + 255) / 256, 4096);
    (void)cudaGetLastError();
    k_warn_runs<<<blocks, 256, 0, st>>>(med, n_keys, below, consecutive, run, out, n);
    return cudaGetLastError();
}

cudaError_t launch_rate_median(const uint32_t* hist, uint32_t n_keys, uint32_t* med, uint32_t* count,
                               cudaStream_t st) {
    if (n_keys == 0) return cudaSuccess;
    (void)cudaGetLastError();
    k_rate_median<<<(n_keys + kMedWarps - 1) / kMedWarps, kMedWarps * 32, 0, st>>>(hist, n_keys, med, count);
    return cudaGetLastError();
}

cudaError_t launch_flag_compact(const double* rate, const uint64_t* stats, uint32_t n_site_keys,
                                double thr, uint32_t min_flows, uint32_t* out_keys,
                                uint32_t* out_count, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out_count, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    uint32_t blocks = (n_site_keys + 255) / 256;
    if (blocks == 0) blocks = 1;
    if (blocks > 4096) blocks = 4096;
    k_flag_compact<<<blocks, 256, 0, st>>>(rate, stats, n_site_keys, thr, min_flows, out_keys, out_count);
    return cudaGetLastError();
}

namespace {
__global__ void k_rates(const uint64_t* __restrict__ eo, const uint64_t* __restrict__ ed, uint64_t n,
                        double* __restrict__ rate) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        rate[i] = dev::rate_of_sums(__ldg(eo + i), __ldg(ed + i));
}
}  // namespace

cudaError_t launch_rates(const uint64_t* e_octets, const uint64_t* e_dur_ms, uint64_t n, double* rate,
                         cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (n + 255) / 256, cap = (uint64_t)(sms > 0 ? sms : 1) * 8;
    k_rates<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(e_octets, e_dur_ms, n, rate);
    return cudaGetLastError();
}

cudaError_t launch_lookup(const AggParams& p, int lookup, const uint32_t* addr, uint64_t n,
                          uint32_t* site_out, uint32_t* pos_out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (n + 255) / 256;
    const int blocks = (int)(want < (uint64_t)sms * 8 ? want : (uint64_t)sms * 8);
    size_t smem = 0;
    (void)cudaGetLastError();  // report this launch's error only
    if (lookup == kLookupSmem) smem = (size_t)p.n_ranges * 4;
    if (lookup == kLookupStaged) smem = (size_t)p.n_blocks * 4;
    if (lookup == kLookupRadix) smem = ((size_t)1 << p.radix_bits) * 4 + 4;
    if (lookup == kLookupRmi) smem = p.rmi.leaves_global ? 0 : (size_t)p.rmi.n_models * 16;
    cudaError_t e;
    switch (lookup) {
        case kLookupSmem:
            e = cudaFuncSetAttribute(k_lookup<kLookupSmem>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            k_lookup<kLookupSmem><<<blocks, 256, smem, st>>>(p, addr, n, site_out, pos_out);
            break;
        case kLookupRmi:
            e = cudaFuncSetAttribute(k_lookup<kLookupRmi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            k_lookup<kLookupRmi><<<blocks, 256, smem, st>>>(p, addr, n, site_out, pos_out);
            break;
        case kLookupHash24:
            k_lookup<kLookupHash24><<<blocks, 256, 0, st>>>(p, addr, n, site_out, pos_out);
            break;
        case kLookupStaged:
            e = cudaFuncSetAttribute(k_lookup<kLookupStaged>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            k_lookup<kLookupStaged><<<blocks, 256, smem, st>>>(p, addr, n, site_out, pos_out);
            break;
        case kLookupRadix:
            e = cudaFuncSetAttribute(k_lookup<kLookupRadix>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            k_lookup<kLookupRadix><<<blocks, 256, smem, st>>>(p, addr, n, site_out, pos_out);
            break;
        default:
            k_lookup<kLookupL2><<<blocks, 256, 0, st>>>(p, addr, n, site_out, pos_out);
    }
    return cudaGetLastError();
}

namespace {
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);
std::once_flag g_ctx_once;
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
}  // namespace

unsigned long long current_context_id() {
    std::call_once(g_ctx_once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_id = reinterpret_cast<CtxGetIdFn>(f);
        (void)cudaGetLastError();
    });
    if (!g_ctx_current || !g_ctx_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != 0 || !ctx || g_ctx_id(ctx, &id) != 0) return 0;
    return id;
}

cudaError_t ensure_smem_optin(const void* fn, int bytes, OptInCache& cache) {
    if (bytes < 46 * 1024) return cudaSuccess;  // within the default 48 KB
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(cache.mu);
    if (dev < 64 && ctx != 0 && cache.ctx[dev] == ctx && cache.bytes[dev] >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    if (dev < 64) {
        if (cache.ctx[dev] != ctx) cache.bytes[dev] = 0;
        cache.ctx[dev] = ctx;
        cache.bytes[dev] = bytes > cache.bytes[dev] ? bytes : cache.bytes[dev];
    }
    return cudaSuccess;
}

}  // namespace gnm
