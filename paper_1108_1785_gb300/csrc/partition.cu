// partition.cu -- regrouping of a launch's records by (window, key group) before the
// aggregation, for key spaces larger than one CTA's direct shared-memory table.
//
// A key group is `part_rows` consecutive keys: as many as one CTA's direct table holds.
// After the regrouping every segment the aggregation kernel meets holds the keys of one
// group only, so a direct table serves it with neither a cache nor global atomics. The
// per-key sums do not depend on the order of the records, so the order the scatter
// produces is free and the results stay exact.
//
// Three kernels, all on the launch's stream:
//   k_part_count    per-CTA histogram of the buckets (window * groups + group) -> counts
//   k_part_scan     one CTA: bucket starts (in place of the counts), the aggregation's
//                   segment descriptors and the finalisation's partial-block ranges
//   k_part_scatter  tiles sorted by group in shared memory, one place reservation per
//                   (tile, group), coalesced runs out
#include <cuda_runtime.h>

#include "gnm_internal.cuh"

namespace gnm {
namespace {

constexpr uint32_t kPartThreads = 1024;
constexpr uint32_t kScanThreads = 1024;
constexpr uint32_t kScanPer = kPartMaxBuckets / kScanThreads;  // buckets per scan thread

// First window (descriptor) whose end lies above record lo.
__device__ __forceinline__ uint32_t first_win(const WinDesc* w, uint32_t n, uint64_t lo) {
    uint32_t a = 0, b = n;
    while (a < b) {
        const uint32_t m = (a + b) >> 1;
        if (w[m].end > lo) b = m;
        else a = m + 1;
    }
    return a;
}

// Bucket sizes: records [blockIdx.x * chunk, +chunk) of the launch, window segment by
// window segment, counted per (window, key group) in shared memory. p.src holds each
// record's key (written by the key kernel).
__global__ void __launch_bounds__(kPartThreads)
    k_part_count(const __grid_constant__ AggParams p, uint64_t chunk, uint32_t rows, uint32_t groups,
                 uint32_t* __restrict__ cnt) {
    extern __shared__ uint32_t hist[];
    const uint32_t nb = p.n_wins * groups;
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    const uint64_t lo = min((uint64_t)blockIdx.x * chunk, p.n_total);
    const uint64_t hi = min(lo + chunk, p.n_total);
    for (uint32_t w = first_win(p.wins, p.n_wins, lo); w < p.n_wins; ++w) {
        const WinDesc wd = p.wins[w];
        if (wd.begin >= hi) break;
        const uint64_t e0 = min(wd.end, hi);
        // four keys per thread and step, their loads in flight together
        for (uint64_t i = max(wd.begin, lo) + threadIdx.x; i < e0; i += 4u * blockDim.x) {
            uint32_t k[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint64_t j = i + (uint64_t)u * blockDim.x;
                k[u] = j < e0 ? __ldcs(p.src + j) : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i + (uint64_t)u * blockDim.x < e0 && chk(p.check_err, k[u] / rows < groups, kChkBucket, k[u]))
                    atomicAdd(&hist[w * groups + k[u] / rows], 1u);
        }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x)
        if (hist[b]) atomicAdd(cnt + b, hist[b]);
}

// Exclusive prefix sum of v[0..n) into out[0..n) by the whole CTA (tmp: kPartThreads words);
// up to 32 values (the usual number of key groups) take one warp's shuffles.
__device__ __forceinline__ void cta_exclusive_scan(const uint32_t* v, uint32_t* out, uint32_t n, uint32_t* tmp) {
    const uint32_t t = threadIdx.x;
    if (n <= 32u) {
        if (t < 32u) {
            const uint32_t x = t < n ? v[t] : 0u;
            uint32_t incl = x;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
                if ((int)t >= d) incl += y;
            }
            if (t < n) out[t] = incl - x;
        }
        __syncthreads();
        return;
    }
    const uint32_t per = (n + kPartThreads - 1) / kPartThreads;
    const uint32_t a = min(t * per, n), b = min(a + per, n);
    uint32_t sum = 0;
    for (uint32_t i = a; i < b; ++i) sum += v[i];
    tmp[t] = sum;
    __syncthreads();
    for (uint32_t d = 1; d < kPartThreads; d <<= 1) {  // Hillis-Steele over the CTA
        const uint32_t add = t >= d ? tmp[t - d] : 0u;
        __syncthreads();
        tmp[t] += add;
        __syncthreads();
    }
    uint32_t run = tmp[t] - sum;
    for (uint32_t i = a; i < b; ++i) {
        out[i] = run;
        run += v[i];
    }
    __syncthreads();
}

// The regrouping itself, tile by tile (kTile records of one window): the tile is sorted by
// key group in shared memory, each group's run of the tile takes its place in the bucket
// with one atomic on cnt (the bucket's next free place), and the runs go out with
// coalesced stores. out: 4 arrays of `stride` words (key within its group, pkts, octets,
// duration = last - first mod 2^32, the only use of the two times). Any split of the
// records into CTAs works: places are reserved per tile.
constexpr uint32_t kTile = 4 * kPartThreads;
constexpr int kTileRecs = (int)(kTile / kPartThreads);  // records per thread and tile

__global__ void __launch_bounds__(kPartThreads)
    k_part_scatter(const __grid_constant__ AggParams p, uint64_t chunk, uint32_t rows, uint32_t groups,
                   uint32_t* __restrict__ cnt, uint32_t* __restrict__ out, uint64_t stride) {
    extern __shared__ __align__(16) uint32_t sh[];
    __shared__ uint32_t tmp[kPartThreads];
    uint32_t* s_rec = sh;                 // [4][kTile] the tile in group order
    uint32_t* s_grp = sh + 4 * kTile;     // [kTile] group of each placed record
    uint32_t* hist = s_grp + kTile;       // [groups] records of the tile per group
    uint32_t* toff = hist + groups;       // [groups] first place of each group in the tile
    uint32_t* gpos = toff + groups;       // [groups] first place of each group's run in its bucket
    uint32_t* o[4] = {out, out + stride, out + 2 * stride, out + 3 * stride};
    const uint32_t tid = threadIdx.x;
    const uint64_t lo = min((uint64_t)blockIdx.x * chunk, p.n_total);
    const uint64_t hi = min(lo + chunk, p.n_total);
    for (uint32_t w = first_win(p.wins, p.n_wins, lo); w < p.n_wins; ++w) {
        const WinDesc wd = p.wins[w];
        if (wd.begin >= hi) break;
        const uint64_t e0 = min(wd.end, hi);
        // a tile's fields are in registers before it is sorted; the next tile of the segment
        // is loaded while this one goes out, so its memory latency overlaps the stores
        uint32_t v[4][kTileRecs];
        auto load = [&](uint64_t t0) {
            const uint32_t n = (uint32_t)min((uint64_t)kTile, e0 - t0);
#pragma unroll
            for (int u = 0; u < kTileRecs; ++u) {
                const uint32_t j = tid + u * kPartThreads;
                const bool ok = j < n;
                const uint64_t i = t0 + (ok ? j : 0u);
                v[0][u] = ok ? __ldcs(p.src + i) : 0u;
                v[1][u] = ok ? __ldcs(p.pkts + i) : 0u;
                v[2][u] = ok ? __ldcs(p.oct + i) : 0u;
                v[3][u] = ok ? __ldcs(p.last + i) - __ldcs(p.first + i) : 0u;  // duration
            }
        };
        if (max(wd.begin, lo) < e0) load(max(wd.begin, lo));
        for (uint64_t t0 = max(wd.begin, lo); t0 < e0; t0 += kTile) {
            const uint32_t n = (uint32_t)min((uint64_t)kTile, e0 - t0);
            for (uint32_t g = tid; g < groups; g += kPartThreads) hist[g] = 0u;
            __syncthreads();
            uint32_t grp[kTileRecs], rk[kTileRecs];
            bool in[kTileRecs];
#pragma unroll
            for (int u = 0; u < kTileRecs; ++u) {
                const uint32_t j = tid + u * kPartThreads;
                grp[u] = v[0][u] / rows;
                // (checked build: a key beyond the groups is left out here as in the count)
                in[u] = j < n && (GNM_CHECKED == 0 || grp[u] < groups);
                rk[u] = in[u] ? atomicAdd(&hist[grp[u]], 1u) : 0u;
            }
            __syncthreads();
            cta_exclusive_scan(hist, toff, groups, tmp);
            for (uint32_t g = tid; g < groups; g += kPartThreads)
                gpos[g] = hist[g] ? atomicAdd(cnt + w * groups + g, hist[g]) : 0u;
            uint32_t placed = n;  // records of the tile that are placed
#if GNM_CHECKED
            placed = 0;
            for (uint32_t g = 0; g < groups; ++g) placed += hist[g];
#endif
#pragma unroll
            for (int u = 0; u < kTileRecs; ++u) {
                if (in[u]) {
                    const uint32_t pos = toff[grp[u]] + rk[u];
                    s_rec[pos] = v[0][u] - grp[u] * rows;
#pragma unroll
                    for (int f = 1; f < 4; ++f) s_rec[f * kTile + pos] = v[f][u];
                    s_grp[pos] = grp[u];
                }
            }
            __syncthreads();
            if (t0 + kTile < e0) load(t0 + kTile);
            for (uint32_t j = tid; j < placed; j += kPartThreads) {
                const uint32_t g = s_grp[j];
                const uint32_t r = gpos[g] + (j - toff[g]);
                if (!chk(p.check_err, r < stride, kChkPosition, r)) continue;
#pragma unroll
                for (int f = 0; f < 4; ++f) o[f][r] = s_rec[f * kTile + j];
            }
            __syncthreads();
        }
    }
}

// Exclusive prefix sum over the CTA of one value per thread; the total goes to *total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s, uint32_t* total) {
    const uint32_t t = threadIdx.x;
    s[t] = v;
    __syncthreads();
    for (uint32_t d = 1; d < kScanThreads; d <<= 1) {  // Hillis-Steele over the CTA
        const uint32_t add = t >= d ? s[t - d] : 0u;
        __syncthreads();
        s[t] += add;
        __syncthreads();
    }
    const uint32_t incl = s[t];
    *total = s[kScanThreads - 1];
    __syncthreads();
    return incl - v;
}

// One CTA. cnt[b] (bucket sizes) becomes the bucket's first place; descs receives the
// non-empty buckets as aggregation segments (in bucket order, so ascending begin), then
// empty descriptors at the end of the records; part_desc[b] = (first partial block, blocks).
__global__ void __launch_bounds__(kScanThreads)
    k_part_scan(const __grid_constant__ AggParams p, uint32_t rows, uint32_t groups, uint64_t agg_chunk,
                uint32_t* __restrict__ cnt, WinDesc* __restrict__ descs, uint2* __restrict__ part_desc) {
    __shared__ uint32_t s[kScanThreads];
    const uint32_t nb = p.n_wins * groups, t = threadIdx.x;
    const uint32_t b0 = t * kScanPer;
    uint32_t c[kScanPer], ctas[kScanPer];
    uint32_t sum = 0;
#pragma unroll
    for (uint32_t j = 0; j < kScanPer; ++j) {
        c[j] = b0 + j < nb ? cnt[b0 + j] : 0u;
        sum += c[j];
    }
    uint32_t total;
    const uint32_t base0 = block_exclusive_scan(sum, s, &total);
    // segment extents and their CTAs (the aggregation's records per CTA: agg_chunk)
    uint32_t nctas = 0, nonempty = 0;
    uint32_t beg = base0;
#pragma unroll
    for (uint32_t j = 0; j < kScanPer; ++j) {
        const uint64_t b = beg, e = (uint64_t)beg + c[j];
        ctas[j] = c[j] ? (uint32_t)((e - 1) / agg_chunk - b / agg_chunk + 1) : 0u;
        nctas += ctas[j];
        nonempty += c[j] ? 1u : 0u;
        beg += c[j];
    }
    uint32_t dummy;
    const uint32_t part0 = block_exclusive_scan(nctas, s, &dummy);
    uint32_t n_nonempty;
    const uint32_t idx0 = block_exclusive_scan(nonempty, s, &n_nonempty);
    beg = base0;
    uint32_t part = part0, idx = idx0;
#pragma unroll
    for (uint32_t j = 0; j < kScanPer; ++j) {
        const uint32_t b = b0 + j;
        if (b < nb) {
            cnt[b] = beg;
            part_desc[b] = make_uint2(part, ctas[j]);
            if (c[j]) {
                const uint32_t w = b / groups;
                WinDesc d;
                d.begin = beg;
                d.end = (uint64_t)beg + c[j];
                d.slot = p.wins[w].slot;
                d.flags = 0u;
                d.ctas = ctas[j];
                d.part_base = part;
                d.n_parts = ctas[j];
                d.key_base = (b - w * groups) * rows;
                descs[idx++] = d;
            }
        }
        beg += c[j];
        part += ctas[j];
    }
    for (uint32_t i = n_nonempty + t; i < nb; i += kScanThreads) {  // unused: past every CTA's records
        WinDesc d;
        d.begin = p.n_total;
        d.end = p.n_total;
        d.slot = 0u;
        d.flags = 0u;
        d.ctas = 0u;
        d.part_base = 0u;
        d.n_parts = 0u;
        d.key_base = 0u;
        descs[i] = d;
    }
}

}  // namespace

uint64_t part_array_stride(uint64_t n) { return (n + 3u) & ~3ull; }

cudaError_t launch_part_count(const AggParams& p, const LaunchShape& s, uint32_t* cnt, cudaStream_t st) {
    const uint32_t nb = p.n_wins * s.part_groups;
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)nb * 4, st);
    if (e != cudaSuccess) return e;
    const uint64_t chunk = (p.n_total + s.part_grid - 1) / s.part_grid;
    (void)cudaGetLastError();
    k_part_count<<<s.part_grid, kPartThreads, (size_t)nb * 4, st>>>(p, chunk, s.part_rows, s.part_groups, cnt);
    return cudaGetLastError();
}

cudaError_t launch_part_scan(const AggParams& p, const LaunchShape& s, uint64_t agg_chunk, uint32_t* cnt,
                             WinDesc* descs, uint2* part_desc, cudaStream_t st) {
    (void)cudaGetLastError();
    k_part_scan<<<1, kScanThreads, 0, st>>>(p, s.part_rows, s.part_groups, agg_chunk, cnt, descs, part_desc);
    return cudaGetLastError();
}

cudaError_t launch_part_scatter(const AggParams& p, const LaunchShape& s, uint32_t* cnt, uint32_t* out,
                                cudaStream_t st) {
    const uint64_t chunk = (p.n_total + s.part_grid - 1) / s.part_grid;
    static OptInCache granted;
    const int bytes = (int)((5 * kTile + 3 * s.part_groups) * 4);
    cudaError_t e = ensure_smem_optin((const void*)k_part_scatter, bytes, granted);
    if (e != cudaSuccess) return e;
    (void)cudaGetLastError();
    k_part_scatter<<<s.part_grid, kPartThreads, (size_t)bytes, st>>>(p, chunk, s.part_rows, s.part_groups, cnt, out,
                                                                      part_array_stride(p.n_total));
    return cudaGetLastError();
}

}  // namespace gnm
