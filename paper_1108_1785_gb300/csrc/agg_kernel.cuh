// agg_kernel.cuh -- the window aggregation kernel (the paper's TransRate step,
// Sec. III.B.2.1) and its device helpers. Included by one translation unit per lookup
// mode so that the variants compile in parallel.
//
// One persistent launch processes any number of windows laid out back to back in one
// struct-of-arrays batch. CTA b owns the contiguous record range
// [b*chunk, (b+1)*chunk); it walks the windows that overlap it, accumulates each
// window's per-(site, direction) sums in shared memory, adds them to the window's
// global accumulator row with one atomic per column and key, and takes a ticket; the
// CTA that takes a window's last ticket finalises it (rates and flags) in place.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gnm_internal.cuh"

namespace gnm {
namespace dev {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint4 ld_stream4(const uint32_t* p) {
    return __ldcs(reinterpret_cast<const uint4*>(p));
}
__device__ __forceinline__ uint32_t ld_stream1(const uint32_t* p) { return __ldcs(p); }

// Local-site membership: any of the (at most GNM_MAX_LOCAL) local prefixes contains a.
__device__ __forceinline__ bool is_local(const AggParams& p, uint32_t a) {
    bool r = false;
#pragma unroll
    for (int i = 0; i < GNM_MAX_LOCAL; ++i)
        if (i < (int)p.n_local) r |= ((a & p.local_mask[i]) == p.local_pfx[i]);
    return r;
}

// Predecessor search over sorted range starts (s[0] = 0): largest i with s[i] <= x.
// R independent searches advance in lock step so their loads overlap.
template <int R, bool kShared>
__device__ __forceinline__ void pred_search(const uint32_t* __restrict__ s, uint32_t n,
                                            const uint32_t (&x)[R], uint32_t (&base)[R]) {
#pragma unroll
    for (int j = 0; j < R; ++j) base[j] = 0;
    uint32_t len = n;
    while (len > 1) {
        const uint32_t half = len >> 1;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const uint32_t v = kShared ? s[base[j] + half] : __ldg(s + base[j] + half);
            base[j] = (v <= x[j]) ? base[j] + half : base[j];
        }
        len -= half;
    }
}

__device__ __forceinline__ uint32_t pred_search1(const uint32_t* __restrict__ s, uint32_t lo,
                                                 uint32_t len, uint32_t x) {
    uint32_t base = lo;
    while (len > 1) {
        const uint32_t half = len >> 1;
        base = (__ldg(s + base + half) <= x) ? base + half : base;
        len -= half;
    }
    return base;
}

// floor(v) clamped to [0, n-1] (n - 1 < 2^24, so the comparison is exact); NaN -> 0.
__device__ __forceinline__ uint32_t clamp_floor(float v, uint32_t n) {
    if (!(v >= 0.f)) return 0u;
    if (v >= (float)(n - 1)) return n - 1;
    return (uint32_t)v;
}

// Root of the learned index: leaf of address x (FP32, one rounding per operation).
__device__ __forceinline__ uint32_t rmi_root(const RmiDev& m, uint32_t x) {
    const float xn = __fmul_rn(__uint2float_rn(x), 2.3283064365386963e-10f);  // x * 2^-32
    float r;
    if (m.root_kind == GNM_RMI_ROOT_LINEAR) {
        r = __fadd_rn(__fmul_rn(m.ra, xn), m.rb);
    } else {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < kMaxHidden; ++j) {
            if (j < (int)m.hidden) {
                const float pre = __fadd_rn(__fmul_rn(m.w1[j], xn), m.b1[j]);
                const float h = pre > 0.f ? pre : 0.f;
                acc = __fadd_rn(acc, __fmul_rn(m.w2[j], h));
            }
        }
        r = __fadd_rn(acc, m.b2);
    }
    return clamp_floor(r, m.n_leaves);
}

// Predicted position of x inside leaf l.
__device__ __forceinline__ uint32_t rmi_leaf_pos(const float* a, const float* b,
                                                 const uint32_t* x0, uint32_t l, uint32_t x,
                                                 uint32_t n) {
    const float d = __ll2float_rn((long long)x - (long long)x0[l]);
    return clamp_floor(__fadd_rn(__fmul_rn(a[l], d), b[l]), n);
}

// Learned-index lookup: model window, exact search inside it, verification, fallback.
__device__ __forceinline__ uint32_t rmi_lookup(const RmiDev& m, const float* a, const float* b,
                                               const uint32_t* x0, const uint32_t* eps,
                                               const uint32_t* __restrict__ starts, uint32_t n,
                                               uint32_t x, unsigned long long* violations) {
    const uint32_t l = rmi_root(m, x);
    const uint32_t e = eps[l];
    if (e == 0xFFFFFFFFu) return pred_search1(starts, 0, n, x);
    const uint32_t pi = rmi_leaf_pos(a, b, x0, l, x, n);
    const uint32_t elo = e & 0xFFFFu, ehi = e >> 16;
    const uint32_t lo = pi > elo ? pi - elo : 0u;
    const uint32_t hi = min(pi + ehi + 1u, n - 1u);  // one past the bound, to verify it
    const uint32_t r = pred_search1(starts, lo, hi - lo + 1u, x);
    const bool ok = (lo == 0u || __ldg(starts + lo) <= x) && (r < hi || hi == n - 1u);
    if (ok) return r;
    atomicAdd(violations, 1ull);
    return pred_search1(starts, 0, n, x);
}

// Staged placement, last level: the 64-byte block of 8 ranges holding x (8 starts, then
// their 8 sites; padding past the last range repeats 0xFFFFFFFF as start and the last site,
// so it only ever matches x = 0xFFFFFFFF, which belongs to the last range anyway).
__device__ __forceinline__ uint32_t staged_block_site(const uint4* b, uint32_t x) {
    const uint4 s0 = __ldg(b), s1 = __ldg(b + 1), w0 = __ldg(b + 2), w1 = __ldg(b + 3);
    const uint32_t c = (s0.y <= x) + (s0.z <= x) + (s0.w <= x) + (s1.x <= x) + (s1.y <= x) +
                       (s1.z <= x) + (s1.w <= x);  // s0.x <= x holds: it is the block's sample
    const uint4 w = c < 4 ? w0 : w1;
    const uint32_t q = c & 3u;
    return q == 0 ? w.x : (q == 1 ? w.y : (q == 2 ? w.z : w.w));
}

// Range index form of the same lookup (largest i with start_i <= x), clamped to n-1.
__device__ __forceinline__ uint32_t staged_block_pos(const uint4* b, uint32_t jb, uint32_t x, uint32_t n) {
    const uint4 s0 = __ldg(b), s1 = __ldg(b + 1);
    const uint32_t c = (s0.y <= x) + (s0.z <= x) + (s0.w <= x) + (s1.x <= x) + (s1.y <= x) +
                       (s1.z <= x) + (s1.w <= x);
    return min(jb * kBlockRanges + c, n - 1);
}

// One classified record.
struct Item {
    uint32_t key;   // site*2+dir, or 2*n_sites + unmatched class
    uint32_t oc, pk, dur;
    bool elig, valid;
};

__device__ __forceinline__ Item classify(const AggParams& p, bool valid, uint32_t src,
                                         uint32_t dst, uint32_t pk, uint32_t oc, uint32_t fi,
                                         uint32_t la, uint32_t site) {
    Item it;
    const bool sl = is_local(p, src), dl = is_local(p, dst);
    const uint32_t nk = 2u * p.n_sites;
    const uint32_t dir = sl ? 1u : 0u;  // outbound when the source is local
    const uint32_t dur = la - fi;       // modulo 2^32
    bool elig = false;
    if (sl == dl) {
        it.key = nk + (sl ? 1u : 0u);   // 0 neither local, 1 both local
    } else if (site == kNoSite) {
        it.key = nk + 2u + dir;         // 2 inbound unregistered, 3 outbound unregistered
    } else {
        it.key = site * 2u + dir;
        const bool ack_ok = (uint64_t)oc >= (uint64_t)p.min_avg * (uint64_t)pk;
        const bool many = pk >= p.min_pkts, longd = dur >= p.min_dur;
        const bool admin_ok = p.admin_rule == GNM_ADMIN_OR ? (many && longd) : (many || longd);
        elig = dur != 0u && ack_ok && admin_ok;
    }
    it.oc = oc;
    it.pk = pk;
    it.dur = dur;
    it.elig = elig;
    it.valid = valid;
    return it;
}

__device__ __forceinline__ void red_add(uint64_t* a, uint64_t v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(a), (unsigned long long)v);
}

// Adds one record's contribution to a packed 5-column row (shared or global).
__device__ __forceinline__ void row_add(uint64_t* row, const Item& it) {
    red_add(row + 0, it.elig ? 0x100000001ull : 0x100000000ull);
    red_add(row + 1, it.oc);
    red_add(row + 2, it.pk);
    if (it.elig) {
        red_add(row + 3, it.oc);
        red_add(row + 4, it.dur);
    }
}

__device__ __forceinline__ void row_add_sums(uint64_t* row, uint64_t packed, uint64_t oc,
                                             uint64_t pk, uint64_t eoc, uint64_t edur, bool any_e) {
    red_add(row + 0, packed);
    red_add(row + 1, oc);
    red_add(row + 2, pk);
    if (any_e) {
        red_add(row + 3, eoc);
        red_add(row + 4, edur);
    }
}

// Sum of a 32-bit value over the lanes of `peers`, exact in 64 bits (16-bit halves).
__device__ __forceinline__ uint64_t peer_sum(unsigned peers, uint32_t v) {
    const uint32_t lo = __reduce_add_sync(peers, v & 0xFFFFu);
    const uint32_t hi = __reduce_add_sync(peers, v >> 16);
    return ((uint64_t)hi << 16) + (uint64_t)lo;
}

// Shared-memory cache slot of `key`: one of the two slots of its bucket pair, taking a
// free one if needed; -1 when both hold other keys (the record then goes to global
// memory). Keys seen early in a CTA's range -- the frequent ones -- keep their slots.
__device__ __forceinline__ int table_slot(uint32_t* tk, uint32_t cap, uint32_t key) {
    uint32_t h = (key * 2654435761u);
    h = (h ^ (h >> 15)) & (cap - 2u);  // even slot of the pair
    volatile uint32_t* vk = tk;
    uint32_t k0 = vk[h];
    if (k0 == key) return (int)h;
    uint32_t k1 = vk[h + 1];
    if (k1 == key) return (int)h + 1;
    if (k0 == kEmptyKey) {
        k0 = atomicCAS(tk + h, kEmptyKey, key);
        if (k0 == kEmptyKey || k0 == key) return (int)h;
    }
    if (k1 == kEmptyKey) {
        k1 = atomicCAS(tk + h + 1, kEmptyKey, key);
        if (k1 == kEmptyKey || k1 == key) return (int)h + 1;
    }
    return -1;
}

template <int TABLE>
__device__ __forceinline__ uint64_t* smem_row(uint64_t* tv, uint32_t* tk, uint32_t cap,
                                              uint32_t key) {
    if (TABLE == kTableDirect) return tv + (size_t)key * kAccCols;
    const int s = table_slot(tk, cap, key);
    return s >= 0 ? tv + (size_t)s * kAccCols : nullptr;
}

// Sums of one item per lane over the lanes that share its key, added by the group
// leader to `row` (or, when row is null, to the key's global accumulator row).
// Warp-collective over the lanes with `part` set.
__device__ __forceinline__ void group_add(const Item& it, unsigned peers, uint64_t* row, uint64_t* gacc) {
    const uint32_t e = it.elig ? 1u : 0u;
    const uint32_t n = __popc(peers);
    const uint32_t ne = __reduce_add_sync(peers, e);
    const uint64_t oc = peer_sum(peers, it.oc);
    const uint64_t pk = peer_sum(peers, it.pk);
    uint64_t eoc = 0, edur = 0;
    if (ne) {  // uniform across the peer group
        eoc = peer_sum(peers, it.elig ? it.oc : 0u);
        edur = peer_sum(peers, it.elig ? it.dur : 0u);
    }
    if ((int)(threadIdx.x & 31u) != __ffs(peers) - 1) return;
    if (row == nullptr) row = gacc + (size_t)it.key * kAccCols;
    row_add_sums(row, ((uint64_t)n << 32) | ne, oc, pk, eoc, edur, ne != 0);
}

// Accumulate one item per lane. Warp-collective: every lane of the warp calls it
// (invalid lanes with valid = false).
//   DIRECT aggregation: each lane adds to its key's shared-memory row; lanes whose key
//   has no row (cache full) are combined per key across the warp and added globally.
//   WARP aggregation: lanes are first combined per key; the group leader adds.
template <int TABLE, int AGG>
__device__ __forceinline__ void accumulate(const Item& it, uint64_t* tv, uint32_t* tk,
                                           uint32_t cap, uint64_t* gacc) {
    if (TABLE != kTableGlobal && AGG == GNM_AGG_DIRECT) {
        uint64_t* row = it.valid ? smem_row<TABLE>(tv, tk, cap, it.key) : nullptr;
        const bool miss = it.valid && row == nullptr;
        if (TABLE == kTableHash && __any_sync(kFull, miss)) {
            const unsigned peers = __match_any_sync(kFull, miss ? it.key : kEmptyKey);
            if (miss) group_add(it, peers, nullptr, gacc);
        }
        if (row) row_add(row, it);
        return;
    }
    const unsigned peers = __match_any_sync(kFull, it.valid ? it.key : kEmptyKey);
    if (!it.valid) return;
    uint64_t* row = nullptr;
    if (TABLE != kTableGlobal) {
        // the leader probes for the whole group
        const int leader = __ffs(peers) - 1;
        uint64_t* r = nullptr;
        if ((int)(threadIdx.x & 31u) == leader) r = smem_row<TABLE>(tv, tk, cap, it.key);
        row = (uint64_t*)__shfl_sync(peers, (unsigned long long)r, leader);
    }
    group_add(it, peers, row, gacc);
}

// Adds the CTA's shared-memory sums to the window's global accumulators and clears them.
template <int TABLE>
__device__ __forceinline__ void flush(uint64_t* tv, uint32_t* tk, uint32_t rows, uint64_t* gacc) {
    for (uint32_t r = threadIdx.x; r < rows; r += blockDim.x) {
        uint64_t* row = tv + (size_t)r * kAccCols;
        const uint64_t packed = row[0];
        uint32_t key = r;
        if (TABLE == kTableHash) {
            key = tk[r];
            tk[r] = kEmptyKey;
        }
        if (packed == 0) continue;
        uint64_t* g = gacc + (size_t)key * kAccCols;
        const bool any_e = (packed & 0xFFFFFFFFull) != 0;
        row_add_sums(g, packed, row[1], row[2], row[3], row[4], any_e);
#pragma unroll
        for (int c = 0; c < kAccCols; ++c) row[c] = 0;
    }
}

// Rates and flags of one window from its accumulators (Sec. III.B.1: rates per site;
// a site is sub-optimal when its rate is below the standard).
__device__ __forceinline__ void finalize_rows(const AggParams& p, uint32_t slot, uint32_t k0,
                                              uint32_t step) {
    const size_t keys = p.keys;
    uint64_t* acc = p.acc + (size_t)slot * keys * kAccCols;
    uint64_t* st = p.stats + (size_t)slot * keys * kNStat;
    const uint32_t nk = 2u * p.n_sites;
    double* rate = p.rate + (size_t)slot * nk;
    uint8_t* flag = p.flag + (size_t)slot * nk;
    for (uint32_t k = k0; k < keys; k += step) {
        uint64_t* a = acc + (size_t)k * kAccCols;
        const uint64_t packed = __ldcg(reinterpret_cast<const unsigned long long*>(a));
        const uint64_t oc = __ldcg(reinterpret_cast<const unsigned long long*>(a + 1));
        const uint64_t pk = __ldcg(reinterpret_cast<const unsigned long long*>(a + 2));
        const uint64_t eo = __ldcg(reinterpret_cast<const unsigned long long*>(a + 3));
        const uint64_t ed = __ldcg(reinterpret_cast<const unsigned long long*>(a + 4));
        const uint64_t ef = packed & 0xFFFFFFFFull;
        // accumulators return to zero for the slot's next window
#pragma unroll
        for (int c = 0; c < kAccCols; ++c) a[c] = 0;
        uint64_t* s = st + (size_t)k * kNStat;
        s[0] = packed >> 32;
        s[1] = oc;
        s[2] = pk;
        s[3] = ef;
        s[4] = eo;
        s[5] = ed;
        if (k < nk) {
            // rate = (octets * 8 bits) / (ms / 1000), one rounding per operation
            const double r = ed ? __ddiv_rn(__dmul_rn(__ull2double_rn(eo), 8000.0),
                                            __ull2double_rn(ed))
                                : __longlong_as_double(0x7FF8000000000000ll);
            rate[k] = r;
            flag[k] = (ef >= (uint64_t)p.min_flows && r < p.threshold) ? 1 : 0;
        }
    }
}

// Smallest window index whose end is past `lo` (windows sorted, disjoint, non-empty).
__device__ __forceinline__ uint32_t first_window(const WinDesc* w, uint32_t n, uint64_t lo) {
    uint32_t a = 0, b = n;
    while (a < b) {
        const uint32_t m = (a + b) >> 1;
        if (w[m].end > lo) b = m;
        else a = m + 1;
    }
    return a;
}

struct Smem {
    uint64_t* tv;       // table values
    uint32_t* tk;       // hash keys
    uint32_t rows;      // table rows
    const uint32_t* s_starts;
    const uint32_t* s_site;
    const float* ra;    // learned index leaf arrays
    const float* rb;
    const uint32_t* rx0;
    const uint32_t* reps;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Shared-memory layout: [table values][hash keys][registry or leaf arrays].
__host__ __device__ inline size_t smem_layout(int lookup, int table, uint32_t n_ranges,
                                              uint32_t keys, uint32_t cap, uint32_t n_leaves,
                                              size_t* off_keys, size_t* off_lookup) {
    const uint32_t rows = table == kTableDirect ? keys : (table == kTableHash ? cap : 0u);
    size_t o = (size_t)rows * kAccCols * 8;
    *off_keys = o;
    if (table == kTableHash) o += (size_t)cap * 4;
    o = align_up(o, 16);
    *off_lookup = o;
    if (lookup == kLookupSmem) o += (size_t)n_ranges * 8;
    if (lookup == kLookupStaged) o += (size_t)((n_ranges + kBlockRanges - 1) / kBlockRanges) * 4;
    if (lookup == kLookupRmi) o += (size_t)n_leaves * 16;
    return align_up(o, 16);
}

// Processes R records per thread: lookups for all of them first (independent loads in
// flight together), then classification and accumulation.
template <int LOOKUP, int TABLE, int AGG, int R>
__device__ __forceinline__ void process(const AggParams& p, const Smem& sm, uint64_t* gacc,
                                        const bool (&valid)[R], const uint32_t (&src)[R],
                                        const uint32_t (&dst)[R], const uint32_t (&pk)[R],
                                        const uint32_t (&oc)[R], const uint32_t (&fi)[R],
                                        const uint32_t (&la)[R]) {
    uint32_t x[R], idx[R], site[R];
#pragma unroll
    for (int j = 0; j < R; ++j) x[j] = is_local(p, src[j]) ? dst[j] : src[j];
    if (LOOKUP == kLookupSmem) {
        pred_search<R, true>(sm.s_starts, p.n_ranges, x, idx);
#pragma unroll
        for (int j = 0; j < R; ++j) site[j] = sm.s_site[idx[j]];
    } else if (LOOKUP == kLookupL2) {
        pred_search<R, false>(p.starts, p.n_ranges, x, idx);
#pragma unroll
        for (int j = 0; j < R; ++j) site[j] = __ldg(p.rsite + idx[j]);
    } else if (LOOKUP == kLookupStaged) {
        pred_search<R, true>(sm.s_starts, p.n_blocks, x, idx);  // block of x
#pragma unroll
        for (int j = 0; j < R; ++j) site[j] = staged_block_site(p.blocks + 4 * (size_t)idx[j], x[j]);
    } else {
#pragma unroll
        for (int j = 0; j < R; ++j) {
            idx[j] = valid[j] ? rmi_lookup(p.rmi, sm.ra, sm.rb, sm.rx0, sm.reps, p.starts,
                                           p.n_ranges, x[j], p.violations)
                              : 0u;
        }
#pragma unroll
        for (int j = 0; j < R; ++j) site[j] = __ldg(p.rsite + idx[j]);
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const Item it = classify(p, valid[j], src[j], dst[j], pk[j], oc[j], fi[j], la[j], site[j]);
        accumulate<TABLE, AGG>(it, sm.tv, sm.tk, p.table_cap, gacc);
    }
}

// Records [lo, hi) one per thread and slot (head/tail of a window, or unaligned arrays).
template <int LOOKUP, int TABLE, int AGG>
__device__ __forceinline__ void scalar_range(const AggParams& p, const Smem& sm, uint64_t* gacc,
                                             uint64_t lo, uint64_t hi) {
    const uint32_t B = blockDim.x;
    for (uint64_t base = lo; base < hi; base += (uint64_t)B * 4u) {  // uniform loop
        bool v[4];
        uint32_t s[4], d[4], pk[4], oc[4], fi[4], la[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint64_t i = base + (uint64_t)j * B + threadIdx.x;
            v[j] = i < hi;
            const uint64_t ii = v[j] ? i : lo;
            s[j] = ld_stream1(p.src + ii);
            d[j] = ld_stream1(p.dst + ii);
            pk[j] = ld_stream1(p.pkts + ii);
            oc[j] = ld_stream1(p.oct + ii);
            fi[j] = ld_stream1(p.first + ii);
            la[j] = ld_stream1(p.last + ii);
        }
        process<LOOKUP, TABLE, AGG, 4>(p, sm, gacc, v, s, d, pk, oc, fi, la);
    }
}

// Records [a0, a0 + 4*G): G aligned groups of four, 16-byte vector loads.
template <int LOOKUP, int TABLE, int AGG, int U>
__device__ __forceinline__ void vector_range(const AggParams& p, const Smem& sm, uint64_t* gacc,
                                             uint64_t a0, uint64_t G) {
    constexpr int R = 4 * U;
    const uint32_t B = blockDim.x;
    for (uint64_t gb = 0; gb < G; gb += (uint64_t)B * U) {  // uniform loop
        bool v[R];
        uint32_t s[R], d[R], pk[R], oc[R], fi[R], la[R];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t g = gb + (uint64_t)u * B + threadIdx.x;
            const bool ok = g < G;
            const uint64_t i = a0 + 4u * (ok ? g : 0u);
            const uint4 vs = ld_stream4(p.src + i), vd = ld_stream4(p.dst + i);
            const uint4 vp = ld_stream4(p.pkts + i), vo = ld_stream4(p.oct + i);
            const uint4 vf = ld_stream4(p.first + i), vl = ld_stream4(p.last + i);
            s[4 * u + 0] = vs.x; s[4 * u + 1] = vs.y; s[4 * u + 2] = vs.z; s[4 * u + 3] = vs.w;
            d[4 * u + 0] = vd.x; d[4 * u + 1] = vd.y; d[4 * u + 2] = vd.z; d[4 * u + 3] = vd.w;
            pk[4 * u + 0] = vp.x; pk[4 * u + 1] = vp.y; pk[4 * u + 2] = vp.z; pk[4 * u + 3] = vp.w;
            oc[4 * u + 0] = vo.x; oc[4 * u + 1] = vo.y; oc[4 * u + 2] = vo.z; oc[4 * u + 3] = vo.w;
            fi[4 * u + 0] = vf.x; fi[4 * u + 1] = vf.y; fi[4 * u + 2] = vf.z; fi[4 * u + 3] = vf.w;
            la[4 * u + 0] = vl.x; la[4 * u + 1] = vl.y; la[4 * u + 2] = vl.z; la[4 * u + 3] = vl.w;
#pragma unroll
            for (int j = 0; j < 4; ++j) v[4 * u + j] = ok;
        }
        process<LOOKUP, TABLE, AGG, R>(p, sm, gacc, v, s, d, pk, oc, fi, la);
    }
}

template <int LOOKUP, int TABLE, int AGG, int U>
__global__ void __launch_bounds__(U == 1 ? 1024 : 512)
    k_aggregate(const __grid_constant__ AggParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_last;
    const uint32_t tid = threadIdx.x, B = blockDim.x;

    const uint64_t lo = min((uint64_t)blockIdx.x * p.chunk, p.n_total);
    const uint64_t hi = min(lo + p.chunk, p.n_total);
    if (lo >= hi) return;  // whole CTA idle

    size_t off_keys, off_lookup;
    smem_layout(LOOKUP, TABLE, p.n_ranges, p.keys, p.table_cap,
                LOOKUP == kLookupRmi ? p.rmi.n_leaves : 0u, &off_keys, &off_lookup);
    Smem sm;
    sm.tv = reinterpret_cast<uint64_t*>(smem_raw);
    sm.tk = reinterpret_cast<uint32_t*>(smem_raw + off_keys);
    sm.rows = TABLE == kTableDirect ? p.keys : (TABLE == kTableHash ? p.table_cap : 0u);
    // stage the table (zero), the registry or the leaf parameters
    for (uint32_t i = tid; i < sm.rows * kAccCols; i += B) sm.tv[i] = 0;
    if (TABLE == kTableHash)
        for (uint32_t i = tid; i < p.table_cap; i += B) sm.tk[i] = kEmptyKey;
    if (LOOKUP == kLookupSmem) {
        uint32_t* st = reinterpret_cast<uint32_t*>(smem_raw + off_lookup);
        uint32_t* si = st + p.n_ranges;
        for (uint32_t i = tid; i < p.n_ranges; i += B) {
            st[i] = __ldg(p.starts + i);
            si[i] = __ldg(p.rsite + i);
        }
        sm.s_starts = st;
        sm.s_site = si;
    }
    if (LOOKUP == kLookupStaged) {
        uint32_t* st = reinterpret_cast<uint32_t*>(smem_raw + off_lookup);
        for (uint32_t i = tid; i < p.n_blocks; i += B) st[i] = __ldg(p.sample + i);
        sm.s_starts = st;
    }
    if (LOOKUP == kLookupRmi) {
        const uint32_t L = p.rmi.n_leaves;
        float* a = reinterpret_cast<float*>(smem_raw + off_lookup);
        float* b = a + L;
        uint32_t* x0 = reinterpret_cast<uint32_t*>(b + L);
        uint32_t* e = x0 + L;
        for (uint32_t i = tid; i < L; i += B) {
            a[i] = __ldg(p.rmi.a + i);
            b[i] = __ldg(p.rmi.b + i);
            x0[i] = __ldg(p.rmi.x0 + i);
            e[i] = __ldg(p.rmi.eps + i);
        }
        sm.ra = a;
        sm.rb = b;
        sm.rx0 = x0;
        sm.reps = e;
    }
    __syncthreads();

    for (uint32_t w = first_window(p.wins, p.n_wins, lo); w < p.n_wins; ++w) {
        const WinDesc wd = p.wins[w];
        if (wd.begin >= hi) break;
        const uint64_t s = max(wd.begin, lo), e = min(wd.end, hi);
        uint64_t* gacc = p.acc + (size_t)wd.slot * p.keys * kAccCols;
        uint64_t a0 = e, a1 = e;
        if (p.vec_ok) {
            const uint32_t mis = (uint32_t)((s + p.phase) & 3u);
            a0 = mis ? min(s + (4u - mis), e) : s;
            a1 = a0 + ((e - a0) & ~3ull);
        }
        scalar_range<LOOKUP, TABLE, AGG>(p, sm, gacc, s, a0);
        if (a1 > a0) vector_range<LOOKUP, TABLE, AGG, U>(p, sm, gacc, a0, (a1 - a0) >> 2);
        scalar_range<LOOKUP, TABLE, AGG>(p, sm, gacc, a1, e);
        if (TABLE != kTableGlobal) {
            __syncthreads();
            flush<TABLE>(sm.tv, sm.tk, sm.rows, gacc);
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const uint32_t t = atomicAdd(p.done + w, 1u);
            s_last = (t + 1u == wd.ctas) ? 1 : 0;
            if (s_last) {
                p.done[w] = 0;  // every other CTA of this window has taken its ticket
                __threadfence();
            }
        }
        __syncthreads();
        if (s_last && (wd.flags & kWinFinalize)) finalize_rows(p, wd.slot, tid, B);
        __syncthreads();
    }
}

template <int LOOKUP, int TABLE, int AGG, int U>
cudaError_t launch_variant(const AggParams& p, const LaunchShape& s, cudaStream_t st) {
    auto k = k_aggregate<LOOKUP, TABLE, AGG, U>;
    static int set_bytes[64];  // opt-in already granted, per device (0 = none yet)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (s.smem > 48 * 1024 && (dev >= 64 || set_bytes[dev] < (int)s.smem)) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
        if (e != cudaSuccess) return e;
        if (dev < 64) set_bytes[dev] = (int)s.smem;
    }
    (void)cudaGetLastError();  // report this launch's error only
    k<<<s.grid, s.block, s.smem, st>>>(p);
    return cudaGetLastError();
}

template <int LOOKUP, int TABLE>
cudaError_t launch_table(const AggParams& p, const LaunchShape& s, cudaStream_t st) {
    if (TABLE == kTableGlobal || s.agg == GNM_AGG_WARP) {
        return s.unroll == 2 ? launch_variant<LOOKUP, TABLE, GNM_AGG_WARP, 2>(p, s, st)
                             : launch_variant<LOOKUP, TABLE, GNM_AGG_WARP, 1>(p, s, st);
    }
    return s.unroll == 2 ? launch_variant<LOOKUP, TABLE, GNM_AGG_DIRECT, 2>(p, s, st)
                         : launch_variant<LOOKUP, TABLE, GNM_AGG_DIRECT, 1>(p, s, st);
}

template <int LOOKUP>
cudaError_t launch_lookup_mode(const AggParams& p, const LaunchShape& s, cudaStream_t st) {
    switch (s.table) {
        case kTableDirect: return launch_table<LOOKUP, kTableDirect>(p, s, st);
        case kTableHash: return launch_table<LOOKUP, kTableHash>(p, s, st);
        default: return launch_table<LOOKUP, kTableGlobal>(p, s, st);
    }
}

}  // namespace dev
}  // namespace gnm
