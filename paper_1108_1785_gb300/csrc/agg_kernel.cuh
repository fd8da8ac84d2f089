// agg_kernel.cuh -- the window aggregation kernel (the paper's TransRate step,
// Sec. III.B.2.1) and its device helpers. Included by one translation unit per lookup
// mode so that the variants compile in parallel.
//
// One persistent launch processes any number of windows laid out back to back in one
// struct-of-arrays batch. CTA b owns the contiguous record range
// [b*chunk, (b+1)*chunk); it walks the windows that overlap it and accumulates each
// window's per-(site, direction) sums in shared memory. At the end of its segment of a
// window it hands them over: with a direct table, as plain stores of its rows to a partial
// block of its own; otherwise with one global atomic per column and key. It then takes the
// window's ticket; the CTA that takes the last one finalises the window (rates and flags)
// when its key space is small, else a grid-wide finalisation kernel follows.
#pragma once
#include <cooperative_groups.h>
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

// Local-site membership of both endpoints: any of the (at most GNM_MAX_LOCAL) local
// prefixes contains the address. The loop stops at n_local (uniform across the grid).
__device__ __forceinline__ void local_pair(const AggParams& p, uint32_t src, uint32_t dst, bool& sl, bool& dl) {
    sl = false;
    dl = false;
#pragma unroll
    for (int i = 0; i < GNM_MAX_LOCAL; ++i) {
        if (i >= (int)p.n_local) break;
        const uint32_t m = p.local_mask[i], q = p.local_pfx[i];
        sl |= (src & m) == q;
        dl |= (dst & m) == q;
    }
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

// Radix-directed search: dir[t] is the range holding the first address of bucket t (the
// top `bits` bits of an address), so x's range lies in [dir[t], dir[t+1]]; a binary search
// over the starts inside that interval finishes (R lookups in lock step, each stopping
// when its interval has one entry).
template <int R, bool kShared = false>
__device__ __forceinline__ void radix_search(const uint32_t* __restrict__ dir, uint32_t bits,
                                             const uint32_t* __restrict__ starts, const uint32_t (&x)[R],
                                             uint32_t (&base)[R], uint32_t n, unsigned long long* err) {
    uint32_t len[R];
    bool more = false;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const uint32_t t = bits ? x[j] >> (32u - bits) : 0u;
        base[j] = dir[t];
        len[j] = dir[t + 1] - base[j] + 1u;
        if (!chk(err, (uint64_t)base[j] + len[j] <= n, kChkWindow, base[j])) {
            base[j] = 0u;
            len[j] = 1u;
        }
        more |= len[j] > 1u;
    }
    while (more) {
        more = false;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            if (len[j] > 1u) {
                const uint32_t half = len[j] >> 1;
                const uint32_t v = kShared ? starts[base[j] + half] : __ldg(starts + base[j] + half);
                base[j] = v <= x[j] ? base[j] + half : base[j];
                len[j] -= half;
                more |= len[j] > 1u;
            }
        }
    }
}

// Predecessor search over (start, site) pairs, R lookups in lock step: narrows each
// [base, base + len) -- whose first start is <= x -- to one range, carrying the site of
// the current base along, so that no separate site load follows the last probe.
template <int R>
__device__ __forceinline__ void pair_search(const uint2* __restrict__ pairs, const uint32_t (&x)[R],
                                            uint32_t (&base)[R], uint32_t (&len)[R], uint32_t (&site)[R]) {
    bool more = false;
#pragma unroll
    for (int j = 0; j < R; ++j) more |= len[j] > 1u;
    while (more) {
        more = false;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            if (len[j] > 1u) {
                const uint32_t half = len[j] >> 1;
                const uint2 v = __ldg(pairs + base[j] + half);
                if (v.x <= x[j]) {
                    base[j] += half;
                    site[j] = v.y;
                }
                len[j] -= half;
                more |= len[j] > 1u;
            }
        }
    }
}

// Block-sample search (key kernel): dir[t] is the BR-range block holding the first address
// of bucket t (the top `bits` bits), so x's block lies in [dir[t], dir[t+1]]; a search over
// the blocks' first starts `smp` (shared memory) picks it, and one load of its BR (start,
// site) pairs (16 bytes for BR = 2, 32 for BR = 4) gives the site. Pairs past the last
// range are start 0xFFFFFFFF with the last range's site, so the count is right for every x.
// With fewer than 2^16 blocks (`packed`) the directory holds one word per bucket: the first
// block in its low 16 bits and the number of blocks after it in the high 16, one load instead
// of two.
template <int BR, int R>
__device__ __forceinline__ void radix_block(const uint32_t* dir, uint32_t bits, const uint32_t* smp,
                                            const uint2* __restrict__ pairs, const uint32_t (&x)[R],
                                            uint32_t (&site)[R], bool packed, uint32_t n_blk,
                                            unsigned long long* err) {
    static_assert(BR == 2 || BR == 4, "blocks of 2 or 4 ranges");
    uint32_t g[R], len[R];
    bool more = false;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const uint32_t t = x[j] >> (32u - bits);
        if (packed) {
            const uint32_t e = dir[t];
            g[j] = e & 0xFFFFu;
            len[j] = (e >> 16) + 1u;
        } else {
            g[j] = dir[t];
            len[j] = dir[t + 1] - g[j] + 1u;
        }
        if (!chk(err, (uint64_t)g[j] + len[j] <= n_blk, kChkBlocks, g[j])) {
            g[j] = 0u;
            len[j] = 1u;
        }
        more |= len[j] > 1u;
    }
    while (more) {
        more = false;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            if (len[j] > 1u) {
                const uint32_t half = len[j] >> 1;
                g[j] = smp[g[j] + half] <= x[j] ? g[j] + half : g[j];
                len[j] -= half;
                more |= len[j] > 1u;
            }
        }
    }
    uint4 lo[R], hi[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const uint4* q = reinterpret_cast<const uint4*>(pairs) + (BR / 2) * (size_t)g[j];
        if (BR == 2) {
            lo[j] = __ldg(q);  // start0 site0 start1 site1
        } else {  // one 32-byte load (a 32-byte aligned block): start0 site0 .. start3 site3
            asm("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                : "=r"(lo[j].x), "=r"(lo[j].y), "=r"(lo[j].z), "=r"(lo[j].w), "=r"(hi[j].x), "=r"(hi[j].y),
                  "=r"(hi[j].z), "=r"(hi[j].w)
                : "l"(q));
        }
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
        if (BR == 2) {
            site[j] = lo[j].z <= x[j] ? lo[j].w : lo[j].y;
        } else {
            const uint32_t c = (lo[j].z <= x[j]) + (hi[j].x <= x[j]) + (hi[j].z <= x[j]);
            site[j] = c == 0 ? lo[j].y : (c == 1 ? lo[j].w : (c == 2 ? hi[j].y : hi[j].w));
        }
    }
}

// Block-sample search with 16-bit tables (key kernel, fewer than 2^16 blocks of 2 ranges):
// dh[t] is the first block whose first start is >= t << 16 for the /16 bucket t of x, so the
// block before it holds the bucket's first address and blocks dh[t] .. dh[t+1]-1 start inside
// the bucket, where their low 16 start bits `s16` order them exactly. The last of those with
// low bits <= x's (or the block before them) holds x; one 16-byte load of its two (start,
// site) pairs gives the site. R lookups in lock step.
template <int R>
__device__ __forceinline__ void radix_block16(const uint16_t* dh, const uint16_t* s16,
                                              const uint2* __restrict__ pairs, const uint32_t (&x)[R],
                                              uint32_t (&site)[R], uint32_t n_blk, unsigned long long* err) {
    uint32_t l[R], n[R];
    bool more = false;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const uint32_t t = x[j] >> 16;
        l[j] = dh[t];
        n[j] = (uint32_t)dh[t + 1] - l[j];
        if (!chk(err, (uint64_t)l[j] + n[j] <= n_blk && dh[t + 1] >= l[j], kChkBlocks, l[j])) {
            l[j] = 1u;
            n[j] = 0u;
        }
        more |= n[j] > 0u;
    }
    while (more) {  // l: first candidate whose low bits exceed x's, within [l, l + n)
        more = false;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            if (n[j] > 0u) {
                const uint32_t half = n[j] >> 1;
                if (s16[l[j] + half] <= (x[j] & 0xFFFFu)) {
                    l[j] += half + 1u;
                    n[j] -= half + 1u;
                } else {
                    n[j] = half;
                }
                more |= n[j] > 0u;
            }
        }
    }
    uint4 v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {  // l >= 1: block 0 starts at address 0, inside bucket 0
        if (!chk(err, l[j] >= 1u, kChkBlocks, l[j])) l[j] = 1u;
        v[j] = __ldg(reinterpret_cast<const uint4*>(pairs) + (l[j] - 1u));
    }
#pragma unroll
    for (int j = 0; j < R; ++j) site[j] = v[j].z <= x[j] ? v[j].w : v[j].y;
}

// The paper's lookup (Sec. III.B.2.1): the site of x's /24 subnet from the hash table of
// the registered networks' /24 subnets (kNoSite when absent). Linear probing; the table is
// at most half full, so every probe sequence ends at the key or at an empty slot.
template <int R>
__device__ __forceinline__ void hash24_sites(const uint2* __restrict__ t, uint32_t mask, const uint32_t (&x)[R],
                                             uint32_t (&site)[R]) {
    uint32_t h[R];
    bool open[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        h[j] = hash24(x[j] >> 8) & mask;
        open[j] = true;
        site[j] = kNoSite;
    }
    bool more = true;
    while (more) {
        more = false;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            if (open[j]) {
                const uint2 e = __ldg(t + h[j]);
                if (e.x == (x[j] >> 8) + 1u) {
                    site[j] = e.y;
                    open[j] = false;
                } else if (e.x == 0u) {
                    open[j] = false;
                } else {
                    h[j] = (h[j] + 1u) & mask;
                    more = true;
                }
            }
        }
    }
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

// Parameters of leaf l: from the staged shared-memory arrays, or (a == null) with one
// 16-byte load of the interleaved global copy.
struct RmiLeaf {
    float a, b;
    uint32_t x0, eps;
};
__device__ __forceinline__ RmiLeaf rmi_leaf(const RmiDev& m, const float* a, const float* b, const uint32_t* x0,
                                            const uint32_t* eps, uint32_t l) {
    RmiLeaf f;
    if (a) {
        f.a = a[l];
        f.b = b[l];
        f.x0 = x0[l];
        f.eps = eps[l];
    } else {
        const uint4 v = __ldg(m.leaf4 + l);
        f.a = __uint_as_float(v.x);
        f.b = __uint_as_float(v.y);
        f.x0 = v.z;
        f.eps = v.w;
    }
    return f;
}

// fl(int64(x) - int64(x0)) on the 32-bit converter: round-to-nearest-even is symmetric in
// sign, so rounding |x - x0| and negating gives the same float as rounding the signed
// 64-bit difference.
__device__ __forceinline__ float rel_offset(uint32_t x, uint32_t x0) {
    return x >= x0 ? __uint2float_rn(x - x0) : -__uint2float_rn(x0 - x);
}

// Predicted position of x inside its leaf.
__device__ __forceinline__ uint32_t rmi_leaf_pos(const RmiLeaf& f, uint32_t x, uint32_t n) {
    return clamp_floor(__fadd_rn(__fmul_rn(f.a, rel_offset(x, f.x0)), f.b), n);
}

// Sub-leaf of x in a split leaf's record: min(((x - x0) mod 2^32) >> shift, count - 1),
// counted from the record's first sub-leaf.
__device__ __forceinline__ uint32_t rmi_sub_model(const RmiLeaf& f, uint32_t x) {
    const uint32_t w = __float_as_uint(f.a);
    return __float_as_uint(f.b) + min((x - f.x0) >> (w & 31u), w >> 8);
}

// Parameters of the model that answers x: the root's leaf, or its sub-leaf when the leaf
// is split (one more dependent load, for the addresses of split leaves only).
__device__ __forceinline__ RmiLeaf rmi_model(const RmiDev& m, const float* a, const float* b, const uint32_t* x0,
                                             const uint32_t* eps, uint32_t x) {
    RmiLeaf f = rmi_leaf(m, a, b, x0, eps, rmi_root(m, x));
    if (f.eps == kEpsSplit) {
        const uint32_t sub = rmi_sub_model(f, x);
        if (chk(m.check_err, sub < m.n_models, kChkModel, sub)) f = rmi_leaf(m, a, b, x0, eps, sub);
        else f.eps = 0xFFFFFFFFu;  // (checked build) no model: the full search
    }
    return f;
}

// Learned-index lookup: model window, exact search inside it, verification, fallback.
__device__ __forceinline__ uint32_t rmi_lookup(const RmiDev& m, const float* a, const float* b,
                                               const uint32_t* x0, const uint32_t* eps,
                                               const uint32_t* __restrict__ starts, uint32_t n,
                                               uint32_t x, unsigned long long* violations) {
    const RmiLeaf f = rmi_model(m, a, b, x0, eps, x);
    const uint32_t e = f.eps;
    if (e == 0xFFFFFFFFu) return pred_search1(starts, 0, n, x);
    const uint32_t pi = rmi_leaf_pos(f, x, n);
    const uint32_t elo = e & 0xFFFFu, ehi = e >> 16;
    const uint32_t lo = pi > elo ? pi - elo : 0u;
    const uint32_t hi = min(pi + ehi + 1u, n - 1u);  // one past the bound, to verify it
    const uint32_t r = pred_search1(starts, lo, hi - lo + 1u, x);
    const bool ok = (lo == 0u || __ldg(starts + lo) <= x) && (r < hi || hi == n - 1u);
    if (ok) return r;
    atomicAdd(violations, 1ull);
    return pred_search1(starts, 0, n, x);
}

// The four (start, site) pairs of 32-byte sector k of `pairs` (one 256-bit load, sm_100).
__device__ __forceinline__ void ld_sector(const uint2* __restrict__ pairs, uint32_t k, uint4& lo, uint4& hi) {
    const uint4* q = reinterpret_cast<const uint4*>(pairs) + 2u * (size_t)k;
    asm("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(lo.x), "=r"(lo.y), "=r"(lo.z), "=r"(lo.w), "=r"(hi.x), "=r"(hi.y), "=r"(hi.z), "=r"(hi.w)
        : "l"(q));
}

// Learned-index lookups of R addresses in lock step over the (start, site) pairs. The model
// gives each a window [lo, hi] (hi one past the proven bound, to verify it); the window is
// searched by 32-byte sectors of four pairs: a binary search over the sectors' first starts
// (one 4-byte probe each) finds the last sector from lo's sector to hi's whose first start
// is <= x, and one 256-bit load of it gives the count c of its starts <= x and the site.
// The answer is exact when c >= 1 (lo's sector does start at or below x) and the range
// after it was seen (c < 4, or a later sector was probed, or the array ends there);
// otherwise the lookup counts a fallback and takes the full search. Pairs past the last
// range have start 0xFFFFFFFF and the last range's site, and the array is padded so that
// the sector of any hi <= n - 1 is whole.
template <int R>
__device__ __forceinline__ void rmi_sites(const RmiDev& m, const float* a, const float* b, const uint32_t* x0,
                                          const uint32_t* eps, const uint2* __restrict__ pairs, uint32_t n,
                                          const bool (&valid)[R], const uint32_t (&x)[R], uint32_t (&site)[R],
                                          unsigned long long* violations) {
    uint32_t sb[R], len[R], s1[R];
    bool more = false;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const RmiLeaf lf = rmi_model(m, a, b, x0, eps, x[j]);
        const uint32_t e = lf.eps;
        uint32_t lo = 0u, hi = 0u;
        if (valid[j] && e == 0xFFFFFFFFu) {  // no proven bound for this leaf: full search
            hi = n - 1u;
        } else if (valid[j]) {
            const uint32_t pi = rmi_leaf_pos(lf, x[j], n);
            const uint32_t elo = e & 0xFFFFu, ehi = e >> 16;
            lo = pi > elo ? pi - elo : 0u;
            hi = min(pi + ehi + 1u, n - 1u);  // one past the bound, to verify it
        }
        sb[j] = lo >> 2;
        s1[j] = hi >> 2;
        len[j] = s1[j] - sb[j] + 1u;
        more |= len[j] > 1u;
    }
    const uint32_t* st = reinterpret_cast<const uint32_t*>(pairs);  // start of pair i at word 2i
    while (more) {
        more = false;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            if (len[j] > 1u) {
                const uint32_t half = len[j] >> 1;
                if (__ldg(st + 8u * (size_t)(sb[j] + half)) <= x[j]) sb[j] += half;
                len[j] -= half;
                more |= len[j] > 1u;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
        uint4 v0, v1;
        ld_sector(pairs, sb[j], v0, v1);
        const uint32_t c = (v0.x <= x[j]) + (v0.z <= x[j]) + (v1.x <= x[j]) + (v1.z <= x[j]);
        site[j] = c <= 1u ? v0.y : (c == 2u ? v0.w : (c == 3u ? v1.y : v1.w));
        const bool ok = c >= 1u && (c < 4u || sb[j] < s1[j] || 4u * sb[j] + 3u >= n - 1u);
        if (valid[j] && !ok) {
            atomicAdd(violations, 1ull);
            uint32_t xb[1] = {x[j]}, bb[1] = {0u}, lb[1] = {n}, sbb[1] = {__ldg(pairs).y};
            pair_search<1>(pairs, xb, bb, lb, sbb);
            site[j] = sbb[0];
        }
    }
}

// Staged placement, last level: position of x inside the 64-byte block jb of 16 range
// starts (the block's first start is its shared-memory sample, <= x). Padding past the
// last range is 0xFFFFFFFF, which only x = 0xFFFFFFFF passes; the clamp to n-1 maps that
// to the last range, which holds it anyway.
__device__ __forceinline__ uint32_t block_count(uint4 v, uint32_t x) {
    return (v.x <= x) + (v.y <= x) + (v.z <= x) + (v.w <= x);
}

__device__ __forceinline__ uint32_t staged_block_pos(const uint4* b, uint32_t jb, uint32_t x, uint32_t n) {
    const uint4 s0 = __ldg(b), s1 = __ldg(b + 1), s2 = __ldg(b + 2), s3 = __ldg(b + 3);
    const uint32_t c = block_count(s0, x) + block_count(s1, x) + block_count(s2, x) + block_count(s3, x);
    return min(jb * kBlockRanges + c - 1u, n - 1u);
}

// One classified record.
struct Item {
    uint32_t key;   // site*2+dir, or 2*n_sites + unmatched class
    uint32_t oc, pk, dur;
    bool elig, valid;
};

__device__ __forceinline__ Item classify(const AggParams& p, bool valid, bool sl, bool dl, uint32_t pk,
                                         uint32_t oc, uint32_t fi, uint32_t la, uint32_t site) {
    Item it;
    const uint32_t nk = 2u * p.n_sites;
    const uint32_t dir = sl ? 1u : 0u;  // outbound when the source is local
    const uint32_t dur = la - fi;       // modulo 2^32
    const bool mixed = sl != dl;        // exactly one endpoint local
    // registered: a site id below n_sites (kNoSite, and any id a caller's own registry
    // arrays hold beyond n_sites, count as unregistered, so keys stay below 2*n_sites + 4)
    const bool reg = site < p.n_sites;
    // unmatched classes: 0 neither local, 1 both local, 2 inbound unregistered, 3 outbound
    it.key = mixed ? (reg ? site * 2u + dir : nk + 2u + dir) : nk + dir;
    const bool ack_ok = (uint64_t)oc >= (uint64_t)p.min_avg * (uint64_t)pk;
    const bool many = pk >= p.min_pkts, longd = dur >= p.min_dur;
    const bool admin_ok = p.admin_rule == GNM_ADMIN_OR ? (many && longd) : (many || longd);
    it.elig = mixed && reg && dur != 0u && ack_ok && admin_ok;
    it.oc = oc;
    it.pk = pk;
    it.dur = dur;
    it.valid = valid;
    return it;
}

__device__ __forceinline__ void red_add(uint64_t* a, uint64_t v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(a), (unsigned long long)v);
}

// Adds summed contributions to a key's global accumulator row (5 u64 columns; column 0
// packs flows << 32 | e_flows, which cannot carry: a window holds < 2^32 records; column
// 1 holds the octets of ineligible flows, column 3 those of eligible ones).
__device__ __forceinline__ void row_add_sums(uint64_t* row, uint64_t packed, uint64_t neoc,
                                             uint64_t pk, uint64_t eoc, uint64_t edur, bool any_e) {
    red_add(row + 0, packed);
    red_add(row + 1, neoc);
    red_add(row + 2, pk);
    if (any_e) {
        red_add(row + 3, eoc);
        red_add(row + 4, edur);
    }
}

// Per-CTA sums in shared memory use 32-bit atomics (64-bit shared atomics serialise the
// lanes of a warp). A row is 5 words, stride 5 (odd, so random rows spread over the 32
// banks):
//   [0] flows (bits 0-15) | e_flows (bits 16-31)   [1] octets of ineligible flows
//   [2] pkts  [3] e_octets  [4] e_dur
// A flow's octets go to [1] or [3] (one atomic, its address picked per lane); the total
// is [1] + [3], formed at finalisation.
// The counts cannot wrap because a CTA flushes at least every kFlushRecords records. The
// sums keep their low 32 bits; the lane whose add wraps a word adds 2^32 to the key's
// global accumulator column directly (rare: a word wraps once per ~4 GB of octets), so
// every total stays exact.
constexpr int kRowWords = 5;
static_assert(kRowWords * 4 == kSmemRowBytes, "host and device disagree on the shared row size");

__device__ __forceinline__ void red32(uint32_t* a, uint32_t v) { atomicAdd(a, v); }

// lo += v (mod 2^32); a wrap adds 2^32 to the global column g (true then).
__device__ __forceinline__ bool add_wrap(uint32_t* lo, uint64_t* g, uint32_t v) {
    const uint32_t old = atomicAdd(lo, v);
    if (old <= ~v) return false;
    red_add(g, 1ull << 32);  // old + v >= 2^32
    return true;
}

__device__ __forceinline__ bool add_wrap64(uint32_t* lo, uint64_t* g, uint64_t v) {
    const uint32_t vl = (uint32_t)v;
    const uint32_t old = atomicAdd(lo, vl);
    const uint64_t h = (v >> 32) + (old > ~vl ? 1ull : 0ull);
    if (!h) return false;
    red_add(g, h << 32);
    return true;
}

struct Smem {
    uint32_t key_base;  // keys of the current segment are relative to it (partitioned launches)
    uint8_t* dirty;     // the window's dirty marks of 32-key accumulator groups, or null
    uint32_t slot;      // the window's result slot (its rate statistics are found from it:
                        // kept out of registers, they cost the hot loop nothing when off)
    uint32_t* t;        // table rows (kRowWords words each)
    uint32_t* tk;       // hash keys
    uint32_t rows;      // table rows
    const uint32_t* s_starts;
    const uint32_t* s_site;
    const uint32_t* s_dir; // kLookupSmem: directory over the top radix_bits bits, or null
    const uint16_t* dh;    // 16-bit block directory and samples (kLookupRadixBlk2H)
    const uint16_t* s16;
    const float* ra;    // learned index leaf arrays
    const float* rb;
    const uint32_t* rx0;
    const uint32_t* reps;
};

// Marks the accumulator group of `key` (relative to sm.key_base) as written; finalisation
// reads and clears only the rows of marked groups (the others are zero).
__device__ __forceinline__ void touch(const Smem& sm, uint32_t key) {
    if (sm.dirty) sm.dirty[(sm.key_base + key) >> 5] = 1;
}

// One record's contribution to shared-memory row r (gk: the key's global row).
__device__ __forceinline__ void srow_add(const Smem& sm, int r, const Item& it, uint64_t* gk) {
    uint32_t* w = sm.t + r * kRowWords;
    red32(w, it.elig ? 0x10001u : 1u);
    const int co = it.elig ? 3 : 1;
    bool g = add_wrap(w + co, gk + co, it.oc);
    g |= add_wrap(w + 2, gk + 2, it.pk);
    if (it.elig) g |= add_wrap(w + 4, gk + 4, it.dur);
    if (g) touch(sm, it.key);
}

__device__ __forceinline__ void srow_add_sums(const Smem& sm, int r, uint32_t key, uint32_t n, uint32_t ne,
                                              uint64_t oc, uint64_t pk, uint64_t eoc, uint64_t edur, uint64_t* gk) {
    uint32_t* w = sm.t + r * kRowWords;
    red32(w, n | (ne << 16));
    bool g = add_wrap64(w + 1, gk + 1, oc - eoc);
    g |= add_wrap64(w + 2, gk + 2, pk);
    if (ne) {
        g |= add_wrap64(w + 3, gk + 3, eoc);
        g |= add_wrap64(w + 4, gk + 4, edur);
    }
    if (g) touch(sm, key);
}

// srow_add for R items of a direct table (row = key) at once: every item's shared atomics
// are issued before any wrap check reads their results, so their latencies overlap; the rare
// wraps are handled after. The same per-atomic wrap test as srow_add, so the same sums.
template <int R>
__device__ __forceinline__ void srow_add_all(const Smem& sm, const Item (&it)[R], uint64_t* gacc) {
    uint32_t o1[R], o2[R], o4[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        o1[j] = 0u;
        o2[j] = 0u;
        o4[j] = 0u;
        if (it[j].valid) {
            uint32_t* w = sm.t + it[j].key * kRowWords;
            red32(w, it[j].elig ? 0x10001u : 1u);
            o1[j] = atomicAdd(w + (it[j].elig ? 3 : 1), it[j].oc);
            o2[j] = atomicAdd(w + 2, it[j].pk);
            if (it[j].elig) o4[j] = atomicAdd(w + 4, it[j].dur);
        }
    }
    // an add wrapped when old > ~v; records without an add have old = 0, which never does
    bool any = false;
#pragma unroll
    for (int j = 0; j < R; ++j) any |= (o1[j] > ~it[j].oc) | (o2[j] > ~it[j].pk) | (o4[j] > ~it[j].dur);
    if (!any) return;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        if (!it[j].valid) continue;
        uint64_t* gk = gacc + (size_t)it[j].key * kAccCols;
        const bool w1 = o1[j] > ~it[j].oc, w2 = o2[j] > ~it[j].pk, w4 = it[j].elig && o4[j] > ~it[j].dur;
        if (w1) red_add(gk + (it[j].elig ? 3 : 1), 1ull << 32);
        if (w2) red_add(gk + 2, 1ull << 32);
        if (w4) red_add(gk + 4, 1ull << 32);
        if (w1 || w2 || w4) touch(sm, it[j].key);
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
    h ^= h >> 15;
    h = __umulhi(h * 0x85EBCA6Bu, cap >> 1) << 1;  // even slot of a pair, any even cap
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

// Shared-memory row of `key` (-1: none).
template <int TABLE>
__device__ __forceinline__ int smem_row(const Smem& sm, uint32_t cap, uint32_t key) {
    if (TABLE == kTableDirect) return (int)key;
    return table_slot(sm.tk, cap, key);
}

// Sums of one item per lane over the lanes of `peers` (all share its key), added by the
// group leader to shared-memory row r, or, when r < 0, to the key's global row.
__device__ __forceinline__ void group_add(const Item& it, unsigned peers, int r, const Smem& sm,
                                          uint64_t* gacc) {
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
    uint64_t* gk = gacc + (size_t)it.key * kAccCols;
    if (r >= 0) {
        srow_add_sums(sm, r, it.key, n, ne, oc, pk, eoc, edur, gk);
    } else {
        touch(sm, it.key);
        row_add_sums(gk, ((uint64_t)n << 32) | ne, oc - eoc, pk, eoc, edur, ne != 0);
    }
}

// Accumulate one item per lane. Warp-collective: every lane of the warp calls it
// (invalid lanes with valid = false).
//   DIRECT aggregation: each lane adds to its key's shared-memory row; lanes whose key
//   has no row (cache full) are combined per key across the warp and added globally.
//   WARP aggregation: lanes are first combined per key; the group leader adds.
template <int TABLE, int AGG>
__device__ __forceinline__ void accumulate(const Item& it, const Smem& sm, uint32_t cap, uint64_t* gacc) {
    if (TABLE != kTableGlobal && AGG == GNM_AGG_DIRECT) {
        const int r = it.valid ? smem_row<TABLE>(sm, cap, it.key) : -1;
        const bool miss = it.valid && r < 0;
        if (TABLE == kTableHash && __any_sync(kFull, miss)) {
            const unsigned peers = __match_any_sync(kFull, miss ? it.key : kEmptyKey);
            if (miss) group_add(it, peers, -1, sm, gacc);
        }
        if (r >= 0) srow_add(sm, r, it, gacc + (size_t)it.key * kAccCols);
        return;
    }
    const unsigned peers = __match_any_sync(kFull, it.valid ? it.key : kEmptyKey);
    if (!it.valid) return;
    int r = -1;
    if (TABLE != kTableGlobal) {  // the leader probes for the whole group
        const int leader = __ffs(peers) - 1;
        int q = -1;
        if ((int)(threadIdx.x & 31u) == leader) q = smem_row<TABLE>(sm, cap, it.key);
        r = __shfl_sync(peers, q, leader);
    }
    group_add(it, peers, r, sm, gacc);
}

// Direct tables with a partial-sum area: the CTA stores its rows (as they are, 16-bit
// counts and low 32-bit sums) to its own block of the area, column by column (word c of
// row r at c * rows + r, so that finalisation reads each column coalesced), and clears
// them; the window's finalisation adds the blocks up. With a multiple of four rows (and so
// 16-byte aligned columns: blocks start 16-byte aligned), a thread takes four rows at a
// time: their 20 words are five 16-byte shared loads (the 80-byte groups of a quarter
// warp's lanes start in 8 different bank quads), transposed in registers into five 16-byte
// column words. Otherwise word by word (row stride 5 is odd: lanes reading consecutive rows
// of one column hit 32 different banks).
__device__ __forceinline__ void dump_rows(const Smem& sm, uint32_t* dst) {
    const uint32_t rows = sm.rows;
    if ((rows & 3u) == 0u) {
        const uint32_t g4 = rows >> 2, cs4 = rows >> 2;  // groups of four rows; column stride in uint4
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        for (uint32_t g = threadIdx.x; g < g4; g += blockDim.x) {
            uint4* q = reinterpret_cast<uint4*>(sm.t + g * 4u * kRowWords);  // rows 4g .. 4g+3
            const uint4 a = q[0], b = q[1], c = q[2], d = q[3], e = q[4];
            q[0] = z;
            q[1] = z;
            q[2] = z;
            q[3] = z;
            q[4] = z;
            uint4* o = reinterpret_cast<uint4*>(dst) + g;
            __stcg(o, make_uint4(a.x, b.y, c.z, d.w));
            __stcg(o + cs4, make_uint4(a.y, b.z, c.w, e.x));
            __stcg(o + 2u * cs4, make_uint4(a.z, b.w, d.x, e.y));
            __stcg(o + 3u * cs4, make_uint4(a.w, c.x, d.y, e.z));
            __stcg(o + 4u * cs4, make_uint4(b.x, c.y, d.z, e.w));
        }
        return;
    }
#pragma unroll 1
    for (int c = 0; c < kRowWords; ++c)
        for (uint32_t r = threadIdx.x; r < rows; r += blockDim.x) {
            __stcg(dst + (size_t)c * rows + r, sm.t[r * kRowWords + c]);
            sm.t[r * kRowWords + c] = 0;
        }
}

// Within a CTA's segment of a window whose rows go to a partial block at its end, between
// pieces of at most kCountPiece records: a row whose 16-bit flows or e_flows count has
// reached 2^15 adds its counts to the window's global accumulators and clears them. Every
// count then starts a piece below 2^15 and ends it below 2^15 + kCountPiece < 2^16, so
// none wraps; the sums (wrap-safe) keep accumulating, and rows with smaller counts too.
__device__ __forceinline__ void flush_counts(const Smem& sm, uint64_t* gacc) {
    for (uint32_t r = threadIdx.x; r < sm.rows; r += blockDim.x) {
        uint32_t* w = sm.t + r * kRowWords;
        const uint32_t cnt = w[0];
        if ((cnt & 0x80008000u) == 0u) continue;
        touch(sm, r);
        red_add(gacc + (size_t)r * kAccCols, ((uint64_t)(cnt & 0xFFFFu) << 32) | (cnt >> 16));
        w[0] = 0;
    }
}

// Adds the CTA's shared-memory sums to the window's global accumulators and clears them.
template <int TABLE>
__device__ __forceinline__ void flush(const Smem& sm, uint64_t* gacc) {
    for (uint32_t r = threadIdx.x; r < sm.rows; r += blockDim.x) {
        uint32_t* w = sm.t + r * kRowWords;
        uint32_t key = r;
        if (TABLE == kTableHash) {
            key = sm.tk[r];
            sm.tk[r] = kEmptyKey;
        }
        const uint32_t cnt = w[0];
        // a row can hold only wrap-carried sums (count 0 is impossible after an add)
        if (cnt == 0 && (w[1] | w[2] | w[3] | w[4]) == 0) continue;
        const uint32_t ef = cnt >> 16;
        touch(sm, key);
        row_add_sums(gacc + (size_t)key * kAccCols, ((uint64_t)(cnt & 0xFFFFu) << 32) | ef, w[1], w[2], w[3], w[4],
                     ef != 0 || (w[3] | w[4]) != 0);
#pragma unroll
        for (int c = 0; c < kRowWords; ++c) w[c] = 0;
    }
}

// IEEE 754 binary64 bits of the integer v rounded to nearest, ties to even, on the integer
// units: the leading 53 bits of v, rounded up when the bits shifted out exceed half a unit
// in the last place (or equal it and the kept last bit is odd).
__device__ __forceinline__ uint64_t f64_bits_rn(uint64_t v) {
    if (v == 0) return 0;
    const int e = 63 - __clzll((long long)v);  // position of the leading one
    uint64_t m;
    int ex = e;
    if (e <= 52) {
        m = v << (52 - e);
    } else {
        const int sh = e - 52;  // 1..11 bits shifted out
        m = v >> sh;
        const uint64_t rem = v & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (m & 1ull))) {
            ++m;
            if (m == (1ull << 53)) {
                m >>= 1;
                ++ex;
            }
        }
    }
    return ((uint64_t)(ex + 1023) << 52) | (m & ((1ull << 52) - 1ull));
}

// Bits of RN(RN(o) * 8000). RN(o) = m * 2^k with a 53-bit integer m, and m * 8000 =
// (m * 125) * 2^(k+6) with m * 125 < 2^60: the product rounds as the integer m * 125 does,
// then 2^(k+6) only moves the exponent (the result is at least 8000, far from the limits).
__device__ __forceinline__ uint64_t f64_bits_times8000(uint64_t o) {
    const uint64_t a = f64_bits_rn(o);
    if (a == 0) return 0;
    const uint64_t m = (a & ((1ull << 52) - 1ull)) | (1ull << 52);
    const int64_t k = (int64_t)(a >> 52) - 1075;
    return f64_bits_rn(m * 125u) + ((uint64_t)(k + 6) << 52);
}

// Bits of RN(a / b) for binary64 operands given as bits, a = 0 or normal, b normal and
// positive, with a quotient in the normal range (here: 2^-64 < a / b < 2^1000), formed on the
// integer and FP32 units (GB300 runs FP64 at 1/64 of the FP32 rate; a division per eligible
// flow in the per-flow rate statistics is on the aggregation's hot path).
// With a = ma * 2^ka and b = mb * 2^kb (53-bit significands ma, mb), the quotient's
// significand is Q = floor(ma * 2^s / mb) with s = 52 when ma >= mb and 53 otherwise, so that
// 2^52 <= Q < 2^53, and the remainder R decides the rounding (to nearest, ties to even) as in
// schoolbook division: Q + 1 when 2R > mb, or 2R = mb and Q is odd. Q is found digit by digit
// (10 bits a step, so R * 2^10 stays below 2^63); each digit is estimated from FP32 values
// within one of the true digit and corrected with the exact integer remainder. A remainder
// left outside [0, mb) would mean a digit more than one off; that case is reported (`ok`
// false) and the caller uses the FP64 division instead, so the result is exact either way.
__device__ __forceinline__ uint64_t f64_div_bits(uint64_t abits, uint64_t bbits, bool& ok) {
    ok = true;
    if (abits == 0) return 0;
    constexpr uint64_t kFrac = (1ull << 52) - 1ull;
    const uint64_t ma = (abits & kFrac) | (1ull << 52), mb = (bbits & kFrac) | (1ull << 52);
    const int ea = (int)(abits >> 52), eb = (int)(bbits >> 52);
    const bool ge = ma >= mb;
    const int s = ge ? 52 : 53;
    int64_t r = (int64_t)(ge ? ma - mb : ma);  // remainder, 0 <= r < mb
    uint64_t q = ge ? 1u : 0u;                  // quotient digits so far
    const int64_t d = (int64_t)mb;
    const float rd = __frcp_rn(__ull2float_rn(mb));
    bool bad = false;
    // five digits of 10 bits, then one of s - 50 (2 or 3) bits
    auto digit = [&](int c) {
        const float est = __ull2float_rn((uint64_t)r) * rd * (float)(1u << c);
        int64_t dig = (int64_t)min(__float2uint_rz(est), (1u << c) - 1u);
        int64_t nr = (r << c) - dig * d;  // |nr| < 2^63: r < 2^53, dig < 2^10
        if (nr < 0) {
            --dig;
            nr += d;
        } else if (nr >= d) {
            ++dig;
            nr -= d;
        }
        bad |= nr < 0 || nr >= d;
        q = (q << c) + (uint64_t)dig;
        r = nr;
    };
#pragma unroll
    for (int i = 0; i < 5; ++i) digit(10);
    digit(s - 50);
    if (bad) {
        ok = false;
        return 0;
    }
    const uint64_t r2 = (uint64_t)r << 1;
    if (r2 > mb || (r2 == mb && (q & 1ull))) ++q;
    int e = ea - eb - s + 52 + 1023;  // biased exponent of Q * 2^(ka - kb - s)
    if (q == (1ull << 53)) {
        q >>= 1;
        ++e;
    }
    return ((uint64_t)e << 52) | (q & kFrac);
}

// The FP64 division of two operands given as bits (out of line: rarely taken).
static __device__ __noinline__ double f64_div_fallback(uint64_t a, uint64_t b) {
    return __ddiv_rn(__longlong_as_double((long long)a), __longlong_as_double((long long)b));
}

// Rate from eligible octets and milliseconds, (RN(eo) * 8000) / RN(ed) with one rounding per
// operation (NaN when ed = 0): the conversions, the product and the division exact on the
// integer units, with the FP64 division as the fallback of f64_div_bits.
__device__ __forceinline__ double rate_of_sums(uint64_t eo, uint64_t ed) {
    if (!ed) return __longlong_as_double(0x7FF8000000000000ll);
    const uint64_t a = f64_bits_times8000(eo), b = f64_bits_rn(ed);
    bool ok;
    const uint64_t q = f64_div_bits(a, b, ok);
    return ok ? __longlong_as_double((long long)q) : f64_div_fallback(a, b);
}

// Rates and flags of one window from its accumulators (Sec. III.B.1: rates per site;
// a site is sub-optimal when its rate is below the standard). kL1: the sums were written
// by an earlier kernel, so loads may go through L1; inside the aggregation kernel they
// bypass L1. Partial blocks hold table_rows rows column by column.
// Partitioned launches (p.part_groups > 0): every key group of window `win` has its own
// run of partial blocks of table_rows rows (p.part_desc), and `parts`/`n_parts` are unused.
// `stage` (kNStat * 32 words of shared memory per warp, or null): a warp writes its 32
// keys' stats rows there and stores them as one contiguous run of 16-byte words.
template <bool kL1 = false>
__device__ __forceinline__ void finalize_rows(const AggParams& p, uint32_t slot, uint32_t k0,
                                              uint32_t step, const uint32_t* parts = nullptr,
                                              uint32_t n_parts = 0, uint32_t win = 0,
                                              uint64_t* stage = nullptr) {
    const uint32_t rows = p.table_rows;
    const uint64_t pstride = part_stride_words(rows);
    const size_t keys = p.keys;
    uint64_t* acc = p.acc + (size_t)slot * keys * kAccCols;
    uint64_t* st = p.stats + (size_t)slot * keys * kNStat;
    const uint32_t nk = 2u * p.n_sites;
    double* rate = p.rate + (size_t)slot * nk;
    uint8_t* flag = p.flag + (size_t)slot * nk;
    uint8_t* dg = p.dirty ? p.dirty + (size_t)slot * p.dirty_groups : nullptr;
    auto ld64 = [](const uint64_t* q) -> uint64_t {
        return kL1 ? *q : __ldcg(reinterpret_cast<const unsigned long long*>(q));
    };
    auto ld32 = [](const uint32_t* q) -> uint32_t { return kL1 ? __ldg(q) : __ldcg(q); };
    // k0 and step are such that a warp's lanes take the 32 keys of one group per pass (k0 is
    // a multiple of 32 plus the lane, step a multiple of 32); the loop is warp-uniform
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll 1
    for (uint32_t kb = k0 - lane; kb < keys; kb += step) {
        const uint32_t k = kb + lane;
        const bool act = k < keys;
        // the group's dirty mark, the first four partial blocks and (for a marked group) the
        // accumulator row are all loaded before any of them is used, so their latencies overlap
        const uint32_t mark = dg ? (kL1 ? dg[kb >> 5] : __ldcg(dg + (kb >> 5))) : 1u;
        uint64_t packed = 0, oc = 0, pk = 0, eo = 0, ed = 0;
        const uint32_t* kp = parts + k;
        uint32_t np = n_parts;
        if (act && p.part_groups) {
            const uint32_t g = k / rows;
            const uint2 pd = p.part_desc[(size_t)win * p.part_groups + g];
            kp = p.partials + (size_t)pd.x * pstride + (k - g * rows);
            np = p.partials ? pd.y : 0u;
            if (np && !chk(p.check_err, ((uint64_t)pd.x + np) * pstride <= p.partial_cap, kChkPartial, pd.x)) np = 0u;
        }
        if (!act) np = 0;
        uint32_t v[4][kRowWords];
        auto load4 = [&](uint32_t q0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t* w = kp + (size_t)(q0 + j) * pstride;
#pragma unroll
                for (int c = 0; c < kRowWords; ++c) v[j][c] = q0 + j < np ? ld32(w + (size_t)c * rows) : 0u;
            }
        };
        auto add4 = [&]() {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                packed += ((uint64_t)(v[j][0] & 0xFFFFu) << 32) | (v[j][0] >> 16);
                oc += v[j][1];
                pk += v[j][2];
                eo += v[j][3];
                ed += v[j][4];
            }
        };
        load4(0);
        // accumulator rows of an unmarked group are zero: neither read nor cleared
        const bool dirty = mark != 0u;
        uint64_t av[kAccCols] = {0, 0, 0, 0, 0};
        uint64_t* a = acc + (size_t)k * kAccCols;
        if (act && dirty) {
#pragma unroll
            for (int c = 0; c < kAccCols; ++c) av[c] = ld64(a + c);
        }
        add4();
        for (uint32_t q0 = 4; q0 < np; q0 += 4) {  // further partial blocks, four at a time
            load4(q0);
            add4();
        }
        __syncwarp();
        if (dg && dirty && lane == 0) dg[kb >> 5] = 0;
        uint64_t sv[kNStat] = {0, 0, 0, 0, 0, 0};
        if (act) {
            if (dirty) {
                packed += av[0];
                oc += av[1];
                pk += av[2];
                eo += av[3];
                ed += av[4];
                // accumulators return to zero for the slot's next window
#pragma unroll
                for (int c = 0; c < kAccCols; ++c) a[c] = 0;
            }
            const uint64_t ef = packed & 0xFFFFFFFFull;
            sv[0] = packed >> 32;
            sv[1] = oc + eo;  // ineligible and eligible flows' octets
            sv[2] = pk;
            sv[3] = ef;
            sv[4] = eo;
            sv[5] = ed;
            if (k < nk) {
                // rate = (octets * 8 bits) / (ms / 1000), one rounding per operation; the
                // conversions and the product are formed exactly on the integer units, the
                // division is the FP64 one (f64_div_bits made this kernel slower: 20 -> 22 us
                // on the hour, its FP64 divisions are not what bounds it)
                const double r = ed ? __ddiv_rn(__longlong_as_double((long long)f64_bits_times8000(eo)),
                                                __longlong_as_double((long long)f64_bits_rn(ed)))
                                    : __longlong_as_double(0x7FF8000000000000ll);
                rate[k] = r;
                flag[k] = (ef >= (uint64_t)p.min_flows && r < p.threshold) ? 1 : 0;
            }
        }
        if (stage) {  // the warp's keys [kb, kb + n) are kNStat * 8 * n contiguous bytes
            const uint32_t n = (uint32_t)min((size_t)32, keys - kb);
#pragma unroll
            for (int c = 0; c < kNStat; ++c) stage[lane * kNStat + c] = sv[c];
            __syncwarp();
            const uint4* src4 = reinterpret_cast<const uint4*>(stage);
            uint4* dst4 = reinterpret_cast<uint4*>(st + (size_t)kb * kNStat);
            for (uint32_t i = lane; i < n * (kNStat / 2); i += 32u) dst4[i] = src4[i];
            __syncwarp();
        } else if (act) {
            uint64_t* s = st + (size_t)k * kNStat;
#pragma unroll
            for (int c = 0; c < kNStat; ++c) s[c] = sv[c];
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


__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Shared-memory layout: [table values][hash keys][registry or leaf arrays].
__host__ __device__ inline size_t smem_layout(int lookup, int table, uint32_t n_ranges,
                                              uint32_t keys, uint32_t cap, uint32_t n_models,
                                              uint32_t radix_bits, size_t* off_keys, size_t* off_lookup) {
    const uint32_t rows = table == kTableDirect ? keys : (table == kTableHash ? cap : 0u);
    size_t o = (size_t)rows * kSmemRowBytes;
    *off_keys = o;
    if (table == kTableHash) o += (size_t)cap * 4;
    o = align_up(o, 16);
    *off_lookup = o;
    if (lookup == kLookupSmem) o += (size_t)n_ranges * 8 + (radix_bits ? (((size_t)1 << radix_bits) + 1) * 4 : 0);
    if (lookup == kLookupStaged) o += (size_t)((n_ranges + kBlockRanges - 1) / kBlockRanges) * 4;
    if (lookup == kLookupRmi) o += (size_t)n_models * 16;
    if (lookup == kLookupRadix) o += ((size_t)1 << radix_bits) * 4 + 4;
    return align_up(o, 16);
}

// Site of each remote address x[j] (kNoSite when unregistered) by the launch's lookup
// method; the R lookups advance together so their loads overlap.
template <int LOOKUP, int R>
__device__ __forceinline__ void lookup_sites(const AggParams& p, const Smem& sm, const bool (&valid)[R],
                                             const uint32_t (&x)[R], uint32_t (&site)[R]) {
    uint32_t idx[R];
    if (LOOKUP == kLookupSmem) {
        if (sm.s_dir) {  // a directory over the top radix_bits bits narrows the search first
            // the same number of steps for every lane (enough for the largest bucket), so the
            // loop has no per-lane exit; a step on a one-range interval keeps it
            uint32_t len[R];
            const bool packed = p.n_ranges < 65536u;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const uint32_t t = x[j] >> (32u - p.radix_bits);
                if (packed) {
                    const uint32_t e = sm.s_dir[t];
                    idx[j] = e & 0xFFFFu;
                    len[j] = (e >> 16) + 1u;
                } else {
                    idx[j] = sm.s_dir[t];
                    len[j] = sm.s_dir[t + 1] - idx[j] + 1u;
                }
                if (!chk(p.check_err, (uint64_t)idx[j] + len[j] <= p.n_ranges, kChkWindow, idx[j])) {
                    idx[j] = 0u;
                    len[j] = 1u;
                }
            }
#pragma unroll 1
            for (uint32_t it = 0; it < p.dir_iters; ++it) {
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const uint32_t half = len[j] >> 1;
                    idx[j] = sm.s_starts[idx[j] + half] <= x[j] ? idx[j] + half : idx[j];
                    len[j] -= half;
                }
            }
        } else {
            pred_search<R, true>(sm.s_starts, p.n_ranges, x, idx);
        }
#pragma unroll
        for (int j = 0; j < R; ++j) site[j] = sm.s_site[idx[j]];
    } else if (LOOKUP == kLookupL2) {
        if (p.pairs) {  // (the allocation-free entry point has plain arrays only)
            uint32_t len[R];
            const uint32_t s0 = __ldg(p.pairs).y;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                idx[j] = 0u;
                len[j] = p.n_ranges;
                site[j] = s0;
            }
            pair_search<R>(p.pairs, x, idx, len, site);
        } else {
            pred_search<R, false>(p.starts, p.n_ranges, x, idx);
#pragma unroll
            for (int j = 0; j < R; ++j) site[j] = __ldg(p.rsite + idx[j]);
        }
    } else if (LOOKUP == kLookupRadix) {
        // the directory gives x's bucket [dir[t], dir[t+1]] of ranges; search it
        uint32_t len[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const uint32_t t = p.radix_bits ? x[j] >> (32u - p.radix_bits) : 0u;
            idx[j] = sm.s_starts[t];
            len[j] = sm.s_starts[t + 1] - idx[j] + 1u;
            if (!chk(p.check_err, (uint64_t)idx[j] + len[j] <= p.n_ranges, kChkWindow, idx[j])) {
                idx[j] = 0u;
                len[j] = 1u;
            }
            site[j] = __ldg(p.pairs + idx[j]).y;
        }
        pair_search<R>(p.pairs, x, idx, len, site);
    } else if (LOOKUP == kLookupStaged) {
        pred_search<R, true>(sm.s_starts, p.n_blocks, x, idx);  // block of x
#pragma unroll
        for (int j = 0; j < R; ++j) idx[j] = staged_block_pos(p.blocks + 4 * (size_t)idx[j], idx[j], x[j], p.n_ranges);
#pragma unroll
        for (int j = 0; j < R; ++j) site[j] = __ldg(p.rsite + idx[j]);
    } else if (LOOKUP == kLookupRadixBlk) {
        radix_block<4, R>(sm.s_starts, p.radix_bits, sm.s_site, p.pairs, x, site, p.n_blk4 < 65536u, p.n_blk4,
                          p.check_err);
    } else if (LOOKUP == kLookupRadixBlk2) {
        radix_block<2, R>(sm.s_starts, p.radix_bits, sm.s_site, p.pairs, x, site, p.n_blk2 < 65536u, p.n_blk2,
                          p.check_err);
    } else if (LOOKUP == kLookupRadixBlk2H) {
        radix_block16<R>(sm.dh, sm.s16, p.pairs, x, site, p.n_blk2, p.check_err);
    } else if (LOOKUP == kLookupRmi) {
        rmi_sites<R>(p.rmi, sm.ra, sm.rb, sm.rx0, sm.reps, p.pairs, p.n_ranges, valid, x, site, p.violations);
    } else if (LOOKUP == kLookupHash24) {
        hash24_sites<R>(p.h24, p.h24_mask, x, site);
    }
}

// Key of a record: site*2+dir for a record between the local site and a registered
// site, else 2*n_sites + unmatched class (0 neither local, 1 both local, 2 inbound from
// an unregistered address, 3 outbound to one).
__device__ __forceinline__ uint32_t record_key(const AggParams& p, bool sl, bool dl, uint32_t site) {
    const uint32_t nk = 2u * p.n_sites;
    const uint32_t dir = sl ? 1u : 0u;  // outbound when the source is local
    const bool mixed = sl != dl;
    return mixed ? (site < p.n_sites ? site * 2u + dir : nk + 2u + dir) : nk + dir;
}

// A record whose key is already known (split launches: a lookup kernel wrote it).
__device__ __forceinline__ Item classify_key(const AggParams& p, bool valid, uint32_t key, uint32_t key_base,
                                             uint32_t pk, uint32_t oc, uint32_t fi, uint32_t la) {
    Item it;
    const uint32_t dur = la - fi;  // modulo 2^32
    const bool ack_ok = (uint64_t)oc >= (uint64_t)p.min_avg * (uint64_t)pk;
    const bool many = pk >= p.min_pkts, longd = dur >= p.min_dur;
    const bool admin_ok = p.admin_rule == GNM_ADMIN_OR ? (many && longd) : (many || longd);
    it.key = key;
    it.elig = key + key_base < 2u * p.n_sites && dur != 0u && ack_ok && admin_ok;
    it.oc = oc;
    it.pk = pk;
    it.dur = dur;
    it.valid = valid;
    return it;
}

// Per-flow rate statistics (Sec. III.B.2.1: minimum, maximum and the median's 10 kb/s
// histogram) of one eligible record of key `key`: bucket = min(10000, floor(4 o / (5 d))),
// rate = o * 8000 / d as in FP64 (one rounding per operation). Rates are >= 0, so their bit
// patterns order like the values; a read first skips the atomics that cannot change them.
static __device__ __noinline__ void rate_stat_add(const AggParams& p, const Smem& sm, uint32_t key, uint32_t oc,
                                                     uint32_t dur) {
    const uint64_t b = ((uint64_t)oc * 4u) / ((uint64_t)dur * 5u);
    const uint32_t bucket = b < 10000u ? (uint32_t)b : 10000u;
    const size_t k = (size_t)sm.slot * 2u * p.n_sites + sm.key_base + key;  // the key's statistics row
    if (p.rlog) {
        // sparse: append (key << 14 | bucket) to the window's log, one counter atomic per
        // group of lanes that arrive together (the host reserved a word per record)
        const cooperative_groups::coalesced_group g = cooperative_groups::coalesced_threads();
        uint32_t base = 0;
        if (g.thread_rank() == 0) base = atomicAdd(p.rlog_cnt + sm.slot, g.size());
        base = g.shfl(base, 0) + g.thread_rank();
        if (base < p.rlog_cap[sm.slot]) p.rlog[sm.slot][base] = ((sm.key_base + key) << 14) | bucket;
    } else {
        atomicAdd(p.hist + k * kRateBuckets + bucket, 1u);
    }
    const double r = rate_of_sums(oc, dur);  // (oc * 8000 is exact in FP64: below 2^45)
    const unsigned long long bits = (unsigned long long)__double_as_longlong(r);
    if (bits > __ldcg(p.rmax + k)) atomicMax(p.rmax + k, bits);
    if (bits < __ldcg(p.rmin + k)) atomicMin(p.rmin + k, bits);
}

// Processes R records per thread: lookups for all of them first (independent loads in
// flight together), then classification and accumulation. With LOOKUP == kLookupKeys the
// `src` field carries each record's precomputed key instead of an address.
template <int LOOKUP, int TABLE, int AGG, int R, bool STATS>
__device__ __forceinline__ void process(const AggParams& p, const Smem& sm, uint64_t* gacc,
                                        const bool (&valid)[R], const uint32_t (&src)[R],
                                        const uint32_t (&dst)[R], const uint32_t (&pk)[R],
                                        const uint32_t (&oc)[R], const uint32_t (&fi)[R],
                                        const uint32_t (&la)[R]) {
    // checked build: a key must name a row of the table and of the window's accumulators
    const uint32_t key_lim = TABLE == kTableDirect ? sm.rows : p.keys - sm.key_base;
    if constexpr (LOOKUP == kLookupKeys) {
        if constexpr (TABLE == kTableDirect && AGG == GNM_AGG_DIRECT) {
            Item its[R];
#pragma unroll
            for (int j = 0; j < R; ++j) {
                its[j] = classify_key(p, valid[j], src[j], sm.key_base, pk[j], oc[j], fi[j], la[j]);
                its[j].valid = its[j].valid && chk(p.check_err, its[j].key < key_lim, kChkKey, its[j].key);
            }
            srow_add_all<R>(sm, its, gacc);
            if (STATS && (p.hist || p.rlog)) {
#pragma unroll
                for (int j = 0; j < R; ++j)
                    if (its[j].valid && its[j].elig) rate_stat_add(p, sm, its[j].key, its[j].oc, its[j].dur);
            }
        } else {
#pragma unroll
            for (int j = 0; j < R; ++j) {
                Item it = classify_key(p, valid[j], src[j], sm.key_base, pk[j], oc[j], fi[j], la[j]);
                it.valid = it.valid && chk(p.check_err, it.key < key_lim, kChkKey, it.key);
                accumulate<TABLE, AGG>(it, sm, p.table_cap, gacc);
                if (STATS && (p.hist || p.rlog) && it.valid && it.elig) rate_stat_add(p, sm, it.key, it.oc, it.dur);
            }
        }
    } else {
        uint32_t x[R], site[R];
        bool sl[R], dl[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            local_pair(p, src[j], dst[j], sl[j], dl[j]);
            x[j] = sl[j] ? dst[j] : src[j];  // the remote endpoint
        }
        lookup_sites<LOOKUP, R>(p, sm, valid, x, site);
        if constexpr (TABLE == kTableDirect && AGG == GNM_AGG_DIRECT) {
            Item its[R];
#pragma unroll
            for (int j = 0; j < R; ++j) {
                its[j] = classify(p, valid[j], sl[j], dl[j], pk[j], oc[j], fi[j], la[j], site[j]);
                its[j].valid = its[j].valid && chk(p.check_err, its[j].key < key_lim, kChkKey, its[j].key);
            }
            srow_add_all<R>(sm, its, gacc);
            if (STATS && (p.hist || p.rlog)) {
#pragma unroll
                for (int j = 0; j < R; ++j)
                    if (its[j].valid && its[j].elig) rate_stat_add(p, sm, its[j].key, its[j].oc, its[j].dur);
            }
        } else {
#pragma unroll
            for (int j = 0; j < R; ++j) {
                Item it = classify(p, valid[j], sl[j], dl[j], pk[j], oc[j], fi[j], la[j], site[j]);
                it.valid = it.valid && chk(p.check_err, it.key < key_lim, kChkKey, it.key);
                accumulate<TABLE, AGG>(it, sm, p.table_cap, gacc);
                if (STATS && (p.hist || p.rlog) && it.valid && it.elig) rate_stat_add(p, sm, it.key, it.oc, it.dur);
            }
        }
    }
}

// Records [lo, hi) one per thread and slot (head/tail of a window, or unaligned arrays).
// STATS: the launch may keep per-flow rate statistics (when false, their code is left out:
// the hot loop then needs fewer registers). Regrouped records (no `first`) hold the
// duration in `last`.
template <int LOOKUP, int TABLE, int AGG, bool STATS>
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
            d[j] = LOOKUP == kLookupKeys ? 0u : ld_stream1(p.dst + ii);
            pk[j] = ld_stream1(p.pkts + ii);
            oc[j] = ld_stream1(p.oct + ii);
            fi[j] = p.first ? ld_stream1(p.first + ii) : 0u;
            la[j] = ld_stream1(p.last + ii);
        }
        process<LOOKUP, TABLE, AGG, 4, STATS>(p, sm, gacc, v, s, d, pk, oc, fi, la);
    }
}

// Records [a0, a0 + 4*G): G aligned groups of four, 16-byte vector loads.
//   U = 1, 2: U groups per thread and step, loaded together, then processed.
//   U = 3 (key launches): one group per thread and step; the next step's group is loaded
//   before this one is processed, so its memory latency overlaps the table atomics.
template <int LOOKUP, int TABLE, int AGG, int U, bool STATS>
__device__ __forceinline__ void vector_range(const AggParams& p, const Smem& sm, uint64_t* gacc,
                                             uint64_t a0, uint64_t G) {
    if constexpr (U == 3) {
        static_assert(LOOKUP == kLookupKeys, "pipelined groups read precomputed keys");
        const uint32_t B = blockDim.x;
        // lanes past the end load group 0 again (in bounds) and process nothing
        auto load = [&](uint64_t g, uint4& k, uint4& pk4, uint4& oc4, uint4& fi4, uint4& la4) {
            const uint64_t i = a0 + 4u * (g < G ? g : 0u);
            k = ld_stream4(p.src + i);
            pk4 = ld_stream4(p.pkts + i);
            oc4 = ld_stream4(p.oct + i);
            fi4 = p.first ? ld_stream4(p.first + i) : make_uint4(0, 0, 0, 0);
            la4 = ld_stream4(p.last + i);
        };
        uint4 ck, cp, co, cf, cl;
        load(threadIdx.x, ck, cp, co, cf, cl);
        for (uint64_t gb = 0; gb < G; gb += B) {  // uniform loop
            uint4 nk, np, no, nf, nl;
            load(gb + B + threadIdx.x, nk, np, no, nf, nl);
            const bool ok = gb + threadIdx.x < G;
            const bool v[4] = {ok, ok, ok, ok};
            const uint32_t s[4] = {ck.x, ck.y, ck.z, ck.w}, d[4] = {0u, 0u, 0u, 0u};
            const uint32_t pk[4] = {cp.x, cp.y, cp.z, cp.w}, oc[4] = {co.x, co.y, co.z, co.w};
            const uint32_t fi[4] = {cf.x, cf.y, cf.z, cf.w}, la[4] = {cl.x, cl.y, cl.z, cl.w};
            process<LOOKUP, TABLE, AGG, 4, STATS>(p, sm, gacc, v, s, d, pk, oc, fi, la);
            ck = nk;
            cp = np;
            co = no;
            cf = nf;
            cl = nl;
        }
    } else {
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
            const uint4 vs = ld_stream4(p.src + i);
            const uint4 vd = LOOKUP == kLookupKeys ? make_uint4(0, 0, 0, 0) : ld_stream4(p.dst + i);
            const uint4 vp = ld_stream4(p.pkts + i), vo = ld_stream4(p.oct + i);
            const uint4 vf = p.first ? ld_stream4(p.first + i) : make_uint4(0, 0, 0, 0);
            const uint4 vl = ld_stream4(p.last + i);
            s[4 * u + 0] = vs.x; s[4 * u + 1] = vs.y; s[4 * u + 2] = vs.z; s[4 * u + 3] = vs.w;
            d[4 * u + 0] = vd.x; d[4 * u + 1] = vd.y; d[4 * u + 2] = vd.z; d[4 * u + 3] = vd.w;
            pk[4 * u + 0] = vp.x; pk[4 * u + 1] = vp.y; pk[4 * u + 2] = vp.z; pk[4 * u + 3] = vp.w;
            oc[4 * u + 0] = vo.x; oc[4 * u + 1] = vo.y; oc[4 * u + 2] = vo.z; oc[4 * u + 3] = vo.w;
            fi[4 * u + 0] = vf.x; fi[4 * u + 1] = vf.y; fi[4 * u + 2] = vf.z; fi[4 * u + 3] = vf.w;
            la[4 * u + 0] = vl.x; la[4 * u + 1] = vl.y; la[4 * u + 2] = vl.z; la[4 * u + 3] = vl.w;
#pragma unroll
            for (int j = 0; j < 4; ++j) v[4 * u + j] = ok;
        }
        process<LOOKUP, TABLE, AGG, R, STATS>(p, sm, gacc, v, s, d, pk, oc, fi, la);
    }
    }
}

// Copies the lookup method's shared-memory structure (registry, block samples, radix
// directory or leaf parameters) to `base` and points `sm` at it.
template <int LOOKUP>
__device__ __forceinline__ void stage_lookup(const AggParams& p, unsigned char* base, Smem& sm) {
    const uint32_t tid = threadIdx.x, B = blockDim.x;
    if (LOOKUP == kLookupSmem) {
        uint32_t* st = reinterpret_cast<uint32_t*>(base);
        uint32_t* si = st + p.n_ranges;
        for (uint32_t i = tid; i < p.n_ranges; i += B) {
            st[i] = __ldg(p.starts + i);
            si[i] = __ldg(p.rsite + i);
        }
        sm.s_starts = st;
        sm.s_site = si;
        sm.s_dir = nullptr;
        if (p.radix_bits && p.dir16) {  // every 2^(16-bits)-th entry of the 16-bit directory
            uint32_t* d = si + p.n_ranges;
            const uint32_t nd = 1u << p.radix_bits, sh = 16u - p.radix_bits;
            if (p.n_ranges < 65536u) {  // one word per bucket: first range, ranges after it
                for (uint32_t i = tid; i < nd; i += B) {
                    const uint32_t r0 = __ldg(p.dir16 + ((size_t)i << sh));
                    const uint32_t r1 = __ldg(p.dir16 + ((size_t)(i + 1u) << sh));
                    d[i] = r0 | ((r1 - r0) << 16);
                }
            } else {
                for (uint32_t i = tid; i <= nd; i += B) d[i] = __ldg(p.dir16 + ((size_t)i << sh));
            }
            sm.s_dir = d;
        }
    }
    if (LOOKUP == kLookupStaged) {
        uint32_t* st = reinterpret_cast<uint32_t*>(base);
        for (uint32_t i = tid; i < p.n_blocks; i += B) st[i] = __ldg(p.sample + i);
        sm.s_starts = st;
    }
    if (LOOKUP == kLookupRadix) {  // every 2^(16-bits)-th entry of the 16-bit directory
        uint32_t* d = reinterpret_cast<uint32_t*>(base);
        const uint32_t nd = 1u << p.radix_bits, sh = 16u - p.radix_bits;
        for (uint32_t i = tid; i <= nd; i += B) d[i] = __ldg(p.dir16 + ((size_t)i << sh));
        sm.s_starts = d;
    }
    if (LOOKUP == kLookupRadixBlk || LOOKUP == kLookupRadixBlk2) {
        // block directory (from the range directory) and block samples
        constexpr uint32_t lg = LOOKUP == kLookupRadixBlk ? 2u : 1u;  // log2(ranges per block)
        const uint32_t* sample = LOOKUP == kLookupRadixBlk ? p.sample4 : p.sample2;
        const uint32_t nb = LOOKUP == kLookupRadixBlk ? p.n_blk4 : p.n_blk2;
        uint32_t* d = reinterpret_cast<uint32_t*>(base);
        const uint32_t nd = 1u << p.radix_bits, sh = 16u - p.radix_bits;
        if (nb < 65536u) {  // one word per bucket: first block (low 16 bits), blocks after it
            for (uint32_t i = tid; i < nd; i += B) {
                const uint32_t b0 = __ldg(p.dir16 + ((size_t)i << sh)) >> lg;
                const uint32_t b1 = __ldg(p.dir16 + ((size_t)(i + 1u) << sh)) >> lg;
                d[i] = b0 | ((b1 - b0) << 16);
            }
        } else {
            for (uint32_t i = tid; i <= nd; i += B) d[i] = __ldg(p.dir16 + ((size_t)i << sh)) >> lg;
        }
        uint32_t* smp = d + (((nd + 1u) + 3u) & ~3u);
        for (uint32_t i = tid; i < nb; i += B) smp[i] = __ldg(sample + i);
        sm.s_starts = d;
        sm.s_site = smp;  // (here: the block samples)
    }
    if (LOOKUP == kLookupRadixBlk2H) {  // 16-bit directory (65537 entries) and block samples
        uint32_t* d = reinterpret_cast<uint32_t*>(base);
        const uint32_t* gd = reinterpret_cast<const uint32_t*>(p.dirh);
        constexpr uint32_t nd = (65537u + 1u) / 2u;  // 32-bit words (the last one half used)
        for (uint32_t i = tid; i < nd; i += B) d[i] = i + 1u < nd ? __ldg(gd + i) : (uint32_t)__ldg(p.dirh + 65536);
        uint16_t* s = reinterpret_cast<uint16_t*>(base + (65537u * 2u + 15u) / 16u * 16u);
        for (uint32_t i = tid; i < p.n_blk2; i += B) s[i] = __ldg(p.smp16 + i);
        sm.dh = reinterpret_cast<const uint16_t*>(d);
        sm.s16 = s;
    }
    if (LOOKUP == kLookupRmi && p.rmi.leaves_global) {  // leaves read from global memory
        sm.ra = nullptr;
        sm.rb = nullptr;
        sm.rx0 = nullptr;
        sm.reps = nullptr;
    } else if (LOOKUP == kLookupRmi) {
        const uint32_t L = p.rmi.n_models;
        float* a = reinterpret_cast<float*>(base);
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
}

template <int LOOKUP, int TABLE, int AGG, int U, bool STATS = true>
__global__ void __launch_bounds__(agg_block_max(LOOKUP, TABLE, AGG, U))
    k_aggregate(const __grid_constant__ AggParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_last;
    const uint32_t tid = threadIdx.x, B = blockDim.x;

    const uint64_t lo = min((uint64_t)blockIdx.x * p.chunk, p.n_total);
    const uint64_t hi = min(lo + p.chunk, p.n_total);
    if (lo >= hi) return;  // whole CTA idle

    size_t off_keys, off_lookup;
    smem_layout(LOOKUP, TABLE, p.n_ranges, p.table_rows, p.table_cap,
                LOOKUP == kLookupRmi && !p.rmi.leaves_global ? p.rmi.n_models : 0u, p.radix_bits, &off_keys,
                &off_lookup);
    Smem sm;
    sm.key_base = 0u;
    sm.dirty = nullptr;
    sm.slot = 0u;
    sm.rows = TABLE == kTableDirect ? p.table_rows : (TABLE == kTableHash ? p.table_cap : 0u);
    sm.t = reinterpret_cast<uint32_t*>(smem_raw);
    sm.tk = reinterpret_cast<uint32_t*>(smem_raw + off_keys);
    // stage the table (zero; 16-byte stores, the table starts 16-byte aligned), the registry
    // or the leaf parameters
    {
        const uint32_t words = sm.rows * kRowWords, w4 = words >> 2;
        for (uint32_t i = tid; i < w4; i += B) reinterpret_cast<uint4*>(sm.t)[i] = make_uint4(0u, 0u, 0u, 0u);
        for (uint32_t i = 4u * w4 + tid; i < words; i += B) sm.t[i] = 0;
    }
    if (TABLE == kTableHash)
        for (uint32_t i = tid; i < p.table_cap; i += B) sm.tk[i] = kEmptyKey;
    stage_lookup<LOOKUP>(p, smem_raw + off_lookup, sm);
    __syncthreads();

    for (uint32_t w = first_window(p.wins, p.n_wins, lo); w < p.n_wins; ++w) {
        const WinDesc wd = p.wins[w];
        if (wd.begin >= hi) break;
        const uint64_t s0 = max(wd.begin, lo), e0 = min(wd.end, hi);
        // (a segment of a partitioned launch holds keys relative to its group's first key)
        uint64_t* gacc = p.acc + ((size_t)wd.slot * p.keys + wd.key_base) * kAccCols;
        sm.key_base = wd.key_base;
        sm.dirty = p.dirty ? p.dirty + (size_t)wd.slot * p.dirty_groups : nullptr;
        sm.slot = wd.slot;
        // pieces of at most kFlushRecords records, so the 16-bit counts cannot wrap. With a
        // partial-sum area the CTA's segment of the window ends in one block of its own
        // (block q = the CTA's position among the window's CTAs), and the pieces before
        // the last hand over only their counts
        const uint32_t q = (uint32_t)(blockIdx.x - wd.begin / p.chunk);
        const uint64_t piece = (TABLE == kTableDirect && p.partials) ? kCountPiece : kFlushRecords;
        for (uint64_t s = s0; s < e0; s += piece) {
            const uint64_t e = min(e0, s + piece);
            uint64_t a0 = e, a1 = e;
            if (p.vec_ok) {
                const uint32_t mis = (uint32_t)((s + p.phase) & 3u);
                a0 = mis ? min(s + (4u - mis), e) : s;
                a1 = a0 + ((e - a0) & ~3ull);
            }
            // (regrouped records, read by key launches only, hold the duration in `last`
            // and no `first`)
            scalar_range<LOOKUP, TABLE, AGG, STATS>(p, sm, gacc, s, a0);
            if (a1 > a0) vector_range<LOOKUP, TABLE, AGG, U, STATS>(p, sm, gacc, a0, (a1 - a0) >> 2);
            scalar_range<LOOKUP, TABLE, AGG, STATS>(p, sm, gacc, a1, e);
            if (TABLE != kTableGlobal) {
                __syncthreads();
                if (TABLE == kTableDirect && p.partials) {
                    if (e >= e0) {
                        if (chk(p.check_err,
                                ((uint64_t)wd.part_base + q + 1) * part_stride_words(sm.rows) <= p.partial_cap,
                                kChkPartial, (uint64_t)wd.part_base + q))
                            dump_rows(sm, p.partials + ((size_t)wd.part_base + q) * part_stride_words(sm.rows));
                    }
                    else
                        flush_counts(sm, gacc);
                } else {
                    flush<TABLE>(sm, gacc);
                }
                __syncthreads();
            }
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
        if (s_last && (wd.flags & kWinFinalize)) {
            if (TABLE == kTableDirect && p.partials)
                finalize_rows(p, wd.slot, tid, B, p.partials + (size_t)wd.part_base * part_stride_words(p.table_rows),
                              chk(p.check_err,
                                  ((uint64_t)wd.part_base + wd.n_parts) * part_stride_words(p.table_rows) <=
                                      p.partial_cap,
                                  kChkPartial, wd.part_base)
                                  ? wd.n_parts
                                  : 0u);
            else
                finalize_rows(p, wd.slot, tid, B);
        }
        __syncthreads();
    }
}

// Split launches, first kernel: the key of every record of [0, n_total) (lookups only;
// the shared memory holds just the lookup structure, so many CTAs fit per SM). The key
// array has the same 16-byte phase as the record arrays.
template <int LOOKUP, int U>
__global__ void __launch_bounds__(keys_block_max(LOOKUP, U)) k_keys(const __grid_constant__ AggParams p,
                                                                    uint32_t* __restrict__ keys) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem sm;
    sm.key_base = 0u;
    sm.dirty = nullptr;
    sm.slot = 0u;
    sm.t = nullptr;
    sm.tk = nullptr;
    sm.rows = 0;
    stage_lookup<LOOKUP>(p, smem_raw, sm);
    // partitioned launches: this CTA's record counts per (window, key group) bucket
    uint32_t* hist = p.key_hist ? reinterpret_cast<uint32_t*>(smem_raw + p.key_hist_off) : nullptr;
    const uint32_t nbk = p.key_hist ? p.n_wins * p.part_groups : 0u;
    for (uint32_t b = threadIdx.x; b < nbk; b += blockDim.x) hist[b] = 0u;
    __syncthreads();
    const uint64_t N = p.n_total;
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // bucket count of record i with key k (the lanes of a warp that share a bucket add once)
    uint32_t wcur = 0;
    auto count = [&](bool ok, uint64_t i, uint32_t k) {
        if (!hist) return;
        if (ok)
            while (wcur + 1 < p.n_wins && p.wins[wcur].end <= i) ++wcur;
        const uint32_t g = ok ? k / p.key_group_rows : 0u;
        const uint32_t b = ok ? wcur * p.part_groups + g : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, b);
        if (ok && chk(p.check_err, g < p.part_groups, kChkBucket, k) &&
            (threadIdx.x & 31u) == (uint32_t)(__ffs(peers) - 1))
            atomicAdd(hist + b, (uint32_t)__popc(peers));
    };
    uint64_t a0 = N, a1 = N;
    if (p.vec_ok) {
        const uint32_t mis = p.phase & 3u;
        a0 = mis ? min((uint64_t)(4u - mis), N) : 0;
        a1 = a0 + ((N - a0) & ~3ull);
    }
    // unaligned head and tail (at most 3 + 3 records), or every record when the arrays'
    // 16-byte phases differ
    const uint64_t ns = a0 + (N - a1);
    for (uint64_t tb = 0; tb < ns; tb += T) {  // uniform loop (the counts are warp-collective)
        const uint64_t t = tb + tid;
        const bool ok = t < ns;
        const uint64_t i = !ok ? 0u : (t < a0 ? t : a1 + (t - a0));
        uint32_t k = 0u;
        if (ok) {
            const uint32_t src = __ldcs(p.src + i), dst = __ldcs(p.dst + i);
            bool sl, dl;
            local_pair(p, src, dst, sl, dl);
            const bool v[1] = {true};
            const uint32_t x[1] = {sl ? dst : src};
            uint32_t site[1];
            lookup_sites<LOOKUP, 1>(p, sm, v, x, site);
            k = record_key(p, sl, dl, site[0]);
            keys[i] = k;
        }
        if (hist) {
            wcur = ok ? min(first_window(p.wins, p.n_wins, i), p.n_wins - 1u) : 0u;
            count(ok, i, k);
        }
    }
    constexpr int R = 4 * U;
    const uint64_t G = (a1 - a0) >> 2;
    if (hist && tid < G) wcur = min(first_window(p.wins, p.n_wins, a0 + 4u * tid), p.n_wins - 1u);
    // one group per thread: the next step's addresses are loaded before this step's
    // lookups, so that their memory latency overlaps them (two groups per thread have no
    // registers left for it)
    constexpr bool kPre = U == 1;
    uint4 pre_s = make_uint4(0, 0, 0, 0), pre_d = pre_s;
    auto fetch = [&](uint64_t gb) {
        const uint64_t g = gb + tid;
        const uint64_t i = a0 + 4u * (g < G ? g : 0u);
        pre_s = ld_stream4(p.src + i);
        pre_d = ld_stream4(p.dst + i);
    };
    if (kPre && G) fetch(0);
    for (uint64_t gb = 0; gb < G; gb += T * U) {
        bool v[R];
        uint32_t s[R], d[R], x[R], site[R];
        bool sl[R], dl[R];
        const uint4 cur_s = pre_s, cur_d = pre_d;
        if (kPre && gb + T < G) fetch(gb + T);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t g = gb + (uint64_t)u * T + tid;
            const bool ok = g < G;
            const uint64_t i = a0 + 4u * (ok ? g : 0u);
            const uint4 vs = kPre ? cur_s : ld_stream4(p.src + i), vd = kPre ? cur_d : ld_stream4(p.dst + i);
            s[4 * u + 0] = vs.x; s[4 * u + 1] = vs.y; s[4 * u + 2] = vs.z; s[4 * u + 3] = vs.w;
            d[4 * u + 0] = vd.x; d[4 * u + 1] = vd.y; d[4 * u + 2] = vd.z; d[4 * u + 3] = vd.w;
#pragma unroll
            for (int j = 0; j < 4; ++j) v[4 * u + j] = ok;
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
            local_pair(p, s[j], d[j], sl[j], dl[j]);
            x[j] = sl[j] ? d[j] : s[j];
        }
        lookup_sites<LOOKUP, R>(p, sm, v, x, site);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t g = gb + (uint64_t)u * T + tid;
            uint4 k;
            k.x = record_key(p, sl[4 * u + 0], dl[4 * u + 0], site[4 * u + 0]);
            k.y = record_key(p, sl[4 * u + 1], dl[4 * u + 1], site[4 * u + 1]);
            k.z = record_key(p, sl[4 * u + 2], dl[4 * u + 2], site[4 * u + 2]);
            k.w = record_key(p, sl[4 * u + 3], dl[4 * u + 3], site[4 * u + 3]);
            if (g < G) __stcg(reinterpret_cast<uint4*>(keys + a0 + 4u * g), k);
            if (hist) {  // (every lane takes part: the counts are warp-collective)
                const uint64_t i0 = a0 + 4u * g;  // (a thread's groups only grow: wcur only advances)
                count(g < G, i0, k.x);
                count(g < G, i0 + 1, k.y);
                count(g < G, i0 + 2, k.z);
                count(g < G, i0 + 3, k.w);
            }
        }
    }
    if (hist) {  // this CTA's counts to the launch's
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < nbk; b += blockDim.x)
            if (hist[b]) atomicAdd(p.key_hist + b, hist[b]);
    }
}

template <int LOOKUP>
cudaError_t launch_keys_impl(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st) {
    auto k = s.keys_unroll == 2 ? k_keys<LOOKUP, 2> : k_keys<LOOKUP, 1>;
    static OptInCache granted[2];  // per unroll variant
    cudaError_t e = ensure_smem_optin((const void*)k, (int)s.keys_smem, granted[s.keys_unroll == 2 ? 1 : 0]);
    if (e != cudaSuccess) return e;
    (void)cudaGetLastError();
    k<<<s.keys_grid, s.keys_block, s.keys_smem, st>>>(p, keys);
    return cudaGetLastError();
}

template <int LOOKUP, int TABLE, int AGG, int U>
cudaError_t launch_variant(const AggParams& p, const LaunchShape& s, cudaStream_t st) {
    auto k = k_aggregate<LOOKUP, TABLE, AGG, U>;
    static OptInCache granted, granted_plain;  // one per kernel
    OptInCache* g = &granted;
    // key launches without rate statistics (the hour workload, the regrouped window) take the
    // variant without their code
    if constexpr (LOOKUP == kLookupKeys)
        if (!p.hist && !p.rlog) {
            k = k_aggregate<LOOKUP, TABLE, AGG, U, false>;
            g = &granted_plain;
        }
    cudaError_t e = ensure_smem_optin((const void*)k, (int)s.smem, *g);
    if (e != cudaSuccess) return e;
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
    if constexpr (LOOKUP == kLookupKeys && TABLE == kTableDirect)
        if (s.unroll == 3) return launch_variant<LOOKUP, TABLE, GNM_AGG_DIRECT, 3>(p, s, st);
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
