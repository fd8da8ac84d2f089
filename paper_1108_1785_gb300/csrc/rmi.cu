// rmi.cu -- the learned index over the flattened range starts: GPU training of a
// two-stage recursive model index (Kraska et al., "The Case for Learned Index
// Structures", 2018) and its per-model error bounds.
//
// Not in the paper: it replaces the full search that assigns a record to a registered
// subnet (the paper's hash table, Sec. III.B.2.1, Sec. IV.A.1). Results stay exact:
// the lookup verifies the model window and falls back to the full binary search.
//
// Arithmetic (identical in training, the error sweep and inference):
//   xn = fl(fl(x) * 2^-32); root -> leaf = clamp(floor(root(xn)), 0, L-1)
//   split leaf -> sub-leaf min(((x - x0) mod 2^32) >> shift, count - 1)
//   d  = fl(int64(x) - int64(x0[m])); pos = clamp(floor(fl(fl(a*d) + b)), 0, n-1)
// Training:
//   root: mean squared error by gradient descent (linear, on a standardised input, so a
//         handful of steps reach the least-squares line) or Adam on mini-batches (the
//         1 -> H -> 1 ReLU MLP), on the training lookups and the plain search's positions;
//   leaves (minimax, default): each leaf's address interval [F, F') comes from the root by
//         bisection; its line minimises the worst-case error over the pieces of the ranges
//         inside the interval (convex in the slope: ternary search, max/min reductions);
//         a leaf whose window stays above the target is split into 2^k equal sub-leaves;
//   leaves (MSE): gradient descent per leaf on the training lookups it receives.
// Every reduction of the root and minimax paths is in a fixed order (per-block partials,
// then one ordered sum; max/min otherwise), so those models are reproducible bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "agg_kernel.cuh"

namespace gnm {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxRed = 3 * kMaxHidden + 2;  // widest reduction (MLP gradient + loss)
constexpr int kFitThreads = 128;
constexpr int kFitIters = 48;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Per-block sums of CNT per-thread doubles, in a fixed order: a shuffle tree per warp,
// then the warps in order; block b writes part[b * CNT + k]. k_sum_partials adds the
// blocks in order.
template <int CNT>
__device__ __forceinline__ void block_partials(const double (&v)[CNT], double* part) {
    __shared__ double sred[kWarps * CNT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < CNT; ++k) {
        const double s = warp_sum(v[k]);
        if (lane == 0) sred[warp * CNT + k] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < CNT; k += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sred[w * CNT + k];
        part[(size_t)blockIdx.x * CNT + k] = t;
    }
}

__global__ void k_sum_partials(const double* __restrict__ part, int nblk, int cnt, double* __restrict__ out) {
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < nblk; ++b) t += part[(size_t)b * cnt + k];
        out[k] = t;
    }
}

__device__ __forceinline__ float xnorm(uint32_t x) {
    return __fmul_rn(__uint2float_rn(x), 2.3283064365386963e-10f);
}

// ------------------------------------------------------------ linear stage (root)

// sum of xn and xn^2 (for standardisation)
__global__ void __launch_bounds__(kThreads) k_moments(const uint32_t* __restrict__ keys, uint64_t n, double* part) {
    double v[2] = {0.0, 0.0};
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const double x = (double)xnorm(__ldg(keys + i));
        v[0] += x;
        v[1] += x * x;
    }
    block_partials<2>(v, part);
}

// Forward + backward of yhat = w*z + c with z = (xn - mu) * inv_sigma and target
// y = pos * scale: sums of r*z, r and r^2.
__global__ void __launch_bounds__(kThreads) k_root_linear_grad(const uint32_t* __restrict__ keys,
                                                               const uint32_t* __restrict__ pos, uint64_t n,
                                                               float mu, float inv_sigma, float scale, float w,
                                                               float c, double* part) {
    double v[3] = {0.0, 0.0, 0.0};
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float z = __fmul_rn(__fsub_rn(xnorm(__ldg(keys + i)), mu), inv_sigma);
        const float y = __fmul_rn(__uint2float_rn(__ldg(pos + i)), scale);
        const float r = __fsub_rn(__fadd_rn(__fmul_rn(w, z), c), y);
        v[0] += (double)r * (double)z;
        v[1] += (double)r;
        v[2] += (double)r * (double)r;
    }
    block_partials<3>(v, part);
}

// The same gradient over explicit (z, y) samples, exposed through the C ABI.
__global__ void __launch_bounds__(kThreads) k_linear_grad(const float* __restrict__ z, const float* __restrict__ y,
                                                          uint64_t n, float w, float c, double* part) {
    double v[3] = {0.0, 0.0, 0.0};
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float zi = __ldg(z + i);
        const float r = __fsub_rn(__fadd_rn(__fmul_rn(w, zi), c), __ldg(y + i));
        v[0] += (double)r * (double)zi;
        v[1] += (double)r;
        v[2] += (double)r * (double)r;
    }
    block_partials<3>(v, part);
}

// ---------------------------------------------------------------- MLP root

// params: w1[H], b1[H], w2[H], b2 (FP32); per sample the terms of r*dout/dtheta and r^2.
template <int H>
__device__ __forceinline__ void mlp_sample(const float* p, float xn, float y, float (&g)[3 * H + 2]) {
    float pre[H], h[H];
    float out = 0.f;
#pragma unroll
    for (int j = 0; j < H; ++j) {
        pre[j] = __fadd_rn(__fmul_rn(p[j], xn), p[H + j]);
        h[j] = pre[j] > 0.f ? pre[j] : 0.f;
        out = __fadd_rn(out, __fmul_rn(p[2 * H + j], h[j]));
    }
    out = __fadd_rn(out, p[3 * H]);
    const float r = __fsub_rn(out, y);
#pragma unroll
    for (int j = 0; j < H; ++j) {
        const float gh = pre[j] > 0.f ? r * p[2 * H + j] : 0.f;  // d r^2 / 2 d h_j
        g[j] += gh * xn;
        g[H + j] += gh;
        g[2 * H + j] += r * h[j];
    }
    g[3 * H] += r;
    g[3 * H + 1] += r * r;
}

// Sums over samples of r*dout/dtheta and r^2 (r = out - y); the caller scales by 2/m
// (gradient) and 1/m (loss). Samples are either all (idx == nullptr) or a mini-batch of
// `n` hashed indices into [0, n_all).
template <int H>
__global__ void __launch_bounds__(kThreads) k_mlp_grad(const float* __restrict__ xs, const float* __restrict__ ys,
                                                       const uint32_t* __restrict__ keys,
                                                       const uint32_t* __restrict__ pos, float yscale,
                                                       uint64_t n, uint64_t n_all, uint64_t seed,
                                                       const float* __restrict__ params, double* part) {
    constexpr int CNT = 3 * H + 2;
    __shared__ float sp[3 * H + 1];
    for (int k = threadIdx.x; k < 3 * H + 1; k += blockDim.x) sp[k] = params[k];
    __syncthreads();
    float g[CNT];
#pragma unroll
    for (int k = 0; k < CNT; ++k) g[k] = 0.f;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        float xn, y;
        if (xs) {
            xn = __ldg(xs + i);
            y = __ldg(ys + i);
        } else {
            // mini-batch element i: SplitMix64 mix of (seed, i), reduced to [0, n_all)
            uint64_t z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            const uint64_t j = (uint64_t)(((unsigned __int128)z * n_all) >> 64);
            xn = xnorm(__ldg(keys + j));
            y = __fmul_rn(__uint2float_rn(__ldg(pos + j)), yscale);
        }
        mlp_sample<H>(sp, xn, y, g);
    }
    double v[CNT];
#pragma unroll
    for (int k = 0; k < CNT; ++k) v[k] = (double)g[k];
    block_partials<CNT>(v, part);
}

// Adam update of the 3H+1 MLP parameters from summed gradients (scaled by 2/m here).
__global__ void k_adam(float* params, float* m, float* v, const double* gsum, int cnt, double inv_m,
                       float lr, float b1, float b2, float eps, int step) {
    const int k = threadIdx.x;
    if (k >= cnt) return;
    const float g = (float)(2.0 * gsum[k] * inv_m);
    m[k] = b1 * m[k] + (1.f - b1) * g;
    v[k] = b2 * v[k] + (1.f - b2) * g * g;
    const float mh = m[k] / (1.f - powf(b1, (float)step));
    const float vh = v[k] / (1.f - powf(b2, (float)step));
    params[k] -= lr * mh / (sqrtf(vh) + eps);
}

// ------------------------------------------------------- leaves: mean squared error

__global__ void k_route(const RmiDev m, const uint32_t* __restrict__ keys, uint64_t n, uint32_t* __restrict__ leaf,
                        uint32_t* __restrict__ x0) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = __ldg(keys + i);
        const uint32_t l = dev::rmi_root(m, x);
        leaf[i] = l;
        atomicMin(x0 + l, x);
    }
}

// per leaf: count, sum d, sum d^2 (d relative to the leaf's smallest key, so d >= 0)
__global__ void k_leaf_moments(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ leaf, uint64_t n,
                               const uint32_t* __restrict__ x0, double* mom) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t l = __ldg(leaf + i);
        const double d = (double)dev::rel_offset(__ldg(keys + i), __ldg(x0 + l));
        atomicAdd(mom + 3 * (size_t)l, 1.0);
        atomicAdd(mom + 3 * (size_t)l + 1, d);
        atomicAdd(mom + 3 * (size_t)l + 2, d * d);
    }
}

// Standardisation of every leaf: mu, 1/sigma (1/sigma = 0 for a single distinct d).
__global__ void k_leaf_standardise(const double* mom, uint32_t L, float* mu, float* isd) {
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    const double c = mom[3 * l];
    if (c == 0.0) {
        mu[l] = 0.f;
        isd[l] = 0.f;
        return;
    }
    const double m = mom[3 * l + 1] / c;
    const double var = mom[3 * l + 2] / c - m * m;
    mu[l] = (float)m;
    isd[l] = var > 1e-12 ? (float)(1.0 / sqrt(var)) : 0.f;
}

// Forward + backward of every leaf's line yhat = w_l * z + c_l: per-leaf sums of r*z,
// r and r^2, with r = yhat - pos.
__global__ void k_leaf_grad(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ pos,
                            const uint32_t* __restrict__ leaf, uint64_t n, const uint32_t* __restrict__ x0,
                            const float* __restrict__ mu, const float* __restrict__ isd,
                            const float* __restrict__ w, const float* __restrict__ c, double* acc) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t l = __ldg(leaf + i);
        const float d = dev::rel_offset(__ldg(keys + i), __ldg(x0 + l));
        const float z = __fmul_rn(__fsub_rn(d, __ldg(mu + l)), __ldg(isd + l));
        const float r = __fsub_rn(__fadd_rn(__fmul_rn(__ldg(w + l), z), __ldg(c + l)), __uint2float_rn(__ldg(pos + i)));
        atomicAdd(acc + 3 * (size_t)l, (double)r * (double)z);
        atomicAdd(acc + 3 * (size_t)l + 1, (double)r);
        atomicAdd(acc + 3 * (size_t)l + 2, (double)r * (double)r);
    }
}

// Gradient step of every leaf (learning rate lr on the mean squared error).
__global__ void k_leaf_step(const double* acc, const double* mom, uint32_t L, float lr, float* w, float* c) {
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    const double m = mom[3 * l];
    if (m == 0.0) return;
    w[l] -= lr * (float)(2.0 * acc[3 * l] / m);
    c[l] -= lr * (float)(2.0 * acc[3 * l + 1] / m);
}

// Fold the standardisation into the leaf line: pos = a*d + b (a >= 0: monotone).
__global__ void k_leaf_fold(const double* mom, uint32_t L, uint32_t n_ranges, const float* mu, const float* isd,
                            const float* w, const float* c, float* a, float* b, uint32_t* x0) {
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    if (mom[3 * l] == 0.0) {  // no training key reached this leaf
        a[l] = 0.f;
        b[l] = (float)((double)l * n_ranges / L);
        x0[l] = 0u;
        return;
    }
    double sl = (double)w[l] * (double)isd[l];
    if (sl < 0.0) sl = 0.0;
    a[l] = (float)sl;
    b[l] = (float)((double)c[l] - sl * (double)mu[l]);
}

// ----------------------------------------------------------- leaves: minimax

// first[l] = smallest address whose leaf is >= l (bisection over [0, 2^32] on the
// root, which is monotone for the linear root); first[0] = 0, first[L] = 2^32.
__global__ void k_leaf_first(const RmiDev m, uint32_t L, unsigned long long* first) {
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l > L) return;
    uint64_t lo = 0, hi = 1ull << 32;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (dev::rmi_root(m, (uint32_t)mid) >= l) hi = mid;
        else lo = mid + 1;
    }
    first[l] = l == 0 ? 0ull : lo;
}

__device__ __forceinline__ float block_max(float v, float* s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = s[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, s[w]);
    return r;
}

__device__ __forceinline__ float block_min(float v, float* s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = s[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fminf(r, s[w]);
    return r;
}

// Piece k of the ranges inside [F, G): offsets (from F) of its first and last address.
__device__ __forceinline__ void piece(const uint32_t* __restrict__ starts, uint32_t n, uint32_t i, uint64_t F,
                                      uint64_t G, float& dlo, float& dhi) {
    const uint64_t s = __ldg(starts + i);
    const uint64_t e = i + 1 < n ? (uint64_t)__ldg(starts + i + 1) : (1ull << 32);
    dlo = (float)((s > F ? s : F) - F);
    dhi = (float)((e < G ? e : G) - 1 - F);
}

// Minimax line of every interval [lo[i], hi[i]) (one CTA per interval): the slope a >= 0
// minimising E(a) = (G(a) - H(a)) / 2 with G(a) = max_k (t_k - a*dlo_k) and
// H(a) = min_k (t_k - a*dhi_k) over the pieces k of the ranges inside the interval
// (t_k = k), by ternary search over [0, (count - 1) / widest piece]; then c = (G + H) / 2.
// Output in the library's convention: pos = floor(a*d + b) with b = i0 + c + 0.5 (i0 the
// interval's first range), and E.
__global__ void __launch_bounds__(kFitThreads) k_fit_minimax(const uint32_t* __restrict__ starts, uint32_t n,
                                                             const unsigned long long* __restrict__ ivl_lo,
                                                             const unsigned long long* __restrict__ ivl_hi,
                                                             uint32_t count, float* out_a, float* out_b,
                                                             float* out_e) {
    __shared__ float s[kFitThreads / 32];
    for (uint32_t iv = blockIdx.x; iv < count; iv += gridDim.x) {
        const uint64_t F = ivl_lo[iv], G = ivl_hi[iv];
        if (F >= G) {
            if (threadIdx.x == 0) {
                out_a[iv] = 0.f;
                out_b[iv] = 0.f;
                out_e[iv] = 0.f;
            }
            continue;
        }
        const uint32_t i0 = dev::pred_search1(starts, 0, n, (uint32_t)F);
        const uint32_t i1 = dev::pred_search1(starts, 0, n, (uint32_t)(G - 1));
        const uint32_t cnt = i1 - i0 + 1;
        float wmax = 0.f;
        for (uint32_t k = threadIdx.x; k < cnt; k += blockDim.x) {
            float dlo, dhi;
            piece(starts, n, i0 + k, F, G, dlo, dhi);
            wmax = fmaxf(wmax, dhi - dlo);
        }
        wmax = block_max(wmax, s);
        float alo = 0.f, ahi = (float)(cnt - 1) / fmaxf(wmax, 1.f);
        for (int it = 0; it < kFitIters; ++it) {
            const float m1 = alo + (ahi - alo) / 3.f, m2 = ahi - (ahi - alo) / 3.f;
            float g1 = -INFINITY, h1 = INFINITY, g2 = -INFINITY, h2 = INFINITY;
            for (uint32_t k = threadIdx.x; k < cnt; k += blockDim.x) {
                float dlo, dhi;
                piece(starts, n, i0 + k, F, G, dlo, dhi);
                const float t = (float)k;
                g1 = fmaxf(g1, t - m1 * dlo);
                h1 = fminf(h1, t - m1 * dhi);
                g2 = fmaxf(g2, t - m2 * dlo);
                h2 = fminf(h2, t - m2 * dhi);
            }
            g1 = block_max(g1, s);
            h1 = block_min(h1, s);
            g2 = block_max(g2, s);
            h2 = block_min(h2, s);
            if (g1 - h1 < g2 - h2) ahi = m2;
            else alo = m1;
        }
        const float a = 0.5f * (alo + ahi);
        float g = -INFINITY, h = INFINITY;
        for (uint32_t k = threadIdx.x; k < cnt; k += blockDim.x) {
            float dlo, dhi;
            piece(starts, n, i0 + k, F, G, dlo, dhi);
            g = fmaxf(g, (float)k - a * dlo);
            h = fminf(h, (float)k - a * dhi);
        }
        g = block_max(g, s);
        h = block_min(h, s);
        if (threadIdx.x == 0) {
            out_a[iv] = a;
            out_b[iv] = __fadd_rn((float)i0, 0.5f * (g + h) + 0.5f);
            out_e[iv] = 0.5f * (g - h);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- error bounds

__device__ __forceinline__ void flush_eps(uint32_t l, uint32_t lo, uint32_t hi, uint32_t* elo, uint32_t* ehi) {
    if (lo) atomicMax(elo + l, lo);
    if (hi) atomicMax(ehi + l, hi);
}

// Exhaustive sweep over every 32-bit address: per model, the largest amount by which the
// predicted position exceeds (eps_lo) or falls short of (eps_hi) the true position.
__global__ void __launch_bounds__(kThreads) k_eps_sweep(const RmiDev m, const uint32_t* __restrict__ starts,
                                                        uint32_t n, uint32_t* elo, uint32_t* ehi) {
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t per = ((1ull << 32) + T - 1) / T;
    const uint64_t xa = tid * per;
    const uint64_t xb = (xa + per < (1ull << 32)) ? xa + per : (1ull << 32);
    if (xa >= xb) return;
    uint32_t t = dev::pred_search1(starts, 0, n, (uint32_t)xa);
    uint64_t next = t + 1 < n ? (uint64_t)__ldg(starts + t + 1) : (1ull << 32);
    uint32_t cl = 0xFFFFFFFFu, cur = 0xFFFFFFFFu, mlo = 0, mhi = 0;
    dev::RmiLeaf lf{0.f, 0.f, 0u, 0u}, f{0.f, 0.f, 0u, 0u};
    for (uint64_t x = xa; x < xb; ++x) {
        while (x >= next) {
            ++t;
            next = t + 1 < n ? (uint64_t)__ldg(starts + t + 1) : (1ull << 32);
        }
        const uint32_t l = dev::rmi_root(m, (uint32_t)x);
        if (l != cl) {
            cl = l;
            lf = dev::rmi_leaf(m, m.a, m.b, m.x0, m.eps, l);
        }
        const uint32_t md = lf.eps == kEpsSplit ? dev::rmi_sub_model(lf, (uint32_t)x) : l;
        if (md != cur) {
            if (cur != 0xFFFFFFFFu) flush_eps(cur, mlo, mhi, elo, ehi);
            cur = md;
            mlo = mhi = 0;
            f = md == l ? lf : dev::rmi_leaf(m, m.a, m.b, m.x0, m.eps, md);
        }
        const uint32_t p = dev::rmi_leaf_pos(f, (uint32_t)x, n);
        if (p > t) mlo = max(mlo, p - t);
        else mhi = max(mhi, t - p);
    }
    flush_eps(cur, mlo, mhi, elo, ehi);
}

// Error bounds from the training samples only.
__global__ void k_eps_samples(const RmiDev m, const uint32_t* __restrict__ keys, const uint32_t* __restrict__ pos,
                              uint64_t n_s, uint32_t n, uint32_t* elo, uint32_t* ehi) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_s; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = __ldg(keys + i), t = __ldg(pos + i);
        const uint32_t l = dev::rmi_root(m, x);
        const dev::RmiLeaf lf = dev::rmi_leaf(m, m.a, m.b, m.x0, m.eps, l);
        const uint32_t md = lf.eps == kEpsSplit ? dev::rmi_sub_model(lf, x) : l;
        const dev::RmiLeaf f = md == l ? lf : dev::rmi_leaf(m, m.a, m.b, m.x0, m.eps, md);
        const uint32_t p = dev::rmi_leaf_pos(f, x, n);
        flush_eps(md, p > t ? p - t : 0u, t > p ? t - p : 0u, elo, ehi);
    }
}

// Packed bounds of every model (split leaves keep their marker).
__global__ void k_pack_eps(const uint32_t* lo, const uint32_t* hi, uint32_t* packed, uint32_t M) {
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= M || packed[l] == kEpsSplit) return;
    packed[l] = (lo[l] > 0xFFFEu || hi[l] > 0xFFFEu) ? 0xFFFFFFFFu : (lo[l] | (hi[l] << 16));
}

// Model parameters interleaved for lookups that read them from global memory.
__global__ void k_pack_leaf4(const float* a, const float* b, const uint32_t* x0, const uint32_t* eps, uint4* out,
                             uint32_t M) {
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= M) return;
    out[l] = make_uint4(__float_as_uint(a[l]), __float_as_uint(b[l]), x0[l], eps[l]);
}

// Over the training lookups: squared error of the predicted position and the width of
// the model window searched (the whole registry where no bound holds).
__global__ void __launch_bounds__(kThreads) k_model_stats(const RmiDev m, const uint32_t* __restrict__ keys,
                                                          const uint32_t* __restrict__ pos, uint64_t n_s,
                                                          uint32_t n, double* part) {
    double v[2] = {0.0, 0.0};
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_s; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = __ldg(keys + i);
        const dev::RmiLeaf f = dev::rmi_model(m, m.a, m.b, m.x0, m.eps, x);
        const double r = (double)dev::rmi_leaf_pos(f, x, n) - (double)__ldg(pos + i);
        v[0] += r * r;
        v[1] += f.eps == 0xFFFFFFFFu ? (double)n : (double)((f.eps & 0xFFFFu) + (f.eps >> 16) + 1u);
    }
    block_partials<2>(v, part);
}

int grid_for(uint64_t n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (n + kThreads - 1) / kThreads;
    const uint64_t cap = (uint64_t)sms * 8;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

template <int H>
cudaError_t launch_mlp_grad(const float* xs, const float* ys, const uint32_t* keys, const uint32_t* pos,
                            float yscale, uint64_t n, uint64_t n_all, uint64_t seed, const float* params,
                            double* part, double* out, cudaStream_t st) {
    const int g = grid_for(n);
    k_mlp_grad<H><<<g, kThreads, 0, st>>>(xs, ys, keys, pos, yscale, n, n_all, seed, params, part);
    k_sum_partials<<<1, 128, 0, st>>>(part, g, 3 * H + 2, out);
    return cudaGetLastError();
}

cudaError_t mlp_grad_dispatch(uint32_t hidden, const float* xs, const float* ys, const uint32_t* keys,
                              const uint32_t* pos, float yscale, uint64_t n, uint64_t n_all, uint64_t seed,
                              const float* params, double* part, double* out, cudaStream_t st) {
    switch (hidden) {
        case 8: return launch_mlp_grad<8>(xs, ys, keys, pos, yscale, n, n_all, seed, params, part, out, st);
        case 16: return launch_mlp_grad<16>(xs, ys, keys, pos, yscale, n, n_all, seed, params, part, out, st);
        case 32: return launch_mlp_grad<32>(xs, ys, keys, pos, yscale, n, n_all, seed, params, part, out, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// --------------------------------------------------------------- host side

size_t rmi_partials_bytes() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return ((size_t)sms * 8 * kMaxRed + kMaxRed) * sizeof(double);
}

struct TrainScratch {
    uint32_t* leaf;     // [n]
    double* red;        // ordered sums [kMaxRed]
    double* part;       // per-block partials [grid][kMaxRed]
    double* mom;        // [3L]
    double* acc;        // [3L]
    float *mu, *isd, *w, *c;  // [L]
    float *la, *lb;           // [L] MSE leaf lines
    uint32_t* lx0;            // [L]
    unsigned long long* first;  // [L + 1]
    float *mp, *mm, *mv;      // MLP params / Adam state [3*32+1]
};

static size_t carve_bytes(uint64_t n, uint32_t L, TrainScratch* s, void* base) {
    char* p = (char*)base;
    size_t used = 0;
    auto take = [&](size_t bytes) {
        char* r = p ? p + used : nullptr;
        used += (bytes + 255) / 256 * 256;
        return (void*)r;
    };
    TrainScratch t;
    t.leaf = (uint32_t*)take(n * 4);
    t.red = (double*)take(kMaxRed * 8);
    t.part = (double*)take(rmi_partials_bytes());
    t.mom = (double*)take((size_t)L * 3 * 8);
    t.acc = (double*)take((size_t)L * 3 * 8);
    t.mu = (float*)take((size_t)L * 4);
    t.isd = (float*)take((size_t)L * 4);
    t.w = (float*)take((size_t)L * 4);
    t.c = (float*)take((size_t)L * 4);
    t.la = (float*)take((size_t)L * 4);
    t.lb = (float*)take((size_t)L * 4);
    t.lx0 = (uint32_t*)take((size_t)L * 4);
    t.first = (unsigned long long*)take((size_t)(L + 1) * 8);
    t.mp = (float*)take(128 * 4);
    t.mm = (float*)take(128 * 4);
    t.mv = (float*)take(128 * 4);
    if (s) *s = t;
    return used;
}

size_t rmi_train_scratch_bytes(uint64_t n, uint32_t L) { return carve_bytes(n, L, nullptr, nullptr) + 1024; }

#define RMI_CU(x)                              \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return e_;      \
    } while (0)

namespace {

// Minimax lines of `lo.size()` intervals on the device (synchronous; host vectors out).
cudaError_t fit_intervals(const uint32_t* starts, uint32_t n, const std::vector<unsigned long long>& lo,
                          const std::vector<unsigned long long>& hi, std::vector<float>& a, std::vector<float>& b,
                          std::vector<float>& e, cudaStream_t st) {
    const size_t k = lo.size();
    a.assign(k, 0.f);
    b.assign(k, 0.f);
    e.assign(k, 0.f);
    if (k == 0) return cudaSuccess;
    void* buf = nullptr;
    RMI_CU(cudaMalloc(&buf, k * (8 + 8 + 4 + 4 + 4)));
    unsigned long long* dlo = (unsigned long long*)buf;
    unsigned long long* dhi = dlo + k;
    float* da = (float*)(dhi + k);
    float* db = da + k;
    float* de = db + k;
    cudaError_t r = cudaMemcpyAsync(dlo, lo.data(), k * 8, cudaMemcpyHostToDevice, st);
    if (r == cudaSuccess) r = cudaMemcpyAsync(dhi, hi.data(), k * 8, cudaMemcpyHostToDevice, st);
    if (r == cudaSuccess) {
        const uint32_t grid = (uint32_t)std::min<size_t>(k, 65535);
        k_fit_minimax<<<grid, kFitThreads, 0, st>>>(starts, n, dlo, dhi, (uint32_t)k, da, db, de);
        r = cudaGetLastError();
    }
    if (r == cudaSuccess) r = cudaMemcpyAsync(a.data(), da, k * 4, cudaMemcpyDeviceToHost, st);
    if (r == cudaSuccess) r = cudaMemcpyAsync(b.data(), db, k * 4, cudaMemcpyDeviceToHost, st);
    if (r == cudaSuccess) r = cudaMemcpyAsync(e.data(), de, k * 4, cudaMemcpyDeviceToHost, st);
    if (r == cudaSuccess) r = cudaStreamSynchronize(st);
    cudaFree(buf);
    return r;
}

// Window width expected from a minimax error E: each side rounds to about E + 0.5 after
// the floor, plus the FP32 rounding of the prediction.
inline bool window_ok(float E, uint32_t target) { return target == 0 || 2.f * E + 3.f <= (float)target; }

// Minimax leaves with split leaves (host orchestration of k_leaf_first and
// k_fit_minimax): fills the model arrays of `out`.
cudaError_t minimax_leaves(const RmiDev& m, const uint32_t* starts, uint32_t n_ranges, const gnm_rmi_config& cfg,
                           unsigned long long* d_first, RmiTrainOut* out, cudaStream_t st) {
    const uint32_t L = m.n_leaves;
    k_leaf_first<<<(L + 1 + 255) / 256, 256, 0, st>>>(m, L, d_first);
    RMI_CU(cudaGetLastError());
    std::vector<unsigned long long> first(L + 1);
    RMI_CU(cudaMemcpyAsync(first.data(), d_first, (size_t)(L + 1) * 8, cudaMemcpyDeviceToHost, st));
    RMI_CU(cudaStreamSynchronize(st));
    for (uint32_t l = 0; l < L; ++l)
        if (first[l] > first[l + 1]) return cudaErrorNotSupported;
    std::vector<unsigned long long> lo(first.begin(), first.end() - 1), hi(first.begin() + 1, first.end());
    std::vector<float> la, lb, le;
    RMI_CU(fit_intervals(starts, n_ranges, lo, hi, la, lb, le, st));
    // split leaves: try 2, 4, 8, ... sub-leaves per failing leaf until every sub-leaf fits
    struct Split {
        uint32_t shift = 0, count = 0;
        std::vector<float> a, b;
        std::vector<uint32_t> x0;
    };
    std::vector<Split> split(L);
    std::vector<uint32_t> failing;
    for (uint32_t l = 0; l < L; ++l)
        if (!window_ok(le[l], cfg.eps_target) && hi[l] - lo[l] > 1) failing.push_back(l);
    const uint32_t max_r = std::min<uint32_t>(cfg.max_split_log2, 16);
    uint64_t n_sub = 0;
    for (uint32_t r = 1; r <= max_r && !failing.empty(); ++r) {
        std::vector<unsigned long long> slo, shi;
        std::vector<uint32_t> sh(failing.size()), cnt(failing.size());
        for (size_t i = 0; i < failing.size(); ++i) {
            const uint32_t l = failing[i];
            const uint64_t W = hi[l] - lo[l];
            uint32_t lg = 0;
            while ((1ull << lg) < W) ++lg;
            sh[i] = lg > r ? lg - r : 0u;
            cnt[i] = (uint32_t)((W + (1ull << sh[i]) - 1) >> sh[i]);
            for (uint32_t j = 0; j < cnt[i]; ++j) {
                slo.push_back(lo[l] + ((uint64_t)j << sh[i]));
                shi.push_back(std::min<unsigned long long>(lo[l] + ((uint64_t)(j + 1) << sh[i]), hi[l]));
            }
        }
        if (n_sub + slo.size() + L > kMaxModels) break;  // keep the last accepted splits
        std::vector<float> sa, sb, se;
        RMI_CU(fit_intervals(starts, n_ranges, slo, shi, sa, sb, se, st));
        std::vector<uint32_t> still;
        size_t o = 0;
        for (size_t i = 0; i < failing.size(); ++i) {
            const uint32_t l = failing[i];
            bool ok = true;
            for (uint32_t j = 0; j < cnt[i]; ++j) ok = ok && window_ok(se[o + j], cfg.eps_target);
            if (ok || sh[i] == 0 || r == max_r) {
                if (split[l].count) n_sub -= split[l].count;
                Split& s = split[l];
                s.shift = sh[i];
                s.count = cnt[i];
                s.a.assign(sa.begin() + o, sa.begin() + o + cnt[i]);
                s.b.assign(sb.begin() + o, sb.begin() + o + cnt[i]);
                s.x0.resize(cnt[i]);
                for (uint32_t j = 0; j < cnt[i]; ++j) s.x0[j] = (uint32_t)slo[o + j];
                n_sub += cnt[i];
            }
            if (!ok && sh[i] > 0 && r < max_r) still.push_back(l);
            o += cnt[i];
        }
        failing.swap(still);
    }
    // models: leaves, then the sub-leaves of split leaves in leaf order
    const uint32_t M = L + (uint32_t)n_sub;
    out->a.assign(M, 0.f);
    out->b.assign(M, 0.f);
    out->x0.assign(M, 0u);
    out->eps.assign(M, 0u);
    out->split.assign(L, 0u);
    out->empty_leaves = 0;
    out->split_leaves = 0;
    uint32_t nxt = L;
    for (uint32_t l = 0; l < L; ++l) {
        const uint32_t fx = (uint32_t)std::min<unsigned long long>(lo[l], 0xFFFFFFFFull);
        out->x0[l] = fx;
        out->empty_leaves += lo[l] >= hi[l];
        if (split[l].count) {
            const Split& s = split[l];
            const uint32_t w = s.shift | ((s.count - 1) << 8);
            std::memcpy(&out->a[l], &w, 4);
            std::memcpy(&out->b[l], &nxt, 4);
            out->eps[l] = kEpsSplit;
            out->split[l] = w;
            ++out->split_leaves;
            for (uint32_t j = 0; j < s.count; ++j, ++nxt) {
                out->a[nxt] = s.a[j];
                out->b[nxt] = s.b[j];
                out->x0[nxt] = s.x0[j];
            }
        } else {
            out->a[l] = la[l];
            out->b[l] = lb[l];
        }
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t rmi_train_device(RmiDev* m, const uint32_t* keys, const uint32_t* pos, uint64_t n,
                             const uint32_t* starts, uint32_t n_ranges, const gnm_rmi_config& cfg, void* scratch,
                             RmiTrainOut* out, cudaStream_t st) {
    const uint32_t L = cfg.n_leaves;
    TrainScratch s;
    carve_bytes(n, L, &s, scratch);
    const int g = grid_for(n);
    double h[kMaxRed];
    // ---- root
    m->n_leaves = L;
    m->root_kind = cfg.root_kind;
    m->hidden = cfg.hidden;
    const float yscale_root = (float)((double)L / n_ranges);
    if (cfg.root_kind == GNM_RMI_ROOT_LINEAR) {
        k_moments<<<g, kThreads, 0, st>>>(keys, n, s.part);
        k_sum_partials<<<1, 128, 0, st>>>(s.part, g, 2, s.red);
        RMI_CU(cudaMemcpyAsync(h, s.red, 16, cudaMemcpyDeviceToHost, st));
        RMI_CU(cudaStreamSynchronize(st));
        const double mu = h[0] / n, var = h[1] / n - mu * mu;
        const double sd = var > 1e-30 ? sqrt(var) : 1.0;
        float w = 0.f, c = 0.f;
        double loss = 0.0;
        for (uint32_t it = 0; it <= cfg.leaf_iters; ++it) {
            k_root_linear_grad<<<g, kThreads, 0, st>>>(keys, pos, n, (float)mu, (float)(1.0 / sd), yscale_root, w, c,
                                                      s.part);
            k_sum_partials<<<1, 128, 0, st>>>(s.part, g, 3, s.red);
            RMI_CU(cudaMemcpyAsync(h, s.red, 24, cudaMemcpyDeviceToHost, st));
            RMI_CU(cudaStreamSynchronize(st));
            loss = h[2] / n;
            if (it == cfg.leaf_iters) break;
            w -= 0.5f * (float)(2.0 * h[0] / n);
            c -= 0.5f * (float)(2.0 * h[1] / n);
        }
        double ra = (double)w / sd;
        if (ra < 0) ra = 0;
        m->ra = (float)ra;
        m->rb = (float)((double)c - ra * mu);
        out->root_loss = loss;
    } else {
        const int H = (int)cfg.hidden;
        const int cnt = 3 * H + 1;
        float p[3 * 32 + 1];
        // knots spread over [0, 1): h_j = relu(xn - j/H); the output layer learns the CDF
        uint64_t r = cfg.seed * 0x9E3779B97F4A7C15ull + 1;
        for (int j = 0; j < H; ++j) {
            r ^= r << 13; r ^= r >> 7; r ^= r << 17;
            const float u = (float)((r >> 11) * (1.0 / 9007199254740992.0));
            p[j] = 1.0f;
            p[H + j] = -(float)j / H;
            p[2 * H + j] = (u - 0.5f) * 0.02f;
        }
        p[3 * H] = 0.f;
        RMI_CU(cudaMemcpyAsync(s.mp, p, cnt * 4, cudaMemcpyHostToDevice, st));
        RMI_CU(cudaMemsetAsync(s.mm, 0, 128 * 4, st));
        RMI_CU(cudaMemsetAsync(s.mv, 0, 128 * 4, st));
        const uint64_t batch = cfg.mlp_batch < n ? cfg.mlp_batch : n;
        const float ys = (float)(1.0 / n_ranges);  // targets in [0, 1): position / n
        for (uint32_t step = 1; step <= cfg.mlp_steps; ++step) {
            RMI_CU(mlp_grad_dispatch(cfg.hidden, nullptr, nullptr, keys, pos, ys, batch, n,
                                     cfg.seed * 1000003ull + step, s.mp, s.part, s.red, st));
            k_adam<<<1, 128, 0, st>>>(s.mp, s.mm, s.mv, s.red, cnt, 1.0 / batch, cfg.mlp_lr, 0.9f, 0.999f, 1e-8f,
                                      (int)step);
        }
        // final loss over all samples (in leaf units)
        RMI_CU(mlp_grad_dispatch(cfg.hidden, nullptr, nullptr, keys, pos, ys, n, n, 0, s.mp, s.part, s.red, st));
        RMI_CU(cudaMemcpyAsync(p, s.mp, cnt * 4, cudaMemcpyDeviceToHost, st));
        RMI_CU(cudaMemcpyAsync(h, s.red, (3 * H + 2) * 8, cudaMemcpyDeviceToHost, st));
        RMI_CU(cudaStreamSynchronize(st));
        out->root_loss = h[3 * H + 1] / n * (double)L * L;
        for (int j = 0; j < H; ++j) {
            m->w1[j] = p[j];
            m->b1[j] = p[H + j];
            m->w2[j] = p[2 * H + j] * (float)L;  // output rescaled from [0,1) to leaf units
        }
        for (int j = H; j < 32; ++j) m->w1[j] = m->b1[j] = m->w2[j] = 0.f;
        m->b2 = p[3 * H] * (float)L;
    }
    // ---- leaves (minimax needs contiguous leaf intervals: a root whose leaf boundaries
    // come out unordered takes the MSE leaves)
    if (cfg.leaf_fit == GNM_RMI_FIT_MINIMAX) {
        const cudaError_t e = minimax_leaves(*m, starts, n_ranges, cfg, s.first, out, st);
        if (e != cudaErrorNotSupported) return e;
    }
    RMI_CU(cudaMemsetAsync(s.lx0, 0xFF, (size_t)L * 4, st));
    RmiDev route = *m;
    k_route<<<g, kThreads, 0, st>>>(route, keys, n, s.leaf, s.lx0);
    RMI_CU(cudaMemsetAsync(s.mom, 0, (size_t)L * 3 * 8, st));
    k_leaf_moments<<<g, kThreads, 0, st>>>(keys, s.leaf, n, s.lx0, s.mom);
    const int gl = (int)((L + 255) / 256);
    k_leaf_standardise<<<gl, 256, 0, st>>>(s.mom, L, s.mu, s.isd);
    RMI_CU(cudaMemsetAsync(s.w, 0, (size_t)L * 4, st));
    RMI_CU(cudaMemsetAsync(s.c, 0, (size_t)L * 4, st));
    for (uint32_t it = 0; it < cfg.leaf_iters; ++it) {
        RMI_CU(cudaMemsetAsync(s.acc, 0, (size_t)L * 3 * 8, st));
        k_leaf_grad<<<g, kThreads, 0, st>>>(keys, pos, s.leaf, n, s.lx0, s.mu, s.isd, s.w, s.c, s.acc);
        k_leaf_step<<<gl, 256, 0, st>>>(s.acc, s.mom, L, 0.5f, s.w, s.c);
    }
    k_leaf_fold<<<gl, 256, 0, st>>>(s.mom, L, n_ranges, s.mu, s.isd, s.w, s.c, s.la, s.lb, s.lx0);
    RMI_CU(cudaGetLastError());
    out->a.assign(L, 0.f);
    out->b.assign(L, 0.f);
    out->x0.assign(L, 0u);
    out->eps.assign(L, 0u);
    out->split.assign(L, 0u);
    std::vector<double> hmom((size_t)L * 3);
    RMI_CU(cudaMemcpyAsync(out->a.data(), s.la, (size_t)L * 4, cudaMemcpyDeviceToHost, st));
    RMI_CU(cudaMemcpyAsync(out->b.data(), s.lb, (size_t)L * 4, cudaMemcpyDeviceToHost, st));
    RMI_CU(cudaMemcpyAsync(out->x0.data(), s.lx0, (size_t)L * 4, cudaMemcpyDeviceToHost, st));
    RMI_CU(cudaMemcpyAsync(hmom.data(), s.mom, (size_t)L * 3 * 8, cudaMemcpyDeviceToHost, st));
    RMI_CU(cudaStreamSynchronize(st));
    out->empty_leaves = 0;
    out->split_leaves = 0;
    for (uint32_t l = 0; l < L; ++l) out->empty_leaves += hmom[3 * l] == 0.0;
    return cudaSuccess;
}

cudaError_t rmi_eps_sweep(const RmiDev& m, const uint32_t* starts, uint32_t n, uint32_t* elo, uint32_t* ehi,
                          int sm_count, cudaStream_t st) {
    RMI_CU(cudaMemsetAsync(elo, 0, (size_t)m.n_models * 4, st));
    RMI_CU(cudaMemsetAsync(ehi, 0, (size_t)m.n_models * 4, st));
    k_eps_sweep<<<sm_count * 8, kThreads, 0, st>>>(m, starts, n, elo, ehi);
    return cudaGetLastError();
}

cudaError_t rmi_eps_from_samples(const RmiDev& m, const uint32_t* keys, const uint32_t* pos, uint64_t n_s,
                                 uint32_t n, uint32_t* elo, uint32_t* ehi, cudaStream_t st) {
    RMI_CU(cudaMemsetAsync(elo, 0, (size_t)m.n_models * 4, st));
    RMI_CU(cudaMemsetAsync(ehi, 0, (size_t)m.n_models * 4, st));
    k_eps_samples<<<grid_for(n_s), kThreads, 0, st>>>(m, keys, pos, n_s, n, elo, ehi);
    return cudaGetLastError();
}

cudaError_t rmi_pack_leaf4(const float* a, const float* b, const uint32_t* x0, const uint32_t* eps, uint4* out,
                           uint32_t M, cudaStream_t st) {
    k_pack_leaf4<<<(M + 255) / 256, 256, 0, st>>>(a, b, x0, eps, out, M);
    return cudaGetLastError();
}

cudaError_t rmi_pack_eps(const uint32_t* lo, const uint32_t* hi, uint32_t* packed, uint32_t M, cudaStream_t st) {
    k_pack_eps<<<(M + 255) / 256, 256, 0, st>>>(lo, hi, packed, M);
    return cudaGetLastError();
}

cudaError_t rmi_model_stats(const RmiDev& m, const uint32_t* keys, const uint32_t* pos, uint64_t n_s, uint32_t n,
                            double* part, double* out2, cudaStream_t st) {
    const int g = grid_for(n_s);
    k_model_stats<<<g, kThreads, 0, st>>>(m, keys, pos, n_s, n, part);
    k_sum_partials<<<1, 128, 0, st>>>(part, g, 2, out2);
    return cudaGetLastError();
}

cudaError_t rmi_linear_grad(const float* z, const float* y, uint64_t n, float w, float c, double* part, double* acc3,
                            cudaStream_t st) {
    const int g = grid_for(n);
    k_linear_grad<<<g, kThreads, 0, st>>>(z, y, n, w, c, part);
    k_sum_partials<<<1, 128, 0, st>>>(part, g, 3, acc3);
    return cudaGetLastError();
}

cudaError_t rmi_mlp_grad(const float* xn, const float* y, uint64_t n, uint32_t hidden, const float* params,
                         double* part, double* grad, cudaStream_t st) {
    return mlp_grad_dispatch(hidden, xn, y, nullptr, nullptr, 1.f, n, n, 0, params, part, grad, st);
}

}  // namespace gnm
