// rmi.cu -- the learned index over the flattened range starts: GPU training of a
// two-stage recursive model index (Kraska et al., "The Case for Learned Index
// Structures", 2018) and its per-leaf error bounds.
//
// Not in the paper: it replaces the full search that assigns a record to a registered
// subnet (the paper's hash table, Sec. III.B.2.1, Sec. IV.A.1). Results stay exact:
// the lookup verifies the model window and falls back to the full binary search.
//
// Arithmetic (identical in training, the error sweep and inference):
//   xn = fl(fl(x) * 2^-32); root -> leaf = clamp(floor(root(xn)), 0, L-1)
//   d  = fl(int64(x) - int64(x0[leaf])); pos = clamp(floor(fl(fl(a*d) + b)), 0, n-1)
// Training minimises the mean squared error of each stage by gradient descent: the
// linear stages on a standardised input (so a handful of steps reach the least-squares
// line), the MLP root (1 -> H -> 1, ReLU) with Adam on mini-batches.
#include <cuda_runtime.h>
#include <stdint.h>

#include "agg_kernel.cuh"

namespace gnm {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Sums of `cnt` per-thread doubles over the block, added atomically to out[0..cnt).
template <int CNT>
__device__ __forceinline__ void block_add(const double (&v)[CNT], double* out, double* sred) {
    for (int k = threadIdx.x; k < CNT; k += blockDim.x) sred[k] = 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < CNT; ++k) {
        const double s = warp_sum(v[k]);
        if ((threadIdx.x & 31) == 0) atomicAdd(sred + k, s);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < CNT; k += blockDim.x) atomicAdd(out + k, sred[k]);
}

__device__ __forceinline__ float xnorm(uint32_t x) {
    return __fmul_rn(__uint2float_rn(x), 2.3283064365386963e-10f);
}

// ------------------------------------------------------------ linear stage (root)

// sum of xn and xn^2 (for standardisation)
__global__ void k_moments(const uint32_t* __restrict__ keys, uint64_t n, double* out2) {
    __shared__ double sred[2];
    double v[2] = {0.0, 0.0};
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const double x = (double)xnorm(__ldg(keys + i));
        v[0] += x;
        v[1] += x * x;
    }
    block_add<2>(v, out2, sred);
}

// Forward + backward of yhat = w*z + c with z = (xn - mu) * inv_sigma and target
// y = pos * scale: accumulates sum(r*z), sum(r), sum(r^2).
__global__ void k_root_linear_grad(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ pos,
                                   uint64_t n, float mu, float inv_sigma, float scale, float w, float c,
                                   double* out3) {
    __shared__ double sred[3];
    double v[3] = {0.0, 0.0, 0.0};
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float z = __fmul_rn(__fsub_rn(xnorm(__ldg(keys + i)), mu), inv_sigma);
        const float y = __fmul_rn(__uint2float_rn(__ldg(pos + i)), scale);
        const float r = __fsub_rn(__fadd_rn(__fmul_rn(w, z), c), y);
        v[0] += (double)r * (double)z;
        v[1] += (double)r;
        v[2] += (double)r * (double)r;
    }
    block_add<3>(v, out3, sred);
}

// The same gradient over explicit (z, y) samples, exposed through the C ABI.
__global__ void k_linear_grad(const float* __restrict__ z, const float* __restrict__ y, uint64_t n, float w,
                              float c, double* out3) {
    __shared__ double sred[3];
    double v[3] = {0.0, 0.0, 0.0};
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float zi = __ldg(z + i);
        const float r = __fsub_rn(__fadd_rn(__fmul_rn(w, zi), c), __ldg(y + i));
        v[0] += (double)r * (double)zi;
        v[1] += (double)r;
        v[2] += (double)r * (double)r;
    }
    block_add<3>(v, out3, sred);
}

// ---------------------------------------------------------------- MLP root

// params: w1[H], b1[H], w2[H], b2 (FP32); grad: same layout, then the loss (FP64 sums of
// 2/m * dL terms are formed on the host side of the call by scaling).
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
                                                       const float* __restrict__ params, double* out) {
    constexpr int CNT = 3 * H + 2;
    __shared__ float sp[3 * H + 1];
    __shared__ double sred[CNT];
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
    block_add<CNT>(v, out, sred);
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

// ----------------------------------------------------------------- leaves

__global__ void k_route(const RmiDev m, const uint32_t* __restrict__ keys, uint64_t n, uint32_t* __restrict__ leaf,
                        uint32_t* __restrict__ x0) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = __ldg(keys + i);
        const uint32_t l = dev::rmi_root(m, x);
        leaf[i] = l;
        atomicMin(x0 + l, x);
    }
}

// per leaf: count, sum d, sum d^2 (d relative to the leaf's smallest key)
__global__ void k_leaf_moments(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ leaf, uint64_t n,
                               const uint32_t* __restrict__ x0, double* mom) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t l = __ldg(leaf + i);
        const double d = (double)__ll2float_rn((long long)__ldg(keys + i) - (long long)__ldg(x0 + l));
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
        const float d = __ll2float_rn((long long)__ldg(keys + i) - (long long)__ldg(x0 + l));
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

// ---------------------------------------------------------------- error bounds

__device__ __forceinline__ void flush_eps(uint32_t l, uint32_t lo, uint32_t hi, uint32_t* elo, uint32_t* ehi) {
    if (lo) atomicMax(elo + l, lo);
    if (hi) atomicMax(ehi + l, hi);
}

// Exhaustive sweep over every 32-bit address: per leaf, the largest amount by which the
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
    uint32_t cur = 0xFFFFFFFFu, mlo = 0, mhi = 0;
    float ca = 0.f, cb = 0.f;
    uint32_t cx0 = 0;
    for (uint64_t x = xa; x < xb; ++x) {
        while (x >= next) {
            ++t;
            next = t + 1 < n ? (uint64_t)__ldg(starts + t + 1) : (1ull << 32);
        }
        const uint32_t l = dev::rmi_root(m, (uint32_t)x);
        if (l != cur) {
            if (cur != 0xFFFFFFFFu) flush_eps(cur, mlo, mhi, elo, ehi);
            cur = l;
            mlo = mhi = 0;
            ca = __ldg(m.a + l);
            cb = __ldg(m.b + l);
            cx0 = __ldg(m.x0 + l);
        }
        const float d = __ll2float_rn((long long)x - (long long)cx0);
        const uint32_t p = dev::clamp_floor(__fadd_rn(__fmul_rn(ca, d), cb), n);
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
        const dev::RmiLeaf f{__ldg(m.a + l), __ldg(m.b + l), __ldg(m.x0 + l), 0u};
        const uint32_t p = dev::rmi_leaf_pos(f, x, n);
        flush_eps(l, p > t ? p - t : 0u, t > p ? t - p : 0u, elo, ehi);
    }
}

__global__ void k_pack_eps(const uint32_t* lo, const uint32_t* hi, uint32_t* packed, uint32_t L) {
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    packed[l] = (lo[l] > 0xFFFFu || hi[l] > 0xFFFFu) ? 0xFFFFFFFFu : (lo[l] | (hi[l] << 16));
}

// Leaf parameters interleaved for lookups that read them from global memory.
__global__ void k_pack_leaf4(const float* a, const float* b, const uint32_t* x0, const uint32_t* eps, uint4* out,
                             uint32_t L) {
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    out[l] = make_uint4(__float_as_uint(a[l]), __float_as_uint(b[l]), x0[l], eps[l]);
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
                            double* out, cudaStream_t st) {
    k_mlp_grad<H><<<grid_for(n), kThreads, 0, st>>>(xs, ys, keys, pos, yscale, n, n_all, seed, params, out);
    return cudaGetLastError();
}

cudaError_t mlp_grad_dispatch(uint32_t hidden, const float* xs, const float* ys, const uint32_t* keys,
                              const uint32_t* pos, float yscale, uint64_t n, uint64_t n_all, uint64_t seed,
                              const float* params, double* out, cudaStream_t st) {
    switch (hidden) {
        case 8: return launch_mlp_grad<8>(xs, ys, keys, pos, yscale, n, n_all, seed, params, out, st);
        case 16: return launch_mlp_grad<16>(xs, ys, keys, pos, yscale, n, n_all, seed, params, out, st);
        case 32: return launch_mlp_grad<32>(xs, ys, keys, pos, yscale, n, n_all, seed, params, out, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// --------------------------------------------------------------- host side

struct TrainScratch {
    uint32_t* pos;      // [n] (owned by caller)
    uint32_t* leaf;     // [n]
    double* red;        // small reductions [128]
    double* mom;        // [3L]
    double* acc;        // [3L]
    float *mu, *isd, *w, *c;  // [L]
    float *mp, *mm, *mv;      // MLP params / Adam state [3*32+1]
};

size_t rmi_train_scratch_bytes(uint64_t n, uint32_t L) {
    return n * 4 + 128 * 8 + (size_t)L * 3 * 8 * 2 + (size_t)L * 4 * 4 + 3 * 128 * 4 + 1024;
}

static TrainScratch carve(void* base, uint64_t n, uint32_t L) {
    char* p = (char*)base;
    auto take = [&](size_t bytes) {
        char* r = p;
        p += (bytes + 255) / 256 * 256;
        return (void*)r;
    };
    TrainScratch s;
    s.pos = nullptr;
    s.leaf = (uint32_t*)take(n * 4);
    s.red = (double*)take(128 * 8);
    s.mom = (double*)take((size_t)L * 3 * 8);
    s.acc = (double*)take((size_t)L * 3 * 8);
    s.mu = (float*)take((size_t)L * 4);
    s.isd = (float*)take((size_t)L * 4);
    s.w = (float*)take((size_t)L * 4);
    s.c = (float*)take((size_t)L * 4);
    s.mp = (float*)take(128 * 4);
    s.mm = (float*)take(128 * 4);
    s.mv = (float*)take(128 * 4);
    return s;
}

#define RMI_CU(x)                              \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return e_;      \
    } while (0)

cudaError_t rmi_train_device(RmiDev* m, float* d_a, float* d_b, uint32_t* d_x0, const uint32_t* keys,
                             const uint32_t* pos, uint64_t n, uint32_t n_ranges, const gnm_rmi_config& cfg,
                             void* scratch, RmiTrainOut* out, cudaStream_t st) {
    const uint32_t L = cfg.n_leaves;
    TrainScratch s = carve(scratch, n, L);
    const int g = grid_for(n);
    double h[4];
    // ---- root
    m->n_leaves = L;
    m->root_kind = cfg.root_kind;
    m->hidden = cfg.hidden;
    const float yscale_root = (float)((double)L / n_ranges);
    if (cfg.root_kind == GNM_RMI_ROOT_LINEAR) {
        RMI_CU(cudaMemsetAsync(s.red, 0, 2 * 8, st));
        k_moments<<<g, kThreads, 0, st>>>(keys, n, s.red);
        RMI_CU(cudaMemcpyAsync(h, s.red, 16, cudaMemcpyDeviceToHost, st));
        RMI_CU(cudaStreamSynchronize(st));
        const double mu = h[0] / n, var = h[1] / n - mu * mu;
        const double sd = var > 1e-30 ? sqrt(var) : 1.0;
        float w = 0.f, c = 0.f;
        double loss = 0.0;
        for (uint32_t it = 0; it <= cfg.leaf_iters; ++it) {
            RMI_CU(cudaMemsetAsync(s.red, 0, 3 * 8, st));
            k_root_linear_grad<<<g, kThreads, 0, st>>>(keys, pos, n, (float)mu, (float)(1.0 / sd), yscale_root, w, c, s.red);
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
            RMI_CU(cudaMemsetAsync(s.red, 0, (3 * H + 2) * 8, st));
            RMI_CU(mlp_grad_dispatch(cfg.hidden, nullptr, nullptr, keys, pos, ys, batch, n,
                                     cfg.seed * 1000003ull + step, s.mp, s.red, st));
            k_adam<<<1, 128, 0, st>>>(s.mp, s.mm, s.mv, s.red, cnt, 1.0 / batch, cfg.mlp_lr, 0.9f, 0.999f, 1e-8f,
                                      (int)step);
        }
        // final loss over all samples (in leaf units)
        RMI_CU(cudaMemsetAsync(s.red, 0, (3 * H + 2) * 8, st));
        RMI_CU(mlp_grad_dispatch(cfg.hidden, nullptr, nullptr, keys, pos, ys, n, n, 0, s.mp, s.red, st));
        double gl[3 * 32 + 2];
        RMI_CU(cudaMemcpyAsync(p, s.mp, cnt * 4, cudaMemcpyDeviceToHost, st));
        RMI_CU(cudaMemcpyAsync(gl, s.red, (3 * H + 2) * 8, cudaMemcpyDeviceToHost, st));
        RMI_CU(cudaStreamSynchronize(st));
        out->root_loss = gl[3 * H + 1] / n * (double)L * L;
        for (int j = 0; j < H; ++j) {
            m->w1[j] = p[j];
            m->b1[j] = p[H + j];
            m->w2[j] = p[2 * H + j] * (float)L;  // output rescaled from [0,1) to leaf units
        }
        for (int j = H; j < 32; ++j) m->w1[j] = m->b1[j] = m->w2[j] = 0.f;
        m->b2 = p[3 * H] * (float)L;
    }
    // ---- leaves
    RMI_CU(cudaMemsetAsync(d_x0, 0xFF, (size_t)L * 4, st));
    RmiDev route = *m;
    k_route<<<g, kThreads, 0, st>>>(route, keys, n, s.leaf, d_x0);
    RMI_CU(cudaMemsetAsync(s.mom, 0, (size_t)L * 3 * 8, st));
    k_leaf_moments<<<g, kThreads, 0, st>>>(keys, s.leaf, n, d_x0, s.mom);
    const int gl = (int)((L + 255) / 256);
    k_leaf_standardise<<<gl, 256, 0, st>>>(s.mom, L, s.mu, s.isd);
    RMI_CU(cudaMemsetAsync(s.w, 0, (size_t)L * 4, st));
    RMI_CU(cudaMemsetAsync(s.c, 0, (size_t)L * 4, st));
    for (uint32_t it = 0; it < cfg.leaf_iters; ++it) {
        RMI_CU(cudaMemsetAsync(s.acc, 0, (size_t)L * 3 * 8, st));
        k_leaf_grad<<<g, kThreads, 0, st>>>(keys, pos, s.leaf, n, d_x0, s.mu, s.isd, s.w, s.c, s.acc);
        k_leaf_step<<<gl, 256, 0, st>>>(s.acc, s.mom, L, 0.5f, s.w, s.c);
    }
    RMI_CU(cudaMemsetAsync(s.acc, 0, (size_t)L * 3 * 8, st));
    k_leaf_grad<<<g, kThreads, 0, st>>>(keys, pos, s.leaf, n, d_x0, s.mu, s.isd, s.w, s.c, s.acc);
    k_leaf_fold<<<gl, 256, 0, st>>>(s.mom, L, n_ranges, s.mu, s.isd, s.w, s.c, d_a, d_b, d_x0);
    RMI_CU(cudaGetLastError());
    // leaf loss and empty leaves
    double* hacc = new double[(size_t)L * 3];
    double* hmom = new double[(size_t)L * 3];
    cudaError_t e = cudaMemcpyAsync(hacc, s.acc, (size_t)L * 3 * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hmom, s.mom, (size_t)L * 3 * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        double sse = 0;
        uint32_t empty = 0;
        for (uint32_t l = 0; l < L; ++l) {
            sse += hacc[3 * l + 2];
            empty += hmom[3 * l] == 0.0;
        }
        out->leaf_loss = sse / n;
        out->empty_leaves = empty;
    }
    delete[] hacc;
    delete[] hmom;
    m->a = d_a;
    m->b = d_b;
    m->x0 = d_x0;
    return e;
}

cudaError_t rmi_eps_sweep(const RmiDev& m, const uint32_t* starts, uint32_t n, uint32_t* elo, uint32_t* ehi,
                          int sm_count, cudaStream_t st) {
    RMI_CU(cudaMemsetAsync(elo, 0, (size_t)m.n_leaves * 4, st));
    RMI_CU(cudaMemsetAsync(ehi, 0, (size_t)m.n_leaves * 4, st));
    k_eps_sweep<<<sm_count * 8, kThreads, 0, st>>>(m, starts, n, elo, ehi);
    return cudaGetLastError();
}

cudaError_t rmi_eps_from_samples(const RmiDev& m, const uint32_t* keys, const uint32_t* pos, uint64_t n_s,
                                 uint32_t n, uint32_t* elo, uint32_t* ehi, cudaStream_t st) {
    RMI_CU(cudaMemsetAsync(elo, 0, (size_t)m.n_leaves * 4, st));
    RMI_CU(cudaMemsetAsync(ehi, 0, (size_t)m.n_leaves * 4, st));
    k_eps_samples<<<grid_for(n_s), kThreads, 0, st>>>(m, keys, pos, n_s, n, elo, ehi);
    return cudaGetLastError();
}

cudaError_t rmi_pack_leaf4(const float* a, const float* b, const uint32_t* x0, const uint32_t* eps, uint4* out,
                           uint32_t L, cudaStream_t st) {
    k_pack_leaf4<<<(L + 255) / 256, 256, 0, st>>>(a, b, x0, eps, out, L);
    return cudaGetLastError();
}

cudaError_t rmi_pack_eps(const uint32_t* lo, const uint32_t* hi, uint32_t* packed, uint32_t L, cudaStream_t st) {
    k_pack_eps<<<(L + 255) / 256, 256, 0, st>>>(lo, hi, packed, L);
    return cudaGetLastError();
}

cudaError_t rmi_linear_grad(const float* z, const float* y, uint64_t n, float w, float c, double* acc3,
                            cudaStream_t st) {
    RMI_CU(cudaMemsetAsync(acc3, 0, 3 * 8, st));
    k_linear_grad<<<grid_for(n), kThreads, 0, st>>>(z, y, n, w, c, acc3);
    return cudaGetLastError();
}

cudaError_t rmi_mlp_grad(const float* xn, const float* y, uint64_t n, uint32_t hidden, const float* params,
                         double* grad, cudaStream_t st) {
    RMI_CU(cudaMemsetAsync(grad, 0, (3 * hidden + 2) * 8, st));
    return mlp_grad_dispatch(hidden, xn, y, nullptr, nullptr, 1.f, n, n, 0, params, grad, st);
}

}  // namespace gnm
