// rmi_api.cu -- C ABI of the learned index: training, error bounds, import/export and the
// gradient entry points used to check the training arithmetic.
#include <algorithm>
#include <cstring>
#include <vector>

#include "ctx.hpp"

using namespace gnm;

namespace {

gnm_status ensure_models(gnm_ctx* c, uint32_t L) {
    if (c->rmi_cap >= L) return GNM_OK;
    cudaFree(c->d_rmi_a);
    cudaFree(c->d_rmi_b);
    cudaFree(c->d_rmi_x0);
    cudaFree(c->d_rmi_eps);
    cudaFree(c->d_rmi_elo);
    cudaFree(c->d_rmi_ehi);
    cudaFree(c->d_rmi_leaf4);
    c->d_rmi_leaf4 = nullptr;
    c->d_rmi_a = c->d_rmi_b = nullptr;
    c->d_rmi_x0 = c->d_rmi_eps = c->d_rmi_elo = c->d_rmi_ehi = nullptr;
    c->rmi_cap = 0;
    GNM_CU(cudaMalloc(&c->d_rmi_a, (size_t)L * 4));
    GNM_CU(cudaMalloc(&c->d_rmi_b, (size_t)L * 4));
    GNM_CU(cudaMalloc(&c->d_rmi_x0, (size_t)L * 4));
    GNM_CU(cudaMalloc(&c->d_rmi_eps, (size_t)L * 4));
    GNM_CU(cudaMalloc(&c->d_rmi_elo, (size_t)L * 4));
    GNM_CU(cudaMalloc(&c->d_rmi_ehi, (size_t)L * 4));
    GNM_CU(cudaMalloc(&c->d_rmi_leaf4, (size_t)L * 16));
    c->rmi_cap = L;
    return GNM_OK;
}

// Uploads a host model (root in m, arrays in t) into the context's model arrays.
gnm_status upload_model(gnm_ctx* c, RmiDev& m, const RmiTrainOut& t, cudaStream_t st) {
    const uint32_t M = (uint32_t)t.a.size();
    GNM_TRY(ensure_models(c, M));
    GNM_CU(cudaMemcpyAsync(c->d_rmi_a, t.a.data(), (size_t)M * 4, cudaMemcpyHostToDevice, st));
    GNM_CU(cudaMemcpyAsync(c->d_rmi_b, t.b.data(), (size_t)M * 4, cudaMemcpyHostToDevice, st));
    GNM_CU(cudaMemcpyAsync(c->d_rmi_x0, t.x0.data(), (size_t)M * 4, cudaMemcpyHostToDevice, st));
    GNM_CU(cudaMemcpyAsync(c->d_rmi_eps, t.eps.data(), (size_t)M * 4, cudaMemcpyHostToDevice, st));
    GNM_CU(cudaStreamSynchronize(st));  // the host vectors may go away
    m.n_models = M;
    m.a = c->d_rmi_a;
    m.b = c->d_rmi_b;
    m.x0 = c->d_rmi_x0;
    m.eps = c->d_rmi_eps;
    c->rmi_split = t.split;
    return GNM_OK;
}

// Error bounds of the model in m (exhaustive or from samples), packed for lookups; the
// eps array already marks split leaves.
gnm_status finish_model(gnm_ctx* c, RmiDev& m, bool exhaustive, const uint32_t* keys, const uint32_t* pos,
                        uint64_t n, cudaStream_t st, double* sweep_ms) {
    const uint32_t nr = (uint32_t)c->h_starts.size();
    cudaEvent_t e0, e1;
    GNM_CU(cudaEventCreate(&e0));
    GNM_CU(cudaEventCreate(&e1));
    GNM_CU(cudaEventRecord(e0, st));
    if (exhaustive) GNM_CU(rmi_eps_sweep(m, c->d_starts, nr, c->d_rmi_elo, c->d_rmi_ehi, c->sm_count, st));
    else GNM_CU(rmi_eps_from_samples(m, keys, pos, n, nr, c->d_rmi_elo, c->d_rmi_ehi, st));
    GNM_CU(rmi_pack_eps(c->d_rmi_elo, c->d_rmi_ehi, c->d_rmi_eps, m.n_models, st));
    GNM_CU(rmi_pack_leaf4(m.a, m.b, m.x0, c->d_rmi_eps, c->d_rmi_leaf4, m.n_models, st));
    GNM_CU(cudaEventRecord(e1, st));
    GNM_CU(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (sweep_ms) *sweep_ms = ms;
    m.eps = c->d_rmi_eps;
    m.leaf4 = c->d_rmi_leaf4;
    m.leaves_global = 0;
    c->rmi = m;
    c->rmi_ready = true;
    return GNM_OK;
}

}  // namespace

extern "C" {

void gnm_rmi_config_default(gnm_rmi_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->root_kind = GNM_RMI_ROOT_LINEAR;
    cfg->n_leaves = 4096;
    cfg->hidden = 32;
    cfg->leaf_iters = 4;
    cfg->mlp_steps = 600;
    cfg->mlp_batch = 65536;
    cfg->mlp_lr = 0.01f;
    cfg->seed = 1;
    cfg->exhaustive_eps = 1;
    cfg->leaf_fit = GNM_RMI_FIT_MINIMAX;
    cfg->eps_target = 64;
    cfg->max_split_log2 = 14;
}

gnm_status gnm_rmi_train(gnm_ctx* c, const uint32_t* keys, uint64_t n, const gnm_rmi_config* cfg_in,
                         gnm_rmi_report* rep, void* stream) {
    if (!c || !keys || !rep) return fail(GNM_E_INVAL, "NULL argument");
    if (!c->have_registry) return fail(GNM_E_STATE, "no registry loaded");
    gnm_rmi_config cfg;
    if (cfg_in) cfg = *cfg_in;
    else gnm_rmi_config_default(&cfg);
    if (n == 0) return fail(GNM_E_INVAL, "no training keys");
    if (cfg.n_leaves == 0 || cfg.n_leaves > (uint32_t)kMaxLeaves) return fail(GNM_E_INVAL, "n_leaves must be 1..1048576");
    if (cfg.root_kind != GNM_RMI_ROOT_LINEAR && cfg.root_kind != GNM_RMI_ROOT_MLP)
        return fail(GNM_E_INVAL, "unknown root kind");
    if (cfg.root_kind == GNM_RMI_ROOT_MLP && cfg.hidden != 8 && cfg.hidden != 16 && cfg.hidden != 32)
        return fail(GNM_E_INVAL, "MLP root width must be 8, 16 or 32");
    if (cfg.leaf_fit != GNM_RMI_FIT_MINIMAX && cfg.leaf_fit != GNM_RMI_FIT_MSE)
        return fail(GNM_E_INVAL, "unknown leaf fit");
    if (cfg.max_split_log2 > 16) return fail(GNM_E_INVAL, "max_split_log2 must be at most 16");
    if (c->h_starts.size() >= (1u << 24)) return fail(GNM_E_INVAL, "learned index needs fewer than 2^24 ranges");
    GNM_CU(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    std::memset(rep, 0, sizeof(*rep));
    rep->n_train = n;
    uint32_t* pos = nullptr;
    void* scratch = nullptr;
    gnm_status status = GNM_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    do {
        if (cudaMalloc(&pos, n * 4) != cudaSuccess ||
            cudaMalloc(&scratch, rmi_train_scratch_bytes(n, cfg.n_leaves)) != cudaSuccess) {
            status = fail(GNM_E_NOMEM, "training scratch allocation failed");
            break;
        }
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            status = fail(GNM_E_CUDA, "event creation failed");
            break;
        }
        cudaEventRecord(e0, st);
        // positions from the plain binary search (the lookups the model learns)
        AggParams p;
        gnm_records none{};
        build_params(c, &none, &p);
        cudaError_t e = launch_lookup(p, kLookupL2, keys, n, nullptr, pos, st);
        RmiDev m{};
        RmiTrainOut to{};
        if (e == cudaSuccess)
            e = rmi_train_device(&m, keys, pos, n, c->d_starts, (uint32_t)c->h_starts.size(), cfg, scratch, &to, st);
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            status = fail(GNM_E_CUDA, std::string("learned-index training: ") + cudaGetErrorString(e));
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        rep->train_ms = ms;
        rep->root_loss = to.root_loss;
        rep->empty_leaves = to.empty_leaves;
        rep->split_leaves = to.split_leaves;
        rep->n_models = (uint32_t)to.a.size();
        c->rmi_ready = false;
        status = upload_model(c, m, to, st);
        if (status == GNM_OK) status = finish_model(c, m, cfg.exhaustive_eps != 0, keys, pos, n, st, &rep->sweep_ms);
        if (status != GNM_OK) break;
        // report: widest window and error over the models, and over the training lookups the
        // mean squared position error and the mean window searched
        const uint32_t M = m.n_models;
        std::vector<uint32_t> lo(M), hi(M);
        if (cudaMemcpy(lo.data(), c->d_rmi_elo, (size_t)M * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(hi.data(), c->d_rmi_ehi, (size_t)M * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
            status = fail(GNM_E_CUDA, "error-bound readback failed");
            break;
        }
        uint32_t mx = 0, mxe = 0;
        for (uint32_t l = 0; l < M; ++l) {
            mx = std::max(mx, lo[l] + hi[l]);
            mxe = std::max(mxe, std::max(lo[l], hi[l]));
        }
        rep->eps_max = mx;
        rep->err_max = mxe;
        double* part = (double*)scratch;  // the training scratch is free again
        double h2[2] = {0.0, 0.0};
        e = rmi_model_stats(c->rmi, keys, pos, n, (uint32_t)c->h_starts.size(), part + 2, part, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h2, part, 16, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            status = fail(GNM_E_CUDA, std::string("learned-index report: ") + cudaGetErrorString(e));
            break;
        }
        rep->leaf_loss = h2[0] / n;
        rep->eps_mean = h2[1] / n;
    } while (false);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(pos);
    cudaFree(scratch);
    return status;
}

gnm_status gnm_rmi_violations(gnm_ctx* c, uint64_t* count, int reset) {
    if (!c || !count) return fail(GNM_E_INVAL, "NULL argument");
    GNM_CU(cudaSetDevice(c->device));
    GNM_CU(cudaDeviceSynchronize());
    unsigned long long v = 0;
    GNM_CU(cudaMemcpy(&v, c->d_violations, 8, cudaMemcpyDeviceToHost));
    *count = v;
    if (reset) GNM_CU(cudaMemset(c->d_violations, 0, 8));
    return GNM_OK;
}

gnm_status gnm_rmi_linear_grad(gnm_ctx* c, const float* z, const float* y, uint64_t n, float w, float cc,
                               double grad[3], void* stream) {
    if (!c || !z || !y || !grad || n == 0) return fail(GNM_E_INVAL, "bad argument");
    GNM_CU(cudaSetDevice(c->device));
    double* d = nullptr;
    GNM_CU(cudaMalloc(&d, 3 * 8 + rmi_partials_bytes()));
    cudaStream_t st = (cudaStream_t)stream;
    double h[3];
    cudaError_t e = rmi_linear_grad(z, y, n, w, cc, d + 3, d, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, 24, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return fail(GNM_E_CUDA, cudaGetErrorString(e));
    grad[0] = 2.0 * h[0] / n;
    grad[1] = 2.0 * h[1] / n;
    grad[2] = h[2] / n;
    return GNM_OK;
}

gnm_status gnm_rmi_mlp_grad(gnm_ctx* c, const float* xn, const float* y, uint64_t n, uint32_t hidden,
                            const float* params, double* grad, void* stream) {
    if (!c || !xn || !y || !params || !grad || n == 0) return fail(GNM_E_INVAL, "bad argument");
    if (hidden != 8 && hidden != 16 && hidden != 32) return fail(GNM_E_INVAL, "hidden must be 8, 16 or 32");
    GNM_CU(cudaSetDevice(c->device));
    const int cnt = 3 * (int)hidden + 1;
    float* dp = nullptr;
    double* dg = nullptr;
    GNM_CU(cudaMalloc(&dp, cnt * 4));
    if (cudaMalloc(&dg, (cnt + 1) * 8 + rmi_partials_bytes()) != cudaSuccess) {
        cudaFree(dp);
        return fail(GNM_E_NOMEM, "allocation failed");
    }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> h(cnt + 1);
    cudaError_t e = cudaMemcpyAsync(dp, params, cnt * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = rmi_mlp_grad(xn, y, n, hidden, dp, dg + (cnt + 1), dg, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), dg, (cnt + 1) * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dp);
    cudaFree(dg);
    if (e != cudaSuccess) return fail(GNM_E_CUDA, cudaGetErrorString(e));
    for (int k = 0; k < cnt; ++k) grad[k] = 2.0 * h[k] / n;
    grad[cnt] = h[cnt] / n;
    return GNM_OK;
}

gnm_status gnm_rmi_export(gnm_ctx* c, int32_t* root_kind, uint32_t* n_leaves, uint32_t* n_models, float* root,
                          uint32_t* split, float* a, float* b, uint32_t* x0, uint32_t* eps_lo, uint32_t* eps_hi) {
    if (!c) return fail(GNM_E_INVAL, "ctx is NULL");
    if (!c->rmi_ready) return fail(GNM_E_STATE, "no learned index");
    GNM_CU(cudaSetDevice(c->device));
    GNM_CU(cudaDeviceSynchronize());
    const RmiDev& m = c->rmi;
    const uint32_t L = m.n_leaves, M = m.n_models;
    if (root_kind) *root_kind = m.root_kind;
    if (n_leaves) *n_leaves = L;
    if (n_models) *n_models = M;
    if (root) {
        root[0] = m.ra;
        root[1] = m.rb;
        for (int j = 0; j < kMaxHidden; ++j) {
            root[2 + j] = m.w1[j];
            root[2 + kMaxHidden + j] = m.b1[j];
            root[2 + 2 * kMaxHidden + j] = m.w2[j];
        }
        root[2 + 3 * kMaxHidden] = m.b2;
    }
    if (split)
        for (uint32_t l = 0; l < L; ++l) split[l] = l < c->rmi_split.size() ? c->rmi_split[l] : 0u;
    if (a) GNM_CU(cudaMemcpy(a, c->d_rmi_a, (size_t)M * 4, cudaMemcpyDeviceToHost));
    if (b) GNM_CU(cudaMemcpy(b, c->d_rmi_b, (size_t)M * 4, cudaMemcpyDeviceToHost));
    if (x0) GNM_CU(cudaMemcpy(x0, c->d_rmi_x0, (size_t)M * 4, cudaMemcpyDeviceToHost));
    if (eps_lo) GNM_CU(cudaMemcpy(eps_lo, c->d_rmi_elo, (size_t)M * 4, cudaMemcpyDeviceToHost));
    if (eps_hi) GNM_CU(cudaMemcpy(eps_hi, c->d_rmi_ehi, (size_t)M * 4, cudaMemcpyDeviceToHost));
    // split leaves' entries hold their routing words on the device; the export shows zeros
    for (uint32_t l = 0; l < L && l < c->rmi_split.size(); ++l)
        if (c->rmi_split[l]) {
            if (a) a[l] = 0.f;
            if (b) b[l] = 0.f;
            if (eps_lo) eps_lo[l] = 0u;
            if (eps_hi) eps_hi[l] = 0u;
        }
    return GNM_OK;
}

gnm_status gnm_rmi_import(gnm_ctx* c, int32_t root_kind, uint32_t L, uint32_t M, const float* root,
                          const uint32_t* split, const float* a, const float* b, const uint32_t* x0, void* stream) {
    if (!c || !root || !a || !b || !x0) return fail(GNM_E_INVAL, "NULL argument");
    if (!c->have_registry) return fail(GNM_E_STATE, "no registry loaded");
    if (L == 0 || L > (uint32_t)kMaxLeaves) return fail(GNM_E_INVAL, "n_leaves must be 1..1048576");
    if (M < L || M > kMaxModels) return fail(GNM_E_INVAL, "n_models must be n_leaves..4194304");
    if (root_kind != GNM_RMI_ROOT_LINEAR && root_kind != GNM_RMI_ROOT_MLP) return fail(GNM_E_INVAL, "unknown root kind");
    if (c->h_starts.size() >= (1u << 24)) return fail(GNM_E_INVAL, "learned index needs fewer than 2^24 ranges");
    RmiTrainOut t;
    t.a.assign(a, a + M);
    t.b.assign(b, b + M);
    t.x0.assign(x0, x0 + M);
    t.eps.assign(M, 0u);
    t.split.assign(L, 0u);
    uint64_t nxt = L;
    for (uint32_t l = 0; split && l < L; ++l) {
        const uint32_t w = split[l];
        if (!w) continue;
        if ((w & 0xFFu) > 31u || (w >> 8) > 0xFFFFu) return fail(GNM_E_INVAL, "split word: shift > 31 or count > 65536");
        const uint32_t base = (uint32_t)nxt;
        nxt += (w >> 8) + 1u;
        if (nxt > M) break;
        std::memcpy(&t.a[l], &w, 4);
        std::memcpy(&t.b[l], &base, 4);
        t.eps[l] = kEpsSplit;
        t.split[l] = w;
    }
    if (nxt != M) return fail(GNM_E_INVAL, "the split table does not add up to n_models");
    GNM_CU(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    RmiDev m{};
    m.root_kind = root_kind;
    m.n_leaves = L;
    m.hidden = kMaxHidden;
    m.ra = root[0];
    m.rb = root[1];
    for (int j = 0; j < kMaxHidden; ++j) {
        m.w1[j] = root[2 + j];
        m.b1[j] = root[2 + kMaxHidden + j];
        m.w2[j] = root[2 + 2 * kMaxHidden + j];
    }
    m.b2 = root[2 + 3 * kMaxHidden];
    c->rmi_ready = false;
    GNM_TRY(upload_model(c, m, t, st));
    return finish_model(c, m, true, nullptr, nullptr, 0, st, nullptr);
}

}  // extern "C"
