// plan.cu -- batched plans (one persistent launch over many windows, captured once into
// a CUDA graph and replayed) and the launch-shape autotuner.
//
// A plan fits the paper's hourly cycle (Sec. III.B.1: the NetPerf thread copies the Flow
// Data Store, a fixed buffer, to the GPU and launches the kernels every hour): the record
// buffers and window shapes stay, only their contents change between launches.
#include <algorithm>
#include <cstring>
#include <iterator>
#include <vector>

#include "ctx.hpp"

namespace gnm {
gnm_status acquire_slot_pinned(gnm_ctx* c, uint64_t wid, cudaStream_t st, uint32_t* out);
void unpin_slot(gnm_ctx* c, uint32_t s);
}  // namespace gnm

struct gnm_plan {
    gnm_ctx* c = nullptr;
    cudaGraphExec_t exec = nullptr;
    gnm::WinDesc* d_wins = nullptr;
    uint32_t* d_done = nullptr;
    uint32_t* d_partials = nullptr;
    uint32_t* d_keys = nullptr;
    std::vector<uint32_t> slots;
    cudaEvent_t ev = nullptr;
    uint32_t launches = 0;
    bool timed = false;
    bool launched = false;
    cudaEvent_t marks[gnm::kMaxPlanKernels + 1] = {};  // before the first kernel and after each
    int32_t kinds[gnm::kMaxPlanKernels] = {};
    unsigned char* d_part = nullptr;
};

using namespace gnm;

static void plan_free(gnm_plan* p) {
    if (!p) return;
    if (p->c) {
        cudaSetDevice(p->c->device);
        if (p->ev) cudaEventSynchronize(p->ev);
        for (uint32_t s : p->slots) {
            unpin_slot(p->c, s);
            // the plan's event dies with it; its work is complete, so nothing to wait for
            if (s < p->c->slots.size() && p->c->slots[s].ev == p->ev) p->c->slots[s].ev = nullptr;
        }
    }
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->d_wins) cudaFree(p->d_wins);
    if (p->d_done) cudaFree(p->d_done);
    if (p->d_partials) cudaFree(p->d_partials);
    if (p->d_keys) cudaFree(p->d_keys);
    if (p->d_part) cudaFree(p->d_part);
    if (p->ev) cudaEventDestroy(p->ev);
    for (auto e : p->marks)
        if (e) cudaEventDestroy(e);
    delete p;
}

extern "C" {

gnm_status gnm_plan_create(gnm_ctx* c, const gnm_records* rec, const uint64_t* offsets,
                           const uint64_t* wids, size_t n_win, gnm_plan** out) {
    return gnm_plan_create_ex(c, rec, offsets, wids, n_win, 0, out);
}

gnm_status gnm_plan_create_ex(gnm_ctx* c, const gnm_records* rec, const uint64_t* offsets,
                              const uint64_t* wids, size_t n_win, uint32_t flags, gnm_plan** out) {
    if (!c || !out || !wids) return fail(GNM_E_INVAL, "NULL argument");
    if (flags & ~GNM_PLAN_KERNEL_TIMES) return fail(GNM_E_INVAL, "unknown plan flags");
    *out = nullptr;
    if (n_win == 0) return fail(GNM_E_INVAL, "a plan needs at least one window");
    GNM_CU(cudaSetDevice(c->device));
    GNM_TRY(check_windows(c, rec, offsets, n_win));
    if (!rec->on_device && offsets[n_win] > offsets[0])
        return fail(GNM_E_INVAL, "plans run over device record buffers");
    for (size_t k = 0; k < n_win; ++k)
        for (size_t j = 0; j < k; ++j)
            if (wids[j] == wids[k]) return fail(GNM_E_INVAL, "duplicate window id in one plan");
    gnm_plan* p = new (std::nothrow) gnm_plan();
    if (!p) return fail(GNM_E_NOMEM, "host allocation failed");
    p->c = c;
    p->timed = (flags & GNM_PLAN_KERNEL_TIMES) != 0;
    auto bail = [&](gnm_status s) {
        plan_free(p);
        return s;
    };
    if (p->timed)
        for (auto& e : p->marks)
            if (cudaEventCreate(&e) != cudaSuccess) return bail(fail(GNM_E_CUDA, "event creation failed"));
    for (size_t k = 0; k < n_win; ++k) {
        uint32_t s;
        gnm_status st = acquire_slot_pinned(c, wids[k], c->aux, &s);
        if (st != GNM_OK) return bail(st);
        p->slots.push_back(s);
    }
    if (cudaStreamSynchronize(c->aux) != cudaSuccess) return bail(fail(GNM_E_CUDA, "slot preparation failed"));
    {  // sparse rate statistics: each window's log holds a word per record of the window
        std::vector<uint64_t> need(n_win);
        for (size_t k = 0; k < n_win; ++k) need[k] = offsets[k + 1] - offsets[k];
        const gnm_status st = reserve_rate_log(c, p->slots.data(), need.data(), n_win, c->aux);
        if (st != GNM_OK) return bail(st);
    }
    gnm_records dr = *rec;
    const uint64_t base = offsets[0];
    if (offsets[n_win] > base) {
        dr.srcaddr += base; dr.dstaddr += base; dr.dPkts += base; dr.dOctets += base; dr.first += base; dr.last += base;
    }
    Prepared pr;
    gnm_status st = prepare_launch(c, &dr, offsets, n_win, p->slots.data(), true, &pr);
    if (st != GNM_OK) return bail(st);
    const size_t nw = std::max<size_t>(std::max<size_t>(pr.wins.size(), pr.n_buckets), 1);
    if (cudaMalloc(&p->d_wins, sizeof(WinDesc) * nw) != cudaSuccess ||
        cudaMalloc(&p->d_done, sizeof(uint32_t) * nw) != cudaSuccess ||
        cudaMemset(p->d_done, 0, sizeof(uint32_t) * nw) != cudaSuccess ||
        (pr.wins.size() && cudaMemcpy(p->d_wins, pr.wins.data(), sizeof(WinDesc) * pr.wins.size(),
                                      cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaEventCreateWithFlags(&p->ev, cudaEventDisableTiming) != cudaSuccess ||
        (pr.partial_words && cudaMalloc(&p->d_partials, pr.partial_words * 4) != cudaSuccess) ||
        (pr.sh.split && pr.n && cudaMalloc(&p->d_keys, (pr.n + 4) * 4) != cudaSuccess) ||
        (pr.part_bytes && cudaMalloc(&p->d_part, pr.part_bytes) != cudaSuccess))
        return bail(fail(GNM_E_CUDA, "plan allocation failed"));
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(GNM_E_CUDA, "stream creation failed"));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = enqueue_prepared(c, pr, offsets, n_win, p->slots.data(), true, p->d_wins, p->d_done, p->d_partials,
                              p->d_keys, p->d_part, cs, &p->launches, p->timed ? p->marks : nullptr, p->kinds);
        e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess && st == GNM_OK) e = cudaGraphInstantiate(&p->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (st != GNM_OK) return bail(st);
    if (e != cudaSuccess) return bail(fail(GNM_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e)));
    *out = p;
    return GNM_OK;
}

gnm_status gnm_plan_launch(gnm_plan* p, void* stream) {
    if (!p) return fail(GNM_E_INVAL, "plan is NULL");
    gnm_ctx* c = p->c;
    GNM_CU(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    for (uint32_t s : p->slots)  // earlier readers and writers of the slots come first
        if (c->slots[s].ev && c->slots[s].ev != p->ev) GNM_CU(cudaStreamWaitEvent(st, c->slots[s].ev, 0));
    GNM_CU(cudaGraphLaunch(p->exec, st));
    GNM_CU(cudaEventRecord(p->ev, st));
    set_slots_done(c, p->slots.data(), p->slots.size(), p->ev, true);
    c->last_launches = p->launches;
    p->launched = true;
    return GNM_OK;
}

gnm_status gnm_plan_kernel_times(gnm_plan* p, float* ms, int32_t* kind, size_t cap, size_t* n_out) {
    if (!p || !n_out) return fail(GNM_E_INVAL, "NULL argument");
    if (!p->timed) return fail(GNM_E_STATE, "plan created without GNM_PLAN_KERNEL_TIMES");
    if (!p->launched) return fail(GNM_E_STATE, "plan never launched");
    *n_out = p->launches;
    if (cap < p->launches) return fail(GNM_E_CAPACITY, "cap smaller than the plan's kernel count");
    GNM_CU(cudaSetDevice(p->c->device));
    GNM_CU(cudaEventSynchronize(p->ev));
    for (uint32_t i = 0; i < p->launches; ++i) {
        if (ms) GNM_CU(cudaEventElapsedTime(&ms[i], p->marks[i], p->marks[i + 1]));
        if (kind) kind[i] = p->kinds[i];
    }
    return GNM_OK;
}

void gnm_plan_destroy(gnm_plan* p) { plan_free(p); }

gnm_status gnm_autotune(gnm_ctx* c, const gnm_records* rec, const uint64_t* offsets, const uint64_t* wids,
                        size_t n_win, gnm_tune_report* rep) {
    if (!c || !rep) return fail(GNM_E_INVAL, "NULL argument");
    GNM_CU(cudaSetDevice(c->device));
    GNM_TRY(check_windows(c, rec, offsets, n_win));
    if (!rec->on_device) return fail(GNM_E_INVAL, "autotuning runs over device record buffers");
    const gnm_config saved = c->cfg;
    const Tuned saved_t = c->tuned;
    c->tuned = Tuned();
    cudaEvent_t e0, e1;
    GNM_CU(cudaEventCreate(&e0));
    GNM_CU(cudaEventCreate(&e1));
    cudaStream_t st = c->aux;
    auto time_cfg = [&](double* ms) -> gnm_status {
        float best = 1e30f;
        for (int r = 0; r < 4; ++r) {
            GNM_CU(cudaEventRecord(e0, st));
            GNM_TRY(gnm_windows_process(c, rec, offsets, wids, n_win, st));
            GNM_CU(cudaEventRecord(e1, st));
            GNM_CU(cudaEventSynchronize(e1));
            float t;
            GNM_CU(cudaEventElapsedTime(&t, e0, e1));
            if (r > 0) best = std::min(best, t);  // first run warms up
        }
        *ms = best;
        return GNM_OK;
    };
    std::memset(rep, 0, sizeof(*rep));
    gnm_status status = time_cfg(&rep->default_ms);
    rep->best_ms = 1e30;
    const int blocks[] = {256, 512, 768, 1024};
    const int unrolls[] = {1, 2, 3};
    const int aggs[] = {GNM_AGG_DIRECT, GNM_AGG_WARP};
    const int places[] = {GNM_PLACE_SMEM, GNM_PLACE_STAGED, GNM_PLACE_L2};
    // the lookup method decides which knob matters: placement (binary search) or
    // directory size (radix)
    LaunchShape base_shape;
    GNM_TRY(choose_shape(c, offsets[n_win] - offsets[0], &base_shape));
    std::vector<int> places_v, bits_v;
    if (base_shape.lookup == kLookupRadix) {
        places_v.push_back(GNM_PLACE_AUTO);
        const int b0 = (int)base_shape.radix_bits;
        for (int d : {0, -2, -1, 1, 2})
            if (b0 + d >= 4 && b0 + d <= 16) bits_v.push_back(b0 + d);
    } else {
        bits_v.push_back(0);
        if (base_shape.lookup == kLookupSmem) {  // no directory (0), or one of 2..32 ranges per bucket
            uint32_t lg = 0;
            while ((1ull << lg) < c->h_starts.size()) ++lg;
            for (int d : {1, 2, 3, 4, 5})
                if ((int)lg - d >= 4 && (int)lg - d <= 14) bits_v.push_back((int)lg - d);
        }
        if (base_shape.lookup == kLookupRmi) places_v = {GNM_PLACE_AUTO, GNM_PLACE_L2};  // leaves staged or not
        else places_v.assign(std::begin(places), std::end(places));
    }
    const int cpss[] = {0, 1};
    std::vector<int> splits_v;
    if (base_shape.lookup == kLookupSmem) splits_v.push_back(GNM_SPLIT_FUSED);
    else splits_v = {GNM_SPLIT_FUSED, GNM_SPLIT_TWO_KERNELS};
    std::vector<int> kdirs_v = {0};
    if (base_shape.lookup == kLookupRadix) kdirs_v = {3, 1, 4, 2};
    for (int sp : splits_v)
    for (int kd : kdirs_v)
    for (int ku : {1, 2})
    for (int b : blocks)
        for (int u : unrolls)
            for (int a : aggs)
                for (int pl : places_v)
                    for (int rb : bits_v)
                        for (int cps : cpss) {
                            if (status != GNM_OK) break;
                            // two groups per thread: up to 512 threads; pipelined groups (3):
                            // split launches with direct aggregation, up to 768 threads; 768
                            // threads for pipelined groups only
                            if (u == 2 && b > 512) continue;
                            if (u == 3 && (b > 768 || sp != GNM_SPLIT_TWO_KERNELS || a != GNM_AGG_DIRECT)) continue;
                            if (b == 768 && u != 3) continue;
                            c->cfg = saved;
                            if (c->cfg.block_threads == 0) c->cfg.block_threads = b;
                            if (c->cfg.unroll == 0) c->cfg.unroll = u;
                            if (c->cfg.aggregation == GNM_AGG_AUTO) c->cfg.aggregation = a;
                            if (c->cfg.placement == GNM_PLACE_AUTO) c->cfg.placement = pl;
                            if (c->cfg.radix_bits == 0) c->cfg.radix_bits = (uint32_t)rb;
                            if (c->cfg.ctas_per_sm == 0) c->cfg.ctas_per_sm = cps;
                            if (c->cfg.split == GNM_SPLIT_AUTO) c->cfg.split = sp;
                            // key kernel knobs: none in fused launches; the 16-bit directory
                            // has no size to tune
                            if (sp == GNM_SPLIT_FUSED && (kd != kdirs_v[0] || ku == 2)) continue;
                            if (kd == 4 && rb != bits_v[0]) continue;
                            // directory sizes matter to the shared-memory placement only
                            if (base_shape.lookup == kLookupSmem && rb != 0 && pl != GNM_PLACE_SMEM) continue;
                            c->tuned.keys_unroll = ku;
                            if (c->cfg.key_directory == 0) c->cfg.key_directory = kd;
                            LaunchShape sh;
                            if (choose_shape(c, offsets[n_win] - offsets[0], &sh) != GNM_OK) continue;  // does not fit
                            double ms;
                            status = time_cfg(&ms);
                            rep->n_tried++;
                            {
                                double& ba = rep->best_ms_by_agg[c->cfg.aggregation == GNM_AGG_WARP ? 2 : 1];
                                if (status == GNM_OK && (ba == 0.0 || ms < ba)) ba = ms;
                            }
                            if (status == GNM_OK && ms < rep->best_ms) {
                                rep->best_ms = ms;
                                rep->block_threads = c->cfg.block_threads;
                                rep->unroll = c->cfg.unroll;
                                rep->aggregation = c->cfg.aggregation;
                                rep->placement = c->cfg.placement;
                                rep->ctas_per_sm = sh.ctas_per_sm;
                                rep->radix_bits = sh.radix_bits;
                                rep->split = sh.split ? GNM_SPLIT_TWO_KERNELS : GNM_SPLIT_FUSED;
                                rep->key_directory = c->cfg.key_directory;
                                rep->keys_unroll = sh.split ? sh.keys_unroll : 0;
                            }
                        }
    c->cfg = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != GNM_OK) {
        c->tuned = saved_t;
        return status;
    }
    c->tuned.block = rep->block_threads;
    c->tuned.unroll = rep->unroll;
    c->tuned.agg = rep->aggregation;
    c->tuned.placement = rep->placement;
    c->tuned.ctas_per_sm = rep->ctas_per_sm;
    c->tuned.radix_bits = rep->radix_bits;
    c->tuned.split = rep->split;
    c->tuned.key_dir = rep->key_directory;
    c->tuned.keys_unroll = rep->keys_unroll;
    // leave the windows holding the results of the chosen shape
    return gnm_windows_process(c, rec, offsets, wids, n_win, st) == GNM_OK && cudaStreamSynchronize(st) == cudaSuccess
               ? GNM_OK
               : GNM_E_CUDA;
}

}  // extern "C"
