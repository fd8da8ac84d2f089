// state.cu -- checkpoint of an open window: its partial sums out to the host in the
// user-facing row layout, and back into a freshly opened window.
//
// Accumulator rows hold (flows << 32 | e_flows, octets of ineligible flows, pkts, e_octets,
// e_dur); rows of a 32-key group that a launch wrote are marked for finalisation, so an
// imported window marks all of its groups.
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "ctx.hpp"

using namespace gnm;

namespace {

gnm_status open_slot(gnm_ctx* c, uint64_t wid, uint32_t* s) {
    if (!c->have_registry) return fail(GNM_E_STATE, "no registry loaded");
    auto it = c->slot_of.find(wid);
    if (it == c->slot_of.end()) return fail(GNM_E_STATE, "unknown or evicted window id " + std::to_string(wid));
    if (!c->slots[it->second].open) return fail(GNM_E_STATE, "window " + std::to_string(wid) + " is not open");
    *s = it->second;
    return GNM_OK;
}

gnm_status carried_only(gnm_ctx* c) {
    if (c->cfg.rate_stats || c->hcap)
        return fail(GNM_E_STATE, "a window checkpoint carries the sums only: this context keeps per-flow rate "
                                 "or per-host statistics");
    return GNM_OK;
}

}  // namespace

extern "C" {

gnm_status gnm_window_export(gnm_ctx* c, uint64_t wid, uint64_t* rows, size_t cap, size_t* n_out) {
    if (!c || !n_out || (cap && !rows)) return fail(GNM_E_INVAL, "NULL argument");
    *n_out = 0;
    uint32_t s;
    GNM_TRY(open_slot(c, wid, &s));
    GNM_TRY(carried_only(c));
    const size_t keys = c->keys;
    *n_out = keys;
    if (cap < keys) return fail(GNM_E_CAPACITY, "rows holds fewer than " + std::to_string(keys) + " rows");
    GNM_CU(cudaSetDevice(c->device));
    const Slot& sl = c->slots[s];
    if (sl.ev) GNM_CU(cudaEventSynchronize(sl.ev));
    std::vector<uint64_t> acc(keys * kAccCols);
    GNM_CU(cudaMemcpy(acc.data(), c->d_acc + (size_t)s * keys * kAccCols, acc.size() * 8, cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < keys; ++k) {
        const uint64_t* a = acc.data() + k * kAccCols;
        uint64_t* r = rows + k * kNStat;
        r[0] = a[0] >> 32;               // flows
        r[1] = a[1] + a[3];              // octets: ineligible + eligible flows'
        r[2] = a[2];                     // pkts
        r[3] = a[0] & 0xFFFFFFFFull;     // e_flows
        r[4] = a[3];                     // e_octets
        r[5] = a[4];                     // e_dur_ms
    }
    return GNM_OK;
}

gnm_status gnm_window_import(gnm_ctx* c, uint64_t wid, const uint64_t* rows, size_t n_rows, void* stream) {
    if (!c || !rows) return fail(GNM_E_INVAL, "NULL argument");
    if (!c->have_registry) return fail(GNM_E_STATE, "no registry loaded");
    GNM_TRY(carried_only(c));
    const size_t keys = c->keys;
    if (n_rows != keys) return fail(GNM_E_INVAL, "n_rows must be " + std::to_string(keys));
    std::vector<uint64_t> acc(keys * kAccCols);
    uint64_t records = 0;
    for (size_t k = 0; k < keys; ++k) {
        const uint64_t* r = rows + k * kNStat;
        if (r[0] >= (1ull << 32) || r[3] > r[0] || r[4] > r[1])
            return fail(GNM_E_INVAL, "row " + std::to_string(k) + " is inconsistent");
        records += r[0];
        uint64_t* a = acc.data() + k * kAccCols;
        a[0] = r[0] << 32 | r[3];
        a[1] = r[1] - r[4];
        a[2] = r[2];
        a[3] = r[4];
        a[4] = r[5];
    }
    if (records >= (1ull << 32)) return fail(GNM_E_INVAL, "the window would hold 2^32 records or more");
    GNM_CU(cudaSetDevice(c->device));
    const cudaStream_t st = (cudaStream_t)stream;
    uint32_t s;
    GNM_TRY(open_window(c, wid, st, false, &s));
    const size_t groups = (keys + 31) / 32;
    GNM_CU(cudaMemcpyAsync(c->d_acc + (size_t)s * keys * kAccCols, acc.data(), acc.size() * 8,
                           cudaMemcpyHostToDevice, st));
    GNM_CU(cudaMemsetAsync(c->d_dirty + (size_t)s * groups, 1, groups, st));
    // synchronous: later work on the window may come on any stream
    GNM_CU(cudaStreamSynchronize(st));
    c->slots[s].records = records;
    return GNM_OK;
}

}  // extern "C"
