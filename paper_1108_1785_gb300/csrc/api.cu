// api.cu -- the C ABI: contexts, registry upload, window processing and result readout.
#include <algorithm>
#include <limits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.hpp"

namespace gnm {

static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }
const char* get_error() { return g_err.c_str(); }
gnm_status fail(gnm_status s, const std::string& m) {
    set_error(m);
    return s;
}

std::string flatten_registry(const uint32_t* prefix, const uint8_t* len, const uint32_t* site,
                             size_t n, uint32_t n_sites, std::vector<uint32_t>* starts,
                             std::vector<uint32_t>* sites);
bool local_overlaps(uint32_t lp, uint8_t ll, const uint32_t* prefix, const uint8_t* len, size_t n);
bool build_hash24(const uint32_t* prefix, const uint8_t* len, const uint32_t* site, size_t n,
                  std::vector<uint32_t>* table, uint32_t* mask);

constexpr uint32_t kRingSize = 32;
constexpr size_t kRegistrySmemMax = 96 * 1024;   // bytes of ranges kept in shared memory
constexpr size_t kSampleSmemMax = 96 * 1024;     // bytes of block samples (staged placement)
constexpr size_t kDirectTableMax = 208 * 1024;   // direct-indexed per-CTA sums
constexpr size_t kHashTableMax = 200 * 1024;     // hashed per-CTA sums
constexpr uint32_t kFinalizeInCtaMaxKeys = 4096;
constexpr uint64_t kPartialBytesMax = 1ull << 30;  // per launch; larger launches flush atomically
constexpr uint64_t kMaxWindowRecords = 0xFFFFFFFFull;

static uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

static void free_dev(void* p) {
    if (p) cudaFree(p);
}

// ------------------------------------------------------------------ slots

static gnm_status wait_slot_on_stream(gnm_ctx* c, uint32_t s, cudaStream_t st) {
    Slot& sl = c->slots[s];
    if (sl.ev) GNM_CU(cudaStreamWaitEvent(st, sl.ev, 0));
    return GNM_OK;
}

static gnm_status acquire_slot_impl(gnm_ctx* c, uint64_t wid, cudaStream_t st, bool pin, uint32_t* out) {
    auto it = c->slot_of.find(wid);
    uint32_t s;
    if (it != c->slot_of.end()) {
        s = it->second;
        if (c->slots[s].pinned) return fail(GNM_E_STATE, "window id belongs to a plan");
    } else {
        s = UINT32_MAX;
        for (uint32_t i = 0; i < c->n_slots; ++i)
            if (!c->slots[i].used) { s = i; break; }
        if (s == UINT32_MAX) {  // evict the oldest window not held by a plan
            uint64_t best = UINT64_MAX;
            for (uint32_t i = 0; i < c->n_slots; ++i)
                if (!c->slots[i].pinned && c->slots[i].age < best) { best = c->slots[i].age; s = i; }
            if (s == UINT32_MAX) return fail(GNM_E_CAPACITY, "every result slot is held by a plan or an open served window");
            c->slot_of.erase(c->slots[s].window_id);
        }
        c->slot_of[wid] = s;
    }
    GNM_TRY(wait_slot_on_stream(c, s, st));
    Slot& sl = c->slots[s];
    if (sl.used && sl.open) {  // partial sums of an unfinished window: clear them
        GNM_CU(cudaMemsetAsync(c->d_acc + (size_t)s * c->keys * kAccCols, 0,
                               (size_t)c->keys * kAccCols * 8, st));
    }
    sl.used = true;
    sl.open = false;
    sl.finalized = false;
    sl.pinned = pin;
    sl.window_id = wid;
    sl.records = 0;
    sl.age = ++c->age;
    *out = s;
    return GNM_OK;
}

gnm_status acquire_slot(gnm_ctx* c, uint64_t wid, cudaStream_t st, uint32_t* out) {
    return acquire_slot_impl(c, wid, st, false, out);
}

gnm_status acquire_slot_pinned(gnm_ctx* c, uint64_t wid, cudaStream_t st, uint32_t* out) {
    return acquire_slot_impl(c, wid, st, true, out);
}

void unpin_slot(gnm_ctx* c, uint32_t s) {
    if (s < c->slots.size()) c->slots[s].pinned = false;
}

void set_slots_done(gnm_ctx* c, const uint32_t* slots, size_t n, cudaEvent_t ev, bool finalized) {
    for (size_t k = 0; k < n; ++k) {
        Slot& sl = c->slots[slots[k]];
        sl.ev = ev;
        sl.open = !finalized;
        sl.finalized = finalized;
    }
}

// Records a completion event on st (a ring entry's) and returns it.
static gnm_status record_event(gnm_ctx* c, cudaStream_t st, cudaEvent_t* ev) {
    LaunchBuf* lb;
    GNM_TRY(acquire_ring(c, 0, &lb));
    GNM_CU(cudaEventRecord(lb->ev, st));
    lb->ev_recorded = true;
    *ev = lb->ev;
    return GNM_OK;
}

void release_slots(gnm_ctx* c) {
    c->slots.clear();
    c->slot_of.clear();
    free_dev(c->d_acc);
    free_dev(c->d_dirty);
    free_dev(c->d_stats);
    free_dev(c->d_rate);
    free_dev(c->d_flag);
    free_dev(c->d_flag_keys);
    free_dev(c->d_hist);
    free_dev(c->d_rmin);
    free_dev(c->d_rmax);
    free_dev(c->d_med);
    free_dev(c->d_mcnt);
    free_dev(c->d_warn_run);
    c->d_warn_run = nullptr;
    for (auto* q : c->rlog) free_dev(q);
    c->rlog.clear();
    c->rlog_cap.clear();
    c->rlog_sorted.clear();
    if (c->h_rlog_ptr) cudaFreeHost(c->h_rlog_ptr);
    if (c->h_rlog_cap) cudaFreeHost(c->h_rlog_cap);
    c->h_rlog_ptr = nullptr;
    c->h_rlog_cap = nullptr;
    free_dev(c->d_rlog_ptr);
    free_dev(c->d_rlog_cap);
    free_dev(c->d_rlog_cnt);
    free_dev(c->d_rlog_tmp);
    free_dev(c->d_rs_hist);
    c->d_rlog_ptr = nullptr;
    c->d_rlog_cap = nullptr;
    c->d_rlog_cnt = nullptr;
    c->d_rlog_tmp = nullptr;
    c->d_rs_hist = nullptr;
    c->rlog_tmp_cap = 0;
    c->rs_hist_cap = 0;
    free_dev(c->d_hkeys);
    free_dev(c->d_hrows);
    free_dev(c->d_hover);
    free_dev(c->d_hrate);
    c->d_hrate = nullptr;
    c->d_hkeys = nullptr;
    c->d_hrows = nullptr;
    c->d_hover = nullptr;
    c->hcap = 0;
    c->d_hist = nullptr;
    c->d_rmin = nullptr;
    c->d_rmax = nullptr;
    c->d_med = nullptr;
    c->d_mcnt = nullptr;
    c->d_acc = nullptr;
    c->d_dirty = nullptr;
    c->d_stats = nullptr;
    c->d_rate = nullptr;
    c->d_flag = nullptr;
    c->d_flag_keys = nullptr;
    c->n_slots = 0;
}

static gnm_status find_window(gnm_ctx* c, uint64_t wid, uint32_t* s) {
    if (!c->have_registry) return fail(GNM_E_STATE, "no registry loaded");
    auto it = c->slot_of.find(wid);
    if (it == c->slot_of.end())
        return fail(GNM_E_STATE, "unknown or evicted window id " + std::to_string(wid));
    *s = it->second;
    return GNM_OK;
}

// ------------------------------------------------------------- launch buffers

gnm_status acquire_ring(gnm_ctx* c, uint32_t n_win, LaunchBuf** out) {
    LaunchBuf& b = c->ring[c->ring_next];
    c->ring_next = (c->ring_next + 1) % kRingSize;
    if (b.ev_recorded) GNM_CU(cudaEventSynchronize(b.ev));  // its previous launch is done
    if (b.cap < n_win || b.cap == 0) {
        const uint32_t cap = std::max<uint32_t>(n_win, 64);
        if (b.h_wins) cudaFreeHost(b.h_wins);
        free_dev(b.d_wins);
        free_dev(b.d_done);
        b.h_wins = nullptr;
        b.d_wins = nullptr;
        b.d_done = nullptr;
        b.cap = 0;
        GNM_CU(cudaMallocHost(&b.h_wins, sizeof(WinDesc) * cap));
        GNM_CU(cudaMalloc(&b.d_wins, sizeof(WinDesc) * cap));
        GNM_CU(cudaMalloc(&b.d_done, sizeof(uint32_t) * cap));
        GNM_CU(cudaMemset(b.d_done, 0, sizeof(uint32_t) * cap));
        b.cap = cap;
    }
    *out = &b;
    return GNM_OK;
}

// Host records that the kernels may read in place: page-locked host memory mapped for the
// device (the runtime reports a device address for it). out[k]: the device address of
// field k's element `base`.
static bool host_addressable(gnm_ctx* c, const gnm_records* rec, uint64_t base, const uint32_t* out[6]) {
    if (c->cfg.host_records == GNM_HOST_STAGE || c->cfg.host_records == GNM_HOST_PIPELINE) return false;
    const uint32_t* f[6] = {rec->srcaddr, rec->dstaddr, rec->dPkts, rec->dOctets, rec->first, rec->last};
    for (int k = 0; k < 6; ++k) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, f[k] + base) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return false;
        out[k] = static_cast<const uint32_t*>(a.devicePointer);
    }
    return true;
}

static gnm_status stage_records(gnm_ctx* c, const gnm_records* rec, uint64_t lo, uint64_t hi,
                                cudaStream_t st, const uint32_t* out[6]) {
    Staging& g = c->staging;
    if (g.ev_recorded) GNM_CU(cudaEventSynchronize(g.ev));
    const uint64_t n = hi - lo;
    if (g.cap < n) {
        for (auto& p : g.d) {
            free_dev(p);
            p = nullptr;
        }
        g.cap = 0;
        const uint64_t cap = std::max<uint64_t>(n, 1 << 16);
        for (auto& p : g.d) GNM_CU(cudaMalloc(&p, cap * 4));
        g.cap = cap;
    }
    const uint32_t* src[6] = {rec->srcaddr, rec->dstaddr, rec->dPkts, rec->dOctets, rec->first, rec->last};
    for (int k = 0; k < 6; ++k) {
        if (n) GNM_CU(cudaMemcpyAsync(g.d[k], src[k] + lo, n * 4, cudaMemcpyHostToDevice, st));
        out[k] = g.d[k];
    }
    GNM_CU(cudaEventRecord(g.ev, st));
    g.ev_recorded = true;
    return GNM_OK;
}

// ------------------------------------------------------------- shapes and params

gnm_status choose_shape(gnm_ctx* c, uint64_t n, LaunchShape* s, size_t n_win) {
    const gnm_config& cfg = c->cfg;
    const uint32_t nr = (uint32_t)c->h_starts.size();
    int mode = cfg.lookup_mode;
    if (mode == GNM_LOOKUP_AUTO)  // a registry that fits shared memory is searched there directly
        mode = c->rmi_ready ? GNM_LOOKUP_RMI
               : (size_t)nr * 8 <= kRegistrySmemMax ? GNM_LOOKUP_BSEARCH : GNM_LOOKUP_RADIX;
    if (mode == GNM_LOOKUP_RMI && !c->rmi_ready)
        return fail(GNM_E_STATE, "lookup mode RMI requested but no learned index is trained");
    size_t lookup_bytes = 0;
    s->radix_bits = 0;
    s->dir_iters = 0;
    s->rmi_global = 0;
    if (mode == GNM_LOOKUP_HASH24) {
        if (!c->d_h24) return fail(GNM_E_INVAL, "lookup mode HASH24: the registry has prefixes longer than /24");
        s->lookup = kLookupHash24;
    } else if (mode == GNM_LOOKUP_RMI) {
        s->lookup = kLookupRmi;
        // leaf parameters staged in shared memory, or read (16 bytes per lookup) from global
        // memory: placement L2, or AUTO when they do not fit
        const size_t leaf_bytes = (size_t)c->rmi.n_models * 16;
        int place = cfg.placement != GNM_PLACE_AUTO ? cfg.placement : c->tuned.placement;
        if (place == GNM_PLACE_STAGED) place = GNM_PLACE_AUTO;
        const bool fits = leaf_bytes + 1024 <= (size_t)c->smem_optin;
        if (place == GNM_PLACE_SMEM && !fits)
            return fail(GNM_E_INVAL, "learned-index leaves too large for shared memory");
        s->rmi_global = place == GNM_PLACE_L2 || !fits;
        lookup_bytes = s->rmi_global ? 0 : leaf_bytes;
    } else if (mode == GNM_LOOKUP_RADIX) {
        uint32_t bits = cfg.radix_bits ? cfg.radix_bits : c->tuned.radix_bits;
        if (bits && (bits < 4 || bits > 16)) return fail(GNM_E_INVAL, "radix_bits must be 4..16");
        if (!bits) {  // about two buckets per range, shrunk while it crowds out direct rows
            uint32_t lg = 0;
            while ((1ull << lg) < nr) ++lg;
            bits = std::min<uint32_t>(14, std::max<uint32_t>(8, lg + 1));  // directory <= 64 KB
            const size_t direct = (size_t)c->keys * kSmemRowBytes;
            const uint32_t floor_bits = std::max<uint32_t>(8, lg > 3 ? lg - 3 : 0);
            while (bits > floor_bits && direct <= kDirectTableMax &&
                   direct + ((size_t)1 << bits) * 4 + 4 + 1024 > (size_t)c->smem_optin)
                --bits;
        }
        s->lookup = kLookupRadix;
        s->radix_bits = bits;
        lookup_bytes = ((size_t)1 << bits) * 4 + 4;
    } else if (mode == GNM_LOOKUP_BSEARCH) {
        int place = cfg.placement != GNM_PLACE_AUTO ? cfg.placement : c->tuned.placement;
        const size_t sample_bytes = (size_t)c->n_blocks * 4;
        if (place == GNM_PLACE_AUTO)
            place = (size_t)nr * 8 <= kRegistrySmemMax ? GNM_PLACE_SMEM
                    : sample_bytes <= kSampleSmemMax   ? GNM_PLACE_STAGED
                                                       : GNM_PLACE_L2;
        if (place == GNM_PLACE_SMEM && (size_t)nr * 8 + 1024 > (size_t)c->smem_optin)
            return fail(GNM_E_INVAL, "registry too large for shared-memory placement");
        if (place == GNM_PLACE_STAGED && sample_bytes + 1024 > (size_t)c->smem_optin)
            return fail(GNM_E_INVAL, "registry too large for staged placement");
        if (place == GNM_PLACE_SMEM) {
            s->lookup = kLookupSmem;
            lookup_bytes = (size_t)nr * 8;
            // radix_bits > 0: a directory over the top bits in front of the search, when it
            // fits beside the ranges (0: the search covers all ranges)
            const uint32_t bits = cfg.radix_bits ? cfg.radix_bits : c->tuned.radix_bits;
            if (bits && (bits < 4 || bits > 16)) return fail(GNM_E_INVAL, "radix_bits must be 4..16");
            const size_t dir_bytes = (((size_t)1 << bits) + 1) * 4;
            if (bits && lookup_bytes + dir_bytes + 1024 <= (size_t)c->smem_optin) {
                s->radix_bits = bits;
                lookup_bytes += dir_bytes;
                // every lane takes the same number of search steps: enough for the largest
                // bucket (ranges [first range of bucket t, first range of bucket t+1])
                const std::vector<uint32_t>& st = c->h_starts;
                uint32_t longest = 1, prev = 0;
                for (uint64_t t = 1; t <= ((uint64_t)1 << bits); ++t) {
                    const uint64_t a = t << (32 - bits);
                    const uint32_t i = a >> 32 ? nr - 1u
                                               : (uint32_t)(std::upper_bound(st.begin(), st.end(), (uint32_t)a) -
                                                            st.begin()) - 1u;
                    longest = std::max(longest, i - prev + 1u);
                    prev = i;
                }
                uint32_t it = 0;
                while ((1u << it) < longest) ++it;
                s->dir_iters = it;
            }
        } else if (place == GNM_PLACE_STAGED) {
            s->lookup = kLookupStaged;
            lookup_bytes = sample_bytes;
        } else if (place == GNM_PLACE_L2) {
            s->lookup = kLookupL2;
        } else {
            return fail(GNM_E_INVAL, "unknown placement");
        }
    } else {
        return fail(GNM_E_INVAL, "unknown lookup mode");
    }
    // split launches: the lookup structure lives in the key kernel only
    int split = cfg.split != GNM_SPLIT_AUTO ? cfg.split : c->tuned.split;
    if (split == GNM_SPLIT_AUTO) split = s->lookup == kLookupSmem ? GNM_SPLIT_FUSED : GNM_SPLIT_TWO_KERNELS;
    if (c->hcap) {  // per-host sums read the key kernel's keys
        if (cfg.split == GNM_SPLIT_FUSED) return fail(GNM_E_INVAL, "per-host statistics need split launches");
        split = GNM_SPLIT_TWO_KERNELS;
    }
    if (split != GNM_SPLIT_FUSED && split != GNM_SPLIT_TWO_KERNELS) return fail(GNM_E_INVAL, "unknown split mode");
    s->split = split == GNM_SPLIT_TWO_KERNELS;
    s->keys_smem = s->split ? (lookup_bytes + 15) / 16 * 16 : 0;
    s->keys_blk = 0;
    s->keys_h16 = 0;
    s->keys_bits = 0;
    if (cfg.key_directory < 0 || cfg.key_directory > 4) return fail(GNM_E_INVAL, "key_directory must be 0..4");
    const int key_dir = cfg.key_directory ? cfg.key_directory : c->tuned.key_dir;
    if (s->split && s->lookup == kLookupRadix && key_dir == 4) {
        // 16-bit directory and samples of 2-range blocks (block indices below 2^16)
        const size_t one = (size_t)c->smem_optin > 1024 ? (size_t)c->smem_optin - 1024 : 0;
        const size_t bytes = (65537 * 2 + 15) / 16 * 16 + ((size_t)c->n_blk2 * 2 + 15) / 16 * 16;
        if (c->d_dirh && bytes <= one) {
            s->keys_blk = 2;
            s->keys_h16 = 1;
            s->keys_bits = 16;
            s->keys_smem = bytes;
        } else {
            return fail(GNM_E_INVAL, "key_directory 4 needs fewer than 65,536 two-range blocks that fit in "
                                     "shared memory");
        }
    }
    if (s->split && s->lookup == kLookupRadix && key_dir != 2 && key_dir != 4 && !s->keys_h16) {
        // block samples in the key kernel's shared memory next to a directory of block
        // indices: 2-range blocks (one 16-byte load) when they fit, else 4-range blocks
        // (32 bytes); else the plain directory
        const size_t one = (size_t)c->smem_optin > 1024 ? (size_t)c->smem_optin - 1024 : 0;
        auto bytes = [&](uint32_t kb, uint32_t nb) {
            return ((((size_t)1 << kb) + 1) * 4 + 15) / 16 * 16 + ((size_t)nb * 4 + 15) / 16 * 16;
        };
        uint32_t kb0 = cfg.radix_bits ? cfg.radix_bits : c->tuned.radix_bits;
        if (kb0 && (kb0 < 4 || kb0 > 16)) return fail(GNM_E_INVAL, "radix_bits must be 4..16");
        for (int br : {2, 4}) {
            if (key_dir == 1 && br == 2) continue;
            if (key_dir == 3 && br == 4) continue;
            const uint32_t nb = br == 2 ? c->n_blk2 : c->n_blk4;
            uint32_t kb = kb0;
            if (!kb)  // the largest directory (<= 14 bits) that fits beside the samples
                for (kb = 14; kb > 8 && bytes(kb, nb) > one; --kb) {}
            if (bytes(kb, nb) <= one) {
                s->keys_blk = br;
                s->keys_bits = kb;
                s->keys_smem = bytes(kb, nb);
                break;
            }
        }
        if (!s->keys_blk && (key_dir == 1 || key_dir == 3))
            return fail(GNM_E_INVAL, "block samples do not fit in shared memory (key_directory " +
                                         std::to_string(key_dir) + ")");
    }
    if (s->split && s->keys_smem + 1024 > (size_t)c->smem_optin)
        return fail(GNM_E_INVAL, "lookup structure too large for shared memory");
    if (!s->split && s->lookup == kLookupRadix && lookup_bytes + 1024 > (size_t)c->smem_optin)
        return fail(GNM_E_INVAL, "radix directory too large for shared memory");
    if (s->split) lookup_bytes = 0;
    const size_t budget = (size_t)c->smem_optin > lookup_bytes + 1024 ? (size_t)c->smem_optin - lookup_bytes - 1024 : 0;
    const size_t direct = (size_t)c->keys * kSmemRowBytes;
    const size_t row = kSmemRowBytes + 4;
    uint32_t cap = 0;
    int tm = cfg.table_mode;
    // partitioned launches: groups of part_rows keys (a multiple of 256 that one direct
    // table holds), at most kPartMaxBuckets (window, group) buckets, fewer than 2^32 records
    const uint32_t part_rows = (uint32_t)(std::min(kDirectTableMax, budget) / kSmemRowBytes) & ~255u;
    const uint32_t part_groups = part_rows ? (c->keys + part_rows - 1) / part_rows : 0u;
    const bool part_ok = s->split && part_rows >= 256 &&
                         (uint64_t)part_groups * std::max<size_t>(n_win, 1) <= kPartMaxBuckets && n < 0xFFFFFFFFull;
    if (tm == GNM_TABLE_AUTO)
        tm = direct <= std::min(kDirectTableMax, budget) ? GNM_TABLE_DIRECT
             : part_ok && part_groups > 1                 ? GNM_TABLE_PARTITION
                                                          : GNM_TABLE_HASH;
    s->part = 0;
    s->part_rows = 0;
    s->part_groups = 0;
    s->part_grid = 0;
    uint32_t rows = c->keys;  // rows of a direct table
    if (tm == GNM_TABLE_PARTITION) {
        if (!part_ok)
            return fail(GNM_E_INVAL, "table_mode PARTITION needs split launches, more keys than one table "
                                     "holds, at most 8192 (window, key group) buckets and < 2^32 records");
        s->table = kTableDirect;
        s->part = 1;
        s->part_rows = part_rows;
        s->part_groups = part_groups;
        rows = part_rows;
    } else if (tm == GNM_TABLE_DIRECT) {
        if (direct > budget) return fail(GNM_E_INVAL, "per-site sums do not fit in shared memory (table_mode DIRECT)");
        s->table = kTableDirect;
    } else if (tm == GNM_TABLE_HASH) {
        if (cfg.hash_slots) {
            cap = cfg.hash_slots;
            if (cap < 256 || cap > 65536 || (cap & 1u))
                return fail(GNM_E_INVAL, "hash_slots must be even, 256..65536");
            if ((size_t)cap * row > budget) return fail(GNM_E_INVAL, "hash_slots do not fit in shared memory");
        } else {  // as many slot pairs as fit
            cap = (uint32_t)(std::min(kHashTableMax, budget) / row) & ~1u;
            if (cap > 65536) cap = 65536;
        }
        s->table = cap >= 256 ? kTableHash : kTableGlobal;
        if (s->table == kTableGlobal) cap = 0;
    } else if (tm == GNM_TABLE_GLOBAL) {
        s->table = kTableGlobal;
    } else {
        return fail(GNM_E_INVAL, "unknown table_mode");
    }
    int agg = cfg.aggregation != GNM_AGG_AUTO ? cfg.aggregation : c->tuned.agg;
    s->agg = agg == GNM_AGG_WARP ? GNM_AGG_WARP : GNM_AGG_DIRECT;
    // untuned defaults: 1024 threads, one group of four records per thread and step; split
    // launches into direct tables: 512 threads with the next group in flight (unroll 3)
    const bool piped = s->split && s->table == kTableDirect && s->agg == GNM_AGG_DIRECT && !cfg.unroll;
    int block = cfg.block_threads ? cfg.block_threads : (c->tuned.block ? c->tuned.block : (piped ? 512 : 1024));
    int unroll = cfg.unroll ? cfg.unroll : (c->tuned.unroll ? c->tuned.unroll : (piped && block <= 768 ? 3 : 1));
    if (block < 64 || block > 1024 || block % 32) return fail(GNM_E_INVAL, "block_threads must be 64..1024, multiple of 32");
    if (unroll < 1 || unroll > 3) return fail(GNM_E_INVAL, "unroll must be 1, 2 or 3");
    if (unroll == 3 && !(s->split && s->table == kTableDirect && s->agg == GNM_AGG_DIRECT)) unroll = 1;
    if (unroll > 1 && block > agg_block_max(s->split ? kLookupKeys : s->lookup, s->table, s->agg, unroll)) unroll = 1;
    s->block = block;
    s->unroll = unroll;
    s->smem = aggregate_smem_bytes(s->split ? kLookupKeys : s->lookup, s->table, nr, rows, cap,
                                   s->lookup == kLookupRmi && !s->rmi_global ? c->rmi.n_models : 0, s->radix_bits);
    if (s->smem > (size_t)c->smem_optin) return fail(GNM_E_INVAL, "shared-memory layout exceeds the device limit");
    int cps = cfg.ctas_per_sm ? cfg.ctas_per_sm : c->tuned.ctas_per_sm;
    const int by_threads = std::max(1, 2048 / block);
    const int by_smem = s->smem ? std::max(1, (int)(c->smem_per_sm / (s->smem + 1024))) : 32;
    const int fit = std::min(by_threads, by_smem);
    if (cps <= 0 || cps > fit) cps = fit;
    s->ctas_per_sm = cps;
    const uint64_t resident = (uint64_t)c->sm_count * cps;
    const uint64_t min_per_cta = (uint64_t)block * 8;  // at least two groups of 4 per thread
    uint64_t grid = std::min<uint64_t>(resident, std::max<uint64_t>(1, ceil_div(n, min_per_cta)));
    s->grid = (int)grid;
    if (s->split) {  // key kernel: as many CTAs per SM as its shared memory allows
        int ku = c->tuned.keys_unroll ? c->tuned.keys_unroll : s->unroll;
        if (ku != 1 && ku != 2) ku = 1;
        const int lk = s->keys_h16 ? kLookupRadixBlk2H
                       : s->keys_blk == 2 ? kLookupRadixBlk2 : s->keys_blk == 4 ? kLookupRadixBlk : s->lookup;
        s->keys_unroll = ku;
        s->keys_block = keys_block_max(lk, ku);
        const int kfit = std::max(1, std::min(2048 / s->keys_block, (int)(c->smem_per_sm / (s->keys_smem + 1024))));
        const uint64_t kres = (uint64_t)c->sm_count * kfit;
        s->keys_grid = (int)std::min<uint64_t>(kres, std::max<uint64_t>(1, ceil_div(n, (uint64_t)s->keys_block * 4 * ku)));
        if (s->part)  // count and scatter: one 1024-thread CTA per SM, at least 4096 records each
            s->part_grid = (int)std::min<uint64_t>((uint64_t)c->sm_count * 2, std::max<uint64_t>(1, ceil_div(n, 4096)));
    } else {
        s->keys_unroll = 1;
        s->keys_block = 0;
        s->keys_grid = 0;
    }
    s->cap = cap;
    return GNM_OK;
}

gnm_status build_params(gnm_ctx* c, const gnm_records* rec, AggParams* p) {
    std::memset(p, 0, sizeof(*p));
    p->src = rec->srcaddr;
    p->dst = rec->dstaddr;
    p->pkts = rec->dPkts;
    p->oct = rec->dOctets;
    p->first = rec->first;
    p->last = rec->last;
    p->starts = c->d_starts;
    p->rsite = c->d_site;
    p->pairs = c->d_pairs;
    p->blocks = reinterpret_cast<const uint4*>(c->d_blocks);
    p->sample = c->d_sample;
    p->dir16 = c->d_dir16;
    p->sample4 = c->d_sample4;
    p->n_blk4 = c->n_blk4;
    p->sample2 = c->d_sample2;
    p->n_blk2 = c->n_blk2;
    p->dirh = c->d_dirh;
    p->smp16 = c->d_smp16;
    p->h24 = c->d_h24;
    p->h24_mask = c->h24_mask;
    p->n_blocks = c->n_blocks;
    p->n_ranges = (uint32_t)c->h_starts.size();
    p->n_sites = c->n_sites;
    p->rmi = c->rmi;
    p->rmi.check_err = c->d_check;
    p->check_err = c->d_check;
    for (uint32_t i = 0; i < GNM_MAX_LOCAL; ++i) {
        p->local_pfx[i] = c->local_pfx[i];
        p->local_mask[i] = c->local_mask[i];
    }
    p->n_local = c->n_local;
    p->min_avg = c->cfg.min_avg_pkt_bytes;
    p->min_pkts = c->cfg.min_pkts;
    p->min_dur = c->cfg.min_dur_ms;
    p->admin_rule = c->cfg.admin_rule;
    p->acc = c->d_acc;
    p->dirty = c->d_dirty;
    p->dirty_groups = (c->keys + 31) / 32;
    p->stats = c->d_stats;
    p->rate = c->d_rate;
    p->flag = c->d_flag;
    p->keys = c->keys;
    p->table_rows = c->keys;
    p->hist = c->d_hist;
    p->rmin = c->d_rmin;
    p->rmax = c->d_rmax;
    p->rlog = c->d_hist ? nullptr : c->d_rlog_ptr;
    p->rlog_cap = c->d_rlog_cap;
    p->rlog_cnt = c->d_rlog_cnt;
    p->hkeys = c->d_hkeys;
    p->hrows = c->d_hrows;
    p->hover = c->d_hover;
    p->hcap = c->hcap;
    p->min_flows = c->cfg.min_flows_to_flag;
    p->threshold = c->cfg.threshold_bps;
    p->violations = c->d_violations;
    return GNM_OK;
}

static gnm_status check_records(const gnm_records* rec, uint64_t need) {
    if (!rec) return fail(GNM_E_INVAL, "records is NULL");
    if (rec->n < need) return fail(GNM_E_INVAL, "records->n is smaller than the windows need");
    if (rec->n == 0) return GNM_OK;
    const uint32_t* f[6] = {rec->srcaddr, rec->dstaddr, rec->dPkts, rec->dOctets, rec->first, rec->last};
    for (auto* q : f) {
        if (!q) return fail(GNM_E_INVAL, "a record field pointer is NULL");
        if (((uintptr_t)q & 3u) != 0) return fail(GNM_E_INVAL, "record arrays must be 4-byte aligned");
    }
    return GNM_OK;
}

gnm_status check_windows(gnm_ctx* c, const gnm_records* rec, const uint64_t* offsets, size_t n_win) {
    if (!c->have_registry) return fail(GNM_E_STATE, "no registry loaded");
    if (!offsets) return fail(GNM_E_INVAL, "offsets are NULL");
    for (size_t k = 0; k < n_win; ++k) {
        if (offsets[k + 1] < offsets[k]) return fail(GNM_E_INVAL, "offsets must be non-decreasing");
        if (offsets[k + 1] - offsets[k] > kMaxWindowRecords) return fail(GNM_E_INVAL, "a window holds 2^32 records or more");
    }
    if (n_win > c->n_slots) return fail(GNM_E_CAPACITY, "more windows in one call than result slots");
    return check_records(rec, offsets[n_win]);
}

gnm_status prepare_launch(gnm_ctx* c, const gnm_records* dr, const uint64_t* offsets, size_t n_win,
                          const uint32_t* slots, bool finalize, Prepared* out) {
    const uint64_t base = offsets[0], N = offsets[n_win] - offsets[0];
    out->n = N;
    out->wins.clear();
    if (N == 0) return GNM_OK;
    AggParams& p = out->p;
    GNM_TRY(build_params(c, dr, &p));
    LaunchShape& sh = out->sh;
    GNM_TRY(choose_shape(c, N, &sh, n_win));
    p.table_cap = sh.cap;
    p.radix_bits = sh.radix_bits;
    p.dir_iters = sh.dir_iters;
    p.rmi.leaves_global = sh.rmi_global ? 1u : 0u;
    p.n_total = N;
    uint64_t chunk = ceil_div(N, (uint64_t)sh.grid);
    chunk = (chunk + 3) & ~3ull;
    sh.grid = (int)ceil_div(N, chunk);
    p.chunk = chunk;
    const uintptr_t a0 = (uintptr_t)dr->srcaddr & 15u;
    const uint32_t* f[6] = {dr->srcaddr, dr->dstaddr, dr->dPkts, dr->dOctets, dr->first, dr->last};
    p.vec_ok = 1;
    for (auto* q : f)
        if (((uintptr_t)q & 15u) != a0) p.vec_ok = 0;
    p.phase = (uint32_t)(a0 >> 2);
    // one CTA finalises a window in place when its key space is small; larger ones are
    // finalised by a grid-wide kernel after the aggregation (partial sums or per window)
    out->fin_in_kernel = finalize && c->keys <= kFinalizeInCtaMaxKeys;
    out->fin_grid = finalize && !out->fin_in_kernel;
    uint64_t parts = 0;
    for (size_t k = 0; k < n_win; ++k) {
        const uint64_t b = offsets[k] - base, e = offsets[k + 1] - base;
        if (b == e) continue;
        WinDesc w;
        w.begin = b;
        w.end = e;
        w.slot = slots[k];
        w.flags = out->fin_in_kernel ? kWinFinalize : 0u;
        w.ctas = (uint32_t)((e - 1) / chunk - b / chunk + 1);
        w.part_base = (uint32_t)parts;
        const uint64_t np = w.ctas;  // one partial block per CTA segment of the window
        w.n_parts = (uint32_t)np;
        w.key_base = 0;
        parts += np;
        out->wins.push_back(w);
    }
    // direct tables of finalising launches hand their sums over through plain stores
    out->partial_words = 0;
    out->n_buckets = 0;
    out->part_bytes = 0;
    if (sh.part) {
        out->n_buckets = (uint32_t)(out->wins.size() * sh.part_groups);
        out->part_bytes = part_layout(N, out->n_buckets).bytes;
        // finalising launches: a block per (bucket, CTA) segment, at most one per CTA plus
        // one per bucket; otherwise (or past the limit) the segments add to the accumulators
        const uint64_t words = ((uint64_t)sh.grid + out->n_buckets) * part_stride_words(sh.part_rows);
        if (out->fin_grid && words * 4 <= kPartialBytesMax) out->partial_words = words;
    } else if (sh.table == kTableDirect && (out->fin_in_kernel || out->fin_grid)) {
        const uint64_t words = parts * part_stride_words(c->keys);
        if (words * 4 <= kPartialBytesMax) out->partial_words = words;
    }
    return GNM_OK;
}

PartLayout part_layout(uint64_t n, uint32_t nb) {
    PartLayout l;
    l.cnt = 4 * part_array_stride(n) * 4;
    l.descs = (l.cnt + (uint64_t)nb * 4 + 15) & ~15ull;
    l.pdesc = l.descs + (uint64_t)nb * sizeof(WinDesc);
    l.bytes = l.pdesc + (uint64_t)nb * sizeof(uint2);
    return l;
}

gnm_status clear_rate_stats(gnm_ctx* c, const uint32_t* slots, size_t n, cudaStream_t st) {
    if (!c->d_hist && !c->d_rlog_cnt && !c->d_hkeys) return GNM_OK;
    const size_t nk = (size_t)2 * c->n_sites, hc = c->hcap;
    for (size_t k = 0; k < n;) {  // runs of consecutive slots: one memset per array
        size_t m = 1;
        while (k + m < n && slots[k + m] == slots[k] + m) ++m;
        const size_t s0 = slots[k];
        if (c->d_hist) GNM_CU(cudaMemsetAsync(c->d_hist + s0 * nk * kRateBuckets, 0, m * nk * kRateBuckets * 4, st));
        if (c->d_rlog_cnt) {
            GNM_CU(cudaMemsetAsync(c->d_rlog_cnt + s0, 0, m * 4, st));
            for (size_t j = s0; j < s0 + m; ++j) c->rlog_sorted[j] = 0;
        }
        if (c->d_hist || c->d_rlog_cnt) {
            GNM_CU(cudaMemsetAsync(c->d_rmax + s0 * nk, 0, m * nk * 8, st));
            GNM_CU(cudaMemsetAsync(c->d_rmin + s0 * nk, 0xFF, m * nk * 8, st));  // above every rate
        }
        if (c->d_hkeys) {
            GNM_CU(cudaMemsetAsync(c->d_hkeys + s0 * hc, 0, m * hc * 8, st));
            GNM_CU(cudaMemsetAsync(c->d_hrows + s0 * hc * kNStat, 0, m * hc * kNStat * 8, st));
            GNM_CU(cudaMemsetAsync(c->d_hover + s0, 0, m * 4, st));
        }
        k += m;
    }
    return GNM_OK;
}

gnm_status reserve_rate_log(gnm_ctx* c, const uint32_t* slots, const uint64_t* need, size_t n, cudaStream_t st) {
    if (!c->d_rlog_cnt) return GNM_OK;
    bool synced = false;
    for (size_t k = 0; k < n; ++k) {
        const uint32_t s = slots[k];
        if (need[k] <= c->rlog_cap[s]) continue;
        if (need[k] > 0xFFFFFFFFull) return fail(GNM_E_INVAL, "a window holds 2^32 records or more");
        if (!synced) {  // nothing queued may still use a log that is replaced
            GNM_CU(cudaStreamSynchronize(st));
            synced = true;
        }
        const uint64_t cap = std::min<uint64_t>(0xFFFFFFFFull,
                                                std::max<uint64_t>({need[k], 2 * c->rlog_cap[s], 1ull << 16}));
        uint32_t* nb = nullptr;
        if (cudaMalloc(&nb, cap * 4) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(GNM_E_NOMEM, "rate-statistics log allocation failed (" + std::to_string(cap * 4) + " bytes)");
        }
        if (c->rlog[s] && c->rlog_cap[s]) {  // an open window keeps the words logged so far
            const cudaError_t e = cudaMemcpyAsync(nb, c->rlog[s], c->rlog_cap[s] * 4, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) {
                cudaFree(nb);
                GNM_CU(e);
            }
        }
        c->h_rlog_ptr[s] = nb;
        c->h_rlog_cap[s] = (uint32_t)cap;
        GNM_CU(cudaMemcpyAsync(c->d_rlog_ptr + s, c->h_rlog_ptr + s, sizeof(uint32_t*), cudaMemcpyHostToDevice, st));
        GNM_CU(cudaMemcpyAsync(c->d_rlog_cap + s, c->h_rlog_cap + s, 4, cudaMemcpyHostToDevice, st));
        GNM_CU(cudaStreamSynchronize(st));
        free_dev(c->rlog[s]);
        c->rlog[s] = nb;
        c->rlog_cap[s] = cap;
    }
    return GNM_OK;
}

gnm_status enqueue_prepared(gnm_ctx* c, Prepared& pr, const uint64_t* offsets, size_t n_win,
                            const uint32_t* slots, bool finalize, WinDesc* d_wins, uint32_t* d_done,
                            uint32_t* d_partials, uint32_t* d_keys, unsigned char* d_part, cudaStream_t st,
                            uint32_t* launches, cudaEvent_t* marks, int32_t* kinds, bool fresh) {
    *launches = 0;
    if (fresh) GNM_TRY(clear_rate_stats(c, slots, n_win, st));
    // an external event node when captured into a graph, so that the host can read it
    auto mark = [&](int32_t kind) -> gnm_status {
        if (!marks) return GNM_OK;
        if (kind >= 0) kinds[*launches - 1] = kind;
        GNM_CU(cudaEventRecordWithFlags(marks[*launches], st, cudaEventRecordExternal));
        return GNM_OK;
    };
    if (pr.n) {
        pr.p.wins = d_wins;
        pr.p.n_wins = (uint32_t)pr.wins.size();
        pr.p.done = d_done;
        pr.p.partials = pr.partial_words ? d_partials : nullptr;
        pr.p.partial_cap = pr.partial_words;
        GNM_TRY(mark(-1));
        if (pr.sh.part) {
            // keys; regrouping by (window, key group); sums per group; grid finalisation
            uint32_t* keys = d_keys + pr.p.phase;
            const PartLayout L = part_layout(pr.n, pr.n_buckets);
            uint32_t* out = reinterpret_cast<uint32_t*>(d_part);
            uint32_t* cnt = reinterpret_cast<uint32_t*>(d_part + L.cnt);
            WinDesc* descs = reinterpret_cast<WinDesc*>(d_part + L.descs);
            uint2* pdesc = reinterpret_cast<uint2*>(d_part + L.pdesc);
            // the key kernel also counts the records of every (window, key group) bucket when
            // its shared memory has room for the counts; else the count kernel does
            const uint32_t nb = pr.p.n_wins * pr.sh.part_groups;
            AggParams pk = pr.p;
            LaunchShape sk = pr.sh;
            if (pr.sh.keys_blk) pk.radix_bits = pr.sh.keys_bits;
            const size_t hist_off = (pr.sh.keys_smem + 15) / 16 * 16;
            const bool fold = hist_off + (size_t)nb * 4 + 1024 <= (size_t)c->smem_optin;
            if (fold) {
                GNM_CU(cudaMemsetAsync(cnt, 0, (size_t)nb * 4, st));
                pk.key_hist = cnt;
                pk.part_groups = pr.sh.part_groups;
                pk.key_group_rows = pr.sh.part_rows;
                pk.key_hist_off = (uint32_t)hist_off;
                sk.keys_smem = hist_off + (size_t)nb * 4;
            }
            GNM_CU(launch_keys(pk, sk, keys, st));
            ++*launches;
            GNM_TRY(mark(GNM_KERNEL_KEYS));
            if (pr.p.hkeys) {
                GNM_CU(launch_host_stats(pr.p, keys, c->sm_count * 4, st));
                ++*launches;
                GNM_TRY(mark(GNM_KERNEL_HOSTS));
            }
            AggParams pp = pr.p;
            pp.src = keys;
            pp.dst = keys;
            if (!fold) {
                GNM_CU(launch_part_count(pp, pr.sh, cnt, st));
                ++*launches;
                GNM_TRY(mark(GNM_KERNEL_PART_COUNT));
            }
            GNM_CU(launch_part_scan(pp, pr.sh, pr.p.chunk, cnt, descs, pdesc, st));
            ++*launches;
            GNM_TRY(mark(GNM_KERNEL_PART_SCAN));
            GNM_CU(launch_part_scatter(pp, pr.sh, cnt, out, st));
            ++*launches;
            GNM_TRY(mark(GNM_KERNEL_PART_SCATTER));
            const uint64_t stride = part_array_stride(pr.n);
            AggParams pa = pr.p;
            pa.src = out;
            pa.dst = out;
            pa.pkts = out + stride;
            pa.oct = out + 2 * stride;
            pa.first = nullptr;  // regrouped records carry the duration as `last`
            pa.last = out + 3 * stride;
            pa.vec_ok = 1;
            pa.phase = 0;
            pa.wins = descs;
            pa.n_wins = pr.n_buckets;
            pa.table_rows = pr.sh.part_rows;
            GNM_CU(launch_aggregate(pa, pr.sh, st));
            ++*launches;
            GNM_TRY(mark(GNM_KERNEL_AGGREGATE));
            if (finalize) {
                AggParams pf = pr.p;
                pf.table_rows = pr.sh.part_rows;
                pf.part_groups = pr.sh.part_groups;
                pf.part_desc = pdesc;
                GNM_CU(launch_finalize_windows(pf, st));
                ++*launches;
                GNM_TRY(mark(GNM_KERNEL_FINALIZE));
            }
        } else if (pr.sh.split) {  // keys first (same 16-byte phase as the records), then the sums
            uint32_t* keys = d_keys + pr.p.phase;
            AggParams pk = pr.p;
            if (pr.sh.keys_blk) pk.radix_bits = pr.sh.keys_bits;
            GNM_CU(launch_keys(pk, pr.sh, keys, st));
            ++*launches;
            GNM_TRY(mark(GNM_KERNEL_KEYS));
            if (pr.p.hkeys) {
                GNM_CU(launch_host_stats(pr.p, keys, c->sm_count * 4, st));
                ++*launches;
                GNM_TRY(mark(GNM_KERNEL_HOSTS));
            }
            AggParams pa = pr.p;
            pa.src = keys;
            pa.dst = keys;
            GNM_CU(launch_aggregate(pa, pr.sh, st));
        } else {
            GNM_CU(launch_aggregate(pr.p, pr.sh, st));
        }
        if (!pr.sh.part) {
            ++*launches;
            GNM_TRY(mark(GNM_KERNEL_AGGREGATE));
            if (finalize && pr.fin_grid) {
                GNM_CU(launch_finalize_windows(pr.p, st));
                ++*launches;
                GNM_TRY(mark(GNM_KERNEL_FINALIZE));
            }
        }
    }
    // empty windows: zero sums, no rate, no flag
    for (size_t k = 0; k < n_win && finalize; ++k) {
        if (offsets[k + 1] != offsets[k]) continue;
        const uint32_t s = slots[k];
        GNM_CU(cudaMemsetAsync(c->d_stats + (size_t)s * c->keys * kNStat, 0, (size_t)c->keys * kNStat * 8, st));
        GNM_CU(cudaMemsetAsync(c->d_rate + (size_t)s * 2 * c->n_sites, 0xFF, (size_t)2 * c->n_sites * 8, st));
        GNM_CU(cudaMemsetAsync(c->d_flag + (size_t)s * 2 * c->n_sites, 0, (size_t)2 * c->n_sites, st));
    }
    return GNM_OK;
}

// Core of every processing call: windows k = [offsets[k], offsets[k+1]) of rec.
// finalize: rates and flags at the end; open_add: add to already open windows.
// GNM_HOST_PIPELINE: chunks of consecutive windows copied to two alternating device buffer
// sets on the context's copy stream, each processed on st once its copy has landed; a
// buffer set is refilled only after the processing that read it.
static gnm_status run_windows_pipelined(gnm_ctx* c, const gnm_records* rec, const uint64_t* offsets,
                                        const uint64_t* wids, size_t n_win, cudaStream_t st, bool finalize) {
    const uint64_t N = offsets[n_win] - offsets[0];
    const uint64_t target = std::max<uint64_t>(N / 8, (uint64_t)1 << 20);
    std::vector<size_t> cut{0};  // chunk k holds windows cut[k] .. cut[k+1]-1
    for (size_t w = 1; w <= n_win; ++w)
        if (w == n_win || offsets[w] - offsets[cut.back()] >= target) cut.push_back(w);
    {
        std::vector<uint64_t> ids(wids, wids + n_win);
        std::sort(ids.begin(), ids.end());
        if (std::adjacent_find(ids.begin(), ids.end()) != ids.end())
            return fail(GNM_E_INVAL, "duplicate window id in one call");
    }
    uint64_t most = 0;
    for (size_t k = 0; k + 1 < cut.size(); ++k) most = std::max(most, offsets[cut[k + 1]] - offsets[cut[k]]);
    PipeStaging& ps = c->pipe;
    if (!ps.copy) {
        GNM_CU(cudaStreamCreateWithFlags(&ps.copy, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            GNM_CU(cudaEventCreateWithFlags(&ps.copied[b], cudaEventDisableTiming));
            GNM_CU(cudaEventCreateWithFlags(&ps.freed[b], cudaEventDisableTiming));
        }
    }
    if (ps.cap < most) {  // grow both sets once the work that reads them is done
        GNM_CU(cudaStreamSynchronize(ps.copy));
        for (int b = 0; b < 2; ++b)
            if (ps.freed_recorded[b]) GNM_CU(cudaEventSynchronize(ps.freed[b]));
        for (auto& set : ps.d)
            for (auto& p : set) {
                free_dev(p);
                p = nullptr;
            }
        ps.cap = 0;
        for (auto& set : ps.d)
            for (auto& p : set) GNM_CU(cudaMalloc(&p, most * 4));
        ps.cap = most;
    }
    const uint32_t* src[6] = {rec->srcaddr, rec->dstaddr, rec->dPkts, rec->dOctets, rec->first, rec->last};
    std::vector<uint64_t> off;
    for (size_t k = 0; k + 1 < cut.size(); ++k) {
        const int b = (int)(k & 1);
        const uint64_t lo = offsets[cut[k]], n = offsets[cut[k + 1]] - lo;
        if (ps.freed_recorded[b]) GNM_CU(cudaStreamWaitEvent(ps.copy, ps.freed[b], 0));
        for (int f = 0; f < 6; ++f)
            if (n) GNM_CU(cudaMemcpyAsync(ps.d[b][f], src[f] + lo, n * 4, cudaMemcpyHostToDevice, ps.copy));
        GNM_CU(cudaEventRecord(ps.copied[b], ps.copy));
        GNM_CU(cudaStreamWaitEvent(st, ps.copied[b], 0));
        gnm_records dk = *rec;
        dk.n = n;
        dk.srcaddr = ps.d[b][0]; dk.dstaddr = ps.d[b][1]; dk.dPkts = ps.d[b][2];
        dk.dOctets = ps.d[b][3]; dk.first = ps.d[b][4]; dk.last = ps.d[b][5];
        dk.on_device = 1;
        off.assign(offsets + cut[k], offsets + cut[k + 1] + 1);
        for (auto& o : off) o -= lo;
        GNM_TRY(run_windows(c, &dk, off.data(), wids + cut[k], cut[k + 1] - cut[k], st, finalize, false));
        GNM_CU(cudaEventRecord(ps.freed[b], st));
        ps.freed_recorded[b] = true;
    }
    return GNM_OK;
}

gnm_status run_windows(gnm_ctx* c, const gnm_records* rec, const uint64_t* offsets,
                       const uint64_t* wids, size_t n_win, cudaStream_t st, bool finalize,
                       bool open_add) {
    if (n_win == 0) return GNM_OK;
    if (!wids) return fail(GNM_E_INVAL, "window ids are NULL");
    GNM_TRY(check_windows(c, rec, offsets, n_win));
    if (!rec->on_device && c->cfg.host_records == GNM_HOST_PIPELINE && !open_add && n_win > 1 &&
        offsets[n_win] > offsets[0])
        return run_windows_pipelined(c, rec, offsets, wids, n_win, st, finalize);
    const uint64_t base = offsets[0], N = offsets[n_win] - offsets[0];
    gnm_records dr = *rec;
    const uint32_t* inplace[6];
    if (N && !rec->on_device && host_addressable(c, rec, base, inplace)) {
        dr.srcaddr = inplace[0]; dr.dstaddr = inplace[1]; dr.dPkts = inplace[2];
        dr.dOctets = inplace[3]; dr.first = inplace[4]; dr.last = inplace[5];
        dr.on_device = 1;
    } else if (N && !rec->on_device) {
        if (c->cfg.host_records == GNM_HOST_IN_PLACE)
            return fail(GNM_E_INVAL, "host_records IN_PLACE: the record arrays are not device-addressable "
                                     "page-locked host memory");
        const uint32_t* d[6];
        GNM_TRY(stage_records(c, rec, base, offsets[n_win], st, d));
        dr.srcaddr = d[0]; dr.dstaddr = d[1]; dr.dPkts = d[2]; dr.dOctets = d[3]; dr.first = d[4]; dr.last = d[5];
    } else if (N) {
        dr.srcaddr += base; dr.dstaddr += base; dr.dPkts += base; dr.dOctets += base; dr.first += base; dr.last += base;
    }
    std::vector<uint32_t> slot(n_win);
    for (size_t k = 0; k < n_win; ++k) {
        if (open_add) {
            uint32_t s;
            GNM_TRY(find_window(c, wids[k], &s));
            Slot& sl = c->slots[s];
            if (!sl.open) return fail(GNM_E_STATE, "window is not open");
            if (sl.records + (offsets[k + 1] - offsets[k]) > kMaxWindowRecords)
                return fail(GNM_E_INVAL, "an open window would reach 2^32 records");
            GNM_TRY(wait_slot_on_stream(c, s, st));
            slot[k] = s;
        } else {
            for (size_t j = 0; j < k; ++j)
                if (wids[j] == wids[k]) return fail(GNM_E_INVAL, "duplicate window id in one call");
            GNM_TRY(acquire_slot(c, wids[k], st, &slot[k]));
        }
    }
    Prepared pr;
    GNM_TRY(prepare_launch(c, &dr, offsets, n_win, slot.data(), finalize, &pr));
    LaunchBuf* lb;
    GNM_TRY(acquire_ring(c, (uint32_t)std::max<size_t>(n_win, pr.n_buckets), &lb));
    const uint64_t key_words = pr.sh.split ? pr.n + 4 : 0;
    if (pr.part_bytes > lb->part_cap) {  // grow this entry's regrouping scratch
        free_dev(lb->d_part);
        lb->d_part = nullptr;
        lb->part_cap = 0;
        GNM_CU(cudaMalloc(&lb->d_part, pr.part_bytes));
        lb->part_cap = pr.part_bytes;
    }
    if (key_words > lb->keys_cap) {  // grow this entry's key array
        free_dev(lb->d_keys);
        lb->d_keys = nullptr;
        lb->keys_cap = 0;
        GNM_CU(cudaMalloc(&lb->d_keys, key_words * 4));
        lb->keys_cap = key_words;
    }
    if (pr.partial_words > lb->partial_cap) {  // grow this entry's partial-sum area
        free_dev(lb->d_partials);
        lb->d_partials = nullptr;
        lb->partial_cap = 0;
        GNM_CU(cudaMalloc(&lb->d_partials, pr.partial_words * 4));
        lb->partial_cap = pr.partial_words;
    }
    if (!pr.wins.empty()) {
        std::memcpy(lb->h_wins, pr.wins.data(), sizeof(WinDesc) * pr.wins.size());
        GNM_CU(cudaMemcpyAsync(lb->d_wins, lb->h_wins, sizeof(WinDesc) * pr.wins.size(), cudaMemcpyHostToDevice, st));
    }
    if (c->d_rlog_cnt) {  // sparse rate statistics: a log word per record of each window
        std::vector<uint64_t> need(n_win);
        for (size_t k = 0; k < n_win; ++k)
            need[k] = (open_add ? c->slots[slot[k]].records : 0) + (offsets[k + 1] - offsets[k]);
        GNM_TRY(reserve_rate_log(c, slot.data(), need.data(), n_win, st));
    }
    GNM_TRY(enqueue_prepared(c, pr, offsets, n_win, slot.data(), finalize, lb->d_wins, lb->d_done,
                             lb->d_partials, lb->d_keys, lb->d_part, st, &c->last_launches, nullptr, nullptr,
                             !open_add));
    GNM_CU(cudaEventRecord(lb->ev, st));
    lb->ev_recorded = true;
    for (size_t k = 0; k < n_win; ++k) c->slots[slot[k]].records += offsets[k + 1] - offsets[k];
    set_slots_done(c, slot.data(), n_win, lb->ev, finalize);
    return GNM_OK;
}

gnm_status reserve_launch_scratch(gnm_ctx* c, uint64_t n) {
    if (!n) return GNM_OK;
    LaunchShape sh;
    GNM_TRY(choose_shape(c, n, &sh, 1));
    const uint64_t key_words = sh.split ? n + 4 : 0;
    const uint64_t part_bytes = sh.part ? part_layout(n, sh.part_groups).bytes : 0;
    for (auto& b : c->ring) {
        if (b.ev_recorded) GNM_CU(cudaEventSynchronize(b.ev));
        if (key_words > b.keys_cap) {
            free_dev(b.d_keys);
            b.d_keys = nullptr;
            b.keys_cap = 0;
            GNM_CU(cudaMalloc(&b.d_keys, key_words * 4));
            b.keys_cap = key_words;
        }
        if (part_bytes > b.part_cap) {
            free_dev(b.d_part);
            b.d_part = nullptr;
            b.part_cap = 0;
            GNM_CU(cudaMalloc(&b.d_part, part_bytes));
            b.part_cap = part_bytes;
        }
    }
    return GNM_OK;
}

gnm_status open_window(gnm_ctx* c, uint64_t wid, cudaStream_t st, bool pin, uint32_t* s) {
    GNM_TRY(acquire_slot_impl(c, wid, st, pin, s));
    GNM_TRY(clear_rate_stats(c, s, 1, st));
    cudaEvent_t ev;
    GNM_TRY(record_event(c, st, &ev));
    set_slots_done(c, s, 1, ev, false);
    return GNM_OK;
}

gnm_status close_window(gnm_ctx* c, uint64_t wid, cudaStream_t st) {
    uint32_t s;
    GNM_TRY(find_window(c, wid, &s));
    Slot& sl = c->slots[s];
    if (!sl.open) return fail(GNM_E_STATE, "window is not open");
    GNM_TRY(wait_slot_on_stream(c, s, st));
    AggParams p;
    gnm_records none{};
    GNM_TRY(build_params(c, &none, &p));
    GNM_CU(launch_finalize(p, s, st));
    c->last_launches = 1;
    cudaEvent_t ev;
    GNM_TRY(record_event(c, st, &ev));
    set_slots_done(c, &s, 1, ev, true);
    return GNM_OK;
}

gnm_status device_checks(gnm_ctx* c) {
#if GNM_CHECKED
    unsigned long long v = 0;
    GNM_CU(cudaMemcpyAsync(&v, c->d_check, 8, cudaMemcpyDeviceToHost, c->aux));
    GNM_CU(cudaStreamSynchronize(c->aux));
    if (v)
        return fail(GNM_E_INTERNAL, std::string("device bounds check failed: ") + check_site_name((uint32_t)(v >> 56)) +
                                        " (value " + std::to_string(v & 0x00FFFFFFFFFFFFFFull) + ")");
#else
    (void)c;
#endif
    return GNM_OK;
}

}  // namespace gnm

using namespace gnm;

extern "C" {

void gnm_config_default(gnm_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->min_avg_pkt_bytes = 100;
    cfg->min_pkts = 10;
    cfg->min_dur_ms = 1000;
    cfg->min_flows_to_flag = 1;
    cfg->admin_rule = GNM_ADMIN_OR;
    cfg->lookup_mode = GNM_LOOKUP_AUTO;
    cfg->placement = GNM_PLACE_AUTO;
    cfg->aggregation = GNM_AGG_AUTO;
    cfg->device = 0;
    cfg->window_slots = 64;
    cfg->threshold_bps = 1e8;
}

gnm_status gnm_create(const gnm_config* cfg, gnm_ctx** out) {
    if (!out) return fail(GNM_E_INVAL, "out is NULL");
    *out = nullptr;
    gnm_ctx* c = new (std::nothrow) gnm_ctx();
    if (!c) return fail(GNM_E_NOMEM, "host allocation failed");
    if (cfg) c->cfg = *cfg;
    else gnm_config_default(&c->cfg);
    if (c->cfg.admin_rule != GNM_ADMIN_OR && c->cfg.admin_rule != GNM_ADMIN_AND) {
        delete c;
        return fail(GNM_E_INVAL, "admin_rule must be GNM_ADMIN_OR or GNM_ADMIN_AND");
    }
    if (c->cfg.window_slots == 0) c->cfg.window_slots = 64;
    if (c->cfg.host_records < GNM_HOST_AUTO || c->cfg.host_records > GNM_HOST_PIPELINE) {
        delete c;
        return fail(GNM_E_INVAL, "host_records must be GNM_HOST_AUTO, _STAGE, _IN_PLACE or _PIPELINE");
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        delete c;
        return fail(GNM_E_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    if (c->cfg.device < 0 || c->cfg.device >= ndev) {
        delete c;
        return fail(GNM_E_INVAL, "device ordinal out of range");
    }
    c->device = c->cfg.device;
    if ((e = cudaSetDevice(c->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&c->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device)) != cudaSuccess) {
        delete c;
        return fail(GNM_E_CUDA, std::string("device query: ") + cudaGetErrorString(e));
    }
    c->ring.resize(kRingSize);
    for (auto& b : c->ring) {
        if (cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming) != cudaSuccess) {
            gnm_destroy(c);
            return fail(GNM_E_CUDA, "event creation failed");
        }
    }
    if (cudaEventCreateWithFlags(&c->staging.ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&c->d_violations, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->d_check, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->d_flag_count, sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(c->d_violations, 0, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(c->d_check, 0, sizeof(unsigned long long)) != cudaSuccess) {
        gnm_destroy(c);
        return fail(GNM_E_CUDA, "context allocation failed");
    }
    *out = c;
    return GNM_OK;
}

void gnm_destroy(gnm_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    release_slots(c);
    for (auto& b : c->ring) {
        if (b.h_wins) cudaFreeHost(b.h_wins);
        free_dev(b.d_wins);
        free_dev(b.d_done);
        free_dev(b.d_partials);
        free_dev(b.d_keys);
        free_dev(b.d_part);
        if (b.ev) cudaEventDestroy(b.ev);
    }
    for (auto* p : c->staging.d) free_dev(p);
    if (c->staging.ev) cudaEventDestroy(c->staging.ev);
    for (auto& set : c->pipe.d)
        for (auto* p : set) free_dev(p);
    for (int b = 0; b < 2; ++b) {
        if (c->pipe.copied[b]) cudaEventDestroy(c->pipe.copied[b]);
        if (c->pipe.freed[b]) cudaEventDestroy(c->pipe.freed[b]);
    }
    if (c->pipe.copy) cudaStreamDestroy(c->pipe.copy);
    if (c->aux) cudaStreamDestroy(c->aux);
    free_dev(c->d_starts);
    free_dev(c->d_site);
    free_dev(c->d_pairs);
    free_dev(c->d_blocks);
    free_dev(c->d_sample);
    free_dev(c->d_dir16);
    free_dev(c->d_sample4);
    free_dev(c->d_sample2);
    free_dev(c->d_dirh);
    free_dev(c->d_smp16);
    free_dev(c->d_h24);
    free_dev(c->d_violations);
    free_dev(c->d_check);
    free_dev(c->d_flag_count);
    free_dev(c->d_rmi_a);
    free_dev(c->d_rmi_b);
    free_dev(c->d_rmi_x0);
    free_dev(c->d_rmi_eps);
    free_dev(c->d_rmi_elo);
    free_dev(c->d_rmi_ehi);
    free_dev(c->d_rmi_leaf4);
    delete c;
}

const char* gnm_last_error(const gnm_ctx*) { return get_error(); }

gnm_status gnm_registry_load(gnm_ctx* c, const uint32_t* prefix, const uint8_t* len,
                             const uint32_t* site_id, size_t n, uint32_t n_sites,
                             const uint32_t* local_prefix, const uint8_t* local_len, size_t n_local) {
    if (!c) return fail(GNM_E_INVAL, "ctx is NULL");
    if (n && (!prefix || !len || !site_id)) return fail(GNM_E_INVAL, "registry arrays are NULL");
    if (n_sites == 0 || n_sites > (1u << 26)) return fail(GNM_E_INVAL, "n_sites must be 1..2^26");
    if (n_local == 0 || n_local > GNM_MAX_LOCAL || !local_prefix || !local_len)
        return fail(GNM_E_INVAL, "need 1..8 local prefixes");
    for (size_t i = 0; i < n_local; ++i) {
        if (local_len[i] > 32) return fail(GNM_E_INVAL, "local prefix length > 32");
        const uint32_t m = local_len[i] == 0 ? 0u : (0xFFFFFFFFu << (32 - local_len[i]));
        if (local_prefix[i] & ~m) return fail(GNM_E_INVAL, "local prefix has host bits set");
        if (local_overlaps(local_prefix[i], local_len[i], prefix, len, n))
            return fail(GNM_E_INVAL, "a local prefix overlaps a registered prefix");
    }
    std::vector<uint32_t> starts, sites;
    const std::string why = flatten_registry(prefix, len, site_id, n, n_sites, &starts, &sites);
    if (!why.empty()) return fail(GNM_E_INVAL, why);
    GNM_CU(cudaSetDevice(c->device));
    GNM_CU(cudaDeviceSynchronize());
    // drop everything that depended on the old registry
    release_slots(c);
    free_dev(c->d_starts);
    free_dev(c->d_site);
    free_dev(c->d_pairs);
    free_dev(c->d_blocks);
    free_dev(c->d_sample);
    free_dev(c->d_dir16);
    free_dev(c->d_sample4);
    free_dev(c->d_sample2);
    free_dev(c->d_dirh);
    free_dev(c->d_smp16);
    free_dev(c->d_h24);
    c->d_dir16 = nullptr;
    c->d_sample4 = nullptr;
    c->n_blk4 = 0;
    c->d_sample2 = nullptr;
    c->n_blk2 = 0;
    c->d_dirh = nullptr;
    c->d_smp16 = nullptr;
    c->d_h24 = nullptr;
    c->h24_mask = 0;
    c->d_starts = nullptr;
    c->d_site = nullptr;
    c->d_pairs = nullptr;
    c->d_blocks = nullptr;
    c->d_sample = nullptr;
    c->n_blocks = 0;
    c->have_registry = false;
    c->rmi_ready = false;
    c->tuned = Tuned();
    const size_t nr = starts.size();
    GNM_CU(cudaMalloc(&c->d_starts, nr * 4));
    GNM_CU(cudaMalloc(&c->d_site, nr * 4));
    GNM_CU(cudaMemcpy(c->d_starts, starts.data(), nr * 4, cudaMemcpyHostToDevice));
    GNM_CU(cudaMemcpy(c->d_site, sites.data(), nr * 4, cudaMemcpyHostToDevice));
    {  // (start, site) pairs: a search probe brings the site of the range it lands on
        std::vector<uint2> pr(nr + 16);
        for (size_t i = 0; i < nr + 16; ++i)
            pr[i] = i < nr ? make_uint2(starts[i], sites[i]) : make_uint2(0xFFFFFFFFu, sites[nr - 1]);
        GNM_CU(cudaMalloc(&c->d_pairs, pr.size() * sizeof(uint2)));
        GNM_CU(cudaMemcpy(c->d_pairs, pr.data(), pr.size() * sizeof(uint2), cudaMemcpyHostToDevice));
    }
    // staged layout: blocks of 16 range starts (the last block padded with 0xFFFFFFFF)
    // and the first start of every block
    const size_t nb = (nr + kBlockRanges - 1) / kBlockRanges;
    std::vector<uint32_t> blk(nb * kBlockRanges), smp(nb);
    for (size_t j = 0; j < nb; ++j) {
        for (size_t k = 0; k < kBlockRanges; ++k) {
            const size_t i = j * kBlockRanges + k;
            blk[j * kBlockRanges + k] = i < nr ? starts[i] : 0xFFFFFFFFu;
        }
        smp[j] = starts[j * kBlockRanges];
    }
    // radix directory: for each /16 t (and t = 65536 for the end), the range holding its
    // first address
    std::vector<uint32_t> dir(65537);
    {
        size_t i = 0;
        for (uint64_t t = 0; t <= 65536; ++t) {
            const uint64_t a = t << 16;
            while (i + 1 < nr && (uint64_t)starts[i + 1] <= a) ++i;
            dir[t] = (uint32_t)i;
        }
        dir[65536] = (uint32_t)(nr - 1);
    }
    GNM_CU(cudaMalloc(&c->d_dir16, dir.size() * 4));
    GNM_CU(cudaMemcpy(c->d_dir16, dir.data(), dir.size() * 4, cudaMemcpyHostToDevice));
    {  // the paper's /24 subnet hash table, for registries of prefixes up to /24
        std::vector<uint32_t> t;
        uint32_t mask = 0;
        if (build_hash24(prefix, len, site_id, n, &t, &mask)) {
            GNM_CU(cudaMalloc(&c->d_h24, t.size() * 4));
            GNM_CU(cudaMemcpy(c->d_h24, t.data(), t.size() * 4, cudaMemcpyHostToDevice));
            c->h24_mask = mask;
        }
    }
    for (size_t br : {(size_t)2, (size_t)4}) {  // key kernel: first start of every 2- and 4-range block
        const size_t nb = (nr + br - 1) / br;
        std::vector<uint32_t> sb(nb);
        for (size_t g = 0; g < nb; ++g) sb[g] = starts[br * g];
        uint32_t** d = br == 2 ? &c->d_sample2 : &c->d_sample4;
        GNM_CU(cudaMalloc(d, nb * 4));
        GNM_CU(cudaMemcpy(*d, sb.data(), nb * 4, cudaMemcpyHostToDevice));
        (br == 2 ? c->n_blk2 : c->n_blk4) = (uint32_t)nb;
        if (br == 2 && nb < 65536) {
            // 16-bit form: per /16 bucket t the first block starting at or after t << 16 (the
            // block before it holds the bucket's first address; the blocks up to the next
            // bucket's entry start inside the bucket, so their low 16 bits order them)
            std::vector<uint16_t> dh(65537), s16(nb);
            size_t g = 0;
            for (uint64_t t = 0; t < 65536; ++t) {
                while (g < nb && (uint64_t)sb[g] < (t << 16)) ++g;
                dh[t] = (uint16_t)g;
            }
            dh[65536] = (uint16_t)nb;
            for (size_t b = 0; b < nb; ++b) s16[b] = (uint16_t)(sb[b] & 0xFFFFu);
            GNM_CU(cudaMalloc(&c->d_dirh, dh.size() * 2));
            GNM_CU(cudaMemcpy(c->d_dirh, dh.data(), dh.size() * 2, cudaMemcpyHostToDevice));
            GNM_CU(cudaMalloc(&c->d_smp16, nb * 2));
            GNM_CU(cudaMemcpy(c->d_smp16, s16.data(), nb * 2, cudaMemcpyHostToDevice));
        }
    }
    GNM_CU(cudaMalloc(&c->d_blocks, blk.size() * 4));
    GNM_CU(cudaMalloc(&c->d_sample, nb * 4));
    GNM_CU(cudaMemcpy(c->d_blocks, blk.data(), blk.size() * 4, cudaMemcpyHostToDevice));
    GNM_CU(cudaMemcpy(c->d_sample, smp.data(), nb * 4, cudaMemcpyHostToDevice));
    c->n_blocks = (uint32_t)nb;
    c->h_starts.swap(starts);
    c->h_site.swap(sites);
    c->n_sites = n_sites;
    c->n_prefixes = (uint32_t)n;
    c->keys = 2 * n_sites + kUnmatched;
    c->n_local = (uint32_t)n_local;
    for (uint32_t i = 0; i < GNM_MAX_LOCAL; ++i) {
        c->local_pfx[i] = i < n_local ? local_prefix[i] : 0u;
        c->local_mask[i] = i < n_local ? (local_len[i] == 0 ? 0u : (0xFFFFFFFFu << (32 - local_len[i]))) : 0u;
    }
    // result slots; accumulators start (and stay, between windows) at zero
    c->n_slots = c->cfg.window_slots;
    const size_t keys = c->keys, slots = c->n_slots;
    GNM_CU(cudaMalloc(&c->d_acc, slots * keys * kAccCols * 8));
    GNM_CU(cudaMalloc(&c->d_stats, slots * keys * kNStat * 8));
    GNM_CU(cudaMalloc(&c->d_rate, slots * 2 * n_sites * 8));
    GNM_CU(cudaMalloc(&c->d_flag, slots * 2 * n_sites));
    GNM_CU(cudaMalloc(&c->d_flag_keys, (size_t)2 * n_sites * 4));
    GNM_CU(cudaMemset(c->d_acc, 0, slots * keys * kAccCols * 8));
    GNM_CU(cudaMalloc(&c->d_dirty, slots * ((keys + 31) / 32)));
    GNM_CU(cudaMemset(c->d_dirty, 0, slots * ((keys + 31) / 32)));
    if (c->cfg.rate_stats < 0 || c->cfg.rate_stats > 2) return fail(GNM_E_INVAL, "rate_stats must be 0, 1 or 2");
    if (c->cfg.rate_stats == 2 && (size_t)2 * n_sites > (1u << 18))
        return fail(GNM_E_INVAL, "rate_stats = 2 needs at most 131,072 sites (keys of 18 bits)");
    if (c->cfg.rate_stats) {  // per-flow rate statistics: per site key and slot
        const size_t nk = (size_t)2 * n_sites;
        if (c->cfg.rate_stats == 1) {  // a histogram of 10001 buckets
            GNM_CU(cudaMalloc(&c->d_hist, slots * nk * kRateBuckets * 4));
        } else {  // a log word per eligible flow, grown per slot as records arrive
            c->rlog.assign(slots, nullptr);
            c->rlog_cap.assign(slots, 0);
            c->rlog_sorted.assign(slots, 0);
            GNM_CU(cudaMallocHost(&c->h_rlog_ptr, slots * sizeof(uint32_t*)));
            GNM_CU(cudaMallocHost(&c->h_rlog_cap, slots * 4));
            GNM_CU(cudaMalloc(&c->d_rlog_ptr, slots * sizeof(uint32_t*)));
            GNM_CU(cudaMalloc(&c->d_rlog_cap, slots * 4));
            GNM_CU(cudaMalloc(&c->d_rlog_cnt, slots * 4));
            GNM_CU(cudaMemset(c->d_rlog_ptr, 0, slots * sizeof(uint32_t*)));
            GNM_CU(cudaMemset(c->d_rlog_cap, 0, slots * 4));
            GNM_CU(cudaMemset(c->d_rlog_cnt, 0, slots * 4));
        }
        GNM_CU(cudaMalloc(&c->d_rmin, slots * nk * 8));
        GNM_CU(cudaMalloc(&c->d_rmax, slots * nk * 8));
        GNM_CU(cudaMalloc(&c->d_med, nk * 4));
        GNM_CU(cudaMalloc(&c->d_mcnt, nk * 4));
        GNM_CU(cudaMalloc(&c->d_warn_run, nk * 4));
        GNM_CU(cudaMemset(c->d_warn_run, 0, nk * 4));
    }
    if (c->cfg.host_capacity) {  // per-host sums: a table at most half full per slot
        uint64_t hc = 1024;
        while (hc < 2ull * c->cfg.host_capacity) hc <<= 1;
        if (hc > (1ull << 31)) return fail(GNM_E_INVAL, "host_capacity too large");
        c->hcap = (uint32_t)hc;
        GNM_CU(cudaMalloc(&c->d_hkeys, slots * hc * 8));
        GNM_CU(cudaMalloc(&c->d_hrows, slots * hc * kNStat * 8));
        GNM_CU(cudaMalloc(&c->d_hover, slots * 4));
        GNM_CU(cudaMalloc(&c->d_hrate, hc * 8));
    }
    c->slots.resize(slots);
    c->have_registry = true;
    return GNM_OK;
}

gnm_status gnm_registry_info_get(gnm_ctx* c, gnm_registry_info* out) {
    if (!c || !out) return fail(GNM_E_INVAL, "NULL argument");
    if (!c->have_registry) return fail(GNM_E_STATE, "no registry loaded");
    std::memset(out, 0, sizeof(*out));
    out->n_ranges = c->h_starts.size();
    for (uint32_t s : c->h_site) out->n_registered += s != GNM_NO_SITE;
    out->n_sites = c->n_sites;
    out->n_prefixes = c->n_prefixes;
    LaunchShape sh;
    if (choose_shape(c, 1u << 20, &sh) == GNM_OK) {
        out->placement = sh.lookup == kLookupSmem ? GNM_PLACE_SMEM
                         : sh.lookup == kLookupStaged ? GNM_PLACE_STAGED : GNM_PLACE_L2;
        out->lookup_mode = sh.lookup == kLookupRmi      ? GNM_LOOKUP_RMI
                           : sh.lookup == kLookupRadix  ? GNM_LOOKUP_RADIX
                           : sh.lookup == kLookupHash24 ? GNM_LOOKUP_HASH24
                                                        : GNM_LOOKUP_BSEARCH;
        out->privatized = sh.table != kTableGlobal;
    }
    out->rmi_ready = c->rmi_ready;
    return GNM_OK;
}

gnm_status gnm_registry_ranges(gnm_ctx* c, uint32_t* starts, uint32_t* site, size_t cap, size_t* n_out) {
    if (!c || !n_out) return fail(GNM_E_INVAL, "NULL argument");
    if (!c->have_registry) return fail(GNM_E_STATE, "no registry loaded");
    *n_out = c->h_starts.size();
    if (cap < c->h_starts.size()) return fail(GNM_E_CAPACITY, "cap smaller than the number of ranges");
    if (starts) std::memcpy(starts, c->h_starts.data(), c->h_starts.size() * 4);
    if (site) std::memcpy(site, c->h_site.data(), c->h_site.size() * 4);
    return GNM_OK;
}

gnm_status gnm_window_process(gnm_ctx* c, const gnm_records* rec, uint64_t wid, void* stream) {
    if (!c || !rec) return fail(GNM_E_INVAL, "NULL argument");
    GNM_CU(cudaSetDevice(c->device));
    const uint64_t off[2] = {0, rec->n};
    return run_windows(c, rec, off, &wid, 1, (cudaStream_t)stream, true, false);
}

gnm_status gnm_windows_process(gnm_ctx* c, const gnm_records* rec, const uint64_t* offsets,
                               const uint64_t* wids, size_t n_win, void* stream) {
    if (!c) return fail(GNM_E_INVAL, "ctx is NULL");
    GNM_CU(cudaSetDevice(c->device));
    return run_windows(c, rec, offsets, wids, n_win, (cudaStream_t)stream, true, false);
}

gnm_status gnm_window_open(gnm_ctx* c, uint64_t wid, void* stream) {
    if (!c) return fail(GNM_E_INVAL, "ctx is NULL");
    if (!c->have_registry) return fail(GNM_E_STATE, "no registry loaded");
    GNM_CU(cudaSetDevice(c->device));
    uint32_t s;
    return open_window(c, wid, (cudaStream_t)stream, false, &s);
}

gnm_status gnm_window_add(gnm_ctx* c, const gnm_records* rec, uint64_t wid, void* stream) {
    if (!c || !rec) return fail(GNM_E_INVAL, "NULL argument");
    GNM_CU(cudaSetDevice(c->device));
    const uint64_t off[2] = {0, rec->n};
    return run_windows(c, rec, off, &wid, 1, (cudaStream_t)stream, false, true);
}

gnm_status gnm_window_close(gnm_ctx* c, uint64_t wid, void* stream) {
    if (!c) return fail(GNM_E_INVAL, "ctx is NULL");
    GNM_CU(cudaSetDevice(c->device));
    return close_window(c, wid, (cudaStream_t)stream);
}

static gnm_status sync_slot(gnm_ctx* c, uint32_t s) {
    Slot& sl = c->slots[s];
    if (!sl.finalized) return fail(GNM_E_STATE, "window is open (not finalised)");
    if (sl.ev) GNM_CU(cudaEventSynchronize(sl.ev));
    return GNM_OK;
}

namespace {

// Sparse rate statistics: sorts slot s's log once (in place) and returns its word count.
gnm_status sorted_rate_log(gnm_ctx* c, uint32_t s, cudaStream_t st, uint32_t* n_out) {
    uint32_t n = 0;
    GNM_CU(cudaMemcpyAsync(&n, c->d_rlog_cnt + s, 4, cudaMemcpyDeviceToHost, st));
    GNM_CU(cudaStreamSynchronize(st));
    if (n > c->rlog_cap[s]) return fail(GNM_E_INTERNAL, "rate-statistics log overflow");
    *n_out = n;
    if (c->rlog_sorted[s] || n <= 1) {
        c->rlog_sorted[s] = 1;
        return GNM_OK;
    }
    const uint64_t hw = radix_sort_hist_words(n, c->sm_count);
    if (n > c->rlog_tmp_cap) {
        free_dev(c->d_rlog_tmp);
        c->d_rlog_tmp = nullptr;
        c->rlog_tmp_cap = 0;
        GNM_CU(cudaMalloc(&c->d_rlog_tmp, (size_t)n * 4));
        c->rlog_tmp_cap = n;
    }
    if (hw > c->rs_hist_cap) {
        free_dev(c->d_rs_hist);
        c->d_rs_hist = nullptr;
        c->rs_hist_cap = 0;
        GNM_CU(cudaMalloc(&c->d_rs_hist, hw * 4));
        c->rs_hist_cap = hw;
    }
    // significant bits of the largest word, ((2S - 1) << 14) | 10000
    const uint32_t top = ((2u * c->n_sites - 1u) << 14) | 10000u;
    int bits = 0;
    while (bits < 32 && (top >> bits)) ++bits;
    uint32_t* res = nullptr;
    GNM_CU(radix_sort_u32(c->rlog[s], c->d_rlog_tmp, n, bits, c->d_rs_hist, c->sm_count, st, &res));
    if (res != c->rlog[s]) GNM_CU(cudaMemcpyAsync(c->rlog[s], res, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    c->rlog_sorted[s] = 1;
    return GNM_OK;
}

// Lower-median bucket and eligible flows of every site key of slot s into d_med / d_mcnt.
gnm_status rate_medians(gnm_ctx* c, uint32_t s, cudaStream_t st) {
    const uint32_t nk = 2u * c->n_sites;
    if (c->d_hist) {
        GNM_CU(launch_rate_median(c->d_hist + (size_t)s * nk * kRateBuckets, nk, c->d_med, c->d_mcnt, st));
        return GNM_OK;
    }
    uint32_t n = 0;
    GNM_TRY(sorted_rate_log(c, s, st, &n));
    GNM_CU(launch_sparse_median(c->rlog[s], n, nk, c->d_med, c->d_mcnt, st));
    return GNM_OK;
}

}  // namespace

gnm_status gnm_window_rate_cells(gnm_ctx* c, uint64_t wid, uint32_t* key, uint32_t* bucket, uint32_t* count,
                                 size_t cap, size_t* n_out) {
    if (!c || !n_out) return fail(GNM_E_INVAL, "NULL argument");
    if (!c->d_hist && !c->d_rlog_cnt) return fail(GNM_E_STATE, "the context keeps no rate statistics (rate_stats = 0)");
    GNM_CU(cudaSetDevice(c->device));
    uint32_t s;
    GNM_TRY(find_window(c, wid, &s));
    if (!c->slots[s].finalized) return fail(GNM_E_STATE, "window is open (not finalised)");
    GNM_TRY(wait_slot_on_stream(c, s, c->aux));
    const size_t nk = (size_t)2 * c->n_sites;
    std::vector<uint32_t> ck, cb, cc;
    if (c->d_hist) {  // non-zero cells of the dense histograms
        std::vector<uint32_t> h(nk * kRateBuckets);
        GNM_CU(cudaMemcpyAsync(h.data(), c->d_hist + (size_t)s * nk * kRateBuckets, h.size() * 4,
                               cudaMemcpyDeviceToHost, c->aux));
        GNM_CU(cudaStreamSynchronize(c->aux));
        for (size_t k = 0; k < nk; ++k)
            for (uint32_t b = 0; b < kRateBuckets; ++b)
                if (h[k * kRateBuckets + b]) {
                    ck.push_back((uint32_t)k);
                    cb.push_back(b);
                    cc.push_back(h[k * kRateBuckets + b]);
                }
    } else {  // runs of the sorted log
        uint32_t n = 0;
        GNM_TRY(sorted_rate_log(c, s, c->aux, &n));
        std::vector<uint32_t> w(n);
        if (n) GNM_CU(cudaMemcpyAsync(w.data(), c->rlog[s], (size_t)n * 4, cudaMemcpyDeviceToHost, c->aux));
        GNM_CU(cudaStreamSynchronize(c->aux));
        for (uint32_t i = 0; i < n;) {
            uint32_t j = i + 1;
            while (j < n && w[j] == w[i]) ++j;
            ck.push_back(w[i] >> 14);
            cb.push_back(w[i] & 0x3FFFu);
            cc.push_back(j - i);
            i = j;
        }
    }
    *n_out = ck.size();
    if (cap < ck.size()) return fail(GNM_E_CAPACITY, "cap smaller than the number of non-empty cells");
    if (key && !ck.empty()) std::memcpy(key, ck.data(), ck.size() * 4);
    if (bucket && !cb.empty()) std::memcpy(bucket, cb.data(), cb.size() * 4);
    if (count && !cc.empty()) std::memcpy(count, cc.data(), cc.size() * 4);
    return GNM_OK;
}

gnm_status gnm_window_rate_stats(gnm_ctx* c, uint64_t wid, double* rmin, double* rmax, uint32_t* median_bucket,
                                 uint32_t* hist) {
    if (!c) return fail(GNM_E_INVAL, "ctx is NULL");
    if (!c->d_hist && !c->d_rlog_cnt) return fail(GNM_E_STATE, "the context keeps no rate statistics (rate_stats = 0)");
    if (hist && !c->d_hist)
        return fail(GNM_E_INVAL, "rate_stats = 2 keeps no dense histograms (gnm_window_rate_cells lists the cells)");
    GNM_CU(cudaSetDevice(c->device));
    uint32_t s;
    GNM_TRY(find_window(c, wid, &s));
    if (!c->slots[s].finalized) return fail(GNM_E_STATE, "window is open (not finalised)");
    GNM_TRY(wait_slot_on_stream(c, s, c->aux));
    const size_t nk = (size_t)2 * c->n_sites;
    const uint32_t* h = c->d_hist ? c->d_hist + (size_t)s * nk * kRateBuckets : nullptr;
    GNM_TRY(rate_medians(c, s, c->aux));
    std::vector<uint32_t> cnt(nk);
    std::vector<unsigned long long> lo(rmin ? nk : 0), hi(rmax ? nk : 0);
    GNM_CU(cudaMemcpyAsync(cnt.data(), c->d_mcnt, nk * 4, cudaMemcpyDeviceToHost, c->aux));
    if (median_bucket) GNM_CU(cudaMemcpyAsync(median_bucket, c->d_med, nk * 4, cudaMemcpyDeviceToHost, c->aux));
    if (rmin) GNM_CU(cudaMemcpyAsync(lo.data(), c->d_rmin + (size_t)s * nk, nk * 8, cudaMemcpyDeviceToHost, c->aux));
    if (rmax) GNM_CU(cudaMemcpyAsync(hi.data(), c->d_rmax + (size_t)s * nk, nk * 8, cudaMemcpyDeviceToHost, c->aux));
    if (hist) GNM_CU(cudaMemcpyAsync(hist, h, nk * kRateBuckets * 4, cudaMemcpyDeviceToHost, c->aux));
    GNM_CU(cudaStreamSynchronize(c->aux));
    const double nan = std::numeric_limits<double>::quiet_NaN();
    for (size_t k = 0; k < nk; ++k) {
        double v;
        if (rmin) {
            std::memcpy(&v, &lo[k], 8);
            rmin[k] = cnt[k] ? v : nan;
        }
        if (rmax) {
            std::memcpy(&v, &hi[k], 8);
            rmax[k] = cnt[k] ? v : nan;
        }
    }
    return GNM_OK;
}

gnm_status gnm_window_hosts(gnm_ctx* c, uint64_t wid, gnm_host_stat* out, size_t cap, size_t* n_out) {
    if (!c || !n_out) return fail(GNM_E_INVAL, "NULL argument");
    if (!c->d_hkeys) return fail(GNM_E_STATE, "the context keeps no per-host sums (host_capacity = 0)");
    GNM_CU(cudaSetDevice(c->device));
    uint32_t s;
    GNM_TRY(find_window(c, wid, &s));
    if (!c->slots[s].finalized) return fail(GNM_E_STATE, "window is open (not finalised)");
    GNM_TRY(sync_slot(c, s));
    const size_t hc = c->hcap;
    std::vector<unsigned long long> keys(hc), rows(hc * kNStat);
    std::vector<double> rate(hc);
    uint32_t lost = 0;
    const unsigned long long* d_rows = c->d_hrows + (size_t)s * hc * kNStat;
    GNM_CU(launch_host_rates(d_rows, (uint32_t)hc, c->d_hrate, c->aux));
    GNM_CU(cudaStreamSynchronize(c->aux));
    GNM_CU(cudaMemcpy(keys.data(), c->d_hkeys + (size_t)s * hc, hc * 8, cudaMemcpyDeviceToHost));
    GNM_CU(cudaMemcpy(rows.data(), d_rows, hc * kNStat * 8, cudaMemcpyDeviceToHost));
    GNM_CU(cudaMemcpy(rate.data(), c->d_hrate, hc * 8, cudaMemcpyDeviceToHost));
    GNM_CU(cudaMemcpy(&lost, c->d_hover + s, 4, cudaMemcpyDeviceToHost));
    std::vector<gnm_host_stat> v;
    for (size_t h = 0; h < hc; ++h) {
        if (!keys[h]) continue;
        const unsigned long long k = keys[h] - 1ull;
        gnm_host_stat r;
        r.addr = (uint32_t)(k >> 1);
        r.dir = (uint32_t)(k & 1ull);
        // the host's site: the flattened range holding its address
        const size_t i = (size_t)(std::upper_bound(c->h_starts.begin(), c->h_starts.end(), r.addr) -
                                  c->h_starts.begin()) - 1;
        r.site = c->h_site[i];
        r.reserved = 0;
        const unsigned long long* q = &rows[h * kNStat];
        r.flows = q[0];
        r.octets = q[1];
        r.pkts = q[2];
        r.e_flows = q[3];
        r.e_octets = q[4];
        r.e_dur_ms = q[5];
        r.rate_bps = rate[h];
        v.push_back(r);
    }
    std::sort(v.begin(), v.end(), [](const gnm_host_stat& a, const gnm_host_stat& b) {
        return a.site != b.site ? a.site < b.site : a.dir != b.dir ? a.dir < b.dir : a.addr < b.addr;
    });
    *n_out = v.size();
    if (cap < v.size()) return fail(GNM_E_CAPACITY, "cap smaller than the number of host rows");
    if (out && !v.empty()) std::memcpy(out, v.data(), v.size() * sizeof(gnm_host_stat));
    if (lost) return fail(GNM_E_CAPACITY, std::to_string(lost) + " records met a full host table (host_capacity)");
    return GNM_OK;
}

gnm_status gnm_warnings_update(gnm_ctx* c, uint64_t wid, uint32_t below_bucket, uint32_t consecutive,
                               uint32_t* keys_out, size_t cap, size_t* n_out) {
    if (!c || !n_out) return fail(GNM_E_INVAL, "NULL argument");
    if (!c->d_warn_run) return fail(GNM_E_STATE, "the context keeps no rate statistics (rate_stats = 0)");
    if (consecutive == 0) return fail(GNM_E_INVAL, "consecutive must be at least 1");
    GNM_CU(cudaSetDevice(c->device));
    uint32_t s;
    GNM_TRY(find_window(c, wid, &s));
    if (!c->slots[s].finalized) return fail(GNM_E_STATE, "window is open (not finalised)");
    GNM_TRY(wait_slot_on_stream(c, s, c->aux));
    const uint32_t nk = 2u * c->n_sites;
    GNM_TRY(rate_medians(c, s, c->aux));
    GNM_CU(launch_warn_runs(c->d_med, nk, below_bucket, consecutive, c->d_warn_run, c->d_flag_keys, c->d_flag_count,
                            c->aux));
    uint32_t cnt = 0;
    GNM_CU(cudaMemcpyAsync(&cnt, c->d_flag_count, 4, cudaMemcpyDeviceToHost, c->aux));
    GNM_CU(cudaStreamSynchronize(c->aux));
    std::vector<uint32_t> keys(cnt);
    if (cnt) GNM_CU(cudaMemcpyAsync(keys.data(), c->d_flag_keys, cnt * 4, cudaMemcpyDeviceToHost, c->aux));
    GNM_CU(cudaStreamSynchronize(c->aux));
    *n_out = cnt;
    if (cap < cnt) return fail(GNM_E_CAPACITY, "cap smaller than the number of warned keys");
    std::sort(keys.begin(), keys.end());
    if (keys_out && cnt) std::memcpy(keys_out, keys.data(), cnt * 4);
    return GNM_OK;
}

gnm_status gnm_warnings_reset(gnm_ctx* c) {
    if (!c) return fail(GNM_E_INVAL, "ctx is NULL");
    if (!c->d_warn_run) return fail(GNM_E_STATE, "the context keeps no rate statistics (rate_stats = 0)");
    GNM_CU(cudaSetDevice(c->device));
    GNM_CU(cudaMemsetAsync(c->d_warn_run, 0, (size_t)2 * c->n_sites * 4, c->aux));
    GNM_CU(cudaStreamSynchronize(c->aux));
    return GNM_OK;
}

gnm_status gnm_warnings_export(gnm_ctx* c, uint32_t* runs) {
    if (!c || !runs) return fail(GNM_E_INVAL, "NULL argument");
    if (!c->d_warn_run) return fail(GNM_E_STATE, "the context keeps no rate statistics (rate_stats = 0)");
    GNM_CU(cudaSetDevice(c->device));
    GNM_CU(cudaMemcpyAsync(runs, c->d_warn_run, (size_t)2 * c->n_sites * 4, cudaMemcpyDeviceToHost, c->aux));
    GNM_CU(cudaStreamSynchronize(c->aux));
    return GNM_OK;
}

gnm_status gnm_warnings_import(gnm_ctx* c, const uint32_t* runs) {
    if (!c || !runs) return fail(GNM_E_INVAL, "NULL argument");
    if (!c->d_warn_run) return fail(GNM_E_STATE, "the context keeps no rate statistics (rate_stats = 0)");
    GNM_CU(cudaSetDevice(c->device));
    GNM_CU(cudaMemcpyAsync(c->d_warn_run, runs, (size_t)2 * c->n_sites * 4, cudaMemcpyHostToDevice, c->aux));
    GNM_CU(cudaStreamSynchronize(c->aux));
    return GNM_OK;
}

gnm_status gnm_window_dense(gnm_ctx* c, uint64_t wid, uint64_t* stats, uint64_t* unmatched,
                            double* rate, uint8_t* flag) {
    if (!c) return fail(GNM_E_INVAL, "ctx is NULL");
    GNM_CU(cudaSetDevice(c->device));
    uint32_t s;
    GNM_TRY(find_window(c, wid, &s));
    GNM_TRY(sync_slot(c, s));
    const size_t nk = 2 * (size_t)c->n_sites;
    const uint64_t* st = c->d_stats + (size_t)s * c->keys * kNStat;
    if (stats) GNM_CU(cudaMemcpyAsync(stats, st, nk * kNStat * 8, cudaMemcpyDeviceToHost, c->aux));
    uint64_t un6[kUnmatched * kNStat];
    if (unmatched) GNM_CU(cudaMemcpyAsync(un6, st + nk * kNStat, sizeof(un6), cudaMemcpyDeviceToHost, c->aux));
    if (rate) GNM_CU(cudaMemcpyAsync(rate, c->d_rate + (size_t)s * nk, nk * 8, cudaMemcpyDeviceToHost, c->aux));
    if (flag) GNM_CU(cudaMemcpyAsync(flag, c->d_flag + (size_t)s * nk, nk, cudaMemcpyDeviceToHost, c->aux));
    GNM_CU(cudaStreamSynchronize(c->aux));
    if (unmatched)
        for (int k = 0; k < kUnmatched; ++k)
            for (int j = 0; j < 3; ++j) unmatched[k * 3 + j] = un6[k * kNStat + j];
    return device_checks(c);
}

// Enqueues on st the copies of windows' results (after each window's last processing):
// stats, the unmatched rows as stored (un6: kUnmatched x kNStat words per window), rates
// and flags; any of them may be null.
static gnm_status enqueue_results(gnm_ctx* c, const uint64_t* wids, size_t n, uint64_t* stats, uint64_t* un6,
                                  double* rate, uint8_t* flag, cudaStream_t st, std::vector<uint32_t>& slot) {
    const size_t nk = 2 * (size_t)c->n_sites;
    slot.resize(n);
    for (size_t k = 0; k < n; ++k) {
        GNM_TRY(find_window(c, wids[k], &slot[k]));
        if (!c->slots[slot[k]].finalized) return fail(GNM_E_STATE, "window is open (not finalised)");
        GNM_TRY(wait_slot_on_stream(c, slot[k], st));
    }
    for (size_t k = 0; k < n;) {
        // windows k..k+m-1 in consecutive slots: one copy per array for the run (rates and
        // flags are contiguous across slots; stats rows carry the unmatched rows between)
        size_t m = 1;
        while (k + m < n && slot[k + m] == slot[k] + m) ++m;
        const uint32_t s = slot[k];
        if (rate) GNM_CU(cudaMemcpyAsync(rate + k * nk, c->d_rate + (size_t)s * nk, m * nk * 8, cudaMemcpyDeviceToHost, st));
        if (flag) GNM_CU(cudaMemcpyAsync(flag + k * nk, c->d_flag + (size_t)s * nk, m * nk, cudaMemcpyDeviceToHost, st));
        // stats: the run's windows are rows of keys * GNM_NSTAT words, the site rows first
        // and the unmatched rows after them: one pitched copy for each part
        const uint64_t* sp = c->d_stats + (size_t)s * c->keys * kNStat;
        const size_t pitch = (size_t)c->keys * kNStat * 8;
        if (stats)
            GNM_CU(cudaMemcpy2DAsync(stats + k * nk * kNStat, nk * kNStat * 8, sp, pitch, nk * kNStat * 8, m,
                                     cudaMemcpyDeviceToHost, st));
        if (un6)
            GNM_CU(cudaMemcpy2DAsync(un6 + k * kUnmatched * kNStat, kUnmatched * kNStat * 8, sp + nk * kNStat,
                                     pitch, kUnmatched * kNStat * 8, m, cudaMemcpyDeviceToHost, st));
        k += m;
    }
    return GNM_OK;
}

gnm_status gnm_windows_results(gnm_ctx* c, const uint64_t* wids, size_t n, uint64_t* stats,
                               uint64_t* unmatched, double* rate, uint8_t* flag) {
    if (!c || (n && !wids)) return fail(GNM_E_INVAL, "NULL argument");
    GNM_CU(cudaSetDevice(c->device));
    std::vector<uint64_t> un6(unmatched ? n * kUnmatched * kNStat : 0);
    std::vector<uint32_t> slot;
    GNM_TRY(enqueue_results(c, wids, n, stats, unmatched ? un6.data() : nullptr, rate, flag, c->aux, slot));
    GNM_CU(cudaStreamSynchronize(c->aux));
    if (unmatched)
        for (size_t k = 0; k < n; ++k)
            for (int q = 0; q < kUnmatched; ++q)
                for (int j = 0; j < 3; ++j) unmatched[(k * kUnmatched + q) * 3 + j] = un6[(k * kUnmatched + q) * kNStat + j];
    return device_checks(c);
}

gnm_status gnm_windows_results_async(gnm_ctx* c, const uint64_t* wids, size_t n, uint64_t* stats,
                                     uint64_t* unmatched6, double* rate, uint8_t* flag, void* cuda_stream) {
    if (!c || (n && !wids)) return fail(GNM_E_INVAL, "NULL argument");
    GNM_CU(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    std::vector<uint32_t> slot;
    GNM_TRY(enqueue_results(c, wids, n, stats, unmatched6, rate, flag, st, slot));
    // the next work on these slots waits for the copies too
    cudaEvent_t ev;
    GNM_TRY(record_event(c, st, &ev));
    for (uint32_t s : slot) c->slots[s].ev = ev;
    return GNM_OK;
}

gnm_status gnm_window_device(gnm_ctx* c, uint64_t wid, const uint64_t** stats, const double** rate,
                             const uint8_t** flag) {
    if (!c) return fail(GNM_E_INVAL, "ctx is NULL");
    uint32_t s;
    GNM_TRY(find_window(c, wid, &s));
    const size_t nk = 2 * (size_t)c->n_sites;
    if (stats) *stats = c->d_stats + (size_t)s * c->keys * kNStat;
    if (rate) *rate = c->d_rate + (size_t)s * nk;
    if (flag) *flag = c->d_flag + (size_t)s * nk;
    return GNM_OK;
}

gnm_status gnm_site_stats(gnm_ctx* c, uint64_t wid, gnm_site_stat* out, size_t cap, size_t* n_out,
                          uint64_t unmatched[12]) {
    if (!c || !n_out) return fail(GNM_E_INVAL, "NULL argument");
    const size_t nk = 2 * (size_t)c->n_sites;
    std::vector<uint64_t> st(nk * kNStat);
    std::vector<double> rate(nk);
    std::vector<uint8_t> flag(nk);
    GNM_TRY(gnm_window_dense(c, wid, st.data(), unmatched, rate.data(), flag.data()));
    size_t n = 0;
    for (size_t k = 0; k < nk; ++k) n += st[k * kNStat] != 0;
    *n_out = n;
    if (cap < n) return fail(GNM_E_CAPACITY, "cap smaller than the number of active keys");
    size_t j = 0;
    for (size_t k = 0; k < nk; ++k) {
        const uint64_t* r = &st[k * kNStat];
        if (r[0] == 0) continue;
        gnm_site_stat& o = out[j++];
        o.site = (uint32_t)(k >> 1);
        o.dir = (uint32_t)(k & 1);
        o.flows = r[0];
        o.octets = r[1];
        o.pkts = r[2];
        o.e_flows = r[3];
        o.e_octets = r[4];
        o.e_dur_ms = r[5];
        o.rate_bps = rate[k];
        o.flag = flag[k];
        o.reserved = 0;
    }
    return GNM_OK;
}

gnm_status gnm_flag_suboptimal(gnm_ctx* c, uint64_t wid, double thr, uint32_t* site_out,
                               uint8_t* dir_out, size_t cap, size_t* n_out) {
    if (!c || !n_out) return fail(GNM_E_INVAL, "NULL argument");
    GNM_CU(cudaSetDevice(c->device));
    uint32_t s;
    GNM_TRY(find_window(c, wid, &s));
    if (!c->slots[s].finalized) return fail(GNM_E_STATE, "window is open (not finalised)");
    GNM_TRY(wait_slot_on_stream(c, s, c->aux));
    const size_t nk = 2 * (size_t)c->n_sites;
    GNM_CU(launch_flag_compact(c->d_rate + (size_t)s * nk, c->d_stats + (size_t)s * c->keys * kNStat,
                               (uint32_t)nk, thr, c->cfg.min_flows_to_flag, c->d_flag_keys,
                               c->d_flag_count, c->aux));
    uint32_t cnt = 0;
    GNM_CU(cudaMemcpyAsync(&cnt, c->d_flag_count, 4, cudaMemcpyDeviceToHost, c->aux));
    GNM_CU(cudaStreamSynchronize(c->aux));
    std::vector<uint32_t> keys(cnt);
    if (cnt) GNM_CU(cudaMemcpyAsync(keys.data(), c->d_flag_keys, cnt * 4, cudaMemcpyDeviceToHost, c->aux));
    GNM_CU(cudaStreamSynchronize(c->aux));
    *n_out = cnt;
    if (cap < cnt) return fail(GNM_E_CAPACITY, "cap smaller than the number of flagged keys");
    std::sort(keys.begin(), keys.end());
    for (uint32_t i = 0; i < cnt; ++i) {
        if (site_out) site_out[i] = keys[i] >> 1;
        if (dir_out) dir_out[i] = (uint8_t)(keys[i] & 1);
    }
    return device_checks(c);
}

gnm_status gnm_window_release(gnm_ctx* c, uint64_t wid) {
    if (!c) return fail(GNM_E_INVAL, "ctx is NULL");
    uint32_t s;
    GNM_TRY(find_window(c, wid, &s));
    Slot& sl = c->slots[s];
    if (sl.pinned) return fail(GNM_E_STATE, "window id belongs to a plan");
    if (sl.open) {  // keep the zero-accumulator invariant
        GNM_CU(cudaSetDevice(c->device));
        if (sl.ev) GNM_CU(cudaEventSynchronize(sl.ev));
        GNM_CU(cudaMemset(c->d_acc + (size_t)s * c->keys * kAccCols, 0, (size_t)c->keys * kAccCols * 8));
    }
    sl.used = false;
    sl.open = false;
    sl.finalized = false;
    sl.age = 0;
    c->slot_of.erase(wid);
    return GNM_OK;
}

gnm_status gnm_lookup(gnm_ctx* c, const uint32_t* addr, uint64_t n, uint32_t* site_out,
                      uint32_t* pos_out, void* stream) {
    if (!c) return fail(GNM_E_INVAL, "ctx is NULL");
    if (!c->have_registry) return fail(GNM_E_STATE, "no registry loaded");
    if (n && !addr) return fail(GNM_E_INVAL, "addr is NULL");
    GNM_CU(cudaSetDevice(c->device));
    LaunchShape sh;
    GNM_TRY(choose_shape(c, n ? n : 1, &sh));
    if (sh.lookup == kLookupHash24 && pos_out)
        return fail(GNM_E_INVAL, "lookup mode HASH24 gives sites, not range positions (pos_out must be NULL)");
    AggParams p;
    gnm_records none{};
    GNM_TRY(build_params(c, &none, &p));
    p.radix_bits = sh.radix_bits;
    p.rmi.leaves_global = sh.rmi_global ? 1u : 0u;
    GNM_CU(launch_lookup(p, sh.lookup, addr, n, site_out, pos_out, (cudaStream_t)stream));
    c->last_launches = 1;
    return GNM_OK;
}

uint32_t gnm_last_launch_count(const gnm_ctx* c) { return c ? c->last_launches : 0; }

gnm_status gnm_rates(const uint64_t* e_octets, const uint64_t* e_dur_ms, uint64_t n, double* rate,
                     void* stream) {
    if (n == 0) return GNM_OK;
    if (!e_octets || !e_dur_ms || !rate) return fail(GNM_E_INVAL, "NULL array");
    const uintptr_t mis = (uintptr_t)e_octets | (uintptr_t)e_dur_ms | (uintptr_t)rate;
    if (mis & 7u) return fail(GNM_E_INVAL, "arrays must be 8-byte aligned");
    GNM_CU(launch_rates(e_octets, e_dur_ms, n, rate, (cudaStream_t)stream));
    return GNM_OK;
}

gnm_status gnm_registry_flatten(const uint32_t* prefix, const uint8_t* len, const uint32_t* site_id,
                                size_t n, uint32_t n_sites, uint32_t* starts, uint32_t* site,
                                size_t cap, size_t* n_out) {
    if (!n_out) return fail(GNM_E_INVAL, "n_out is NULL");
    if (n && (!prefix || !len || !site_id)) return fail(GNM_E_INVAL, "registry arrays are NULL");
    if (n_sites == 0 || n_sites > (1u << 26)) return fail(GNM_E_INVAL, "n_sites must be 1..2^26");
    std::vector<uint32_t> st, si;
    const std::string why = flatten_registry(prefix, len, site_id, n, n_sites, &st, &si);
    if (!why.empty()) return fail(GNM_E_INVAL, why);
    *n_out = st.size();
    if (cap < st.size()) return fail(GNM_E_CAPACITY, "cap smaller than the number of ranges");
    if (starts) std::memcpy(starts, st.data(), st.size() * 4);
    if (site) std::memcpy(site, si.data(), si.size() * 4);
    return GNM_OK;
}

int gnm_checked_build(void) { return GNM_CHECKED; }

gnm_status gnm_device_checks(gnm_ctx* c, uint64_t* word) {
    if (!c) return fail(GNM_E_INVAL, "ctx is NULL");
    GNM_CU(cudaSetDevice(c->device));
    GNM_CU(cudaDeviceSynchronize());
    unsigned long long v = 0;
    GNM_CU(cudaMemcpy(&v, c->d_check, 8, cudaMemcpyDeviceToHost));
    if (word) *word = v;
    const gnm_status st = device_checks(c);
    GNM_CU(cudaMemset(c->d_check, 0, 8));
    return st;
}

gnm_status gnm_debug_corrupt(gnm_ctx* c, int32_t what, uint32_t index, uint32_t value) {
    if (!c) return fail(GNM_E_INVAL, "ctx is NULL");
#if GNM_CHECKED
    if (what != GNM_DEBUG_RMI_SPLIT_BASE) return fail(GNM_E_INVAL, "unknown corruption");
    if (!c->rmi_ready) return fail(GNM_E_STATE, "no learned index");
    if (index >= c->rmi.n_leaves || index >= c->rmi_split.size() || !c->rmi_split[index])
        return fail(GNM_E_INVAL, "index is not a split leaf");
    GNM_CU(cudaSetDevice(c->device));
    GNM_CU(cudaDeviceSynchronize());
    // the split leaf's first sub-leaf, in the model arrays and in their interleaved copy
    GNM_CU(cudaMemcpy(const_cast<float*>(c->rmi.b) + index, &value, 4, cudaMemcpyHostToDevice));
    GNM_CU(cudaMemcpy(reinterpret_cast<uint32_t*>(c->d_rmi_leaf4 + index) + 1, &value, 4, cudaMemcpyHostToDevice));
    return GNM_OK;
#else
    (void)what;
    (void)index;
    (void)value;
    return fail(GNM_E_STATE, "state can be corrupted only in the checked build (libgnm_checked.so)");
#endif
}

}  // extern "C"
