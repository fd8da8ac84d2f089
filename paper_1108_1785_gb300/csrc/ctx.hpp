// ctx.hpp -- host-side state of a gnm context (library-internal).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "gnm.h"
#include "gnm_internal.cuh"

namespace gnm {

// Thread-local message of the last failure.
void set_error(const std::string& msg);
const char* get_error();

#define GNM_CU(call)                                                                     \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            (void)cudaGetLastError(); /* do not leak a non-sticky error into later calls */ \
            ::gnm::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));        \
            return GNM_E_CUDA;                                                           \
        }                                                                                \
    } while (0)

#define GNM_TRY(expr)                     \
    do {                                  \
        gnm_status s_ = (expr);           \
        if (s_ != GNM_OK) return s_;      \
    } while (0)

gnm_status fail(gnm_status s, const std::string& msg);

// One result slot on the device.
struct Slot {
    bool used = false;
    bool open = false;        // accumulating, not finalised
    bool finalized = false;
    bool pinned = false;      // owned by a plan: never evicted or reassigned
    uint64_t window_id = 0;
    uint64_t records = 0;     // records added so far (must stay below 2^32)
    uint64_t age = 0;         // assignment order, for eviction
    cudaEvent_t ev = nullptr; // recorded after the last work that wrote the slot (not owned;
                              // re-recording it later only makes waits more conservative)
};

// Per-launch device scratch: window descriptors and finalise tickets.
struct LaunchBuf {
    WinDesc* h_wins = nullptr;   // pinned
    WinDesc* d_wins = nullptr;
    uint32_t* d_done = nullptr;  // zero between launches (each launch resets it)
    uint32_t cap = 0;
    uint32_t* d_partials = nullptr;  // per-(window, CTA) partial sums
    uint64_t partial_cap = 0;        // in u32 words
    uint32_t* d_keys = nullptr;      // per-record keys of split launches
    uint64_t keys_cap = 0;           // in u32 words
    unsigned char* d_part = nullptr; // regrouped records and bucket tables of partitioned launches
    uint64_t part_cap = 0;           // in bytes
    cudaEvent_t ev = nullptr;
    bool ev_recorded = false;
};

struct Staging {
    uint32_t* d[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    uint64_t cap = 0;
    cudaEvent_t ev = nullptr;
    bool ev_recorded = false;
};

// Pipelined staging of host records (GNM_HOST_PIPELINE): two buffer sets, the copy of one
// chunk of windows on `copy` overlapping the processing of the previous chunk.
struct PipeStaging {
    uint32_t* d[2][6] = {};
    uint64_t cap = 0;                       // records per buffer set
    cudaStream_t copy = nullptr;            // non-blocking copy stream
    cudaEvent_t copied[2] = {nullptr, nullptr};
    cudaEvent_t freed[2] = {nullptr, nullptr};  // recorded on the processing stream after a chunk
    bool freed_recorded[2] = {false, false};
};

struct Tuned {
    int block = 0, ctas_per_sm = 0, unroll = 0, agg = 0, placement = 0, split = 0, key_dir = 0, keys_unroll = 0;
    uint32_t radix_bits = 0;
};

}  // namespace gnm

struct gnm_ctx {
    gnm_config cfg{};
    int device = 0;
    int sm_count = 0;
    int smem_optin = 0;      // max dynamic shared memory per block
    int smem_per_sm = 0;
    // registry
    bool have_registry = false;
    uint32_t n_sites = 0;
    uint32_t n_prefixes = 0;
    uint32_t keys = 0;       // 2*n_sites + 4
    std::vector<uint32_t> h_starts, h_site;
    uint32_t* d_starts = nullptr;
    uint32_t* d_site = nullptr;
    uint2* d_pairs = nullptr;       // (start, site) interleaved, 16 padding entries at the end
    uint32_t* d_blocks = nullptr;   // staged placement: [n_blocks][8 starts, 8 sites]
    uint32_t* d_sample = nullptr;   // staged placement: first start of every block
    uint32_t n_blocks = 0;
    uint32_t* d_dir16 = nullptr;    // radix directory: range of each /16's first address
    uint32_t* d_sample4 = nullptr;  // key kernel: first start of every 4-range block
    uint32_t n_blk4 = 0;
    uint32_t* d_sample2 = nullptr;  // key kernel: first start of every 2-range block
    uint32_t n_blk2 = 0;
    uint16_t* d_dirh = nullptr;     // key kernel, n_blk2 < 2^16: 16-bit directory of 2-range blocks
    uint16_t* d_smp16 = nullptr;    // ... and the low 16 bits of their first starts
    uint2* d_h24 = nullptr;         // /24 subnet hash table (registries of prefixes up to /24)
    uint32_t h24_mask = 0;
    uint32_t local_pfx[GNM_MAX_LOCAL] = {0};
    uint32_t local_mask[GNM_MAX_LOCAL] = {0};
    uint32_t n_local = 0;
    // window results
    uint32_t n_slots = 0;
    uint64_t* d_acc = nullptr;
    uint8_t* d_dirty = nullptr;   // [slots][ceil(keys / 32)] written-group marks of d_acc
    uint64_t* d_stats = nullptr;
    double* d_rate = nullptr;
    uint8_t* d_flag = nullptr;
    uint32_t* d_hist = nullptr;           // rate statistics (cfg.rate_stats): [slots][2S][10001]
    unsigned long long* d_rmin = nullptr; // [slots][2S]
    unsigned long long* d_rmax = nullptr; // [slots][2S]
    uint32_t* d_med = nullptr;            // [2S] readout scratch: median buckets
    uint32_t* d_mcnt = nullptr;           // [2S] readout scratch: eligible flows
    uint32_t* d_warn_run = nullptr;       // [2S] windows in a row with a below-standard median
    // sparse rate statistics (cfg.rate_stats == 2): per slot a log of (key << 14 | bucket)
    // words of the eligible flows, sorted when the statistics are first read
    std::vector<uint32_t*> rlog;          // [slots] device logs
    std::vector<uint64_t> rlog_cap;       // [slots] capacity in words
    std::vector<char> rlog_sorted;        // [slots] sorted since the window was cleared
    uint32_t** h_rlog_ptr = nullptr;      // [slots] page-locked mirrors of the tables below
    uint32_t* h_rlog_cap = nullptr;
    uint32_t** d_rlog_ptr = nullptr;      // [slots] device copy of rlog
    uint32_t* d_rlog_cap = nullptr;       // [slots] device copy of rlog_cap
    uint32_t* d_rlog_cnt = nullptr;       // [slots] words appended
    uint32_t* d_rlog_tmp = nullptr;       // sort scratch (words) and histograms
    uint64_t rlog_tmp_cap = 0;
    uint32_t* d_rs_hist = nullptr;
    uint64_t rs_hist_cap = 0;
    unsigned long long* d_hkeys = nullptr; // per-host sums (cfg.host_capacity): [slots][hcap] keys
    unsigned long long* d_hrows = nullptr; // [slots][hcap][6] sums
    uint32_t* d_hover = nullptr;           // [slots] hosts lost to a full table
    double* d_hrate = nullptr;             // [hcap] readout scratch: host rates
    uint32_t hcap = 0;
    std::vector<gnm::Slot> slots;
    std::unordered_map<uint64_t, uint32_t> slot_of;
    uint64_t age = 0;
    // scratch
    std::vector<gnm::LaunchBuf> ring;
    uint32_t ring_next = 0;
    gnm::Staging staging;
    gnm::PipeStaging pipe;
    unsigned long long* d_violations = nullptr;
    unsigned long long* d_check = nullptr;  // the checked build's error word (site << 56 | value)
    uint32_t* d_flag_keys = nullptr;
    uint32_t* d_flag_count = nullptr;
    // learned index
    bool rmi_ready = false;
    gnm::RmiDev rmi{};
    float* d_rmi_a = nullptr;
    float* d_rmi_b = nullptr;
    uint32_t* d_rmi_x0 = nullptr;
    uint4* d_rmi_leaf4 = nullptr;  // leaf parameters interleaved (16 bytes per leaf)
    uint32_t* d_rmi_eps = nullptr;  // packed
    uint32_t* d_rmi_elo = nullptr;
    uint32_t* d_rmi_ehi = nullptr;
    uint32_t rmi_cap = 0;
    std::vector<uint32_t> rmi_split;  // per leaf: 0, or shift | (count - 1) << 8
    // tuning
    gnm::Tuned tuned;
    uint32_t last_launches = 0;
    cudaStream_t aux = nullptr;  // private non-blocking stream for readouts
};

namespace gnm {
// shared by api.cu, plan.cu and rmi_api.cu
gnm_status build_params(gnm_ctx* c, const gnm_records* rec, AggParams* p);
gnm_status choose_shape(gnm_ctx* c, uint64_t n_records, LaunchShape* s, size_t n_win = 1);
gnm_status acquire_slot(gnm_ctx* c, uint64_t window_id, cudaStream_t st, uint32_t* slot_out);
void release_slots(gnm_ctx* c);
gnm_status check_windows(gnm_ctx* c, const gnm_records* rec, const uint64_t* offsets, size_t n_win);

// A launch over windows [offsets[k], offsets[k+1]) of device records `dr` (already
// rebased so that offsets[0] is element 0): parameters, shape and descriptors.
struct Prepared {
    AggParams p;
    LaunchShape sh;
    std::vector<WinDesc> wins;   // non-empty windows only
    bool fin_in_kernel = false;
    bool fin_grid = false;       // finalise in a grid-wide kernel after the aggregation
    uint64_t n = 0;
    uint64_t partial_words = 0;  // u32 words of per-(window, CTA) partial sums (0: none)
    uint32_t n_buckets = 0;      // partitioned launches: (window, key group) buckets
    uint64_t part_bytes = 0;     // partitioned launches: their scratch (part_layout)
};
// Scratch of a partitioned launch of n records and nb buckets: the five regrouped record
// arrays, then the bucket counts, segment descriptors and partial-block ranges.
struct PartLayout {
    uint64_t cnt, descs, pdesc, bytes;
};
PartLayout part_layout(uint64_t n, uint32_t nb);
gnm_status prepare_launch(gnm_ctx* c, const gnm_records* dr, const uint64_t* offsets, size_t n_win,
                          const uint32_t* slots, bool finalize, Prepared* out);
// Enqueues the kernels of a prepared launch (descriptors already on the device).
// marks (optional, 4 timing events): recorded before the first kernel and after each
// one; kinds[i] receives the gnm_kernel_kind of kernel i.
// fresh: the windows start in this launch (their rate statistics are cleared first).
gnm_status enqueue_prepared(gnm_ctx* c, Prepared& pr, const uint64_t* offsets, size_t n_win,
                            const uint32_t* slots, bool finalize, WinDesc* d_wins, uint32_t* d_done,
                            uint32_t* d_partials, uint32_t* d_keys, unsigned char* d_part, cudaStream_t st,
                            uint32_t* launches, cudaEvent_t* marks = nullptr, int32_t* kinds = nullptr,
                            bool fresh = true);
constexpr int kMaxPlanKernels = 7;  // keys, hosts, count, scan, scatter, aggregate, finalise
// Next launch-scratch entry of the ring (waits for its previous use).
gnm_status acquire_ring(gnm_ctx* c, uint32_t n_win, LaunchBuf** out);
void set_slots_done(gnm_ctx* c, const uint32_t* slots, size_t n, cudaEvent_t ev, bool finalized);
void unpin_slot(gnm_ctx* c, uint32_t s);
// Grows every launch-ring entry's scratch for single-window launches of up to n records.
gnm_status reserve_launch_scratch(gnm_ctx* c, uint64_t n);
// Clears the rate statistics of slots[0..n) on st (windows that start there).
gnm_status clear_rate_stats(gnm_ctx* c, const uint32_t* slots, size_t n, cudaStream_t st);
// Checked build: GNM_E_INTERNAL (naming the check) when a device bounds check has failed
// since the context's error word was last cleared; the default build returns GNM_OK.
gnm_status device_checks(gnm_ctx* c);
// Sparse rate statistics: room for need[k] log words in slot slots[k] (keeping the words
// already logged); synchronises `st` when a log grows, so call it outside stream capture.
gnm_status reserve_rate_log(gnm_ctx* c, const uint32_t* slots, const uint64_t* need, size_t n, cudaStream_t st);
// Windows k = [offsets[k], offsets[k+1]) of rec on stream st. finalize: rates and flags at
// the end; open_add: add to windows already open instead of starting them.
gnm_status run_windows(gnm_ctx* c, const gnm_records* rec, const uint64_t* offsets, const uint64_t* wids,
                       size_t n_win, cudaStream_t st, bool finalize, bool open_add);
// Starts window wid with zero sums in a slot (pin: the slot is never evicted until unpinned).
gnm_status open_window(gnm_ctx* c, uint64_t wid, cudaStream_t st, bool pin, uint32_t* slot_out);
// Finalises an open window on st: rates and flags from its sums, which are zeroed.
gnm_status close_window(gnm_ctx* c, uint64_t wid, cudaStream_t st);
}  // namespace gnm
