// gnm_internal.cuh -- device-side layouts and launch parameters shared by the library's
// translation units (never by the oracle).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "gnm.h"
#include "hash24.hpp"

// The checked build (-DGNM_CHECKED=1, libgnm_checked.so) tests every index at the points
// where kernels trust data -- a record's key before the table, accumulator and histogram
// accesses it drives, a registry search's starting window before its loads, a learned-index
// model number, a regrouping bucket and position, a partial block -- and on a failure skips
// the access and records the first failure in a device word that the host reports as
// GNM_E_INTERNAL. In the default build the checks compile away.
#ifndef GNM_CHECKED
#define GNM_CHECKED 0
#endif

namespace gnm {

// Check sites of the checked build (the top byte of the device error word).
enum : uint32_t {
    kChkKey = 1,          // a record's key beyond its table / accumulator rows
    kChkWindow = 2,       // a registry search window beyond the ranges
    kChkBlocks = 3,       // a block-sample search window beyond the blocks
    kChkModel = 4,        // a learned-index model number beyond the models
    kChkBucket = 5,       // a regrouping bucket beyond the launch's buckets
    kChkPosition = 6,     // a regrouped record position beyond the records
    kChkPartial = 7,      // a partial-sum block beyond the partial area
    kChkHostKey = 8,      // a per-host key beyond the site keys
};

__host__ __device__ inline const char* check_site_name(uint32_t s) {
    switch (s) {
        case kChkKey: return "record key beyond its table or accumulator rows";
        case kChkWindow: return "registry search window beyond the ranges";
        case kChkBlocks: return "block-sample search window beyond the blocks";
        case kChkModel: return "learned-index model number beyond the models";
        case kChkBucket: return "regrouping bucket beyond the launch's buckets";
        case kChkPosition: return "regrouped record position beyond the records";
        case kChkPartial: return "partial-sum block beyond the partial area";
        case kChkHostKey: return "per-host key beyond the site keys";
        default: return "unknown check";
    }
}

constexpr uint32_t kNoSite = GNM_NO_SITE;
constexpr int kNStat = GNM_NSTAT;   // columns of a user-facing stats row
constexpr uint32_t kRateBuckets = GNM_RATE_BUCKETS;  // 10 kb/s buckets, the last for >= 100 Mb/s
constexpr int kAccCols = 5;         // accumulator row: flows<<32|e_flows, ineligible oct, pkts, e_oct, e_dur
constexpr size_t kSmemRowBytes = 20;  // per-CTA shared-memory row: packed counts + 4 low words
constexpr int kUnmatched = 4;       // classes appended after the 2*n_sites site rows
constexpr int kMaxLeaves = 1 << 20;
constexpr uint32_t kMaxModels = 1u << 22;  // leaves plus sub-leaves of split leaves
// eps word of a split leaf's record: its `a` bits hold shift | (count - 1) << 8 and its `b`
// bits the index of its first sub-leaf; x0 is the leaf's first address. Packed bounds never
// take this value (each half is at most 0xFFFE, else the word is 0xFFFFFFFF).
constexpr uint32_t kEpsSplit = 0xFFFFFFFEu;
constexpr int kMaxHidden = 32;
constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;

// One window of a launch: records [begin, end) of the launch's struct-of-arrays.
struct WinDesc {
    uint64_t begin, end;
    uint32_t slot;       // result slot
    uint32_t flags;      // kWinFinalize
    uint32_t ctas;       // CTAs whose record range overlaps the window (ticket target)
    uint32_t part_base;  // first partial-sum block of the window (when partials are used)
    uint32_t n_parts;    // partial-sum blocks of the window (one per CTA piece)
    uint32_t key_base;   // first key of the segment's key group (partitioned launches), else 0
};
// Words between consecutive partial-sum blocks of `rows` 20-byte rows: padded to 16 bytes
// so that the blocks can be read with 16-byte loads.
__host__ __device__ constexpr uint64_t part_stride_words(uint64_t rows) { return (rows * 5u + 3u) & ~3ull; }

// A CTA flushes its shared sums at least every kFlushRecords records (16-bit counts).
constexpr uint64_t kFlushRecords = 65532;  // < 2^16, multiple of 4
// Direct tables with partial blocks: pieces after which only rows with counts >= 2^15 flush.
constexpr uint64_t kCountPiece = 32764;    // 2^15 + kCountPiece < 2^16, multiple of 4
constexpr uint32_t kWinFinalize = 1u;

// Learned index: root parameters by value, per-model arrays in device memory (the root's
// n_leaves leaves, then the sub-leaves of split leaves).
struct RmiDev {
    int32_t root_kind;     // GNM_RMI_ROOT_*
    uint32_t n_leaves;
    uint32_t n_models;     // n_leaves + sub-leaves; the length of a, b, x0, eps, leaf4
    uint32_t hidden;
    float ra, rb;          // linear root, on xn = float(x) * 2^-32
    float w1[kMaxHidden], b1[kMaxHidden], w2[kMaxHidden], b2;
    const float* a;
    const float* b;
    const uint32_t* x0;
    const uint32_t* eps;   // packed eps_lo | eps_hi << 16; 0xFFFFFFFF: always full search;
                           // kEpsSplit: a split leaf
    const uint4* leaf4;    // per model (a bits, b bits, x0, eps) interleaved: one 16-byte load
    uint32_t leaves_global;  // this launch reads leaf4 from global memory instead of staging
    unsigned long long* check_err;  // the checked build's error word
};

struct AggParams {
    // struct-of-arrays records of this launch
    const uint32_t* src;
    const uint32_t* dst;
    const uint32_t* pkts;
    const uint32_t* oct;
    const uint32_t* first;
    const uint32_t* last;
    uint64_t n_total;
    uint64_t chunk;              // records per CTA (multiple of 4)
    const WinDesc* wins;
    uint32_t n_wins;
    uint32_t vec_ok;             // all six arrays share the same 16-byte phase
    uint32_t phase;              // (address / 4) mod 4 of element 0
    // registry
    const uint32_t* starts;
    const uint32_t* rsite;
    const uint2* pairs;          // (start, site) of every range, then 16 padding entries
    const uint4* blocks;         // staged placement: 16 starts per block (64 bytes)
    const uint32_t* sample;      // staged placement: first start of every block
    const uint32_t* dir16;       // radix directory over the top 16 bits (65537 entries)
    uint32_t radix_bits;         // directory bits used by this launch (<= 16)
    uint32_t dir_iters;          // shared-memory registry behind a directory: search steps that
                                 // narrow its largest bucket to one range
    const uint32_t* sample4;     // key kernel: first start of every 4-range block of pairs
    uint32_t n_blk4;
    const uint32_t* sample2;     // key kernel: first start of every 2-range block of pairs
    uint32_t n_blk2;
    const uint16_t* dirh;        // key kernel (n_blk2 < 2^16): per /16 bucket t, the first 2-range
                                 // block whose first start is >= t << 16 (65537 entries)
    const uint16_t* smp16;       // the low 16 bits of every 2-range block's first start
    const uint2* h24;            // /24 subnet hash table: (subnet + 1, site), 0 = empty
    uint32_t h24_mask;           // table slots - 1
    uint32_t n_blocks;
    uint32_t n_ranges;
    uint32_t n_sites;
    uint32_t pad1;
    // learned index (lookup mode RMI)
    RmiDev rmi;
    // local site
    uint32_t local_pfx[GNM_MAX_LOCAL];
    uint32_t local_mask[GNM_MAX_LOCAL];
    uint32_t n_local;
    // filters
    uint32_t min_avg, min_pkts, min_dur;
    int32_t admin_rule;
    // results
    uint64_t* acc;               // [slots][keys][kAccCols] accumulators (zeroed per window)
    uint8_t* dirty;              // [slots][dirty_groups]: nonzero when a launch may have written an
                                 // accumulator row of the 32-key group since it was last finalised
                                 // (null: every row is read)
    uint64_t* stats;             // [slots][keys][kNStat] finalised sums
    uint32_t* hist;              // [slots][2*n_sites][kRateBuckets] rate histograms, or null
    unsigned long long* rmin;    // [slots][2*n_sites] least rate (bits of a double >= 0)
    unsigned long long* rmax;    // [slots][2*n_sites] greatest rate
    // sparse rate statistics (hist == null): per slot a log of (key << 14 | bucket) words of
    // the eligible flows, its capacity in words and the words appended so far (or null)
    uint32_t* const* rlog;
    const uint32_t* rlog_cap;
    uint32_t* rlog_cnt;
    unsigned long long* hkeys;   // [slots][hcap] host table keys ((addr << 1 | dir) + 1; 0 empty), or null
    unsigned long long* hrows;   // [slots][hcap][kNStat] host sums
    uint32_t* hover;             // [slots] hosts that found no free entry
    uint32_t hcap;               // host table entries per slot (power of two)
    double* rate;                // [slots][2*n_sites]
    uint8_t* flag;               // [slots][2*n_sites]
    uint32_t keys;               // 2*n_sites + 4
    uint32_t table_rows;         // rows of a direct shared-memory table: keys, or one key group
    uint32_t part_groups;        // key groups per window of a partitioned launch (0: none)
    uint32_t dirty_groups;       // ceil(keys / 32)
    const uint2* part_desc;      // [window][group]: (first partial block, blocks) of a partitioned launch
    uint32_t table_cap;          // shared-memory hash slots (table mode 1)
    uint32_t min_flows;
    uint32_t pad0;
    double threshold;
    // scratch
    uint32_t* partials;          // per (window, CTA) dumps of the shared rows, or null
    uint32_t* done;              // [n_wins] finalise tickets, zero between launches
    unsigned long long* violations;  // learned-index fallbacks
    unsigned long long* check_err;   // the checked build's error word (site << 56 | value)
    // key kernel of a partitioned launch: per (window, key group) record counts (global,
    // zeroed before the launch), the keys per group, and the shared-memory offset of the
    // kernel's own counts (or key_hist == null)
    uint32_t* key_hist;
    uint32_t key_group_rows;
    uint32_t key_hist_off;
    uint64_t partial_cap;            // words of `partials` (checked build)
    uint64_t part_cap;               // records of a partitioned launch's regrouped arrays (checked build)
};

// The checked build's test: false when !ok, recording the first failure as site << 56 |
// value; in the default build always true, and the compiler drops the test.
__device__ __forceinline__ bool chk(unsigned long long* err, bool ok, uint32_t site, uint64_t value) {
#if GNM_CHECKED
    if (!ok && err) atomicCAS(err, 0ull, ((unsigned long long)site << 56) | (value & 0x00FFFFFFFFFFFFFFull));
    return ok;
#else
    (void)err;
    (void)site;
    (void)value;
    return true;
#endif
}

// kLookupKeys: the aggregation reads per-record keys that a lookup kernel wrote (split
// launches), instead of addresses.
// kLookupRadixBlk / kLookupRadixBlk2 (key kernel only): a directory of blocks of 4 (2)
// ranges and the blocks' first starts in shared memory; one 32-byte (16-byte) load of the
// block's (start, site) pairs ends the lookup.
// kLookupRadixBlk2H (key kernel only): 2-range blocks found through a directory over the top
// 16 address bits and the blocks' low 16 start bits, both 16-bit, in shared memory.
// kLookupHash24: the paper's /24 subnet hash table (registries of prefixes up to /24).
enum { kLookupL2 = 0, kLookupSmem = 1, kLookupRmi = 2, kLookupStaged = 3, kLookupRadix = 4, kLookupKeys = 5,
       kLookupRadixBlk = 6, kLookupRadixBlk2 = 7, kLookupHash24 = 8, kLookupRadixBlk2H = 9 };


// Largest block of the key kernel for a lookup and records-per-thread unroll: two groups
// of lookups per thread fit 64 registers (1024 threads) only for the lighter lookups.
__host__ __device__ constexpr int keys_block_max(int lookup, int unroll) {
    return (unroll == 1 || lookup == kLookupRadixBlk2 || lookup == kLookupRadixBlk2H || lookup == kLookupRadix ||
            lookup == kLookupL2)
               ? 1024
               : 512;
}
constexpr uint32_t kBlockRanges = 16;  // ranges per staged block (16 starts, 64 bytes)
enum { kTableDirect = 0, kTableHash = 1, kTableGlobal = 2 };

// Largest block of the aggregation kernel: two groups of 4 records per thread (40 words
// of records in flight per thread) take more than the 64 registers of 1024-thread blocks;
// a group in flight while the previous one is processed (unroll 3) fits 80 registers.
__host__ __device__ constexpr int agg_block_max(int lookup, int table, int agg, int unroll) {
    return (void)lookup, (void)table, (void)agg, unroll == 1 ? 1024 : unroll == 3 ? 768 : 512;
}

// Launch shape chosen by the host.
struct LaunchShape {
    int block;
    int ctas_per_sm;
    int unroll;      // 1 or 2 four-record groups per thread per iteration
    int lookup;      // kLookup*
    int table;       // kTable*
    int agg;         // GNM_AGG_DIRECT / GNM_AGG_WARP (shared-memory tables only)
    int grid;
    uint32_t cap;    // hash-table slots (kTableHash)
    uint32_t radix_bits;  // kLookupRadix directory bits
    uint32_t dir_iters;   // kLookupSmem with a directory: fixed search steps (see AggParams)
    int rmi_global;       // kLookupRmi: leaf parameters read from global memory (L2/L1)
    size_t smem;
    // split launches: a lookup kernel (this lookup method) writes keys, then the
    // aggregation kernel reads them (kLookupKeys)
    int split;
    int keys_grid, keys_block;
    size_t keys_smem;
    int keys_blk;          // radix key kernel: ranges per block of its shared block samples (0: none)
    int keys_h16;          // ... with the 16-bit directory and 16-bit samples (2-range blocks)
    uint32_t keys_bits;    // its directory bits
    int keys_unroll;       // key kernel: groups of 4 records per thread and step (1 or 2)
    // partitioned launches (split launches whose keys exceed one direct table): records are
    // regrouped by (window, group of part_rows keys) before the aggregation
    int part;
    uint32_t part_rows, part_groups;
    int part_grid;
};

// partition.cu: count, scan and scatter of a partitioned launch. `p` is the launch's
// parameters (records, windows, keys of the key kernel at p.src); cnt (n_wins * groups
// words) holds the bucket sizes, then their next free places; `out` receives the
// regrouped records (key within its group, pkts, octets, first, last: 5 arrays of
// part_array_stride(n) words); `descs` the aggregation's segment descriptors (n_wins *
// groups entries), `part_desc` the finalisation's partial-block ranges per bucket.
constexpr uint32_t kPartMaxBuckets = 8192;
uint64_t part_array_stride(uint64_t n);
cudaError_t launch_part_count(const AggParams& p, const LaunchShape& s, uint32_t* cnt, cudaStream_t st);
cudaError_t launch_part_scan(const AggParams& p, const LaunchShape& s, uint64_t agg_chunk, uint32_t* cnt,
                             WinDesc* descs, uint2* part_desc, cudaStream_t st);
cudaError_t launch_part_scatter(const AggParams& p, const LaunchShape& s, uint32_t* cnt, uint32_t* out,
                                cudaStream_t st);

// aggregate*.cu
cudaError_t launch_aggregate(const AggParams& p, const LaunchShape& s, cudaStream_t st);
cudaError_t launch_keys(const AggParams& p, const LaunchShape& s, uint32_t* keys, cudaStream_t st);
size_t aggregate_smem_bytes(int lookup, int table, uint32_t n_ranges, uint32_t keys,
                            uint32_t table_cap, uint32_t n_leaves, uint32_t radix_bits);
cudaError_t launch_finalize(const AggParams& p, uint32_t slot, cudaStream_t st);
// Finalises every window of a launch from its partial-sum blocks (grid over windows x keys).
cudaError_t launch_finalize_windows(const AggParams& p, cudaStream_t st);
// Runs of below-standard medians: run[k] = med[k] < below ? run[k] + 1 : 0; keys whose run
// reaches `consecutive` are appended to out (count via *n).
cudaError_t launch_warn_runs(const uint32_t* med, uint32_t n_keys, uint32_t below, uint32_t consecutive,
                             uint32_t* run, uint32_t* out, uint32_t* n, cudaStream_t st);
// Per-host sums of a split launch: after the key kernel (keys at `keys`, same phase as the
// records), every record of a registered site adds to its (remote host, dir) entry of its
// window's host table.
cudaError_t launch_host_stats(const AggParams& p, const uint32_t* keys, int grid, cudaStream_t st);
// FP64 rate of each of n host entries (rows of kNStat sums).
cudaError_t launch_host_rates(const unsigned long long* rows, uint32_t n, double* rate, cudaStream_t st);
// rsort.cu: LSD radix sort of n words (bits significant bits, 8 per pass) between keys and
// tmp; *result is whichever holds the sorted words. hist needs radix_sort_hist_words(n).
size_t radix_sort_hist_words(uint32_t n, int sms);
cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* tmp, uint32_t n, int bits, uint32_t* hist, int sms,
                           cudaStream_t st, uint32_t** result);
// Lower-median bucket and eligible-flow count of every key from a sorted sparse log.
cudaError_t launch_sparse_median(const uint32_t* sorted, uint32_t n, uint32_t n_keys, uint32_t* med, uint32_t* count,
                                 cudaStream_t st);
// Lower-median bucket and eligible-flow count of every site key of one slot's histograms.
cudaError_t launch_rate_median(const uint32_t* hist, uint32_t n_keys, uint32_t* med, uint32_t* count,
                               cudaStream_t st);
cudaError_t launch_flag_compact(const double* rate, const uint64_t* stats, uint32_t n_site_keys,
                                double thr, uint32_t min_flows, uint32_t* out_keys,
                                uint32_t* out_count, cudaStream_t st);
cudaError_t launch_lookup(const AggParams& p, int lookup, const uint32_t* addr, uint64_t n,
                          uint32_t* site_out, uint32_t* pos_out, cudaStream_t st);
// Rates of n given (eligible octets, eligible milliseconds) sums (the rate step alone).
cudaError_t launch_rates(const uint64_t* e_octets, const uint64_t* e_dur_ms, uint64_t n, double* rate,
                         cudaStream_t st);

// Unique id of the calling thread's current CUDA context (the driver's cuCtxGetId,
// reached through the runtime's driver entry point, so the library does not link the
// driver library itself); 0 when there is no current context or it cannot be read.
unsigned long long current_context_id();

// Per-device record of the dynamic shared memory a kernel has been granted, valid for one
// context: a device reset or a new primary context starts again from nothing.
struct OptInCache {
    std::mutex mu;
    unsigned long long ctx[64] = {};
    int bytes[64] = {};
};
// Grants kernel `fn` `bytes` of dynamic shared memory (cudaFuncSetAttribute) unless the
// current context already granted as much; thread-safe.
cudaError_t ensure_smem_optin(const void* fn, int bytes, OptInCache& cache);

// rmi.cu
// A trained model on the host: the root (in RmiDev) and per model a, b, x0 and the initial
// eps word (kEpsSplit for split leaves, else 0 until the bounds are computed).
struct RmiTrainOut {
    double root_loss = 0.0;
    uint32_t empty_leaves = 0, split_leaves = 0;
    std::vector<float> a, b;
    std::vector<uint32_t> x0, eps;
    std::vector<uint32_t> split;  // per leaf: 0, or shift | (count - 1) << 8
};
size_t rmi_train_scratch_bytes(uint64_t n, uint32_t n_leaves);
size_t rmi_partials_bytes();  // per-block partial sums of the ordered reductions
// Root and leaves (model arrays in `out`, on the host). `pos` holds the plain search's
// positions of the n device keys; `starts` the device range starts.
cudaError_t rmi_train_device(RmiDev* model, const uint32_t* keys, const uint32_t* pos, uint64_t n,
                             const uint32_t* starts, uint32_t n_ranges, const gnm_rmi_config& cfg,
                             void* scratch, RmiTrainOut* out, cudaStream_t st);
// Over n_s training lookups: out2[0] = sum of squared position errors, out2[1] = sum of the
// window widths searched.
cudaError_t rmi_model_stats(const RmiDev& model, const uint32_t* keys, const uint32_t* pos, uint64_t n_s,
                            uint32_t n_ranges, double* part, double* out2, cudaStream_t st);
cudaError_t rmi_eps_sweep(const RmiDev& model, const uint32_t* starts, uint32_t n_ranges,
                          uint32_t* d_eps_lo, uint32_t* d_eps_hi, int sm_count, cudaStream_t st);
cudaError_t rmi_eps_from_samples(const RmiDev& model, const uint32_t* keys, const uint32_t* pos,
                                 uint64_t n, uint32_t n_ranges, uint32_t* d_eps_lo,
                                 uint32_t* d_eps_hi, cudaStream_t st);
cudaError_t rmi_pack_eps(const uint32_t* lo, const uint32_t* hi, uint32_t* packed,
                         uint32_t n_leaves, cudaStream_t st);
cudaError_t rmi_pack_leaf4(const float* a, const float* b, const uint32_t* x0, const uint32_t* eps, uint4* out,
                           uint32_t L, cudaStream_t st);
cudaError_t rmi_linear_grad(const float* z, const float* y, uint64_t n, float w, float c,
                            double* d_part, double* d_acc3, cudaStream_t st);
cudaError_t rmi_mlp_grad(const float* xn, const float* y, uint64_t n, uint32_t hidden,
                         const float* d_params, double* d_part, double* d_grad, cudaStream_t st);

}  // namespace gnm
