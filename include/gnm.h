/*
 * gnm.h -- C ABI of the GB300 flow-analysis library (G-NetMon hot path).
 *
 * Paper: W. Wu, P. DeMar, D. Holmgren, A. Singh, R. Pordes, "G-NetMon: A GPU-accelerated
 * Network Performance Monitoring System for Large Scale Scientific Collaborations".
 *
 * The library computes, for every window of NetFlow-v5-shaped flow records:
 *   - the remote endpoint's collaboration site, by longest-prefix match against the
 *     registered subnets (Sec. III.B.1 "Site Registration Thread", Sec. III.B.2.1
 *     "Catalog Kernel" / "TransRate Kernel");
 *   - per (site, direction) unsigned 64-bit sums of flows, octets and packets of every
 *     record between the local site and a registered site, and of flows, octets and
 *     durations of the records that pass the ACK and administrative filters
 *     (Sec. III.B.2.1);
 *   - the site transfer rate in bits per second, 8000 * sum(octets) / sum(duration ms)
 *     over eligible records, and a sub-optimal flag when the rate is strictly below a
 *     supplied standard (Sec. III.B.1 "NetPerf Monitoring Thread", Sec. IV.B).
 *
 * Conventions (all calls):
 *   - every call returns a gnm_status and never throws or aborts; on failure
 *     gnm_last_error() holds a message for the calling thread;
 *   - a context is used by one host thread at a time;
 *   - record arrays are owned by the caller and never freed or retained by the library;
 *     device pointers must stay valid until the work queued on the stream has finished;
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream);
 *     work is queued on it and no call synchronises the host unless it returns host
 *     data (gnm_site_stats, gnm_flag_suboptimal, gnm_window_dense and the reports);
 *   - site ids are dense in [0, n_sites); direction 0 = inbound (remote endpoint is the
 *     source), 1 = outbound (remote endpoint is the destination);
 *   - an output array that is too small gives GNM_E_CAPACITY with *n_out set to the
 *     required count.
 */
#ifndef GNM_H
#define GNM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GNM_NO_SITE 0xFFFFFFFFu
#define GNM_NSTAT 6     /* flows, octets, pkts, e_flows, e_octets, e_dur_ms */
#define GNM_MAX_LOCAL 8 /* local-site prefixes */

typedef enum {
    GNM_OK = 0,
    GNM_E_INVAL = 1,    /* bad argument or registry */
    GNM_E_NOMEM = 2,    /* host or device allocation failed */
    GNM_E_CUDA = 3,     /* a CUDA runtime call failed */
    GNM_E_STATE = 4,    /* wrong call order, unknown window id */
    GNM_E_CAPACITY = 5, /* output array too small; *n_out holds the required count */
    GNM_E_TIMEOUT = 6,  /* a bounded device or host wait gave up */
    GNM_E_INTERNAL = 7  /* a device-side consistency check failed */
} gnm_status;

/* Prefix-match methods. BSEARCH: binary search over all range starts (placement below).
 * RMI: the learned index (gnm_rmi_train). RADIX: a directory indexed by the top
 * `radix_bits` address bits -- the paper's direct-indexed site catalog (Sec. III.B.2.1
 * hashes /24 subnets) generalised to any prefix length -- gives each bucket's range
 * interval, and a binary search inside the bucket finishes. HASH24: the paper's own GPU
 * Site Catalog (Sec. III.B.2.1): every registered network expanded into its /24 subnets
 * in a hash table (the longest registered prefix wins each subnet), one probe sequence per
 * lookup; only for registries whose prefixes are all /24 or shorter (GNM_E_INVAL
 * otherwise), and gnm_lookup gives sites but no range positions with it. AUTO: RMI when
 * trained, else BSEARCH when the registry fits shared memory, else RADIX. */
enum { GNM_LOOKUP_AUTO = 0, GNM_LOOKUP_BSEARCH = 1, GNM_LOOKUP_RMI = 2, GNM_LOOKUP_RADIX = 3,
       GNM_LOOKUP_HASH24 = 4 };
/* Where the flattened registry is searched: wholly in shared memory (SMEM), wholly in L2
 * (L2), or STAGED: the first start of every block of 16 ranges in shared memory, the
 * 64-byte blocks of 16 starts and the sites in L2 (two L2 accesses per lookup). With RMI
 * the ranges are always searched in L2 and the placement is that of the learned index's
 * leaf parameters: staged in shared memory (SMEM; GNM_E_INVAL when they do not fit), read
 * from global memory with one 16-byte load per lookup (L2), or AUTO: staged when they fit
 * (up to about 14,000 leaves), else read from global memory. */
enum { GNM_PLACE_AUTO = 0, GNM_PLACE_SMEM = 1, GNM_PLACE_L2 = 2, GNM_PLACE_STAGED = 3 };
enum { GNM_AGG_AUTO = 0, GNM_AGG_DIRECT = 1, GNM_AGG_WARP = 2 };
enum { GNM_ADMIN_OR = 0, GNM_ADMIN_AND = 1 };
/* Per-CTA accumulation: a shared-memory row per key (DIRECT, when all keys fit), a
 * shared-memory hash table of the keys a CTA meets with global atomics for the overflow
 * (HASH), warp-aggregated global atomics only (GLOBAL), or PARTITION (split launches):
 * the records are first regrouped by (window, group of keys that one direct table holds),
 * then every CTA segment meets one group only. AUTO: DIRECT when all keys fit, else
 * PARTITION for split launches of at most 8192 (window, group) buckets, else HASH. */
enum { GNM_TABLE_AUTO = 0, GNM_TABLE_DIRECT = 1, GNM_TABLE_HASH = 2, GNM_TABLE_GLOBAL = 3,
       GNM_TABLE_PARTITION = 4 };
enum { GNM_SPLIT_AUTO = 0, GNM_SPLIT_FUSED = 1, GNM_SPLIT_TWO_KERNELS = 2 };

/* Filters and execution knobs. The paper fixes none of the filter constants
 * (Sec. III.B.2.1 says only "average packet size ... usually small" and "small number
 * of packets with short durations"); the defaults are this library's reading. */
typedef struct {
    uint32_t min_avg_pkt_bytes; /* eligible needs dOctets >= this * dPkts (default 100) */
    uint32_t min_pkts;          /* administrative filter: packets (default 10) */
    uint32_t min_dur_ms;        /* administrative filter: duration (default 1000) */
    uint32_t min_flows_to_flag; /* a key needs this many eligible flows to be flagged (1) */
    int32_t admin_rule;         /* GNM_ADMIN_OR: exclude if few packets OR short (default);
                                   GNM_ADMIN_AND: exclude only if both */
    int32_t lookup_mode;        /* GNM_LOOKUP_*: prefix-match method */
    int32_t placement;          /* GNM_PLACE_*: registry in shared memory or L2 */
    int32_t aggregation;        /* GNM_AGG_*: shared-memory atomics per record, or
                                   warp-aggregated */
    int32_t device;             /* CUDA device ordinal (default 0) */
    uint32_t window_slots;      /* per-window result slots kept on the device (64) */
    double threshold_bps;       /* flag standard used when a window is finalised (1e8) */
    int32_t block_threads;      /* 0: tuned default; else 128..1024, multiple of 32 */
    int32_t ctas_per_sm;        /* 0: tuned default; else 1..8 */
    int32_t unroll;             /* 0: tuned default; else 1 or 2 (4-record groups per
                                   thread per iteration), or 3: one group, the next
                                   group's loads issued before this one is processed
                                   (split launches with direct tables; else 1) */
    int32_t table_mode;         /* GNM_TABLE_*: where a CTA accumulates its sums */
    uint32_t hash_slots;        /* GNM_TABLE_HASH size: 0 = largest that fits, else an
                                   even number in 256..65536 */
    uint32_t radix_bits;        /* GNM_LOOKUP_RADIX directory bits: 0 = sized from the
                                   registry, else 4..16. With the shared-memory placement of
                                   GNM_LOOKUP_BSEARCH: 4..16 = a directory of that many bits in
                                   front of the search (when it fits), 0 = none */
    int32_t split;              /* GNM_SPLIT_*: one fused kernel, or a lookup kernel that
                                   writes a 4-byte key per record followed by the
                                   aggregation kernel (registries outside shared memory) */
    int32_t key_directory;      /* split RADIX lookups: 3 (1) = the key kernel keeps the
                                   first start of every 2-range (4-range) block in shared
                                   memory beside a directory of block indices, and one
                                   16-byte (32-byte) load of the block's (start, site)
                                   pairs ends a lookup; 4 = as 3 with a 16-bit directory
                                   over the top 16 address bits and the blocks' low 16
                                   start bits (fewer than 65,536 blocks; GNM_E_INVAL
                                   otherwise); 2 = the range directory and a search over
                                   L2; 0 = 3, else 1, whichever fits first */
    int32_t host_records;       /* GNM_HOST_*: how kernels get host (on_device = 0) records */
    int32_t rate_stats;         /* per-flow rate statistics per window (gnm_window_rate_stats):
                                   1: each result slot also holds a 10001-bucket histogram per
                                   key (40 KB per key); 2: each result slot logs one 32-bit
                                   (key, bucket) word per eligible flow instead (4 bytes per
                                   record of the window, grown as records arrive), sorted on
                                   the GPU when first read (needs n_sites <= 131,072; a log
                                   that grows synchronises the stream, so do not capture such
                                   calls); both keep 16 bytes per key for the least and
                                   greatest rate. 0: off */
    uint32_t host_capacity;     /* > 0: per-host sums per window (gnm_window_hosts) for up to
                                   this many (remote host, dir) pairs per window; each result
                                   slot holds a table of 2^ceil(log2(2 * capacity)) entries of
                                   56 bytes; launches then run the key kernel first. 0: off */
} gnm_config;

/* Host records: AUTO reads them in place when every array is page-locked host memory that
 * the device can address (cudaHostAlloc / cudaHostRegister; the kernels then read it over
 * the host link, with no staging copy), else STAGE; STAGE copies them to a device staging
 * buffer first; IN_PLACE requires addressable page-locked arrays (GNM_E_INVAL otherwise).
 * PIPELINE (gnm_windows_process of two or more windows): the windows are split into chunks
 * of consecutive windows (about an eighth of the records each, at least 1M records), each
 * chunk is copied to one of two device buffer sets on a stream of the context's own, and
 * processed on the caller's stream as soon as its copy has landed, so that copying a chunk
 * overlaps processing the one before it (meant for host links that copy faster than
 * kernels read through them; on a GB300's NVLink-C2C, AUTO's in-place reads were faster:
 * 7.6 against 5.6 G records/s on the hour workload); other calls stage as STAGE. */
enum { GNM_HOST_AUTO = 0, GNM_HOST_STAGE = 1, GNM_HOST_IN_PLACE = 2, GNM_HOST_PIPELINE = 3 };

/* One struct-of-arrays batch of NetFlow v5 fields (Sec. IV.A.3: 48-byte v5 records; only
 * the six fields below are read). Element i of every array is record i. Device arrays
 * that share the same address modulo 16 bytes are read with 16-byte vector loads; any
 * other 4-byte alignment is read element by element. */
typedef struct {
    uint64_t n;
    const uint32_t *srcaddr, *dstaddr; /* IPv4 addresses, host byte order */
    const uint32_t *dPkts, *dOctets;   /* packets and layer-3 bytes of the flow */
    const uint32_t *first, *last;      /* router uptime (ms) at first / last packet */
    const uint16_t *srcport, *dstport; /* not read; may be NULL */
    const uint8_t *prot;               /* not read; may be NULL */
    int32_t on_device;                 /* 1: device pointers; 0: host pointers (copied
                                          through a library-owned staging buffer) */
} gnm_records;

typedef struct {
    uint32_t site, dir;
    uint64_t flows, octets, pkts, e_flows, e_octets, e_dur_ms;
    double rate_bps; /* NaN when e_dur_ms == 0 */
    uint32_t flag;   /* against the context's threshold_bps */
    uint32_t reserved;
} gnm_site_stat;

typedef struct {
    uint64_t n_ranges;      /* disjoint address ranges after flattening */
    uint64_t n_registered;  /* ranges that carry a site */
    uint32_t n_sites;
    uint32_t n_prefixes;
    int32_t placement;      /* resolved GNM_PLACE_* (binary search) */
    int32_t lookup_mode;    /* resolved GNM_LOOKUP_* */
    int32_t privatized;     /* per-CTA shared-memory sums in use */
    int32_t rmi_ready;
} gnm_registry_info;

typedef struct gnm_ctx gnm_ctx;

/* Fills *cfg with the defaults listed above. */
void gnm_config_default(gnm_config *cfg);

/* Creates a context on cfg->device (NULL cfg = defaults). Owns all device state. */
gnm_status gnm_create(const gnm_config *cfg, gnm_ctx **out);

/* Releases the context and all device memory it owns (synchronises its work). */
void gnm_destroy(gnm_ctx *ctx);

/* Message of the last failure on this thread (empty string if none). */
const char *gnm_last_error(const gnm_ctx *ctx);

/* Registers the collaboration sites' subnets and the local site (Sec. III.B.1 "Site
 * Registration Thread"; the "Site Catalog"). prefix[i]/len[i] is a CIDR block, host
 * order, with site_id[i] < n_sites. Prefixes may nest: an address belongs to the site of
 * the longest prefix that contains it. Rejected with GNM_E_INVAL: len > 32, host bits
 * set, the same (prefix, len) twice, site_id >= n_sites, n_local == 0 or > GNM_MAX_LOCAL,
 * a local prefix that overlaps a registered one. All arrays are host memory and are
 * copied. Replaces any earlier registry (and drops the learned index and all window
 * results). The flattened ranges are uploaded once and stay resident. */
gnm_status gnm_registry_load(gnm_ctx *ctx, const uint32_t *prefix, const uint8_t *len,
                             const uint32_t *site_id, size_t n, uint32_t n_sites,
                             const uint32_t *local_prefix, const uint8_t *local_len,
                             size_t n_local);

gnm_status gnm_registry_info_get(gnm_ctx *ctx, gnm_registry_info *out);

/* The rate step alone (Sec. III.B.1 and Sec. III.B.2.1: a site's transfer rate from its
 * eligible flows' bytes and durations): rate[i] = (e_octets[i] * 8000) / e_dur_ms[i] in bits
 * per second, each operand converted to binary64 and each operation rounded to nearest
 * (ties to even), NaN when e_dur_ms[i] = 0 -- the same bits as the rates the window calls
 * report, for sums gathered elsewhere (e.g. the sums of one site over several windows or
 * GPUs). e_octets, e_dur_ms and rate are device arrays of n entries (8-byte aligned) on the
 * current device, owned by the caller; the kernel is queued on cuda_stream (NULL: the legacy
 * stream) and the call does not wait for it. No context is needed. GNM_E_INVAL for NULL or
 * misaligned arrays (n = 0 accepts anything), GNM_E_CUDA when the launch fails. */
gnm_status gnm_rates(const uint64_t *e_octets, const uint64_t *e_dur_ms, uint64_t n, double *rate,
                     void *cuda_stream);

/* Host-only form of the registry step (no context, no GPU): validates the registry as
 * gnm_registry_load does and writes the flattened ranges (see gnm_registry_ranges).
 * *n_out receives the number of ranges (GNM_E_CAPACITY if cap is smaller). */
gnm_status gnm_registry_flatten(const uint32_t *prefix, const uint8_t *len,
                                const uint32_t *site_id, size_t n, uint32_t n_sites,
                                uint32_t *starts, uint32_t *site, size_t cap, size_t *n_out);

/* Copies the flattened registry to host arrays: starts[i] is the first address of
 * range i (starts[0] = 0, strictly increasing), site[i] its site or GNM_NO_SITE.
 * GNM_E_CAPACITY if cap < n_ranges. */
gnm_status gnm_registry_ranges(gnm_ctx *ctx, uint32_t *starts, uint32_t *site, size_t cap,
                               size_t *n_out);

/* Processes one window (Sec. III.B.1: the NetPerf thread hands a batch of records to the
 * kernels; Sec. III.B.2.1 TransRate Kernel). Results go to the window's device slot
 * (reusing the oldest slot when all are taken) and are finalised (rates, flags) in the
 * same launch. window_id is any caller-chosen key; processing an id again replaces its
 * results. Host records (on_device = 0) are copied on `stream` first. n must be below
 * 2^32 so that the 64-bit sums cannot overflow. */
gnm_status gnm_window_process(gnm_ctx *ctx, const gnm_records *rec, uint64_t window_id,
                              void *stream);

/* Many windows in one launch: window k is records [offsets[k], offsets[k+1]) of the
 * struct-of-arrays `rec` (rec->n >= offsets[n_win]); offsets is host memory,
 * non-decreasing, offsets[0] may be > 0. Each window gets its own slot and is finalised
 * when its last CTA finishes. Empty windows are allowed. */
gnm_status gnm_windows_process(gnm_ctx *ctx, const gnm_records *rec, const uint64_t *offsets,
                               const uint64_t *window_ids, size_t n_win, void *stream);

/* Streaming form of a window: open (zero the sums), add any number of batches, close
 * (finalise). Between open and close the window's sums are partial. */
gnm_status gnm_window_open(gnm_ctx *ctx, uint64_t window_id, void *stream);
gnm_status gnm_window_add(gnm_ctx *ctx, const gnm_records *rec, uint64_t window_id,
                          void *stream);
gnm_status gnm_window_close(gnm_ctx *ctx, uint64_t window_id, void *stream);

/* Checkpoint of an open window (the paper's receiver keeps the period's records on disk
 * until they are processed, Sec. III.B.1; here the state to keep is the window's partial
 * sums). gnm_window_export copies the sums accumulated so far to `rows`: keys rows (keys =
 * 2*n_sites + 4: the site keys site*2+dir, then the four unmatched classes) of GNM_NSTAT
 * uint64 in the gnm_window_dense order (flows, octets, pkts, e_flows, e_octets, e_dur_ms).
 * Synchronous; host memory; the window stays open. gnm_window_import opens `window_id` (as
 * gnm_window_open) with `rows` (n_rows = keys, as exported, possibly by another context over
 * the same registry and filters) as its sums so far; gnm_window_add then continues it and
 * gnm_window_close finalises it exactly as if every record had been added here. Returns
 * when the sums are on the device. Errors: GNM_E_STATE for an unknown, evicted or closed
 * window (export), and in contexts keeping per-flow rate or per-host statistics (those are
 * not carried); GNM_E_CAPACITY when cap < keys (*n_out = keys); GNM_E_INVAL when n_rows !=
 * keys or a row is inconsistent (e_flows > flows, e_octets > octets, flows >= 2^32, or the
 * flows of all rows reach 2^32). */
gnm_status gnm_window_export(gnm_ctx *ctx, uint64_t window_id, uint64_t *rows, size_t cap,
                             size_t *n_out);
gnm_status gnm_window_import(gnm_ctx *ctx, uint64_t window_id, const uint64_t *rows, size_t n_rows,
                             void *stream);

/* Per-site statistics of a window (synchronises with the window's work). Writes the
 * keys with at least one flow, ordered by (site, dir), into out[0..*n_out). unmatched,
 * if not NULL, receives 4 classes x {flows, octets, pkts}: 0 neither endpoint local,
 * 1 both endpoints local, 2 inbound from an unregistered address, 3 outbound to one.
 * GNM_E_STATE for an unknown or evicted window id. */
gnm_status gnm_site_stats(gnm_ctx *ctx, uint64_t window_id, gnm_site_stat *out, size_t cap,
                          size_t *n_out, uint64_t unmatched[12]);

/* Sub-optimal (site, dir) keys of a window: at least min_flows_to_flag eligible flows
 * and rate strictly below threshold_bps (Sec. III.B.1, Sec. IV.B "less than"). Computed
 * on the device against this threshold, compacted, then copied to site_out/dir_out. */
gnm_status gnm_flag_suboptimal(gnm_ctx *ctx, uint64_t window_id, double threshold_bps,
                               uint32_t *site_out, uint8_t *dir_out, size_t cap, size_t *n_out);

/* Per-flow transfer-rate statistics of a finalised window (contexts created with
 * rate_stats = 1 or 2; GNM_E_STATE otherwise). Sec. III.B.2.1: the maximum, minimum and median
 * of the rates of each (site, dir)'s flows, the median from a histogram of 10 kb/s buckets
 * whose last bucket holds every rate from 100 Mb/s up. Over the eligible flows of key
 * site*2+dir, with rate = (double)octets * 8000.0 / (double)duration_ms (one rounding per
 * operation) and bucket = min(10000, floor(4 * octets / (5 * duration_ms))):
 *   rmin[k], rmax[k]     least and greatest rate; NaN without eligible flows
 *   median_bucket[k]     bucket of the ceil(n/2)-th smallest of the key's n rates (the
 *                        lower median): its rate lies in [10 kb/s * b, 10 kb/s * (b+1));
 *                        GNM_NO_MEDIAN without eligible flows
 *   hist[k * 10001 + b]  flows of key k in bucket b (rate_stats = 1 only; must be NULL
 *                        with rate_stats = 2, GNM_E_INVAL otherwise)
 * Arrays have 2*n_sites entries (hist 2*n_sites*10001); each may be NULL. The medians are
 * the same in both modes. */
#define GNM_RATE_BUCKETS 10001u
#define GNM_NO_MEDIAN 0xFFFFFFFFu
gnm_status gnm_window_rate_stats(gnm_ctx *ctx, uint64_t window_id, double *rmin, double *rmax,
                                 uint32_t *median_bucket, uint32_t *hist);

/* The non-empty cells of a finalised window's rate histograms (rate_stats = 1 or 2), in
 * (key, bucket) order: key[i] = site*2+dir, bucket[i] (as in gnm_window_rate_stats),
 * count[i] > 0 flows. *n_out = number of cells; GNM_E_CAPACITY (with *n_out set) when cap
 * is smaller. Host arrays, each may be NULL. */
gnm_status gnm_window_rate_cells(gnm_ctx *ctx, uint64_t window_id, uint32_t *key, uint32_t *bucket,
                                 uint32_t *count, size_t cap, size_t *n_out);

/* Median-rate warnings across windows (Sec. III.B.1, Sec. IV.B: a warning for a site
 * whose median transfer rate stays below a standard, 1 Mb/s, for two consecutive periods).
 * The context keeps a run length per (site, dir) key on the device. Each call takes the
 * next window in time order (finalised, rate_stats = 1): a key whose lower-median bucket
 * is below `below_bucket` (100 for 1 Mb/s) extends its run, any other key -- including one
 * without eligible flows -- restarts at zero. Keys whose run has reached `consecutive`
 * windows are written, ascending, to keys_out (key = site*2+dir; a site is warned about when
 * either direction is); *n_out gets their number (GNM_E_CAPACITY when cap is smaller, the
 * runs being updated all the same). gnm_warnings_reset sets every run to zero. */
gnm_status gnm_warnings_update(gnm_ctx *ctx, uint64_t window_id, uint32_t below_bucket, uint32_t consecutive,
                               uint32_t *keys_out, size_t cap, size_t *n_out);
gnm_status gnm_warnings_reset(gnm_ctx *ctx);
/* The warning runs as host arrays of 2*n_sites u32 (export), or set from them (import):
 * monitoring stopped after some window resumes, in another context over the same registry,
 * with the next window as if it had never stopped. */
gnm_status gnm_warnings_export(gnm_ctx *ctx, uint32_t *runs);
gnm_status gnm_warnings_import(gnm_ctx *ctx, const uint32_t *runs);

/* Per-host sums of a finalised window (contexts with host_capacity > 0; Sec. III.B.2.1:
 * statistics "for each host in a registered site"): one row per remote address of a
 * registered site and direction, with the six sums of a site key and the rate of its
 * eligible flows (as gnm_site_stats), sorted by (site, dir, addr). GNM_E_CAPACITY when cap
 * is smaller than the number of rows (*n_out set), or when the window met more hosts than
 * host_capacity (its rows are then incomplete; *n_out = the rows kept). */
typedef struct {
    uint32_t addr;
    uint32_t site;
    uint32_t dir;
    uint32_t reserved;
    uint64_t flows, octets, pkts, e_flows, e_octets, e_dur_ms;
    double rate_bps;
} gnm_host_stat;
gnm_status gnm_window_hosts(gnm_ctx *ctx, uint64_t window_id, gnm_host_stat *out, size_t cap, size_t *n_out);

/* Dense copies of a window's results to host arrays (each may be NULL):
 * stats[(2*n_sites) x GNM_NSTAT] (row site*2+dir), unmatched[12], rate[2*n_sites],
 * flag[2*n_sites] (against the context threshold). Synchronises with the window. */
gnm_status gnm_window_dense(gnm_ctx *ctx, uint64_t window_id, uint64_t *stats,
                            uint64_t *unmatched, double *rate, uint8_t *flag);

/* The dense results of n windows in one call: window k's arrays start at stats +
 * k*(2*n_sites)*GNM_NSTAT, unmatched + k*12, rate + k*2*n_sites, flag + k*2*n_sites (each
 * may be NULL). One synchronisation for all of them. */
gnm_status gnm_windows_results(gnm_ctx *ctx, const uint64_t *window_ids, size_t n,
                               uint64_t *stats, uint64_t *unmatched, double *rate,
                               uint8_t *flag);

/* gnm_windows_results enqueued on cuda_stream (a cudaStream_t; NULL: the legacy default
 * stream), without waiting. The copies start after each window's last processing. The next
 * processing of these windows (or of the slots they hold) waits for the copies, so results of
 * one batch of windows can be read while another batch is processed. The host arrays are
 * read once the stream is synchronised; they should be page-locked, or the copies are not
 * asynchronous. stats, rate and flag are laid out as in gnm_windows_results. unmatched6
 * holds the unmatched rows as stored: window k's class c in unmatched6[(k*4 + c)*GNM_NSTAT
 * ...], words 0..2 its flows, octets and packets (those gnm_windows_results reports). Errors
 * found by the checked build's device checks surface at the next synchronising call. */
gnm_status gnm_windows_results_async(gnm_ctx *ctx, const uint64_t *window_ids, size_t n,
                                     uint64_t *stats, uint64_t *unmatched6, double *rate,
                                     uint8_t *flag, void *cuda_stream);

/* Device addresses of a window's dense results (same layouts as gnm_window_dense; the
 * stats block has 2*n_sites+4 rows, the last four being the unmatched classes with
 * e_* columns zero). Valid until the slot is reused or the registry is replaced. No
 * synchronisation: order reads after the window's stream. */
gnm_status gnm_window_device(gnm_ctx *ctx, uint64_t window_id, const uint64_t **stats,
                             const double **rate, const uint8_t **flag);

/* Forgets a window id (its slot becomes free). */
gnm_status gnm_window_release(gnm_ctx *ctx, uint64_t window_id);

/* Longest-prefix match of n device addresses: site_out[i] (device, may be NULL) gets the
 * site or GNM_NO_SITE, pos_out[i] (device, may be NULL) the index of the flattened range.
 * Uses the context's lookup mode. */
gnm_status gnm_lookup(gnm_ctx *ctx, const uint32_t *addr, uint64_t n, uint32_t *site_out,
                      uint32_t *pos_out, void *stream);

/* ----------------------------------------------------------------- learned index */

/* Two-stage recursive model index over the flattened range starts (not in the paper;
 * Kraska et al. 2018). It predicts the position of an address; an exact search within
 * [pred - eps_lo, pred + eps_hi] of the leaf finishes the lookup and a full binary search
 * is the fallback whenever that window does not hold the answer, so results never depend
 * on the model.
 *
 * Leaves are fitted by default by minimising their worst-case error over every address
 * they own (GNM_RMI_FIT_MINIMAX: a Chebyshev line over the range pieces of the leaf's
 * address interval, whose positions are the plain binary search's answers), since that
 * error is the proven bound; GNM_RMI_FIT_MSE fits them by gradient descent on the mean
 * squared error of the training lookups instead. With minimax leaves, a leaf whose window
 * would exceed eps_target is split into 2^k equal sub-leaves (one more linear model level
 * for that leaf's addresses only; the hybrid form of Kraska et al.'s index). Models are
 * numbered leaves first (0..n_leaves-1), then the sub-leaves of split leaves in leaf order.
 * Minimax training (root, leaves, splits) is deterministic: the same keys, configuration
 * and GPU give the same model bit for bit. MSE leaves sum with FP64 atomics and may differ
 * in the last bits between runs. */
enum { GNM_RMI_ROOT_LINEAR = 0, GNM_RMI_ROOT_MLP = 1 };
enum { GNM_RMI_FIT_MINIMAX = 0, GNM_RMI_FIT_MSE = 1 };

typedef struct {
    int32_t root_kind;   /* GNM_RMI_ROOT_* */
    uint32_t n_leaves;   /* 1..1048576 (4096) */
    uint32_t hidden;     /* MLP root width: 8, 16 or 32 (32) */
    uint32_t leaf_iters; /* gradient steps for the linear root and for MSE leaves (4) */
    uint32_t mlp_steps;  /* Adam steps for the MLP root (600) */
    uint32_t mlp_batch;  /* samples per Adam step (65536) */
    float mlp_lr;        /* Adam learning rate (0.01) */
    uint32_t seed;       /* initialisation and mini-batch sampling seed */
    int32_t exhaustive_eps; /* 1: error bounds from all 2^32 addresses (default);
                               0: from the training samples only (the verify-and-
                               fall-back path keeps results exact either way) */
    int32_t leaf_fit;       /* GNM_RMI_FIT_MINIMAX (default) or GNM_RMI_FIT_MSE */
    uint32_t eps_target;    /* minimax leaves: a leaf whose window eps_lo + eps_hi is
                               estimated above this is split (64); 0: never split */
    uint32_t max_split_log2; /* at most 2^max_split_log2 sub-leaves per leaf (14, <= 16) */
} gnm_rmi_config;

typedef struct {
    uint64_t n_train;
    double root_loss;             /* mean squared error of the root (leaf units) */
    double leaf_loss;             /* mean squared error of the predicted position over
                                     the training lookups */
    uint32_t eps_max;             /* max over models of eps_lo + eps_hi (window - 1) */
    uint32_t err_max;             /* max over models of max(eps_lo, eps_hi): the largest
                                     |predicted - true position| over all addresses */
    double eps_mean;              /* mean window width eps_lo + eps_hi + 1 over the
                                     training lookups */
    uint32_t empty_leaves;        /* leaves that own no address (minimax) or no training key */
    uint32_t n_models;            /* leaves + sub-leaves */
    uint32_t split_leaves;        /* leaves split into sub-leaves */
    double train_ms, sweep_ms;
} gnm_rmi_report;

void gnm_rmi_config_default(gnm_rmi_config *cfg);

/* Trains the learned index on the GPU from n device addresses `keys` (the lookups the
 * plain binary search answers; their positions are computed by it), then computes the
 * per-leaf error bounds. Contexts whose lookup_mode is GNM_LOOKUP_AUTO use the learned
 * index from then on. Needs fewer than 2^24 ranges. Allocates and frees its own training
 * scratch and synchronises `stream`. */
gnm_status gnm_rmi_train(gnm_ctx *ctx, const uint32_t *keys, uint64_t n,
                         const gnm_rmi_config *cfg, gnm_rmi_report *report, void *stream);

/* Number of lookups since the last reset whose model window missed the answer and fell
 * back to the full binary search (0 when the error bounds hold). */
gnm_status gnm_rmi_violations(gnm_ctx *ctx, uint64_t *count, int reset);

/* Gradient of the mean squared error of one linear stage yhat = w*z + c over n device
 * samples (z float, y float): grad[0] = dL/dw, grad[1] = dL/dc, grad[2] = L (host out).
 * Exposed so the training arithmetic can be checked against an FP64 reference. */
gnm_status gnm_rmi_linear_grad(gnm_ctx *ctx, const float *z, const float *y, uint64_t n,
                               float w, float c, double grad[3], void *stream);

/* Gradient of the mean squared error of the 1 -> H -> 1 ReLU root over n device samples
 * (xn float in [0,1), y float). params (host) = w1[H], b1[H], w2[H], b2; grad (host) has
 * the same layout, followed by the loss. */
gnm_status gnm_rmi_mlp_grad(gnm_ctx *ctx, const float *xn, const float *y, uint64_t n,
                            uint32_t hidden, const float *params, double *grad, void *stream);

/* Copies the trained model to host arrays (any may be NULL; call once with NULL arrays to
 * read the sizes): root[2 + 3*32 + 1] (ra, rb, w1[32], b1[32], w2[32], b2);
 * split[n_leaves]: 0 for a leaf that is not split, else ((count - 1) << 8) | shift: the
 * leaf's addresses [F, F') go to `count` sub-leaves of 2^shift addresses each from F (the
 * last one takes the remainder), address x to sub-leaf min((x - F) >> shift, count - 1);
 * a/b/x0/eps_lo/eps_hi[n_models] per model (zeros for split leaves). Position of x in
 * model m: clamp(floor(fl(fl(a[m] * fl(x - x0[m])) + b[m])), 0, n_ranges - 1). */
gnm_status gnm_rmi_export(gnm_ctx *ctx, int32_t *root_kind, uint32_t *n_leaves, uint32_t *n_models,
                          float *root, uint32_t *split, float *a, float *b, uint32_t *x0,
                          uint32_t *eps_lo, uint32_t *eps_hi);

/* Installs a model (same layout as gnm_rmi_export; split may be NULL when no leaf is
 * split, and n_models must then equal n_leaves) and computes its error bounds by the
 * exhaustive sweep over all 2^32 addresses. GNM_E_INVAL when the split table does not add
 * up to n_models, a count exceeds 65,536 or a shift exceeds 31. */
gnm_status gnm_rmi_import(gnm_ctx *ctx, int32_t root_kind, uint32_t n_leaves, uint32_t n_models,
                          const float *root, const uint32_t *split, const float *a, const float *b,
                          const uint32_t *x0, void *stream);

/* ------------------------------------------------------- batched plans and tuning */

typedef struct gnm_plan gnm_plan;

/* A reusable launch of gnm_windows_process over fixed device buffers and window shapes,
 * captured once into a CUDA graph: the per-record key kernel (registries outside shared
 * memory), the persistent aggregation kernel and, for registries of more than 4096 keys,
 * the per-window finalisation kernel. The record buffers and window shapes stay fixed;
 * their contents may change between launches. */
gnm_status gnm_plan_create(gnm_ctx *ctx, const gnm_records *rec, const uint64_t *offsets,
                           const uint64_t *window_ids, size_t n_win, gnm_plan **out);

/* gnm_plan_create with flags. GNM_PLAN_KERNEL_TIMES adds timing events between the
 * graph's kernels (a few microseconds per launch), read by gnm_plan_kernel_times. */
#define GNM_PLAN_KERNEL_TIMES 1u
gnm_status gnm_plan_create_ex(gnm_ctx *ctx, const gnm_records *rec, const uint64_t *offsets,
                              const uint64_t *window_ids, size_t n_win, uint32_t flags, gnm_plan **out);
gnm_status gnm_plan_launch(gnm_plan *plan, void *stream);

/* Kernels of a plan's launch, in order */
typedef enum { GNM_KERNEL_KEYS = 0, GNM_KERNEL_AGGREGATE = 1, GNM_KERNEL_FINALIZE = 2, GNM_KERNEL_PART_COUNT = 3,
               GNM_KERNEL_PART_SCAN = 4, GNM_KERNEL_PART_SCATTER = 5, GNM_KERNEL_HOSTS = 6 } gnm_kernel_kind;

/* Device durations (ms, CUDA events) of each kernel of the plan's last launch, which it
 * waits for; kind[i] names kernel i. *n_out = the plan's kernel count (GNM_E_CAPACITY
 * if cap is smaller); GNM_E_STATE for a plan created without GNM_PLAN_KERNEL_TIMES or
 * never launched. */
gnm_status gnm_plan_kernel_times(gnm_plan *plan, float *ms, int32_t *kind, size_t cap, size_t *n_out);
void gnm_plan_destroy(gnm_plan *plan);

typedef struct {
    int32_t block_threads, ctas_per_sm, unroll, aggregation, placement;
    double best_ms, default_ms;
    uint32_t n_tried;
    uint32_t radix_bits;
    int32_t split;
    int32_t key_directory;
    int32_t keys_unroll;      /* key kernel: groups of 4 records per thread and step */
    /* the fastest candidate of each aggregation (index GNM_AGG_DIRECT, GNM_AGG_WARP; 0 where
     * none of that aggregation ran): per-lane shared-memory atomics against one atomic per
     * distinct key of a warp after __match_any_sync */
    double best_ms_by_agg[3];
} gnm_tune_report;

/* Times candidate launch shapes (block size, CTAs per SM, records per thread,
 * aggregation, registry placement or radix directory bits, fused or split launches, key
 * kernel directory) on these windows with CUDA events, keeps the fastest in the context
 * and reports it. Results of the windows are those of the last run. */
gnm_status gnm_autotune(gnm_ctx *ctx, const gnm_records *rec, const uint64_t *offsets,
                        const uint64_t *window_ids, size_t n_win, gnm_tune_report *report);

/* Number of kernels the last processing call enqueued (for launch accounting). */
uint32_t gnm_last_launch_count(const gnm_ctx *ctx);

/* ------------------------------------------------------------------- serving */

/* A streaming front end over one context. In the paper a receiver thread buffers arriving
 * records in host memory and the monitoring thread hands each period's buffer to the GPU
 * at once (Sec. III.B.1 "FlowData Receiver Thread", "NetPerf Monitoring Thread"); here
 * batches go to the GPU as they arrive and are added to per-window device state, and a
 * window's rates and flags (Sec. III.B.2.1) are final once its closing batch is processed.
 *
 * Admission: the records of admitted, unfinished batches (24 bytes each) never exceed
 * budget_bytes. Host batches in page-locked, device-mapped memory are read in place by the
 * kernels over the host link when the context's host_records is AUTO or IN_PLACE (no copy,
 * no arena space); other host batches are copied into a device arena of budget_bytes owned
 * by the server (IN_PLACE refuses them with GNM_E_INVAL); device batches only count
 * against the budget. A batch that does not fit waits
 * in a FIFO queue; a window's first batch also waits while every result slot is held by
 * an open window (later batches of open windows pass it). Queued batches are admitted in
 * gnm_stream_submit and gnm_stream_poll as earlier batches finish (continuous batching).
 * Each admitted batch is copied (if staged) and processed on the next of n_cuda_streams
 * CUDA streams, so the copies of some batches overlap the kernels of others; the kernels of
 * one window run in submission order, those of different windows overlap. The caller keeps
 * a host batch's arrays unchanged until its window is reported.
 *
 * Window latency = host time from the gnm_stream_submit call that closes the window to
 * the completion of its finalisation on the device (a host callback queued after it).
 * Results of a reported window are read with gnm_window_dense / gnm_site_stats /
 * gnm_flag_suboptimal on the context. A closed window keeps its result slot until the
 * gnm_stream_submit or gnm_stream_poll call after the poll that reported it; from then on
 * the context may reuse the slot for a newer window (oldest first).
 *
 * Threads: the server and its context are used from one host thread at a time; no other
 * call may process windows on the context while the server is open. Host arrays of a
 * batch must stay valid until gnm_stream_poll has reported its window. */
typedef struct gnm_stream gnm_stream;

typedef struct {
    uint64_t budget_bytes;    /* device bytes of records in flight (default 4 GiB) */
    uint32_t n_cuda_streams;  /* CUDA streams batches are spread over (default 4, 1..64) */
    uint32_t max_queued;      /* queued batches before submit returns GNM_E_CAPACITY (65536) */
    uint64_t max_batch_records; /* largest batch expected: the context's launch scratch is
                                   reserved for it at open, so that no allocation falls
                                   between batches (default 1,048,576; larger batches still
                                   work and grow it) */
} gnm_stream_config;

typedef struct {
    uint64_t window_id;
    uint64_t records;         /* records added to the window */
    double latency_ms;        /* closing submit -> rates and flags final */
    int32_t status;           /* GNM_OK, or the first error of the window's work */
    int32_t reserved;
    double queued_ms;         /* closing submit -> its finalisation enqueued (the part of the
                                 latency spent on the host: admission queue, submission) */
} gnm_window_done;

typedef struct {
    uint64_t batches;             /* submitted */
    uint64_t batches_queued;      /* not admitted by the submit call that brought them */
    uint64_t records;             /* submitted */
    uint64_t windows_closed;
    uint64_t windows_done;
    uint64_t inflight_bytes;      /* now: admitted batches not yet finished on the GPU */
    uint64_t peak_inflight_bytes; /* never above budget_bytes */
    double p50_ms, p99_ms, max_ms, mean_ms;  /* window latency over the windows done */
} gnm_stream_stats;

void gnm_stream_config_default(gnm_stream_config *cfg);

/* Opens a server on ctx, which must hold a registry. Allocates the arena (budget_bytes of
 * device memory) and the streams: GNM_E_NOMEM / GNM_E_CUDA if that fails. */
gnm_status gnm_stream_open(gnm_ctx *ctx, const gnm_stream_config *cfg, gnm_stream **out);

/* Submits a batch of records (host or device SoA, fields as in gnm_window_process) for
 * window `window_id`. The first batch of a window opens it; close_window = 1 closes the
 * window after this batch (n = 0 closes it with no records). Errors: GNM_E_INVAL for a
 * batch above the budget or malformed arrays, GNM_E_STATE for a batch of a window whose
 * close was already submitted, GNM_E_CAPACITY when the batch cannot be admitted now and
 * max_queued batches are waiting already (the batch is then not taken). */
gnm_status gnm_stream_submit(gnm_stream *s, const gnm_records *batch, uint64_t window_id,
                             int close_window);

/* Submits n_batches batches that are slices of one record pool (host or device):
 * batch i = records [begin[i], begin[i] + count[i]) of `pool` for window wids[i], closing it
 * when close_flags[i] (close_flags may be NULL: none close). The batches are taken in order
 * as by gnm_stream_submit; at the first error it stops and returns it, *n_accepted holding
 * the batches taken. Host pool arrays must stay valid until their windows are reported. */
gnm_status gnm_stream_submit_many(gnm_stream *s, const gnm_records *pool, const uint64_t *begin,
                                  const uint64_t *count, const uint64_t *window_ids, const uint8_t *close_flags,
                                  size_t n_batches, size_t *n_accepted);

/* Admits what fits and reports up to cap windows completed since the last report
 * (*n_out set; more stay for the next call). wait_all = 1 first waits until every
 * submitted batch is processed and every closed window is done, or until the batches
 * left wait for result slots held by the windows this call reports (call again after
 * reading them); GNM_E_STATE when they wait for slots that only closing an open window
 * frees. A failed window is reported with its error and has no results. */
gnm_status gnm_stream_poll(gnm_stream *s, gnm_window_done *out, size_t cap, size_t *n_out,
                           int wait_all);

gnm_status gnm_stream_stats_get(gnm_stream *s, gnm_stream_stats *out);

/* Waits for the work in flight, drops batches still queued, releases the server's memory
 * and streams. Windows left open stay open (unpinned) in the context. */
void gnm_stream_close(gnm_stream *s);

/* ------------------------------------------------------------ without allocation */

/* ------------------------------------------------------------- checked build */

/* The library is also built with device-side bounds checks (libgnm_checked.so, same ABI;
 * not in the paper). Its kernels test every index where they trust data -- a record's key
 * before the table, accumulator and histogram accesses it drives; a registry search's
 * starting window before its loads; a learned-index model number; a regrouping bucket
 * and position; a partial-sum block -- and on a failure skip the access and record the
 * first failure in the context's error word. Readouts (gnm_window_dense,
 * gnm_windows_results, gnm_site_stats, gnm_flag_suboptimal) then return GNM_E_INTERNAL
 * naming the check. The default build has no checks and never reports through this word. */

/* 1 in the checked build, 0 in the default one. */
int gnm_checked_build(void);

/* Synchronises the device, returns the context's error word in *word (may be NULL; top
 * byte = check, low 56 bits = the offending value; 0 = no failure), clears it, and returns
 * GNM_E_INTERNAL when it was set (always GNM_OK in the default build). */
gnm_status gnm_device_checks(gnm_ctx *ctx, uint64_t *word);

/* Checked build only (GNM_E_STATE in the default build): overwrites one value of the
 * context's device state from the host, so tests can show that a corrupt index is caught
 * without any access out of bounds. GNM_DEBUG_RMI_SPLIT_BASE: the first-sub-leaf number of
 * split leaf `index` of the learned index becomes `value`. */
enum { GNM_DEBUG_RMI_SPLIT_BASE = 1 };
gnm_status gnm_debug_corrupt(gnm_ctx *ctx, int32_t what, uint32_t index, uint32_t value);

/* Largest n_sites gnm_window_process_noalloc accepts (its fixed scratch is 1 MiB). */
#define GNM_NOALLOC_MAX_SITES 13102u

/* One window, as gnm_window_process computes it, for callers that cannot call cudaMalloc:
 * a process whose device memory is held up front by another allocator (a framework's
 * caching allocator, a fixed budget), or a latency-critical loop that cannot afford
 * cudaMalloc's implicit device synchronisation. The paper has no counterpart to this call.
 * It needs no context and allocates nothing: the caller owns every input and output, and
 * the kernel's scratch (window descriptor, finalise ticket, per-key partial sums) is one
 * fixed 1 MiB array in the library's device image, which every GPU that loads the library
 * keeps until the process exits -- hence n_sites <= GNM_NOALLOC_MAX_SITES (GNM_E_INVAL with
 * a message beyond it). The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress), and so does the first call after the device's context changed
 * (cudaDeviceReset, a new primary context); make those calls before any stream capture.
 * All calls on a device share the one array and clear it before use: calls that overlap
 * on the GPU (other streams, other host threads) race on it and must not be issued.
 * Arguments: cfg (host; NULL = defaults; filters and threshold_bps apply), starts/site
 * (device, n_ranges entries: the flattened registry, e.g. gnm_registry_flatten's output
 * copied to the device; a range whose site id is GNM_NO_SITE or at least n_sites counts as
 * unregistered), n_sites, the local prefixes (host), rec (device records,
 * n < 2^32), and the device results stats[(2*n_sites+4) x GNM_NSTAT] (layout of
 * gnm_window_device), rate[2*n_sites], flag[2*n_sites]. Work is queued on `stream`; the
 * call does not synchronise the host. */
gnm_status gnm_window_process_noalloc(const gnm_config *cfg, const uint32_t *starts,
                                      const uint32_t *site, uint32_t n_ranges, uint32_t n_sites,
                                      const uint32_t *local_prefix, const uint8_t *local_len,
                                      size_t n_local, const gnm_records *rec, uint64_t *stats,
                                      double *rate, uint8_t *flag, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GNM_H */
