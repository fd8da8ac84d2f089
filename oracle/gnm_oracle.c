/*
 * gnm_oracle.c -- plain, slow, obviously correct CPU definition of the G-NetMon
 * flow-analysis hot path (Wu et al., "G-NetMon: A GPU-accelerated Network Performance
 * Monitoring System for Large Scale Scientific Collaborations").
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. It shares no code, header, table or helper
 * with the CUDA library; the two meet only through the seeded input generator.
 *
 * What it computes, per window of flow records (Sec. III.B.1 "NetPerf Monitoring
 * Thread", Sec. III.B.2.1 "TransRate Kernel"):
 *   1. direction of each record from the local-site prefixes (a record between the
 *      local site and another site is recognised by its source or destination address);
 *   2. the site of the remote endpoint by longest-prefix match against the registered
 *      subnets (Sec. III.B.1 "Site Registration Thread"; nested prefixes resolve to the
 *      longest one);
 *   3. the two record filters of Sec. III.B.2.1: reverse-path pure-ACK records (small
 *      average packet size) and short administrative records (few packets, short
 *      duration) are excluded from the transfer-rate calculation;
 *   4. per (site, direction) unsigned 64-bit sums of flows, octets and packets of all
 *      records, and of flows, octets and durations of the eligible ones;
 *   5. the per-site transfer rate (bits per second over the eligible records) and the
 *      sub-optimal flag "rate below a supplied standard" (Sec. III, Sec. IV.B).
 *
 * Two prefix matchers are given, deliberately different algorithms:
 *   - orc_lpm_scan: the paper's "non-hash-table" sequential search over every
 *     registered subnet (Sec. IV.A.1), extended to keep the longest match;
 *   - orc_lpm_lookup: one hash table per prefix length, probed from the longest length
 *     down (the paper's hash-table idea, Sec. III.B.2.1 "Catalog Kernel", generalised
 *     from /24 entries to every length).
 *
 * Readings where the paper is silent (also listed in the design notes):
 *   - site rate = 8000 * sum(eligible octets) / sum(eligible duration ms): the
 *     aggregate form of the per-flow rate bytes*8/duration;
 *   - eligible <=> dur > 0, dOctets >= min_avg_pkt_bytes * dPkts (average packet size
 *     test without division), and the administrative test, which by default excludes a
 *     record with dPkts < min_pkts OR dur < min_dur_ms (admin_rule 0); admin_rule 1
 *     excludes only records with both;
 *   - dur = (uint32)(Last - First), i.e. modulo 2^32 (router uptime wraps);
 *   - flag <=> e_flows >= min_flows_to_flag and rate < threshold (strict, NaN never).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -pthread.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NO_SITE 0xFFFFFFFFu
#define ORC_NSTAT 6 /* flows, octets, pkts, e_flows, e_octets, e_dur_ms */

/* network mask of a prefix length; mask(0) = 0, no shift by 32 */
static uint32_t orc_mask(unsigned len) { return len == 0 ? 0u : (0xFFFFFFFFu << (32u - len)); }

/* ---------------------------------------------------------------- sequential search */

/* Longest-prefix match by scanning every registered prefix (Sec. IV.A.1 sequential
 * search). Ties cannot occur because a (prefix, length) pair appears at most once. */
static uint32_t orc_scan_one(const uint32_t *pfx, const uint8_t *len, const uint32_t *site,
                             size_t n_pfx, uint32_t x) {
    int best_len = -1;
    uint32_t best = ORC_NO_SITE;
    for (size_t i = 0; i < n_pfx; i++) {
        if ((x & orc_mask(len[i])) == pfx[i] && (int)len[i] > best_len) {
            best_len = len[i];
            best = site[i];
        }
    }
    return best;
}

void orc_lpm_scan(const uint32_t *pfx, const uint8_t *len, const uint32_t *site, size_t n_pfx,
                  const uint32_t *x, size_t n, uint32_t *out) {
    for (size_t k = 0; k < n; k++) out[k] = orc_scan_one(pfx, len, site, n_pfx, x[k]);
}

/* ------------------------------------------------------- per-length hash tables */

typedef struct {
    uint32_t cap;   /* power of two, 0 if the length is absent */
    uint32_t *key;  /* masked network address */
    uint32_t *val;  /* site id */
    uint8_t *used;
} orc_table;

typedef struct orc_lpm {
    orc_table t[33];
    int lens_desc[33]; /* lengths present, longest first */
    int n_lens;
    /* the raw registry, kept for the sequential-search variant */
    uint32_t *pfx, *site;
    uint8_t *len;
    size_t n;
} orc_lpm;

static uint32_t orc_hash(uint32_t k, uint32_t cap) {
    /* multiplicative hashing, then fold to the table size */
    uint32_t h = k * 2654435761u;
    h ^= h >> 16;
    return h & (cap - 1u);
}

void orc_lpm_free(orc_lpm *m) {
    if (!m) return;
    for (int l = 0; l <= 32; l++) {
        free(m->t[l].key);
        free(m->t[l].val);
        free(m->t[l].used);
    }
    free(m->pfx);
    free(m->site);
    free(m->len);
    free(m);
}

/* Builds the matcher. Returns NULL and sets *err: 1 length > 32, 2 host bits set,
 * 3 the same (prefix, length) twice, 4 out of memory. */
orc_lpm *orc_lpm_build(const uint32_t *pfx, const uint8_t *len, const uint32_t *site, size_t n,
                       int *err) {
    *err = 0;
    orc_lpm *m = (orc_lpm *)calloc(1, sizeof(orc_lpm));
    if (!m) { *err = 4; return NULL; }
    size_t cnt[33] = {0};
    for (size_t i = 0; i < n; i++) {
        if (len[i] > 32) { *err = 1; orc_lpm_free(m); return NULL; }
        if ((pfx[i] & ~orc_mask(len[i])) != 0) { *err = 2; orc_lpm_free(m); return NULL; }
        cnt[len[i]]++;
    }
    for (int l = 0; l <= 32; l++) {
        if (!cnt[l]) continue;
        uint32_t cap = 16;
        while (cap < 2 * cnt[l]) cap <<= 1;
        m->t[l].cap = cap;
        m->t[l].key = (uint32_t *)calloc(cap, sizeof(uint32_t));
        m->t[l].val = (uint32_t *)calloc(cap, sizeof(uint32_t));
        m->t[l].used = (uint8_t *)calloc(cap, 1);
        if (!m->t[l].key || !m->t[l].val || !m->t[l].used) { *err = 4; orc_lpm_free(m); return NULL; }
    }
    for (size_t i = 0; i < n; i++) {
        orc_table *t = &m->t[len[i]];
        uint32_t h = orc_hash(pfx[i], t->cap);
        while (t->used[h]) {
            if (t->key[h] == pfx[i]) { *err = 3; orc_lpm_free(m); return NULL; }
            h = (h + 1) & (t->cap - 1);
        }
        t->used[h] = 1;
        t->key[h] = pfx[i];
        t->val[h] = site[i];
    }
    m->n_lens = 0;
    for (int l = 32; l >= 0; l--)
        if (cnt[l]) m->lens_desc[m->n_lens++] = l;
    m->n = n;
    m->pfx = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    m->site = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    m->len = (uint8_t *)malloc(n ? n : 1);
    if (!m->pfx || !m->site || !m->len) { *err = 4; orc_lpm_free(m); return NULL; }
    if (n) {
        memcpy(m->pfx, pfx, n * sizeof(uint32_t));
        memcpy(m->site, site, n * sizeof(uint32_t));
        memcpy(m->len, len, n);
    }
    return m;
}

/* Probe the present lengths from longest to shortest; the first hit is the longest
 * matching prefix. */
static uint32_t orc_hash_one(const orc_lpm *m, uint32_t x) {
    for (int j = 0; j < m->n_lens; j++) {
        int l = m->lens_desc[j];
        const orc_table *t = &m->t[l];
        uint32_t k = x & orc_mask((unsigned)l);
        uint32_t h = orc_hash(k, t->cap);
        while (t->used[h]) {
            if (t->key[h] == k) return t->val[h];
            h = (h + 1) & (t->cap - 1);
        }
    }
    return ORC_NO_SITE;
}

void orc_lpm_lookup(const orc_lpm *m, const uint32_t *x, size_t n, uint32_t *out) {
    for (size_t k = 0; k < n; k++) out[k] = orc_hash_one(m, x[k]);
}

/* Disjoint ranges by definition: the set of prefixes containing an address changes only
 * at a prefix's first address or one past its last, so the LPM site is constant between
 * consecutive such boundaries. Writes the sorted range starts (first = 0) and the site of
 * each range (ORC_NO_SITE for gaps), merging neighbours with equal sites. Returns the
 * number of ranges, or -(needed) if cap is too small. */
static int orc_cmp_u32(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

long long orc_flatten(const orc_lpm *m, uint32_t *starts, uint32_t *site_out, size_t cap) {
    size_t nb = 1 + 2 * m->n;
    uint32_t *b = (uint32_t *)malloc(nb * sizeof(uint32_t));
    if (!b) return 0;
    size_t k = 0;
    b[k++] = 0;
    for (size_t i = 0; i < m->n; i++) {
        b[k++] = m->pfx[i];
        uint64_t end = (uint64_t)m->pfx[i] + ((uint64_t)1 << (32 - m->len[i]));
        if (end < ((uint64_t)1 << 32)) b[k++] = (uint32_t)end;
    }
    qsort(b, k, sizeof(uint32_t), orc_cmp_u32);
    size_t out = 0;
    uint32_t prev_site = 0;
    for (size_t i = 0; i < k; i++) {
        if (i > 0 && b[i] == b[i - 1]) continue;
        uint32_t s = orc_hash_one(m, b[i]);
        if (out > 0 && s == prev_site) continue;
        if (out < cap) { starts[out] = b[i]; site_out[out] = s; }
        out++;
        prev_site = s;
    }
    free(b);
    return out <= cap ? (long long)out : -(long long)out;
}

/* ------------------------------------------------------------------- window */

typedef struct {
    const uint32_t *local_pfx;
    const uint8_t *local_len;
    size_t n_local;
    uint32_t n_sites;
    uint32_t min_avg_pkt_bytes, min_pkts, min_dur_ms;
    int admin_rule;
    int use_scan; /* 1: sequential search instead of the hash tables */
} orc_params;

static int orc_is_local(const orc_params *p, uint32_t a) {
    for (size_t i = 0; i < p->n_local; i++)
        if ((a & orc_mask(p->local_len[i])) == p->local_pfx[i]) return 1;
    return 0;
}

/* Record eligibility for the transfer-rate calculation (Sec. III.B.2.1). */
static int orc_eligible(const orc_params *p, uint32_t pkts, uint32_t octets, uint32_t dur) {
    if (dur == 0) return 0;
    /* average packet size octets/pkts >= min_avg, written without division */
    if ((uint64_t)octets < (uint64_t)p->min_avg_pkt_bytes * (uint64_t)pkts) return 0;
    int few_pkts = pkts < p->min_pkts;
    int short_dur = dur < p->min_dur_ms;
    if (p->admin_rule == 0) return !(few_pkts || short_dur);
    return !(few_pkts && short_dur);
}

/* stats: (2*n_sites) rows of ORC_NSTAT u64, row = site*2 + dir (dir 0 inbound, 1
 * outbound). unmatched: 4 classes x {flows, octets, pkts}: 0 neither endpoint local,
 * 1 both local, 2 inbound remote unregistered, 3 outbound remote unregistered.
 * Both arrays are accumulated into (the caller zeroes them). */
static void orc_window_range(const orc_params *p, const orc_lpm *m, const uint32_t *src,
                             const uint32_t *dst, const uint32_t *pkts, const uint32_t *octets,
                             const uint32_t *first, const uint32_t *last, size_t lo, size_t hi,
                             uint64_t *stats, uint64_t *unmatched) {
    for (size_t i = lo; i < hi; i++) {
        int sl = orc_is_local(p, src[i]);
        int dl = orc_is_local(p, dst[i]);
        uint64_t *row = NULL;
        int cls = -1;
        uint32_t dur = last[i] - first[i];
        if (sl && !dl) {          /* outbound: remote is the destination */
            uint32_t s = p->use_scan ? orc_scan_one(m->pfx, m->len, m->site, m->n, dst[i])
                                     : orc_hash_one(m, dst[i]);
            if (s == ORC_NO_SITE) cls = 3;
            else row = stats + ((size_t)s * 2 + 1) * ORC_NSTAT;
        } else if (dl && !sl) {   /* inbound: remote is the source */
            uint32_t s = p->use_scan ? orc_scan_one(m->pfx, m->len, m->site, m->n, src[i])
                                     : orc_hash_one(m, src[i]);
            if (s == ORC_NO_SITE) cls = 2;
            else row = stats + ((size_t)s * 2 + 0) * ORC_NSTAT;
        } else {
            cls = sl ? 1 : 0;
        }
        if (cls >= 0) {
            unmatched[cls * 3 + 0] += 1;
            unmatched[cls * 3 + 1] += octets[i];
            unmatched[cls * 3 + 2] += pkts[i];
            continue;
        }
        row[0] += 1;
        row[1] += octets[i];
        row[2] += pkts[i];
        if (orc_eligible(p, pkts[i], octets[i], dur)) {
            row[3] += 1;
            row[4] += octets[i];
            row[5] += dur;
        }
    }
}

int orc_window(const orc_lpm *m, const uint32_t *local_pfx, const uint8_t *local_len,
               size_t n_local, uint32_t n_sites, uint32_t min_avg_pkt_bytes, uint32_t min_pkts,
               uint32_t min_dur_ms, int admin_rule, int use_scan, const uint32_t *src,
               const uint32_t *dst, const uint32_t *pkts, const uint32_t *octets,
               const uint32_t *first, const uint32_t *last, size_t n, uint64_t *stats,
               uint64_t *unmatched) {
    orc_params p = {local_pfx, local_len, n_local, n_sites, min_avg_pkt_bytes, min_pkts,
                    min_dur_ms, admin_rule, use_scan};
    memset(stats, 0, (size_t)n_sites * 2 * ORC_NSTAT * sizeof(uint64_t));
    memset(unmatched, 0, 12 * sizeof(uint64_t));
    orc_window_range(&p, m, src, dst, pkts, octets, first, last, 0, n, stats, unmatched);
    return 0;
}

/* Same result computed by n_threads POSIX threads over contiguous record slices, each
 * with private sums that are then added (integer addition is order-free). */
typedef struct {
    const orc_params *p;
    const orc_lpm *m;
    const uint32_t *src, *dst, *pkts, *octets, *first, *last;
    size_t lo, hi;
    uint64_t *stats, *unmatched;
} orc_job;

static void *orc_job_run(void *arg) {
    orc_job *j = (orc_job *)arg;
    orc_window_range(j->p, j->m, j->src, j->dst, j->pkts, j->octets, j->first, j->last, j->lo,
                     j->hi, j->stats, j->unmatched);
    return NULL;
}

int orc_window_mt(const orc_lpm *m, const uint32_t *local_pfx, const uint8_t *local_len,
                  size_t n_local, uint32_t n_sites, uint32_t min_avg_pkt_bytes, uint32_t min_pkts,
                  uint32_t min_dur_ms, int admin_rule, const uint32_t *src, const uint32_t *dst,
                  const uint32_t *pkts, const uint32_t *octets, const uint32_t *first,
                  const uint32_t *last, size_t n, uint64_t *stats, uint64_t *unmatched,
                  int n_threads) {
    if (n_threads < 1) n_threads = 1;
    orc_params p = {local_pfx, local_len, n_local, n_sites, min_avg_pkt_bytes, min_pkts,
                    min_dur_ms, admin_rule, 0};
    size_t rows = (size_t)n_sites * 2 * ORC_NSTAT;
    uint64_t *priv = (uint64_t *)calloc((size_t)n_threads * (rows + 12), sizeof(uint64_t));
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    orc_job *jobs = (orc_job *)malloc(sizeof(orc_job) * (size_t)n_threads);
    if (!priv || !th || !jobs) { free(priv); free(th); free(jobs); return -1; }
    for (int t = 0; t < n_threads; t++) {
        orc_job *j = &jobs[t];
        j->p = &p; j->m = m;
        j->src = src; j->dst = dst; j->pkts = pkts; j->octets = octets;
        j->first = first; j->last = last;
        j->lo = n * (size_t)t / (size_t)n_threads;
        j->hi = n * (size_t)(t + 1) / (size_t)n_threads;
        j->stats = priv + (size_t)t * (rows + 12);
        j->unmatched = j->stats + rows;
        pthread_create(&th[t], NULL, orc_job_run, j);
    }
    memset(stats, 0, rows * sizeof(uint64_t));
    memset(unmatched, 0, 12 * sizeof(uint64_t));
    for (int t = 0; t < n_threads; t++) {
        pthread_join(th[t], NULL);
        for (size_t r = 0; r < rows; r++) stats[r] += jobs[t].stats[r];
        for (int r = 0; r < 12; r++) unmatched[r] += jobs[t].unmatched[r];
    }
    free(priv); free(th); free(jobs);
    return 0;
}

/* --------------------------------------------------------------- rate and flag */

/* rate = (octets * 8 bits) / (duration ms / 1000) in bits per second, evaluated as
 * ((double)e_octets * 8000.0) / (double)e_dur_ms, each operation rounded to nearest;
 * NaN when no eligible duration was seen. */
void orc_rates(const uint64_t *stats, size_t n_keys, double *rate) {
    for (size_t k = 0; k < n_keys; k++) {
        uint64_t eo = stats[k * ORC_NSTAT + 4], ed = stats[k * ORC_NSTAT + 5];
        if (ed == 0) { rate[k] = NAN; continue; }
        double num = (double)eo * 8000.0;
        rate[k] = num / (double)ed;
    }
}

/* A key is sub-optimal when it has at least min_flows eligible flows and its rate is
 * strictly below the threshold (Sec. III.B.1, Sec. IV.B "less than"). */
void orc_flags(const uint64_t *stats, const double *rate, size_t n_keys, double threshold,
               uint32_t min_flows, uint8_t *flag) {
    for (size_t k = 0; k < n_keys; k++) {
        uint64_t ef = stats[k * ORC_NSTAT + 3];
        flag[k] = (ef >= (uint64_t)min_flows && rate[k] < threshold) ? 1 : 0;
    }
}

/* ------------------------------------------------------------- median (next) */

/* Per-flow rate bucket of the paper's median histogram (Sec. III.B.2.1): bucket n holds
 * rates in [n*10 kb/s, (n+1)*10 kb/s), rates above 100 Mb/s go to the last bucket 10000.
 * rate = 8000*o/dur b/s, so n = floor(8000*o / (dur*10000)) = floor(4*o / (5*dur)). */
uint32_t orc_rate_bucket(uint32_t octets, uint32_t dur) {
    uint64_t n = ((uint64_t)octets * 4u) / ((uint64_t)dur * 5u);
    return n > 10000u ? 10000u : (uint32_t)n;
}

/* Per-flow transfer-rate statistics of a window (Sec. III.B.2.1: maximum, minimum and
 * median of the rates of each site's flows; the median from the 10001-bucket histogram).
 * Over the eligible flows of each key (site*2 + dir, as in orc_window):
 *   hist[key * 10001 + b]  flows whose rate falls in bucket b (orc_rate_bucket)
 *   rmin[key], rmax[key]   least and greatest (double)octets * 8000.0 / (double)dur,
 *                          NaN when the key has no eligible flow
 *   med[key]               the bucket holding the ceil(n/2)-th smallest of the key's n
 *                          rates (the lower median), 0xFFFFFFFF when n = 0
 * Records of unmatched classes carry no rate statistics. */
int orc_rate_stats(const orc_lpm *m, const uint32_t *local_pfx, const uint8_t *local_len,
                   size_t n_local, uint32_t n_sites, uint32_t min_avg_pkt_bytes, uint32_t min_pkts,
                   uint32_t min_dur_ms, int admin_rule, const uint32_t *src, const uint32_t *dst,
                   const uint32_t *pkts, const uint32_t *octets, const uint32_t *first,
                   const uint32_t *last, size_t n, uint32_t *hist, double *rmin, double *rmax,
                   uint32_t *med) {
    orc_params p = {local_pfx, local_len, n_local, n_sites, min_avg_pkt_bytes, min_pkts,
                    min_dur_ms, admin_rule, 0};
    const size_t nk = (size_t)n_sites * 2;
    memset(hist, 0, nk * 10001u * sizeof(uint32_t));
    for (size_t k = 0; k < nk; k++) {
        rmin[k] = NAN;
        rmax[k] = NAN;
    }
    for (size_t i = 0; i < n; i++) {
        int sl = orc_is_local(&p, src[i]);
        int dl = orc_is_local(&p, dst[i]);
        if (sl == dl) continue;                    /* neither or both local */
        uint32_t s = orc_hash_one(m, sl ? dst[i] : src[i]);
        if (s == ORC_NO_SITE) continue;            /* remote endpoint unregistered */
        uint32_t dur = last[i] - first[i];
        if (!orc_eligible(&p, pkts[i], octets[i], dur)) continue;
        size_t k = (size_t)s * 2 + (sl ? 1 : 0);
        hist[k * 10001u + orc_rate_bucket(octets[i], dur)] += 1;
        double r = (double)octets[i] * 8000.0 / (double)dur;
        if (isnan(rmin[k]) || r < rmin[k]) rmin[k] = r;
        if (isnan(rmax[k]) || r > rmax[k]) rmax[k] = r;
    }
    for (size_t k = 0; k < nk; k++) {
        uint64_t total = 0;
        for (uint32_t b = 0; b <= 10000u; b++) total += hist[k * 10001u + b];
        med[k] = 0xFFFFFFFFu;
        if (total == 0) continue;
        uint64_t want = (total + 1) / 2, cum = 0;
        for (uint32_t b = 0; b <= 10000u; b++) {
            cum += hist[k * 10001u + b];
            if (cum >= want) {
                med[k] = b;
                break;
            }
        }
    }
    return 0;
}
