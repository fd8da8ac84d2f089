// noalloc.cu -- one-window processing that allocates no device memory.
//
// For callers that cannot call cudaMalloc: processes whose device memory is reserved up
// front by another allocator (a framework's caching allocator, a fixed budget), and
// latency-critical monitoring loops where cudaMalloc's implicit device synchronisation
// would stall other streams. The caller passes the flattened registry, the records and
// the result arrays (all device memory it owns); the kernel's scratch -- the window
// descriptor, the finalise ticket and the per-key accumulators -- lives in the fixed
// array below, which every GPU that loads this library holds until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "ctx.hpp"

namespace gnm {
namespace {

constexpr size_t kNoAllocBytes = 1u << 20;  // 1 MiB of scratch per device
constexpr size_t kNoAllocHeader = 256;      // descriptor, ticket, fallback counter
constexpr uint32_t kNoAllocMaxSites = GNM_NOALLOC_MAX_SITES;
static_assert(kNoAllocHeader + (2ull * kNoAllocMaxSites + kUnmatched) * kAccCols * 8 <= kNoAllocBytes,
              "the largest accepted registry must fit the fixed scratch");
constexpr int kMaxDevices = 64;

// The scratch. Host code must not pass the symbol itself to a kernel (on the host it
// names a host-side stand-in); its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};
unsigned long long g_ctx[kMaxDevices] = {0};

// Device address of the scratch on the current device: looked up once per device and
// context (set-up), again only after the device's context changed (a cudaDeviceReset or a
// new primary context reloads the library's device image).
gnm_status scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(GNM_E_INVAL, "device ordinal beyond the supported range");
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_addr[dev] || ctx == 0 || ctx != g_ctx[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            g_addr[dev] = nullptr;
            return fail(GNM_E_CUDA, std::string("cudaGetSymbolAddress of the scratch array: ") + cudaGetErrorString(e));
        }
        g_addr[dev] = p;
        g_ctx[dev] = current_context_id();  // the lookup made the device's context current
    }
    *out = static_cast<unsigned char*>(g_addr[dev]);
    return GNM_OK;
}

// Writes the one-window descriptor into the scratch header (device code may name the
// array directly).
__global__ void k_noalloc_desc(WinDesc d) {
    *reinterpret_cast<WinDesc*>(g_noalloc_scratch) = d;
}

}  // namespace
}  // namespace gnm

using namespace gnm;

extern "C" gnm_status gnm_window_process_noalloc(const gnm_config* cfg_in, const uint32_t* starts,
                                                 const uint32_t* site, uint32_t n_ranges, uint32_t n_sites,
                                                 const uint32_t* local_prefix, const uint8_t* local_len,
                                                 size_t n_local, const gnm_records* rec, uint64_t* stats,
                                                 double* rate, uint8_t* flag, void* stream) {
    gnm_config cfg;
    if (cfg_in) cfg = *cfg_in;
    else gnm_config_default(&cfg);
    if (!starts || !site || n_ranges == 0) return fail(GNM_E_INVAL, "registry ranges are missing");
    if (n_sites == 0) return fail(GNM_E_INVAL, "n_sites must be at least 1");
    if (n_sites > kNoAllocMaxSites)
        return fail(GNM_E_INVAL, "n_sites " + std::to_string(n_sites) + " exceeds the allocation-free limit of " +
                                     std::to_string(kNoAllocMaxSites) + " sites (1 MiB of fixed scratch)");
    if (n_local == 0 || n_local > GNM_MAX_LOCAL || !local_prefix || !local_len)
        return fail(GNM_E_INVAL, "need 1..8 local prefixes");
    if (!rec || !stats || !rate || !flag) return fail(GNM_E_INVAL, "records or result arrays are NULL");
    if (rec->n && !rec->on_device) return fail(GNM_E_INVAL, "records must be device arrays");
    if (rec->n > 0xFFFFFFFFull) return fail(GNM_E_INVAL, "a window holds 2^32 records or more");
    if (cfg.admin_rule != GNM_ADMIN_OR && cfg.admin_rule != GNM_ADMIN_AND)
        return fail(GNM_E_INVAL, "admin_rule must be GNM_ADMIN_OR or GNM_ADMIN_AND");
    if (rec->n) {
        const uint32_t* f[6] = {rec->srcaddr, rec->dstaddr, rec->dPkts, rec->dOctets, rec->first, rec->last};
        for (auto* q : f)
            if (!q || ((uintptr_t)q & 3u)) return fail(GNM_E_INVAL, "record arrays must be non-NULL and 4-byte aligned");
    }
    int dev = 0;
    GNM_CU(cudaGetDevice(&dev));
    unsigned char* scr = nullptr;
    GNM_TRY(scratch_address(dev, &scr));
    int sms = 0, optin = 0, per_sm = 0;
    GNM_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GNM_CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    GNM_CU(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t keys = 2 * n_sites + kUnmatched;
    const size_t used = kNoAllocHeader + (size_t)keys * kAccCols * 8;

    AggParams p;
    std::memset(&p, 0, sizeof(p));
    p.src = rec->srcaddr;
    p.dst = rec->dstaddr;
    p.pkts = rec->dPkts;
    p.oct = rec->dOctets;
    p.first = rec->first;
    p.last = rec->last;
    p.starts = starts;
    p.rsite = site;
    p.n_ranges = n_ranges;
    p.n_sites = n_sites;
    for (size_t i = 0; i < n_local; ++i) {
        if (local_len[i] > 32) return fail(GNM_E_INVAL, "local prefix length > 32");
        p.local_mask[i] = local_len[i] == 0 ? 0u : (0xFFFFFFFFu << (32 - local_len[i]));
        p.local_pfx[i] = local_prefix[i];
        if (p.local_pfx[i] & ~p.local_mask[i]) return fail(GNM_E_INVAL, "local prefix has host bits set");
    }
    p.n_local = (uint32_t)n_local;
    p.min_avg = cfg.min_avg_pkt_bytes;
    p.min_pkts = cfg.min_pkts;
    p.min_dur = cfg.min_dur_ms;
    p.admin_rule = cfg.admin_rule;
    p.acc = reinterpret_cast<uint64_t*>(scr + kNoAllocHeader);
    p.stats = stats;
    p.rate = rate;
    p.flag = flag;
    p.keys = keys;
    p.table_rows = keys;
    p.min_flows = cfg.min_flows_to_flag;
    p.threshold = cfg.threshold_bps;
    p.wins = reinterpret_cast<const WinDesc*>(scr);
    p.done = reinterpret_cast<uint32_t*>(scr + 64);
    p.violations = reinterpret_cast<unsigned long long*>(scr + 128);
    p.check_err = reinterpret_cast<unsigned long long*>(scr + 192);  // (checked build)
    p.n_wins = 1;
    p.n_total = rec->n;

    // clear what must start at zero (the array keeps the previous call's contents)
    GNM_CU(cudaMemsetAsync(scr, 0, used, st));
    if (rec->n == 0) {  // empty window: zero sums, no rate, no flag
        GNM_CU(cudaMemsetAsync(stats, 0, (size_t)keys * kNStat * 8, st));
        GNM_CU(cudaMemsetAsync(rate, 0xFF, (size_t)2 * n_sites * 8, st));
        GNM_CU(cudaMemsetAsync(flag, 0, (size_t)2 * n_sites, st));
        return GNM_OK;
    }
    // launch shape: registry in shared memory when it fits, per-key shared-memory rows
    // when they fit, else the two-slot cache
    LaunchShape sh;
    std::memset(&sh, 0, sizeof(sh));
    sh.lookup = (size_t)n_ranges * 8 <= 96 * 1024 ? kLookupSmem : kLookupL2;
    const size_t lookup_bytes = sh.lookup == kLookupSmem ? (size_t)n_ranges * 8 : 0;
    const size_t budget = (size_t)optin > lookup_bytes + 1024 ? (size_t)optin - lookup_bytes - 1024 : 0;
    uint32_t cap = 0;
    if ((size_t)keys * kSmemRowBytes <= std::min<size_t>(120 * 1024, budget)) {
        sh.table = kTableDirect;
    } else {
        cap = (uint32_t)(std::min<size_t>(200 * 1024, budget) / (kSmemRowBytes + 4)) & ~1u;
        sh.table = cap >= 256 ? kTableHash : kTableGlobal;
        if (sh.table == kTableGlobal) cap = 0;
    }
    sh.cap = cap;
    sh.agg = GNM_AGG_DIRECT;
    sh.block = 1024;
    sh.unroll = 1;
    sh.smem = aggregate_smem_bytes(sh.lookup, sh.table, n_ranges, keys, cap, 0, 0);
    const int fit = std::max(1, std::min(2048 / sh.block, (int)(per_sm / (sh.smem + 1024))));
    const uint64_t min_per_cta = (uint64_t)sh.block * 8;
    uint64_t grid = std::min<uint64_t>((uint64_t)sms * fit, std::max<uint64_t>(1, (rec->n + min_per_cta - 1) / min_per_cta));
    uint64_t chunk = (rec->n + grid - 1) / grid;
    chunk = (chunk + 3) & ~3ull;
    grid = (rec->n + chunk - 1) / chunk;
    sh.grid = (int)grid;
    sh.ctas_per_sm = fit;
    p.table_cap = cap;
    p.chunk = chunk;
    const uintptr_t a0 = (uintptr_t)rec->srcaddr & 15u;
    const uint32_t* f[6] = {rec->srcaddr, rec->dstaddr, rec->dPkts, rec->dOctets, rec->first, rec->last};
    p.vec_ok = 1;
    for (auto* q : f)
        if (((uintptr_t)q & 15u) != a0) p.vec_ok = 0;
    p.phase = (uint32_t)(a0 >> 2);
    WinDesc d;
    d.begin = 0;
    d.end = rec->n;
    d.slot = 0;
    d.flags = kWinFinalize;
    d.ctas = (uint32_t)grid;
    d.part_base = 0;
    d.n_parts = 0;
    d.key_base = 0;
    (void)cudaGetLastError();
    k_noalloc_desc<<<1, 1, 0, st>>>(d);
    GNM_CU(cudaGetLastError());
    GNM_CU(launch_aggregate(p, sh, st));
    return GNM_OK;
}
