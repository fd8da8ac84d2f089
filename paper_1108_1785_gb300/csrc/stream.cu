// stream.cu -- streaming front end over one context: memory-budget admission, continuous
// batching over several CUDA streams, per-window latency.
//
// Host-side runtime only; the device work is the context's own window kernels
// (run_windows with open_add for each batch, close_window for the finalisation).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "ctx.hpp"

namespace gnm {
namespace {

constexpr uint64_t kRecordBytes = 24;   // six u32 fields
constexpr uint64_t kArenaAlign = 256;   // every staged field starts on a 256-byte boundary
constexpr uint32_t kMaxCudaStreams = 64;
constexpr int64_t kCallbackWaitNs = 10'000'000'000;  // bound on waiting for a finished stream's callbacks

int64_t now_ns() {
    const int64_t t = std::chrono::duration_cast<std::chrono::nanoseconds>(
                          std::chrono::steady_clock::now().time_since_epoch())
                          .count();
    return t > 0 ? t : 1;
}

uint64_t round_up(uint64_t a, uint64_t b) { return (a + b - 1) / b * b; }

// First-fit allocator over [0, size) with coalescing of freed neighbours.
class Arena {
public:
    void reset(uint64_t size) {
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(uint64_t n, uint64_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const uint64_t o = it->first, rest = it->second - n;
            free_.erase(it);
            if (rest) free_[o + n] = rest;
            *off = o;
            return true;
        }
        return false;
    }
    void release(uint64_t off, uint64_t n) {
        auto next = free_.lower_bound(off);
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                off = prev->first;
                n += prev->second;
                free_.erase(prev);
            }
        }
        if (next != free_.end() && off + n == next->first) {
            n += next->second;
            free_.erase(next);
        }
        free_[off] = n;
    }

private:
    std::map<uint64_t, uint64_t> free_;  // offset -> size
};

struct Win {
    uint64_t wid = 0;
    bool open = false;          // holds a pinned result slot
    bool close_submitted = false;
    bool closed = false;        // finalisation enqueued
    bool failed = false;
    uint32_t slot = 0;
    uint64_t records = 0;
    int64_t t_close = 0;        // host time of the closing submit
    int64_t t_enq = 0;          // host time its finalisation was enqueued
    int32_t status = GNM_OK;
    std::atomic<int64_t> t_done{0};  // set by the completion callback (or on failure)
};

struct Batch {
    gnm_records rec{};
    uint64_t wid = 0;
    uint64_t seq = 0;
    bool close = false;
    uint64_t bytes = 0;         // budget charge: 24 bytes per record
    uint64_t arena_off = 0, arena_bytes = 0;
    cudaEvent_t ev = nullptr;   // recorded after the batch's kernels
    int stream = 0;
    bool in_place = false;      // host batch read by the kernels at dev[] (mapped memory)
    const uint32_t* dev[6] = {};
};

// Device addresses of a host batch's six arrays when all of them are page-locked host
// memory mapped for the device; false otherwise.
bool mapped_fields(const gnm_records* r, const uint32_t* out[6]) {
    const uint32_t* f[6] = {r->srcaddr, r->dstaddr, r->dPkts, r->dOctets, r->first, r->last};
    for (int k = 0; k < 6; ++k) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, f[k]) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return false;
        out[k] = static_cast<const uint32_t*>(a.devicePointer);
    }
    return true;
}

void CUDART_CB on_window_done(void* arg) {
    // runs on the CUDA callback thread once the finalisation has completed; no CUDA calls
    static_cast<Win*>(arg)->t_done.store(now_ns(), std::memory_order_release);
}

}  // namespace
}  // namespace gnm

using namespace gnm;

struct gnm_stream {
    gnm_ctx* c = nullptr;
    gnm_stream_config cfg{};
    unsigned char* d_arena = nullptr;
    Arena arena;
    std::vector<cudaStream_t> streams;
    uint32_t next_stream = 0;
    std::vector<cudaEvent_t> event_pool;
    std::deque<Batch> queue;
    std::vector<Batch> inflight;
    std::unordered_map<uint64_t, std::unique_ptr<Win>> wins;
    std::vector<Win*> closing;  // finalisation enqueued, completion not yet reported
    std::vector<uint32_t> to_unpin;  // slots of windows reported by the last poll
    std::vector<double> latencies_ms;
    uint64_t seq = 0;
    uint64_t inflight_bytes = 0;
    gnm_stream_stats st{};
};

namespace gnm {
namespace {

gnm_status get_event(gnm_stream* s, cudaEvent_t* ev) {
    if (!s->event_pool.empty()) {
        *ev = s->event_pool.back();
        s->event_pool.pop_back();
        return GNM_OK;
    }
    GNM_CU(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
    return GNM_OK;
}

void release_batch(gnm_stream* s, Batch& b) {
    if (b.arena_bytes) s->arena.release(b.arena_off, b.arena_bytes);
    b.arena_bytes = 0;
    s->inflight_bytes -= b.bytes;
    if (b.ev) s->event_pool.push_back(b.ev);
    b.ev = nullptr;
}

// A window whose work failed: its slot is released (its sums are unusable) and its
// remaining batches are dropped; it is reported with the error once its closing batch
// has been taken from the queue.
void fail_window(gnm_stream* s, Win& w, gnm_status err) {
    if (!w.failed) {
        w.failed = true;
        w.status = err;
    }
    if (w.open) {
        unpin_slot(s->c, w.slot);
        (void)gnm_window_release(s->c, w.wid);
        w.open = false;
    }
}

void finish_failed(gnm_stream* s, Win& w) {
    if (w.closed) return;
    w.closed = true;
    w.t_done.store(now_ns(), std::memory_order_release);
    s->closing.push_back(&w);
    ++s->st.windows_closed;
}

// Waits (bounded) until the completion callbacks of the reported-closed windows have run;
// false if one has not (its stream failed).
bool wait_callbacks(gnm_stream* s) {
    const int64_t t0 = now_ns();
    for (Win* w : s->closing)
        while (w->t_done.load(std::memory_order_acquire) == 0) {
            if (now_ns() - t0 > kCallbackWaitNs) return false;
            std::this_thread::yield();
        }
    return true;
}

// Retires finished batches (frees their arena space and budget).
gnm_status retire(gnm_stream* s) {
    for (size_t i = 0; i < s->inflight.size();) {
        Batch& b = s->inflight[i];
        const cudaError_t e = cudaEventQuery(b.ev);
        if (e == cudaErrorNotReady) {
            ++i;
            continue;
        }
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(GNM_E_CUDA, std::string("batch completion: ") + cudaGetErrorString(e));
        }
        release_batch(s, b);
        s->inflight[i] = s->inflight.back();
        s->inflight.pop_back();
    }
    return GNM_OK;
}

// Copies (host batches) and processes one admitted batch on stream b.stream; closes the
// window after it when asked.
gnm_status enqueue(gnm_stream* s, Batch& b, Win& w) {
    gnm_ctx* c = s->c;
    cudaStream_t st = s->streams[b.stream];
    const uint64_t n = b.rec.n;
    if (n && !w.failed) {
        gnm_records dr = b.rec;
        if (b.in_place) {
            dr.srcaddr = b.dev[0]; dr.dstaddr = b.dev[1]; dr.dPkts = b.dev[2];
            dr.dOctets = b.dev[3]; dr.first = b.dev[4]; dr.last = b.dev[5];
            dr.on_device = 1;
        } else if (!b.rec.on_device) {
            const uint32_t* src[6] = {b.rec.srcaddr, b.rec.dstaddr, b.rec.dPkts, b.rec.dOctets, b.rec.first, b.rec.last};
            const uint32_t* dst[6];
            const uint64_t field = round_up(n * 4, kArenaAlign);
            for (int k = 0; k < 6; ++k) {
                uint32_t* d = reinterpret_cast<uint32_t*>(s->d_arena + b.arena_off + k * field);
                GNM_CU(cudaMemcpyAsync(d, src[k], n * 4, cudaMemcpyHostToDevice, st));
                dst[k] = d;
            }
            dr.srcaddr = dst[0]; dr.dstaddr = dst[1]; dr.dPkts = dst[2];
            dr.dOctets = dst[3]; dr.first = dst[4]; dr.last = dst[5];
            dr.on_device = 1;
        }
        const uint64_t off[2] = {0, n};
        const gnm_status r = run_windows(c, &dr, off, &b.wid, 1, st, false, true);
        if (r != GNM_OK) return r;
        w.records += n;
    }
    GNM_TRY(get_event(s, &b.ev));
    GNM_CU(cudaEventRecord(b.ev, st));
    if (b.close && w.failed) {
        finish_failed(s, w);
    } else if (b.close) {
        GNM_TRY(close_window(c, b.wid, st));  // the slot stays pinned until the window is reported
        w.t_enq = now_ns();
        w.open = false;
        w.closed = true;
        s->closing.push_back(&w);
        ++s->st.windows_closed;
        GNM_CU(cudaLaunchHostFunc(st, on_window_done, &w));
    }
    return GNM_OK;
}

// Admits queued batches in order. Memory is first come, first served (a batch that does
// not fit stops the scan); a window that cannot get a result slot is skipped together with
// its later batches, so that open windows can still reach their closing batch.
gnm_status admit(gnm_stream* s, bool* progressed) {
    *progressed = false;
    std::unordered_set<uint64_t> skipped;
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Batch& b = *it;
        Win& w = *s->wins.at(b.wid);
        if (skipped.count(b.wid)) {
            ++it;
            continue;
        }
        if (s->inflight_bytes + b.bytes > s->cfg.budget_bytes) break;
        b.arena_bytes = 0;
        if (b.rec.n && !b.rec.on_device && !b.in_place && !w.failed) {
            const uint64_t need = 6 * round_up(b.rec.n * 4, kArenaAlign);
            if (!s->arena.alloc(need, &b.arena_off)) break;
            b.arena_bytes = need;
        }
        b.stream = (int)(s->next_stream % s->streams.size());
        if (!w.open && !w.failed) {
            const gnm_status r = open_window(s->c, b.wid, s->streams[b.stream], true, &w.slot);
            if (r == GNM_E_CAPACITY) {  // every slot is held by an open window
                if (b.arena_bytes) s->arena.release(b.arena_off, b.arena_bytes);
                b.arena_bytes = 0;
                skipped.insert(b.wid);
                ++it;
                continue;
            }
            if (r != GNM_OK) {
                if (b.arena_bytes) s->arena.release(b.arena_off, b.arena_bytes);
                b.arena_bytes = 0;
                fail_window(s, w, r);
            } else {
                w.open = true;
            }
        }
        ++s->next_stream;
        s->inflight_bytes += b.bytes;
        s->st.peak_inflight_bytes = std::max(s->st.peak_inflight_bytes, s->inflight_bytes);
        const gnm_status r = enqueue(s, b, w);
        if (r != GNM_OK) {
            // the stream may still read the arena: wait for it before the space is reused
            (void)cudaStreamSynchronize(s->streams[b.stream]);
            (void)cudaGetLastError();
            release_batch(s, b);
            fail_window(s, w, r);
            if (b.close) finish_failed(s, w);
        } else {
            s->inflight.push_back(b);
        }
        it = s->queue.erase(it);
        *progressed = true;
    }
    return GNM_OK;
}

gnm_status pump(gnm_stream* s, bool* progressed) {
    for (uint32_t slot : s->to_unpin) unpin_slot(s->c, slot);  // reported: may be reused now
    s->to_unpin.clear();
    GNM_TRY(retire(s));
    return admit(s, progressed);
}

// Placement of a host batch under the context's host_records: in place (dev filled) when
// mapped and allowed, else staged; IN_PLACE refuses unmapped arrays.
gnm_status host_placement(gnm_stream* s, const gnm_records* b, bool* in_place, const uint32_t* dev[6]) {
    *in_place = false;
    if (!b->n || b->on_device || s->c->cfg.host_records == GNM_HOST_STAGE) return GNM_OK;
    *in_place = mapped_fields(b, dev);
    if (!*in_place && s->c->cfg.host_records == GNM_HOST_IN_PLACE)
        return fail(GNM_E_INVAL, "host_records IN_PLACE: the batch's arrays are not device-addressable "
                                 "page-locked host memory");
    return GNM_OK;
}

// Takes a batch (checked here); dev: the device addresses of a host batch read in place, or null.
gnm_status submit_batch(gnm_stream* s, const gnm_records* b, uint64_t wid, int close_window,
                        const uint32_t* const* dev) {
    if (b->n > 0xFFFFFFFFull) return fail(GNM_E_INVAL, "a batch holds 2^32 records or more");
    if (b->n * kRecordBytes > s->cfg.budget_bytes)
        return fail(GNM_E_INVAL, "batch of " + std::to_string(b->n) + " records exceeds the budget");
    if (b->n) {
        const uint32_t* f[6] = {b->srcaddr, b->dstaddr, b->dPkts, b->dOctets, b->first, b->last};
        for (auto* q : f)
            if (!q || ((uintptr_t)q & 3u)) return fail(GNM_E_INVAL, "record arrays must be non-NULL and 4-byte aligned");
    }
    auto it = s->wins.find(wid);
    if (it != s->wins.end() && it->second->close_submitted)
        return fail(GNM_E_STATE, "window " + std::to_string(wid) + " is already closed");
    GNM_CU(cudaSetDevice(s->c->device));
    const bool new_window = it == s->wins.end();
    if (new_window) {
        auto w = std::make_unique<Win>();
        w->wid = wid;
        it = s->wins.emplace(wid, std::move(w)).first;
    }
    Win& w = *it->second;
    Batch q;
    q.rec = *b;
    q.wid = wid;
    q.seq = ++s->seq;
    q.close = close_window != 0;
    q.bytes = b->n * kRecordBytes;
    if (dev) {
        q.in_place = true;
        for (int k = 0; k < 6; ++k) q.dev[k] = dev[k];
    }
    if (q.close) {
        w.close_submitted = true;
        w.t_close = now_ns();
    }
    s->queue.push_back(q);
    ++s->st.batches;
    s->st.records += b->n;
    bool progressed;
    GNM_TRY(pump(s, &progressed));
    if (!s->queue.empty() && s->queue.back().seq == q.seq) {  // not admitted: it has to wait
        if (s->queue.size() > s->cfg.max_queued) {  // no room: take it back
            s->queue.pop_back();
            --s->st.batches;
            s->st.records -= b->n;
            if (q.close) {
                w.close_submitted = false;
                w.t_close = 0;
            }
            if (new_window) s->wins.erase(wid);
            return fail(GNM_E_CAPACITY, "admission queue is full");
        }
        ++s->st.batches_queued;
    }
    return GNM_OK;
}

double percentile(std::vector<double> v, double q) {  // nearest rank
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    size_t k = (size_t)std::ceil(q * (double)v.size());
    k = std::min(std::max<size_t>(k, 1), v.size());
    return v[k - 1];
}

}  // namespace
}  // namespace gnm

extern "C" {

void gnm_stream_config_default(gnm_stream_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->budget_bytes = 4ull << 30;
    cfg->n_cuda_streams = 4;
    cfg->max_queued = 65536;
    cfg->max_batch_records = 1u << 20;
}

gnm_status gnm_stream_open(gnm_ctx* c, const gnm_stream_config* cfg_in, gnm_stream** out) {
    if (!c || !out) return fail(GNM_E_INVAL, "NULL argument");
    *out = nullptr;
    if (!c->have_registry) return fail(GNM_E_STATE, "no registry loaded");
    gnm_stream_config cfg;
    if (cfg_in) cfg = *cfg_in;
    else gnm_stream_config_default(&cfg);
    if (cfg.budget_bytes < kRecordBytes) return fail(GNM_E_INVAL, "budget_bytes below one record");
    if (cfg.n_cuda_streams == 0 || cfg.n_cuda_streams > kMaxCudaStreams)
        return fail(GNM_E_INVAL, "n_cuda_streams must be 1..64");
    if (cfg.max_queued == 0) return fail(GNM_E_INVAL, "max_queued must be at least 1");
    GNM_CU(cudaSetDevice(c->device));
    std::unique_ptr<gnm_stream> s(new (std::nothrow) gnm_stream());
    if (!s) return fail(GNM_E_NOMEM, "host allocation failed");
    s->c = c;
    s->cfg = cfg;
    // the arena holds budget_bytes of records plus the alignment padding of each field
    const uint64_t arena = cfg.budget_bytes + 6 * kArenaAlign;
    if (cudaMalloc(&s->d_arena, arena) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(GNM_E_NOMEM, "device arena of " + std::to_string(arena) + " bytes");
    }
    s->arena.reset(arena);
    if (const gnm_status r = reserve_launch_scratch(c, std::min<uint64_t>(cfg.max_batch_records,
                                                                          cfg.budget_bytes / kRecordBytes));
        r != GNM_OK) {
        cudaFree(s->d_arena);
        s->d_arena = nullptr;
        return r;
    }
    for (uint32_t k = 0; k < cfg.n_cuda_streams; ++k) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            (void)cudaGetLastError();
            gnm_stream_close(s.release());
            return fail(GNM_E_CUDA, "stream creation failed");
        }
        s->streams.push_back(st);
    }
    *out = s.release();
    return GNM_OK;
}

gnm_status gnm_stream_submit_many(gnm_stream* s, const gnm_records* pool, const uint64_t* begin,
                                  const uint64_t* count, const uint64_t* wids, const uint8_t* close_flags,
                                  size_t n_batches, size_t* n_accepted) {
    if (!s || !pool || !n_accepted || (n_batches && (!begin || !count || !wids)))
        return fail(GNM_E_INVAL, "NULL argument");
    *n_accepted = 0;
    GNM_CU(cudaSetDevice(s->c->device));
    // the pool's placement is decided once for all its slices
    bool in_place = false;
    const uint32_t* pdev[6];
    const bool fields = pool->srcaddr && pool->dstaddr && pool->dPkts && pool->dOctets && pool->first && pool->last;
    if (pool->n && fields) GNM_TRY(host_placement(s, pool, &in_place, pdev));
    for (size_t i = 0; i < n_batches; ++i) {
        if (count[i] && (begin[i] > pool->n || count[i] > pool->n - begin[i]))
            return fail(GNM_E_INVAL, "batch " + std::to_string(i) + " lies outside the pool");
        gnm_records b = *pool;
        b.n = count[i];
        const uint32_t* dev[6];
        if (count[i]) {
            b.srcaddr += begin[i];
            b.dstaddr += begin[i];
            b.dPkts += begin[i];
            b.dOctets += begin[i];
            b.first += begin[i];
            b.last += begin[i];
            for (int k = 0; k < 6; ++k) dev[k] = in_place ? pdev[k] + begin[i] : nullptr;
        }
        GNM_TRY(submit_batch(s, &b, wids[i], close_flags ? close_flags[i] : 0, count[i] && in_place ? dev : nullptr));
        *n_accepted = i + 1;
    }
    return GNM_OK;
}


gnm_status gnm_stream_submit(gnm_stream* s, const gnm_records* b, uint64_t wid, int close_window) {
    if (!s || !b) return fail(GNM_E_INVAL, "NULL argument");
    GNM_CU(cudaSetDevice(s->c->device));
    bool in_place;
    const uint32_t* dev[6];
    if (b->n && !b->on_device && b->srcaddr && b->dstaddr && b->dPkts && b->dOctets && b->first && b->last)
        GNM_TRY(host_placement(s, b, &in_place, dev));
    else
        in_place = false;
    return submit_batch(s, b, wid, close_window, in_place ? dev : nullptr);
}


gnm_status gnm_stream_poll(gnm_stream* s, gnm_window_done* out, size_t cap, size_t* n_out, int wait_all) {
    if (!s || !n_out || (cap && !out)) return fail(GNM_E_INVAL, "NULL argument");
    *n_out = 0;
    GNM_CU(cudaSetDevice(s->c->device));
    bool progressed;
    GNM_TRY(pump(s, &progressed));
    if (wait_all) {
        while (!s->queue.empty() || !s->inflight.empty()) {
            if (s->inflight.empty() && !progressed) {
                // the queue waits for result slots; those of windows reported now free up
                // at the next call, any others only when an open window is closed
                bool reportable = false;
                for (Win* w : s->closing) reportable = reportable || !w->failed;
                if (reportable) break;
                return fail(GNM_E_STATE, "queued batches wait for a result slot: close an open window");
            }
            if (!s->inflight.empty()) GNM_CU(cudaEventSynchronize(s->inflight.front().ev));
            GNM_TRY(pump(s, &progressed));
        }
        for (auto st : s->streams) GNM_CU(cudaStreamSynchronize(st));
        if (!wait_callbacks(s)) return fail(GNM_E_TIMEOUT, "a window's completion callback did not run");
    }
    size_t n = 0;
    for (size_t i = 0; i < s->closing.size() && n < cap;) {
        Win* w = s->closing[i];
        const int64_t t = w->t_done.load(std::memory_order_acquire);
        if (t == 0) {
            ++i;
            continue;
        }
        gnm_window_done& d = out[n++];
        d.window_id = w->wid;
        d.records = w->records;
        d.latency_ms = (double)(t - w->t_close) * 1e-6;
        d.status = w->status;
        d.reserved = 0;
        d.queued_ms = w->t_enq ? (double)(w->t_enq - w->t_close) * 1e-6 : 0.0;
        if (w->status == GNM_OK) {
            s->latencies_ms.push_back(d.latency_ms);
            s->to_unpin.push_back(w->slot);
        }
        ++s->st.windows_done;
        s->closing.erase(s->closing.begin() + (long)i);
        s->wins.erase(w->wid);
    }
    *n_out = n;
    return GNM_OK;
}

gnm_status gnm_stream_stats_get(gnm_stream* s, gnm_stream_stats* out) {
    if (!s || !out) return fail(GNM_E_INVAL, "NULL argument");
    // batches that finished since the last call are retired first, so that the figures
    // are those of now (a window can be reported done by its callback before the poll that
    // reported it had seen its last batch finish)
    GNM_CU(cudaSetDevice(s->c->device));
    GNM_TRY(retire(s));
    *out = s->st;
    out->inflight_bytes = s->inflight_bytes;
    const auto& v = s->latencies_ms;
    out->p50_ms = percentile(v, 0.50);
    out->p99_ms = percentile(v, 0.99);
    out->max_ms = v.empty() ? 0.0 : *std::max_element(v.begin(), v.end());
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_ms = v.empty() ? 0.0 : sum / (double)v.size();
    return GNM_OK;
}

void gnm_stream_close(gnm_stream* s) {
    if (!s) return;
    cudaSetDevice(s->c->device);
    for (auto st : s->streams) cudaStreamSynchronize(st);
    if (!wait_callbacks(s))  // a callback may still come: keep what it writes to
        for (auto& kv : s->wins) (void)kv.second.release();
    for (auto& b : s->inflight) release_batch(s, b);
    s->inflight.clear();
    s->queue.clear();
    for (uint32_t slot : s->to_unpin) unpin_slot(s->c, slot);
    for (Win* w : s->closing)
        if (!w->failed) unpin_slot(s->c, w->slot);
    for (auto& kv : s->wins)
        if (kv.second && kv.second->open) unpin_slot(s->c, kv.second->slot);
    for (auto ev : s->event_pool) cudaEventDestroy(ev);
    for (auto st : s->streams) cudaStreamDestroy(st);
    if (s->d_arena) cudaFree(s->d_arena);
    (void)cudaGetLastError();
    delete s;
}

}  // extern "C"
