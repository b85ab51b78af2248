// pac_serve.cu -- continuous batching of PAC queries (include/pac.h, part 5).
//
// One worker thread per server.  Submitted queries wait in arrival order.
// The worker retires finished launches (their arena ranges and staging come
// back), then admits from the head of the queue as many queries as the free
// arena, max_inflight and max_batch allow, plans them as one batch placed in
// the arena (pac_batch.h: host layout, bind, image staged in pinned memory),
// and enqueues the batch on the next of n_streams streams: image copy,
// scratch memset, aggregation, merge and release kernels, a copy of the
// batch's status word and of the device-time span its aggregation kernel ran
// in, and a host callback that stamps the completion time.
// The worker never holds its lock across a CUDA call, and callbacks take no
// lock, so a callback can never wait on the worker.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "pac_batch.h"
#include "pac_ctx.h"
#include "pac_validate.h"

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator of ranges of [0, size) (host bookkeeping only).
class RangeAlloc {
  public:
    explicit RangeAlloc(size_t size) { free_[0] = size; }
    bool alloc(size_t n, size_t align, size_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            const size_t start = (it->first + align - 1) / align * align;
            const size_t end = it->first + it->second;
            if (start + n > end) continue;
            const size_t f0 = it->first;
            free_.erase(it);
            if (start > f0) free_[f0] = start - f0;
            if (start + n < end) free_[start + n] = end - (start + n);
            *off = start;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        auto it = free_.emplace(off, n).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    std::map<size_t, size_t> free_;
};

struct Ticket {
    pac_query q{};
    std::vector<pac_agg_spec> specs;
    size_t need = 0;
    Clock::time_point t_submit;
    int state = 0;  // 0 queued, 1 running, 2 done
    double latency_ms = 0.0;
    pac_status status = PAC_OK;
};

struct Flight {
    int stream_idx = -1;
    pac_batch *plan = nullptr;
    size_t arena_off = 0, arena_bytes = 0;
    size_t stage_off = 0, stage_bytes = 0;
    std::vector<uint64_t> tickets;
    unsigned char *h_head = nullptr;  // pinned copy of the status word and the kernel's span
    uint32_t status_seen = 0;
    uint64_t span_lo = 0, span_hi = 0;  // device ns the aggregation kernel ran in (0, 0: none)
    std::atomic<bool> done{false};
    Clock::time_point t_done;
    struct pac_server *srv = nullptr;
    pac_status launch_error = PAC_OK;
};

pac_status status_from_bits(uint32_t h) {
    if (h & pacgpu::kStatusTimeout) return PAC_E_TIMEOUT;
    if (h & pacgpu::kStatusBadGroup) return PAC_E_INVALID;
    if (h & pacgpu::kStatusOverflow) return PAC_E_OVERFLOW;
    return PAC_OK;
}

}  // namespace

struct pac_server {
    pac_ctx *ctx = nullptr;  // the worker's own context
    int device = 0;
    pac_serve_config cfg{};
    pacgpu::BatchConfig bcfg = pacgpu::kBatchDefault;
    void *arena = nullptr;
    char *pinned = nullptr;
    size_t pinned_bytes = 0;
    RangeAlloc *arena_alloc = nullptr, *pin_alloc = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<Flight *> stream_busy;  // the flight each stream is running (nullptr: idle)
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Ticket> tickets;
    std::vector<Flight *> flights;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    // statistics
    std::vector<double> lat;
    std::vector<std::pair<uint64_t, uint64_t>> spans;  // device-time spans of the batches' aggregation kernels
    uint64_t batches = 0, batched_queries = 0;
    int inflight_q = 0, max_inflight_seen = 0;
    size_t arena_used = 0, arena_hw = 0;
};

namespace {

// Bytes copied back from the plan's head: the status word (offset 8) up to
// the end of the two span words.
constexpr size_t kHeadCopy = pacgpu::kPlanSpanOffset + 16 - 8;

void CUDART_CB on_done(void *p) {
    Flight *f = static_cast<Flight *>(p);
    f->t_done = Clock::now();
    uint64_t span[2];
    std::memcpy(&f->status_seen, f->h_head, 4);
    std::memcpy(span, f->h_head + (pacgpu::kPlanSpanOffset - 8), 16);
    if (span[0] && span[1]) {
        f->span_lo = ~span[0];
        f->span_hi = span[1];
    }
    f->done.store(true, std::memory_order_release);
    f->srv->cv_work.notify_one();
}

// Retires finished flights (lock held; no CUDA call).
void retire(pac_server *s) {
    for (size_t i = 0; i < s->flights.size();) {
        Flight *f = s->flights[i];
        if (!f->done.load(std::memory_order_acquire)) {
            i++;
            continue;
        }
        const pac_status st = f->launch_error != PAC_OK ? f->launch_error : status_from_bits(f->status_seen);
        for (uint64_t id : f->tickets) {
            Ticket &t = s->tickets[id];
            t.state = 2;
            t.status = st;
            t.latency_ms = std::chrono::duration<double, std::milli>(f->t_done - t.t_submit).count();
            s->lat.push_back(t.latency_ms);
        }
        if (f->span_hi) s->spans.emplace_back(f->span_lo, f->span_hi);
        s->inflight_q -= static_cast<int>(f->tickets.size());
        if (f->stream_idx >= 0 && s->stream_busy[f->stream_idx] == f) s->stream_busy[f->stream_idx] = nullptr;
        if (f->arena_bytes) s->arena_alloc->release(f->arena_off, f->arena_bytes);
        if (f->stage_bytes) s->pin_alloc->release(f->stage_off, f->stage_bytes);
        s->arena_used -= f->arena_bytes;
        pacgpu::plan_destroy(f->plan);  // host side only: the arena owns the device block
        delete f;
        s->flights[i] = s->flights.back();
        s->flights.pop_back();
        s->cv_done.notify_all();
    }
}

// Plans, places and enqueues the queries `ids` (lock NOT held).  Returns
// the flight, or nullptr when the arena or staging cannot hold the plan now.
Flight *launch_batch(pac_server *s, const std::vector<uint64_t> &ids, int si, std::unique_lock<std::mutex> &lk) {
    std::vector<pac_query> qs;
    qs.reserve(ids.size());
    for (uint64_t id : ids) qs.push_back(s->tickets[id].q);
    lk.unlock();
    pac_batch *b = nullptr;
    pac_status st = pacgpu::plan_build(s->ctx, qs.data(), static_cast<int>(qs.size()), s->bcfg, &b);
    lk.lock();
    if (st != PAC_OK) {
        // a query passed the submit-time checks, so this is an allocation failure
        Flight *f = new Flight();
        f->srv = s;
        f->tickets = ids;
        f->launch_error = st;
        f->done.store(true);
        f->t_done = Clock::now();
        return f;
    }
    size_t aoff = 0, poff = 0;
    const size_t stage = (b->image.size() + 15) / 16 * 16 + 256;
    if (!s->arena_alloc->alloc(b->device_bytes, 256, &aoff)) {
        pacgpu::plan_destroy(b);
        return nullptr;
    }
    if (!s->pin_alloc->alloc(stage, 256, &poff)) {
        s->arena_alloc->release(aoff, b->device_bytes);
        pacgpu::plan_destroy(b);
        return nullptr;
    }
    Flight *f = new Flight();
    f->srv = s;
    f->plan = b;
    f->arena_off = aoff;
    f->arena_bytes = b->device_bytes;
    f->stage_off = poff;
    f->stage_bytes = stage;
    f->tickets = ids;
    s->arena_used += b->device_bytes;
    s->arena_hw = std::max(s->arena_hw, s->arena_used);
    const cudaStream_t stream = s->streams[si];
    f->stream_idx = si;
    s->stream_busy[si] = f;
    lk.unlock();
    char *dev = static_cast<char *>(s->arena) + aoff;
    char *pin = s->pinned + poff;
    pacgpu::plan_bind(b, dev);
    b->d_status = reinterpret_cast<uint32_t *>(dev + 8);  // inside the zeroed head of the block
    f->h_head = reinterpret_cast<unsigned char *>(pin + (b->image.size() + 15) / 16 * 16);
    std::memcpy(pin, b->image.data(), b->image.size());
    st = pacgpu::plan_setup_kernel(s->ctx, b);
    if (st == PAC_OK) st = pacgpu::plan_enqueue(s->ctx, b, stream, pin);
    cudaError_t e = cudaSuccess;
    if (st == PAC_OK) e = cudaMemcpyAsync(f->h_head, b->d_status, kHeadCopy, cudaMemcpyDeviceToHost, stream);
    if (st == PAC_OK && e == cudaSuccess) e = cudaLaunchHostFunc(stream, on_done, f);
    lk.lock();
    if (st != PAC_OK || e != cudaSuccess) {
        // nothing of this batch will complete through the stream: fail its tickets
        cudaGetLastError();
        f->launch_error = st != PAC_OK ? st : PAC_E_CUDA;
        cudaStreamSynchronize(stream);
        f->t_done = Clock::now();
        f->done.store(true);
    }
    return f;
}

void worker_main(pac_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        retire(s);
        if (s->stop && s->queue.empty() && s->flights.empty()) break;
        bool launched = false;
        const int room = std::min(s->cfg.max_batch, s->cfg.max_inflight - s->inflight_q);
        // launch only on an idle stream: while all streams are busy, arrivals
        // queue up and go out together as one larger batch
        int si = -1;
        for (int k = 0; k < static_cast<int>(s->streams.size()); k++)
            if (!s->stream_busy[k]) {
                si = k;
                break;
            }
        if (!s->queue.empty() && room > 0 && si >= 0) {
            std::vector<uint64_t> ids;
            size_t need = 0;
            for (size_t i = 0; i < s->queue.size() && static_cast<int>(ids.size()) < room; i++) {
                const Ticket &t = s->tickets[s->queue[i]];
                if (!ids.empty() && need + t.need > s->cfg.mem_budget - s->arena_used) break;
                need += t.need;
                ids.push_back(s->queue[i]);
            }
            while (!ids.empty()) {
                Flight *f = launch_batch(s, ids, si, lk);
                if (f) {
                    for (size_t k = 0; k < ids.size(); k++) s->queue.pop_front();
                    for (uint64_t id : ids) s->tickets[id].state = 1;
                    s->inflight_q += static_cast<int>(ids.size());
                    s->max_inflight_seen = std::max(s->max_inflight_seen, s->inflight_q);
                    s->batches++;
                    s->batched_queries += ids.size();
                    s->flights.push_back(f);
                    launched = true;
                    break;
                }
                // the arena cannot hold this many now: try half as many
                ids.resize(ids.size() / 2);
            }
        }
        if (!launched) s->cv_work.wait_for(lk, std::chrono::microseconds(100));
    }
}

}  // namespace

extern "C" {

pac_status pac_serve_create(pac_ctx *ctx, const pac_serve_config *cfg, pac_server **srv) {
    if (!ctx || !cfg || !srv) return PAC_E_INVALID;
    *srv = nullptr;
    if (cfg->mem_budget == 0 || cfg->max_inflight < 1 || cfg->max_batch < 1 || cfg->n_streams < 1 ||
        cfg->n_streams > 32 || cfg->reserved != 0)
        return fail(ctx, PAC_E_INVALID, "bad server configuration");
    pac_server *s = new (std::nothrow) pac_server();
    if (!s) return fail(ctx, PAC_E_NOMEM, "server allocation");
    s->device = ctx->device;
    s->cfg = *cfg;
    pac_status st = pac_create(&s->ctx, ctx->device);
    if (st != PAC_OK) {
        delete s;
        return fail(ctx, st, "server context");
    }
    s->pinned_bytes = std::min<size_t>(std::max<size_t>(cfg->mem_budget / 8, 16u << 20), 512u << 20);
    cudaError_t e = cudaMalloc(&s->arena, cfg->mem_budget);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&s->pinned), s->pinned_bytes);
    for (int i = 0; e == cudaSuccess && i < cfg->n_streams; i++) {
        cudaStream_t q;
        e = cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking);
        if (e == cudaSuccess) s->streams.push_back(q);
    }
    s->stream_busy.assign(s->streams.size(), nullptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (cudaStream_t q : s->streams) cudaStreamDestroy(q);
        if (s->pinned) cudaFreeHost(s->pinned);
        if (s->arena) cudaFree(s->arena);
        pac_destroy(s->ctx);
        delete s;
        return fail(ctx, e == cudaErrorMemoryAllocation ? PAC_E_NOMEM : PAC_E_CUDA, "server resources: %s",
                    cudaGetErrorString(e));
    }
    s->arena_alloc = new RangeAlloc(cfg->mem_budget);
    s->pin_alloc = new RangeAlloc(s->pinned_bytes);
    s->worker = std::thread(worker_main, s);
    *srv = s;
    return PAC_OK;
}

pac_status pac_serve_submit(pac_server *s, const pac_query *q, uint64_t *ticket) {
    if (!s || !q || !ticket) return PAC_E_INVALID;
    pac_ctx tmp;  // host-only checks: messages stay out of the worker's context
    tmp.device = s->device;
    pac_status st = pacgpu::check_query(&tmp, q);
    if (st != PAC_OK) return st;
    Ticket t;
    t.specs.assign(q->specs, q->specs + q->n_specs);
    t.q = *q;
    pac_batch *b = nullptr;
    st = pacgpu::plan_build(&tmp, q, 1, s->bcfg, &b);
    if (st != PAC_OK) return st;
    t.need = b->device_bytes;
    const size_t stage = (b->image.size() + 15) / 16 * 16 + 256;
    pacgpu::plan_destroy(b);
    if (t.need > s->cfg.mem_budget || stage > s->pinned_bytes) return PAC_E_NOMEM;
    t.t_submit = Clock::now();
    std::lock_guard<std::mutex> g(s->mu);
    const uint64_t id = s->next_id++;
    Ticket &slot = s->tickets[id] = std::move(t);
    slot.q.specs = slot.specs.data();
    s->queue.push_back(id);
    *ticket = id;
    s->cv_work.notify_one();
    return PAC_OK;
}

pac_status pac_serve_poll(pac_server *s, uint64_t ticket, int32_t *done, double *latency_ms) {
    if (!s || !done) return PAC_E_INVALID;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return PAC_E_INVALID;
    *done = it->second.state == 2 ? 1 : 0;
    if (!*done) return PAC_OK;
    if (latency_ms) *latency_ms = it->second.latency_ms;
    const pac_status st = it->second.status;
    s->tickets.erase(it);
    return st;
}

pac_status pac_serve_wait(pac_server *s, uint64_t ticket, double *latency_ms) {
    if (!s) return PAC_E_INVALID;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return PAC_E_INVALID;
    s->cv_done.wait(lk, [&] { return it->second.state == 2; });
    if (latency_ms) *latency_ms = it->second.latency_ms;
    const pac_status st = it->second.status;
    s->tickets.erase(it);
    return st;
}

pac_status pac_serve_stats(pac_server *s, const char *name, double *value) {
    if (!s || !name || !value) return PAC_E_INVALID;
    std::lock_guard<std::mutex> g(s->mu);
    auto pct = [&](double p) {
        if (s->lat.empty()) return 0.0;
        std::vector<double> v(s->lat);
        std::sort(v.begin(), v.end());
        const size_t k = static_cast<size_t>(p * static_cast<double>(v.size() - 1) + 0.5);
        return v[std::min(k, v.size() - 1)];
    };
    if (!strcmp(name, "completed")) *value = static_cast<double>(s->lat.size());
    else if (!strcmp(name, "batches")) *value = static_cast<double>(s->batches);
    else if (!strcmp(name, "mean_batch"))
        *value = s->batches ? static_cast<double>(s->batched_queries) / static_cast<double>(s->batches) : 0.0;
    else if (!strcmp(name, "p50_ms")) *value = pct(0.50);
    else if (!strcmp(name, "p99_ms")) *value = pct(0.99);
    else if (!strcmp(name, "max_ms")) *value = pct(1.0);
    else if (!strcmp(name, "max_inflight_seen")) *value = s->max_inflight_seen;
    else if (!strcmp(name, "arena_high_water")) *value = static_cast<double>(s->arena_hw);
    else if (!strcmp(name, "max_device_overlap")) {
        // most batches whose aggregation kernels were running at one instant
        std::vector<std::pair<uint64_t, int>> ev;
        for (const auto &iv : s->spans) {
            ev.emplace_back(iv.first, 1);
            ev.emplace_back(iv.second, -1);
        }
        std::sort(ev.begin(), ev.end(), [](const auto &a, const auto &b) {
            return a.first != b.first ? a.first < b.first : a.second < b.second;  // ends before starts
        });
        int cur = 0, best = 0;
        for (const auto &e : ev) best = std::max(best, cur += e.second);
        *value = best;
    } else return PAC_E_INVALID;
    return PAC_OK;
}

void pac_serve_destroy(pac_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (cudaStream_t q : s->streams) {
        cudaStreamSynchronize(q);
        cudaStreamDestroy(q);
    }
    cudaFreeHost(s->pinned);
    cudaFree(s->arena);
    delete s->arena_alloc;
    delete s->pin_alloc;
    pac_destroy(s->ctx);
    delete s;
}

}  // extern "C"
