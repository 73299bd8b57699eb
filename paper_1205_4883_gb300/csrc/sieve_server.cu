// sieve_server.cu -- continuous batching of sieve requests (see the serving
// section of gbsieve.h).
//
// A scheduler thread owns the GPU side.  Each tick it takes, from every
// admitted request that still has segments to sieve, a run of consecutive
// segments (a sub-range that starts on one of the request's segment
// boundaries, so its wheel grid and its words of the odd-only bitmap line up
// with the whole request's), up to tick_segments segments in all, and
// launches one count-mode and/or one bitmap-mode persistent kernel over them.
// Two ticks alternate between two sets of buffers, so the next tick is
// already queued while the current one runs.  When a tick's event has fired,
// its counts are added to their requests; a request whose last run is done is
// completed; a finished list request is handed to one of four finisher threads,
// which compacts its bitmap on its own stream and copies the primes by DMA into
// a pinned host arena (through a pinned bounce buffer to the heap when the arena
// is full), so the scheduler keeps launching ticks meanwhile.
// Host waits poll events and condition variables; no kernel waits on anything.

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "host.h"

using namespace gbs;

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t ticket = 0;
    uint64_t lo = 0, hi = 0;
    int kind = SIEVE_REQ_COUNT;
    RangeDesc plan;                 // the whole range, planned once
    uint64_t next_seg = 0;          // next segment to schedule
    uint64_t done_segs = 0;         // segments whose counts have been added
    uint64_t count = 0;
    uint32_t *d_bitmap = nullptr;   // list requests: arena memory
    uint64_t *d_list = nullptr;
    uint64_t list_cap = 0;
    size_t arena_off = 0, arena_bytes = 0;
    std::unique_ptr<unsigned char[]> heap;  // list result on the heap (when the pinned arena is full)
    void *h_list = nullptr;                 // the list result handed out: pinned arena or `heap`
    size_t harena_off = 0, harena_bytes = 0;
    int status = SIEVE_OK;
    bool done = false;
    Clock::time_point t_submit;
    double latency_us = 0;
};

struct Run {
    Req *req;
    uint64_t seg_a, seg_b;
};

struct Tick {
    LaunchBuffers lb[2];  // [0] count-mode runs, [1] bitmap-mode runs
    std::vector<Run> runs[2];
    cudaStream_t stream = nullptr;  // the stream this tick slot launches on
    cudaEvent_t ev0 = nullptr, ev = nullptr;  // around the tick's work (timing events)
    uint64_t segments = 0;
    bool busy = false;
};

// First-fit allocator over one arena (offsets, 256-byte aligned): the device
// arena of bitmaps and device lists, and the pinned host arena of list results.
struct Arena {
    unsigned char *base = nullptr;
    size_t size = 0, used = 0;
    std::map<size_t, size_t> free_blocks;  // offset -> bytes
    bool alloc(size_t bytes, size_t *off) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t roff = it->first + bytes;
                free_blocks.erase(it);
                if (rest) free_blocks[roff] = rest;
                used += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        used -= bytes;
        auto it = free_blocks.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_blocks.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_blocks.erase(next);
        }
        if (it != free_blocks.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_blocks.erase(it);
            }
        }
    }
};

// A host thread that completes list requests, with its own stream, compaction
// scratch and pinned bounce buffer, so that several run side by side.
struct Finisher {
    cudaStream_t stream = nullptr;
    CompactScratch cs;
    uint64_t *bounce = nullptr;  // pinned, kBounceWords
    std::thread th;
};
constexpr int kFinishers = 4;

}  // namespace

struct sieve_server {
    sieve_ctx *owner = nullptr;
    sieve_ctx *view = nullptr;  // private context view: borrowed resident state, own buffers
    sieve_server_cfg cfg{};
    cudaStream_t stream = nullptr;   // sieve ticks (slot 0, and slot 1 with serial_ticks)
    cudaStream_t stream2 = nullptr;  // slot 1 of the ticks unless serial_ticks
    Tick ticks[2];
    int next_tick = 0;
    Arena arena;

    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_finish;
    std::deque<Req *> to_finish;       // list requests whose sieving is done
    bool finisher_stop = false;
    Finisher fin[kFinishers];          // compaction and copy-out of finished list requests
    Arena host_arena;                  // pinned: list results, copied in by DMA, freed on release

    std::map<uint64_t, std::unique_ptr<Req>> reqs;
    std::deque<Req *> active;  // admitted, segments left to schedule or in flight
    std::deque<uint64_t> done_q;  // tickets completed and not yet reported by sieve_server_wait_any
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread th;

    sieve_server_counters st{};
};

namespace {

// Upper bound on the primes in [lo, hi): 2 w / ln w for w > 1 (Montgomery and
// Vaughan, "The large sieve", Mathematika 20, 1973), plus slack.
uint64_t prime_count_bound(uint64_t w) {
    if (w < 16) return w + 2;
    return (uint64_t)(2.0 * (double)w / std::log((double)w)) + 64;
}

// The sub-range of `r` made of its segments [a, b): it starts on a segment
// boundary, so its own plan uses the same wheel grid and its bitmap words are
// whole words of the request's bitmap.
RangeDesc plan_run(sieve_server *srv, const Req &r, uint64_t a, uint64_t b, int mode) {
    const uint64_t span = 30ull * srv->view->params.seg_bytes;
    const uint64_t lo = a == 0 ? r.lo : (uint64_t)(30 * r.plan.Bbase) + a * span;
    const uint64_t hi = b == r.plan.nseg ? r.hi : (uint64_t)(30 * r.plan.Bbase) + b * span;
    uint32_t *bm = nullptr;
    if (mode == kModeBitmap) bm = r.d_bitmap + ((lo | 1) - (r.lo | 1)) / 64;
    return plan_range(srv->view, lo, hi, srv->view->params.seg_bytes, mode, bm);
}

// Mark an admitted request finished (lock held); it leaves the in-flight count.
void complete(sieve_server *srv, Req *r, int status) {
    r->status = status;
    r->latency_us = std::chrono::duration<double, std::micro>(Clock::now() - r->t_submit).count();
    r->done = true;
    srv->done_q.push_back(r->ticket);
    srv->st.completed++;
    srv->st.integers += r->hi - r->lo;
    srv->st.in_flight--;
}

constexpr size_t kBounceWords = 2u << 20;  // 16 MiB of uint64 per finisher
constexpr size_t kHostArenaBytes = 1ull << 30;  // pinned host memory for list results (default)

// Bytes per list element: uint64 primes, or uint32 offsets from lo.
size_t list_elem(const Req *r) { return r->kind == SIEVE_REQ_LIST_OFFSETS ? 4 : 8; }

// Called without the lock: compaction of a finished list request into its
// device list (the primes, or their offsets from lo), then one DMA copy into the
// pinned host arena -- or, when the arena has no room, a chunked copy to the
// heap through the pinned buffer.
int finish_list(sieve_server *srv, Finisher &f, Req *r) {
    uint64_t n = 0;
    const bool offsets = r->kind == SIEVE_REQ_LIST_OFFSETS;
    const size_t es = list_elem(r);
    int rc = compact_with(srv->view, f.stream, f.cs, r->d_bitmap, r->lo, r->hi, r->d_list, r->list_cap, &n,
                          offsets ? 0 : 1, offsets ? r->lo : 0);
    if (rc) return rc;
    bool pinned = false;
    if (n && srv->host_arena.size) {
        std::lock_guard<std::mutex> lk(srv->mu);
        pinned = srv->host_arena.alloc(n * es, &r->harena_off);
        if (pinned) r->harena_bytes = n * es;
    }
    if (pinned) {
        r->h_list = srv->host_arena.base + r->harena_off;
        cudaError_t e = cudaMemcpyAsync(r->h_list, r->d_list, n * es, cudaMemcpyDeviceToHost, f.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(f.stream);
        if (e != cudaSuccess) return cuda_fail(srv->view, e, "list copy");
        r->count = n;
        return SIEVE_OK;
    }
    r->heap.reset(new (std::nothrow) unsigned char[n ? n * es : 8]);
    if (!r->heap) return SIEVE_ENOMEM;
    r->h_list = r->heap.get();
    const unsigned char *src = reinterpret_cast<const unsigned char *>(r->d_list);
    const uint64_t chunk = kBounceWords * 8 / es;  // elements per pass through the bounce buffer
    for (uint64_t done = 0; done < n; done += chunk) {
        const uint64_t k = std::min<uint64_t>(chunk, n - done);
        cudaError_t e = cudaMemcpyAsync(f.bounce, src + done * es, k * es, cudaMemcpyDeviceToHost, f.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(f.stream);
        if (e != cudaSuccess) return cuda_fail(srv->view, e, "list copy");
        std::memcpy(r->heap.get() + done * es, f.bounce, k * es);
    }
    r->count = n;
    return SIEVE_OK;
}

// Fold a finished tick into its requests (lock held).
void harvest(sieve_server *srv, Tick &t) {
    bool any = false;
    for (int mode = 0; mode < 2; ++mode) {
        for (size_t i = 0; i < t.runs[mode].size(); ++i) {
            const Run &run = t.runs[mode][i];
            Req *r = run.req;
            r->count += t.lb[mode].h_acc[i];
            r->done_segs += run.seg_b - run.seg_a;
            if (r->done_segs != r->plan.nseg) continue;
            srv->active.erase(std::remove(srv->active.begin(), srv->active.end(), r), srv->active.end());
            if (r->kind != SIEVE_REQ_COUNT) {
                srv->to_finish.push_back(r);
                srv->cv_finish.notify_one();
            } else {
                complete(srv, r, SIEVE_OK);
                any = true;
            }
        }
        t.runs[mode].clear();
    }
    t.busy = false;
    srv->st.ticks++;
    srv->st.segments += t.segments;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.ev0, t.ev) == cudaSuccess) srv->st.tick_gpu_ms += ms;
    if (any) srv->cv_done.notify_all();
}

// Finisher threads: complete list requests (compaction and copy-out).
void finisher(sieve_server *srv, Finisher *f) {
    cudaSetDevice(srv->view->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        srv->cv_finish.wait(lk, [&] { return srv->finisher_stop || !srv->to_finish.empty(); });
        if (srv->to_finish.empty()) break;  // stop requested and nothing left
        Req *r = srv->to_finish.front();
        srv->to_finish.pop_front();
        lk.unlock();
        const int rc = finish_list(srv, *f, r);
        lk.lock();
        srv->arena.release(r->arena_off, r->arena_bytes);
        srv->st.device_bytes_reserved = srv->arena.used;
        complete(srv, r, rc);
        srv->cv_done.notify_all();
    }
}

// Take runs from the active requests and launch them on tick t (lock held).
int launch_tick(sieve_server *srv, Tick &t) {
    uint64_t budget = srv->cfg.tick_segments;
    size_t with_work = 0;
    for (Req *r : srv->active)
        if (r->next_seg < r->plan.nseg) ++with_work;
    if (!with_work) return 0;
    const uint64_t share = std::max<uint64_t>(1, budget / with_work);
    size_t m[2] = {0, 0};
    // round-robin start so that no request is always last
    const size_t n_act = srv->active.size();
    const size_t start = n_act ? (size_t)(srv->st.ticks % n_act) : 0;
    for (size_t q = 0; q < n_act && budget; ++q) {
        Req *r = srv->active[(start + q) % n_act];
        if (r->next_seg >= r->plan.nseg) continue;
        const uint64_t take = std::min<uint64_t>({r->plan.nseg - r->next_seg, share, budget});
        const int mode = r->kind != SIEVE_REQ_COUNT ? kModeBitmap : kModeCount;
        if (m[mode] >= t.lb[mode].cap) continue;
        t.lb[mode].h_ranges()[m[mode]++] = plan_run(srv, *r, r->next_seg, r->next_seg + take, mode);
        t.runs[mode].push_back(Run{r, r->next_seg, r->next_seg + take});
        r->next_seg += take;
        budget -= take;
    }
    if (!m[0] && !m[1]) return 0;
    t.segments = srv->cfg.tick_segments - budget;
    cudaError_t e = cudaEventRecord(t.ev0, t.stream);
    if (e != cudaSuccess) return cuda_fail(srv->view, e, "tick event");
    for (int mode = 0; mode < 2; ++mode) {
        if (!m[mode]) continue;
        int rc = launch_ranges(srv->view, t.stream, srv->view->params, mode, t.lb[mode], m[mode], nullptr);
        if (rc) return rc;
        e = cudaMemcpyAsync(t.lb[mode].h_acc, t.lb[mode].d_acc + 1, m[mode] * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, t.stream);
        if (e != cudaSuccess) return cuda_fail(srv->view, e, "tick copy");
    }
    e = cudaEventRecord(t.ev, t.stream);
    if (e != cudaSuccess) return cuda_fail(srv->view, e, "tick event");
    t.busy = true;
    return 1;
}

void fail_all(sieve_server *srv, int rc) {
    for (Tick &t : srv->ticks)
        for (auto &rs : t.runs) rs.clear();
    for (Req *r : srv->active) {
        if (r->kind != SIEVE_REQ_COUNT) srv->arena.release(r->arena_off, r->arena_bytes);
        complete(srv, r, rc);
    }
    srv->active.clear();
    srv->cv_done.notify_all();
}

void scheduler(sieve_server *srv) {
    cudaSetDevice(srv->view->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        // fold in the ticks that have finished
        bool any_busy = false;
        for (Tick &t : srv->ticks) {
            if (!t.busy) continue;
            cudaError_t q = cudaEventQuery(t.ev);
            if (q == cudaSuccess) {
                harvest(srv, t);
            } else if (q != cudaErrorNotReady) {
                t.busy = false;
                fail_all(srv, cuda_fail(srv->view, q, "tick"));
            } else {
                any_busy = true;
            }
        }
        // keep up to two ticks queued
        bool launched = false;
        for (int k = 0; k < 2; ++k) {
            Tick &t = srv->ticks[srv->next_tick];
            if (t.busy) break;
            int rc = launch_tick(srv, t);
            if (rc < 0) {
                fail_all(srv, rc);
                break;
            }
            if (rc == 0) break;
            launched = any_busy = true;
            srv->next_tick ^= 1;
        }
        if (srv->stop && srv->active.empty() && !any_busy) break;
        if (launched) continue;
        if (any_busy) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        } else {
            srv->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

}  // namespace

extern "C" {

int sieve_server_create(sieve_ctx *ctx, const sieve_server_cfg *cfg, sieve_server **out) {
    if (!ctx || !out) return SIEVE_EINVAL;
    *out = nullptr;
    std::unique_ptr<sieve_server> srv(new (std::nothrow) sieve_server);
    if (!srv) return SIEVE_ENOMEM;
    srv->owner = ctx;
    if (cfg) srv->cfg = *cfg;
    if (!srv->cfg.max_requests) srv->cfg.max_requests = 1024;
    if (!srv->cfg.tick_segments) srv->cfg.tick_segments = 4u * (uint32_t)ctx->num_sms;
    if (!srv->cfg.max_device_bytes) srv->cfg.max_device_bytes = 4ull << 30;

    sieve_ctx *v = new (std::nothrow) sieve_ctx;
    if (!v) return SIEVE_ENOMEM;
    srv->view = v;
    v->shadow = true;
    v->device = ctx->device;
    v->num_sms = ctx->num_sms;
    v->hi_max = ctx->hi_max;
    v->prime_limit = ctx->prime_limit;
    v->d_primes = ctx->d_primes;
    v->d_magic = ctx->d_magic;
    v->h_primes = ctx->h_primes;
    v->h_prime_bucket = ctx->h_prime_bucket;
    v->d_tile = ctx->d_tile;
    v->tile_stride = ctx->tile_stride;
    v->params = ctx->params;
    auto bail = [&](int rc) {
        sieve_server_destroy(srv.release());
        return rc;
    };
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&srv->stream, cudaStreamNonBlocking);
    // Finishers on the highest-priority streams: a sieve CTA holds a whole SM (all
    // its registers), so compaction kernels run only where one has left; with
    // priority their CTAs take a freed SM before the next tick's waiting CTAs.
    int prio_low = 0, prio_high = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    for (Finisher &f : srv->fin)
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&f.stream, cudaStreamNonBlocking, prio_high);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "server streams"));
    v->stream = srv->stream;
    // the Miller-Rabin path keeps raw words in one scratch of the view, which two
    // ticks in flight would share: the server sieves every segment in full
    v->params.mr_percent = 0;
    if (!srv->cfg.serial_ticks) e = cudaStreamCreateWithFlags(&srv->stream2, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "server streams"));
    for (int k = 0; k < 2; ++k) {
        Tick &t = srv->ticks[k];
        t.stream = k == 1 && srv->stream2 ? srv->stream2 : srv->stream;
        for (auto &lb : t.lb) {
            int rc = alloc_launch_buffers(v, lb, srv->cfg.max_requests);
            if (rc) return bail(rc);
        }
        e = cudaEventCreate(&t.ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&t.ev);
        if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "server event"));
    }
    e = cudaMalloc(&srv->arena.base, srv->cfg.max_device_bytes);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "server arena"));
    srv->arena.size = srv->cfg.max_device_bytes;
    srv->arena.free_blocks[0] = srv->arena.size;
    for (Finisher &f : srv->fin) {
        e = cudaMallocHost(&f.bounce, kBounceWords * sizeof(uint64_t));
        if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "server bounce buffer"));
    }
    // list results go here by DMA; without it (pinning refused) they take the bounce path
    unsigned char *ha = nullptr;
    const size_t hbytes = srv->cfg.host_arena_bytes ? srv->cfg.host_arena_bytes : kHostArenaBytes;
    if (cudaMallocHost(&ha, hbytes) == cudaSuccess) {
        srv->host_arena.base = ha;
        srv->host_arena.size = hbytes;
        srv->host_arena.free_blocks[0] = hbytes;
    } else {
        cudaGetLastError();  // clear the refused allocation's error
    }
    srv->th = std::thread(scheduler, srv.get());
    for (Finisher &f : srv->fin) f.th = std::thread(finisher, srv.get(), &f);
    *out = srv.release();
    return SIEVE_OK;
}

int sieve_server_submit(sieve_server *srv, const sieve_req *req, uint64_t *ticket) {
    if (!srv || !req || !ticket) return SIEVE_EINVAL;
    if (req->lo > req->hi || (req->kind != SIEVE_REQ_COUNT && req->kind != SIEVE_REQ_LIST &&
                              req->kind != SIEVE_REQ_LIST_OFFSETS))
        return SIEVE_EINVAL;
    if (req->hi > srv->view->hi_max) return SIEVE_ERANGE;
    if (req->kind == SIEVE_REQ_LIST_OFFSETS && req->hi - req->lo > (1ull << 32)) return SIEVE_ERANGE;
    std::unique_ptr<Req> r(new (std::nothrow) Req);
    if (!r) return SIEVE_ENOMEM;
    r->lo = req->lo;
    r->hi = req->hi;
    r->kind = req->kind;
    r->t_submit = Clock::now();
    const int mode = r->kind != SIEVE_REQ_COUNT ? kModeBitmap : kModeCount;
    r->plan = plan_range(srv->view, r->lo, r->hi, srv->view->params.seg_bytes, mode, nullptr);
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) return SIEVE_EINVAL;
    if (srv->reqs.size() >= srv->cfg.max_requests) {
        srv->st.rejected++;
        return SIEVE_EBUSY;
    }
    if (r->kind != SIEVE_REQ_COUNT && r->hi > r->lo) {
        const uint64_t words = bitmap_words_of(r->lo, r->hi);
        r->list_cap = prime_count_bound(r->hi - r->lo);
        const size_t bm_bytes = ((words * 4 + 255) & ~(size_t)255);
        r->arena_bytes = bm_bytes + r->list_cap * sizeof(uint64_t);
        if (!srv->arena.alloc(r->arena_bytes, &r->arena_off)) {
            srv->st.rejected++;
            return SIEVE_EBUSY;
        }
        r->d_bitmap = reinterpret_cast<uint32_t *>(srv->arena.base + r->arena_off);
        r->d_list = reinterpret_cast<uint64_t *>(srv->arena.base + r->arena_off + bm_bytes);
        srv->st.device_bytes_reserved = srv->arena.used;
    }
    r->ticket = srv->next_ticket++;
    *ticket = r->ticket;
    srv->st.submitted++;
    Req *raw = r.get();
    srv->reqs.emplace(r->ticket, std::move(r));
    srv->st.in_flight++;
    if (raw->plan.nseg == 0) {  // empty range: nothing to sieve
        complete(srv, raw, SIEVE_OK);
        srv->cv_done.notify_all();
        return SIEVE_OK;
    }
    srv->active.push_back(raw);
    srv->cv_work.notify_one();
    return SIEVE_OK;
}

int sieve_server_poll(sieve_server *srv, uint64_t ticket, sieve_result *res, int64_t timeout_us) {
    if (!srv || !res) return SIEVE_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return SIEVE_ENOENT;
    Req *r = it->second.get();
    if (!r->done) {
        auto ready = [&] { return r->done; };
        if (timeout_us < 0)
            srv->cv_done.wait(lk, ready);
        else if (!srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
            return SIEVE_ETIMEOUT;
    }
    res->status = r->status;
    res->kind = r->kind;
    res->count = r->count;
    const bool ok = r->status == SIEVE_OK;
    res->primes = (r->kind == SIEVE_REQ_LIST && ok) ? static_cast<const uint64_t *>(r->h_list) : nullptr;
    res->offsets = (r->kind == SIEVE_REQ_LIST_OFFSETS && ok) ? static_cast<const uint32_t *>(r->h_list) : nullptr;
    res->latency_us = r->latency_us;
    return SIEVE_OK;
}

int sieve_server_wait_any(sieve_server *srv, uint64_t *tickets, size_t cap, size_t *n, int64_t timeout_us) {
    if (!srv || !n || (!tickets && cap)) return SIEVE_EINVAL;
    *n = 0;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto ready = [&] { return !srv->done_q.empty(); };
    if (!ready()) {
        if (timeout_us < 0)
            srv->cv_done.wait(lk, ready);
        else if (!srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
            return SIEVE_ETIMEOUT;
    }
    size_t k = 0;
    while (k < cap && !srv->done_q.empty()) {
        tickets[k++] = srv->done_q.front();
        srv->done_q.pop_front();
    }
    *n = k;
    return SIEVE_OK;
}

int sieve_server_release(sieve_server *srv, uint64_t ticket) {
    if (!srv) return SIEVE_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return SIEVE_ENOENT;
    if (!it->second->done) return SIEVE_EBUSY;
    if (it->second->harena_bytes) srv->host_arena.release(it->second->harena_off, it->second->harena_bytes);
    srv->reqs.erase(it);
    return SIEVE_OK;
}

int sieve_server_stats(sieve_server *srv, sieve_server_counters *st) {
    if (!srv || !st) return SIEVE_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    *st = srv->st;
    return SIEVE_OK;
}

void sieve_server_destroy(sieve_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->th.joinable()) srv->th.join();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->finisher_stop = true;
    }
    srv->cv_finish.notify_all();
    for (Finisher &f : srv->fin)
        if (f.th.joinable()) f.th.join();
    if (srv->view) {
        cudaSetDevice(srv->view->device);
        if (srv->stream) cudaStreamSynchronize(srv->stream);
        if (srv->stream2) cudaStreamSynchronize(srv->stream2);
        for (Tick &t : srv->ticks) {
            for (auto &lb : t.lb) free_launch_buffers(srv->view, lb);
            if (t.ev0) cudaEventDestroy(t.ev0);
            if (t.ev) cudaEventDestroy(t.ev);
        }
        for (Finisher &f : srv->fin) free_compact_scratch(srv->view, f.cs);
        srv->view->stream = nullptr;  // the view does not own the stream
        sieve_destroy(srv->view);
    }
    if (srv->arena.base) cudaFree(srv->arena.base);
    for (Finisher &f : srv->fin) {
        if (f.bounce) cudaFreeHost(f.bounce);
        if (f.stream) cudaStreamDestroy(f.stream);
    }
    srv->reqs.clear();  // results in the host arena die with it
    if (srv->host_arena.base) cudaFreeHost(srv->host_arena.base);
    if (srv->stream) cudaStreamDestroy(srv->stream);
    if (srv->stream2) cudaStreamDestroy(srv->stream2);
    delete srv;
}

}  // extern "C"
