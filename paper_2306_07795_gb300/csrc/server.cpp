// server.cpp -- native request server (include/bmmc_server.h).
//
// Submission plans the request in the caller's thread (bmmc_plan_create_ex),
// so planning cost scales with the number of submitting threads; in
// CONTINUOUS mode only the first pass is planned then, and the second pass of
// a two-pass plan is derived right after the first pass is launched, while it
// runs.  In CONTINUOUS mode a scheduler thread then admits requests in submission order
// while their input + output + workspace bytes fit the budget and their output
// and workspace fit the arena, launches each on the least-loaded stream (small
// ones admitted together share one batch launch), and retires launches as
// their events complete.  A request that finds nothing queued ahead of it and
// the scheduler idle is admitted and launched in the submitting thread.  PLAIN
// mode does planning, allocation and launch in the submitting thread on one
// stream.  The paper has no serving counterpart (Sec. 6 times one array at a
// time); every request runs the passes of Sec. 5.1 / 5.2 unchanged.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bmmc.h"
#include "bmmc_batch.h"
#include "bmmc_server.h"
#include "plan_internal.hpp"
#include "debug_hooks.hpp"

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxStreams = 32;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// An NVTX range for the scope (no cost unless a profiler is attached):
// submission, admission and retirement show on a profiler's timeline.
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
};

// First-fit allocator over one device block; free ranges kept coalesced.
class Arena {
public:
    void init(uint8_t *base, size_t size)
    {
        base_ = base;
        size_ = size;
        free_.clear();
        free_[0] = size;
    }
    void *alloc(size_t bytes)
    {
        bytes = align_up(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_ += bytes;
                return base_ + off;
            }
        }
        return nullptr;
    }
    void release(void *p, size_t bytes)
    {
        if (!p) return;
        bytes = align_up(bytes ? bytes : 1);
        size_t off = (uint8_t *)p - base_;
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }

private:
    uint8_t *base_ = nullptr;
    size_t size_ = 0;
    size_t used_ = 0;
    std::map<size_t, size_t> free_;
};

struct Req {
    uint64_t id = 0;
    const void *in = nullptr;
    bmmc_plan plan = nullptr;
    bool cached = false;     // plan belongs to the plan cache (pinned by this request)
    std::string key;         // its cache key
    size_t array_bytes = 0;  // 2^n * e
    size_t ws_bytes = 0;
    uint64_t bytes = 0;      // in + out + ws, for the budget
    void *out = nullptr;
    void *ws = nullptr;
    double submit_ms = 0;
    int status = BMMC_OK;
};

struct Launch {
    std::vector<Req *> reqs;
    cudaEvent_t ev = nullptr;
    bmmc_batch batch = nullptr;
    void *table = nullptr;
    size_t table_bytes = 0;
    void *group_ws = nullptr;
    size_t group_ws_bytes = 0;
};

}  // namespace

struct bmmc_server_s {
    bmmc_server_config cfg;
    int device = -1;
    int nstreams = 1;
    cudaStream_t streams[kMaxStreams] = {};
    cudaEvent_t start = nullptr;
    std::chrono::steady_clock::time_point t0;
    uint8_t *arena_mem = nullptr;
    Arena arena;           // guarded by sched_mu
    std::vector<cudaEvent_t> events;  // free events, guarded by sched_mu

    // submission side
    std::mutex mu;
    std::condition_variable cv;       // new submissions / stop
    std::condition_variable drained;  // outstanding reached 0
    std::deque<Req *> submitted;
    // requests the worker has taken from `submitted` and not yet queued in
    // `waiting` (set under mu, cleared under sched_mu)
    std::atomic<size_t> in_transit{0};
    std::vector<bmmc_server_result> results;
    uint64_t outstanding = 0;
    bool stop = false;
    bool hold = false;
    std::thread worker;

    // scheduler side (worker thread in CONTINUOUS; callers under sched_mu in PLAIN)
    std::mutex sched_mu;
    std::deque<Req *> waiting;
    std::deque<Launch> inflight[kMaxStreams];
    std::map<void *, size_t> kept;  // kept outputs and their sizes
    uint64_t used = 0;

    // Plan cache (plans are immutable, so requests for the same permutation
    // share one).  An entry used by a request in flight is pinned; when the
    // cache is full the least recently used unpinned entry is evicted.
    struct CachedPlan {
        bmmc_plan plan = nullptr;
        uint32_t refs = 0;
        std::list<const std::string *>::iterator lru;  // valid while refs == 0
    };
    std::mutex plan_mu;
    std::unordered_map<std::string, CachedPlan> plans;
    std::list<const std::string *> lru;  // unpinned entries, least recent first
    uint64_t n_plan_hits = 0;

    // counters
    uint64_t n_submitted = 0, n_completed = 0, n_single = 0, n_groups = 0,
             n_grouped = 0, peak_bytes = 0, peak_inflight = 0, n_inflight = 0,
             n_inline = 0;

    double now_ms() const
    {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
            .count();
    }
};

namespace {

cudaEvent_t take_event(bmmc_server_s *s)
{
    if (s->events.empty()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
    cudaEvent_t e = s->events.back();
    s->events.pop_back();
    return e;
}

// Give back a request's plan: unpin a cached one, destroy any other.
void release_plan(bmmc_server_s *s, Req *r)
{
    if (!r->plan) return;
    if (r->cached) {
        std::lock_guard<std::mutex> lk(s->plan_mu);
        auto it = s->plans.find(r->key);
        if (it != s->plans.end() && it->second.refs > 0 && --it->second.refs == 0)
            it->second.lru = s->lru.insert(s->lru.end(), &it->first);
    } else {
        bmmc_plan_destroy(r->plan);
    }
    r->plan = nullptr;
}

// Completion of one launch (sched_mu held).  Records results, frees bytes.
void finish(bmmc_server_s *s, Launch &L)
{
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s->start, L.ev);
    std::vector<bmmc_server_result> done;
    done.reserve(L.reqs.size());
    for (Req *r : L.reqs) {
        s->used -= r->bytes;
        if (r->ws) s->arena.release(r->ws, r->ws_bytes);
        bmmc_server_result res;
        res.id = r->id;
        res.status = r->status;
        res.submit_ms = r->submit_ms;
        res.done_ms = ms;
        res.out = r->out;
        if (!s->cfg.keep_outputs) {
            s->arena.release(r->out, r->array_bytes);
            res.out = nullptr;
        } else {
            s->kept[r->out] = r->array_bytes;
        }
        done.push_back(res);
        release_plan(s, r);
        delete r;
    }
    if (L.batch) bmmc_batch_destroy(L.batch);
    if (L.table) s->arena.release(L.table, L.table_bytes);
    if (L.group_ws) s->arena.release(L.group_ws, L.group_ws_bytes);
    s->events.push_back(L.ev);
    s->n_inflight -= L.reqs.size();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->results.insert(s->results.end(), done.begin(), done.end());
        s->n_completed += done.size();
        s->outstanding -= done.size();
        if (s->outstanding == 0) s->drained.notify_all();
    }
}

// Retire completed launches at the heads of the stream queues.
bool retire(bmmc_server_s *s)
{
    NvtxScope range("bmmc server retire");
    bool any = false;
    for (int i = 0; i < s->nstreams; ++i) {
        auto &q = s->inflight[i];
        while (!q.empty() && cudaEventQuery(q.front().ev) == cudaSuccess) {
            finish(s, q.front());
            q.pop_front();
            any = true;
        }
    }
    cudaGetLastError();  // clear cudaErrorNotReady
    return any;
}

// Launches in flight up to which a new request follows a large one on the
// priority stream (see stream_for).
constexpr uint64_t kFollowMax = 3;

int least_loaded(bmmc_server_s *s)
{
    int best = 0;
    for (int i = 1; i < s->nstreams; ++i)
        if (s->inflight[i].size() < s->inflight[best].size()) best = i;
    return best;
}

// The stream a request runs on.  With large_log2 set, a large request that
// is launched while at most one other launch is in flight (the server is
// nearly idle) runs on the high-priority stream 0, and requests that arrive
// while it runs, as long as few are in flight, queue behind it on that
// stream, as they would in the plain loop, instead of taking SMs and
// bandwidth from it.  Under load every request goes to the least loaded of
// streams 1..S-1: a large request on the priority stream would then hold back
// the many small ones queued behind it.
int stream_for(bmmc_server_s *s, const Req *r)
{
    if (s->cfg.large_log2 <= 0 || s->nstreams < 2) return least_loaded(s);
    if (r->array_bytes >= ((size_t)1 << s->cfg.large_log2) && s->n_inflight <= 1) return 0;
    if (!s->inflight[0].empty() && s->n_inflight <= kFollowMax) return 0;
    int best = 1;
    for (int i = 2; i < s->nstreams; ++i)
        if (s->inflight[i].size() < s->inflight[best].size()) best = i;
    return best;
}

void note_peaks(bmmc_server_s *s)
{
    s->peak_bytes = std::max<uint64_t>(s->peak_bytes, s->used);
    s->peak_inflight = std::max<uint64_t>(s->peak_inflight, s->n_inflight);
}

// Derive the tables a request's plan still lacks (sched_mu held: every
// launch, and so every completion of a plan, even a cached one shared by
// several requests, happens under it).
int complete_plan(bmmc_server_s *, Req *r) { return bmmc::plan_derive_rest(r->plan); }

// Launch one request on stream si (sched_mu held, buffers allocated).  A
// request that fails to launch still completes, with its error status, once
// the stream reaches its event.
void launch_single(bmmc_server_s *s, Req *r, int si)
{
    Launch L;
    L.ev = take_event(s);
    const bmmc_stream_t st = (bmmc_stream_t)s->streams[si];
    int rc;
    if (r->plan->derived < r->plan->npass) {
        // The first pass runs while the host derives the second pass's tables.
        rc = bmmc::plan_launch_pass(r->plan, 0, r->in, r->ws, st);
        if (rc == BMMC_OK) rc = complete_plan(s, r);
        if (rc == BMMC_OK) rc = bmmc::plan_launch_pass(r->plan, 1, r->ws, r->out, st);
    } else {
        rc = bmmc_execute_ws(r->plan, r->in, r->out, r->ws, st);
    }
    if (rc != BMMC_OK) r->status = rc;
    if (!L.ev || cudaEventRecord(L.ev, s->streams[si]) != cudaSuccess) {
        // no event: wait here so that completion is known
        cudaStreamSynchronize(s->streams[si]);
        if (!L.ev) cudaEventCreate(&L.ev);
        cudaEventRecord(L.ev, s->streams[si]);
        if (r->status == BMMC_OK) r->status = BMMC_ERR_CUDA;
    }
    L.reqs.push_back(r);
    s->inflight[si].push_back(L);
    s->n_single += 1;
    s->n_inflight += 1;
}

// Try to launch several admitted small requests as one batch.  On failure
// (no arena room for its tables) returns false and launches nothing.
bool launch_group(bmmc_server_s *s, std::vector<Req *> &g, int si)
{
    std::vector<bmmc_plan> plans;
    std::vector<const void *> ins;
    std::vector<void *> outs;
    for (Req *r : g)  // a batch takes complete plans only
        if (complete_plan(s, r) != BMMC_OK) return false;
    for (Req *r : g) {
        plans.push_back(r->plan);
        ins.push_back(r->in);
        outs.push_back(r->out);
    }
    Launch L;
    L.table_bytes = bmmc_batch_table_bytes(plans.data(), (int)g.size());
    L.group_ws_bytes = bmmc_batch_workspace_bytes(plans.data(), (int)g.size());
    L.table = s->arena.alloc(L.table_bytes);
    if (!L.table) return false;
    if (L.group_ws_bytes) {
        L.group_ws = s->arena.alloc(L.group_ws_bytes);
        if (!L.group_ws) {
            s->arena.release(L.table, L.table_bytes);
            return false;
        }
    }
    int rc = bmmc_batch_create(&L.batch, plans.data(), (int)g.size(), ins.data(), outs.data(),
                               L.group_ws, L.table, (bmmc_stream_t)s->streams[si]);
    if (rc != BMMC_OK) {
        s->arena.release(L.table, L.table_bytes);
        if (L.group_ws) s->arena.release(L.group_ws, L.group_ws_bytes);
        return false;
    }
    L.ev = take_event(s);
    if (!L.ev) {
        bmmc_batch_destroy(L.batch);
        s->arena.release(L.table, L.table_bytes);
        if (L.group_ws) s->arena.release(L.group_ws, L.group_ws_bytes);
        return false;
    }
    const int rc_exec = bmmc_batch_execute(L.batch, (bmmc_stream_t)s->streams[si]);
    cudaEventRecord(L.ev, s->streams[si]);
    if (rc_exec != BMMC_OK)
        for (Req *r : g) r->status = rc_exec;
    // grouped requests use the group workspace, not their own
    for (Req *r : g) {
        if (r->ws) s->arena.release(r->ws, r->ws_bytes);
        r->ws = nullptr;
    }
    L.reqs = g;
    s->inflight[si].push_back(L);
    s->n_groups += 1;
    s->n_grouped += g.size();
    s->n_inflight += g.size();
    return true;
}

// Allocate a request's output (and workspace); false if the arena is full.
bool allocate(bmmc_server_s *s, Req *r)
{
    r->out = s->arena.alloc(r->array_bytes);
    if (!r->out) return false;
    if (r->ws_bytes) {
        r->ws = s->arena.alloc(r->ws_bytes);
        if (!r->ws) {
            s->arena.release(r->out, r->array_bytes);
            r->out = nullptr;
            return false;
        }
    }
    return true;
}

// Admit waiting requests in order while they fit; launch them.  Returns true
// if anything was launched.
bool admit(bmmc_server_s *s)
{
    NvtxScope range("bmmc server admit");
    std::vector<Req *> admitted;
    while (!s->waiting.empty()) {
        Req *r = s->waiting.front();
        const bool idle = (s->used == 0 && admitted.empty());
        if (!idle && s->used + r->bytes > s->cfg.budget_bytes) break;
        if (!allocate(s, r)) break;
        s->waiting.pop_front();
        s->used += r->bytes;
        admitted.push_back(r);
    }
    if (admitted.empty()) return false;
    std::vector<Req *> small;
    for (Req *r : admitted) {
        if (s->cfg.group_max_bytes && r->array_bytes <= s->cfg.group_max_bytes)
            small.push_back(r);
    }
    const bool group = s->cfg.group_min > 0 && (int)small.size() >= s->cfg.group_min;
    if (group && launch_group(s, small, least_loaded(s))) {
        for (Req *r : admitted)
            if (r->array_bytes > s->cfg.group_max_bytes)
                launch_single(s, r, stream_for(s, r));
    } else {
        for (Req *r : admitted) launch_single(s, r, stream_for(s, r));
    }
    note_peaks(s);
    return true;
}

// Admit and launch one request now if the budget and the arena allow
// (sched_mu held, nothing waiting ahead of it).
bool admit_one(bmmc_server_s *s, Req *r)
{
    const bool idle = s->used == 0;
    if (!idle && s->used + r->bytes > s->cfg.budget_bytes) return false;
    if (!allocate(s, r)) return false;
    s->used += r->bytes;
    launch_single(s, r, stream_for(s, r));
    note_peaks(s);
    return true;
}

// Make the server's device current in the calling thread; returns the
// device to restore (or -1).
int enter_device(const bmmc_server_s *s)
{
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return -1;
    if (cur == s->device) return -1;
    cudaSetDevice(s->device);
    return cur;
}

void worker_main(bmmc_server_s *s)
{
    cudaSetDevice(s->device);
    // Requests taken from `submitted` and not yet queued in `waiting`; kept
    // across turns so that a failed host allocation loses none of them.
    std::deque<Req *> fresh;
    for (;;) {
        // blocked: requests wait for admission (poll completions at once);
        // busy: launches in flight (retire them, but no hurry: latency comes
        // from CUDA events, and polling beside the submitting thread slows its
        // launches)
        bool busy, blocked;
        {
            std::lock_guard<std::mutex> lk2(s->sched_mu);
            blocked = !s->waiting.empty() || !fresh.empty();
            busy = blocked || s->n_inflight != 0;
        }
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if ((!blocked && s->submitted.empty()) || (s->hold && !s->stop)) {
                if (s->stop && s->submitted.empty() && !busy) return;
                if (busy) s->cv.wait_for(lk, std::chrono::microseconds(100));
                else s->cv.wait_for(lk, std::chrono::milliseconds(1));
                if (s->hold && !s->stop) {
                    lk.unlock();
                    std::lock_guard<std::mutex> lk2(s->sched_mu);
                    retire(s);  // keep retiring while admission is held
                    continue;
                }
            }
            if (fresh.empty()) fresh.swap(s->submitted);
            s->in_transit.store(fresh.size());
        }
        std::lock_guard<std::mutex> lk2(s->sched_mu);
        try {
            while (!fresh.empty()) {
                s->waiting.push_back(fresh.front());
                fresh.pop_front();
            }
            s->in_transit.store(0);
            bool progress = retire(s);
            progress |= admit(s);
            if (!progress && s->n_inflight) std::this_thread::yield();
        } catch (const std::bad_alloc &) {
            // Host memory ran out while queueing or admitting: what is not
            // queued yet stays in `fresh` (still counted in transit, so no
            // later request overtakes it) and the next turn retries, instead
            // of this thread ending the process.
            std::this_thread::yield();
        }
    }
}

// Put a new plan in the cache (plan_mu held), evicting the least recently
// used unpinned entry if the cache is full.  False if every entry is pinned.
bool cache_insert(bmmc_server_s *s, const std::string &key, bmmc_plan plan)
{
    if (s->plans.size() >= (size_t)s->cfg.plan_cache) {
        if (s->lru.empty()) return false;
        const std::string victim = *s->lru.front();
        s->lru.pop_front();
        auto it = s->plans.find(victim);
        bmmc_plan_destroy(it->second.plan);
        s->plans.erase(it);
    }
    auto &ent = s->plans[key];
    ent.plan = plan;
    ent.refs = 1;
    return true;
}

// Pin a cached entry for one more request (plan_mu held).
bmmc_plan cache_pin(bmmc_server_s *s, bmmc_server_s::CachedPlan &ent)
{
    if (ent.refs++ == 0) s->lru.erase(ent.lru);
    return ent.plan;
}

// Plan a request (caller's thread), through the plan cache if it has one.
int prepare(bmmc_server_s *s, Req *r, int n, const uint64_t *rows, uint64_t c, size_t e)
{
    const bool use_cache = s->cfg.plan_cache > 0 && n >= 1 && n <= 64;
    if (use_cache) {
        // key: n, e, c and the rows, as raw bytes (the flags are the server's)
        r->key.resize(sizeof(int) + sizeof(size_t) + sizeof(uint64_t) * (1 + (size_t)n));
        char *k = &r->key[0];
        memcpy(k, &n, sizeof(int));
        memcpy(k + sizeof(int), &e, sizeof(size_t));
        memcpy(k + sizeof(int) + sizeof(size_t), &c, sizeof(uint64_t));
        memcpy(k + sizeof(int) + sizeof(size_t) + sizeof(uint64_t), rows,
               sizeof(uint64_t) * (size_t)n);
        std::lock_guard<std::mutex> lk(s->plan_mu);
        auto it = s->plans.find(r->key);
        if (it != s->plans.end()) {
            r->plan = cache_pin(s, it->second);
            r->cached = true;
            s->n_plan_hits += 1;
        }
    }
    if (!r->plan) {
        bmmc_plan_options o;
        memset(&o, 0, sizeof(o));
        o.flags = s->cfg.plan_flags;
        bmmc_plan p = nullptr;
        // Continuous mode plans the first pass only: the second pass's tables
        // are derived at launch, while the first pass runs.
        const bool staged = s->cfg.mode == BMMC_SERVER_CONTINUOUS;
        int rc = staged ? bmmc::plan_create_first_pass(&p, n, rows, c, e, &o)
                        : bmmc_plan_create_ex(&p, n, rows, c, e, &o);
        if (rc != BMMC_OK) return rc;
        r->plan = p;
        if (use_cache) {
            std::lock_guard<std::mutex> lk(s->plan_mu);
            auto it = s->plans.find(r->key);
            if (it != s->plans.end()) {  // planned meanwhile by another thread
                bmmc_plan_destroy(p);
                r->plan = cache_pin(s, it->second);
                r->cached = true;
            } else {
                r->cached = cache_insert(s, r->key, p);
            }
        }
    }
    r->array_bytes = ((size_t)1 << n) * e;
    r->ws_bytes = bmmc_plan_workspace_bytes(r->plan);
    r->bytes = 2 * (uint64_t)r->array_bytes + r->ws_bytes;
    if (align_up(r->array_bytes) + align_up(r->ws_bytes) > s->arena.size()) {
        release_plan(s, r);
        return BMMC_ERR_TOO_LARGE;
    }
    return BMMC_OK;
}

}  // namespace

extern "C" {

int bmmc_server_create(bmmc_server *out, const bmmc_server_config *cfg)
{
    try {
        if (!out || !cfg) return BMMC_ERR_INVALID;
        *out = nullptr;
        for (int r : cfg->reserved)
            if (r) return BMMC_ERR_UNSUPPORTED;
        if (cfg->mode != BMMC_SERVER_CONTINUOUS && cfg->mode != BMMC_SERVER_PLAIN)
            return BMMC_ERR_UNSUPPORTED;
        if (cfg->streams < 1 || cfg->streams > kMaxStreams) return BMMC_ERR_UNSUPPORTED;
        if (cfg->arena_bytes < kAlign || cfg->budget_bytes == 0) return BMMC_ERR_UNSUPPORTED;
        if (cfg->plan_flags > BMMC_PLAN_SINGLE_PASS) return BMMC_ERR_UNSUPPORTED;
        if (cfg->plan_cache < 0) return BMMC_ERR_UNSUPPORTED;
        bmmc_server_s *s = new (std::nothrow) bmmc_server_s();
        if (!s) return BMMC_ERR_OOM;
        s->cfg = *cfg;
        s->nstreams = cfg->mode == BMMC_SERVER_PLAIN ? 1 : cfg->streams;
        if (cudaGetDevice(&s->device) != cudaSuccess) {
            delete s;
            return BMMC_ERR_CUDA;
        }
        if (bmmc::debug_fail_alloc() ||
            cudaMalloc((void **)&s->arena_mem, cfg->arena_bytes) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return BMMC_ERR_OOM;
        }
        s->arena.init(s->arena_mem, cfg->arena_bytes);
        int prio_low = 0, prio_high = 0;
        cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
        for (int i = 0; i < s->nstreams; ++i) {
            const bool high = i == 0 && s->cfg.large_log2 > 0 && s->nstreams >= 2 &&
                              s->cfg.mode == BMMC_SERVER_CONTINUOUS;
            cudaStreamCreateWithPriority(&s->streams[i], cudaStreamNonBlocking,
                                         high ? prio_high : prio_low);
        }
        for (int i = 0; i < 64; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) == cudaSuccess) s->events.push_back(e);
        }
        cudaEventCreate(&s->start);
        cudaDeviceSynchronize();
        cudaEventRecord(s->start, s->streams[0]);
        cudaEventSynchronize(s->start);
        s->t0 = std::chrono::steady_clock::now();
        if (cudaGetLastError() != cudaSuccess) {
            bmmc_server_destroy(s);
            return BMMC_ERR_CUDA;
        }
        if (cfg->mode == BMMC_SERVER_CONTINUOUS) s->worker = std::thread(worker_main, s);
        *out = s;
        return BMMC_OK;
    } catch (const std::bad_alloc &) {
        return BMMC_ERR_OOM;
    } catch (...) {
        return BMMC_ERR_INVALID;
    }
}

int bmmc_server_submit(bmmc_server s, uint64_t id, int n, const uint64_t *A_rows, uint64_t c,
                       size_t elem_bytes, const void *in)
{
    NvtxScope range("bmmc server submit");
    try {
        if (!s || !in) return BMMC_ERR_INVALID;
        if ((uintptr_t)in & 15u) return BMMC_ERR_ALIGN;
        Req *r = new (std::nothrow) Req();
        if (!r) return BMMC_ERR_OOM;
        r->id = id;
        r->in = in;
        r->submit_ms = s->now_ms();
        int rc = prepare(s, r, n, A_rows, c, elem_bytes);
        if (rc != BMMC_OK) {
            delete r;
            return rc;
        }
        if (s->cfg.mode == BMMC_SERVER_CONTINUOUS) {
            auto enqueue = [s, r]() {
                std::lock_guard<std::mutex> lk(s->mu);
                s->submitted.push_back(r);
                s->cv.notify_one();
                return BMMC_OK;
            };
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->outstanding += 1;
                s->n_submitted += 1;
                if (s->hold || s->stop || !s->submitted.empty()) {
                    s->submitted.push_back(r);
                    s->cv.notify_one();
                    return BMMC_OK;
                }
            }
            // Inline dispatch: when nothing submitted earlier is still queued
            // and the scheduler is not busy, admit and launch in this thread, as
            // the plain loop would, instead of waking the scheduler.  Requests
            // taken by the scheduler but not yet queued (in_transit) keep their
            // place: this one then queues behind them.
            std::unique_lock<std::mutex> lk2(s->sched_mu, std::try_to_lock);
            if (!lk2.owns_lock() || s->in_transit.load() != 0) {
                if (lk2.owns_lock()) lk2.unlock();
                return enqueue();
            }
            bool launched = false;
            if (s->waiting.empty()) {
                const int prev = enter_device(s);
                // launch first; retire finished launches after it (or before
                // a second try when the budget or the arena was full), so that
                // their bookkeeping does not delay this request
                launched = admit_one(s, r);
                retire(s);
                if (!launched) launched = admit_one(s, r);
                if (prev >= 0) cudaSetDevice(prev);
            }
            if (!launched) s->waiting.push_back(r);
            if (launched) s->n_inline += 1;
            lk2.unlock();
            if (!launched) {
                std::lock_guard<std::mutex> lk(s->mu);
                s->cv.notify_one();  // the scheduler admits r when room frees
            }
            // a launched request is retired by the scheduler's next turn (at
            // most 100 us away) or by the next submission
            return BMMC_OK;
        }
        // PLAIN: allocate (waiting for completions if the arena is full), launch.
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->outstanding += 1;
            s->n_submitted += 1;
        }
        std::lock_guard<std::mutex> lk(s->sched_mu);
        retire(s);
        while (!allocate(s, r)) {
            if (s->inflight[0].empty()) {  // cannot happen: prepare checked the size
                release_plan(s, r);
                delete r;
                return BMMC_ERR_OOM;
            }
            cudaEventSynchronize(s->inflight[0].front().ev);
            retire(s);
        }
        s->used += r->bytes;
        launch_single(s, r, 0);
        note_peaks(s);
        return BMMC_OK;
    } catch (const std::bad_alloc &) {
        return BMMC_ERR_OOM;
    } catch (...) {
        return BMMC_ERR_INVALID;
    }
}

int bmmc_server_drain(bmmc_server s)
{
    if (!s) return BMMC_ERR_INVALID;
    if (s->cfg.mode == BMMC_SERVER_CONTINUOUS) {
        std::unique_lock<std::mutex> lk(s->mu);
        s->drained.wait(lk, [s] { return s->outstanding == 0; });
        return BMMC_OK;
    }
    std::lock_guard<std::mutex> lk(s->sched_mu);
    while (!s->inflight[0].empty()) {
        cudaEventSynchronize(s->inflight[0].front().ev);
        retire(s);
    }
    return BMMC_OK;
}

int bmmc_server_hold(bmmc_server s, int hold)
{
    if (!s) return BMMC_ERR_INVALID;
    if (s->cfg.mode != BMMC_SERVER_CONTINUOUS) return BMMC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(s->mu);
    s->hold = hold != 0;
    s->cv.notify_all();
    return BMMC_OK;
}

double bmmc_server_now_ms(bmmc_server s) { return s ? s->now_ms() : -1.0; }

int bmmc_server_results(bmmc_server s, bmmc_server_result *res, int max)
{
    try {
        if (!s || (!res && max > 0) || max < 0) return BMMC_ERR_INVALID;
        std::lock_guard<std::mutex> lk(s->mu);
        int k = (int)std::min<size_t>((size_t)max, s->results.size());
        for (int i = 0; i < k; ++i) res[i] = s->results[i];
        s->results.erase(s->results.begin(), s->results.begin() + k);
        return k;
    } catch (const std::bad_alloc &) {
        return BMMC_ERR_OOM;
    } catch (...) {
        return BMMC_ERR_INVALID;
    }
}

int bmmc_server_release(bmmc_server s, void *out)
{
    if (!s || !out) return BMMC_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->sched_mu);
    auto it = s->kept.find(out);
    if (it == s->kept.end()) return BMMC_ERR_INVALID;
    s->arena.release(it->first, it->second);
    s->kept.erase(it);
    return BMMC_OK;
}

int bmmc_server_stats(bmmc_server s, char *buf, size_t len)
{
    try {
        if (!s) return BMMC_ERR_INVALID;
        char tmp[768];
        uint64_t single, inl, groups, grouped, peak_b, peak_i, sub, comp, hits, cached;
        {
            std::lock_guard<std::mutex> lk(s->sched_mu);
            single = s->n_single;
            inl = s->n_inline;
            groups = s->n_groups;
            grouped = s->n_grouped;
            peak_b = s->peak_bytes;
            peak_i = s->peak_inflight;
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            sub = s->n_submitted;
            comp = s->n_completed;
        }
        {
            std::lock_guard<std::mutex> lk(s->plan_mu);
            hits = s->n_plan_hits;
            cached = s->plans.size();
        }
        int k = snprintf(tmp, sizeof(tmp),
                         "{\"mode\": \"%s\", \"streams\": %d, \"submitted\": %llu, "
                         "\"completed\": %llu, \"single_launches\": %llu, "
                         "\"inline_launches\": %llu, "
                         "\"group_launches\": %llu, \"grouped_requests\": %llu, "
                         "\"peak_bytes_in_flight\": %llu, \"peak_requests_in_flight\": %llu, "
                         "\"plan_cache_hits\": %llu, \"plans_cached\": %llu}",
                         s->cfg.mode == BMMC_SERVER_PLAIN ? "plain" : "continuous", s->nstreams,
                         (unsigned long long)sub, (unsigned long long)comp,
                         (unsigned long long)single, (unsigned long long)inl,
                         (unsigned long long)groups,
                         (unsigned long long)grouped, (unsigned long long)peak_b,
                         (unsigned long long)peak_i, (unsigned long long)hits,
                         (unsigned long long)cached);
        if (buf && len) {
            size_t cpy = (size_t)k < len - 1 ? (size_t)k : len - 1;
            memcpy(buf, tmp, cpy);
            buf[cpy] = 0;
        }
        return k;
    } catch (const std::bad_alloc &) {
        return BMMC_ERR_OOM;
    } catch (...) {
        return BMMC_ERR_INVALID;
    }
}

void bmmc_server_destroy(bmmc_server s)
{
    if (!s) return;
    if (s->worker.joinable()) {
        bmmc_server_hold(s, 0);
        bmmc_server_drain(s);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
            s->cv.notify_all();
        }
        s->worker.join();
    } else if (s->cfg.mode == BMMC_SERVER_PLAIN) {
        bmmc_server_drain(s);
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (s->device >= 0) cudaSetDevice(s->device);
    for (int i = 0; i < s->nstreams; ++i)
        if (s->streams[i]) cudaStreamDestroy(s->streams[i]);
    for (cudaEvent_t e : s->events) cudaEventDestroy(e);
    if (s->start) cudaEventDestroy(s->start);
    if (s->arena_mem) cudaFree(s->arena_mem);
    if (prev >= 0) cudaSetDevice(prev);
    for (auto &kv : s->plans) bmmc_plan_destroy(kv.second.plan);
    delete s;
}

}  // extern "C"
