// engine.cu -- concurrent searches: a pool of worker threads, each with its own
// CUDA stream, fed from one request queue and admitted against one budget of
// device memory.
//
// The paper runs one search at a time.  On one GB300 a search of a short
// series is latency-bound (tens of small kernels, a few microseconds each),
// so many of them are run side by side: each worker enqueues its request's
// kernels on its own stream, and the GPU overlaps the streams.
//
// Memory: the engine allocates one device arena of its budget at creation and
// hands out blocks of it on the host (first fit, 256-byte aligned, coalescing
// free list): every plan lives in a block of exactly its footprint
// (dd_plan_footprint), a host series is staged in a block of 4 m bytes.  A
// request is admitted when its blocks can be allocated, so the workspaces in
// use (resident plans of idle workers included) never exceed the budget.  A
// worker keeps its last plan and reuses it for the same (m, n); a worker that
// finds nothing admissible releases what it holds, so that resident plans
// never block a request.
// Scheduling: a worker takes the first queued request that fits; a request that
// does not fit is passed over by smaller ones behind it, at most kMaxBypass
// times, after which nothing is admitted past it until it fits.

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "dd_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxBypass = 32;

struct Request {
    int64_t id;
    const float* T;
    int64_t m;
    int32_t n;
    int32_t flags;
    Clock::time_point submitted;
    size_t need;   // plan footprint (0: invalid sizes, fails without memory)
    int bypassed;  // times a later request was admitted before this one
};

// Blocks of the engine's device arena, handed out on the host: first fit over a
// free list ordered by offset, adjacent free blocks merged on release.
class Arena {
public:
    static constexpr size_t kAlignA = 256;
    void reset(size_t bytes) {
        free_.clear();
        if (bytes) free_[0] = bytes;
    }
    static size_t round(size_t b) { return (b + kAlignA - 1) / kAlignA * kAlignA; }
    // offset of a new block of b bytes, or SIZE_MAX
    size_t alloc(size_t b) {
        b = round(b);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < b) continue;
            const size_t off = it->first, rest = it->second - b;
            free_.erase(it);
            if (rest) free_[off + b] = rest;
            return off;
        }
        return SIZE_MAX;
    }
    // takes exactly [off, off + b) if it lies inside one free block (undoing a release)
    bool alloc_at(size_t off, size_t b) {
        b = round(b);
        auto it = free_.upper_bound(off);
        if (it == free_.begin()) return false;
        --it;
        const size_t s0 = it->first, sz = it->second;
        if (s0 > off || s0 + sz < off + b) return false;
        free_.erase(it);
        if (off > s0) free_[s0] = off - s0;
        if (s0 + sz > off + b) free_[off + b] = s0 + sz - (off + b);
        return true;
    }
    void release(size_t off, size_t b) {
        b = round(b);
        auto it = free_.emplace(off, b).first;
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
    std::map<size_t, size_t> free_;  // offset -> bytes
};

struct Worker {
    std::thread thread;
    cudaStream_t stream = nullptr;
    dd::PlanShared shared{};           // side stream and fork / join events lent to the worker's plans
    size_t ws_off = SIZE_MAX;          // arena block of the resident plan's workspace
    size_t ws_bytes = 0;
    size_t stage_off = SIZE_MAX;       // arena block of the device copy of a host series
    size_t stage_bytes = 0;
    dd_result_t* res_dev = nullptr;
    dd_result_t* res_host = nullptr;   // pinned
    dd_plan_s* plan = nullptr;         // last plan, reused for the same (m, n)
    size_t held() const { return ws_bytes + stage_bytes; }
};

// Device bytes of the plan of any series with m <= m_max, n <= n_max.  The
// footprint grows with m.  For fixed m it falls with n (fewer subsequences)
// except where it steps up: while n < paa_w the SAX dictionary grows with n
// (words have min(paa_w, n) letters), and the padded tensor-core row length
// grows by 64 at n = 65, 129, ...  So the largest footprint is at one of
// those n.
size_t max_footprint(int64_t m_max, int32_t n_max, const dd_options_t* o) {
    size_t best = dd_plan_footprint(m_max, n_max, o);
    auto take = [&](int64_t n) {
        if (n < 1 || n > n_max) return;
        const size_t f = dd_plan_footprint(m_max, (int32_t)n, o);
        if (f > best) best = f;
    };
    for (int64_t n = 1; n <= o->paa_w; n++) take(n);
    for (int64_t n = 65; n <= n_max; n += 64) take(n);
    return best;
}

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

size_t stage_need(const Request& r) { return (r.flags & DD_SERIES_HOST) ? sizeof(float) * (size_t)r.m : 0; }

}  // namespace

struct dd_engine_s {
    int device = 0;
    dd_options_t opt{};
    int64_t m_max = 0;
    size_t budget = 0;                 // device bytes of the arena
    char* arena_base = nullptr;
    Arena arena;                       // guarded by mu
    std::vector<Worker> workers;
    std::mutex mu;
    std::condition_variable cv_work;   // queue changed, memory freed, or stopping
    std::condition_variable cv_done;   // a completion arrived
    std::deque<Request> queue;
    std::deque<dd_completion_t> done;
    int64_t outstanding = 0;
    bool stopping = false;

    void run(Worker& w);
    bool pick(Worker& w, Request& r);
    void release(Worker& w);
    dd_result_t serve(Worker& w, const Request& r);
};

namespace {

dd_result_t failed(dd_status_t st) {
    dd_result_t r;
    std::memset(&r, 0, sizeof(r));
    r.index = -1;
    r.status = st;
    return r;
}

}  // namespace

// Frees the worker's plan and arena blocks (its stream is idle).  Caller holds mu.
void dd_engine_s::release(Worker& w) {
    dd::destroy_plan(w.plan, false);
    w.plan = nullptr;
    if (w.ws_off != SIZE_MAX) arena.release(w.ws_off, w.ws_bytes);
    if (w.stage_off != SIZE_MAX) arena.release(w.stage_off, w.stage_bytes);
    w.ws_off = w.stage_off = SIZE_MAX;
    w.ws_bytes = w.stage_bytes = 0;
}

// Chooses the next request for worker w and allocates its blocks (caller holds
// mu): the first queued request whose blocks can be allocated, passing over at
// most kMaxBypass times a request whose cannot.  A request that cannot succeed
// (invalid sizes, more than the whole budget) is taken at once and fails
// without memory.  On success the request leaves the queue.
bool dd_engine_s::pick(Worker& w, Request& r) {
    for (size_t k = 0; k < queue.size(); k++) {
        Request& q = queue[k];
        bool take = false;
        if (q.need == 0 || Arena::round(q.need) + Arena::round(stage_need(q)) > budget ||
            ((q.flags & DD_SERIES_HOST) && q.m > m_max)) {
            take = true;
        } else {
            const bool same = w.plan && w.plan->m == q.m && w.plan->n == q.n;
            // a new plan replaces the resident one: its block is free for the new one
            const size_t old_off = w.ws_off, old_bytes = w.ws_bytes;
            size_t ws_off = w.ws_off;
            if (!same) {
                if (old_off != SIZE_MAX) arena.release(old_off, old_bytes);
                ws_off = arena.alloc(q.need);
            }
            size_t st_off = w.stage_off;
            bool ok = ws_off != SIZE_MAX;
            const bool grow_stage = stage_need(q) > w.stage_bytes;
            if (ok && grow_stage) {
                if (w.stage_off != SIZE_MAX) arena.release(w.stage_off, w.stage_bytes);
                st_off = arena.alloc(stage_need(q));
                if (st_off == SIZE_MAX) {
                    ok = false;
                    // put the old staging block back where it was (just freed, nobody took it)
                    if (w.stage_off != SIZE_MAX) arena.alloc_at(w.stage_off, w.stage_bytes);
                }
            }
            if (!ok) {
                if (!same) {
                    if (ws_off != SIZE_MAX) arena.release(ws_off, q.need);
                    if (old_off != SIZE_MAX) arena.alloc_at(old_off, old_bytes);
                }
            } else {
                if (!same) {
                    dd::destroy_plan(w.plan, false);  // its block now belongs to the new plan
                    w.plan = nullptr;
                    w.ws_off = ws_off;
                    w.ws_bytes = q.need;
                }
                if (grow_stage) {
                    w.stage_off = st_off;
                    w.stage_bytes = stage_need(q);
                }
                take = true;
            }
        }
        if (take) {
            r = q;
            for (size_t j = 0; j < k; j++) queue[j].bypassed++;
            queue.erase(queue.begin() + (long)k);
            return true;
        }
        if (q.bypassed >= kMaxBypass) return false;  // nothing goes past a starved request
    }
    return false;
}

dd_result_t dd_engine_s::serve(Worker& w, const Request& r) {
    if (r.n < 1 || r.m < 1 || r.need == 0) return failed(DD_EINVAL);
    if (Arena::round(r.need) + Arena::round(stage_need(r)) > budget || ((r.flags & DD_SERIES_HOST) && r.m > m_max))
        return failed(DD_ENOMEM);
    if (!w.plan) {
        const dd_status_t st = dd::create_plan(&w.plan, r.m, r.n, &opt, arena_base + w.ws_off, w.ws_bytes, true,
                                               w.stream, &w.shared);
        if (st != DD_OK) {
            w.plan = nullptr;
            return failed(st);
        }
    }
    const float* src = r.T;
    cudaError_t e = cudaSuccess;
    if (r.flags & DD_SERIES_HOST) {
        float* stage = reinterpret_cast<float*>(arena_base + w.stage_off);
        e = cudaMemcpyAsync(stage, r.T, sizeof(float) * (size_t)r.m, cudaMemcpyHostToDevice, w.stream);
        src = stage;
    }
    if (e != cudaSuccess) return failed(DD_ECUDA);
    dd_status_t st = dd_find_discord_async(w.plan, src, w.res_dev, w.stream);
    if (st != DD_OK) return failed(st);
    e = cudaMemcpyAsync(w.res_host, w.res_dev, sizeof(dd_result_t), cudaMemcpyDeviceToHost, w.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return failed(DD_ECUDA);
    }
    return *w.res_host;
}

void dd_engine_s::run(Worker& w) {
    cudaSetDevice(device);
    for (;;) {
        Request r;
        {
            std::unique_lock<std::mutex> lk(mu);
            for (;;) {
                if (stopping) return;
                if (pick(w, r)) break;
                if (!queue.empty() && w.held() > 0) {
                    // nothing fits while this worker holds memory: give it back and look again
                    release(w);
                    cv_work.notify_all();
                    continue;
                }
                cv_work.wait(lk);
            }
        }
        const Clock::time_point t0 = Clock::now();
        dd_completion_t c;
        std::memset(&c, 0, sizeof(c));
        c.id = r.id;
        c.result = serve(w, r);
        const Clock::time_point t1 = Clock::now();
        c.queue_ms = ms_between(r.submitted, t0);
        c.service_ms = ms_between(t0, t1);
        {
            std::lock_guard<std::mutex> lk(mu);
            done.push_back(c);
        }
        cv_done.notify_all();
        cv_work.notify_all();  // memory may have been freed
    }
}

extern "C" {

dd_status_t dd_engine_create_budget(dd_engine_t* engine, int32_t workers, const dd_options_t* opt, int64_t m_max,
                                    int32_t n_max, size_t budget_bytes) {
    if (!engine) return DD_EINVAL;
    *engine = nullptr;
    if (workers < 1 || workers > 64) return DD_EINVAL;
    dd_options_t o;
    if (opt)
        o = *opt;
    else
        dd_options_default(&o);
    if (dd_plan_footprint(m_max, n_max, &o) == 0) return DD_EINVAL;
    dd_engine_s* E = new (std::nothrow) dd_engine_s();
    if (!E) return DD_ENOMEM;
    E->opt = o;
    E->m_max = m_max;
    E->budget = budget_bytes ? budget_bytes
                             : (size_t)workers * (max_footprint(m_max, n_max, &o) + sizeof(float) * (size_t)m_max);
    E->budget = Arena::round(E->budget);
    cudaError_t e = cudaGetDevice(&E->device);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&E->arena_base), E->budget);
    if (e == cudaSuccess) E->arena.reset(E->budget);
    E->workers.resize((size_t)workers);
    for (Worker& w : E->workers) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w.shared.side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.shared.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.shared.join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&w.res_dev), sizeof(dd_result_t));
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&w.res_host), sizeof(dd_result_t));
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        dd_engine_destroy(E);
        return e == cudaErrorMemoryAllocation ? DD_ENOMEM : DD_ECUDA;
    }
    for (Worker& w : E->workers) w.thread = std::thread([E, &w] { E->run(w); });
    *engine = E;
    return DD_OK;
}

dd_status_t dd_engine_create(dd_engine_t* engine, int32_t workers, const dd_options_t* opt, int64_t m_max,
                             int32_t n_max) {
    return dd_engine_create_budget(engine, workers, opt, m_max, n_max, 0);
}

dd_status_t dd_engine_submit(dd_engine_t E, int64_t id, const float* T, int64_t m, int32_t n, int32_t flags) {
    if (!E || !T || (flags != DD_SERIES_DEVICE && flags != DD_SERIES_HOST)) return DD_EINVAL;
    {
        std::lock_guard<std::mutex> lk(E->mu);
        if (E->stopping) return DD_EBUSY;
        E->queue.push_back(Request{id, T, m, n, flags, Clock::now(), dd_plan_footprint(m, n, &E->opt), 0});
        E->outstanding++;
    }
    E->cv_work.notify_one();
    return DD_OK;
}

int32_t dd_engine_poll(dd_engine_t E, dd_completion_t* out, int32_t cap, int32_t wait_ms) {
    if (!E || (cap > 0 && !out) || cap < 0) return -DD_EINVAL;
    std::unique_lock<std::mutex> lk(E->mu);
    // nothing queued, running or finished: nothing to wait for
    if (E->done.empty() && E->outstanding == 0) return 0;
    if (E->done.empty() && wait_ms != 0) {
        auto ready = [&] { return !E->done.empty(); };
        if (wait_ms < 0)
            E->cv_done.wait(lk, ready);
        else
            E->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
    }
    int32_t k = 0;
    while (k < cap && !E->done.empty()) {
        out[k++] = E->done.front();
        E->done.pop_front();
    }
    E->outstanding -= k;
    return k;
}

int64_t dd_engine_outstanding(dd_engine_t E) {
    if (!E) return 0;
    std::lock_guard<std::mutex> lk(E->mu);
    return E->outstanding;
}

void dd_engine_destroy(dd_engine_t E) {
    if (!E) return;
    {
        std::lock_guard<std::mutex> lk(E->mu);
        E->stopping = true;
        E->queue.clear();
    }
    E->cv_work.notify_all();
    for (Worker& w : E->workers)
        if (w.thread.joinable()) w.thread.join();
    for (Worker& w : E->workers) {
        if (w.stream) cudaStreamSynchronize(w.stream);
        if (w.stream) E->release(w);
        if (w.stream) cudaStreamSynchronize(w.stream);
        if (w.res_dev) cudaFree(w.res_dev);
        if (w.res_host) cudaFreeHost(w.res_host);
        if (w.shared.side) cudaStreamDestroy(w.shared.side);
        if (w.shared.fork) cudaEventDestroy(w.shared.fork);
        if (w.shared.join) cudaEventDestroy(w.shared.join);
        if (w.stream) cudaStreamDestroy(w.stream);
    }
    if (E->arena_base) cudaFree(E->arena_base);
    delete E;
}

}  // extern "C"
