// engine.cu -- concurrent searches: a pool of worker threads, each with its own
// CUDA stream, device workspace and plan, fed from one FIFO request queue.
//
// The paper runs one search at a time.  On one GB300 a search of a short
// series is latency-bound (tens of small kernels, a few microseconds each),
// so many of them are run side by side: each worker enqueues its request's
// kernels on its own stream, and the GPU overlaps the streams.  A worker
// keeps its last plan and reuses it for the same (m, n); a new shape builds
// a plan inside the worker's workspace, initialised on the worker's stream,
// so no worker waits for another one's searches.

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "dd_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id;
    const float* T;
    int64_t m;
    int32_t n;
    int32_t flags;
    Clock::time_point submitted;
};

struct Worker {
    std::thread thread;
    cudaStream_t stream = nullptr;
    void* ws = nullptr;                // plan workspace
    size_t ws_bytes = 0;
    float* stage = nullptr;            // device copy of host series
    dd_result_t* res_dev = nullptr;
    dd_result_t* res_host = nullptr;   // pinned
    dd_plan_s* plan = nullptr;         // last plan, reused for the same (m, n)
};

// Device bytes that fit a plan of any series with m <= m_max, n <= n_max.  The
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

}  // namespace

struct dd_engine_s {
    int device = 0;
    dd_options_t opt{};
    int64_t m_max = 0;
    std::vector<Worker> workers;
    std::mutex mu;
    std::condition_variable cv_work;   // queue not empty / stopping
    std::condition_variable cv_done;   // a completion arrived
    std::deque<Request> queue;
    std::deque<dd_completion_t> done;
    int64_t outstanding = 0;
    bool stopping = false;

    void run(Worker& w);
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

dd_result_t dd_engine_s::serve(Worker& w, const Request& r) {
    if (r.n < 1 || r.m < 1) return failed(DD_EINVAL);
    const size_t need = dd_plan_footprint(r.m, r.n, &opt);
    if (need == 0) return failed(DD_EINVAL);
    if (need > w.ws_bytes || ((r.flags & DD_SERIES_HOST) && r.m > m_max)) return failed(DD_ENOMEM);
    if (!w.plan || w.plan->m != r.m || w.plan->n != r.n) {
        dd::destroy_plan(w.plan, false);  // the worker's stream is idle here
        w.plan = nullptr;
        const dd_status_t st = dd::create_plan(&w.plan, r.m, r.n, &opt, w.ws, w.ws_bytes, true, w.stream);
        if (st != DD_OK) {
            w.plan = nullptr;
            return failed(st);
        }
    }
    const float* src = r.T;
    cudaError_t e = cudaSuccess;
    if (r.flags & DD_SERIES_HOST) {
        e = cudaMemcpyAsync(w.stage, r.T, sizeof(float) * (size_t)r.m, cudaMemcpyHostToDevice, w.stream);
        src = w.stage;
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
            cv_work.wait(lk, [&] { return stopping || !queue.empty(); });
            if (stopping) return;
            r = queue.front();
            queue.pop_front();
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
    }
}

extern "C" {

dd_status_t dd_engine_create(dd_engine_t* engine, int32_t workers, const dd_options_t* opt, int64_t m_max,
                             int32_t n_max) {
    if (!engine) return DD_EINVAL;
    *engine = nullptr;
    if (workers < 1 || workers > 64) return DD_EINVAL;
    dd_options_t o;
    if (opt)
        o = *opt;
    else
        dd_options_default(&o);
    if (dd_plan_footprint(m_max, n_max, &o) == 0) return DD_EINVAL;
    const size_t ws = max_footprint(m_max, n_max, &o);
    dd_engine_s* E = new (std::nothrow) dd_engine_s();
    if (!E) return DD_ENOMEM;
    E->opt = o;
    E->m_max = m_max;
    cudaError_t e = cudaGetDevice(&E->device);
    E->workers.resize((size_t)workers);
    for (Worker& w : E->workers) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMalloc(&w.ws, ws);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&w.stage), sizeof(float) * (size_t)m_max);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&w.res_dev), sizeof(dd_result_t));
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&w.res_host), sizeof(dd_result_t));
        w.ws_bytes = ws;
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

dd_status_t dd_engine_submit(dd_engine_t E, int64_t id, const float* T, int64_t m, int32_t n, int32_t flags) {
    if (!E || !T || (flags != DD_SERIES_DEVICE && flags != DD_SERIES_HOST)) return DD_EINVAL;
    {
        std::lock_guard<std::mutex> lk(E->mu);
        if (E->stopping) return DD_EBUSY;
        E->queue.push_back(Request{id, T, m, n, flags, Clock::now()});
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
        dd::destroy_plan(w.plan, false);
        if (w.ws) cudaFree(w.ws);
        if (w.stage) cudaFree(w.stage);
        if (w.res_dev) cudaFree(w.res_dev);
        if (w.res_host) cudaFreeHost(w.res_host);
        if (w.stream) cudaStreamDestroy(w.stream);
    }
    delete E;
}

}  // extern "C"
