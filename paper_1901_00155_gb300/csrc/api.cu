// api.cu -- the C ABI of libdd.so (declared in include/dd.h): plans, their
// device workspace, and the entry points that enqueue preparation + search.
#include <algorithm>
#include <vector>
#include <cstring>
#include <new>

#include "dd_internal.cuh"

using dd::Ctrl;

namespace {

constexpr size_t kAlign = 256;
constexpr int32_t kBatchWorkers = 32;  // engine workers of a batched call
constexpr int kPad = 64;  // zero elements after the series copies

struct Carver {
    char* base;
    size_t off = 0;
    template <class T>
    T* take(size_t count) {
        off = (off + kAlign - 1) / kAlign * kAlign;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

bool valid_options(const dd_options_t& o) {
    if (o.precision != DD_FP32 && o.precision != DD_TC_FP16 && o.precision != DD_TC_BF16) return false;
    if (o.paa_w < 1 || o.alphabet < 2 || o.alphabet > dd::kMaxAlphabet) return false;
    double dict = 1.0;
    for (int i = 0; i < o.paa_w; i++) dict *= o.alphabet;
    if (dict > dd::kMaxDict) return false;
    if (o.early_abandon != 0 && o.early_abandon != 1) return false;
    if (o.paa_mode != 0 && o.paa_mode != 1) return false;
    if (o.phase1_max < 0 || o.refine_k < 0 || o.local_cols < 0 || o.word_cols < 0) return false;
    if (o.shard_count < 0 || o.shard_index < 0 || o.shard_index >= (o.shard_count > 1 ? o.shard_count : 1))
        return false;
    if (o.znorm != 0 && o.znorm != 1) return false;
    if (o.diag != 0 && o.diag != 1) return false;
    for (int i = 0; i < 3; i++)
        if (o.reserved[i] != 0) return false;
    return true;
}

// The diagonal-recurrence workspace (and per-window search) is held.
bool has_diag(const dd_options_t& o) { return o.znorm == 1 || o.diag == 1; }

bool valid_sizes(int64_t m, int32_t n) {
    if (n < 1 || m < 1 || (int64_t)n > m) return false;
    const int64_t N = m - n + 1;
    if (N < 2 * (int64_t)n) return false;
    if (m > (int64_t)0x7fffffff - 4096) return false;  // int32 row / column indices
    return true;
}

// Words never have more PAA segments than a subsequence has points.
void clamp_word(dd_options_t& o, int32_t n) {
    if (o.paa_w > n) o.paa_w = n;
}

int dict_size(const dd_options_t& o) {
    int d = 1;
    for (int i = 0; i < o.paa_w; i++) d *= o.alphabet;
    return d;
}

// Lays the plan's arrays out in `base` (or only measures when base == null).
size_t carve(dd_plan_s* p, char* base) {
    Carver c{base};
    const int64_t m = p->m, N = p->N;
    const int D = p->D;
    const int nscan = (int)((m + dd::kScanElems - 1) / dd::kScanElems);
    const int nh = (int)((N + dd::kHistRows - 1) / dd::kHistRows);
    const int nblk = (int)((N + dd::kCompactRows - 1) / dd::kCompactRows);
    p->ctrl = c.take<Ctrl>(1);
    p->stats = c.take<double>(16);
    p->part = c.take<double>(3 * dd::kStatBlocks);
    p->beta = c.take<double>(dd::kMaxAlphabet);
    p->Tbuf = c.take<float>(m + kPad);
    p->t64 = c.take<double>(m + kPad);
    p->t32 = c.take<float>(m + kPad);
    p->P1 = c.take<double>(m + 1);
    p->P2 = c.take<double>(m + 1);
    p->bsum = c.take<double>(4 * (size_t)nscan);
    p->mu_w = c.take<double>(N);
    p->c_w = c.take<double>(N);
    p->code = c.take<int32_t>(N);
    p->hist = c.take<int32_t>(D);
    p->blockcnt = c.take<int32_t>((size_t)nh * D);
    p->word_start = c.take<int32_t>(D);
    p->order = c.take<int32_t>(N);
    p->pos_of = c.take<int32_t>(N);
    p->rmin = c.take<uint32_t>(N);
    for (int k = 0; k < 4; k++) p->list[k] = c.take<int32_t>(N);
    p->cstat_stride = nblk;
    p->cstat = c.take<unsigned long long>((size_t)dd::kCompactSites * nblk);
    p->res_dev = c.take<dd_result_t>(1);
    p->excl = c.take<uint8_t>(N);
    p->seq_rows = c.take<int32_t>(N);
    p->mubin = c.take<int32_t>(N);
    p->hist_mu = c.take<int32_t>(dd::kMuBins);
    p->blockcnt_mu = c.take<int32_t>((size_t)nh * dd::kMuBins);
    p->binstart = c.take<int32_t>(dd::kMuBins + 1);
    p->sig = c.take<int32_t>(N);
    p->sigpos = c.take<int32_t>(N);
    p->ranges = c.take<int4>(N / 128 + 2);
    if (p->opt.precision != DD_FP32) {
        p->kpad = (p->n + 63) / 64 * 64;
        p->S16 = c.take<uint16_t>((size_t)N * p->kpad);
        p->A16 = c.take<uint16_t>((size_t)N * p->kpad);
        p->coldat = c.take<float4>(N + 2 * dd::kTcColPad);
        p->rowmu = c.take<float>(N);
        p->rowc = c.take<float>(N);
        p->rowsc = c.take<float>(N);
        p->alpha = c.take<float>(N);
        p->gam = c.take<float>(N);
        p->q2 = c.take<float>(N);
        p->ex64 = c.take<double>(N);
        p->rmin32 = c.take<uint32_t>(N);
    }
    if (has_diag(p->opt)) {
        if (!p->ex64) p->ex64 = c.take<double>(N);
        p->wmu64 = c.take<double>(N);
        p->wr64 = c.take<double>(N);
        p->wdat = c.take<float4>(N + dd::kDgPad);
        p->wmu32 = c.take<float>(N + dd::kDgPad);
        p->wscr = c.take<float2>(N);
        p->dkey = c.take<unsigned long long>(N);
        p->dub = c.take<float>(N);
    }
    return (c.off + kAlign - 1) / kAlign * kAlign;
}

__global__ void k_mark(uint8_t* a, int64_t lo, int64_t hi) {
    const int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < hi) a[i] = 1;
}

__global__ void k_iota(int32_t* a, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = (int32_t)i;
}

dd_status_t from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return DD_OK;
    if (e == cudaErrorMemoryAllocation) return DD_ENOMEM;
    return DD_ECUDA;
}

struct BusyGuard {
    dd_plan_s* p;
    bool ok;
    explicit BusyGuard(dd_plan_s* q) : p(q) {
        int expected = 0;
        ok = p->busy.compare_exchange_strong(expected, 1);
    }
    ~BusyGuard() {
        if (ok) p->busy.store(0);
    }
};

void rec(dd_plan_s* p, cudaEvent_t e, cudaStream_t s) {
    if (p->capturing)
        cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
        cudaEventRecord(e, s);
}

void prof_begin(dd_plan_s* p, cudaStream_t s) {
    p->ev_used = 0;
    if (p->profiling) rec(p, p->call_ev[0], s);
}

void prof_stop(dd_plan_s* p, cudaStream_t s) {
    if (p->profiling) rec(p, p->call_ev[1], s);
}

// Reads back the events of a finished synchronous call.
void prof_read(dd_plan_s* p, int64_t pairs) {
    if (!p->profiling) return;
    cudaEventSynchronize(p->call_ev[1]);
    dd_profile_t r{};
    r.precision = p->opt.precision;
    r.dist_launches = p->ev_used / 2;
    for (int k = 0; k + 1 < p->ev_used; k += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p->ev[k], p->ev[k + 1]) == cudaSuccess) r.dist_ms += ms;
    }
    float call = 0.f;
    if (cudaEventElapsedTime(&call, p->call_ev[0], p->call_ev[1]) == cudaSuccess) r.call_ms = call;
    r.computed_pairs = pairs;
    p->prof = r;
}

// Everything one synchronous search enqueues: the search and the copy of its
// result to pinned host memory.
cudaError_t enqueue_sync(dd_plan_s* p, const float* T_dev, cudaStream_t s) {
    prof_begin(p, s);
    cudaError_t e = dd::launch_search(p, T_dev, p->res_dev, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(p->res_host, p->res_dev, sizeof(dd_result_t), cudaMemcpyDeviceToHost, s);
    prof_stop(p, s);
    return e;
}

// Replays (capturing first if needed) the graph of `kind` for (T, out).
cudaError_t graph_launch(dd_plan_s* p, int kind, const float* T_dev, dd_result_t* out_dev, cudaStream_t s) {
    if (!p->gexec || p->g_T != T_dev || p->g_out != out_dev || p->g_kind != kind || p->g_prof != p->profiling) {
        if (p->gexec) {
            cudaGraphExecDestroy(p->gexec);
            p->gexec = nullptr;
        }
        if (!p->cap_stream) {
            cudaError_t e0 = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
            if (e0 != cudaSuccess) return e0;
        }
        cudaError_t e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        p->capturing = true;
        int64_t launches = 0;
        cudaError_t ee;
        if (kind == 0) {
            ee = enqueue_sync(p, T_dev, p->cap_stream);
        } else {
            ee = dd::launch_search(p, T_dev, out_dev, p->cap_stream);
        }
        launches = p->launches;
        const int used = p->ev_used;
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(p->cap_stream, &g);
        p->capturing = false;
        if (ee != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return ee != cudaSuccess ? ee : e;
        }
        e = cudaGraphInstantiate(&p->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            p->gexec = nullptr;
            return e;
        }
        p->g_T = T_dev;
        p->g_out = out_dev;
        p->g_kind = kind;
        p->g_prof = p->profiling;
        p->launches = launches;
        p->ev_used = used;
        p->g_launches = launches;
        p->g_ev_used = used;
        p->g_nwaves = p->nwaves;
        for (int w = 0; w < p->nwaves; w++) p->g_waves[w] = p->waves[w];
        p->g_bodies = p->bodies;
    }
    p->launches = p->g_launches;
    p->ev_used = p->g_ev_used;
    p->nwaves = p->g_nwaves;
    for (int w = 0; w < p->g_nwaves; w++) p->waves[w] = p->g_waves[w];
    p->bodies = p->g_bodies;
    return cudaGraphLaunch(p->gexec, s);
}

dd_status_t search_sync(dd_plan_s* p, const float* T_dev, dd_result_t* out, cudaStream_t s) {
    if (!p->res_host) {  // engine plans allocate their pinned result slot on first synchronous use
        if (cudaMallocHost(reinterpret_cast<void**>(&p->res_host), sizeof(dd_result_t)) != cudaSuccess) {
            cudaGetLastError();
            p->res_host = nullptr;
            return DD_ENOMEM;
        }
    }
    cudaError_t e = p->use_graph ? graph_launch(p, 0, T_dev, nullptr, s) : enqueue_sync(p, T_dev, s);
    if (e != cudaSuccess) return from_cuda(e);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    *out = *p->res_host;
    prof_read(p, out->computed_pairs);
    return (dd_status_t)out->status;
}

}  // namespace

namespace dd {
void prof_mark(dd_plan_s* p, cudaStream_t s, bool start) {
    if (!p->profiling) return;
    if (p->ev_used >= (int)p->ev.size()) return;  // pool exhausted: later launches untimed
    if (p->in_cond) return;                       // conditional graph bodies hold no event nodes
    (void)start;
    cudaEvent_t e = p->ev[p->ev_used++];
    if (p->capturing)
        cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
        cudaEventRecord(e, s);
}
}  // namespace dd

namespace {

}  // namespace

namespace dd {

// Builds a plan. Public plans (engine == false) allocate their workspace unless
// one is given, initialise on the legacy stream and wait for the device. Engine
// plans live in a worker's workspace and are initialised on that worker's
// stream, so building one never waits for another worker's searches. They run
// without graph capture (every shape is used once or a few times) and have no
// pinned result buffer.
dd_status_t create_plan(dd_plan_s** plan, int64_t m, int32_t n, const dd_options_t* opt, void* workspace,
                        size_t workspace_bytes, bool engine, cudaStream_t init, const PlanShared* borrowed) {
    if (!plan) return DD_EINVAL;
    *plan = nullptr;
    dd_options_t o;
    if (opt)
        o = *opt;
    else
        dd_options_default(&o);
    if (!valid_options(o) || !valid_sizes(m, n)) return DD_EINVAL;
    clamp_word(o, n);
    if (o.precision != DD_FP32 && !dd::tc_supported(n)) return DD_ENOTSUP;
    if (o.znorm == 1 && (o.precision != DD_FP32 || o.shard_count > 1)) return DD_ENOTSUP;
    if (has_diag(o) && m - n + 1 > ((int64_t)1 << 26)) return DD_ENOTSUP;
    if (workspace && (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) return DD_EINVAL;
    if (engine && !workspace) return DD_EINVAL;
    dd_plan_s* p = new (std::nothrow) dd_plan_s();
    if (!p) return DD_ENOMEM;
    p->m = m;
    p->n = n;
    p->N = m - n + 1;
    p->opt = o;
    p->D = dict_size(o);
    p->use_graph = !engine;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
        delete p;
        return from_cuda(e);
    }
    const size_t need = carve(p, nullptr);
    p->ws_bytes = need;
    if (workspace) {
        if (workspace_bytes < need) {
            delete p;
            return DD_ENOMEM;
        }
        p->ws = workspace;
        p->own_ws = false;
    } else {
        e = cudaMalloc(&p->ws, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete p;
            return DD_ENOMEM;
        }
        p->own_ws = true;
    }
    carve(p, static_cast<char*>(p->ws));
    if (!engine) {
        e = cudaMallocHost(reinterpret_cast<void**>(&p->res_host), sizeof(dd_result_t));
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (p->own_ws) cudaFree(p->ws);
            delete p;
            return DD_ENOMEM;
        }
    }
    {
        // golden-ratio stride, coprime with N
        int64_t st = (int64_t)(0.6180339887498949 * (double)p->N);
        if (st < 1) st = 1;
        auto gcd = [](int64_t x, int64_t y) {
            while (y) {
                const int64_t t = x % y;
                x = y;
                y = t;
            }
            return x;
        };
        while (gcd(st, p->N) != 1) st++;
        p->mu_stride = st % p->N == 0 ? 1 : st;
    }
    dd::host_breakpoints(o.alphabet, p->beta_host);
    e = cudaMemcpyAsync(p->beta, p->beta_host, sizeof(double) * (o.alphabet - 1), cudaMemcpyHostToDevice, init);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->t64 + p->m, 0, sizeof(double) * kPad, init);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->t32 + p->m, 0, sizeof(float) * kPad, init);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->excl, 0, (size_t)p->N, init);
    // index arrays that the search builds on its side stream hold valid row indices
    // (0) from the start, so no read of them can leave the series, whatever the order
    if (e == cudaSuccess) e = cudaMemsetAsync(p->order, 0, sizeof(int32_t) * (size_t)p->N, init);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->pos_of, 0, sizeof(int32_t) * (size_t)p->N, init);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->code, 0, sizeof(int32_t) * (size_t)p->N, init);
    if (e == cudaSuccess && p->wdat) e = cudaMemsetAsync(p->wdat + p->N, 0, sizeof(float4) * dd::kDgPad, init);
    if (e == cudaSuccess && p->wmu32) e = cudaMemsetAsync(p->wmu32 + p->N, 0, sizeof(float) * dd::kDgPad, init);
    if (e == cudaSuccess) {
        k_iota<<<(unsigned)((p->N + 255) / 256), 256, 0, init>>>(p->seq_rows, p->N);
        e = cudaGetLastError();
    }
    if (borrowed) {
        p->own_side = false;
        p->side_stream = borrowed->side;
        p->ev_fork = borrowed->fork;
        p->ev_join = borrowed->join;
    } else {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->side_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
    }
    if (e == cudaSuccess && !engine) e = cudaStreamCreateWithFlags(&p->body_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && o.precision != DD_FP32) e = dd::tc_make_maps(p);
    if (e == cudaSuccess && o.precision != DD_FP32) e = dd::tc_init_plan(p, init);
    // the host copy above reads p->beta_host: wait for the init stream before returning
    if (e == cudaSuccess) e = engine ? cudaStreamSynchronize(init) : cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        destroy_plan(p, !engine);
        return from_cuda(e);
    }
    *plan = p;
    return DD_OK;
}

// Releases a plan. wait_device: wait for all device work first (public plans,
// whose last call's stream is unknown here); engine workers destroy plans only
// after synchronising their own stream.
void destroy_plan(dd_plan_s* p, bool wait_device) {
    if (!p) return;
    if (wait_device) cudaDeviceSynchronize();
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (p->own_side) {
        if (p->side_stream) cudaStreamDestroy(p->side_stream);
        if (p->ev_fork) cudaEventDestroy(p->ev_fork);
        if (p->ev_join) cudaEventDestroy(p->ev_join);
    }
    if (p->body_stream) cudaStreamDestroy(p->body_stream);
    for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : p->call_ev)
        if (e) cudaEventDestroy(e);
    if (p->res_host) cudaFreeHost(p->res_host);
    if (p->own_ws && p->ws) cudaFree(p->ws);
    delete p;
}

}  // namespace dd

extern "C" {

void dd_options_default(dd_options_t* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = DD_FP32;
    opt->paa_w = 4;
    opt->alphabet = 4;
    opt->early_abandon = 1;
    opt->paa_mode = 0;
    opt->phase1_max = 4096;
    opt->refine_k = 128;
    opt->local_cols = 64;
    opt->word_cols = 512;
}

size_t dd_plan_footprint(int64_t m, int32_t n, const dd_options_t* opt) {
    dd_options_t o;
    if (opt)
        o = *opt;
    else
        dd_options_default(&o);
    if (!valid_options(o) || !valid_sizes(m, n)) return 0;
    clamp_word(o, n);
    dd_plan_s tmp;
    tmp.m = m;
    tmp.n = n;
    tmp.N = m - n + 1;
    tmp.opt = o;
    tmp.D = dict_size(o);
    return carve(&tmp, nullptr);
}


dd_status_t dd_plan_create(dd_plan_t* plan, int64_t m, int32_t n, const dd_options_t* opt, void* workspace,
                           size_t workspace_bytes) {
    return dd::create_plan(plan, m, n, opt, workspace, workspace_bytes, false, nullptr);
}

void dd_plan_destroy(dd_plan_t p) { dd::destroy_plan(p, true); }

dd_status_t dd_find_discord(dd_plan_t p, const float* T_dev, dd_result_t* out, void* stream) {
    if (!p || !T_dev || !out) return DD_EINVAL;
    BusyGuard g(p);
    if (!g.ok) return DD_EBUSY;
    return search_sync(p, T_dev, out, static_cast<cudaStream_t>(stream));
}

dd_status_t dd_find_discords(dd_plan_t p, const float* T_dev, int32_t k, dd_result_t* out, void* stream) {
    if (!p || !T_dev || !out || k < 1) return DD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t N = p->N, n = p->n;
    std::vector<uint8_t> ex((size_t)N, 0);  // host copy of the exclusion mask, to know when rows run out
    int64_t left = N;
    dd_status_t st = DD_OK;
    int32_t j = 0;
    for (; j < k && left > 0; j++) {
        st = dd_find_discord(p, T_dev, &out[j], stream);
        if (st != DD_OK || out[j].index < 0) {
            j++;
            break;
        }
        const int64_t d = out[j].index;
        const int64_t lo = d - n + 1 > 0 ? d - n + 1 : 0, hi = d + n < N ? d + n : N;
        for (int64_t i = lo; i < hi; i++) left -= ex[(size_t)i] ? 0 : 1, ex[(size_t)i] = 1;
        k_mark<<<(unsigned)((hi - lo + 255) / 256), 256, 0, s>>>(p->excl, lo, hi);
        if (cudaGetLastError() != cudaSuccess) {
            st = DD_ECUDA;
            j++;
            break;
        }
    }
    for (; j < k; j++) {
        std::memset(&out[j], 0, sizeof(dd_result_t));
        out[j].index = -1;
        out[j].status = DD_OK;
    }
    // leave the mask cleared for ordinary searches
    cudaError_t e = cudaMemsetAsync(p->excl, 0, (size_t)N, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess && st == DD_OK) st = DD_ECUDA;
    return st;
}

dd_status_t dd_find_discord_async(dd_plan_t p, const float* T_dev, dd_result_t* out_dev, void* stream) {
    if (!p || !T_dev || !out_dev) return DD_EINVAL;
    BusyGuard g(p);
    if (!g.ok) return DD_EBUSY;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (p->use_graph) return from_cuda(graph_launch(p, 1, T_dev, out_dev, s));
    return from_cuda(dd::launch_search(p, T_dev, out_dev, s));
}

dd_status_t dd_find_discord_host(dd_plan_t p, const float* T_host, dd_result_t* out, void* stream) {
    if (!p || !T_host || !out) return DD_EINVAL;
    BusyGuard g(p);
    if (!g.ok) return DD_EBUSY;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(p->Tbuf, T_host, sizeof(float) * p->m, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return from_cuda(e);
    return search_sync(p, p->Tbuf, out, s);
}

dd_status_t dd_find_discord_batched(int32_t count, const float* const* T_dev, const int64_t* m, const int32_t* n,
                                    const dd_options_t* opt, dd_result_t* out, void* stream) {
    if (count < 0 || (count > 0 && (!T_dev || !m || !n || !out))) return DD_EINVAL;
    if (count == 0) return DD_OK;
    dd_options_t o;
    if (opt)
        o = *opt;
    else
        dd_options_default(&o);
    // the shapes the engine must hold; invalid series fail on their own
    int64_t m_max = 0;
    int32_t n_max = 0;
    for (int32_t k = 0; k < count; k++)
        if (dd_plan_footprint(m[k], n[k], &o) > 0) {
            m_max = m[k] > m_max ? m[k] : m_max;
            n_max = n[k] > n_max ? n[k] : n_max;
        }
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return DD_ECUDA;
    for (int32_t k = 0; k < count; k++) {
        std::memset(&out[k], 0, sizeof(dd_result_t));
        out[k].index = -1;
        out[k].status = DD_EINVAL;
    }
    if (m_max == 0) return DD_EINVAL;
    dd_engine_t E = nullptr;
    // a search of a short series is a chain of small kernels: up to 32 run side by side
    dd_status_t st = dd_engine_create(&E, count < kBatchWorkers ? count : kBatchWorkers, &o, m_max, n_max);
    if (st != DD_OK) return st;
    // longest series first, so that the last ones to start are short
    std::vector<int32_t> ord((size_t)count);
    for (int32_t k = 0; k < count; k++) ord[(size_t)k] = k;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return m[a] > m[b]; });
    for (int32_t k : ord) dd_engine_submit(E, k, T_dev[k], m[k], n[k], DD_SERIES_DEVICE);
    std::vector<dd_completion_t> c((size_t)count);
    int32_t got = 0;
    while (got < count) {
        const int32_t r = dd_engine_poll(E, c.data(), count, -1);
        if (r < 0) break;
        for (int32_t j = 0; j < r; j++) out[c[(size_t)j].id] = c[(size_t)j].result;
        got += r;
    }
    dd_engine_destroy(E);
    dd_status_t first = DD_OK;
    for (int32_t k = 0; k < count && first == DD_OK; k++)
        if (out[k].status != DD_OK) first = (dd_status_t)out[k].status;
    return first;
}

dd_status_t dd_nn_profile(dd_plan_t p, const float* T_dev, float* nn2_dev, void* stream) {
    if (!p || !T_dev || !nn2_dev) return DD_EINVAL;
    BusyGuard g(p);
    if (!g.ok) return DD_EBUSY;
    return from_cuda(dd::launch_profile(p, T_dev, nullptr, 0, nn2_dev, static_cast<cudaStream_t>(stream)));
}

dd_status_t dd_nn_profile_diag(dd_plan_t p, const float* T_dev, float* nn2_dev, int32_t* nn_index_dev, void* stream) {
    if (!p || !T_dev || !nn2_dev) return DD_EINVAL;
    if (!p->dkey) return DD_ENOTSUP;
    BusyGuard g(p);
    if (!g.ok) return DD_EBUSY;
    return from_cuda(dd::launch_profile_diag(p, T_dev, nn2_dev, nn_index_dev, static_cast<cudaStream_t>(stream)));
}

dd_status_t dd_nn_rows(dd_plan_t p, const float* T_dev, const int32_t* rows_dev, int32_t count, float* nn2_dev,
                       void* stream) {
    if (!p || !T_dev || !rows_dev || !nn2_dev || count < 0 || count > p->N) return DD_EINVAL;
    if (count == 0) return DD_OK;
    BusyGuard g(p);
    if (!g.ok) return DD_EBUSY;
    return from_cuda(dd::launch_profile(p, T_dev, rows_dev, count, nn2_dev, static_cast<cudaStream_t>(stream)));
}

dd_status_t dd_prep(dd_plan_t p, const float* T_dev, void* stream) {
    if (!p || !T_dev) return DD_EINVAL;
    BusyGuard g(p);
    if (!g.ok) return DD_EBUSY;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    p->launches = 0;
    cudaError_t e = cudaMemsetAsync(p->ctrl, 0, sizeof(Ctrl), s);
    if (e == cudaSuccess) e = dd::launch_prep(p, T_dev, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    int nonfinite = 0;
    e = cudaMemcpy(&nonfinite, &p->ctrl->nonfinite, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return from_cuda(e);
    return nonfinite ? DD_ENONFINITE : DD_OK;
}

dd_status_t dd_plan_view(dd_plan_t p, dd_view_t* v) {
    if (!p || !v) return DD_EINVAL;
    v->m = p->m;
    v->N = p->N;
    v->n = p->n;
    v->dict_size = p->D;
    v->stats = p->stats;
    v->P1 = p->P1;
    v->P2 = p->P2;
    v->mu_w = p->mu_w;
    v->c_w = p->c_w;
    v->code = p->code;
    v->freq_hist = p->hist;
    v->order = p->order;
    v->word_start = p->word_start;
    v->ncand = &p->ctrl->ncand;
    v->t32 = p->t32;
    return DD_OK;
}

dd_status_t dd_plan_bound_view(dd_plan_t p, dd_bound_view_t* v) {
    if (!p || !v) return DD_EINVAL;
    if (p->opt.precision == DD_FP32 || !p->alpha) return DD_ENOTSUP;
    v->N = p->N;
    v->precision = p->opt.precision;
    v->beta = dd::kTcBeta;
    v->alpha = p->alpha;
    v->gam = p->gam;
    v->q2 = p->q2;
    return DD_OK;
}

dd_status_t dd_plan_order_view(dd_plan_t p, dd_order_view_t* v) {
    if (!p || !v) return DD_EINVAL;
    v->N = p->N;
    v->stride = p->mu_stride;
    v->bins = dd::kMuBins;
    v->sig = p->sig;
    v->sigpos = p->sigpos;
    v->mubin = p->mubin;
    v->binstart = p->binstart;
    v->geom = p->stats + 6;  // stats[6..9]: lo, w, 1/sigma, 1/w
    return DD_OK;
}

int64_t dd_plan_last_launches(dd_plan_t p) {
    if (!p) return -1;
    // a graph replay skips the kernels of conditional bodies whose gate did not pass
    int64_t n = p->launches;
    for (const dd_plan_s::CondBody& b : p->bodies) {
        int v = 1;
        if (cudaMemcpy(&v, b.taken, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (v == 0) n -= b.launches;
    }
    return n;
}

dd_status_t dd_plan_set_profiling(dd_plan_t p, int32_t enable) {
    if (!p) return DD_EINVAL;
    if (enable && p->ev.empty()) {
        p->ev.resize(256);
        for (auto& e : p->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return DD_ECUDA;
        for (auto& e : p->call_ev)
            if (cudaEventCreate(&e) != cudaSuccess) return DD_ECUDA;
    }
    p->profiling = enable != 0;
    return DD_OK;
}

int32_t dd_plan_get_waves(dd_plan_t p, dd_wave_t* out, int32_t cap) {
    if (!p || (cap > 0 && !out)) return -DD_EINVAL;
    BusyGuard g(p);
    if (!g.ok) return -DD_EBUSY;
    const int nw = p->nwaves;
    if (nw == 0 || cap <= 0) return nw;
    unsigned long long pairs[dd::kMaxWaves], items[dd::kMaxWaves];
    int rows[dd::kMaxWaves];
    cudaError_t e = cudaMemcpy(pairs, p->ctrl->wave_pairs, sizeof(pairs), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(items, p->ctrl->wave_items, sizeof(items), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(rows, p->ctrl->wave_rows, sizeof(rows), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return -DD_ECUDA;
    for (int w = 0; w < nw && w < cap; w++) {
        dd_wave_t r{};
        r.kind = p->waves[w].kind;
        r.rows = rows[w];
        r.items = (int64_t)items[w];
        r.pairs = (int64_t)pairs[w];
        r.ms = -1.0;
        const int k = p->waves[w].ev;
        float ms = 0.f;
        if (p->profiling && k >= 0 && k + 1 < p->ev_used &&
            cudaEventElapsedTime(&ms, p->ev[k], p->ev[k + 1]) == cudaSuccess)
            r.ms = ms;
        out[w] = r;
    }
    return nw;
}

dd_status_t dd_plan_set_graph(dd_plan_t p, int32_t enable) {
    if (!p) return DD_EINVAL;
    BusyGuard g(p);
    if (!g.ok) return DD_EBUSY;
    p->use_graph = enable != 0;
    return DD_OK;
}

dd_status_t dd_plan_inject(dd_plan_t p, int32_t what) {
    if (!p || (what != DD_INJECT_NONE && what != DD_INJECT_STALL_TC)) return DD_EINVAL;
    BusyGuard g(p);
    if (!g.ok) return DD_EBUSY;
    p->inject = what;
    return DD_OK;
}

dd_status_t dd_plan_get_profile(dd_plan_t p, dd_profile_t* out) {
    if (!p || !out) return DD_EINVAL;
    *out = p->prof;
    return DD_OK;
}

const char* dd_status_string(dd_status_t s) {
    switch (s) {
        case DD_OK: return "ok";
        case DD_EINVAL: return "invalid argument";
        case DD_ENOMEM: return "out of memory";
        case DD_ENONFINITE: return "series holds NaN or Inf";
        case DD_ETIMEOUT: return "device-side wait timed out";
        case DD_ECUDA: return "CUDA error";
        case DD_EBUSY: return "plan busy";
        case DD_ENOTSUP: return "not supported";
    }
    return "unknown status";
}

}  // extern "C"
