// dd_internal.cuh -- plan layout, device control block and kernel entry points
// shared by the CUDA translation units of libdd.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "../../include/dd.h"

namespace dd {

// ---------------------------------------------------------------- constants
constexpr int kMaxAlphabet = 64;
constexpr int kMaxDict = 4096;           // alphabet^paa_w limit (word index fits one smem sort)
constexpr int kStatBlocks = 1024;        // partial-sum blocks of the Eq. 2 statistics
constexpr int kScanElems = 4096;         // elements per block of the FP64 prefix scan
constexpr int kHistRows = 4096;          // rows per block of the word histogram / scatter
constexpr int kCompactRows = 2048;       // list entries per block of the compaction
constexpr int kCompactSites = 16;        // compactions per search (one look-back status array each)
constexpr int kTopkBins = 4096;          // bins of the top-k radix select (float bits >> 19)
constexpr int kMuBins = 4096;            // bins of the mean-bucketed row order
constexpr int kMaxLaunchSlots = 512;     // work counters per search
constexpr int kMaxListSlots = 256;       // list counts per search
constexpr int kMaxWaves = 64;            // distance waves traced per call
constexpr int kDgPad = 2048 + 64;        // padding entries after the diagonal-recurrence data (>= one CTA's diagonals)

// Relative term beta of the Gram form's per-row bound F_i(D): 2 x 6 u32 (u32 = 2^-24,
// safety factor 2) for the FP32 rounding of the epilogue's sum D.
constexpr float kTcBeta = 12.0f * 5.9604644775390625e-08f;
constexpr int kTcAtom = 64;      // Gram form: 16-bit operand elements per row chunk (one 128-byte line of S)
constexpr int kTcColPad = 256;   // Gram form: per-column constants padded by one 256-column tile on each side

// FP32 direct-difference tile kernel
constexpr int kF32BM = 128;  // rows per tile
constexpr int kF32BN = 128;  // columns per tile
constexpr int kF32BK = 32;   // k-chunk
constexpr int kF32Threads = 256;

// Device control block: zeroed once at the start of every search (one memset),
// so every counter below is written by exactly one search.
struct Ctrl {
    unsigned long long key;       // argmax key: float bits(nn^2) << 32 | (0xffffffff - i)
    unsigned long long pairs;     // distance pairs computed
    unsigned int bsf;             // best-so-far nn^2 (float bits, non-negative floats order as uints)
    int nonfinite;                // T held NaN/Inf
    int degenerate;               // sigma == 0
    int ncand;                    // |Cand|
    int n1;                       // rows run in phase 1
    int n2;                       // rows in phase 2 (N - n1)
    int ncomplete;                // rows that completed a full scan
    int err;                      // device-side error code (0 = none)
    unsigned int topk_thr;        // top-k threshold (float bits)
    int fmin;                     // smallest non-zero word frequency (Cand words)
    unsigned int tc_scmax;        // Gram form: max sqrt(c_j) (float bits)
    unsigned int tc_cmax;         // Gram form: max c_j (float bits)
    unsigned int tc_mumax;        // Gram form: max |sqrt(n) mu_j| (float bits)
    int ncandidates;              // rows rescored in FP64
    int best_idx;                 // smallest index attaining best64
    unsigned long long best64;    // exact nn^2 of the discord (double bits)
    unsigned long long wlb;       // per-window search: exact nn^2 of the row with the largest bound (double bits)
    int smax[64];                 // largest per-tile segment count of each tile-range launch
    int cnt[kMaxListSlots];       // list counts written by compactions
    int work[kMaxLaunchSlots];    // dynamic-schedule work counters, one per launch
    unsigned long long wave_pairs[kMaxWaves];  // per distance wave (by launch slot)
    unsigned long long wave_items[kMaxWaves];
    int wave_rows[kMaxWaves];
    int cond[8];                  // value each conditional graph node of the search took (1 = body ran)
    int cticket[kCompactSites];   // block tickets of each compaction (blocks take their place in start order)
    int stat_ticket[2];           // blocks done with the two passes of the Eq. 2 statistics
    int topk_ticket[6];           // blocks done with each top-k histogram pass (three selections per search)
    int best_ticket;              // blocks done with the exact maximum over the candidates
    int resc_nch;                 // FP64 rescoring: column chunks of the longest candidate range
    int topk_bin;                 // top-k select: bin of the first pass holding the k-th row (-1: take all)
    int topk_need;                // rows still needed from that bin
    int topk_hist[kTopkBins];     // radix-select histogram, pass 1 (float bits >> 19)
    int topk_hist2[kTopkBins];    // pass 2 inside topk_bin (float bits >> 7, low 12 bits)
};

// A list of rows (orig indices).  Row r of the list is base[off + r] with
// off = *off_dev (or 0) and the count *cnt_dev.
struct ListRef {
    const int32_t* base;
    const int32_t* off_dev;  // may be null
    const int32_t* cnt_dev;
};

// Column schedule of one wave.
//   mode 0: every row tile scans virtual columns [v_lo, v_hi) of the word
//           order, read backwards (virtual v -> position N-1-v);
//   mode 1: each row tile scans `local_cols` rows that share the SAX word of
//           its first row (Index_Word neighbourhood), starting half a word away;
//   mode 2: each row tile scans its own range of the mean-bucketed order
//           (ranges[t] = (L, H, C, segments)) in segments of seg_cols
//           columns, alternating right / left of C, nearest first;
//   mode 3: (tensor-core form, list = the mean-bucketed order itself) row tile
//           [q0, q0+128) against the 256 columns [q0-64, q0+192).
// Column sets of a wave.  mode 0: positions [v_lo, v_hi) of `order`; 1: the
// tile's first row's SAX word (local_cols of them); 2: lower-bound segments of
// the mean order (ranges); 3: the band tile around the row tile (Gram form);
// 4: time-local -- local_cols columns on each side of the tile's rows in time,
// just outside their exclusion zones.
struct ColSpec {
    int mode;
    int v_lo, v_hi;
    int local_cols;
    int seg_cols;  // FP32 form, lower-bound scans: columns per work item (0: the default)
};

struct PrepArrays {
    const float* T;
    int64_t m, N;
    int n;
    int w, A, D, paa_mode;
    double* stats;      // [8]
    double* part;       // [2*kStatBlocks]
    double* t64;        // [m + pad]
    float* t32;         // [m + pad]
    double* P1;         // [m+1]
    double* P2;         // [m+1]
    double* bsum;       // [4 * nscan]
    double* mu_w;       // [N]
    double* c_w;        // [N]
    const double* beta; // [A-1] breakpoints
    int32_t* code;      // [N]
    int32_t* hist;      // [D]
    int32_t* blockcnt;  // [nhist * D]
    int32_t* word_start;// [D]
    int32_t* order;     // [N]
    int32_t* pos_of;    // [N]
    int phase1_max;
    Ctrl* ctrl;
};

// In the Gram form every row also carries r32[i]: the smallest rigorous upper
// bound on d^2 that a direct FP32 wave found for it (FP32 distance plus its
// error bound; +inf when none).  An upper bound on the row's nearest-neighbour
// distance is then min(D + F_i(D), r32[i]).  A lower bound after a full scan
// of the row's columns stays D' - F_i(D') - gam^2 with D' = min(D, r32[i]):
// D' is still at most the value the Gram tiles computed for the true
// nearest column, and x - F_i(x) increases with x.
struct TcBound {
    const float* alpha;
    const float* gam;
    const float* q2;
    float beta;
    int on;
    const uint32_t* r32;  // may be null
    const uint8_t* excl;  // rows that may not be a discord (top-k search); all zero otherwise
};

__device__ __forceinline__ float row_ub(const TcBound& b, int i, float D) {
    if (!b.on) return D;
    const float u = D + (b.alpha[i] + b.beta * D + b.gam[i] * sqrtf(fmaxf(D, 0.f) + b.q2[i]));
    return b.r32 ? fminf(u, __uint_as_float(b.r32[i])) : u;
}
__device__ __forceinline__ float row_lb(const TcBound& b, int i, float D) {
    if (!b.on) return D;
    if (b.r32) D = fminf(D, __uint_as_float(b.r32[i]));
    const float g = b.gam[i];
    const float v = D - (b.alpha[i] + b.beta * D + g * sqrtf(fmaxf(D, 0.f) + b.q2[i])) - g * g;
    return v > 0.f ? v : 0.f;
}

struct ScanArgs {
    const float* t32;
    int N, n;
    ListRef rows;
    const int32_t* order;
    const int32_t* pos_of;
    const int32_t* code;
    const int32_t* hist;
    const int32_t* word_start;
    ColSpec col;
    const int32_t* sig;       // mean-bucketed order (mode 2)
    const int4* ranges;       // per row tile (mode 2)
    const int* smax;          // largest segment count over the tiles (mode 2)
    int seg_cols;             // columns per segment (mode 2)
    uint32_t* rmin;           // per orig row: float bits of the running minimum
    const Ctrl* ctrl_ro;      // bsf, flags
    Ctrl* ctrl;
    int abandon;
    int work_slot;
    int min_seg_tiles;
    int target_items;
    int wave;                 // trace slot (< kMaxWaves) or -1
    int min_rows;             // the wave runs only when the list has more rows than this
    // Gram-form plans run the time-local wave (mode 4) with this kernel: it then
    // tests rows against tb (the Gram bound) and writes rigorous FP32 upper
    // bounds into r32 instead of plain minima into rmin
    TcBound tb;
    uint32_t* r32;
    const double* stats;      // [2] = max |t^| of the series (FP32 error bound)
    // fused batch (batch.cu): per list tile its series, per series its best-so-far
    // (float bits); null for a single-series search
    const int32_t* tser;
    const uint32_t* sbsf;
    int bm;                   // rows per tile: 0 or 128 (default), 64, 32
};

// Upper / lower bounds of a row's nearest-neighbour distance from its running
// minimum D: identical to D for the FP32 form; D +- F_i(D) for the Gram form.

struct TcArgs {
    int N, n, nka, stages, seg_cols, mode;
    ListRef rows;
    int a_direct, a_row0;
    const int32_t* sig;
    const float4* coldat;
    const float* rowmu;
    const float* rowc;
    const float* alpha;
    const float* gam;
    const float* q2;
    float beta;
    int4* ranges;  // per row tile (mode 2); the kernel narrows them as rows finish
    const int* smax;
    uint32_t* rmin;
    Ctrl* ctrl;
    const double* stats;
    int abandon, work_slot;
    uint32_t idesc;
    int wave;               // trace slot (< kMaxWaves) or -1
    const uint32_t* r32;    // per orig row: FP32 upper bound of the time-local wave (see TcBound)
    const int32_t* sigpos;  // orig row -> position in the mean order
    int local_k;            // mode 2: > 0 limits row i to positions within local_k of its own
    int stall;              // fault injection (tests): issue no operand copy
    // fused batch (batch.cu): per list tile its series, per series its best-so-far
    // (float bits); null for a single-series search
    const int32_t* tser;
    const uint32_t* sbsf;
};

}  // namespace dd

// Plan: everything a search needs, carved out of one device workspace.
struct dd_plan_s {
    int64_t m = 0, N = 0;
    int32_t n = 0;
    dd_options_t opt{};
    int device = 0;
    int sm_count = 0;
    int D = 0;
    size_t ws_bytes = 0;
    void* ws = nullptr;
    bool own_ws = false;
    std::atomic<int> busy{0};
    int64_t launches = 0;

    // arrays (device)
    dd::Ctrl* ctrl = nullptr;
    double* stats = nullptr;
    double* part = nullptr;
    double* beta = nullptr;
    float* Tbuf = nullptr;
    double* t64 = nullptr;
    float* t32 = nullptr;
    double* P1 = nullptr;
    double* P2 = nullptr;
    double* bsum = nullptr;
    double* mu_w = nullptr;
    double* c_w = nullptr;
    int32_t* code = nullptr;
    int32_t* hist = nullptr;
    int32_t* blockcnt = nullptr;
    int32_t* word_start = nullptr;
    int32_t* order = nullptr;
    int32_t* pos_of = nullptr;
    uint32_t* rmin = nullptr;
    uint32_t* rmin32 = nullptr;
    uint8_t* excl = nullptr;     // per row: 1 = excluded from being the discord (dd_find_discords)  // Gram form: FP32 upper bounds from the time-local wave (TcBound::r32)
    int32_t* list[4] = {nullptr, nullptr, nullptr, nullptr};
    unsigned long long* cstat = nullptr;  // [kCompactSites][nblk] look-back status words of the compactions
    int cstat_stride = 0;                 // nblk = ceil(N / kCompactRows)
    dd_result_t* res_dev = nullptr;
    dd_result_t* res_host = nullptr;  // pinned
    int32_t* seq_rows = nullptr;      // 0..N-1
    int32_t* mubin = nullptr;         // [N] mean bin of each row
    int32_t* hist_mu = nullptr;       // [kMuBins]
    int32_t* blockcnt_mu = nullptr;   // [nh * kMuBins]
    int32_t* binstart = nullptr;      // [kMuBins + 1]
    int32_t* sig = nullptr;           // [N] rows in mean-bucketed order
    int64_t mu_stride = 0;            // stride permutation feeding the mean-bin sort (gcd with N = 1)
    int32_t* sigpos = nullptr;        // [N] position of each row in sig
    int4* ranges = nullptr;           // [N/128 + 1] per-tile column range (L, H, C, segments)

    // Gram (tensor-core) form
    int kpad = 0;                     // n rounded up to 64 (one 128-byte swizzle atom)
    void* S16 = nullptr;              // [kpad/64][N][64] centred rows in mean-bucketed order (FP16/BF16), k-chunk major
    void* A16 = nullptr;              // [kpad/64][N][64] rows of the current list, packed the same way
    float4* coldat = nullptr;         // [N + 512] per column in mean-bucketed order: (sqrt(n) mu, c, index, 0),
                                      // 256 padding entries on each side (c = +inf)
    float* rowmu = nullptr;           // [N] sqrt(n) mu (orig order)
    float* rowc = nullptr;            // [N] c
    float* rowsc = nullptr;           // [N] sqrt(c) rounded up
    float* alpha = nullptr;           // [N] error bound terms
    float* gam = nullptr;
    float* q2 = nullptr;
    double* ex64 = nullptr;           // [N] exact FP64 nn^2 of the rescored rows

    // diagonal-recurrence profile and per-window form (opt.diag or opt.znorm == 1)
    double* wmu64 = nullptr;          // [N] window means, two-pass FP64
    double* wr64 = nullptr;           // [N] per window: 1 / sigma (0 for a constant window)
    float4* wdat = nullptr;           // [N + kDgPad] (df, dg, 1/sqrt(c), e) per window, (df, dg, c, sqrt(n) mu) globally
    float* wmu32 = nullptr;           // [N + kDgPad] window means rounded to FP32
    float2* wscr = nullptr;           // [N] per window: (fl32(1 / sigma), E) of the FP32 screen
    unsigned long long* dkey = nullptr;  // [N] nearest-neighbour key: float bits << 32 | partner
    float* dub = nullptr;             // [N] per-window search: rigorous upper bound of nn^2
    CUtensorMap mapS_A, mapS_B, mapP_A;

    double beta_host[dd::kMaxAlphabet];

    // captured search graph (replayed while the input/output pointers and the
    // profiling switch stay the same)
    cudaStream_t cap_stream = nullptr;
    struct WaveMeta {
        int kind;  // dd_wave_kind_t
        int ev;    // index of its start event in ev[], -1 if untimed
    };
    WaveMeta waves[dd::kMaxWaves];  // host-side metadata of the last call's waves (by launch slot)
    int nwaves = 0;
    WaveMeta g_waves[dd::kMaxWaves];  // the same for the captured graph
    int g_nwaves = 0;
    cudaStream_t side_stream = nullptr;
    cudaStream_t body_stream = nullptr;  // captures the bodies of conditional graph nodes
    int inject = 0;                      // dd_plan_inject: consumed by the next distance launch
    struct CondBody {
        const int* taken; // device flag: the body ran (set by the node's condition kernel)
        int64_t launches; // kernels inside the body
    };
    std::vector<CondBody> bodies;        // conditional bodies of the last captured call
    std::vector<CondBody> g_bodies;      // the same for the cached graph
    bool in_cond = false;                // capturing a conditional body (no event nodes there)  // SAX / word order run here, beside the mean order
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool own_side = true;                // the side stream and fork / join events belong to the plan
    cudaGraphExec_t gexec = nullptr;
    const void* g_T = nullptr;
    const void* g_out = nullptr;
    int g_kind = -1;
    bool g_prof = false;
    bool capturing = false;
    bool use_graph = true;
    int64_t g_launches = 0;
    int g_ev_used = 0;

    // tracing (dd_plan_set_profiling)
    bool profiling = false;
    std::vector<cudaEvent_t> ev;   // pool: pairs (start, stop) around distance launches
    int ev_used = 0;
    cudaEvent_t call_ev[2] = {nullptr, nullptr};
    dd_profile_t prof{};
};

namespace dd {

// prep.cu
cudaError_t launch_prep(dd_plan_s* p, const float* T, cudaStream_t s);
cudaError_t launch_prep_common(dd_plan_s* p, const float* T, cudaStream_t s);
cudaError_t launch_prep_words(dd_plan_s* p, cudaStream_t s);
cudaError_t launch_prep_mean(dd_plan_s* p, cudaStream_t s);
// search.cu
cudaError_t launch_search(dd_plan_s* p, const float* T, dd_result_t* out_dev, cudaStream_t s);
cudaError_t launch_profile(dd_plan_s* p, const float* T, const int32_t* rows, int count, float* nn2,
                           cudaStream_t s);
// scan_fp32.cu
cudaError_t launch_scan_fp32(const ScanArgs& a, int grid, cudaStream_t s);
// scan_tc.cu
size_t tc_smem_bytes(int kpad);
int tc_stages(int kpad);
bool tc_supported(int n);
cudaError_t tc_make_maps(dd_plan_s* p);
// api.cu: plan construction shared by the public entry point and the engine.
// Engine plans may borrow their worker's side stream and fork / join events
// (borrowed = non-null: {side stream, fork event, join event}), which the plan
// then neither creates nor destroys.
struct PlanShared {
    cudaStream_t side;
    cudaEvent_t fork, join;
};
dd_status_t create_plan(dd_plan_s** plan, int64_t m, int32_t n, const dd_options_t* opt, void* workspace,
                        size_t workspace_bytes, bool engine, cudaStream_t init, const PlanShared* borrowed = nullptr);
void destroy_plan(dd_plan_s* p, bool wait_device);
cudaError_t tc_init_plan(dd_plan_s* p, cudaStream_t s);
cudaError_t launch_tc_prep(dd_plan_s* p, cudaStream_t s);
cudaError_t launch_gather_rows(dd_plan_s* p, ListRef L, cudaStream_t s);
cudaError_t launch_scan_tc(dd_plan_s* p, const TcArgs& a, bool a_packed, cudaStream_t s);
// rescore.cu
cudaError_t launch_rescore(dd_plan_s* p, ListRef cand, TcBound bound, int work_slot, dd_result_t* out_dev,
                           cudaStream_t s);
// api.cu: event pair around a distance launch when profiling (start=true before, false after)
void prof_mark(dd_plan_s* p, cudaStream_t s, bool start);
int scan_fp32_grid(const dd_plan_s* p);

// rescore.cu: argmax over a rescored list (ties -> smallest index) into the result
cudaError_t launch_best(dd_plan_s* p, ListRef cand, dd_result_t* out_dev, cudaStream_t s);
// diag.cu: diagonal-recurrence profile (dd_nn_profile_diag, and dd_nn_profile of a
// per-window plan), per-window rows and the per-window discord search
cudaError_t launch_profile_diag(dd_plan_s* p, const float* T, float* nn2, int32_t* idx, cudaStream_t s);
cudaError_t launch_rows_window(dd_plan_s* p, const float* T, const int32_t* rows, int count, float* nn2,
                               cudaStream_t s);
cudaError_t launch_search_window(dd_plan_s* p, const float* T, dd_result_t* out_dev, cudaStream_t s);

void host_breakpoints(int A, double* beta);

}  // namespace dd
