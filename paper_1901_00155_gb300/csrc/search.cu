// search.cu -- the search stage of PhiDD (Algorithm 2) on the device:
//   PotentialDiscord (Algorithm 3) over the Cand rows, then RefineDiscord
//   (Algorithm 4) over the other rows, as waves of distance tiles with
//   stream compaction of the surviving rows between waves, and the final
//   argmax (Algorithm 1's best-so-far update, ties -> smallest index).
//
// Waves, in order: the first (nearest-mean) wave for every row; the fill
// wave (Gram form) for rows it left unbounded; Cand; the rows with the largest
// upper bounds; when many rows survive, the time-local wave (Algorithm 4's
// index-order scan) and a second top-k; the word wave (FP32 form); the rest;
// and in the Gram form an FP32 settle wave before the FP64 rescoring when many
// candidates remain.  Everything is enqueued on one stream (the SAX words on
// a side branch) with all counts kept on the device, so a search needs no
// host round trip and is captured once into a CUDA graph, whose conditional
// nodes skip the waves that are not needed.
#include "dd_internal.cuh"

namespace dd {
namespace {

__global__ void k_set_int(int* p, int v) { *p = v; }

// Count of the Cand list: the word order (Eq. 10) puts the words of smallest
// frequency first, so Cand (Eq. 7) is order[0 .. ncand); it runs in phase 1
// only when it has at most phase1_max rows.
__global__ void k_cand_count(const Ctrl* ctrl, int phase1_max, int* cnt) {
    *cnt = ctrl->ncand <= phase1_max ? ctrl->ncand : 0;
}

// Rank values at or above this (the running minimum's initial value) mean the
// row has no finite upper bound yet.
constexpr uint32_t kNoBound = 0x7f000000u;

// A row is alive unless one of its distances is proven strictly below the
// best-so-far: FP32 form D < bsf (Algorithms 3/4); Gram form min(D + F_i(D),
// r32_i) < bsf, bsf being a proven lower bound there.  Rows excluded from being
// the discord (top-k search) are never alive.  Non-negative floats order like
// their bit patterns.
__device__ __forceinline__ bool is_alive(const TcBound& b, int i, uint32_t rbits, uint32_t bsf_bits) {
    if (b.excl && b.excl[i]) return false;  // may not be the discord: never a candidate, never completes
    if (!b.on) return rbits >= bsf_bits;
    if (bsf_bits == 0) return true;  // nothing has completed: every upper bound reaches bsf = 0
    // min(D + F(D), r32) >= bsf, F >= 0: decided by D and r32 alone unless D < bsf <= r32
    const float B = __uint_as_float(bsf_bits), D = __uint_as_float(rbits);
    if (b.r32 && __uint_as_float(b.r32[i]) < B) return false;
    if (!(D < B)) return true;
    return !(D + (b.alpha[i] + b.beta * D + b.gam[i] * sqrtf(fmaxf(D, 0.f) + b.q2[i])) < B);
}

// is_alive (and the rank test against thr) for U rows at once: every load of
// the U rows is issued before any of them is used, so a thread waits on one
// memory latency per step instead of one per row.  Entries i < 0 are not rows
// (false).  keep: alive with a rank value in [thr, thr_hi).  The alive
// decisions are the ones is_alive makes; rank gets the value
// rows are ranked by for the top-k waves: the running minimum, or in the Gram
// form the smaller of it and the row's FP32 upper bound (non-negative floats
// order like their bit patterns).
template <int U>
__device__ __forceinline__ void alive_batch(const TcBound& b, const int (&iv)[U], const uint32_t* __restrict__ rmin,
                                            uint32_t bsf_bits, uint32_t thr, uint32_t thr_hi, bool (&keep)[U],
                                            uint32_t (&rank)[U]) {
    uint32_t rb[U], r32[U];
    bool ex[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int i = iv[u];
        rb[u] = i >= 0 ? rmin[i] : 0u;
        r32[u] = i >= 0 && b.r32 ? b.r32[i] : 0xffffffffu;
        ex[u] = i >= 0 && b.excl ? b.excl[i] != 0 : false;
    }
    const float B = __uint_as_float(bsf_bits);
    int st[U];  // 0: not alive, 1: alive, 2: decided by the bound F_i
#pragma unroll
    for (int u = 0; u < U; u++) {
        int v;
        if (iv[u] < 0 || ex[u]) v = 0;
        else if (!b.on) v = rb[u] >= bsf_bits;
        else if (bsf_bits == 0) v = 1;
        else if (b.r32 && __uint_as_float(r32[u]) < B) v = 0;
        else v = __uint_as_float(rb[u]) < B ? 2 : 1;
        st[u] = v;
    }
    float al[U], ga[U], q2[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const bool need = st[u] == 2;
        al[u] = need ? b.alpha[iv[u]] : 0.f;
        ga[u] = need ? b.gam[iv[u]] : 0.f;
        q2[u] = need ? b.q2[iv[u]] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
        bool a = st[u] == 1;
        if (st[u] == 2) {
            const float D = __uint_as_float(rb[u]);
            a = !(D + (al[u] + b.beta * D + ga[u] * sqrtf(fmaxf(D, 0.f) + q2[u])) < B);
        }
        // rank value: min(rmin, r32) (r32 reads as all ones where there is none)
        rank[u] = min(rb[u], r32[u]);
        keep[u] = a && rank[u] >= thr && rank[u] < thr_hi;
    }
}

// Order-preserving compaction of a row list in one pass (decoupled look-back).
// Predicates: pred 0: alive against the best-so-far; pred 1: alive and rank
// value >= the top-k threshold (and finite); pred 2: member of Cand; pred 3:
// alive with no finite upper bound yet (the running minimum still holds its
// initial value).
// With sigpos set, rows outside positions [p_lo, p_hi) of the mean order are
// dropped too.
//
// Block b (a ticket taken at start, so every lower block has started) keeps
// entries [2048 b, 2048 b + 2048) in 8 coalesced rounds of 256 (thread t holds
// entry 256 q + t of round q, the rounds' loads issued together); ranks come
// from warp ballots.  Warp 0 publishes
// the block's count, then looks back over the status words of the blocks
// before it, 128 at a time, adding counts up to the nearest one that holds an
// inclusive prefix, and publishes its own inclusive prefix; the block then
// scatters its entries from there.  A status word is (flag << 62) | count:
// flag 1 = the block's own count, 2 = the inclusive prefix.  The block holding
// the last entry writes the total.  A wait on a predecessor is bounded by
// %globaltimer (2 s): on expiry the search records DD_ETIMEOUT.  Status words
// and tickets are zeroed per search.
constexpr unsigned long long kStAgg = 1ull << 62, kStPre = 2ull << 62;

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(256, 4) k_compact(ListRef in, const uint32_t* __restrict__ rmin, TcBound tb,
                                                 Ctrl* ctrl, int pred, const int32_t* __restrict__ code,
                                                 const int32_t* __restrict__ hist, int phase1_max,
                                                 const int32_t* __restrict__ sigpos, int p_lo, int p_hi, int site,
                                                 unsigned long long* __restrict__ status, int32_t* __restrict__ out,
                                                 int* __restrict__ cnt_out) {
    __shared__ int sh_b, sh_base;
    __shared__ int wcnt[8][8];  // [round][warp]
    const int cnt = *in.cnt_dev;
    if (threadIdx.x == 0) sh_b = atomicAdd(&ctrl->cticket[site], 1);
    __syncthreads();
    const int b = sh_b;
    const int nb = cnt > 0 ? (cnt + kCompactRows - 1) / kCompactRows : 1;  // blocks that hold entries
    if (b >= nb) return;  // no entries here, and no block waits on a later one
    const int off = in.off_dev ? *in.off_dev : 0;
    const uint32_t bsf = ctrl->bsf;
    const uint32_t thr = pred == 1 ? ctrl->topk_thr : (pred == 3 ? kNoBound : 0u);
    const uint32_t thr_hi = pred == 1 ? kNoBound : 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    // the block's entries: 8 independent coalesced loads per thread
    int i8[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const int r = b * kCompactRows + q * 256 + threadIdx.x;
        i8[q] = r < cnt ? in.base[off + r] : -1;
    }
    bool k8[8];
    if (pred == 2) {
        // Cand (Eq. 7): rows whose word has the smallest frequency
        const bool on = ctrl->ncand <= phase1_max;
        const int fmin = ctrl->fmin;
        int c8[8];
#pragma unroll
        for (int q = 0; q < 8; q++) c8[q] = i8[q] >= 0 ? code[i8[q]] : 0;
#pragma unroll
        for (int q = 0; q < 8; q++) k8[q] = on && i8[q] >= 0 && hist[c8[q]] == fmin;
    } else {
        uint32_t rk[8];
        alive_batch<8>(tb, i8, rmin, bsf, thr, thr_hi, k8, rk);
    }
    if (sigpos) {
        // keep only rows at positions [p_lo, p_hi) of the mean order (a shard)
        int s8[8];
#pragma unroll
        for (int q = 0; q < 8; q++) s8[q] = i8[q] >= 0 ? sigpos[i8[q]] : -1;
#pragma unroll
        for (int q = 0; q < 8; q++) k8[q] = k8[q] && s8[q] >= p_lo && s8[q] < p_hi;
    }
    unsigned bal[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
        bal[q] = __ballot_sync(0xffffffffu, k8[q]);
        if (lane == 0) wcnt[q][wid] = __popc(bal[q]);
    }
    __syncthreads();
    int total = 0;
#pragma unroll
    for (int q = 0; q < 8; q++)
#pragma unroll
        for (int w = 0; w < 8; w++) total += wcnt[q][w];
    if (wid == 0) {
        int prefix = 0;
        if (b == 0) {
            if (lane == 0) atomicExch(status, kStPre | (unsigned long long)(unsigned)total);
        } else {
            if (lane == 0) atomicExch(status + b, kStAgg | (unsigned long long)(unsigned)total);
            int j = b - 1;  // the nearest predecessor not yet added
            unsigned long long t0 = 0;
            bool ok = true;
            for (uint32_t it = 0; ok; ++it) {
                // a window of the 128 nearest predecessors not yet added:
                // position w = 32 k + lane is block j - w
                unsigned long long v[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int jj = j - (32 * k + lane);
                    v[k] = jj >= 0 ? *(volatile const unsigned long long*)(status + jj) : kStPre;  // before block 0: 0
                }
                int fp = 128;  // nearest position holding an inclusive prefix
                bool wait = false;
#pragma unroll
                for (int k = 3; k >= 0; k--) {
                    const unsigned pre = __ballot_sync(0xffffffffu, (v[k] & kStPre) != 0);
                    if (pre) fp = 32 * k + __ffs(pre) - 1;
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const unsigned ready = __ballot_sync(0xffffffffu, (v[k] & (kStPre | kStAgg)) != 0);
                    const int top = fp - 32 * k;  // positions 32 k .. 32 k + top of this word are needed
                    const unsigned need = top >= 31 ? 0xffffffffu : (top >= 0 ? (2u << top) - 1u : 0u);
                    wait = wait || (ready & need) != need;
                }
                if (wait) {  // a predecessor in the window has not published
                    if ((it & 63u) == 0u) {
                        // lane 0's clock decides for the whole warp (the loop stays warp-uniform)
                        const unsigned long long t = __shfl_sync(0xffffffffu, gtimer(), 0);
                        if (t0 == 0) t0 = t;
                        if (t - t0 > 2000000000ull) {
                            if (lane == 0) atomicExch(&ctrl->err, DD_ETIMEOUT);
                            ok = false;
                        }
                    }
                    continue;
                }
                int val = 0;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int w = 32 * k + lane;
                    val += w <= fp && j - w >= 0 ? (int)(unsigned)(v[k] & 0xffffffffull) : 0;
                }
                val = __reduce_add_sync(0xffffffffu, val);
                prefix += val;
                if (fp < 128) break;
                j -= 128;
            }
            if (lane == 0) atomicExch(status + b, kStPre | (unsigned long long)(unsigned)(prefix + total));
        }
        if (lane == 0) {
            sh_base = prefix;
            if (b == nb - 1) *cnt_out = prefix + total;
        }
    }
    __syncthreads();
    int pos = sh_base;
#pragma unroll
    for (int q = 0; q < 8; q++) {
        int before = 0;
#pragma unroll
        for (int w = 0; w < 8; w++) before += w < wid ? wcnt[q][w] : 0;
        if (bal[q] & (1u << lane)) out[pos + before + __popc(bal[q] & lt)] = i8[q];
#pragma unroll
        for (int w = 0; w < 8; w++) pos += wcnt[q][w];
    }
}

// Top-k threshold of one pass, run by the last block (256 threads) of that
// pass's histogram launch: the bin (from the top) whose cumulative count
// reaches the number of rows still wanted.  Thread t sums 16 bins in
// descending order; a block inclusive scan of those sums finds the one bin
// where the running count crosses it.  Pass 0 records the bin and the rows
// still needed inside it; pass 1 refines the threshold to 2^7 ulps.
constexpr int kTopkThreads = 256;
__device__ void topk_threshold(Ctrl* ctrl, int k, int pass, const int* hist) {
    __shared__ int part[kTopkThreads / 32];
    __shared__ int found, above, total;
    const int sel = pass == 0 ? 0 : ctrl->topk_bin;
    if (sel < 0) return;  // pass 0 took every row (uniform over the block)
    const int want = pass == 0 ? k : ctrl->topk_need;
    constexpr int kPer = kTopkBins / kTopkThreads;
    const int t = threadIdx.x;  // bins [4095 - kPer t - (kPer - 1), 4095 - kPer t]
    int c[kPer], s = 0;
#pragma unroll
    for (int q = 0; q < kPer; q++) {
        c[q] = __ldcg(&hist[kTopkBins - 1 - kPer * t - q]);
        s += c[q];
    }
    const int lane = t & 31, wid = t >> 5;
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) part[wid] = incl;
    if (t == 0) found = 0x7fffffff;
    __syncthreads();
    if (wid == 0) {
        const int v = lane < kTopkThreads / 32 ? part[lane] : 0;
        int cc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, cc, o);
            if (lane >= o) cc += u;
        }
        if (lane < kTopkThreads / 32) part[lane] = cc - v;
    }
    __syncthreads();
    int run = part[wid] + incl - s;
#pragma unroll
    for (int q = 0; q < kPer; q++) {
        const int before = run;
        run += c[q];
        if (before < want && run >= want) {
            atomicMin(&found, kPer * t + q);
            above = before;  // written by the single crossing thread
            total = run;
        }
    }
    __syncthreads();
    if (t == 0) {
        if (found == 0x7fffffff) {  // fewer rows than wanted
            if (pass == 0) {
                ctrl->topk_thr = 0u;  // take them all
                ctrl->topk_bin = -1;
            } else {
                ctrl->topk_thr = (uint32_t)sel << 19;
            }
        } else {
            const int b = kTopkBins - 1 - found;
            if (pass == 0) {
                // refine only when the first pass would take over twice the rows wanted
                ctrl->topk_bin = total > 2 * want ? b : -1;
                ctrl->topk_need = want - above;
                ctrl->topk_thr = (uint32_t)b << 19;
            } else {
                ctrl->topk_thr = ((uint32_t)sel << 19) | ((uint32_t)b << 7);
            }
        }
    }
}

// Top-k radix select over the rows' running minima (alive rows with a finite
// upper bound only), two
// passes of 12 bits each: pass 0 histograms float bits >> 19; pass 1
// histograms bits 7..18 of the rows inside the bin that holds the k-th row.
// The last block of each pass (a ticket per selection and pass) computes the
// pass's threshold.
__global__ void __launch_bounds__(kTopkThreads) k_topk_hist(ListRef in, const uint32_t* __restrict__ rmin,
                                                            TcBound tb, Ctrl* ctrl, int pass, const int* gate, int k,
                                                            int site) {
    __shared__ int h[kTopkBins];
    __shared__ bool last;
    if (gate && *gate <= k) {  // too few rows to be worth a separate wave: select no row
        if (pass == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
            ctrl->topk_thr = 0xffffffffu;
            ctrl->topk_bin = -1;
        }
        return;
    }
    for (int b = threadIdx.x; b < kTopkBins; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const int cnt = *in.cnt_dev;
    const int off = in.off_dev ? *in.off_dev : 0;
    const uint32_t bsf = ctrl->bsf;
    const int sel = pass == 0 ? 0 : ctrl->topk_bin;
    if (sel >= 0) {
        // 4 rows per thread and step, their loads issued together
        constexpr int U = 4;
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r0 < cnt; r0 += U * stride) {
            int iv[U];
#pragma unroll
            for (int u = 0; u < U; u++) iv[u] = r0 + u * stride < cnt ? in.base[off + r0 + u * stride] : -1;
            bool ok[U];
            uint32_t rk[U];
            // rows without a finite upper bound are not ranked (their full scans
            // could not be pruned; they are scanned with the rest, abandoning early)
            alive_batch<U>(tb, iv, rmin, bsf, 0u, kNoBound, ok, rk);
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (!ok[u]) continue;
                const uint32_t b = rk[u];
                if (pass == 0)
                    atomicAdd(&h[b >> 19], 1);
                else if ((int)(b >> 19) == sel)
                    atomicAdd(&h[(b >> 7) & (kTopkBins - 1)], 1);
            }
        }
    }
    __syncthreads();
    int* dst = pass == 0 ? ctrl->topk_hist : ctrl->topk_hist2;
    for (int b = threadIdx.x; b < kTopkBins; b += blockDim.x)
        if (h[b]) atomicAdd(&dst[b], h[b]);
    __threadfence();  // this block's counts are visible before its ticket
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&ctrl->topk_ticket[site], 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    topk_threshold(ctrl, k, pass, dst);
}

// Rows alive after the last wave have scanned every column: their running
// minimum is their nearest-neighbour distance.  Best-so-far and argmax key.
// (Gram form: the best-so-far takes the row's proven lower bound D - F_i(D).)
__global__ void __launch_bounds__(256) k_complete(ListRef in, const uint32_t* __restrict__ rmin, TcBound tb,
                                                  Ctrl* ctrl) {
    const int cnt = *in.cnt_dev;
    const int off = in.off_dev ? *in.off_dev : 0;
    const uint32_t bsf = ctrl->bsf;
    unsigned long long best = 0;
    uint32_t bmax = 0;
    int done = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < cnt; r += gridDim.x * blockDim.x) {
        const int i = in.base[off + r];
        const uint32_t b = rmin[i];
        if (!is_alive(tb, i, b, bsf)) continue;
        const unsigned long long key = ((unsigned long long)b << 32) | (unsigned long long)(0xffffffffu - (uint32_t)i);
        best = key > best ? key : best;
        const uint32_t lbits = tb.on ? __float_as_uint(row_lb(tb, i, __uint_as_float(b))) : b;
        bmax = lbits > bmax ? lbits : bmax;
        done++;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long ok = __shfl_xor_sync(0xffffffffu, best, o);
        best = ok > best ? ok : best;
        uint32_t ob = __shfl_xor_sync(0xffffffffu, bmax, o);
        bmax = ob > bmax ? ob : bmax;
        done += __shfl_xor_sync(0xffffffffu, done, o);
    }
    if ((threadIdx.x & 31) == 0 && done) {
        atomicMax(&ctrl->key, best);
        atomicMax(&ctrl->bsf, bmax);
        atomicAdd(&ctrl->ncomplete, done);
    }
}

// Column range of every 128-row tile of a list in the mean-bucketed order.
// kind 0 (local): the tile's own positions widened by K on each side.
// kind 1 (lower bound): for each row, the bins within sqrt(R / n) of its mean,
// R = its running minimum; d^2 >= n (mu_i - mu_j)^2 means no column outside
// can lower R.  A row with no finite R gets every column.
__global__ void __launch_bounds__(128) k_tile_ranges(ListRef L, int kind, int K, int seg_cols,
                                                     const int32_t* __restrict__ sigpos,
                                                     const int32_t* __restrict__ mubin,
                                                     const int32_t* __restrict__ binstart,
                                                     const uint32_t* __restrict__ rmin, TcBound tb,
                                                     const double* stats, int n, int N, int4* __restrict__ ranges,
                                                     int* smax) {
    __shared__ int red[4][4];
    const int cnt = *L.cnt_dev;
    const int off = L.off_dev ? *L.off_dev : 0;
    // one tile per block iteration (the grid is sized for a few tiles per SM, not for the longest list)
    for (int t = blockIdx.x; t * 128 < cnt; t += gridDim.x) {
        __syncthreads();  // red[] of the previous tile has been read
        const int r = t * 128 + threadIdx.x;
        int lo = 0x7fffffff, hi = -1, qmin = 0x7fffffff, qmax = -1;
        if (r < cnt) {
            const int i = L.base[off + r];
            const int q = sigpos[i];
            qmin = qmax = q;
            if (kind == 0) {
                lo = q - K;
                hi = q + 1 + K;
            } else {
                const float R = row_ub(tb, i, __uint_as_float(rmin[i]));
                const double w = stats[7];
                if (!(R < 1e30f) || !(w > 0.0)) {
                    lo = 0;
                    hi = N;
                } else {
                    const double h = sqrt((double)R / (double)n) * (1.0 + 1e-4) + 1e-12;
                    const double kb = ceil(h / w) + 1.0;
                    const int k = kb < (double)kMuBins ? (int)kb : kMuBins;  // NaN -> every bin
                    const int b = mubin[i];
                    lo = binstart[b - k < 0 ? 0 : b - k];
                    hi = binstart[b + k + 1 > kMuBins ? kMuBins : b + k + 1];
                }
            }
        }
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        qmin = __reduce_min_sync(0xffffffffu, qmin);
        qmax = __reduce_max_sync(0xffffffffu, qmax);
        const int wid = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) {
            red[0][wid] = lo;
            red[1][wid] = hi;
            red[2][wid] = qmin;
            red[3][wid] = qmax;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w2 = 1; w2 < 4; w2++) {
                lo = min(lo, red[0][w2]);
                hi = max(hi, red[1][w2]);
                qmin = min(qmin, red[2][w2]);
                qmax = max(qmax, red[3][w2]);
            }
            lo = lo < 0 ? 0 : lo;
            hi = hi > N ? N : hi;
            int C = (qmin + qmax + 1) / 2;
            C = C < lo ? lo : (C > hi ? hi : C);
            const int side = max(hi - C, C - lo);
            const int nseg = 2 * ((side + seg_cols - 1) / seg_cols);
            ranges[t] = make_int4(lo, hi, C, nseg);
            atomicMax(smax, nseg);
        }
    }
}

// Gram form, after a direct FP32 full scan of the candidate rows (run only when
// the list has more than min_rows rows, like that scan): every row still alive
// scanned all the columns its lower bound admits, so its FP32 upper bound r32
// came from its nearest column, and r32 - 2 margin(r32) is a rigorous lower
// bound on its nearest-neighbour distance.  Raises the best-so-far with them.
__global__ void __launch_bounds__(256) k_complete32(ListRef in, const uint32_t* __restrict__ rmin, TcBound tb,
                                                    const double* stats, int n, int min_rows, Ctrl* ctrl) {
    const int cnt = *in.cnt_dev;
    if (cnt <= min_rows) return;
    const int off = in.off_dev ? *in.off_dev : 0;
    const uint32_t bsf = ctrl->bsf;
    const float u = 5.9604644775390625e-08f;
    const float nf = (float)n, M = (float)stats[2];
    const float gn = nf * u / (1.f - nf * u);
    const float mu6 = 6.f * u * M;
    uint32_t best = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < cnt; r += gridDim.x * blockDim.x) {
        const int i = in.base[off + r];
        if (!is_alive(tb, i, rmin[i], bsf)) continue;
        const float up = __uint_as_float(tb.r32[i]);
        if (!(up < 1e30f)) continue;
        const float margin = 2.f * ((gn + 4.f * u) * up + 8.f * u * M * sqrtf(nf * up) + nf * mu6 * mu6) + 1e-30f;
        const float lb = up - 2.f * margin;
        if (lb > 0.f) best = max(best, __float_as_uint(lb));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best > bsf) atomicMax(&ctrl->bsf, best);
}

// Appends the rows of src to the list dst[0, *cnt) (one block): at most cap
// entries in all; *cnt becomes the new length.
__global__ void __launch_bounds__(1024) k_append_list(ListRef src, int32_t* __restrict__ dst, int* __restrict__ cnt,
                                                      int cap) {
    __shared__ int n0;
    if (threadIdx.x == 0) n0 = *cnt;
    __syncthreads();
    const int ns = *src.cnt_dev;
    const int off = src.off_dev ? *src.off_dev : 0;
    const int take = min(ns, max(cap - n0, 0));
    for (int r = threadIdx.x; r < take; r += blockDim.x) dst[n0 + r] = src.base[off + r];
    __syncthreads();
    if (threadIdx.x == 0) *cnt = n0 + take;
}

__global__ void k_copy_list(ListRef src, int32_t* __restrict__ dst, int* __restrict__ cnt_out) {
    const int cnt = *src.cnt_dev;
    const int off = src.off_dev ? *src.off_dev : 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < cnt; r += gridDim.x * blockDim.x)
        dst[r] = src.base[off + r];
    if (blockIdx.x == 0 && threadIdx.x == 0) *cnt_out = cnt;
}

// Value of a conditional graph node: run its body only when *cnt > thr.
__global__ void k_set_cond(cudaGraphConditionalHandle h, const int* cnt, int thr, int* taken) {
    const unsigned v = *cnt > thr ? 1u : 0u;
    cudaGraphSetConditional(h, v);
    *taken = (int)v;
}

__global__ void k_finalize(const Ctrl* ctrl, dd_result_t* out) {
    if (threadIdx.x != 0) return;
    dd_result_t r;
    r.exact = 0;
    r.computed_pairs = (int64_t)ctrl->pairs;
    r.candidates = ctrl->ncomplete;
    if (ctrl->nonfinite) {
        r.status = DD_ENONFINITE;
        r.index = -1;
        r.nn_distance = 0.0;
    } else if (ctrl->degenerate) {
        // sigma == 0: the normalised series is identically zero, every
        // distance is 0 and the first subsequence wins the tie.
        r.status = DD_OK;
        r.index = 0;
        r.nn_distance = 0.0;
    } else if (ctrl->err) {
        r.status = ctrl->err;
        r.index = -1;
        r.nn_distance = 0.0;
    } else if (ctrl->key == 0ull) {
        r.status = DD_ECUDA;
        r.index = -1;
        r.nn_distance = 0.0;
    } else {
        r.status = DD_OK;
        r.index = (int64_t)(0xffffffffu - (uint32_t)(ctrl->key & 0xffffffffull));
        r.nn_distance = sqrt((double)__uint_as_float((uint32_t)(ctrl->key >> 32)));
    }
    *out = r;
}

// nn2[k] = running minimum of rows[k] (exhaustive profile output); NaN for an
// entry that is not a row (marked -1 by k_sanitize_rows).
__global__ void k_gather_min(const int32_t* __restrict__ rows, int count, const uint32_t* __restrict__ rmin,
                             float* __restrict__ nn2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) nn2[k] = rows[k] >= 0 ? __uint_as_float(rmin[rows[k]]) : __int_as_float(0x7fc00000);
}

// A caller's row list, copied with every entry outside [0, N) replaced by -1
// (which every kernel of the wave treats as no row).
__global__ void k_sanitize_rows(const int32_t* __restrict__ rows, int count, int64_t N, int32_t* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) out[k] = rows[k] >= 0 && rows[k] < N ? rows[k] : -1;
}

// ---------------------------------------------------------------------------
// Host-side sequencing (no synchronisation; counts stay on the device).
constexpr int kSegCols = 512;
constexpr int kSegColsFull = 128;  // FP32 full scans: one column tile per item, so few rows spread over the SMs
constexpr int kSettleMin = 64;   // candidate rows above which the Gram form settles them in FP32 first
constexpr int kSettleTop = 128;  // of those, settled first to raise the best-so-far (above this many)
constexpr int kTimeCols = 256;   // time-local wave: columns on each side of a row tile
constexpr int kFillCols = 2048;  // half-width of the neighbourhood of rows the band wave left unbounded

struct Seq {
    dd_plan_s* p;
    cudaStream_t s;
    int work_slot = 0;
    int cnt_slot = 0;
    int smax_slot = 0;
    cudaError_t err = cudaSuccess;
    bool tc = false;
    TcBound tb{};

    Seq(dd_plan_s* plan, cudaStream_t stream) : p(plan), s(stream) {
        tc = p->opt.precision != DD_FP32;
        if (tc) {
            tb.alpha = p->alpha;
            tb.gam = p->gam;
            tb.q2 = p->q2;
            tb.beta = kTcBeta;
            tb.on = 1;
            tb.r32 = p->rmin32;
        }
        tb.excl = p->excl;
    }

    void check() {
        if (err == cudaSuccess) err = cudaGetLastError();
    }
    void keep(cudaError_t e) {
        if (err == cudaSuccess) err = e;
    }
    int* cnt_ptr(int slot) { return &p->ctrl->cnt[slot]; }

    // Cand (Eq. 7) as the head of the word order; a shard keeps only its own positions
    ListRef cand_list(int32_t* out) {
        if (p_lo != 0 || p_hi != (int)p->N) return compact(constant_list(p->order, (int)p->N), out, 2, true);
        const int slot = cnt_slot++;
        k_cand_count<<<1, 1, 0, s>>>(p->ctrl, p->opt.phase1_max, cnt_ptr(slot));
        p->launches++;
        check();
        return ListRef{p->order, nullptr, cnt_ptr(slot)};
    }

    ListRef constant_list(const int32_t* base, int count) {
        const int slot = cnt_slot++;
        k_set_int<<<1, 1, 0, s>>>(cnt_ptr(slot), count);
        p->launches++;
        return ListRef{base, nullptr, cnt_ptr(slot)};
    }

    // One wave of distance tiles for the rows of `rows`.  a_direct: the list
    // is the mean-bucketed order itself (its operand rows need no packing).
    // force_fp32: run the wave with the FP32 kernel in a Gram-form plan too (it then
    // publishes rigorous FP32 upper bounds to rmin32, see TcBound).
    void scan(int kind, ListRef rows, ColSpec col, int abandon, const int* smax = nullptr, bool a_direct = false,
              bool force_fp32 = false, int min_rows = 0) {
        if (tc && col.mode == 1) return;  // the same-word wave runs in the FP32 form only
        const int slot = work_slot++;
        if (work_slot > kMaxLaunchSlots) {
            err = cudaErrorInvalidValue;
            return;
        }
        int wave = -1;
        if (p->nwaves < kMaxWaves) {
            wave = p->nwaves++;
            p->waves[wave] = dd_plan_s::WaveMeta{kind, (p->profiling && !p->in_cond) ? p->ev_used : -1};
        }
        if (!tc || force_fp32) {
            ScanArgs a{};
            if (tc) {
                a.tb = tb;
                a.r32 = p->rmin32;
                a.stats = p->stats;
            }
            a.t32 = p->t32;
            a.N = (int)p->N;
            a.n = p->n;
            a.rows = rows;
            a.order = p->order;
            a.pos_of = p->pos_of;
            a.code = p->code;
            a.hist = p->hist;
            a.word_start = p->word_start;
            a.col = col;
            a.sig = p->sig;
            a.ranges = p->ranges;
            a.smax = smax;
            a.seg_cols = col.seg_cols > 0 ? col.seg_cols : kSegCols;
            a.rmin = p->rmin;
            a.ctrl_ro = p->ctrl;
            a.ctrl = p->ctrl;
            a.abandon = abandon;
            a.work_slot = slot;
            // time-local and same-word waves: spread a tile's few columns over blocks
            a.min_seg_tiles = col.mode == 4 || col.mode == 1 ? 1 : 4;
            a.min_rows = min_rows;
            a.wave = wave;
            const int grid = scan_fp32_grid(p);
            a.target_items = grid * 2;
            prof_mark(p, s, true);
            keep(launch_scan_fp32(a, grid, s));
            prof_mark(p, s, false);
            p->launches++;
            return;
        }
        if (!a_direct) keep(launch_gather_rows(p, rows, s));
        TcArgs t{};
        t.N = (int)p->N;
        t.n = p->n;
        t.nka = p->kpad / 64;
        t.stages = tc_stages(p->kpad);
        t.seg_cols = kSegCols;
        t.mode = col.mode == 2 || col.mode == 3 ? col.mode : 0;
        t.rows = rows;
        t.a_direct = a_direct ? 1 : 0;
        t.a_row0 = a_direct ? (int)(rows.base - p->sig) : 0;  // direct lists are slices of the mean order
        t.sig = p->sig;
        t.coldat = p->coldat;
        t.rowmu = p->rowmu;
        t.rowc = p->rowc;
        t.alpha = p->alpha;
        t.gam = p->gam;
        t.q2 = p->q2;
        t.beta = tb.beta;
        t.ranges = p->ranges;
        t.sigpos = p->sigpos;
        t.local_k = t.mode == 2 ? col.local_cols : 0;
        t.stall = p->inject == DD_INJECT_STALL_TC ? 1 : 0;
        p->inject = 0;
        t.smax = smax;
        t.rmin = p->rmin;
        t.ctrl = p->ctrl;
        t.stats = p->stats;
        t.abandon = abandon;
        t.work_slot = slot;
        const uint32_t ty = p->opt.precision == DD_TC_BF16 ? 1u : 0u;
        t.wave = wave;
        t.r32 = p->rmin32;
        t.idesc = (1u << 4) | (ty << 7) | (ty << 10) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        prof_mark(p, s, true);
        keep(launch_scan_tc(p, t, !a_direct, s));
        prof_mark(p, s, false);
        p->launches++;
    }

    // Column ranges of the list's tiles (kind 0: local +-K, kind 1: lower bound).
    const int* ranges(ListRef rows, int kind, int K, int seg = kSegCols) {
        const int slot = smax_slot++;
        if (smax_slot > 64) {
            err = cudaErrorInvalidValue;
            return nullptr;
        }
        const int tiles = (int)((p->N + 127) / 128);
        const int grid = tiles < p->sm_count * 8 ? tiles : p->sm_count * 8;
        k_tile_ranges<<<grid, 128, 0, s>>>(rows, kind, K, seg, p->sigpos, p->mubin, p->binstart, p->rmin, tb,
                                            p->stats, p->n, (int)p->N, p->ranges, &p->ctrl->smax[slot]);
        p->launches++;
        check();
        return &p->ctrl->smax[slot];
    }

    // Order-preserving compaction of `in` into `out`; returns the new list.
    int p_lo = 0, p_hi = 0;  // this search's shard of the mean order

    // Launches between begin_if and end_if run only when *cnt > thr.  Inside a
    // graph capture they form the body of a conditional node whose value a
    // kernel sets on the device, so a skipped block costs one node instead of
    // one per launch.  Outside a capture they are launched as usual (each of
    // them checks the same gate itself).  No events are recorded in a body.
    cudaStream_t saved = nullptr;
    bool in_if = false;
    int* if_taken = nullptr;
    int ncond = 0;
    int64_t if_start = 0;

    void begin_if(const int* cnt, int thr) {
        if (!p->capturing || err != cudaSuccess) return;
        cudaStreamCaptureStatus st;
        cudaGraph_t g = nullptr;
        keep(cudaStreamGetCaptureInfo(s, &st, nullptr, &g));
        cudaGraphConditionalHandle h{};
        keep(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
        if (err != cudaSuccess) return;
        if (ncond >= 8) {
            err = cudaErrorInvalidValue;
            return;
        }
        if_taken = &p->ctrl->cond[ncond++];
        k_set_cond<<<1, 1, 0, s>>>(h, cnt, thr, if_taken);
        p->launches++;
        check();
        const cudaGraphNode_t* deps = nullptr;
        const cudaGraphEdgeData* ed = nullptr;
        size_t nd = 0;
        keep(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, &ed, &nd));
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeIf;
        np.conditional.size = 1;
        cudaGraphNode_t cn = nullptr;
        keep(cudaGraphAddNode(&cn, g, deps, ed, nd, &np));
        if (err != cudaSuccess) return;
        keep(cudaStreamUpdateCaptureDependencies(s, &cn, nullptr, 1, cudaStreamSetCaptureDependencies));
        keep(cudaStreamBeginCaptureToGraph(p->body_stream, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal));
        if (err != cudaSuccess) return;
        saved = s;
        s = p->body_stream;
        in_if = true;
        p->in_cond = true;
        if_start = p->launches;
    }

    void end_if() {
        if (!in_if) return;
        cudaGraph_t body = nullptr;
        keep(cudaStreamEndCapture(s, &body));
        s = saved;
        in_if = false;
        p->in_cond = false;
        p->bodies.push_back(dd_plan_s::CondBody{if_taken, p->launches - if_start});
    }

    // cnt_out: write the count there instead of a new slot (refreshing a list in place)
    int csite = 0;
    ListRef compact(ListRef in, int32_t* out, int pred, bool shard_only = false, int* cnt_out = nullptr) {
        const int nblk = p->cstat_stride;
        if (csite >= kCompactSites) {
            err = cudaErrorInvalidValue;
            return in;
        }
        const int site = csite++;
        int* cnt = cnt_out;
        if (!cnt) {
            const int slot = cnt_slot++;
            if (cnt_slot > kMaxListSlots) {
                err = cudaErrorInvalidValue;
                return in;
            }
            cnt = cnt_ptr(slot);
        }
        k_compact<<<nblk, 256, 0, s>>>(in, p->rmin, tb, p->ctrl, pred, p->code, p->hist, p->opt.phase1_max,
                                       shard_only ? p->sigpos : nullptr, p_lo, p_hi, site,
                                       p->cstat + (size_t)site * nblk, out, cnt);
        p->launches += 1;
        check();
        return ListRef{out, nullptr, cnt};
    }

    // dst[0, *src.cnt) = src rows, count into cnt_out
    // Appends src to the list at dst whose count is *cnt (at most N entries).
    void append(ListRef src, int32_t* dst, const int* cnt) {
        k_append_list<<<1, 1024, 0, s>>>(src, dst, const_cast<int*>(cnt), (int)p->N);
        p->launches++;
        check();
    }

    void copy_list(ListRef src, int32_t* dst, int* cnt_out) {
        k_copy_list<<<p->sm_count * 2, 256, 0, s>>>(src, dst, cnt_out);
        p->launches++;
        check();
    }

    void complete(ListRef in) {
        const int g = (int)((p->N + 1023) / 1024);
        k_complete<<<g < 1024 ? g : 1024, 256, 0, s>>>(in, p->rmin, tb, p->ctrl);
        p->launches++;
        check();
    }

    // gate: skip (select nothing) unless *gate > k
    int topk_calls = 0;
    void topk(ListRef in, int k, const int* gate = nullptr) {
        // the control block starts zeroed: only later calls clear the histograms
        if (topk_calls++ > 0)
            keep(cudaMemsetAsync(p->ctrl->topk_hist, 0, sizeof(p->ctrl->topk_hist) + sizeof(p->ctrl->topk_hist2),
                                 s));
        const int site = 2 * (topk_calls - 1);
        if (site + 1 >= (int)(sizeof(p->ctrl->topk_ticket) / sizeof(int))) {
            err = cudaErrorInvalidValue;
            return;
        }
        for (int pass = 0; pass < 2; pass++)
            k_topk_hist<<<2 * p->sm_count, kTopkThreads, 0, s>>>(in, p->rmin, tb, p->ctrl, pass, gate, k,
                                                                 site + pass);
        p->launches += 2;
        check();
    }

    // Full scan of each row of `in`: every column whose lower bound
    // n (mu_i - mu_j)^2 can still undercut the row's upper bound, nearest mean
    // first, abandoning against the best-so-far; survivors complete.
    void full(int kind, ListRef in) {
        // the FP32 kernel computes whole 128-row tiles even for a few rows: one
        // column tile per item spreads a short list over more SMs
        const int seg = tc ? kSegCols : kSegColsFull;
        const int* sm = ranges(in, 1, 0, seg);
        scan(kind, in, ColSpec{2, 0, 0, 0, seg}, 1, sm);
        complete(in);
    }
};

}  // namespace

cudaError_t launch_search(dd_plan_s* p, const float* T, dd_result_t* out_dev, cudaStream_t s) {
    if (p->opt.znorm == 1) return launch_search_window(p, T, out_dev, s);
    p->launches = 0;
    p->nwaves = 0;
    p->bodies.clear();
    cudaError_t e = cudaMemsetAsync(p->ctrl, 0, sizeof(Ctrl), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(p->cstat, 0, sizeof(unsigned long long) * kCompactSites * p->cstat_stride, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->rmin, 0x7f, sizeof(uint32_t) * p->N, s);
    if (e == cudaSuccess && p->rmin32) e = cudaMemsetAsync(p->rmin32, 0x7f, sizeof(uint32_t) * p->N, s);
    if (e != cudaSuccess) return e;
    // The SAX words and the word order (needed from Algorithm 3 on) are built on
    // a side stream.  In the Gram form they start after the mean order (whose
    // latency-bound sort they would otherwise crowd) and run beside the operand
    // build and the first wave; the FP32 form's exhaustive wave visits columns
    // in the word order, so there they start right after the statistics.
    const bool tc_plan = p->opt.precision != DD_FP32;
    auto fork_words = [&]() -> cudaError_t {
        cudaError_t f = cudaEventRecord(p->ev_fork, s);
        if (f == cudaSuccess) f = cudaStreamWaitEvent(p->side_stream, p->ev_fork, 0);
        if (f == cudaSuccess) f = launch_prep_words(p, p->side_stream);
        if (f == cudaSuccess) f = cudaEventRecord(p->ev_join, p->side_stream);
        return f;
    };
    e = launch_prep_common(p, T, s);
    if (e == cudaSuccess && !tc_plan) e = fork_words();
    if (e == cudaSuccess) e = launch_prep_mean(p, s);
    if (e == cudaSuccess && tc_plan) e = fork_words();
    if (e != cudaSuccess) return e;

    Seq q(p, s);
    if (q.tc) q.keep(launch_tc_prep(p, s));
    const dd_options_t& o = p->opt;
    // every row of this shard (all rows unless sharded), in the mean-bucketed order
    const int G = o.shard_count > 1 ? o.shard_count : 1;
    const int64_t p_lo = p->N * o.shard_index / G, p_hi = p->N * (o.shard_index + 1) / G;
    ListRef all = q.constant_list(p->sig + p_lo, (int)(p_hi - p_lo));
    q.p_lo = (int)p_lo;
    q.p_hi = (int)p_hi;
    bool joined = false;
    auto join = [&]() {
        if (!joined) q.keep(cudaStreamWaitEvent(s, p->ev_join, 0));
        joined = true;
    };
    ListRef rest = all;  // the rows the last wave scanned
    if (!o.early_abandon) {
        // every row scans every column; the argmax runs over all rows.  The FP32
        // form visits the columns in the word order: wait for the side stream.
        join();
        q.scan(DD_WAVE_EXHAUSTIVE, all, ColSpec{0, 0, (int)p->N, 0}, 0, nullptr, true);
        q.complete(all);
    } else {
        // Upper bounds for every row from its nearest-mean neighbourhood.
        if (o.local_cols > 0) {
            if (q.tc) {
                // tensor-core form: one 128 x 256 band tile per row tile
                q.scan(DD_WAVE_BAND, all, ColSpec{3, 0, 0, 0}, 1, nullptr, true);
                // rows the band left without a finite upper bound (every column of
                // their band tile was within n of them in time): a wider
                // neighbourhood in the mean order, row by row
                ListRef lone = q.compact(all, p->list[0], 3);
                const int* sm = q.ranges(lone, 0, kFillCols);
                q.scan(DD_WAVE_LOCAL, lone, ColSpec{2, 0, 0, kFillCols}, 1, sm);
            } else {
                const int* sm = q.ranges(all, 0, o.local_cols);
                q.scan(DD_WAVE_LOCAL, all, ColSpec{2, 0, 0, 0}, 1, sm, true);
            }
        }
        join();
        // Algorithm 3 (PotentialDiscord): full scans of the Cand rows (rarest SAX
        // words).  They run in one wave with the rows of largest upper bound
        // (the likeliest discords), which raise the best-so-far further: the
        // top rows are selected first, from the first wave's bounds, and the
        // Cand rows appended to their list (a row in both is scanned twice in
        // the wave; Cand rows beyond N entries stay alive for the rest wave).
        // Few rows die in these waves, so the selections read every row; a row
        // once ruled out stays ruled out (the best-so-far only grows, upper
        // bounds only shrink), so the final candidates are a subset of the
        // last wave's rows.
        ListRef cand = q.cand_list(p->list[0]);
        const ListRef alive = all;
        if (o.refine_k > 0) {
            q.topk(alive, o.refine_k);
            ListRef first = q.compact(alive, p->list[2], 1);
            q.append(cand, p->list[2], first.cnt_dev);
            q.full(DD_WAVE_CAND, first);
        } else {
            q.full(DD_WAVE_CAND, cand);
        }
        // rows still alive after the top wave (recomputed below if more waves run)
        rest = q.compact(alive, p->list[2], 0);
        // Algorithm 4 scans a row's other candidates in index order, which for a
        // periodic series meets a match one period away; the mean order scatters
        // those.  So when more than refine_k rows survive, every one of them (in
        // time order) first scans the columns just outside its exclusion zone,
        // with direct FP32 differences (in the Gram form their rigorous upper
        // bounds go to rmin32).  Those bounds are close to each row's nearest-
        // neighbour distance where the first-wave bounds of a periodic series are
        // not, so the rows are ranked again and the new top rows fully scanned:
        // the best-so-far then reaches the discord before the rest.
        q.begin_if(rest.cnt_dev, o.refine_k);
        ListRef tl = q.compact(q.constant_list(p->seq_rows, (int)p->N), p->list[3], 0, true);
        q.scan(DD_WAVE_TIME, tl, ColSpec{4, 0, 0, kTimeCols}, 1, nullptr, false, true, o.refine_k);
        if (o.refine_k > 0) {
            q.topk(alive, o.refine_k, rest.cnt_dev);
            ListRef top2 = q.compact(alive, p->list[0], 1);
            q.full(DD_WAVE_TOP, top2);
        }
        q.compact(alive, p->list[2], 0, false, const_cast<int*>(rest.cnt_dev));  // refresh `rest`
        q.end_if();
        // Algorithm 4 (RefineDiscord) over the remaining rows: rows sharing the
        // SAX word first (Index_Word), then every column the bound allows.
        if (o.word_cols > 0 && !q.tc) {
            ListRef words = q.constant_list(p->order, (int)p->N);
            ListRef wl = q.compact(words, p->list[3], 0);
            q.scan(DD_WAVE_WORD, wl, ColSpec{1, 0, 0, o.word_cols}, 1);
            rest = q.compact(alive, p->list[2], 0);
        }
        q.full(DD_WAVE_REST, rest);
    }
    join();
    if (q.tc) {
        // rows still alive after the last wave (a subset of the rows it scanned)
        ListRef cands = q.compact(rest, p->list[3], 0);
        if (o.early_abandon) {
            // Many rows the Gram bound cannot rule out (data whose nearest-neighbour
            // distances lie within the bound of each other): settle them first with
            // direct FP32 full scans, whose error bound is far tighter, and raise the
            // best-so-far with their FP32 lower bounds.  Skipped on the device for
            // short lists.
            q.begin_if(cands.cnt_dev, kSettleMin);
            // The rows of largest upper bound first (none when at most kSettleTop rows
            // remain): their FP32 lower bounds raise bsf close to the discord's distance,
            // so that the full settle wave below abandons the other rows early instead
            // of scanning all their columns.
            q.topk(cands, kSettleTop, cands.cnt_dev);
            ListRef st = q.compact(cands, p->list[0], 1);
            const int* sm1 = q.ranges(st, 1, 0);
            q.scan(DD_WAVE_SETTLE, st, ColSpec{2, 0, 0, 0}, 1, sm1, false, true, 0);
            const int g1 = (int)((p->N + 1023) / 1024);
            k_complete32<<<g1 < 1024 ? g1 : 1024, 256, 0, q.s>>>(st, p->rmin, q.tb, p->stats, p->n, 0, p->ctrl);
            p->launches++;
            q.check();
            const int* sm = q.ranges(cands, 1, 0);
            q.scan(DD_WAVE_SETTLE, cands, ColSpec{2, 0, 0, 0}, 1, sm, false, true, kSettleMin);
            const int g = (int)((p->N + 1023) / 1024);
            k_complete32<<<g < 1024 ? g : 1024, 256, 0, q.s>>>(cands, p->rmin, q.tb, p->stats, p->n, kSettleMin,
                                                               p->ctrl);
            p->launches++;
            q.check();
            // the survivors, back in place of the candidate list
            ListRef c2 = q.compact(cands, p->list[2], 0);
            q.copy_list(c2, p->list[3], const_cast<int*>(cands.cnt_dev));
            q.end_if();
        }
        // every row the bounds cannot rule out, rescored exactly in FP64
        q.keep(launch_rescore(p, cands, q.tb, q.work_slot++, out_dev, s));
    } else {
        k_finalize<<<1, 32, 0, s>>>(p->ctrl, out_dev);
        p->launches++;
    }
    q.check();
    return q.err;
}

cudaError_t launch_profile(dd_plan_s* p, const float* T, const int32_t* rows, int count, float* nn2,
                           cudaStream_t s) {
    if (p->opt.znorm == 1)
        return rows ? launch_rows_window(p, T, rows, count, nn2, s) : launch_profile_diag(p, T, nn2, nullptr, s);
    p->launches = 0;
    p->nwaves = 0;
    p->bodies.clear();
    cudaError_t e = cudaMemsetAsync(p->ctrl, 0, sizeof(Ctrl), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(p->rmin, 0x7f, sizeof(uint32_t) * p->N, s);
    if (e == cudaSuccess && p->rmin32) e = cudaMemsetAsync(p->rmin32, 0x7f, sizeof(uint32_t) * p->N, s);
    if (e != cudaSuccess) return e;
    e = launch_prep(p, T, s);
    if (e != cudaSuccess) return e;
    Seq q(p, s);
    if (q.tc) q.keep(launch_tc_prep(p, s));
    const int32_t* r = p->seq_rows;
    const int c = rows ? count : (int)p->N;
    if (rows) {  // the caller's rows, with out-of-range entries marked (count <= N, checked by the caller)
        k_sanitize_rows<<<(c + 255) / 256, 256, 0, s>>>(rows, c, p->N, p->list[0]);
        p->launches++;
        r = p->list[0];
    }
    ListRef L = q.constant_list(r, c);
    q.scan(DD_WAVE_EXHAUSTIVE, L, ColSpec{0, 0, (int)p->N, 0}, 0);
    k_gather_min<<<(c + 255) / 256, 256, 0, s>>>(r, c, p->rmin, nn2);
    p->launches++;
    q.check();
    return q.err;
}

}  // namespace dd
