// rescore.cu -- exact FP64 nearest-neighbour distances of the rows the
// tensor-core bound could not rule out, and the final argmax (Algorithm 4
// returns sqrt(dist_bsf); Section 2.1: the discord maximises the nearest
// non-self-match distance, ties -> smallest index).
//
// A candidate row i has an upper bound ub_i >= nn_i^2 from its Gram-form scan.
// Its nearest neighbour j* satisfies n (mu_i - mu_j*)^2 <= d^2(i, j*) <= ub_i,
// so scanning the mean-bucketed order over the bins within sqrt(ub_i / n) of
// mu_i, in FP64 direct differences on t^ (Eq. 1 squared), gives nn_i^2
// exactly (to FP64 rounding).  FP64 is slow on GB300, so each column is first
// evaluated in FP32 (direct differences on the FP32 copy of t^); a column whose
// FP32 value exceeds ub_i by more than that value's proven error bound cannot
// be the nearest neighbour and is skipped.  Work items = (candidate, chunk of
// the range), handed out dynamically; chunk minima meet in an atomicMin on the
// double's bits (non-negative doubles order like their bit patterns).
#include "dd_internal.cuh"

namespace dd {
namespace {

constexpr int kChunk = 64;  // columns per work item: a candidate's range spreads over many blocks

__device__ __forceinline__ void lb_range(float R, int i, int n, int N, const double* stats, const int32_t* mubin,
                                         const int32_t* binstart, int& L, int& H) {
    const double w = stats[7];
    if (!(R < 1e30f) || !(w > 0.0)) {
        L = 0;
        H = N;
        return;
    }
    const double h = sqrt((double)R / (double)n) * (1.0 + 1e-4) + 1e-12;
    const double kb = ceil(h / w) + 1.0;
    const int k = kb < (double)kMuBins ? (int)kb : kMuBins;  // NaN -> every bin
    const int b = mubin[i];
    L = binstart[b - k < 0 ? 0 : b - k];
    H = binstart[b + k + 1 > kMuBins ? kMuBins : b + k + 1];
}

__global__ void __launch_bounds__(256) k_rescore64(ListRef cand, TcBound bound, const uint32_t* __restrict__ rmin,
                                                   const int32_t* __restrict__ sig,
                                                   const int32_t* __restrict__ mubin,
                                                   const int32_t* __restrict__ binstart, const double* stats,
                                                   const double* __restrict__ t64, const float* __restrict__ t32,
                                                   int n, int N, const int32_t* __restrict__ rL,
                                                   const int32_t* __restrict__ rH,
                                                   unsigned long long* __restrict__ ex64, Ctrl* ctrl, int slot) {
    __shared__ int sh_item;
    __shared__ double red[8];
    if (ctrl->nonfinite || ctrl->degenerate) return;
    const float u32 = 5.9604644775390625e-08f;
    const float nf = (float)n;
    const float gn32 = nf * u32 / (1.f - nf * u32);
    const float maxabs = (float)stats[2];
    const int cnt = *cand.cnt_dev;
    const int off = cand.off_dev ? *cand.off_dev : 0;
    const int nchunk = ctrl->resc_nch;  // chunks of the longest candidate range
    const long long items = (long long)cnt * nchunk;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) sh_item = atomicAdd(&ctrl->work[slot], 1);
        __syncthreads();
        const int item = sh_item;
        if (item < 0 || item >= items) {
            // a negative claim: the 32-bit work counter wrapped (more than 2^31 items)
            if (item < 0 && threadIdx.x == 0) atomicExch(&ctrl->err, DD_ENOTSUP);
            break;
        }
        const int r = item / nchunk, c = item % nchunk;
        const int i = cand.base[off + r];
        const float D = __uint_as_float(rmin[i]);
        const int L = rL[r], H = rH[r];
        const int a0 = L + c * kChunk;
        if (a0 >= H) continue;
        const int a1 = min(H, a0 + kChunk);
        double best = INFINITY;
        const double* x = t64 + i;
        const float* x32 = t32 + i;
        const float ub = row_ub(bound, i, D);
        // one warp per column: the lanes stride the subsequence (coalesced loads of
        // both operands) and the partial sums meet in a shuffle reduction
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
        for (int p = a0 + wid; p < a1; p += nwarp) {
            const int j = sig[p];
            const int d = i - j;
            if (d < n && d > -n) continue;
            // FP32 screen: |s32 - s| <= (gamma_n + 4u) s32 + 8u M sqrt(n s32) + n (6 u M)^2, M = max|t^|,
            // u = 2^-24 (inputs rounded to FP32, differences, FMA accumulation of at most n terms per
            // partial sum plus the reduction); doubled for safety.
            const float* y32 = t32 + j;
            float s32 = 0.f;
            for (int k = lane; k < n; k += 32) {
                const float df = x32[k] - y32[k];
                s32 = fmaf(df, df, s32);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s32 += __shfl_xor_sync(0xffffffffu, s32, o);
            const float margin = 2.f * ((gn32 + 4.f * u32) * s32 + 8.f * u32 * maxabs * sqrtf(nf * s32) +
                                        nf * (6.f * u32 * maxabs) * (6.f * u32 * maxabs)) + 1e-30f;
            if (s32 - margin > ub) continue;
            const double* y = t64 + j;
            double s = 0.0;
            for (int k = lane; k < n; k += 32) {
                const double df = x[k] - y[k];
                s = fma(df, df, s);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            best = fmin(best, s);
        }
        // every lane holds its warp's minimum
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = red[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); w++) b = fmin(b, red[w]);
            if (b < INFINITY) atomicMin(ex64 + r, (unsigned long long)__double_as_longlong(b));
        }
    }
}

// The result over the rescored candidates: best64 = the largest exact value,
// then the smallest index attaining it, then the result struct.  Every block
// takes part in the maximum; the last block to finish (a ticket) picks the
// index and writes the result.
__global__ void __launch_bounds__(256) k_best_final(ListRef cand, const unsigned long long* __restrict__ ex64,
                                                    Ctrl* ctrl, dd_result_t* out) {
    __shared__ bool last;
    __shared__ int red[8];
    const int cnt = *cand.cnt_dev;
    const int off = cand.off_dev ? *cand.off_dev : 0;
    unsigned long long m = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < cnt; r += gridDim.x * blockDim.x) {
        const unsigned long long v = ex64[r];
        m = v > m ? v : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, m, o);
        m = u > m ? u : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&ctrl->best64, m);
    __threadfence();  // this block's maximum is visible before its ticket
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&ctrl->best_ticket, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const unsigned long long best = *(volatile const unsigned long long*)&ctrl->best64;
    int idx = 0x7fffffff;
    for (int r = threadIdx.x; r < cnt; r += blockDim.x)
        if (ex64[r] == best) idx = min(idx, cand.base[off + r]);
    idx = __reduce_min_sync(0xffffffffu, idx);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = idx;
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) idx = min(idx, red[w]);
    const int best_idx = min(idx, *(volatile const int*)&ctrl->best_idx);
    ctrl->best_idx = best_idx;
    ctrl->ncandidates = cnt;
    dd_result_t res;
    res.exact = 1;
    res.computed_pairs = (int64_t)ctrl->pairs;
    res.candidates = cnt;
    if (ctrl->nonfinite) {
        res.status = DD_ENONFINITE;
        res.index = -1;
        res.nn_distance = 0.0;
    } else if (ctrl->degenerate) {
        res.status = DD_OK;
        res.index = 0;
        res.nn_distance = 0.0;
    } else if (ctrl->err) {
        res.status = ctrl->err;
        res.index = -1;
        res.nn_distance = 0.0;
    } else if (best_idx == 0x7fffffff) {
        res.status = DD_ECUDA;
        res.index = -1;
        res.nn_distance = 0.0;
    } else {
        res.status = DD_OK;
        res.index = best_idx;
        res.nn_distance = sqrt(__longlong_as_double((long long)best));
    }
    *out = res;
}

__global__ void k_init_best(Ctrl* ctrl) {
    if (threadIdx.x == 0) ctrl->best_idx = 0x7fffffff;
}

// Per candidate: its exact value starts at +inf, and its column range [L, H) of
// the mean order (the lower-bound range of its upper bound) is stored; the
// largest number of kChunk-column chunks of any range sizes the work items.
__global__ void k_init_rescore(ListRef cand, TcBound bound, const uint32_t* __restrict__ rmin,
                               const int32_t* __restrict__ mubin, const int32_t* __restrict__ binstart,
                               const double* stats, int n, int N, unsigned long long* __restrict__ ex64,
                               int32_t* __restrict__ rL, int32_t* __restrict__ rH, Ctrl* ctrl) {
    const int cnt = *cand.cnt_dev;
    const int off = cand.off_dev ? *cand.off_dev : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->best_idx = 0x7fffffff;
    int nch = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < cnt; r += gridDim.x * blockDim.x) {
        const int i = cand.base[off + r];
        int L, H;
        lb_range(row_ub(bound, i, __uint_as_float(rmin[i])), i, n, N, stats, mubin, binstart, L, H);
        rL[r] = L;
        rH[r] = H;
        ex64[r] = 0x7ff0000000000000ull;
        nch = max(nch, (H - L + kChunk - 1) / kChunk);
    }
    nch = __reduce_max_sync(0xffffffffu, nch);
    if ((threadIdx.x & 31) == 0 && nch > 0) atomicMax(&ctrl->resc_nch, nch);
}

}  // namespace

cudaError_t launch_best(dd_plan_s* p, ListRef cand, dd_result_t* out_dev, cudaStream_t s) {
    const unsigned long long* ex = reinterpret_cast<const unsigned long long*>(p->ex64);
    k_init_best<<<1, 32, 0, s>>>(p->ctrl);
    k_best_final<<<p->sm_count, 256, 0, s>>>(cand, ex, p->ctrl, out_dev);
    p->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_rescore(dd_plan_s* p, ListRef cand, TcBound bound, int work_slot, dd_result_t* out_dev,
                           cudaStream_t s) {
    // the column ranges of the candidates live in two row lists that are free by now
    k_init_rescore<<<p->sm_count, 256, 0, s>>>(cand, bound, p->rmin, p->mubin, p->binstart, p->stats, p->n,
                                               (int)p->N, reinterpret_cast<unsigned long long*>(p->ex64), p->list[0],
                                               p->list[1], p->ctrl);
    k_rescore64<<<2 * p->sm_count, 256, 0, s>>>(cand, bound, p->rmin, p->sig, p->mubin, p->binstart, p->stats, p->t64,
                                                 p->t32, p->n, (int)p->N, p->list[0], p->list[1],
                                                 reinterpret_cast<unsigned long long*>(p->ex64), p->ctrl, work_slot);
    k_best_final<<<p->sm_count, 256, 0, s>>>(cand, reinterpret_cast<const unsigned long long*>(p->ex64), p->ctrl,
                                              out_dev);
    p->launches += 3;
    return cudaGetLastError();
}

}  // namespace dd
