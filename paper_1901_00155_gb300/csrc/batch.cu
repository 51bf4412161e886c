// batch.cu -- fused discord search of many independent series (tensor-core
// Gram form): every step of the search is one launch over all series of a
// batch, and the distance tiles of all series are claimed from one device work
// queue by the persistent tcgen05 kernel (scan_tc.cu).
//
// Per series s the method is the one of the single-series search: Eq. 2
// normalisation of s on its own, Eq. 5 row statistics from FP64 prefix sums,
// the mean-bucketed row order (d^2(i, j) >= n (mu_i - mu_j)^2 prunes columns
// exactly), Gram tiles with the per-row error bound F_i(D), Algorithm 4's
// early abandon against s's own best-so-far, and exact FP64 rescoring of
// every row the bound cannot rule out; the discord maximises the nearest
// non-self-match distance (Section 2.1), ties -> smallest index.
//
// Layout.  Series with the same subsequence length n form a group.  A group
// concatenates its series' rows: series s owns rows / positions
// [base_s, base_s + Npad_s), Npad_s = roundup(N_s, 128) + 256; its N_s real rows
// come first (row base_s + i is window i; position base_s + p is the p-th row of
// s in mean order) and the rest is padding (no row; column constants c = +inf).
// Row tiles therefore never span two series, and the 256 padding columns keep
// every distance tile of a series (band tiles reach 64 columns past a row
// tile, segment tiles at most 255 past a segment) inside its own region.
//
// Steps of one group (all launches cover every series of the group):
//   k_b_prep     one block per series: Eq. 2 statistics, normalised series,
//                prefix sums, row statistics, mean bins, mean-order counting sort,
//                per-column constants
//   k_b_build    operand matrix S (centred FP16 / BF16 rows, mean order) and the
//                per-row bound terms
//   band wave    every row tile against the 256 columns around it (mean order)
//   k_b_top      per series, the rows with the largest upper bounds (one tile)
//   top wave     full lower-bound scans of those rows (mode 2 segments)
//   k_b_surv     per series: best-so-far = the largest lower bound of the top
//                rows; the rows whose upper bound still reaches it are compacted
//                into whole tiles of their own series
//   rest wave    their scans, abandoned against the series' best-so-far
//   k_b_cands    per series: best-so-far raised by the completed survivors; the
//                candidates go to the FP64 rescoring, or, when there are more
//                than settle_min of them, into settle tiles of settle_rows rows
//   settle wave  direct FP32 full scans of the settle tiles (scan_fp32.cu),
//                rigorous FP32 upper bounds r32, rows abandoned against the
//                series' best-so-far
//   k_b_cands2   per series: best-so-far raised by the settled rows' FP32
//                lower bounds; the settled rows that still reach it go to FP64
//   k_b_rescore  exact FP64 nearest-neighbour distances of the candidates
//   k_b_best     per series: the largest exact value, smallest index -> result
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "dd_internal.cuh"

namespace dd {

// One series of a batch.  The host writes the layout fields, the device the
// statistics and the result fields.
struct BSer {
    const float* T;       // input values (device)
    int64_t m;            // values
    int64_t vbase;        // first value of the series in the group's t32 / t64 / P1 / P2 (= base)
    int32_t n, N;         // subsequence length, rows
    int32_t base, npad;   // first row / position in the group; rows + padding
    int32_t rb0, rb1;     // 64-row blocks [rb0, rb1) of the group's operand build
    int32_t slot;         // index of the series in the caller's list
    int32_t pad0;
    // written by the device
    double mu, sigma, maxabs, lo, w, inv_w, P2end, scale;
    unsigned scmax, cmax, mumax;  // float bits
    int valid, nonfinite, degenerate;
    int ncand, best_idx;
    unsigned long long best64;
};

// Per group: the control block the tensor-core kernel uses, the group's
// operand scale, and the counters of the per-series kernels.
struct BGrp {
    Ctrl ctrl;
    double gstats[16];  // [2] largest max|t^|, [3] operand scale (power of two), [7] largest mean-bin width
    int prep_next, prep_ticket, top_next, surv_next, cand_next, best_ticket;
    int band_rows, top_rows, rest_rows, rest_tiles, ncand;
    int settle_rows, settle_tiles, cand2_next;
    int pad[2];
    // FP64 rescoring: candidates (bits 40..63) and column chunks (bits 0..39)
    // taken so far, one atomic per candidate, so that chunk bases follow slots
    unsigned long long cand_packed;
};

namespace {

constexpr int kPT = 1024;       // threads of the one-block-per-series kernels
constexpr int kBTop = 128;      // rows of the top tile of each series
constexpr int kBRows = 64;      // rows per block of the operand build
constexpr int kBChunks = 16;    // 64-element chunks per pass of the operand build
constexpr int kColPad = kTcColPad;
constexpr int kPadRows = 256;   // padding rows after the rounded-up rows of a series
constexpr int kRChunk = 64;     // columns per FP64 rescoring work item
constexpr int kNoRow = -(1 << 30);

// Group arrays (rows / positions of the group; t32 .. P2 and the per-series
// arrays are batch-wide).
struct BArr {
    BSer* ser;
    int s0, ns;            // series [s0, s0 + ns) of the batch form this group
    int64_t P;             // rows / positions of the group
    int n, kpad;
    BGrp* G;
    float* t32;            // the series' values at their rows' offsets (base + k)
    double* t64;
    double* P1;
    double* P2;
    int32_t* binstart;     // [series][kMuBins + 1]
    uint32_t* sbsf;        // [series] best-so-far (float bits)
    dd_result_t* res;      // [series] results, by slot
    double* mu_w;
    double* c_w;
    int32_t* mubin;
    int32_t* sig;
    int32_t* sigpos;
    int32_t* rser;
    uint32_t* rmin;
    float* rowmu;
    float* rowc;
    float* rowsc;
    float* alpha;
    float* gam;
    float* q2;
    uint8_t* flag;         // 1: in the top tile, 2: survivor
    float4* coldat;        // [P + 2 kColPad]
    void* S16;             // [kpad / 64][P][64]
    int32_t* list_top;     // [ns * 128]
    int32_t* list_rest;    // [P]
    int4* ranges_top;      // [ns]
    int4* ranges_rest;     // [P / 128]
    int32_t* tser_rest;    // [P / 128]
    int32_t* cand;         // [P]
    unsigned long long* ex64;  // [P]
    int32_t* rL;
    int32_t* rH;
    int64_t* cbase;        // [P] first rescoring chunk of each candidate
    uint32_t* r32;         // [P] rigorous FP32 upper bound of nn^2 from the settle wave (float bits)
    int32_t* list_settle;  // [P]
    int4* ranges_settle;   // [P / 32] (tiles of settle_rows rows)
    int32_t* tser_settle;  // [P / 32]
    int seg_cols;
    int settle_min;        // candidates of a series above which they are settled in FP32 first
    int settle_rows;       // rows per settle tile (32, 64 or 128)
    int bf16;
};

__device__ __forceinline__ double bwarp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum over kPT threads; every thread gets the result.
__device__ double bblock_sum(double v, double* sh) {
    v = bwarp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = lane < kPT / 32 ? sh[lane] : 0.0;
    r = bwarp_sum(r);
    return r;
}

// Block-wide maximum of non-negative float bit patterns (or any unsigned).
__device__ unsigned bblock_umax(unsigned v, unsigned* sh) {
    v = __reduce_max_sync(0xffffffffu, v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    unsigned r = lane < kPT / 32 ? sh[lane] : 0u;
    return __reduce_max_sync(0xffffffffu, r);
}

__device__ float bblock_fmax(float v, float* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    float r = lane < kPT / 32 ? sh[lane] : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    return r;
}

__device__ int bblock_isum(int v, int* sh) {
    v = __reduce_add_sync(0xffffffffu, v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int r = lane < kPT / 32 ? sh[lane] : 0;
    return __reduce_add_sync(0xffffffffu, r);
}

// Exclusive block scan (kPT threads) of two doubles per thread.
__device__ void bexscan2(double& a, double& b, double* sh1, double* sh2) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double ua = __shfl_up_sync(0xffffffffu, ia, o);
        const double ub = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += ua;
            ib += ub;
        }
    }
    __syncthreads();
    if (lane == 31) {
        sh1[wid] = ia;
        sh2[wid] = ib;
    }
    __syncthreads();
    if (wid == 0) {
        const double wa = sh1[lane], wb = sh2[lane];
        double sa = wa, sb = wb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double ua = __shfl_up_sync(0xffffffffu, sa, o);
            const double ub = __shfl_up_sync(0xffffffffu, sb, o);
            if (lane >= o) {
                sa += ua;
                sb += ub;
            }
        }
        sh1[lane] = sa - wa;
        sh2[lane] = sb - wb;
    }
    __syncthreads();
    a = sh1[wid] + (ia - a);
    b = sh2[wid] + (ib - b);
}

// Exclusive block scan (kPT threads) of one int per thread; *total gets the sum.
__device__ int bexscan_i(int v, int* sh, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int iv = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, iv, o);
        if (lane >= o) iv += u;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = iv;
    __syncthreads();
    if (wid == 0) {
        const int w0 = sh[lane];
        int s = w0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += u;
        }
        sh[lane] = s - w0;
        if (lane == 31) sh[32] = s;
    }
    __syncthreads();
    *total = sh[32];
    return sh[wid] + (iv - v);
}

// FP16 operand scale of one series: a power of two that puts max |x'| <= 2 max|t^|
// near 2^14 (BF16: 1).
__device__ double operand_scale(double maxabs, int bf16) {
    if (bf16) return 1.0;
    const double mx = 2.0 * maxabs;
    if (!(mx > 0.0)) return 1.0;
    int e = (int)floor(log2(16384.0 / mx));
    e = e > 24 ? 24 : (e < -24 ? -24 : e);
    return ldexp(1.0, e);
}

__device__ __forceinline__ int claim_series(int* ctr, int* sh) {
    __syncthreads();  // every thread has read the previous claim
    if (threadIdx.x == 0) *sh = atomicAdd(ctr, 1);
    __syncthreads();
    return *sh;
}

// Padding rows / positions [lo, hi) of a group: no row, no column.
__device__ void pad_rows(const BArr& A, int s, int64_t lo, int64_t hi) {
    for (int64_t p = lo + threadIdx.x; p < hi; p += kPT) {
        A.sig[p] = -1;
        A.coldat[kColPad + p] = make_float4(0.f, INFINITY, __int_as_float(kNoRow), 0.f);
        A.rser[p] = s;
        A.rmin[p] = __float_as_uint(INFINITY);
        A.r32[p] = __float_as_uint(INFINITY);
        A.flag[p] = 0;
        A.mubin[p] = 0;
        A.rowmu[p] = 0.f;
        A.rowc[p] = 0.f;
        A.rowsc[p] = 0.f;
        A.sigpos[p] = (int32_t)p;
    }
}


// ---- per series: Eq. 2, normalisation, prefix sums, Eq. 5 rows, mean order ----
// One block (kPT threads) per series, series claimed dynamically (the host lists
// a group's series longest first).  The last block to finish sets the group's
// operand scale (the smallest of its series' scales: every operand of the
// group then fits) and its largest mean-bin width.
__global__ void __launch_bounds__(kPT) k_b_prep(BArr A) {
    __shared__ int hist[kMuBins];
    __shared__ double sh1[32], sh2[32];
    __shared__ unsigned shu[32];
    __shared__ float shf[32];
    __shared__ int shi[33];
    __shared__ int s_claim;
    __shared__ double carry[2];
    const int tid = threadIdx.x;
    BGrp* G = A.G;
    for (;;) {
        const int k = claim_series(&G->prep_next, &s_claim);
        if (k >= A.ns) break;
        const int s = A.s0 + k;
        BSer& S = A.ser[s];
        const float* T = S.T;
        const int64_t m = S.m;
        const int n = S.n, N = S.N, base = S.base;
        // Eq. 2, pass 1: FP64 sum, FP32 extremes (input values: exact), finiteness
        double sum = 0.0;
        float mx = -INFINITY, mn = INFINITY;
        int bad = 0;
        for (int64_t i = tid; i < m; i += kPT) {
            const float v = T[i];
            if (!isfinite(v)) bad = 1;
            sum += (double)v;
            mx = fmaxf(mx, v);
            mn = fminf(mn, v);
        }
        bad = __syncthreads_or(bad);
        sum = bblock_sum(sum, sh1);
        const double gmx = (double)bblock_fmax(mx, shf), gmn = -(double)bblock_fmax(-mn, shf);
        const double mu = sum / (double)m;
        // pass 2: two-pass sum of squared deviations
        double q = 0.0;
        for (int64_t i = tid; i < m; i += kPT) {
            const double d = (double)T[i] - mu;
            q += d * d;
        }
        q = bblock_sum(q, sh1);
        const double sigma = sqrt(q / (double)m);
        const bool valid = !bad && sigma > 0.0;
        if (!valid) {
            // a non-finite or constant series takes no part in the waves
            if (tid == 0) {
                S.valid = 0;
                S.nonfinite = bad;
                S.degenerate = bad ? 0 : 1;
            }
            pad_rows(A, s, base, (int64_t)base + S.npad);
            if (tid == 0) A.binstart[(int64_t)s * (kMuBins + 1)] = base;
            continue;
        }
        const double inv_sigma = 1.0 / sigma;
        const double maxabs = fmax(fabs(gmx - mu), fabs(gmn - mu)) / sigma;
        const double lo = (gmn - mu) / sigma, hi = (gmx - mu) / sigma;
        const double w = (hi - lo) / (double)kMuBins;
        const double inv_w = w > 0.0 ? 1.0 / w : 0.0;
        // normalised values and FP64 exclusive prefix sums, 4 kPT values per round
        double* t64 = A.t64 + S.vbase;
        float* t32 = A.t32 + S.vbase;
        double* P1 = A.P1 + S.vbase;
        double* P2 = A.P2 + S.vbase;
        if (tid == 0) {
            P1[0] = 0.0;
            P2[0] = 0.0;
        }
        double c1 = 0.0, c2 = 0.0;
        for (int64_t t0 = 0; t0 < m; t0 += 4 * kPT) {
            double v[4];
            double s1 = 0.0, s2 = 0.0;
#pragma unroll
            for (int qq = 0; qq < 4; qq++) {
                const int64_t i = t0 + 4 * tid + qq;
                v[qq] = i < m ? ((double)T[i] - mu) * inv_sigma : 0.0;
                if (i < m) {
                    t64[i] = v[qq];
                    t32[i] = (float)v[qq];
                }
                s1 += v[qq];
                s2 += v[qq] * v[qq];
            }
            double e1 = s1, e2 = s2;
            bexscan2(e1, e2, sh1, sh2);
            double a1 = c1 + e1, a2 = c2 + e2;
#pragma unroll
            for (int qq = 0; qq < 4; qq++) {
                const int64_t i = t0 + 4 * tid + qq;
                a1 += v[qq];
                a2 += v[qq] * v[qq];
                if (i < m) {
                    P1[i + 1] = a1;
                    P2[i + 1] = a2;
                }
            }
            if (tid == kPT - 1) {
                carry[0] = a1;
                carry[1] = a2;
            }
            __syncthreads();
            c1 = carry[0];
            c2 = carry[1];
        }
        __syncthreads();  // the prefix sums are visible to the whole block
        // Eq. 5 rows, the mean bin of each row and the histogram of the bins
        for (int b = tid; b < kMuBins; b += kPT) hist[b] = 0;
        __syncthreads();
        const double sqrt_n = sqrt((double)n), inv_n = 1.0 / (double)n;
        unsigned scm = 0u, ccm = 0u, amm = 0u;
        for (int i = tid; i < N; i += kPT) {
            const double S1 = P1[i + n] - P1[i];
            const double S2 = P2[i + n] - P2[i];
            const double mui = S1 * inv_n;
            double c = S2 - S1 * mui;
            const double noise = 64.0 * 1.1102230246251565e-16 * (fabs(P2[i + n]) + fabs(P2[i]));
            if (c <= noise) c = 0.0;
            const int64_t g = (int64_t)base + i;
            A.mu_w[g] = mui;
            A.c_w[g] = c;
            const double bb = floor((mui - lo) * inv_w);
            const int bin = bb >= 0.0 ? (bb < (double)kMuBins ? (int)bb : kMuBins - 1) : 0;
            A.mubin[g] = bin;
            atomicAdd(&hist[bin], 1);
            const float rmu = (float)(mui * sqrt_n);
            const float cc = __double2float_ru(c);
            const float sc = __fsqrt_ru(cc);
            A.rowmu[g] = rmu;
            A.rowc[g] = (float)c;
            A.rowsc[g] = sc;
            A.rmin[g] = __float_as_uint(INFINITY);
            A.r32[g] = __float_as_uint(INFINITY);
            A.flag[g] = 0;
            A.rser[g] = s;
            scm = max(scm, __float_as_uint(sc));
            ccm = max(ccm, __float_as_uint(cc));
            amm = max(amm, __float_as_uint(fabsf(rmu)));
        }
        scm = bblock_umax(scm, shu);
        ccm = bblock_umax(ccm, shu);
        amm = bblock_umax(amm, shu);
        // bin starts (positions of the group), then the counting sort
        int h[4], hs = 0;
#pragma unroll
        for (int qq = 0; qq < 4; qq++) {
            h[qq] = hist[4 * tid + qq];
            hs += h[qq];
        }
        int total;
        int start = bexscan_i(hs, shi, &total);
        int32_t* bst = A.binstart + (int64_t)s * (kMuBins + 1);
        __syncthreads();
#pragma unroll
        for (int qq = 0; qq < 4; qq++) {
            bst[4 * tid + qq] = base + start;
            hist[4 * tid + qq] = base + start;  // cursor
            start += h[qq];
        }
        if (tid == 0) bst[kMuBins] = base + N;
        __syncthreads();
        for (int i = tid; i < N; i += kPT) {
            const int64_t g = (int64_t)base + i;
            const int p = atomicAdd(&hist[A.mubin[g]], 1);
            A.sig[p] = (int32_t)g;
            A.sigpos[g] = p;
            A.coldat[kColPad + p] = make_float4(A.rowmu[g], A.rowc[g], __int_as_float((int)g), 0.f);
        }
        pad_rows(A, s, (int64_t)base + N, (int64_t)base + S.npad);
        if (tid == 0) {
            S.valid = 1;
            S.nonfinite = 0;
            S.degenerate = 0;
            S.mu = mu;
            S.sigma = sigma;
            S.maxabs = maxabs;
            S.lo = lo;
            S.w = w;
            S.inv_w = inv_w;
            S.P2end = P2[m];
            S.scale = operand_scale(maxabs, A.bf16);
            S.scmax = scm;
            S.cmax = ccm;
            S.mumax = amm;
        }
    }
    // the last block: group operand scale and largest bin width
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(&G->prep_ticket, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last || tid != 0) return;
    __threadfence();
    double sc = 0.0, wmax = 0.0, amax = 0.0;
    for (int k = 0; k < A.ns; k++) {
        const volatile BSer& S = A.ser[A.s0 + k];
        if (!S.valid) continue;
        sc = sc == 0.0 ? S.scale : fmin(sc, S.scale);
        wmax = fmax(wmax, S.w);
        amax = fmax(amax, S.maxabs);
    }
    G->gstats[2] = amax;  // largest max |t^| (the FP32 error bounds of the settle wave)
    G->gstats[3] = sc > 0.0 ? sc : 1.0;
    G->gstats[7] = wmax;
}


// ---- operand matrix and per-row bound terms -----------------------------------
// Block b of the group builds rows [64 k, 64 k + 64) of the series whose blocks
// [rb0, rb1) hold b: the centred rows s (t^_{i+k} - mu_i) at their mean-order
// positions (FP32 centring, one rounding to 16 bits, zero for k >= n), the
// bound terms F_i of those rows (the single-series form: operand rounding, FP32
// accumulation, subnormal operands, FP32 epilogue, safety factor 2, with the
// series' own maxima and the group's operand scale s), and zero rows at the
// padding positions among [base + 64 k, base + 64 k + 64).
__device__ __forceinline__ uint32_t bpack16(float y0, float y1, __half*) {
    const __half2 h = __floats2half2_rn(y0, y1);
    return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t bpack16(float y0, float y1, __nv_bfloat16*) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(y0, y1);
    return *reinterpret_cast<const uint32_t*>(&h);
}

template <typename T16>
__global__ void __launch_bounds__(256) k_b_build(BArr A, int nblocks) {
    constexpr int TKA = kTcAtom;
    constexpr int kSeg = kBRows + kBChunks * TKA;
    __shared__ __align__(16) float seg[kSeg + 1];
    __shared__ float smu[kBRows];
    __shared__ int spos[kBRows];
    __shared__ int s_ser;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int kpad = A.kpad;
    const int64_t P = A.P;
    const float s = (float)A.G->gstats[3];
    T16* Sm = reinterpret_cast<T16*>(A.S16);
    for (int b = blockIdx.x; b < nblocks; b += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int lo = A.s0, hi = A.s0 + A.ns - 1;  // the series with rb0 <= b < rb1
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (A.ser[mid].rb0 <= b) lo = mid; else hi = mid - 1;
            }
            s_ser = lo;
        }
        __syncthreads();
        const BSer& S = A.ser[s_ser];
        const int n = S.n;
        const int N = S.valid ? S.N : 0;
        const int base = S.base;
        const int64_t m = S.m;
        const int i0 = (b - S.rb0) * kBRows;
        if (threadIdx.x < kBRows) {
            const int i = i0 + threadIdx.x;
            const int64_t g = (int64_t)base + i;
            smu[threadIdx.x] = i < N ? (float)A.mu_w[g] : 0.f;
            spos[threadIdx.x] = i < N ? A.sigpos[g] : -1;
            float al = 0.f, ga = 0.f, qq = 0.f;
            if (i < N) {
                // per-row bound terms (see k_tc_rowbound in tc_prep.cu for the derivation)
                const float u32 = 5.9604644775390625e-08f;
                const float uacc = 2.384185791015625e-07f;
                const float nf = (float)n;
                const float sqrt_n = sqrtf(nf);
                const float scmax = __uint_as_float(S.scmax), cmax = __uint_as_float(S.cmax);
                const float mumax = __uint_as_float(S.mumax);
                const float maxabs = (float)S.maxabs;
                const float u_in = A.bf16 ? 0.00390625f : 0.00048828125f;
                const float gn = nf * uacc / (1.f - nf * uacc);
                const float uo = u_in + 2.f * u32;
                const float Kg = 2.f * ((2.f * uo + uo * uo) + gn * (1.f + uo) * (1.f + uo));
                const float sci = A.rowsc[g];
                const float Q = sci * scmax;
                const float ci = A.rowc[g];
                const float ea = 2.01f * u32 * maxabs + 2.9802322387695312e-08f / s;
                const float eta = 2.f * (ea * sqrt_n * (sci + scmax) + nf * ea * ea);
                const float ec = 512.f * 1.1102230246251565e-16f * (1.f + (float)S.P2end);
                const float A0 = Kg * Q + eta + 4.f * u32 * (ci + cmax) + 2.f * ec + 8.f * u32 * Q;
                const float G0 = 2.f * u32 * (fabsf(A.rowmu[g]) + mumax);
                al = 2.002f * A0;
                ga = 2.002f * G0;
                qq = 2.002f * Q;
            }
            if (i < S.npad) {
                A.alpha[g] = al;
                A.gam[g] = ga;
                A.q2[g] = qq;
            }
        }
        // zero operand rows at the padding positions of this block's range
        {
            const int per = kpad / 8;  // uint4 per row
            const int p_lo = max(i0, N), p_hi = min(i0 + kBRows, S.npad);
            uint4* Sv = reinterpret_cast<uint4*>(A.S16);
            for (int t = threadIdx.x; t < (p_hi - p_lo) * per; t += blockDim.x) {
                const int64_t p = (int64_t)base + p_lo + t / per;
                const int c = t % per;
                Sv[((int64_t)(c >> 3) * P + p) * 8 + (c & 7)] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        if (i0 >= N) continue;
        const float* t32 = A.t32 + S.vbase;
        const unsigned long long s2 = [&] {
            unsigned long long r;
            asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(s));
            return r;
        }();
        for (int k0 = 0; k0 < kpad; k0 += kBChunks * TKA) {
            const int nch = min(kpad - k0, kBChunks * TKA) / TKA;
            __syncthreads();
            for (int x = threadIdx.x; x < kBRows + nch * TKA + 1; x += blockDim.x) {
                const int64_t gi = (int64_t)i0 + k0 + x;
                seg[x] = gi < m ? t32[gi] : 0.f;
            }
            __syncthreads();
            for (int r = wid; r < kBRows; r += nwarp) {
                const int p = spos[r];
                if (p < 0) break;
                const float mu = smu[r];
                unsigned long long mu2;
                asm("mov.b64 %0, {%1, %1};" : "=l"(mu2) : "f"(mu));
                T16* dst = Sm + ((int64_t)(k0 / TKA) * P + p) * TKA + 2 * lane;
                for (int c = 0; c < nch; c++, dst += P * TKA) {
                    const int k = k0 + c * TKA + 2 * lane;
                    float2 x = make_float2(seg[r + c * TKA + 2 * lane], seg[r + c * TKA + 2 * lane + 1]);
                    unsigned long long v;
                    asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(x.x), "f"(x.y));
                    asm("sub.rn.f32x2 %0, %0, %1;" : "+l"(v) : "l"(mu2));
                    asm("mul.rn.f32x2 %0, %0, %1;" : "+l"(v) : "l"(s2));
                    asm("mov.b64 {%0, %1}, %2;" : "=f"(x.x), "=f"(x.y) : "l"(v));
                    *reinterpret_cast<uint32_t*>(dst) =
                        bpack16(k < n ? x.x : 0.f, k + 1 < n ? x.y : 0.f, (T16*)nullptr);
                }
            }
        }
    }
}


// Upper bound of row g from its running minimum (Gram form: D + F_g(D)).
__device__ __forceinline__ float b_ub(const BArr& A, int64_t g) {
    const float D = __uint_as_float(A.rmin[g]);
    return D + (A.alpha[g] + kTcBeta * D + A.gam[g] * sqrtf(fmaxf(D, 0.f) + A.q2[g]));
}
// Lower bound of the true nn^2 of a row whose scan completed: D - F(D) - gam^2.
__device__ __forceinline__ float b_lb(const BArr& A, int64_t g) {
    const float D = __uint_as_float(A.rmin[g]);
    const float ga = A.gam[g];
    const float v = D - (A.alpha[g] + kTcBeta * D + ga * sqrtf(fmaxf(D, 0.f) + A.q2[g])) - ga * ga;
    return v > 0.f ? v : 0.f;
}

// Column segments of a row tile of series S around position C: alternately
// right and left of C, nearest first (mode 2 of the tensor-core kernel).
__device__ __forceinline__ int4 b_range(const BSer& S, int C, int seg) {
    const int L = S.base, H = S.base + S.N;
    C = C < L ? L : (C > H ? H : C);
    const int right = (H - C + seg - 1) / seg, left = (C - L + seg - 1) / seg;
    return make_int4(L, H, C, 2 * (right > left ? right : left));
}

// Largest bin b (of `bins`) with sum_{b' >= b} hist[b'] >= need, and that
// suffix sum without bin b; one warp.
__device__ void b_select_bin(const int* hist, int bins, int need, int* out_bin, int* out_above) {
    const int lane = threadIdx.x & 31;
    const int per = bins / 32;
    int cnt = 0;
    for (int b = lane * per; b < (lane + 1) * per; b++) cnt += hist[b];
    // suffix sums over the lanes: lanes hold consecutive bin ranges
    int suf = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_down_sync(0xffffffffu, suf, o);
        if (lane + o < 32) suf += u;
    }
    const int above_lane = suf - cnt;  // rows in the lanes above this one
    const unsigned hit = __ballot_sync(0xffffffffu, above_lane < need && suf >= need);
    const int L = hit ? 31 - __clz(hit) : 0;
    if (lane == L) {
        int above = above_lane, b = (lane + 1) * per - 1;
        for (; b > lane * per; b--) {
            if (above + hist[b] >= need) break;
            above += hist[b];
        }
        *out_bin = b;
        *out_above = above;
    }
}

// ---- per series: the rows with the largest finite upper bounds (one tile) -------
// Rows the band left without a finite bound are not ranked (their full scans
// could not be pruned).  Two 12-bit radix passes over the bound's float bits
// find the threshold; ties at the last level are taken in any order.
__global__ void __launch_bounds__(kPT) k_b_top(BArr A) {
    __shared__ int hist[kMuBins];
    __shared__ int s_claim, s_b1, s_a1, s_b2, s_a2, s_cnt, s_tie;
    __shared__ int shi[33];
    const int tid = threadIdx.x;
    BGrp* G = A.G;
    for (;;) {
        const int k = claim_series(&G->top_next, &s_claim);
        if (k >= A.ns) break;
        const int s = A.s0 + k;
        const BSer& S = A.ser[s];
        int32_t* out = A.list_top + (int64_t)k * kBTop;
        if (!S.valid) {
            if (tid < kBTop) out[tid] = -1;
            if (tid == 0) A.ranges_top[k] = make_int4(S.base, S.base, S.base, 0);
            continue;
        }
        const int base = S.base, N = S.N;
        for (int b = tid; b < kMuBins; b += kPT) hist[b] = 0;
        if (tid == 0) {
            s_cnt = 0;
            s_tie = 0;
        }
        __syncthreads();
        int nfin = 0;
        for (int i = tid; i < N; i += kPT) {
            const float u = b_ub(A, (int64_t)base + i);
            if (u < INFINITY) {  // NaN and +inf are not ranked
                atomicAdd(&hist[(__float_as_uint(u) & 0x7fffffffu) >> 19], 1);
                nfin++;
            }
        }
        nfin = bblock_isum(nfin, shi);
        const bool all = nfin <= kBTop;
        if (!all) {
            if (tid < 32) b_select_bin(hist, kMuBins, kBTop, &s_b1, &s_a1);
            __syncthreads();
            const int b1 = s_b1, need = kBTop - s_a1;
            for (int b = tid; b < kMuBins; b += kPT) hist[b] = 0;
            __syncthreads();
            for (int i = tid; i < N; i += kPT) {
                const float u = b_ub(A, (int64_t)base + i);
                const unsigned ub = __float_as_uint(u) & 0x7fffffffu;
                if (u < INFINITY && (int)(ub >> 19) == b1) atomicAdd(&hist[(ub >> 7) & 0xfff], 1);
            }
            __syncthreads();
            if (tid < 32) b_select_bin(hist, kMuBins, need, &s_b2, &s_a2);
            __syncthreads();
        }
        const int b1 = all ? -1 : s_b1, b2 = all ? -1 : s_b2;
        const int need2 = all ? 0 : kBTop - s_a1 - s_a2;
        for (int i = tid; i < N; i += kPT) {
            const int64_t g = (int64_t)base + i;
            const float u = b_ub(A, g);
            if (!(u < INFINITY)) continue;
            const unsigned ub = __float_as_uint(u) & 0x7fffffffu;
            const int c1 = (int)(ub >> 19), c2 = (int)((ub >> 7) & 0xfff);
            bool take = all || c1 > b1 || (c1 == b1 && c2 > b2);
            if (!take && c1 == b1 && c2 == b2) take = atomicAdd(&s_tie, 1) < need2;
            if (take) {
                const int slot = atomicAdd(&s_cnt, 1);
                if (slot < kBTop) {
                    out[slot] = (int32_t)g;
                    A.flag[g] = 1;
                }
            }
        }
        __syncthreads();
        const int cnt = min(s_cnt, kBTop);
        for (int j = cnt + tid; j < kBTop; j += kPT) out[j] = -1;
        if (tid == 0) {
            const int4 r = cnt > 0 ? b_range(S, base + N / 2, A.seg_cols) : make_int4(base, base, base, 0);
            A.ranges_top[k] = r;
            if (r.w > 0) atomicMax(&G->ctrl.smax[0], r.w);
        }
    }
}


// ---- per series: best-so-far from the top rows, survivors into whole tiles -------
// The top rows completed full scans, so bsf_s = max of their lower bounds is a
// lower bound of s's discord distance.  Every other row whose upper bound
// reaches bsf_s survives; they are written in mean order into ceil(cnt / 128)
// tiles of their own (entries past cnt are -1), whose place in the list is
// taken with one atomic per series.
__global__ void __launch_bounds__(kPT) k_b_surv(BArr A) {
    __shared__ int s_claim, s_t0;
    __shared__ int shi[33];
    __shared__ unsigned shu[32];
    const int tid = threadIdx.x, lane = tid & 31;
    BGrp* G = A.G;
    for (;;) {
        const int k = claim_series(&G->surv_next, &s_claim);
        if (k >= A.ns) break;
        const int s = A.s0 + k;
        const BSer& S = A.ser[s];
        if (!S.valid) {
            if (tid == 0) A.sbsf[s] = 0u;
            continue;
        }
        const int base = S.base, N = S.N;
        unsigned lbm = 0u;
        if (tid < kBTop) {
            const int g = A.list_top[(int64_t)k * kBTop + tid];
            if (g >= 0) lbm = __float_as_uint(b_lb(A, g));
        }
        lbm = bblock_umax(lbm, shu);
        const float bsf = __uint_as_float(lbm);
        // count, then write in mean order (one round of kPT positions at a time)
        int cnt = 0;
        for (int p = tid; p < N; p += kPT) {
            const int g = A.sig[base + p];
            cnt += (g >= 0 && A.flag[g] == 0 && !(b_ub(A, g) < bsf)) ? 1 : 0;
        }
        cnt = bblock_isum(cnt, shi);
        const int ntile = (cnt + kBTop - 1) / kBTop;
        if (tid == 0) {
            A.sbsf[s] = lbm;
            s_t0 = ntile > 0 ? atomicAdd(&G->rest_tiles, ntile) : 0;
            if (ntile > 0) atomicAdd(&G->rest_rows, ntile * kBTop);
        }
        __syncthreads();
        if (ntile == 0) continue;
        const int t0 = s_t0;
        int32_t* out = A.list_rest + (int64_t)t0 * kBTop;
        int run = 0;
        for (int p0 = 0; p0 < N; p0 += kPT) {
            const int p = p0 + tid;
            int g = -1;
            bool alive = false;
            if (p < N) {
                g = A.sig[base + p];
                alive = g >= 0 && A.flag[g] == 0 && !(b_ub(A, g) < bsf);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, alive);
            int total;
            const int wofs = bexscan_i(lane == 0 ? __popc(bal) : 0, shi, &total);
            const int wbase = __shfl_sync(0xffffffffu, wofs, 0);
            if (alive) {
                out[run + wbase + __popc(bal & ((1u << lane) - 1u))] = g;
                A.flag[g] = 2;
            }
            run += total;
        }
        for (int j = cnt + tid; j < ntile * kBTop; j += kPT) out[j] = -1;
        __syncthreads();
        for (int t = tid; t < ntile; t += kPT) {
            const int first = out[(int64_t)t * kBTop];
            const int last = out[(int64_t)t * kBTop + min(kBTop, cnt - t * kBTop) - 1];
            const int C = (A.sigpos[first] + A.sigpos[last]) / 2;
            const int4 r = b_range(S, C, A.seg_cols);
            A.ranges_rest[t0 + t] = r;
            A.tser_rest[t0 + t] = s;
            atomicMax(&G->ctrl.smax[1], r.w);
        }
    }
}

// ---- per series: final best-so-far, candidates and their FP64 column ranges -------
// A candidate i's nearest neighbour j* has n (mu_i - mu_j*)^2 <= d^2 <= ub_i, so
// its exact scan only needs the positions of the mean bins within sqrt(ub_i / n)
// of mu_i.
__device__ void b_lb_range(const BArr& A, const BSer& S, int s, int64_t g, float ub, int& L, int& H) {
    L = S.base;
    H = S.base + S.N;
    const double w = S.w;
    if (!(ub < 1e30f) || !(w > 0.0)) return;
    const double h = sqrt((double)ub / (double)S.n) * (1.0 + 1e-4) + 1e-12;
    const double kb = ceil(h / w) + 1.0;
    const int kk = kb < (double)kMuBins ? (int)kb : kMuBins;
    const int b = A.mubin[g];
    const int32_t* bst = A.binstart + (int64_t)s * (kMuBins + 1);
    L = bst[b - kk < 0 ? 0 : b - kk];
    H = bst[b + kk + 1 > kMuBins ? kMuBins : b + kk + 1];
}

// Adds row g to the FP64 rescoring list: one atomic gives its slot and its
// first column chunk, so chunk bases ascend with slots.
__device__ void b_add_cand(const BArr& A, int64_t g, int L, int H) {
    const int nc = (H - L + kRChunk - 1) / kRChunk;
    const unsigned long long old = atomicAdd(&A.G->cand_packed, (1ull << 40) | (unsigned long long)nc);
    const int slot = (int)(old >> 40);
    A.cand[slot] = (int32_t)g;
    A.rL[slot] = L;
    A.rH[slot] = H;
    A.cbase[slot] = (int64_t)(old & ((1ull << 40) - 1));
    A.ex64[slot] = 0x7ff0000000000000ull;
}

// Rigorous FP32 error bound of a direct FP32 distance e (the FP32 tile kernel's).
__device__ __forceinline__ float b_margin32(float e, float n, float M) {
    const float u = 5.9604644775390625e-08f;
    const float gn = n * u / (1.f - n * u);
    const float mu6 = 6.f * u * M;
    return 2.f * ((gn + 4.f * u) * e + 8.f * u * M * sqrtf(n * e) + n * mu6 * mu6) + 1e-30f;
}

// A survivor whose upper bound still reaches bsf_s was never abandoned (bounds
// only fall and bsf_s was fixed during the wave), so its scan completed and its
// lower bound counts; bsf_s is raised to the largest.  The candidates are the
// top rows and survivors whose upper bound reaches the raised bsf_s.  Up to
// settle_min of them go to the FP64 rescoring at once; more (rows whose Gram
// bounds overlap, e.g. the windows around an anomaly of a noisy periodic
// series) are first settled by direct FP32 full scans, whose tiles of
// settle_rows rows share every staged column among their rows (a few rows
// already outrun the column-by-column FP32 screen of the rescoring): they are
// written in mean order into whole tiles of the settle list, each tile's
// column range the union of its rows' lower-bound ranges.
__global__ void __launch_bounds__(kPT) k_b_cands(BArr A) {
    __shared__ int s_claim, s_t0;
    __shared__ unsigned shu[32];
    __shared__ int shi[33];
    const int tid = threadIdx.x, lane = tid & 31;
    BGrp* G = A.G;
    for (;;) {
        const int k = claim_series(&G->cand_next, &s_claim);
        if (k >= A.ns) break;
        const int s = A.s0 + k;
        BSer& S = A.ser[s];
        if (!S.valid) continue;
        const int base = S.base, N = S.N;
        const float bsf0 = __uint_as_float(A.sbsf[s]);
        unsigned lbm = A.sbsf[s];
        for (int i = tid; i < N; i += kPT) {
            const int64_t g = (int64_t)base + i;
            if (A.flag[g] == 2 && !(b_ub(A, g) < bsf0)) lbm = max(lbm, __float_as_uint(b_lb(A, g)));
        }
        lbm = bblock_umax(lbm, shu);
        const float bsf = __uint_as_float(lbm);
        int cnt = 0;
        for (int i = tid; i < N; i += kPT) {
            const int64_t g = (int64_t)base + i;
            cnt += (A.flag[g] != 0 && !(b_ub(A, g) < bsf)) ? 1 : 0;
        }
        cnt = bblock_isum(cnt, shi);
        if (tid == 0) {
            S.ncand = cnt;
            A.sbsf[s] = lbm;
        }
        if (cnt <= A.settle_min) {
            for (int i = tid; i < N; i += kPT) {
                const int64_t g = (int64_t)base + i;
                if (A.flag[g] == 0) continue;
                const float ub = b_ub(A, g);
                if (ub < bsf) continue;
                int L, H;
                b_lb_range(A, S, s, g, ub, L, H);
                b_add_cand(A, g, L, H);
            }
            continue;
        }
        const int TR = A.settle_rows;  // rows per settle tile
        const int ntile = (cnt + TR - 1) / TR;
        if (tid == 0) {
            s_t0 = atomicAdd(&G->settle_tiles, ntile);
            atomicAdd(&G->settle_rows, ntile * TR);
        }
        __syncthreads();
        const int t0 = s_t0;
        int32_t* out = A.list_settle + (int64_t)t0 * TR;
        int run = 0;
        for (int p0 = 0; p0 < N; p0 += kPT) {
            const int p = p0 + tid;
            int g = -1;
            bool alive = false;
            if (p < N) {
                g = A.sig[base + p];
                alive = g >= 0 && A.flag[g] != 0 && !(b_ub(A, g) < bsf);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, alive);
            int total;
            const int wofs = bexscan_i(lane == 0 ? __popc(bal) : 0, shi, &total);
            const int wbase = __shfl_sync(0xffffffffu, wofs, 0);
            if (alive) {
                out[run + wbase + __popc(bal & ((1u << lane) - 1u))] = g;
                A.flag[g] = 3;
            }
            run += total;
        }
        for (int j = cnt + tid; j < ntile * TR; j += kPT) out[j] = -1;
        __syncthreads();
        for (int t = tid; t < ntile; t += kPT) {
            int L = base + N, H = base;
            const int rows = min(TR, cnt - t * TR);
            for (int r = 0; r < rows; r++) {
                const int g = out[(int64_t)t * TR + r];
                int l, h;
                b_lb_range(A, S, s, g, b_ub(A, g), l, h);
                L = min(L, l);
                H = max(H, h);
            }
            const int C = (L + H) / 2;
            const int right = (H - C + A.seg_cols - 1) / A.seg_cols, left = (C - L + A.seg_cols - 1) / A.seg_cols;
            const int4 r = make_int4(L, H, C, 2 * (right > left ? right : left));
            A.ranges_settle[t0 + t] = r;
            A.tser_settle[t0 + t] = s;
            atomicMax(&G->ctrl.smax[2], r.w);
        }
    }
}

// After the FP32 settle wave (abandoned against bsf_s, fixed during the wave): a
// settled row whose upper bound min(D + F(D), r32) still reaches bsf_s was never
// abandoned, so it scanned every column its lower bound admits, its FP32 upper
// bound r32 came from its nearest column and r32 - 2 margin(r32) is a rigorous
// lower bound of its nn^2.  bsf_s is raised with them; the settled rows whose
// upper bound still reaches it go to the FP64 rescoring.
__global__ void __launch_bounds__(kPT) k_b_cands2(BArr A) {
    __shared__ int s_claim;
    __shared__ unsigned shu[32];
    __shared__ int shi[33];
    const int tid = threadIdx.x;
    BGrp* G = A.G;
    const float M = (float)G->gstats[2];
    for (;;) {
        const int k = claim_series(&G->cand2_next, &s_claim);
        if (k >= A.ns) break;
        const int s = A.s0 + k;
        BSer& S = A.ser[s];
        if (!S.valid || S.ncand <= A.settle_min) continue;
        const int base = S.base, N = S.N;
        const float nf = (float)S.n;
        const float bsf0 = __uint_as_float(A.sbsf[s]);
        unsigned lbm = A.sbsf[s];
        for (int i = tid; i < N; i += kPT) {
            const int64_t g = (int64_t)base + i;
            if (A.flag[g] != 3) continue;
            const float up = __uint_as_float(A.r32[g]);
            // a row abandoned during the settle wave (upper bound below bsf_s) did not finish
            if (!(up < 1e30f) || fminf(b_ub(A, g), up) < bsf0) continue;
            const float lb = up - 2.f * b_margin32(up, nf, M);
            if (lb > 0.f) lbm = max(lbm, __float_as_uint(lb));
        }
        lbm = bblock_umax(lbm, shu);
        const float bsf = __uint_as_float(lbm);
        int cnt = 0;
        for (int i = tid; i < N; i += kPT) {
            const int64_t g = (int64_t)base + i;
            if (A.flag[g] != 3) continue;
            const float ub = fminf(b_ub(A, g), __uint_as_float(A.r32[g]));
            if (ub < bsf) continue;
            int L, H;
            b_lb_range(A, S, s, g, ub, L, H);
            b_add_cand(A, g, L, H);
            cnt++;
        }
        cnt = bblock_isum(cnt, shi);
        if (tid == 0) {
            S.ncand = cnt;
            A.sbsf[s] = lbm;
        }
    }
}

// ---- exact FP64 nearest-neighbour distances of the candidates ------------------
// Work items (candidate, 64-column chunk of its range), claimed dynamically; each
// column is screened in FP32 first (direct differences on the FP32 copy of t^,
// with a proven error bound), and only columns that could still reach the
// candidate's upper bound are evaluated in FP64 (Eq. 1 squared on t^).
__global__ void __launch_bounds__(256) k_b_rescore(BArr A) {
    __shared__ int sh_item;
    __shared__ double red[8];
    BGrp* G = A.G;
    const float u32 = 5.9604644775390625e-08f;
    const unsigned long long pk = G->cand_packed;
    const int cnt = (int)(pk >> 40);
    const long long items = (long long)(pk & ((1ull << 40) - 1));  // chunks of all candidates
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    if (items > 0x7fffffffll) {  // the 32-bit work counter would wrap
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&G->ctrl.err, DD_ENOTSUP);
        return;
    }
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) sh_item = atomicAdd(&G->ctrl.work[3], 1);
        __syncthreads();
        const int item = sh_item;
        if (item < 0 || item >= items) {
            if (item < 0 && threadIdx.x == 0) atomicExch(&G->ctrl.err, DD_ENOTSUP);
            break;
        }
        // the candidate whose chunk range holds the item (bases ascend with slots)
        int lo = 0, hi = cnt - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (A.cbase[mid] <= item)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int r = lo;
        const int c = (int)(item - A.cbase[r]);
        const int g = A.cand[r];
        const BSer& S = A.ser[A.rser[g]];
        const int a0 = A.rL[r] + c * kRChunk, H = A.rH[r];
        if (a0 >= H) continue;
        const int a1 = min(H, a0 + kRChunk);
        const int n = S.n;
        const int i = g - S.base;
        const double* x = A.t64 + S.vbase + i;
        const float* x32 = A.t32 + S.vbase + i;
        const float ub = fminf(b_ub(A, g), __uint_as_float(A.r32[g]));
        const float nf = (float)n;
        const float gn32 = nf * u32 / (1.f - nf * u32);
        const float maxabs = (float)S.maxabs;
        double best = INFINITY;
        for (int p = a0 + wid; p < a1; p += nwarp) {
            const int j = A.sig[p] - S.base;
            const int d = i - j;
            if (d < n && d > -n) continue;
            const float* y32 = A.t32 + S.vbase + j;
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
            const double* y = A.t64 + S.vbase + j;
            double sd = 0.0;
            for (int k = lane; k < n; k += 32) {
                const double df = x[k] - y[k];
                sd = fma(df, df, sd);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
            best = fmin(best, sd);
        }
        if (lane == 0) red[wid] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = red[0];
            for (int w = 1; w < nwarp; w++) b = fmin(b, red[w]);
            if (b < INFINITY) atomicMin(A.ex64 + r, (unsigned long long)__double_as_longlong(b));
        }
    }
}

// ---- per series: the discord and its result ---------------------------------------
// Every block joins the per-series maxima of the exact values; the last block
// to finish picks, per series, the smallest index attaining the maximum and
// writes every result of the group.
__global__ void __launch_bounds__(256) k_b_best(BArr A) {
    __shared__ bool last;
    BGrp* G = A.G;
    const int cnt = (int)(G->cand_packed >> 40);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < cnt; r += gridDim.x * blockDim.x) {
        const int g = A.cand[r];
        atomicMax(&A.ser[A.rser[g]].best64, A.ex64[r]);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&G->best_ticket, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
        const int g = A.cand[r];
        BSer& S = A.ser[A.rser[g]];
        if (A.ex64[r] == *(volatile unsigned long long*)&S.best64) atomicMin(&S.best_idx, g - S.base);
    }
    __threadfence();
    __syncthreads();
    const int err = *(volatile int*)&G->ctrl.err;
    for (int k = threadIdx.x; k < A.ns; k += blockDim.x) {
        const volatile BSer& S = A.ser[A.s0 + k];
        dd_result_t res;
        res.exact = 1;
        res.computed_pairs = 0;
        res.candidates = S.ncand;
        res.index = -1;
        res.nn_distance = 0.0;
        if (S.nonfinite) {
            res.status = DD_ENONFINITE;
        } else if (S.degenerate) {
            // sigma == 0: every distance is 0 and the first subsequence wins the tie
            res.status = DD_OK;
            res.index = 0;
        } else if (err) {
            res.status = err;
        } else if (S.best_idx == 0x7fffffff || S.best64 == 0x7ff0000000000000ull) {
            res.status = DD_ECUDA;
        } else {
            res.status = DD_OK;
            res.index = S.best_idx;
            res.nn_distance = sqrt(__longlong_as_double((long long)S.best64));
        }
        A.res[S.slot] = res;
    }
}

// Per group, before its first launch: the list counts the waves read, and the
// column constants of the kColPad entries on each side of the group (no column).
__global__ void k_b_init(BArr A) {
    if (threadIdx.x == 0) {
        A.G->band_rows = (int)A.P;
        A.G->top_rows = A.ns * kBTop;
    }
    for (int t = threadIdx.x; t < 2 * kColPad; t += blockDim.x) {
        const int64_t ix = t < kColPad ? t : A.P + t;  // [0, pad) and [pad + P, 2 pad + P)
        A.coldat[ix] = make_float4(0.f, INFINITY, __int_as_float(kNoRow), 0.f);
    }
}


constexpr size_t kBAlign = 256;
constexpr int kMaxGroups = 64;  // distinct subsequence lengths in one call

struct BCarver {
    char* base;
    size_t off = 0;
    template <class T>
    T* take(size_t count) {
        off = (off + kBAlign - 1) / kBAlign * kBAlign;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

int kpad_of(int n) { return (n + kTcAtom - 1) / kTcAtom * kTcAtom; }
// rows of a series with m values: its values, rounded up to whole tiles, and 256 padding
// rows (>= N + 256 rows, and room for the m + 1 prefix sums at the same offsets)
int64_t npad_of(int64_t m) { return (m + 127) / 128 * 128 + kPadRows; }

// Carves one group's arrays (base == null: measures).  S16 / A16 come last.
void carve_group(BCarver& c, BArr& A, void** A16, int64_t P, int ns, int kpad) {
    A.G = c.take<BGrp>(1);
    A.P = P;
    A.kpad = kpad;
    A.coldat = c.take<float4>((size_t)P + 2 * kColPad);
    A.t32 = c.take<float>((size_t)P + 64);
    A.t64 = c.take<double>((size_t)P + 64);
    A.P1 = c.take<double>((size_t)P + 64);
    A.P2 = c.take<double>((size_t)P + 64);
    A.r32 = c.take<uint32_t>((size_t)P);
    A.list_settle = c.take<int32_t>((size_t)P);
    A.ranges_settle = c.take<int4>((size_t)P / 32 + 1);
    A.tser_settle = c.take<int32_t>((size_t)P / 32 + 1);
    A.mu_w = c.take<double>((size_t)P);
    A.c_w = c.take<double>((size_t)P);
    A.ex64 = c.take<unsigned long long>((size_t)P);
    A.mubin = c.take<int32_t>((size_t)P);
    A.sig = c.take<int32_t>((size_t)P);
    A.sigpos = c.take<int32_t>((size_t)P);
    A.rser = c.take<int32_t>((size_t)P);
    A.rmin = c.take<uint32_t>((size_t)P);
    A.rowmu = c.take<float>((size_t)P);
    A.rowc = c.take<float>((size_t)P);
    A.rowsc = c.take<float>((size_t)P);
    A.alpha = c.take<float>((size_t)P);
    A.gam = c.take<float>((size_t)P);
    A.q2 = c.take<float>((size_t)P);
    A.flag = c.take<uint8_t>((size_t)P);
    A.list_top = c.take<int32_t>((size_t)ns * kBTop);
    A.list_rest = c.take<int32_t>((size_t)P);
    A.ranges_top = c.take<int4>((size_t)ns + 1);
    A.ranges_rest = c.take<int4>((size_t)P / 128 + 1);
    A.tser_rest = c.take<int32_t>((size_t)P / 128 + 1);
    A.cand = c.take<int32_t>((size_t)P);
    A.rL = c.take<int32_t>((size_t)P);
    A.rH = c.take<int32_t>((size_t)P);
    A.cbase = c.take<int64_t>((size_t)P);
    A.S16 = c.take<uint16_t>((size_t)P * kpad);
    *A16 = c.take<uint16_t>((size_t)P * kpad);
}

struct BWide {
    BSer* ser;
    dd_result_t* res;
    uint32_t* sbsf;
    int32_t* binstart;
};

void carve_wide(BCarver& c, BWide& W, int max_series) {
    W.ser = c.take<BSer>((size_t)max_series);
    W.res = c.take<dd_result_t>((size_t)max_series);
    W.sbsf = c.take<uint32_t>((size_t)max_series);
    W.binstart = c.take<int32_t>((size_t)max_series * (kMuBins + 1));
}

int64_t rcap_of(int max_series, int64_t max_values) { return max_values + (128 + kPadRows) * (int64_t)max_series; }

size_t batch_bytes(int max_series, int64_t max_values, int n_max) {
    BCarver c{nullptr};
    BWide W{};
    carve_wide(c, W, max_series);
    // the largest group, then the fixed part of every further group
    BArr A{};
    void* a16 = nullptr;
    carve_group(c, A, &a16, rcap_of(max_series, max_values), max_series, kpad_of(n_max));
    const int extra = (max_series < kMaxGroups ? max_series : kMaxGroups) - 1;
    for (int k = 0; k < extra; k++) carve_group(c, A, &a16, 0, 1, kTcAtom);
    return (c.off + kBAlign - 1) / kBAlign * kBAlign + kBAlign * 64;
}

}  // namespace
}  // namespace dd

// ------------------------------------------------------------------ the batch object
struct dd_batch_s {
    int max_series = 0;
    int64_t max_values = 0;
    int32_t n_max = 0;
    dd_options_t opt{};
    dd_batch_config_t cfg{};
    int device = 0, sm_count = 0;
    void* arena = nullptr;
    size_t arena_bytes = 0;
    dd::BWide W{};
    size_t wide_end = 0;
    dd::BSer* ser_host = nullptr;       // pinned staging of the series descriptors
    dd_result_t* res_host = nullptr;    // pinned results
    cudaStream_t cs = nullptr;          // capture stream
    std::vector<cudaStream_t> gs;       // one per group: the groups' launch chains run side by side
    std::vector<cudaEvent_t> gev;       // fork / join events of the group streams
    cudaGraphExec_t gexec = nullptr;    // graph of the last layout
    std::vector<int64_t> gkey;          // its layout: (m, n) of every series, in call order
    std::vector<dd_plan_s*> gplans;     // per group: the tensor maps and operand pointers
    std::vector<dd::BArr> garr;
    std::vector<int> slot_grouped;      // grouped position -> caller's slot
    std::vector<std::pair<int32_t, dd_batch_config_t>> sched;  // per-n schedules (dd_batch_set_schedule)
    std::atomic<int> busy{0};
    int64_t calls = 0, replays = 0;
};

namespace {

// The schedule of the group of subsequence length n.
const dd_batch_config_t& schedule_of(const dd_batch_s* b, int32_t n) {
    for (const auto& e : b->sched)
        if (e.first == n) return e.second;
    return b->cfg;
}

bool valid_config(const dd_batch_config_t& c) {
    if (c.seg_cols < 256 || c.seg_cols > (1 << 16) || c.seg_cols % 256 != 0) return false;
    if (c.settle_min < 0) return false;
    if (c.settle_rows != 32 && c.settle_rows != 64 && c.settle_rows != 128) return false;
    if (c.reserved[0] != 0) return false;
    return true;
}

bool batch_valid_series(int64_t m, int32_t n, int32_t n_max) {
    if (n < 1 || m < 1 || (int64_t)n > m || n > n_max) return false;
    const int64_t N = m - n + 1;
    if (N < 2 * (int64_t)n) return false;
    return m <= (int64_t)0x7fffffff - 4096;
}

void drop_layout(dd_batch_s* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    for (dd_plan_s* gp : b->gplans) delete gp;
    b->gplans.clear();
    b->garr.clear();
    b->gkey.clear();
}

dd_result_t invalid_result() {
    dd_result_t r;
    std::memset(&r, 0, sizeof(r));
    r.index = -1;
    r.status = DD_EINVAL;
    return r;
}

// Enqueues one group's launches on s (captured into the batch's graph).
cudaError_t enqueue_group(dd_batch_s* b, dd::BArr& A, dd_plan_s* gp, int nblocks, cudaStream_t s) {
    using namespace dd;
    const int sm = b->sm_count;
    const int gser = A.ns < 2 * sm ? A.ns : 2 * sm;
    cudaError_t e = cudaMemsetAsync(A.G, 0, sizeof(BGrp), s);
    if (e != cudaSuccess) return e;
    k_b_init<<<1, 256, 0, s>>>(A);
    k_b_prep<<<gser, kPT, 0, s>>>(A);
    const int gb = nblocks < sm * 8 ? nblocks : sm * 8;
    if (A.bf16)
        k_b_build<__nv_bfloat16><<<gb, 256, 0, s>>>(A, nblocks);
    else
        k_b_build<__half><<<gb, 256, 0, s>>>(A, nblocks);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    Ctrl* ctrl = &A.G->ctrl;
    TcArgs t{};
    t.N = (int)A.P;
    t.n = A.n;
    t.nka = A.kpad / kTcAtom;
    t.stages = tc_stages(A.kpad);
    t.seg_cols = A.seg_cols;
    t.sig = A.sig;
    t.coldat = A.coldat;
    t.rowmu = A.rowmu;
    t.rowc = A.rowc;
    t.alpha = A.alpha;
    t.gam = A.gam;
    t.q2 = A.q2;
    t.beta = kTcBeta;
    t.sigpos = A.sigpos;
    t.rmin = A.rmin;
    t.ctrl = ctrl;
    t.stats = A.G->gstats;
    t.abandon = 1;
    t.wave = -1;
    const uint32_t ty = A.bf16 ? 1u : 0u;
    t.idesc = (1u << 4) | (ty << 7) | (ty << 10) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    // band: every row tile of the group against the 256 columns around it
    TcArgs band = t;
    band.mode = 3;
    band.rows = ListRef{A.sig, nullptr, &A.G->band_rows};
    band.a_direct = 1;
    band.a_row0 = 0;
    band.work_slot = 0;
    if ((e = launch_scan_tc(gp, band, false, s)) != cudaSuccess) return e;
    // the top tile of every series: full lower-bound scans
    k_b_top<<<gser, kPT, 0, s>>>(A);
    const ListRef top{A.list_top, nullptr, &A.G->top_rows};
    if ((e = launch_gather_rows(gp, top, s)) != cudaSuccess) return e;
    TcArgs tw = t;
    tw.mode = 2;
    tw.rows = top;
    tw.ranges = A.ranges_top;
    tw.smax = &ctrl->smax[0];
    tw.work_slot = 1;
    if ((e = launch_scan_tc(gp, tw, true, s)) != cudaSuccess) return e;
    // survivors against their own series' best-so-far
    k_b_surv<<<gser, kPT, 0, s>>>(A);
    const ListRef rest{A.list_rest, nullptr, &A.G->rest_rows};
    if ((e = launch_gather_rows(gp, rest, s)) != cudaSuccess) return e;
    TcArgs rw = t;
    rw.mode = 2;
    rw.rows = rest;
    rw.ranges = A.ranges_rest;
    rw.smax = &ctrl->smax[1];
    rw.work_slot = 2;
    rw.tser = A.tser_rest;
    rw.sbsf = A.sbsf;
    if ((e = launch_scan_tc(gp, rw, true, s)) != cudaSuccess) return e;
    k_b_cands<<<gser, kPT, 0, s>>>(A);
    // direct FP32 full scans of the candidates of series with more than kBSettle
    {
        ScanArgs f{};
        f.t32 = A.t32;
        f.N = (int)A.P;
        f.n = A.n;
        f.rows = ListRef{A.list_settle, nullptr, &A.G->settle_rows};
        f.col = ColSpec{2, 0, 0, 0, 0};
        f.sig = A.sig;
        f.ranges = A.ranges_settle;
        f.smax = &ctrl->smax[2];
        f.seg_cols = A.seg_cols;
        f.rmin = A.rmin;
        f.ctrl_ro = ctrl;
        f.ctrl = ctrl;
        f.abandon = 1;
        f.tser = A.tser_settle;
        f.sbsf = A.sbsf;
        f.bm = A.settle_rows;
        f.work_slot = 4;
        f.min_seg_tiles = 4;
        f.target_items = 4 * sm;
        f.wave = -1;
        f.tb = TcBound{A.alpha, A.gam, A.q2, kTcBeta, 1, nullptr, nullptr};
        f.r32 = A.r32;
        f.stats = A.G->gstats;
        if ((e = launch_scan_fp32(f, 2 * sm, s)) != cudaSuccess) return e;
    }
    k_b_cands2<<<gser, kPT, 0, s>>>(A);
    // the warp-per-column screen is latency-bound: up to 5 resident blocks per SM (48 registers)
    k_b_rescore<<<8 * sm, 256, 0, s>>>(A);
    k_b_best<<<sm, 256, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

void dd_batch_config_default(dd_batch_config_t* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->seg_cols = 512;
    cfg->settle_min = 4;
    cfg->settle_rows = 64;
}

size_t dd_batch_footprint(int32_t max_series, int64_t max_values, int32_t n_max) {
    if (max_series < 1 || max_series > (1 << 16) || max_values < 1 || n_max < 1 || n_max > (1 << 16)) return 0;
    if (dd::rcap_of(max_series, max_values) > (int64_t)1 << 30) return 0;
    return dd::batch_bytes(max_series, max_values, n_max);
}

dd_status_t dd_batch_create(dd_batch_t* batch, int32_t max_series, int64_t max_values, int32_t n_max,
                            const dd_options_t* opt, const dd_batch_config_t* cfg) {
    if (!batch) return DD_EINVAL;
    *batch = nullptr;
    dd_options_t o;
    if (opt)
        o = *opt;
    else
        dd_options_default(&o);
    if (o.precision != DD_TC_FP16 && o.precision != DD_TC_BF16) return DD_ENOTSUP;
    if (o.znorm != 0 || o.shard_count > 1 || o.diag != 0) return DD_ENOTSUP;
    dd_batch_config_t c;
    if (cfg)
        c = *cfg;
    else
        dd_batch_config_default(&c);
    if (!valid_config(c)) return DD_EINVAL;
    const size_t bytes = dd_batch_footprint(max_series, max_values, n_max);
    if (bytes == 0) return DD_EINVAL;
    dd_batch_s* b = new (std::nothrow) dd_batch_s();
    if (!b) return DD_ENOMEM;
    b->max_series = max_series;
    b->max_values = max_values;
    b->n_max = n_max;
    b->opt = o;
    b->cfg = c;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaMalloc(&b->arena, bytes);
    if (e == cudaSuccess) {
        b->arena_bytes = bytes;
        e = cudaMallocHost(reinterpret_cast<void**>(&b->ser_host), sizeof(dd::BSer) * (size_t)max_series);
    }
    if (e == cudaSuccess)
        e = cudaMallocHost(reinterpret_cast<void**>(&b->res_host), sizeof(dd_result_t) * (size_t)max_series);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        dd_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? DD_ENOMEM : DD_ECUDA;
    }
    dd::BCarver cv{static_cast<char*>(b->arena)};
    dd::carve_wide(cv, b->W, max_series);
    b->wide_end = cv.off;
    *batch = b;
    return DD_OK;
}

void dd_batch_destroy(dd_batch_t b) {
    if (!b) return;
    if (b->cs) cudaStreamSynchronize(b->cs);
    drop_layout(b);
    for (cudaStream_t x : b->gs) cudaStreamDestroy(x);
    for (cudaEvent_t x : b->gev) cudaEventDestroy(x);
    if (b->arena) cudaFree(b->arena);
    if (b->ser_host) cudaFreeHost(b->ser_host);
    if (b->res_host) cudaFreeHost(b->res_host);
    if (b->cs) cudaStreamDestroy(b->cs);
    delete b;
}

int64_t dd_batch_graph_replays(dd_batch_t b) { return b ? b->replays : -1; }

dd_status_t dd_batch_set_schedule(dd_batch_t b, int32_t n, const dd_batch_config_t* cfg) {
    if (!b || n < 1) return DD_EINVAL;
    if (cfg && !valid_config(*cfg)) return DD_EINVAL;
    int expected = 0;
    if (!b->busy.compare_exchange_strong(expected, 1)) return DD_EBUSY;
    auto it = std::find_if(b->sched.begin(), b->sched.end(), [&](const auto& e) { return e.first == n; });
    if (it != b->sched.end()) b->sched.erase(it);
    if (cfg) b->sched.emplace_back(n, *cfg);
    b->gkey.clear();  // the next call captures its graph with the new schedule
    b->busy.store(0);
    return DD_OK;
}

}  // extern "C"

extern "C" dd_status_t dd_batch_search(dd_batch_t b, int32_t count, const float* const* T_dev, const int64_t* m,
                                       const int32_t* n, dd_result_t* out, void* stream) {
    using namespace dd;
    if (!b || count < 0 || (count > 0 && (!T_dev || !m || !n || !out))) return DD_EINVAL;
    // a failure of the whole call marks every result with its status
    auto fail = [&](dd_status_t st) {
        for (int32_t k = 0; k < count; k++) {
            out[k] = invalid_result();
            out[k].status = st;
        }
        return st;
    };
    int expected = 0;
    if (!b->busy.compare_exchange_strong(expected, 1)) return fail(DD_EBUSY);
    struct Release {
        dd_batch_s* b;
        ~Release() { b->busy.store(0); }
    } rel{b};
    if (count == 0) return DD_OK;
    if (count > b->max_series) return fail(DD_ENOMEM);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // validity, then the grouped order: n ascending, longest series first in a group
    std::vector<int64_t> key;
    key.reserve(3 * (size_t)count + 1);
    key.push_back(count);
    std::vector<int> order;
    for (int32_t k = 0; k < count; k++) {
        const bool ok = T_dev[k] != nullptr && batch_valid_series(m[k], n[k], b->n_max);
        key.push_back(m[k]);
        key.push_back(n[k]);
        key.push_back(ok ? 1 : 0);
        if (ok) order.push_back(k);
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        if (n[a] != n[c]) return n[a] < n[c];
        return m[a] > m[c];
    });
    const int nvalid = (int)order.size();
    int64_t values = 0;
    for (int k : order) values += m[k];
    if (values > b->max_values) return fail(DD_ENOMEM);
    if (key != b->gkey) {
        // a new layout: carve the groups, make their tensor maps, capture the graph
        drop_layout(b);
        BCarver cv{static_cast<char*>(b->arena)};
        cv.off = b->wide_end;
        int ngroups = 0;
        std::vector<int> nblocks;
        for (int j0 = 0; j0 < nvalid;) {
            int j1 = j0;
            while (j1 < nvalid && n[order[(size_t)j1]] == n[order[(size_t)j0]]) j1++;
            if (++ngroups > kMaxGroups) {
                drop_layout(b);
                return fail(DD_ENOTSUP);
            }
            BArr A{};
            A.ser = b->W.ser;
            A.s0 = j0;
            A.ns = j1 - j0;
            A.n = n[order[(size_t)j0]];
            A.bf16 = b->opt.precision == DD_TC_BF16 ? 1 : 0;
            const dd_batch_config_t& gc = schedule_of(b, A.n);
            A.seg_cols = gc.seg_cols;
            A.settle_min = gc.settle_min;
            A.settle_rows = gc.settle_rows;
            A.binstart = b->W.binstart;
            A.sbsf = b->W.sbsf;
            A.res = b->W.res;
            int64_t base = 0;
            int rb = 0;
            for (int j = j0; j < j1; j++) {
                const int k = order[(size_t)j];
                BSer& L = b->ser_host[j];
                std::memset(&L, 0, sizeof(BSer));
                L.m = m[k];
                L.n = n[k];
                L.N = (int32_t)(m[k] - n[k] + 1);
                L.base = (int32_t)base;
                L.npad = (int32_t)npad_of(m[k]);
                L.rb0 = rb;
                L.rb1 = rb + L.npad / kBRows;
                L.vbase = base;
                L.slot = k;
                base += L.npad;
                rb = L.rb1;
            }
            void* a16 = nullptr;
            carve_group(cv, A, &a16, base, A.ns, kpad_of(A.n));
            if (cv.off > b->arena_bytes || base > ((int64_t)1 << 30)) {
                drop_layout(b);
                return fail(DD_ENOMEM);
            }
            dd_plan_s* gp = new (std::nothrow) dd_plan_s();
            if (!gp) {
                drop_layout(b);
                return fail(DD_ENOMEM);
            }
            gp->N = base;
            gp->n = A.n;
            gp->m = base + A.n - 1;
            gp->kpad = A.kpad;
            gp->S16 = A.S16;
            gp->A16 = a16;
            gp->sigpos = A.sigpos;
            gp->sm_count = b->sm_count;
            gp->device = b->device;
            gp->opt = b->opt;
            b->gplans.push_back(gp);
            if (tc_make_maps(gp) != cudaSuccess) {
                drop_layout(b);
                return fail(DD_ECUDA);
            }
            b->garr.push_back(A);
            nblocks.push_back(rb);
            j0 = j1;
        }
        b->slot_grouped.assign(order.begin(), order.end());
        // capture
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess && nvalid > 0)
            e = cudaMemcpyAsync(b->W.ser, b->ser_host, sizeof(BSer) * (size_t)nvalid, cudaMemcpyHostToDevice, b->cs);
        // group g on stream g (forked from and joined back into the capture stream)
        const size_t ng = b->garr.size();
        while (e == cudaSuccess && b->gs.size() < ng) {
            cudaStream_t x = nullptr;
            cudaEvent_t f = nullptr, j = nullptr;
            e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
            if (e == cudaSuccess) b->gs.push_back(x);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f, cudaEventDisableTiming);
            if (e == cudaSuccess) b->gev.push_back(f);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
            if (e == cudaSuccess) b->gev.push_back(j);
        }
        for (size_t gi = 0; gi < ng && e == cudaSuccess; gi++) {
            e = cudaEventRecord(b->gev[2 * gi], b->cs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->gs[gi], b->gev[2 * gi], 0);
            if (e == cudaSuccess) e = enqueue_group(b, b->garr[gi], b->gplans[gi], nblocks[gi], b->gs[gi]);
            if (e == cudaSuccess) e = cudaEventRecord(b->gev[2 * gi + 1], b->gs[gi]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cs, b->gev[2 * gi + 1], 0);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->res_host, b->W.res, sizeof(dd_result_t) * (size_t)count, cudaMemcpyDeviceToHost,
                                b->cs);
        const cudaError_t e2 = cudaStreamEndCapture(b->cs, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            drop_layout(b);
            return fail(DD_ECUDA);
        }
        b->gkey = key;
    } else {
        b->replays++;
    }
    // this call's series pointers and fresh per-series state
    for (int j = 0; j < nvalid; j++) {
        BSer& L = b->ser_host[j];
        const int k = order[(size_t)j];
        L.T = T_dev[k];
        const int64_t keep_m = L.m, keep_vb = L.vbase;
        const int32_t keep[8] = {L.n, L.N, L.base, L.npad, L.rb0, L.rb1, L.slot, 0};
        std::memset(&L, 0, sizeof(BSer));
        L.T = T_dev[k];
        L.m = keep_m;
        L.vbase = keep_vb;
        L.n = keep[0];
        L.N = keep[1];
        L.base = keep[2];
        L.npad = keep[3];
        L.rb0 = keep[4];
        L.rb1 = keep[5];
        L.slot = keep[6];
        L.best_idx = 0x7fffffff;
    }
    b->calls++;
    cudaError_t e = cudaGraphLaunch(b->gexec, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(DD_ECUDA);
    dd_status_t first = DD_OK;
    std::vector<char> ok((size_t)count, 0);
    for (int j = 0; j < nvalid; j++) ok[(size_t)order[(size_t)j]] = 1;
    for (int32_t k = 0; k < count; k++) {
        out[k] = ok[(size_t)k] ? b->res_host[k] : invalid_result();
        if (first == DD_OK && out[k].status != DD_OK) first = (dd_status_t)out[k].status;
    }
    return first;
}
