// prep.cu -- preparation stage of PhiDD (Algorithm 2, before the search):
//   Eq. 2   z-normalisation of the whole series (FP64 mean and population sigma)
//           and the FP32 / FP64 normalised copies,
//           FP64 exclusive prefix sums P1 = sum t^, P2 = sum t^^2,
//   Eq. 5   per-row statistics of the subsequence matrix (mean mu_i, centred
//           sum of squares c_i) from the prefix sums,
//   Eq. 3/4/9  PAA -> SAX word code per row,
//   Eq. 8/7/10 word histogram (Freq), candidate set (Cand = rarest words) and
//           the word index (Index_Word) as one row order: words by ascending
//           frequency, rows ascending within a word (stable counting sort).
#include <cmath>

#include "dd_internal.cuh"

namespace dd {
namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum of one double per thread; result valid in thread 0.
template <int NT>
__device__ double block_sum_d(double v, double* sh) {
    v = warp_sum_d(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = (lane < NT / 32) ? sh[lane] : 0.0;
        r = warp_sum_d(r);
    }
    __syncthreads();
    return r;
}

template <int NT>
__device__ double block_max_d(double v, double* sh) {
    v = warp_max_d(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = (lane < NT / 32) ? sh[lane] : 0.0;
        r = warp_max_d(r);
    }
    __syncthreads();
    return r;
}

// ---- Eq. 2, pass 1: per-block sums of T, min/max, finiteness ----------------
// The extremes are taken in FP32 (exact: they are input values); the sum in
// FP64.  The last block to finish reduces the partials in a fixed order:
// mu = (1/m) sum t.
__device__ bool last_block(int* ticket) {
    __shared__ bool last;
    __threadfence();  // this block's partials are visible before its ticket
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
    __syncthreads();
    return last;
}

__global__ void __launch_bounds__(256) k_stats_sum(const float* __restrict__ T, int64_t m, double* part,
                                                   double* stats, Ctrl* ctrl) {
    __shared__ double sh[32];
    double s = 0.0;
    float mx = -INFINITY, mn = INFINITY;
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        float v = T[i];
        if (!isfinite(v)) bad = 1;
        s += (double)v;
        mx = fmaxf(mx, v);
        mn = fminf(mn, v);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(&ctrl->nonfinite, 1);
    double bs = block_sum_d<256>(s, sh);
    double bmx = block_max_d<256>((double)mx, sh);
    double bmn = -block_max_d<256>(-(double)mn, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = bs;
        part[kStatBlocks + blockIdx.x] = bmx;
        part[2 * kStatBlocks + blockIdx.x] = bmn;
    }
    if (!last_block(&ctrl->stat_ticket[0])) return;
    const int nb = (int)gridDim.x;
    const volatile double* vp = part;
    s = 0.0;
    double gmx = -INFINITY, gmn = INFINITY;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        s += vp[b];
        gmx = fmax(gmx, vp[kStatBlocks + b]);
        gmn = fmin(gmn, vp[2 * kStatBlocks + b]);
    }
    bs = block_sum_d<256>(s, sh);
    bmx = block_max_d<256>(gmx, sh);
    bmn = -block_max_d<256>(-gmn, sh);
    if (threadIdx.x == 0) {
        stats[0] = bs / (double)m;
        stats[4] = bmx;
        stats[5] = bmn;
    }
}

// ---- Eq. 2, pass 2: sum of squared deviations (two-pass variance) ------------
// The last block to finish reduces the partials in a fixed order: sigma, the
// largest |t^|, and the geometry of the mean bins.
__global__ void __launch_bounds__(256) k_stats_var(const float* __restrict__ T, int64_t m, double* stats,
                                                   double* part, Ctrl* ctrl) {
    __shared__ double sh[32];
    const double mu = stats[0];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        double d = (double)T[i] - mu;
        s += d * d;
    }
    double bs = block_sum_d<256>(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
    if (!last_block(&ctrl->stat_ticket[1])) return;
    const int nb = (int)gridDim.x;
    const volatile double* vp = part;
    s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += vp[b];
    bs = block_sum_d<256>(s, sh);
    if (threadIdx.x == 0) {
        double sigma = sqrt(bs / (double)m);
        stats[1] = sigma;
        // max |t^| over the series
        double a = fmax(fabs(stats[4] - mu), fabs(stats[5] - mu));
        stats[2] = sigma > 0.0 ? a / sigma : 0.0;
        if (!(sigma > 0.0)) ctrl->degenerate = 1;
        stats[8] = sigma > 0.0 ? 1.0 / sigma : 0.0;
        // mean-bin geometry: bins of width w over [min t^, max t^]
        const double lo = sigma > 0.0 ? (stats[5] - mu) / sigma : 0.0;
        const double hi = sigma > 0.0 ? (stats[4] - mu) / sigma : 0.0;
        const double w = (hi - lo) / (double)kMuBins;
        stats[6] = lo;
        stats[7] = w;
        stats[9] = w > 0.0 ? 1.0 / w : 0.0;
    }
}

// ---- Eq. 2 normalisation + FP64 prefix scan (3 passes) -----------------------
// Block b covers elements [b*kScanElems, (b+1)*kScanElems); 1024 threads x 4.
__global__ void __launch_bounds__(1024) k_norm_blocks(const float* __restrict__ T, int64_t m,
                                                      const double* stats, double* __restrict__ t64,
                                                      float* __restrict__ t32, double* bsum, int nscan) {
    __shared__ double sh[32];
    const double mu = stats[0], inv_sigma = stats[8];
    const int64_t base = (int64_t)blockIdx.x * kScanElems + 4 * threadIdx.x;
    double s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        int64_t i = base + q;
        if (i < m) {
            double v = ((double)T[i] - mu) * inv_sigma;
            t64[i] = v;
            t32[i] = (float)v;
            s1 += v;
            s2 += v * v;
        }
    }
    double b1 = block_sum_d<1024>(s1, sh);
    double b2 = block_sum_d<1024>(s2, sh);
    if (threadIdx.x == 0) {
        bsum[blockIdx.x] = b1;
        bsum[nscan + blockIdx.x] = b2;
    }
}

// Exclusive block scan of two doubles per thread (1024 threads).
__device__ void block_exscan2(double& a, double& b, double* sh1, double* sh2) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double ua = __shfl_up_sync(0xffffffffu, ia, o);
        double ub = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += ua;
            ib += ub;
        }
    }
    if (lane == 31) {
        sh1[wid] = ia;
        sh2[wid] = ib;
    }
    __syncthreads();
    if (wid == 0) {
        double wa = sh1[lane], wb = sh2[lane];
        double sa = wa, sb = wb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            double ua = __shfl_up_sync(0xffffffffu, sa, o);
            double ub = __shfl_up_sync(0xffffffffu, sb, o);
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

// Exclusive scan of the block totals (one block; each thread a run of
// consecutive totals, then a block scan of the run sums).
__global__ void __launch_bounds__(1024) k_norm_scan_totals(double* bsum, int nscan) {
    __shared__ double sh1[32], sh2[32];
    const int per = (nscan + 1023) / 1024;
    const int lo = threadIdx.x * per, hi = min(nscan, lo + per);
    double a1 = 0.0, a2 = 0.0;
    for (int b = lo; b < hi; b++) {
        a1 += bsum[b];
        a2 += bsum[nscan + b];
    }
    double e1 = a1, e2 = a2;
    block_exscan2(e1, e2, sh1, sh2);
    double c1 = e1, c2 = e2;
    for (int b = lo; b < hi; b++) {
        const double x1 = bsum[b], x2 = bsum[nscan + b];
        bsum[2 * nscan + b] = c1;
        bsum[3 * nscan + b] = c2;
        c1 += x1;
        c2 += x2;
    }
}

__global__ void __launch_bounds__(1024) k_norm_prefix(const double* __restrict__ t64, int64_t m,
                                                      const double* bsum, int nscan, double* __restrict__ P1,
                                                      double* __restrict__ P2) {
    __shared__ double sh1[32], sh2[32];
    const int64_t base = (int64_t)blockIdx.x * kScanElems + 4 * threadIdx.x;
    double v[4];
    double s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        int64_t i = base + q;
        v[q] = (i < m) ? t64[i] : 0.0;
        s1 += v[q];
        s2 += v[q] * v[q];
    }
    double e1 = s1, e2 = s2;
    block_exscan2(e1, e2, sh1, sh2);
    double c1 = bsum[2 * nscan + blockIdx.x] + e1;
    double c2 = bsum[3 * nscan + blockIdx.x] + e2;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        int64_t i = base + q;
        c1 += v[q];
        c2 += v[q] * v[q];
        if (i < m) {
            P1[i + 1] = c1;
            P2[i + 1] = c2;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P1[0] = 0.0;
        P2[0] = 0.0;
    }
}

// ---- Eq. 5 rows: mean and centred sum of squares from the prefix sums -------
// Also each row's bin of the mean-bucketed order (below): its mean mu_i over
// [min t^, max t^] in kMuBins equal bins.
__global__ void __launch_bounds__(256) k_window_stats(const double* __restrict__ P1, const double* __restrict__ P2,
                                                      int64_t N, int n, double inv_n, const double* stats,
                                                      double* __restrict__ mu_w, double* __restrict__ c_w,
                                                      int32_t* __restrict__ bin) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double S1 = P1[i + n] - P1[i];
    const double S2 = P2[i + n] - P2[i];
    const double mu = S1 * inv_n;
    double c = S2 - S1 * mu;
    // Within the rounding of the prefix sums a constant row has c == 0.
    const double noise = 64.0 * 1.1102230246251565e-16 * (fabs(P2[i + n]) + fabs(P2[i]));
    if (c <= noise) c = 0.0;
    mu_w[i] = mu;
    c_w[i] = c;
    const double b = floor((mu - stats[6]) * stats[9]);
    // NaN (non-finite series) and out-of-range values land in the end bins
    bin[i] = (b >= 0.0) ? (b < (double)kMuBins ? (int)b : kMuBins - 1) : 0;
}

// ---- Eq. 3 (PAA) + Eq. 4 (SAX letters) + Eq. 9 (word code) -----------------
// Segment s of a row covers [floor(s n / w), floor((s+1) n / w)), length L_s.
// The letter test beta <= (seg_sum / L_s - mu) / sd is evaluated as
// seg_sum - mu L_s >= beta L_s sd (sd > 0, L_s > 0): the same decision
// without an FP64 division per segment.
__global__ void __launch_bounds__(256) k_sax(const double* __restrict__ P1, const double* __restrict__ mu_w,
                                             const double* __restrict__ c_w, int64_t N, int n, double inv_n, int w,
                                             int A, int paa_mode, const double* __restrict__ beta,
                                             int32_t* __restrict__ code) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double mu = mu_w[i];
    const double c = c_w[i];
    // The FP64 test lhs >= beta_j * scale is taken in FP32 when the two FP32
    // sides differ by more than their rounding (<= 6 u32 of their magnitudes;
    // 1e-6 used), which then gives the same answer; otherwise in FP64.
    const float sd32 = sqrtf((float)(c * inv_n));
    int32_t h = 0;
    for (int s = 0; s < w; s++) {
        const int a = (int)(((int64_t)s * n) / w), b = (int)(((int64_t)(s + 1) * n) / w);
        const double len = (double)(b - a);
        const double seg = P1[i + b] - P1[i + a];
        double lhs;
        float scale32;
        const bool centred = paa_mode == 0 && c > 0.0;
        if (paa_mode == 0) {
            lhs = centred ? fma(-mu, len, seg) : 0.0;
            scale32 = centred ? (float)len * sd32 : 1.f;
        } else {
            lhs = seg;
            scale32 = (float)len;
        }
        const float lhs32 = (float)lhs;
        int letter = 0;
        while (letter < A - 1) {
            const float thr32 = (float)beta[letter] * scale32;
            bool ge;
            if (fabsf(lhs32 - thr32) > 1e-6f * (fabsf(lhs32) + fabsf(thr32)) + 1e-37f) {
                ge = lhs32 >= thr32;
            } else {
                const double scale = centred ? len * sqrt(c * inv_n) : (paa_mode == 0 ? 1.0 : len);
                ge = lhs >= beta[letter] * scale;
            }
            if (!ge) break;
            letter++;
        }
        h = h * A + letter;
    }
    code[i] = h;
}

__device__ __forceinline__ int64_t seq_row(int64_t r, int64_t N, int64_t stride) {
    return stride > 0 ? (int64_t)(((unsigned long long)r * (unsigned long long)stride) % (unsigned long long)N) : r;
}

// ---- Eq. 8: word histogram, one block-local count per word -----------------
// Keys of a counting sort: input element e is row in_perm[e] (or the stride
// permutation seq_row(e)); its key is (keys[row] >> shift) & mask.
struct KeySrc {
    const int32_t* keys;
    const int32_t* in_perm;
    int64_t stride;
    int shift;
    int mask;
};

__device__ __forceinline__ int64_t key_row(const KeySrc& k, int64_t e, int64_t N) {
    return k.in_perm ? (int64_t)k.in_perm[e] : seq_row(e, N, k.stride);
}
__device__ __forceinline__ int key_of(const KeySrc& k, int64_t row) { return (k.keys[row] >> k.shift) & k.mask; }

// Rows and keys of elements e0, e0 + step, ..., e0 + (G - 1) step, their loads
// issued together (entries past N or past `lim` get row -1, key -1).
template <int G>
__device__ __forceinline__ void load_keys(const KeySrc& ks, int64_t e0, int64_t step, int64_t lim, int64_t N,
                                          int64_t (&row)[G], int (&key)[G]) {
#pragma unroll
    for (int u = 0; u < G; u++) {
        const int64_t e = e0 + u * step;
        row[u] = e < lim && e < N ? key_row(ks, e, N) : -1;
    }
#pragma unroll
    for (int u = 0; u < G; u++) key[u] = row[u] >= 0 ? key_of(ks, row[u]) : -1;
}

__global__ void __launch_bounds__(1024) k_word_hist(KeySrc ks, int64_t N, int D, int32_t* __restrict__ hist,
                                                    int32_t* __restrict__ blockcnt) {
    extern __shared__ int32_t sh_cnt[];
    constexpr int G = kHistRows / 1024;  // elements per thread (blockDim.x == 1024)
    const int64_t base = (int64_t)blockIdx.x * kHistRows;
    int64_t row[G];
    int key[G];
    load_keys<G>(ks, base + threadIdx.x, 1024, base + kHistRows, N, row, key);
    for (int h = threadIdx.x; h < D; h += blockDim.x) sh_cnt[h] = 0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < G; u++)
        if (key[u] >= 0) atomicAdd(&sh_cnt[key[u]], 1);
    __syncthreads();
    for (int h = threadIdx.x; h < D; h += blockDim.x) {
        int c = sh_cnt[h];
        blockcnt[(int64_t)blockIdx.x * D + h] = c;
        if (c) atomicAdd(&hist[h], c);
    }
}

// Exclusive scan down each column h of the [nblk][D] block-count matrix,
// starting at start[h]: 32 columns per block, the rows split in 16 chunks
// (chunk sums, then a scan over the chunks, then the writes).
constexpr int kColChunks = 16;
__device__ __forceinline__ void colscan_cols(int32_t* __restrict__ blockcnt, int D, int nblk, int h, int c, int hl,
                                             int start_h, int (*sh)[32]) {
    const int CH = (nblk + kColChunks - 1) / kColChunks;
    const int b0 = c * CH, b1 = min(nblk, b0 + CH);
    int sum = 0;
    if (h < D)
        for (int b = b0; b < b1; b++) sum += blockcnt[(int64_t)b * D + h];
    sh[c][hl] = sum;
    __syncthreads();
    int run = start_h;
    for (int q = 0; q < c; q++) run += sh[q][hl];
    if (h < D)
        for (int b = b0; b < b1; b++) {
            const int64_t ix = (int64_t)b * D + h;
            const int v = blockcnt[ix];
            blockcnt[ix] = run;
            run += v;
        }
}

__global__ void __launch_bounds__(32 * kColChunks) k_colscan(int32_t* __restrict__ blockcnt, int D, int nblk,
                                                             const int32_t* __restrict__ start) {
    __shared__ int sh[kColChunks][32];
    const int hl = threadIdx.x, c = threadIdx.y;
    const int h = blockIdx.x * 32 + hl;
    colscan_cols(blockcnt, D, nblk, h, c, hl, h < D ? start[h] : 0, sh);
}

// Bin offsets of the mean-bucketed order: binstart[b] = the number of rows in
// bins below b (exclusive scan of the histogram), so binstart[b] is the first
// position whose row lies in bin >= b; binstart[kMuBins] = N.  One block of
// 1024 threads, 4 bins each.
__global__ void __launch_bounds__(1024) k_bin_start(const int32_t* __restrict__ hist, int64_t N,
                                                   int32_t* __restrict__ binstart) {
    __shared__ int part[32];
    constexpr int kPer = kMuBins / 1024;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    int c[kPer], s = 0;
#pragma unroll
    for (int q = 0; q < kPer; q++) {
        c[q] = hist[kPer * t + q];
        s += c[q];
    }
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) part[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int v = part[lane];
        int cc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, cc, o);
            if (lane >= o) cc += u;
        }
        part[lane] = cc - v;
    }
    __syncthreads();
    int run = part[wid] + incl - s;
#pragma unroll
    for (int q = 0; q < kPer; q++) {
        binstart[kPer * t + q] = run;
        run += c[q];
    }
    if (t == 0) binstart[kMuBins] = (int32_t)N;
}

// ---- Eq. 7 / Eq. 10 plan: words ordered by (frequency, word), offsets,
// |Cand|, and each block's base offset per word (column scan). One block.
__global__ void __launch_bounds__(1024) k_word_plan(const int32_t* __restrict__ hist, int D, int nblk,
                                                    int32_t* __restrict__ blockcnt, int32_t* __restrict__ word_start,
                                                    int phase1_max, int64_t N, Ctrl* ctrl) {
    __shared__ unsigned long long keys[kMaxDict];
    __shared__ int sh_min;
    int P = 1;
    while (P < D) P <<= 1;
    if (threadIdx.x == 0) sh_min = 0x7fffffff;
    __syncthreads();
    for (int h = threadIdx.x; h < P; h += blockDim.x) {
        if (h < D) {
            int c = hist[h];
            if (c > 0) atomicMin(&sh_min, c);
            unsigned long long f = c > 0 ? (unsigned long long)c : 0xffffffffull;
            keys[h] = (f << 32) | (unsigned long long)h;
        } else {
            keys[h] = ~0ull;
        }
    }
    __syncthreads();
    // bitonic sort ascending
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < P; t += blockDim.x) {
                int ixj = t ^ j;
                if (ixj > t) {
                    unsigned long long a = keys[t], b = keys[ixj];
                    bool up = ((t & k) == 0);
                    if ((a > b) == up) {
                        keys[t] = b;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        int run = 0, ncand = 0;
        const int fmin = sh_min;
        for (int r = 0; r < D; r++) {
            int h = (int)(keys[r] & 0xffffffffull);
            unsigned long long fk = keys[r] >> 32;
            int c = fk == 0xffffffffull ? 0 : (int)fk;  // the sort key holds the frequency
            word_start[h] = run;
            run += c;
            if (c == fmin) ncand += c;
        }
        ctrl->ncand = ncand;
        ctrl->fmin = fmin;
        int n1 = ncand < phase1_max ? ncand : phase1_max;
        ctrl->n1 = n1;
        ctrl->n2 = (int)(N - n1);
    }
    __syncthreads();
    (void)blockcnt;
    (void)nblk;
}

// ---- Eq. 10: stable scatter of rows into word order ------------------------
// Block b handles rows [b*kHistRows, (b+1)*kHistRows); warp w a contiguous
// slice of it, in rounds of 32 rows whose loads are issued 4 rounds at a time;
// ranks inside a round come from __match_any_sync.  Stable scatter: element e
// (in input order) of key h goes to position (block base of h) + (rank of e
// among the block's elements of key h).  The per-warp counters hold
// block-local positions in 16 bits (a block has kHistRows < 2^16 rows), two
// keys to a word, so that several blocks fit on an SM for large key ranges;
// the block base of a key is added when a row is placed.
__device__ __forceinline__ int get16(const uint32_t* w, int h) {
    return (int)((w[h >> 1] >> ((h & 1) * 16)) & 0xffffu);
}

__global__ void __launch_bounds__(1024, 2) k_word_scatter(KeySrc ks, int64_t N, int D,
                                                          const int32_t* __restrict__ blockbase,
                                                          int32_t* __restrict__ order, int32_t* __restrict__ pos_of) {
    extern __shared__ uint32_t sh_wc[];  // [nwarps][ceil(D / 2)], 16-bit counters
    constexpr int G = 4;
    const int nw = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int D2 = (D + 1) >> 1;
    for (int x = threadIdx.x; x < nw * D2; x += blockDim.x) sh_wc[x] = 0u;
    __syncthreads();
    const int per = kHistRows / nw;  // a multiple of 32 G (nw <= 32 divides kHistRows)
    const int64_t base = (int64_t)blockIdx.x * kHistRows + (int64_t)wid * per;
    uint32_t* wc = sh_wc + wid * D2;
    for (int g0 = 0; g0 < per; g0 += 32 * G) {
        int64_t row[G];
        int key[G];
        load_keys<G>(ks, base + g0 + lane, 32, base + per, N, row, key);
#pragma unroll
        for (int u = 0; u < G; u++)
            if (key[u] >= 0) atomicAdd(&wc[key[u] >> 1], 1u << ((key[u] & 1) * 16));
    }
    __syncthreads();
    // per key, exclusive scan over the warps (both halves of a word at once:
    // neither half can carry into the other)
    for (int h2 = threadIdx.x; h2 < D2; h2 += blockDim.x) {
        uint32_t run = 0u;
        for (int q = 0; q < nw; q++) {
            const uint32_t c = sh_wc[q * D2 + h2];
            sh_wc[q * D2 + h2] = run;
            run += c;
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t bb = (int64_t)blockIdx.x * D;
    for (int g0 = 0; g0 < per; g0 += 32 * G) {
        int64_t row[G];
        int key[G];
        load_keys<G>(ks, base + g0 + lane, 32, base + per, N, row, key);
        int kb[G];  // block base of each key
#pragma unroll
        for (int u = 0; u < G; u++) kb[u] = key[u] >= 0 ? blockbase[bb + key[u]] : 0;
#pragma unroll
        for (int u = 0; u < G; u++) {
            const bool ok = key[u] >= 0;
            const int h = ok ? key[u] : -1 - lane;  // unique dummy keys for idle lanes
            const unsigned peers = __match_any_sync(0xffffffffu, h);
            const int rank = __popc(peers & lt);
            const int loc = ok ? get16(wc, h) : 0;
            __syncwarp();
            if (ok) {
                const int pos = kb[u] + loc + rank;
                order[pos] = (int32_t)row[u];
                if (pos_of) pos_of[row[u]] = pos;
                if (rank == 0) atomicAdd(&wc[h >> 1], (uint32_t)__popc(peers) << ((h & 1) * 16));
            }
            __syncwarp();
        }
    }
}

// ---- mean-bucketed row order --------------------------------------------------
// Rows binned by their mean mu_i over [min t^, max t^] (kMuBins equal bins,
// computed with the row statistics).  For globally normalised subsequences
// d^2(i, j) >= n (mu_i - mu_j)^2, so the rows whose distance to row i can be
// below R lie in the bins within sqrt(R / n) of mu_i: a contiguous range of
// this order.

// Warps per block of the stable scatter: per-warp 16-bit counters for every
// key fit in 64 KB of shared memory, and the warps split the block's rows
// evenly.
int scatter_warps(int D) {
    int nw = (64 * 1024 / 4) / ((D + 1) / 2);  // at most 64 KB of counters: several blocks per SM
    if (nw > 32) nw = 32;
    if (nw < 1) nw = 1;
    while (kHistRows % nw) nw--;
    return nw;
}

}  // namespace

// Preparation, part 1: Eq. 2 statistics, normalisation, prefix sums, row statistics.
cudaError_t launch_prep_common(dd_plan_s* p, const float* T, cudaStream_t s) {
    cudaError_t ea = cudaFuncSetAttribute(k_word_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, 192 * 1024);
    if (ea != cudaSuccess) return ea;
    const int64_t m = p->m, N = p->N;
    const int n = p->n;
    int nb = (int)((m + 2047) / 2048);
    if (nb > kStatBlocks) nb = kStatBlocks;
    if (nb < 1) nb = 1;
    k_stats_sum<<<nb, 256, 0, s>>>(T, m, p->part, p->stats, p->ctrl);
    k_stats_var<<<nb, 256, 0, s>>>(T, m, p->stats, p->part, p->ctrl);
    const int nscan = (int)((m + kScanElems - 1) / kScanElems);
    k_norm_blocks<<<nscan, 1024, 0, s>>>(T, m, p->stats, p->t64, p->t32, p->bsum, nscan);
    k_norm_scan_totals<<<1, 1024, 0, s>>>(p->bsum, nscan);
    k_norm_prefix<<<nscan, 1024, 0, s>>>(p->t64, m, p->bsum, nscan, p->P1, p->P2);
    const int gN = (int)((N + 255) / 256);
    k_window_stats<<<gN, 256, 0, s>>>(p->P1, p->P2, N, n, 1.0 / (double)n, p->stats, p->mu_w, p->c_w, p->mubin);
    p->launches += 6;
    return cudaGetLastError();
}

// Part 2: SAX words (Eq. 3, 4, 9), Freq / Cand / Index_Word (Eq. 7, 8, 10).
cudaError_t launch_prep_words(dd_plan_s* p, cudaStream_t s) {
    const int64_t N = p->N;
    const int n = p->n;
    const int D = p->D;
    const int gN = (int)((N + 255) / 256);
    k_sax<<<gN, 256, 0, s>>>(p->P1, p->mu_w, p->c_w, N, n, 1.0 / (double)n, p->opt.paa_w, p->opt.alphabet,
                             p->opt.paa_mode, p->beta, p->code);
    const int nh = (int)((N + kHistRows - 1) / kHistRows);
    cudaMemsetAsync(p->hist, 0, sizeof(int32_t) * D, s);
    const KeySrc words{p->code, nullptr, 0, 0, 0x7fffffff};
    k_word_hist<<<nh, 1024, sizeof(int32_t) * D, s>>>(words, N, D, p->hist, p->blockcnt);
    k_word_plan<<<1, 1024, 0, s>>>(p->hist, D, nh, p->blockcnt, p->word_start, p->opt.phase1_max, N, p->ctrl);
    k_colscan<<<(D + 31) / 32, dim3(32, kColChunks), 0, s>>>(p->blockcnt, D, nh, p->word_start);
    int nw = scatter_warps(D);
    k_word_scatter<<<nh, nw * 32, sizeof(uint32_t) * nw * ((D + 1) / 2), s>>>(words, N, D, p->blockcnt, p->order,
                                                                            p->pos_of);
    p->launches += 5;
    return cudaGetLastError();
}

// Part 3: the mean-bucketed order and its bin offsets.
cudaError_t launch_prep_mean(dd_plan_s* p, cudaStream_t s) {
    const int64_t N = p->N;
    const int nh = (int)((N + kHistRows - 1) / kHistRows);
    // mean-bucketed order (sig): rows sorted by mean bin with one stable
    // counting sort over the kMuBins bins; the input follows a golden-ratio
    // stride permutation, so the rows of a bin are not in time order and
    // neighbours in this order are seldom overlapping subsequences
    const KeySrc ks{p->mubin, nullptr, p->mu_stride, 0, kMuBins - 1};
    cudaMemsetAsync(p->hist_mu, 0, sizeof(int32_t) * kMuBins, s);
    k_word_hist<<<nh, 1024, sizeof(int32_t) * kMuBins, s>>>(ks, N, kMuBins, p->hist_mu, p->blockcnt_mu);
    k_bin_start<<<1, 1024, 0, s>>>(p->hist_mu, N, p->binstart);
    k_colscan<<<(kMuBins + 31) / 32, dim3(32, kColChunks), 0, s>>>(p->blockcnt_mu, kMuBins, nh, p->binstart);
    const int nw = scatter_warps(kMuBins);
    k_word_scatter<<<nh, nw * 32, sizeof(uint32_t) * nw * (kMuBins / 2), s>>>(ks, N, kMuBins, p->blockcnt_mu,
                                                                            p->sig, p->sigpos);
    p->launches += 4;
    return cudaGetLastError();
}

cudaError_t launch_prep(dd_plan_s* p, const float* T, cudaStream_t s) {
    cudaError_t e = launch_prep_common(p, T, s);
    if (e == cudaSuccess) e = launch_prep_words(p, s);
    if (e == cudaSuccess) e = launch_prep_mean(p, s);
    return e;
}

// Breakpoints of the SAX alphabet (text after Eq. 4): Phi(beta_j) = j / A for
// the standard normal CDF Phi.  Newton iterations on Phi(x) - p from x = 0
// for the lower half; the upper half by symmetry, the median exactly 0.
void host_breakpoints(int A, double* beta) {
    const double inv_sqrt2pi = 0.39894228040143267794;
    for (int j = 1; 2 * j < A; j++) {
        const double p = (double)j / (double)A;
        double x = 0.0;
        for (int it = 0; it < 100; it++) {
            const double cdf = 0.5 * std::erfc(-x * 0.70710678118654752440);
            const double pdf = inv_sqrt2pi * std::exp(-0.5 * x * x);
            const double step = (cdf - p) / pdf;
            x -= step;
            if (std::fabs(step) < 1e-17) break;
        }
        beta[j - 1] = x;
        beta[A - j - 1] = -x;
    }
    if (A % 2 == 0) beta[A / 2 - 1] = 0.0;
}

}  // namespace dd
