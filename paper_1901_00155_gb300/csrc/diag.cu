// diag.cu -- exhaustive nearest-neighbour profile by the diagonal recurrence of
// centred dot products, and the per-window z-normalised discord search built
// on it.
//
// For subsequences i, j of a series y (Section 2.1), with window means mu and
// centred sums of squares c (the rows of the subsequence matrix, Eq. 5), the
// centred dot product C(i, j) = sum_k (y_{i+k} - mu_i)(y_{j+k} - mu_j) obeys,
// along a diagonal j - i = const,
//     C(i+1, j+1) = C(i, j) + df_i dg_j + df_j dg_i,
//     df_r = (y_{r+n} - y_r) / 2,   dg_r = (y_{r+n} - mu_{r+1}) + (y_r - mu_r)
// (expanding both sides, the cross terms cancel).  From C the squared
// distance (Eq. 1) is
//     global normalisation (Eq. 2, y = t^):  d^2 = c_i + c_j - 2C + n (mu_i - mu_j)^2
//     per-window normalisation (y = T):       d^2 = n (e_i + e_j - 2 C / sqrt(c_i c_j))
// where e = 1 for a non-constant window and 0 for a constant one, whose
// normalised form is the zero vector (then the C term is absent).  So a pair
// costs O(1) work instead of the O(n) of Eq. 1.
//
// k_diag: one CTA = 2048 consecutive diagonals x 2048 consecutive rows, whose
// row data it stages once in shared memory.  Each lane owns 8 consecutive
// diagonals and walks the rows, all lanes of the CTA on the same row at a
// time; every diagonal is re-seeded with a direct FP32 dot product at the
// CTA's first row, so rounding accumulates over at most 2048 steps.  A pair's score goes into a 32-bit key whose low 8 bits hold the
// diagonal inside the warp, so one float minimum tracks the value and its
// argument.  Per step:
//   - row minimum: each lane keeps one key per row for 8 steps; a transposing
//     shuffle reduction then leaves row r's minimum over the warp's 256
//     diagonals in one lane, which merges it across the CTA's warps in shared
//     memory and then (every 32 rows, one CTA barrier) into the global 64-bit
//     key (value bits << 32 | partner index) with atomicMin, once per row and
//     CTA;
//   - column minimum: a column moves through a lane's 8 diagonals in 8 steps
//     and then into the next lower lane; its running key and column data pass
//     down with __shfl_down_sync, leave the warp at lane 0, merge across
//     warps in a shared-memory ring, and go to the global key when they leave
//     the CTA.
// The arguments found this way are exact up to the recurrence's FP32
// rounding and the 8 key bits (2^-15 relative); k_diag_finish recomputes each
// row's distance to its argument directly (FP32, FP64 or as a rigorous FP32
// upper bound), so what is reported is the distance to a real non-self match.
//
// Per-window discord search (the variant in which every subsequence is
// z-normalised on its own; the mean lower bound of the global form is void
// there, every window having mean 0): profile -> rigorous FP32 upper bound
// ub_x >= nn_x^2 from the distance to each row's argument -> exact FP64
// rescoring of the row with the largest bound, giving a lower bound LB0 <=
// nn^2 of the discord -> exact FP64 rescoring of every row with ub_x >= LB0
// (a superset of the discord) -> argmax, ties to the smallest index.
#include <cfloat>

#include "dd_internal.cuh"

namespace dd {
namespace {

constexpr int kDgD = 8;                          // diagonals per lane
constexpr int kDgWarps = 8;
constexpr int kDgThreads = 32 * kDgWarps;
constexpr int kDgWarpDiags = 32 * kDgD;          // 256
constexpr int kDgTD = kDgWarps * kDgWarpDiags;   // 2048 diagonals per CTA
constexpr int kDgRS = 2048;                      // rows per CTA (one re-seed each)
constexpr int kDgRing = 2 * kDgTD;               // column-key ring (power of two)
constexpr int kDgFlush = 4;                      // groups of 8 rows between CTA-wide merges
constexpr size_t kDgSmem = sizeof(float4) * kDgRS + sizeof(unsigned long long) * kDgRing;
constexpr float kDgNone = 3.0e38f;               // score of a pair outside the triangle
constexpr unsigned long long kEmpty = ~0ull;
constexpr int kWChunk = 512;                     // columns per rescoring work item
static_assert(kDgPad >= kDgTD + 16, "series data padding must cover a CTA's diagonals");
static_assert((kDgRing & (kDgRing - 1)) == 0, "ring size must be a power of two");

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Window statistics, two-pass in FP64 in the element order of the oracle's
// definition (no contraction into FMA): mu_r, c_r.  Per-window form: 1/sigma
// (FP64), 1/sqrt(c) and e for the recurrence, and for the FP32 screen
// 1/sigma rounded to FP32 with E_r, a bound on || z~_r - z_r || (the error of
// the FP32 normalised window computed as (y - fl32(mu)) * fl32(1/sigma)):
//   E_r = 3.01 u sqrt(n) + 1.0001 (n / sqrt(c)) (u |mu| + 1.0001 n u64 (|mu| + sqrt(c)))
// (relative rounding of the subtraction, the reciprocal and the product, and
// the offset error of fl32(mu) scaled by 1/sigma; |y - mu| <= sqrt(c) bounds
// the FP64 mean's error), rounded up.  Global form: c and sqrt(n) mu.
template <bool kWindow>
__global__ void __launch_bounds__(256) k_wstats(const float* __restrict__ y, int N, int n, double* __restrict__ mu64,
                                                double* __restrict__ r64, float4* __restrict__ wdat,
                                                float* __restrict__ wmu32, float2* __restrict__ wscr, Ctrl* ctrl) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const float* x = y + r;
    double s = 0.0;
    for (int q = 0; q < n; q++) s = __dadd_rn(s, (double)x[q]);
    double mu = __ddiv_rn(s, (double)n);
    double c = 0.0;
    for (int q = 0; q < n; q++) {
        const double d = __dsub_rn((double)x[q], mu);
        c = __dadd_rn(c, __dmul_rn(d, d));
    }
    if (!isfinite(c) || !isfinite(mu)) {
        atomicExch(&ctrl->nonfinite, 1);
        mu = 0.0;
        c = 0.0;
    }
    mu64[r] = mu;
    wmu32[r] = (float)mu;
    if (kWindow) {
        const double sg = __dsqrt_rn(__ddiv_rn(c, (double)n));
        const double rs = sg > 0.0 ? __drcp_rn(sg) : 0.0;
        r64[r] = rs;
        float E = 0.f;
        float inv = 0.f;
        if (c > 0.0) {
            const double u = 5.9604644775390625e-08, u64 = 1.1102230246251565e-16;
            const double sc = sqrt(c), am = fabs(mu), nd = (double)n;
            const double e = 3.01 * u * sqrt(nd) + 1.0001 * (nd / sc) * (u * am + 1.0001 * nd * u64 * (am + sc));
            E = (float)(e * (1.0 + 1e-6));
            inv = (float)(1.0 / sc);
        }
        wdat[r] = make_float4(0.f, 0.f, inv, c > 0.0 ? 1.f : 0.f);
        wscr[r] = make_float2((float)rs, E);
    } else {
        wdat[r] = make_float4(0.f, 0.f, (float)c, (float)(sqrt((double)n) * mu));
    }
}

// Recurrence coefficients df_r, dg_r of the step r -> r+1 (zero for the last row).
__global__ void __launch_bounds__(256) k_wdiff(const float* __restrict__ y, int N, int n,
                                               const double* __restrict__ mu64, float4* __restrict__ wdat) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    float df = 0.f, dg = 0.f;
    if (r + 1 < N) {
        const double a = (double)y[r + n], b = (double)y[r];
        df = (float)((a - b) * 0.5);
        dg = (float)((a - mu64[r + 1]) + (b - mu64[r]));
    }
    reinterpret_cast<float2*>(wdat + r)[0] = make_float2(df, dg);
}

__device__ __forceinline__ float dg_key(float sc, uint32_t tag) {
    return __uint_as_float((__float_as_uint(sc) & 0xFFFFFF00u) | tag);
}

// 64-bit key of a 32-bit pair key found at diagonal base kw: (value bits << 32
// | partner).  partner_sign = +1: the partner is row + diagonal (row keys),
// -1: column - diagonal (column keys).  Returns false for masked pairs.
__device__ __forceinline__ bool key64(float kf, int kw, long long at, int sign, unsigned long long& out) {
    const uint32_t b = __float_as_uint(kf);
    const float val = __uint_as_float(b & 0xFFFFFF00u);
    if (!(val < 1e38f)) return false;
    const long long diag = (long long)kw + (long long)(b & 0xFFu);
    const long long partner = at + sign * diag;
    const float vc = val > 0.f ? val : 0.f;
    out = ((unsigned long long)__float_as_uint(vc) << 32) | (unsigned long long)(uint32_t)partner;
    return true;
}

// Lane state of k_diag: the centred dot products of the lane's 8 diagonals
// and its window of 8 columns (slot p holds the column of diagonal d at step
// u when p = (u + d) mod 8): recurrence data, score terms and running key.
struct DiagLane {
    float C[kDgD];
    float cdf[kDgD], cdg[kDgD], cf[kDgD], cg[kDgD], ck[kDgD];
};

// Eight steps (rows rbase .. rbase+7) of one lane.  kFull: every pair of the
// CTA lies inside the triangle r + k < N (no masking).  rows: the CTA's row
// data in shared memory (row r at rows[r - r0]).
template <bool kWindow, bool kFull>
__device__ __forceinline__ void diag_group(DiagLane& L, float (&rk)[8], const float4* __restrict__ wdat,
                                           const float4* rows, int rbase, int r0, long long kw, long long kb, int N,
                                           int lane, float* colst) {
#pragma unroll
    for (int u = 0; u < 8; u++) {
        const int r = rbase + u;
        // the column entering the warp at the end of this step (same address in
        // every lane: one broadcast load, issued a step's work ahead of its use)
        const float4 R = rows[r - r0];
        const float rowfac = -2.f * R.z;
        float ra = kDgNone, rb = kDgNone;  // the row minimum in two chains (shorter dependency)
#pragma unroll
        for (int d = 0; d < kDgD; d++) {
            const int p = (u + d) & 7;
            float sc;
            if (kWindow) {
                sc = fmaf(L.C[d] * rowfac, L.cf[p], R.w + L.cg[p]);
            } else {
                const float dm = R.w - L.cg[p];
                sc = fmaf(dm, dm, fmaf(-2.f, L.C[d], R.z + L.cf[p]));
            }
            if (!kFull && (long long)r + kb + d >= (long long)N) sc = kDgNone;
            const float kf = dg_key(sc, (uint32_t)(lane * kDgD + d));
            if (d & 1)
                rb = fminf(rb, kf);
            else
                ra = fminf(ra, kf);
            L.ck[p] = fminf(L.ck[p], kf);
            L.C[d] = fmaf(R.x, L.cdg[p], L.C[d]);
            L.C[d] = fmaf(L.cdf[p], R.y, L.C[d]);
        }
        rk[u] = fminf(ra, rb);
        // the column of diagonal 0 leaves this lane for lane - 1; lane + 1's
        // enters as diagonal 7 (lane 31 loads the warp's new column)
        const int pl = u & 7;
        float ik = __shfl_down_sync(0xffffffffu, L.ck[pl], 1);
        float i0 = __shfl_down_sync(0xffffffffu, L.cdf[pl], 1);
        float i1 = __shfl_down_sync(0xffffffffu, L.cdg[pl], 1);
        float i2 = __shfl_down_sync(0xffffffffu, L.cf[pl], 1);
        float i3 = __shfl_down_sync(0xffffffffu, L.cg[pl], 1);
        if (lane == 0) colst[u] = L.ck[pl];
        if (lane == 31) {
            const float4 v = wdat[(long long)r + 1 + kb + (kDgD - 1)];
            ik = kDgNone;
            i0 = v.x;
            i1 = v.y;
            i2 = v.z;
            i3 = v.w;
        }
        L.ck[pl] = ik;
        L.cdf[pl] = i0;
        L.cdg[pl] = i1;
        L.cf[pl] = i2;
        L.cg[pl] = i3;
    }
}

// Transposing minimum over the warp of rk[0..7] (one key per row of the
// group): afterwards lane l holds the minimum for row (l & 7) in rk[0].
__device__ __forceinline__ void rows_reduce(float (&rk)[8], int lane) {
#pragma unroll
    for (int q = 0; q < 8; q++) rk[q] = fminf(rk[q], __shfl_xor_sync(0xffffffffu, rk[q], 16));
#pragma unroll
    for (int q = 0; q < 8; q++) rk[q] = fminf(rk[q], __shfl_xor_sync(0xffffffffu, rk[q], 8));
    {
        const bool hi = (lane & 4) != 0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const float send = hi ? rk[q] : rk[q + 4];
            const float keep = hi ? rk[q + 4] : rk[q];
            rk[q] = fminf(keep, __shfl_xor_sync(0xffffffffu, send, 4));
        }
    }
    {
        const bool hi = (lane & 2) != 0;
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const float send = hi ? rk[q] : rk[q + 2];
            const float keep = hi ? rk[q + 2] : rk[q];
            rk[q] = fminf(keep, __shfl_xor_sync(0xffffffffu, send, 2));
        }
    }
    {
        const bool hi = (lane & 1) != 0;
        const float send = hi ? rk[0] : rk[1];
        const float keep = hi ? rk[1] : rk[0];
        rk[0] = fminf(keep, __shfl_xor_sync(0xffffffffu, send, 1));
    }
}

// The CTA's rows, in groups of 8; rows and the columns that left the CTA are
// merged into the global keys every kDgFlush groups (one CTA barrier each).
template <bool kWindow, bool kFull>
__device__ __forceinline__ void diag_rows(DiagLane& L, const float4* __restrict__ wdat, const float4* rows, int r0,
                                          int S, int k0, long long kw, long long kb, int N, int w, int lane,
                                          unsigned long long* ring, unsigned long long (*rowst)[8 * kDgFlush],
                                          float (*colst)[8], unsigned long long* __restrict__ key) {
    const int ngrp = S >> 3;
    for (int grp = 0; grp < ngrp; grp++) {
        const int rbase = r0 + grp * 8;
        const int buf = (grp / kDgFlush) & 1;
        float rk[8];
        diag_group<kWindow, kFull>(L, rk, wdat, rows, rbase, r0, kw, kb, N, lane, colst[w]);
        rows_reduce(rk, lane);
        __syncwarp();
        if (lane < 8) {
            unsigned long long v;
            // row rbase + lane: partner = row + diagonal
            if (key64(rk[0], (int)kw, (long long)rbase + lane, 1, v))
                atomicMin(&rowst[buf][(grp % kDgFlush) * 8 + lane], v);
            // the column that left lane 0 at step `lane`: partner = column - diagonal
            const long long c = (long long)rbase + lane + kw;
            if (key64(colst[w][lane], (int)kw, c, -1, v)) atomicMin(&ring[c & (kDgRing - 1)], v);
        }
        if (grp % kDgFlush == kDgFlush - 1 || grp == ngrp - 1) {
            __syncthreads();
            const int first = grp - grp % kDgFlush;  // first group of this flush window
            const int nrow = (grp - first + 1) * 8;
            const int wbase = r0 + first * 8;
            const int t = threadIdx.x;
            if (t < nrow) {
                const unsigned long long v = rowst[buf][t];
                if (v != kEmpty) atomicMin(&key[wbase + t], v);
                rowst[buf][t] = kEmpty;
            } else if (t >= 128 && t - 128 < nrow) {
                // columns that left the CTA (warp 0's lane 0) during the window
                const long long c = (long long)wbase + (t - 128) + k0;
                const int slot = (int)(c & (kDgRing - 1));
                const unsigned long long v = ring[slot];
                if (v != kEmpty) atomicMin(&key[c], v);
                ring[slot] = kEmpty;
            }
        }
    }
}

// Grid: one CTA per (diagonal block b, row block g), item = b * nseg + g.
template <bool kWindow>
__global__ void __launch_bounds__(kDgThreads, 2) k_diag(const float* __restrict__ y, int64_t m, int N, int n,
                                                        const float4* __restrict__ wdat,
                                                        const float* __restrict__ wmu32, int nseg,
                                                        unsigned long long* __restrict__ key, const Ctrl* ctrl) {
    extern __shared__ float4 dg_smem[];
    float4* rows = dg_smem;                                                              // [kDgRS]
    unsigned long long* ring = reinterpret_cast<unsigned long long*>(dg_smem + kDgRS);   // [kDgRing]
    __shared__ unsigned long long rowst[2][8 * kDgFlush];
    __shared__ float colst[kDgWarps][8];
    if (ctrl->nonfinite) return;
    const int b = blockIdx.x / nseg, g = blockIdx.x % nseg;
    const int k0 = n + b * kDgTD;
    const int r0 = g * kDgRS;
    if (k0 >= N || r0 >= N - k0) return;  // no pair of this block lies in the triangle
    const int rhi = min(r0 + kDgRS, N - k0);
    const int S = ((rhi - r0) + 7) & ~7;
    const bool full = (long long)r0 + S + k0 + kDgTD - 1 <= (long long)N;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kDgRing; i += kDgThreads) ring[i] = kEmpty;
    if (tid < 16 * kDgFlush) rowst[tid / (8 * kDgFlush)][tid % (8 * kDgFlush)] = kEmpty;
    for (int i = tid; i < S; i += kDgThreads) rows[i] = wdat[r0 + i];
    const long long kw = (long long)k0 + (long long)w * kDgWarpDiags;  // the warp's first diagonal
    const long long kb = kw + (long long)lane * kDgD;                   // this lane's first diagonal

    DiagLane L;
    // Seeds: C(r0, r0 + k) by direct FP32 dot products of the centred windows.
    {
        const float mr = wmu32[r0];
        float cm[kDgD];
        bool vd[kDgD];
#pragma unroll
        for (int d = 0; d < kDgD; d++) {
            const long long col = (long long)r0 + kb + d;
            vd[d] = col < (long long)N;
            cm[d] = wmu32[vd[d] ? col : 0];
            L.C[d] = 0.f;
        }
        const long long base = (long long)r0 + kb;
        for (int q0 = 0; q0 < n; q0 += 8) {
            float yb[16];
#pragma unroll
            for (int t = 0; t < 16; t++) {
                const long long ix = base + q0 + t;
                yb[t] = y[ix < m ? ix : m - 1];
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int q = q0 + u;
                const float a = q < n ? y[r0 + q] - mr : 0.f;
#pragma unroll
                for (int d = 0; d < kDgD; d++) L.C[d] = fmaf(a, yb[u + d] - cm[d], L.C[d]);
            }
        }
#pragma unroll
        for (int d = 0; d < kDgD; d++)
            if (!vd[d]) L.C[d] = 0.f;
    }
    // column window at the first row
#pragma unroll
    for (int d = 0; d < kDgD; d++) {
        const float4 v = wdat[(long long)r0 + kb + d];
        L.cdf[d] = v.x;
        L.cdg[d] = v.y;
        L.cf[d] = v.z;
        L.cg[d] = v.w;
        L.ck[d] = kDgNone;
    }
    __syncthreads();
    if (full)
        diag_rows<kWindow, true>(L, wdat, rows, r0, S, k0, kw, kb, N, w, lane, ring, rowst, colst, key);
    else
        diag_rows<kWindow, false>(L, wdat, rows, r0, S, k0, kw, kb, N, w, lane, ring, rowst, colst, key);
    // columns still inside the lanes' windows: slot p holds diagonal p (S is a
    // multiple of 8), column r0 + S + kb + p
#pragma unroll
    for (int p = 0; p < kDgD; p++) {
        unsigned long long v;
        const long long c = (long long)r0 + S + kb + p;
        if (key64(L.ck[p], (int)kw, c, -1, v)) atomicMin(&ring[c & (kDgRing - 1)], v);
    }
    __syncthreads();
    for (int t = tid; t < kDgTD + 8; t += kDgThreads) {
        const long long c = (long long)r0 + S + k0 + t;
        const unsigned long long v = ring[c & (kDgRing - 1)];
        if (v != kEmpty) atomicMin(&key[c], v);
    }
}

// FP32 screen of the per-window distance between rows x and j: s32 = the
// FP32 sum of squared differences of the FP32 normalised windows (one warp,
// lanes striding the window).  |z~ - z| <= E per window, the differences and
// squares round by u each and the sum of at most n + 8 terms by gamma, so
//   (sqrt(s32) (1 - sl) - 2 (E_x + E_j))^2 (1 - 8u) <= d^2 <= (sqrt(s32) (1 + sl) + 2 (E_x + E_j))^2 (1 + 8u)
// with sl = 2 (gamma_{n+8} + 2u) (factors doubled against the rounding of the
// bound's own evaluation).
__device__ __forceinline__ float wscreen(const float* __restrict__ T, int x, int j, int n, float mx, float zx,
                                         float mj, float zj, int lane) {
    float s = 0.f;
    for (int q = lane; q < n; q += 32) {
        const float a = (T[x + q] - mx) * zx;
        const float b = (T[j + q] - mj) * zj;
        const float d = a - b;
        s = fmaf(d, d, s);
    }
    return warp_sum(s);
}

struct WBound {
    float sl, u8;
    __device__ __forceinline__ explicit WBound(int n) {
        const float u = 5.9604644775390625e-08f;
        const float nu = (float)(n + 8) * u;
        sl = 2.f * (nu / (1.f - nu) + 2.f * u);
        u8 = 8.f * u;
    }
    __device__ __forceinline__ float upper(float s32, float E) const {
        const float r = sqrtf(s32) * (1.f + sl) + 2.f * E;
        return r * r * (1.f + u8);
    }
    __device__ __forceinline__ float lower(float s32, float E) const {
        const float r = sqrtf(s32) * (1.f - sl) - 2.f * E;
        return r > 0.f ? r * r * (1.f - u8) : 0.f;
    }
};

// Exact per-window distance in FP64 (z = (T - mu) / sigma with the FP64
// window statistics, the reciprocal precomputed), one warp.
__device__ __forceinline__ double wexact(const float* __restrict__ T, int x, int j, int n, double mx, double rx,
                                         double mj, double rj, int lane) {
    double s = 0.0;
    for (int q = lane; q < n; q += 32) {
        const double a = ((double)T[x + q] - mx) * rx;
        const double b = ((double)T[j + q] - mj) * rj;
        const double d = a - b;
        s = fma(d, d, s);
    }
    return warp_sum64(s);
}

// One warp per row x: the distance to the row's argument j = key & 0xffffffff.
//   mode 0 (global profile):  FP32 direct differences on t^ (Eq. 1 squared);
//   mode 1 (window profile):  exact FP64 per-window distance;
//   mode 2 (window search):   the FP32 screen's rigorous upper bound -> ub[x],
//                             and the argmax of ub over rows that may be the
//                             discord -> ctrl->key (bits << 32 | ~x).
// Thread 0 also publishes the pair count of the exhaustive wave.
template <int kMode>
__global__ void __launch_bounds__(256) k_diag_finish(const float* __restrict__ y, int N, int n,
                                                     const unsigned long long* __restrict__ key,
                                                     const double* __restrict__ mu64, const double* __restrict__ r64,
                                                     const float* __restrict__ wmu32, const float2* __restrict__ wscr,
                                                     const uint8_t* __restrict__ excl, float* __restrict__ out,
                                                     int32_t* __restrict__ idx_out, Ctrl* ctrl,
                                                     unsigned long long pairs, int wave, long long items) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->pairs = pairs;
        if (wave >= 0) {
            ctrl->wave_pairs[wave] = pairs;
            ctrl->wave_items[wave] = (unsigned long long)items;
            ctrl->wave_rows[wave] = N;
        }
    }
    if (ctrl->nonfinite) return;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const WBound wb(n);
    for (int x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < N; x += warps) {
        const unsigned long long v = key[x];
        const long long j64 = (long long)(v & 0xffffffffull);
        if (v == kEmpty || j64 >= N || (j64 - x < n && x - j64 < n)) {
            if (lane == 0) {
                atomicExch(&ctrl->err, DD_ECUDA);
                if (kMode != 2) out[x] = __int_as_float(0x7fffffff);
                if (idx_out) idx_out[x] = -1;
            }
            continue;
        }
        const int j = (int)j64;
        if (kMode == 0) {
            float s = 0.f;
            for (int q = lane; q < n; q += 32) {
                const float d = y[x + q] - y[j + q];
                s = fmaf(d, d, s);
            }
            s = warp_sum(s);
            if (lane == 0) out[x] = s;
        } else if (kMode == 1) {
            const double s = wexact(y, x, j, n, mu64[x], r64[x], mu64[j], r64[j], lane);
            if (lane == 0) out[x] = (float)s;
        } else {
            const float2 ax = wscr[x], aj = wscr[j];
            const float s32 = wscreen(y, x, j, n, wmu32[x], ax.x, wmu32[j], aj.x, lane);
            const float ub = wb.upper(s32, ax.y + aj.y);
            if (lane == 0) {
                out[x] = ub;
                if (!excl[x])
                    atomicMax(&ctrl->key, ((unsigned long long)__float_as_uint(ub) << 32) |
                                              (unsigned long long)(0xffffffffu - (uint32_t)x));
            }
        }
        if (lane == 0 && idx_out) idx_out[x] = j;
    }
}

// Exact FP64 nearest-neighbour distance of the rows of a list (per-window
// form).  Work items = (list entry, chunk of 512 columns), handed out
// dynamically; one warp per column.  use_bound: skip a column whose screened
// lower bound exceeds the row's upper bound ub[x] (it cannot be the nearest
// neighbour); otherwise every column is evaluated exactly.  Chunk minima meet
// in an atomicMin on the double's bits (non-negative doubles order like their
// bit patterns) in ex64[entry].
__global__ void __launch_bounds__(256) k_wrescore(ListRef rows, const float* __restrict__ T, int N, int n,
                                                  const double* __restrict__ mu64, const double* __restrict__ r64,
                                                  const float* __restrict__ wmu32, const float2* __restrict__ wscr,
                                                  const float* __restrict__ ub, int use_bound,
                                                  unsigned long long* __restrict__ ex64, Ctrl* ctrl, int slot) {
    __shared__ int sh_item;
    __shared__ double red[8];
    if (ctrl->nonfinite) return;
    const int cnt = *rows.cnt_dev;
    const int off = rows.off_dev ? *rows.off_dev : 0;
    const int nchunk = (N + kWChunk - 1) / kWChunk;
    const long long items = (long long)cnt * nchunk;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const WBound wb(n);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) sh_item = atomicAdd(&ctrl->work[slot], 1);
        __syncthreads();
        const long long item = sh_item;
        if (item < 0 || item >= items) {
            // a negative claim: the 32-bit work counter wrapped (more than 2^31 items)
            if (item < 0 && threadIdx.x == 0) atomicExch(&ctrl->err, DD_ENOTSUP);
            break;
        }
        const int r = (int)(item / nchunk), c = (int)(item % nchunk);
        const int x = rows.base[off + r];
        if (x < 0 || x >= N) {
            if (threadIdx.x == 0) atomicExch(&ctrl->err, DD_EINVAL);
            continue;
        }
        const float thr = use_bound ? ub[x] : INFINITY;
        const double mx = mu64[x], rx = r64[x];
        const float2 ax = wscr[x];
        const float mx32 = wmu32[x];
        const int a1 = min(N, (c + 1) * kWChunk);
        double best = INFINITY;
        for (int j = c * kWChunk + wid; j < a1; j += nwarp) {
            if (j - x < n && x - j < n) continue;
            if (use_bound) {
                const float2 aj = wscr[j];
                const float s32 = wscreen(T, x, j, n, mx32, ax.x, wmu32[j], aj.x, lane);
                if (wb.lower(s32, ax.y + aj.y) > thr) continue;
            }
            best = fmin(best, wexact(T, x, j, n, mx, rx, mu64[j], r64[j], lane));
        }
        if (lane == 0) red[wid] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = red[0];
            for (int w = 1; w < nwarp; w++) b = fmin(b, red[w]);
            if (b < INFINITY) atomicMin(ex64 + r, (unsigned long long)__double_as_longlong(b));
        }
    }
}

// The row with the largest upper bound (ctrl->key) -> a one-entry list, and
// its result slot reset.
__global__ void k_wpick(const Ctrl* ctrl, int32_t* list, int* cnt, unsigned long long* lb) {
    if (threadIdx.x != 0) return;
    const unsigned long long k = ctrl->key;
    *lb = 0x7ff0000000000000ull;  // +inf
    if (k == 0 || ctrl->nonfinite) {
        *cnt = 0;
        return;
    }
    list[0] = (int32_t)(0xffffffffu - (uint32_t)(k & 0xffffffffull));
    *cnt = 1;
}

// Every row that may be the discord (ub >= LB0, not excluded) -> list, with its
// rescoring slot reset (warp-aggregated append; order is irrelevant, the
// final argmax breaks ties by index).
__global__ void __launch_bounds__(256) k_wcand(const float* __restrict__ ub, const uint8_t* __restrict__ excl, int N,
                                               const unsigned long long* lbbits, int32_t* __restrict__ list,
                                               int* cnt, unsigned long long* __restrict__ ex64, const Ctrl* ctrl) {
    if (ctrl->nonfinite) return;
    const unsigned long long lbb = *lbbits;
    const double lb = lbb == 0x7ff0000000000000ull ? 0.0 : __longlong_as_double((long long)lbb) * (1.0 - 1e-9);
    // every upper bound 0 (e.g. only constant windows): every row's distance is 0 and the
    // row with the largest key, the smallest index, is the discord -- rescore it alone
    const unsigned long long k = ctrl->key;
    const bool all_zero = k != 0 && (k >> 32) == 0;
    const int r0 = (int)(0xffffffffu - (uint32_t)(k & 0xffffffffull));
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * blockDim.x; base < N; base += gridDim.x * blockDim.x) {
        const int x = base + threadIdx.x;
        const bool take = x < N && !excl[x] && (all_zero ? x == r0 : (double)ub[x] >= lb);
        const unsigned mask = __ballot_sync(0xffffffffu, take);
        if (!mask) continue;
        int at = 0;
        if (lane == 0) at = atomicAdd(cnt, __popc(mask));
        at = __shfl_sync(0xffffffffu, at, 0) + __popc(mask & ((1u << lane) - 1u));
        if (take) {
            list[at] = x;
            ex64[at] = 0x7ff0000000000000ull;
        }
    }
}

__global__ void k_set_count(int* p, int v) {
    if (threadIdx.x == 0) *p = v;
}

__global__ void __launch_bounds__(256) k_gather64(const unsigned long long* __restrict__ ex64, int count,
                                                  float* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) out[k] = (float)__longlong_as_double((long long)ex64[k]);
}

}  // namespace

// ---- launchers --------------------------------------------------------------

namespace {

int diag_blocks(int N, int n) { return (N - n + kDgTD - 1) / kDgTD; }
int diag_segs(int N, int n) { return (N - n + kDgRS - 1) / kDgRS; }

// Window statistics and recurrence coefficients of y (T itself per window,
// t^ globally), then the exhaustive recurrence into p->dkey.
cudaError_t diag_core(dd_plan_s* p, const float* y, bool window, int wave, cudaStream_t s) {
    const int N = (int)p->N, n = p->n;
    cudaError_t e = cudaMemsetAsync(p->dkey, 0xff, sizeof(unsigned long long) * (size_t)N, s);
    if (e != cudaSuccess) return e;
    const unsigned gs = (unsigned)((N + 255) / 256);
    if (window)
        k_wstats<true><<<gs, 256, 0, s>>>(y, N, n, p->wmu64, p->wr64, p->wdat, p->wmu32, p->wscr, p->ctrl);
    else
        k_wstats<false><<<gs, 256, 0, s>>>(y, N, n, p->wmu64, p->wr64, p->wdat, p->wmu32, p->wscr, p->ctrl);
    k_wdiff<<<gs, 256, 0, s>>>(y, N, n, p->wmu64, p->wdat);
    const int B = diag_blocks(N, n), G = diag_segs(N, n);
    const long long grid = (long long)B * G;
    if (grid < 1 || grid > 0x7fffffffll) return cudaErrorInvalidValue;
    if (wave >= 0) prof_mark(p, s, true);
    // 64 KiB of dynamic shared memory (row data + column ring): opt in on the current device
    cudaError_t attr = window ? cudaFuncSetAttribute(k_diag<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)kDgSmem)
                              : cudaFuncSetAttribute(k_diag<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)kDgSmem);
    if (attr != cudaSuccess) return attr;
    if (window)
        k_diag<true><<<(unsigned)grid, kDgThreads, kDgSmem, s>>>(y, p->m, N, n, p->wdat, p->wmu32, G, p->dkey,
                                                                 p->ctrl);
    else
        k_diag<false><<<(unsigned)grid, kDgThreads, kDgSmem, s>>>(y, p->m, N, n, p->wdat, p->wmu32, G, p->dkey,
                                                                  p->ctrl);
    if (wave >= 0) prof_mark(p, s, false);
    p->launches += 3;
    return cudaGetLastError();
}

unsigned long long diag_pairs(int64_t N, int n) {
    const unsigned long long k = (unsigned long long)(N - n);
    return k * (k + 1) / 2;
}

long long diag_items(int N, int n) {
    long long items = 0;
    const int B = diag_blocks(N, n), G = diag_segs(N, n);
    for (int b = 0; b < B; b++) {
        const long long rows = (long long)N - n - (long long)b * kDgTD;  // rows of the block's first diagonal
        if (rows > 0) items += (rows + kDgRS - 1) / kDgRS < G ? (rows + kDgRS - 1) / kDgRS : G;
    }
    return items;
}

int record_wave(dd_plan_s* p, int kind) {
    if (p->nwaves >= kMaxWaves) return -1;
    const int w = p->nwaves++;
    p->waves[w] = dd_plan_s::WaveMeta{kind, (p->profiling && !p->in_cond) ? p->ev_used : -1};
    return w;
}

unsigned finish_grid(const dd_plan_s* p) { return (unsigned)(4 * p->sm_count); }

}  // namespace

cudaError_t launch_profile_diag(dd_plan_s* p, const float* T, float* nn2, int32_t* idx, cudaStream_t s) {
    p->launches = 0;
    p->nwaves = 0;
    p->bodies.clear();
    const bool window = p->opt.znorm == 1;
    cudaError_t e = cudaMemsetAsync(p->ctrl, 0, sizeof(Ctrl), s);
    if (e != cudaSuccess) return e;
    const float* y = T;
    if (!window) {
        e = launch_prep_common(p, T, s);  // Eq. 2: t^ (FP32 copy), finiteness
        if (e != cudaSuccess) return e;
        y = p->t32;
    }
    const int wave = record_wave(p, DD_WAVE_DIAG);
    e = diag_core(p, y, window, wave, s);
    if (e != cudaSuccess) return e;
    const int N = (int)p->N, n = p->n;
    if (window)
        k_diag_finish<1><<<finish_grid(p), 256, 0, s>>>(y, N, n, p->dkey, p->wmu64, p->wr64, p->wmu32, p->wscr,
                                                         p->excl, nn2, idx, p->ctrl, diag_pairs(N, n), wave,
                                                         diag_items(N, n));
    else
        k_diag_finish<0><<<finish_grid(p), 256, 0, s>>>(y, N, n, p->dkey, p->wmu64, p->wr64, p->wmu32, p->wscr,
                                                         p->excl, nn2, idx, p->ctrl, diag_pairs(N, n), wave,
                                                         diag_items(N, n));
    p->launches++;
    return cudaGetLastError();
}

cudaError_t launch_rows_window(dd_plan_s* p, const float* T, const int32_t* rows, int count, float* nn2,
                               cudaStream_t s) {
    p->launches = 0;
    p->nwaves = 0;
    p->bodies.clear();
    const int N = (int)p->N, n = p->n;
    cudaError_t e = cudaMemsetAsync(p->ctrl, 0, sizeof(Ctrl), s);
    if (e != cudaSuccess) return e;
    const unsigned gs = (unsigned)((N + 255) / 256);
    k_wstats<true><<<gs, 256, 0, s>>>(T, N, n, p->wmu64, p->wr64, p->wdat, p->wmu32, p->wscr, p->ctrl);
    p->launches++;
    // at most N rows per pass (the size of the FP64 result array)
    for (int done = 0, pass = 0; done < count && pass < kMaxListSlots; pass++) {
        const int c = count - done < N ? count - done : N;
        e = cudaMemsetAsync(p->ex64, 0x7f, sizeof(double) * (size_t)c, s);
        if (e != cudaSuccess) return e;
        k_set_count<<<1, 32, 0, s>>>(&p->ctrl->cnt[pass], c);
        k_wrescore<<<2 * p->sm_count, 256, 0, s>>>(ListRef{rows + done, nullptr, &p->ctrl->cnt[pass]}, T, N, n,
                                                   p->wmu64, p->wr64, p->wmu32, p->wscr, nullptr, 0,
                                                   reinterpret_cast<unsigned long long*>(p->ex64), p->ctrl, pass);
        k_gather64<<<(unsigned)((c + 255) / 256), 256, 0, s>>>(reinterpret_cast<const unsigned long long*>(p->ex64),
                                                               c, nn2 + done);
        p->launches += 3;
        done += c;
        if (done < count && pass + 1 == kMaxListSlots) return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_search_window(dd_plan_s* p, const float* T, dd_result_t* out_dev, cudaStream_t s) {
    p->launches = 0;
    p->nwaves = 0;
    p->bodies.clear();
    const int N = (int)p->N, n = p->n;
    cudaError_t e = cudaMemsetAsync(p->ctrl, 0, sizeof(Ctrl), s);
    if (e != cudaSuccess) return e;
    const int wave = record_wave(p, DD_WAVE_DIAG);
    e = diag_core(p, T, true, wave, s);
    if (e != cudaSuccess) return e;
    unsigned long long* ex = reinterpret_cast<unsigned long long*>(p->ex64);
    // upper bounds and the row with the largest one
    k_diag_finish<2><<<finish_grid(p), 256, 0, s>>>(T, N, n, p->dkey, p->wmu64, p->wr64, p->wmu32, p->wscr, p->excl,
                                                     p->dub, nullptr, p->ctrl, diag_pairs(N, n), wave,
                                                     diag_items(N, n));
    // LB0: its exact nearest-neighbour distance
    int* cnt0 = &p->ctrl->cnt[0];
    int* cnt1 = &p->ctrl->cnt[1];
    unsigned long long* lb = &p->ctrl->wlb;
    k_wpick<<<1, 32, 0, s>>>(p->ctrl, p->list[3], cnt0, lb);
    k_wrescore<<<2 * p->sm_count, 256, 0, s>>>(ListRef{p->list[3], nullptr, cnt0}, T, N, n, p->wmu64, p->wr64,
                                               p->wmu32, p->wscr, p->dub, 1, lb, p->ctrl, 0);
    // every row whose bound reaches LB0, rescored exactly
    k_wcand<<<(unsigned)(2 * p->sm_count), 256, 0, s>>>(p->dub, p->excl, N, lb, p->list[0], cnt1, ex, p->ctrl);
    k_wrescore<<<2 * p->sm_count, 256, 0, s>>>(ListRef{p->list[0], nullptr, cnt1}, T, N, n, p->wmu64, p->wr64,
                                               p->wmu32, p->wscr, p->dub, 1, ex, p->ctrl, 1);
    p->launches += 5;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_best(p, ListRef{p->list[0], nullptr, cnt1}, out_dev, s);
}

}  // namespace dd
