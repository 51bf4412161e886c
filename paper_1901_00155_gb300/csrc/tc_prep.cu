// tc_prep.cu -- preparation for the tensor-core Gram form (scan_tc.cu): per-row
// and per-column constants, the per-row error bound terms F_i, the centred
// FP16 / BF16 operand matrix S in the mean-bucketed order, and the packing of
// listed rows for TMA.
//
// For globally normalised subsequences (Eq. 2) with means mu_i and centred
// sums of squares c_i (Eq. 5 rows), ||x_i - x_j||^2 = c_i + c_j +
// n (mu_i - mu_j)^2 - 2 <x'_i, x'_j>; S holds the scaled centred rows x'_i.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>

#include "dd_internal.cuh"

namespace dd {
namespace {

constexpr int TKA = kTcAtom;        // 16-bit elements per row chunk (one 128-byte line)
constexpr int kColPad = kTcColPad;  // padding of the per-column constant array on each side

// Per row (orig order) and per column (mean-bucketed order): sqrt(n) mu_i,
// c_i (FP32), sqrt(c_i) rounded up; maxima over all rows.
__global__ void __launch_bounds__(256) k_tc_rowconst(const double* __restrict__ mu_w, const double* __restrict__ c_w,
                                                     const int32_t* __restrict__ sigpos, int64_t N, double sqrt_n,
                                                     float4* __restrict__ coldat,
                                                     float* __restrict__ rowmu, float* __restrict__ rowc,
                                                     float* __restrict__ rowsc, Ctrl* ctrl) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float sc = 0.f, cc = 0.f, am = 0.f;
    if (i < N) {
        const float mu = (float)(mu_w[i] * sqrt_n);
        const float c = (float)c_w[i];
        cc = __double2float_ru(c_w[i]);
        sc = __fsqrt_ru(cc);
        am = fabsf(mu);
        const int p = sigpos[i];
        coldat[kColPad + p] = make_float4(mu, c, __int_as_float((int)i), 0.f);
        rowmu[i] = mu;
        rowc[i] = c;
        rowsc[i] = sc;
    }
    // non-negative floats order like their bit patterns; one atomic per block
    __shared__ unsigned red[3][8];
    const unsigned bsc = __reduce_max_sync(0xffffffffu, __float_as_uint(sc));
    const unsigned bcc = __reduce_max_sync(0xffffffffu, __float_as_uint(cc));
    const unsigned bam = __reduce_max_sync(0xffffffffu, __float_as_uint(am));
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = bsc;
        red[1][threadIdx.x >> 5] = bcc;
        red[2][threadIdx.x >> 5] = bam;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        unsigned v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) v = max(v, red[threadIdx.x][w]);
        unsigned int* dst = threadIdx.x == 0 ? &ctrl->tc_scmax : (threadIdx.x == 1 ? &ctrl->tc_cmax : &ctrl->tc_mumax);
        atomicMax(dst, v);
    }
}

// Per-row error bound F_i(D) = alpha_i + beta D + gam_i sqrt(D + q2_i) on
// |D - d^2| for a distance D computed by the Gram tiles (safety factor 2):
//   operands rounded to u_in (FP16 2^-11, BF16 2^-8), products exact in FP32,
//   accumulation of n terms with unit 2^-23 (directed rounding allowed):
//     |g~ - g| <= ((2 u_in + u_in^2) + gamma_n (1 + u_in)^2) sum|x'y'|,
//     sum|x'y'| <= sqrt(c_i) sqrt(c_j) <= sc_i sc_max = Q_i;
//   subnormal operands add <= 2^-25 / s per element (scale s);
//   FP32 rounding of c~, sqrt(n) mu~, the epilogue FMAs and the final sum is
//   bounded through dm^2 <= D + 2 Q_i and |dm| <= sqrt(D + 2 Q_i).
__global__ void __launch_bounds__(256) k_tc_rowbound(const float* __restrict__ rowsc, const float* __restrict__ rowc,
                                                     const float* __restrict__ rowmu, int64_t N, float sqrt_n,
                                                     float u_in, const double* stats, const double* P2end,
                                                     const Ctrl* ctrl, float* __restrict__ alpha,
                                                     float* __restrict__ gam, float* __restrict__ q2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float u32 = 5.9604644775390625e-08f;   // 2^-24
    const float uacc = 2.384185791015625e-07f;   // 2^-22: allows truncating accumulation
    const float n = sqrt_n * sqrt_n;
    const float scmax = __uint_as_float(ctrl->tc_scmax);
    const float cmax = __uint_as_float(ctrl->tc_cmax);
    const float mumax = __uint_as_float(ctrl->tc_mumax);
    const float s = (float)stats[3];
    const float maxabs = (float)stats[2];
    const float gn = n * uacc / (1.f - n * uacc);
    const float uo = u_in + 2.f * u32;  // operand: FP32 centring then one 16-bit rounding
    const float Kg = 2.f * ((2.f * uo + uo * uo) + gn * (1.f + uo) * (1.f + uo));
    const float sci = rowsc[i];
    const float Q = sci * scmax;
    const float ci = rowc[i];
    // absolute operand errors: FP32 centring (2.01 u32 max|t^|) and 16-bit subnormals (2^-25 / s)
    const float ea = 2.01f * u32 * maxabs + 2.9802322387695312e-08f / s;
    const float eta = 2.f * (ea * sqrt_n * (sci + scmax) + n * ea * ea);
    const float ec = 512.f * 1.1102230246251565e-16f * (1.f + (float)*P2end);
    const float A0 = Kg * Q + eta + 4.f * u32 * (ci + cmax) + 2.f * ec + 8.f * u32 * Q;
    const float G0 = 2.f * u32 * (fabsf(rowmu[i]) + mumax);
    alpha[i] = 2.002f * A0;
    gam[i] = 2.002f * G0;
    q2[i] = 2.002f * Q;
}


// Centred rows in the mean-bucketed order: S[p][k] = s (t^_{i+k} - mu_i),
// p = sigpos[i], computed in FP32 from the FP32 copy of t^ and rounded once to
// FP16 / BF16; zero for k in [n, kpad).  (The FP32 centring error, at most
// 2 u32 max|t^| per element, is part of the row bound.)
//
// A block builds kBsRows consecutive rows (time order).  They are windows of
// one stretch of t^, which the block stages in shared memory once per pass of
// up to kBsChunks 64-element chunks, so the series is read about once rather
// than n times.  Each chunk of a row is one 128-byte line of S (chunk-major
// layout), written by one warp (2 elements per lane, 4-byte stores) at the
// row's place in the mean order; a warp walks its rows, and each row's chunks,
// by pointer increments, with the bounds test k < n only in chunks that reach n.
constexpr int kBsRows = 64, kBsChunks = 16;

// Two 16-bit roundings packed into one word (element y0 at the lower address).
__device__ __forceinline__ uint32_t pack16(float y0, float y1, __half*) {
    const __half2 h = __floats2half2_rn(y0, y1);
    return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack16(float y0, float y1, __nv_bfloat16*) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(y0, y1);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// (x - mu) s for both elements of a pair with packed FP32 arithmetic (sm_100+
// f32x2): each element is rounded exactly as by a scalar subtract then multiply.
__device__ __forceinline__ float2 centre2(float2 x, unsigned long long mu2, unsigned long long s2) {
    unsigned long long v;
    asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(x.x), "f"(x.y));
    asm("sub.rn.f32x2 %0, %0, %1;" : "+l"(v) : "l"(mu2));
    asm("mul.rn.f32x2 %0, %0, %1;" : "+l"(v) : "l"(s2));
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ unsigned long long dup2(float x) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(x));
    return r;
}

template <typename T16>
__global__ void __launch_bounds__(256) k_build_S(const float* __restrict__ t32, const double* __restrict__ mu_w,
                                                 const int32_t* __restrict__ sigpos, int64_t N, int n, int kpad,
                                                 const double* stats, T16* __restrict__ S) {
    // seg[0][x] = t^_{i0 + k0 + x}; seg[1][x] = seg[0][x + 1], so that a lane's
    // two elements are one aligned 8-byte shared load for odd rows too
    constexpr int kSeg = kBsRows + kBsChunks * TKA;
    __shared__ __align__(16) float seg[2][kSeg];
    __shared__ float smu[kBsRows];
    __shared__ int spos[kBsRows];
    const int64_t i0 = (int64_t)blockIdx.x * kBsRows;
    const int64_t m = N + n - 1;
    const float s = (float)stats[3];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    if (threadIdx.x < kBsRows) {
        const int64_t i = i0 + threadIdx.x;
        // one FP64 -> FP32 conversion per row (FP64 throughput is low on this GPU)
        smu[threadIdx.x] = i < N ? (float)mu_w[i] : 0.f;
        spos[threadIdx.x] = i < N ? sigpos[i] : -1;
    }
    for (int k0 = 0; k0 < kpad; k0 += kBsChunks * TKA) {
        const int nch = min(kpad - k0, kBsChunks * TKA) / TKA;  // chunks of this pass
        // chunks whose 64 elements all lie below n (no zero padding inside)
        const int nfull = n - k0 >= nch * TKA ? nch : max(n - k0, 0) / TKA;
        __syncthreads();  // the previous pass has finished reading seg
        for (int x = threadIdx.x; x < kBsRows + nch * TKA; x += blockDim.x) {
            const int64_t g = i0 + k0 + x;
            const float v = g < m ? t32[g] : 0.f;
            seg[0][x] = v;
            if (x > 0) seg[1][x - 1] = v;
        }
        __syncthreads();
        // warp w: rows w, w + nwarp, ..., every chunk of each
        for (int r = wid; r < kBsRows; r += nwarp) {
            const int p = spos[r];
            if (p < 0) break;  // this row and every later one lie past N
            const float mu = smu[r];
            const float2* src = reinterpret_cast<const float2*>((r & 1) ? &seg[1][r - 1] : &seg[0][r]) + lane;
            T16* dst = S + ((int64_t)(k0 / TKA) * N + p) * TKA + 2 * lane;
            const unsigned long long mu2 = dup2(mu), s2 = dup2(s);
            int c = 0;
#pragma unroll 4
            for (; c < nfull; c++, src += TKA / 2, dst += N * TKA) {
                const float2 y = centre2(*src, mu2, s2);
                *reinterpret_cast<uint32_t*>(dst) = pack16(y.x, y.y, (T16*)nullptr);
            }
            for (int k = k0 + c * TKA + 2 * lane; c < nch; c++, k += TKA, src += TKA / 2, dst += N * TKA) {
                const float2 y = centre2(*src, mu2, s2);
                *reinterpret_cast<uint32_t*>(dst) = pack16(k < n ? y.x : 0.f, k + 1 < n ? y.y : 0.f, (T16*)nullptr);
            }
        }
    }
}

// Operand scale: a power of two that puts max |x'| <= 2 max|t^| near 2^14 (FP16).
__global__ void k_tc_scale(double* stats, int is_bf16) {
    if (threadIdx.x != 0) return;
    double s = 1.0;
    if (!is_bf16) {
        const double mx = 2.0 * stats[2];
        if (mx > 0.0) {
            int e = (int)floor(log2(16384.0 / mx));
            if (e > 24) e = 24;
            if (e < -24) e = -24;
            s = ldexp(1.0, e);
        }
    }
    stats[3] = s;
}

// Packs the operand rows of a list (in list order) for TMA.
__global__ void __launch_bounds__(256) k_gather_rows(ListRef L, const int32_t* __restrict__ sigpos,
                                                     const uint4* __restrict__ S, int kpad, int64_t N,
                                                     uint4* __restrict__ P) {
    const int cnt = *L.cnt_dev;
    const int off = L.off_dev ? *L.off_dev : 0;
    const int per_row = kpad / 8;  // uint4 per row (8 per 64-element chunk)
    const int64_t total = (int64_t)cnt * per_row;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = g / per_row;
        const int c = (int)(g % per_row);
        const int i = L.base[off + r];
        const int64_t plane = (int64_t)(c >> 3) * N;  // chunk-major: [chunk][row][8 uint4]
        // an entry that is not a row (-1) packs zeros; its tile row is masked anyway
        P[(plane + r) * 8 + (c & 7)] = i >= 0 ? S[(plane + sigpos[i]) * 8 + (c & 7)] : make_uint4(0u, 0u, 0u, 0u);
    }
}

}  // namespace

cudaError_t launch_tc_prep(dd_plan_s* p, cudaStream_t s) {
    const int64_t N = p->N;
    const int n = p->n;
    const bool bf16 = p->opt.precision == DD_TC_BF16;
    const int gN = (int)((N + 255) / 256);
    k_tc_scale<<<1, 32, 0, s>>>(p->stats, bf16 ? 1 : 0);
    k_tc_rowconst<<<gN, 256, 0, s>>>(p->mu_w, p->c_w, p->sigpos, N, std::sqrt((double)n), p->coldat, p->rowmu,
                                     p->rowc, p->rowsc, p->ctrl);
    const float u_in = bf16 ? 0.00390625f : 0.00048828125f;
    k_tc_rowbound<<<gN, 256, 0, s>>>(p->rowsc, p->rowc, p->rowmu, N, (float)std::sqrt((double)n), u_in, p->stats,
                                     p->P2 + p->m, p->ctrl, p->alpha, p->gam, p->q2);
    const int g = (int)((N + kBsRows - 1) / kBsRows);
    if (bf16)
        k_build_S<__nv_bfloat16><<<g, 256, 0, s>>>(p->t32, p->mu_w, p->sigpos, N, n, p->kpad, p->stats,
                                                   reinterpret_cast<__nv_bfloat16*>(p->S16));
    else
        k_build_S<__half><<<g, 256, 0, s>>>(p->t32, p->mu_w, p->sigpos, N, n, p->kpad, p->stats,
                                            reinterpret_cast<__half*>(p->S16));
    p->launches += 4;
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(dd_plan_s* p, ListRef L, cudaStream_t s) {
    const int g = p->sm_count * 4;
    k_gather_rows<<<g, 256, 0, s>>>(L, p->sigpos, reinterpret_cast<const uint4*>(p->S16), p->kpad, p->N,
                                    reinterpret_cast<uint4*>(p->A16));
    p->launches++;
    return cudaGetLastError();
}

}  // namespace dd
