// noalloc.cu -- dd_nn_profile_static: the exhaustive nearest-neighbour
// profile of dd_nn_profile (FP32 direct differences), for callers that must
// not allocate device memory.  It needs no plan: its scratch (the Eq. 2
// statistics and the normalised series) lives in one file-scope device array
// of fixed size, so the call itself never allocates.
//
// Limits and caveats (also stated in include/dd.h):
//   * series of at most kStaticMaxM points (larger ones are rejected);
//   * every call on a device shares the one array, so calls whose work
//     overlaps on the GPU (other streams, other host threads) race;
//   * the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current; make that first call
//     before any stream capture.
#include <mutex>

#include "dd_internal.cuh"

namespace dd {
namespace {

constexpr int64_t kStaticMaxM = 1 << 18;  // 262,144 points
constexpr int kStaticParts = 256;          // partial-sum blocks
constexpr int kPadS = 64;

struct StaticScratch {
    double stats[8];                  // [0] mu  [1] sigma  [2] non-finite flag
    double part[2 * kStaticParts];
    float t32[kStaticMaxM + kPadS];   // normalised series (Eq. 2), zero padded
};

// The only storage this entry point uses.  Every GPU that loads the library
// holds it (about 1 MiB) until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[sizeof(StaticScratch)];

std::mutex g_lock;
void* g_addr[256];
bool g_ready[256];

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// Eq. 2 pass 1: block sums of T and a count of non-finite values.
__global__ void __launch_bounds__(256) k_s_sum(const float* __restrict__ T, int64_t m, StaticScratch* s) {
    __shared__ double sh[8];
    double a = 0.0, bad = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = T[i];
        if (!isfinite(v)) bad += 1.0;
        a += (double)v;
    }
    a = block_sum(a, sh);
    bad = block_sum(bad, sh);
    if (threadIdx.x == 0) {
        s->part[blockIdx.x] = a;
        s->part[kStaticParts + blockIdx.x] = bad;
    }
}

__global__ void __launch_bounds__(256) k_s_mu(int64_t m, StaticScratch* s) {
    __shared__ double sh[8];
    const double a = block_sum(s->part[threadIdx.x], sh);
    const double bad = block_sum(s->part[kStaticParts + threadIdx.x], sh);
    if (threadIdx.x == 0) {
        s->stats[0] = a / (double)m;
        s->stats[2] = bad;
    }
}

// Eq. 2 pass 2: two-pass population variance.
__global__ void __launch_bounds__(256) k_s_var(const float* __restrict__ T, int64_t m, StaticScratch* s) {
    __shared__ double sh[8];
    const double mu = s->stats[0];
    double a = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = (double)T[i] - mu;
        a += d * d;
    }
    a = block_sum(a, sh);
    if (threadIdx.x == 0) s->part[blockIdx.x] = a;
}

__global__ void __launch_bounds__(256) k_s_sigma(int64_t m, StaticScratch* s) {
    __shared__ double sh[8];
    const double a = block_sum(s->part[threadIdx.x], sh);
    if (threadIdx.x == 0) s->stats[1] = sqrt(a / (double)m);
}

// t^ = (t - mu) / sigma (0 when sigma == 0), zero padding; output reset to +inf.
__global__ void __launch_bounds__(256) k_s_norm(const float* __restrict__ T, int64_t m, int64_t N,
                                                StaticScratch* s, float* __restrict__ nn2) {
    const double mu = s->stats[0], sigma = s->stats[1];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m + kPadS;
         i += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.f;
        if (i < m && sigma > 0.0) v = (float)(((double)T[i] - mu) / sigma);
        s->t32[i] = v;
        if (i < N) nn2[i] = INFINITY;
    }
}

// 64 rows x 256 columns per block; rows and columns are consecutive
// subsequences, staged 64 k at a time; each thread an 8x8 micro-tile of
// sum_k (x_k - y_k)^2 in FP32; row minima outside the exclusion zone
// |i - j| < n meet in an atomicMin on the float bits of nn2.
constexpr int SR = 64, SC = 256, SK = 64;

__global__ void __launch_bounds__(256) k_s_profile(int64_t N, int n, const StaticScratch* __restrict__ s,
                                                   float* __restrict__ nn2) {
    __shared__ float xr[SR + SK];
    __shared__ float yc[SC + SK];
    if (s->stats[2] != 0.0) return;  // non-finite input: the output is set to NaN below
    const int64_t i0 = (int64_t)blockIdx.x * SR, j0 = (int64_t)blockIdx.y * SC;
    const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; a++)
#pragma unroll
        for (int b = 0; b < 8; b++) acc[a][b] = 0.f;
    for (int k0 = 0; k0 < n; k0 += SK) {
        __syncthreads();
        for (int q = tid; q < SR + SK; q += blockDim.x) {
            const int64_t g = i0 + k0 + q;
            xr[q] = g < N + n - 1 ? s->t32[g] : 0.f;
        }
        for (int q = tid; q < SC + SK; q += blockDim.x) {
            const int64_t g = j0 + k0 + q;
            yc[q] = g < N + n - 1 ? s->t32[g] : 0.f;
        }
        __syncthreads();
        const int kmax = min(SK, n - k0);
        for (int k = 0; k < kmax; k++) {
            float x[8], y[8];
#pragma unroll
            for (int a = 0; a < 8; a++) x[a] = xr[ty * 8 + a + k];
#pragma unroll
            for (int b = 0; b < 8; b++) y[b] = yc[tx * 8 + b + k];
#pragma unroll
            for (int a = 0; a < 8; a++)
#pragma unroll
                for (int b = 0; b < 8; b++) {
                    const float d = x[a] - y[b];
                    acc[a][b] = fmaf(d, d, acc[a][b]);
                }
        }
    }
#pragma unroll
    for (int a = 0; a < 8; a++) {
        const int64_t i = i0 + ty * 8 + a;
        float mn = INFINITY;
#pragma unroll
        for (int b = 0; b < 8; b++) {
            const int64_t j = j0 + tx * 8 + b;
            const int64_t d = i - j;
            if (i < N && j < N && (d >= n || d <= -n)) mn = fminf(mn, acc[a][b]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        if (tx == 0 && i < N && mn < INFINITY) atomicMin(reinterpret_cast<unsigned*>(nn2) + i, __float_as_uint(mn));
    }
}

__global__ void __launch_bounds__(256) k_s_nan(int64_t N, const StaticScratch* __restrict__ s, float* nn2) {
    if (s->stats[2] == 0.0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        nn2[i] = __int_as_float(0x7fc00000);
}

}  // namespace
}  // namespace dd

extern "C" dd_status_t dd_nn_profile_static(const float* T_dev, int64_t m, int32_t n, float* nn2_dev,
                                            void* stream) {
    using namespace dd;
    if (!T_dev || !nn2_dev || n < 1 || m < 1 || (int64_t)n > m) return DD_EINVAL;
    const int64_t N = m - n + 1;
    if (N < 2 * (int64_t)n) return DD_EINVAL;
    if (m > kStaticMaxM) return DD_EINVAL;  // beyond the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return DD_ECUDA;
    void* addr = nullptr;
    {
        std::lock_guard<std::mutex> g(g_lock);
        if (!g_ready[dev]) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess || ptr == nullptr) return DD_ECUDA;
            g_addr[dev] = ptr;
            g_ready[dev] = true;
        }
        addr = g_addr[dev];
    }
    StaticScratch* s = static_cast<StaticScratch*>(addr);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // An error left pending by earlier work on this thread is the caller's: report it without
    // launching and leave it pending, so that the launch check below sees only this call's errors.
    if (cudaPeekAtLastError() != cudaSuccess) return DD_ECUDA;
    k_s_sum<<<kStaticParts, 256, 0, st>>>(T_dev, m, s);
    k_s_mu<<<1, kStaticParts, 0, st>>>(m, s);
    k_s_var<<<kStaticParts, 256, 0, st>>>(T_dev, m, s);
    k_s_sigma<<<1, kStaticParts, 0, st>>>(m, s);
    k_s_norm<<<256, 256, 0, st>>>(T_dev, m, N, s, nn2_dev);
    dim3 grid((unsigned)((N + SR - 1) / SR), (unsigned)((N + SC - 1) / SC));
    k_s_profile<<<grid, 256, 0, st>>>(N, n, s, nn2_dev);
    k_s_nan<<<64, 256, 0, st>>>(N, s, nn2_dev);
    return cudaGetLastError() == cudaSuccess ? DD_OK : DD_ECUDA;
}
