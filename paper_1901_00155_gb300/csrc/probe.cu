// probe.cu -- measured arithmetic peaks of this device's CUDA cores (no counterpart in
// the paper).  They are the roofline denominators of the kernels that do not run on the
// tensor cores: the FP32 FMA rate bounds the plain FP32 distance tiles (Eq. 1 squared,
// one subtract and one FMA per element) and the diagonal recurrence, the FP64 FMA rate
// the exact rescoring.
//
// Every thread runs 8 independent FMA chains x <- x * b + c (|b| < 1, so the chains
// converge and never overflow or go subnormal); enough warps per SM cover the pipe
// latency.  The rate is FMA lane operations per second over a launch of about 20 ms,
// timed with CUDA events after a warm-up launch.
#include "dd_internal.cuh"

namespace dd {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 4;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_rate(T* out, int iters, T b, T c) {
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 8; u++) {
#pragma unroll
            for (int k = 0; k < kChains; k++) x[k] = fma(x[k], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    if (s == (T)-1.0) out[blockIdx.x & 31] = s;  // never true: keeps the chains live
}

template <typename T>
cudaError_t timed(T* out, int grid, int iters, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
    const T b = (T)0.999, c = (T)1e-3;
    k_fma_rate<T><<<grid, kProbeThreads, 0, s>>>(out, iters, b, c);  // warm-up
    cudaError_t e = cudaEventRecord(e0, s);
    if (e != cudaSuccess) return e;
    k_fma_rate<T><<<grid, kProbeThreads, 0, s>>>(out, iters, b, c);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    return e;
}

template <typename T>
cudaError_t probe(double* rate, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = sms * kProbeBlocksPerSm;
    T* out = nullptr;
    e = cudaMalloc(&out, 32 * sizeof(T));
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    int iters = 256;
    // grow the launch until it lasts about 20 ms (at most a few doublings past 2 ms)
    for (int round = 0; e == cudaSuccess && round < 24; round++) {
        e = timed<T>(out, grid, iters, s, e0, e1, &ms);
        if (e != cudaSuccess || ms >= 15.f) break;
        const double scale = ms > 0.5f ? 20.0 / ms : 8.0;
        const double next = (double)iters * scale;
        iters = next > 1e9 ? 1000000000 : (int)next;
    }
    if (e == cudaSuccess) {
        const double fmas = (double)grid * kProbeThreads * (double)iters * 8.0 * kChains;
        *rate = fmas / (ms * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return e;
}

}  // namespace
}  // namespace dd

extern "C" dd_status_t dd_probe_fma_rate(int32_t fp64, double* fma_per_s, void* stream) {
    if (!fma_per_s || (fp64 != 0 && fp64 != 1)) return DD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const cudaError_t e = fp64 ? dd::probe<double>(fma_per_s, s) : dd::probe<float>(fma_per_s, s);
    if (e == cudaSuccess) return DD_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DD_ENOMEM : DD_ECUDA;
}
