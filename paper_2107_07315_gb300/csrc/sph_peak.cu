// Measured FP32 and FP64 fused multiply-add rates of the current device, the
// denominators of the pair kernels' rooflines.  Every thread runs eight
// independent FMA chains on registers (enough independent work to keep the
// pipes busy at a few resident warps per scheduler); the grid fills every SM
// several times.  Timed with CUDA events after a warm-up launch.
#include <cstdio>

#include "sph_internal.cuh"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma(T *out, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
#pragma unroll 16
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    T s = (T)0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    // a store the compiler cannot drop: the chains' result
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

template <typename T>
cudaError_t rate(int sms, int iters, double *tflops)
{
    const int blocks = sms * 8;
    T *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, sizeof(T) * (size_t)blocks * kPeakThreads);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a and b keep x bounded: x -> 0.5 x + 0.25 converges to 0.5
    k_fma<T><<<blocks, kPeakThreads>>>(buf, iters / 4, (T)0.5, (T)0.25);
    cudaEventRecord(e0);
    k_fma<T><<<blocks, kPeakThreads>>>(buf, iters, (T)0.5, (T)0.25);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms > 0.f)
        *tflops = 2.0 * kChains * (double)iters * blocks * kPeakThreads / (ms * 1e-3) / 1e12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace

extern "C" sph_status sph_peak_rates(double out[4])
{
    if (!out) return SPH_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sph::record_error("sph_peak_rates: no CUDA device");
        return SPH_ERR_NODEVICE;
    }
    out[0] = out[1] = 0.0;
    out[2] = sms;
    out[3] = 0.0;
    if (rate<float>(sms, 1 << 16, &out[0]) != cudaSuccess ||
        rate<double>(sms, 1 << 10, &out[1]) != cudaSuccess) {
        cudaGetLastError();
        sph::record_error("sph_peak_rates: microbenchmark launch failed");
        return SPH_ERR_CUDA;
    }
    return SPH_OK;
}
