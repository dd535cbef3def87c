// FMA throughput of the CUDA cores (FP32 and FP64): the denominator of the
// roofline of arithmetic-bound kernels (the complex128 contraction on GB300,
// whose FP64 rate is far below its memory bandwidth in flops per byte).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/qt.h"

namespace {

constexpr int kChains = 8;       // independent FMA chains per thread (hides the FMA latency)
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

template <typename R>
__global__ void __launch_bounds__(kThreads) k_fma(const R* seed, R* out, int iters) {
    R a[kChains];
    const R m = seed[0], c = seed[1];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed[2] + (R)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
    }
    R s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == (R)-1.2345) out[blockIdx.x] = s;  // never true for the seeds used; keeps the chains live
}

template <typename R>
int measure(double* tflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QT_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QT_ECUDA;
    R* buf = nullptr;
    if (cudaMalloc(&buf, sizeof(R) * (3 + (size_t)sms * kBlocksPerSm)) != cudaSuccess) return QT_ENOMEM;
    const R h_seed[3] = {(R)0.999999, (R)1e-7, (R)0.5};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = QT_OK;
    const int iters = sizeof(R) == 8 ? 1 << 12 : 1 << 16;  // ~10-50 ms per launch on either pipe
    const int grid = sms * kBlocksPerSm;
    float ms = 0.f;
    if (cudaMemcpy(buf, h_seed, sizeof(h_seed), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = QT_ECUDA;
    } else {
        k_fma<R><<<grid, kThreads>>>(buf, buf + 3, iters);  // warm-up (clocks ramp)
        k_fma<R><<<grid, kThreads>>>(buf, buf + 3, iters);
        cudaEventRecord(e0);
        for (int r = 0; r < 3; ++r) k_fma<R><<<grid, kThreads>>>(buf, buf + 3, iters);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
            rc = QT_ECUDA;
    }
    if (rc == QT_OK) {
        const double flops = 3.0 * 2.0 * kChains * (double)iters * kThreads * grid;
        *tflops = flops / (ms * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    cudaGetLastError();
    return rc;
}

}  // namespace

extern "C" int qt_fma_peak(int32_t dtype, double* tflops) {
    if (!tflops || (dtype != QT_C64 && dtype != QT_C128)) return QT_EINVAL;
    return dtype == QT_C128 ? measure<double>(tflops) : measure<float>(tflops);
}
