// gks_probe.cu -- FMA-chain throughput probe: the measured float32 / float64
// arithmetic peak that the sweep kernels are compared against.
#include <cuda_runtime.h>

#include "../../include/gks.h"

namespace {

constexpr int CHAINS = 16;  // independent FMA chains per thread (covers the pipeline latency)

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* out, int iters, T b, T c)
{
    T a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
gks_status probe(double target_ms, double* tflops)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GKS_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GKS_ECUDA;
    const int blocks = sms * 8, threads = 256;
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return GKS_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int iters = 256;
    double ms = 0.0;
    gks_status st = GKS_OK;
    for (int round = 0; round < 12; ++round) {  // grow until one launch takes target_ms
        cudaEventRecord(e0);
        k_fma_chains<T><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-7));
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = GKS_ECUDA; break; }
        float f = 0.f;
        cudaEventElapsedTime(&f, e0, e1);
        ms = f;
        if (ms >= target_ms || round == 11) break;
        iters = (int)(iters * (ms > 0.05 ? target_ms / ms * 1.05 : 8.0));
    }
    if (st == GKS_OK) {
        const double flops = 2.0 * CHAINS * (double)iters * blocks * threads;
        *tflops = flops / (ms * 1e-3) / 1e12;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return st;
}

}  // namespace

extern "C" gks_status gks_alu_peak(int precision, double target_ms, double* tflops)
{
    if (!tflops || !(target_ms > 0.0)) return GKS_EINVAL;
    return precision == GKS_FP32_FLUX ? probe<float>(target_ms, tflops) : probe<double>(target_ms, tflops);
}
