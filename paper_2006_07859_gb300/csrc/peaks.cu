// Throughput microbenchmarks for the roofline of the pair kernels: FP32 FMA, MUFU (rsqrt) and FP64
// FMA issue rates, each from independent dependency chains on a full grid.  Loop trip counts are
// fixed, no thread waits on another.
#include <cuda_runtime.h>

#include "tpe_internal.cuh"

namespace {

__global__ void k_fp32(int iters, float seed, float *out)
{
    float a[8];
    for (int k = 0; k < 8; ++k) a[k] = seed + threadIdx.x * 1e-7f + k;
    const float m = 0.9999999f, c = 1e-7f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
    float s = 0;
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 12345.678f) out[0] = s;  // keep the work observable
}

__global__ void k_mufu(int iters, float seed, float *out)
{
    float a[8];
    for (int k = 0; k < 8; ++k) a[k] = seed + threadIdx.x * 1e-7f + k + 1.0f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = rsqrtf(a[k]);
    float s = 0;
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 12345.678f) out[0] = s;
}

__global__ void k_fp64(int iters, double seed, double *out)
{
    double a[8];
    for (int k = 0; k < 8; ++k) a[k] = seed + threadIdx.x * 1e-7 + k;
    const double m = 0.9999999, c = 1e-7;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
    double s = 0;
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 12345.678) out[0] = s;
}

template <class F>
double time_kernel(F launch)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    launch();  // warm-up
    cudaEventRecord(a);
    launch();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms * 1e-3;
}

}  // namespace

extern "C" TPE_API int tp_measure_peaks(double *fp32_flops, double *mufu_ops, double *fp64_flops)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float *fo = nullptr;
    double *dfo = nullptr;
    if (cudaMalloc(&fo, 16) != cudaSuccess) return 2;
    if (cudaMalloc(&dfo, 16) != cudaSuccess) {
        cudaFree(fo);
        return 2;
    }
    const int blocks = sms * 8, threads = 256;
    const int it32 = 1 << 16, itm = 1 << 13, it64 = 1 << 10;
    double t = time_kernel([&] { k_fp32<<<blocks, threads>>>(it32, 1.0f, fo); });
    if (fp32_flops) *fp32_flops = (double)blocks * threads * it32 * 8 * 2 / t;
    t = time_kernel([&] { k_mufu<<<blocks, threads>>>(itm, 1.0f, fo); });
    if (mufu_ops) *mufu_ops = (double)blocks * threads * itm * 8 / t;
    t = time_kernel([&] { k_fp64<<<blocks, threads>>>(it64, 1.0, dfo); });
    if (fp64_flops) *fp64_flops = (double)blocks * threads * it64 * 8 * 2 / t;
    cudaError_t e = cudaGetLastError();
    cudaFree(fo);
    cudaFree(dfo);
    return e == cudaSuccess ? 0 : 2;
}
