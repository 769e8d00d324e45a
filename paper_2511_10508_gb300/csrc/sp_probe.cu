// sp_probe.cu -- FP64 throughput probe: the sustained rate of independent FP64
// fused multiply-adds on this device, the ceiling that FP64 step kernels (bound
// by the FP64 pipe) are compared with besides the nominal unit count.
#include "sp_internal.h"

namespace sp {

constexpr int kProbeChains = 16, kProbeIters = 4096, kProbeThreads = 256, kProbeCtasPerSm = 8;

__global__ void __launch_bounds__(kProbeThreads) fp64_probe_kernel(double *sink, double seed, int iters) {
    double a[kProbeChains];
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) a[i] = seed + threadIdx.x + i;
    const double b = 1e-30 * seed, c = 0.999999;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) a[i] = __fma_rn(a[i], c, b);
    }
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) t += a[i];
    if (t == -1.0) sink[0] = t;  // never true: keeps the chains live
}

}  // namespace sp

extern "C" int sp_probe_fp64_rate(void *stream, double *gops) {
    if (!gops) return SP_EINVAL;
    *gops = 0.0;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SP_ECUDA;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SP_OK;
    if (cudaMalloc(&sink, sizeof(double)) != cudaSuccess) return SP_ENOMEM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = SP_ECUDA;
    const int blocks = nsm * sp::kProbeCtasPerSm;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && rc == SP_OK; ++rep) {  // the first launch warms up
        cudaEventRecord(e0, st);
        sp::fp64_probe_kernel<<<blocks, sp::kProbeThreads, 0, st>>>(sink, 1.0, sp::kProbeIters);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = SP_ECUDA;
    }
    if (rc == SP_OK && ms > 0.f) {
        const double ops = (double)blocks * sp::kProbeThreads * sp::kProbeIters * sp::kProbeChains;
        *gops = ops / (ms * 1e-3) / 1e9;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
}

extern "C" int sp_binary_version(int *version) {
    if (!version) return SP_EINVAL;
    *version = 0;
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, sp::fp64_probe_kernel) != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    *version = a.binaryVersion;
    return SP_OK;
}
