// peaks.cu -- a measurement helper, not part of the method: the FP64 fused
// multiply-add rate of the current GPU, the denominator of the roofline of
// the FP64 stage kernels (which are bound by FP64 arithmetic on a part whose
// FP64 rate is a small fraction of its FP32 rate).
//
// Every thread runs kChains independent FMA chains x <- x * m + c for a fixed
// number of iterations, enough warps per SM to hide the FMA latency; the rate
// is 2 flops per FMA over the CUDA-event time of the launch (the best of a
// few launches after a warm-up launch).
#include "nlse.h"
#include "nlse_internal.h"

namespace nlse {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kIters = 4096;

__global__ void __launch_bounds__(kThreads) fp64_fma_chains(double* out, double m, double c) {
    double x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = 1.0 + 1e-3 * (threadIdx.x + j);
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = __fma_rn(x[j], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;   // keeps the chains alive
}

}  // namespace
}  // namespace nlse

extern "C" int nlse_measure_fp64_rate(double* flops_per_s, void* stream) {
    if (!flops_per_s) return nlse::report_error(NLSE_EINVAL, "flops_per_s is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                     cudaSuccess)
        return nlse::report_error(NLSE_ECUDA, "device query failed");
    const int blocks = nsm * 8;
    double* out = nullptr;
    if (cudaMalloc((void**)&out, sizeof(double) * blocks * nlse::kThreads) != cudaSuccess)
        return nlse::report_error(NLSE_ENOMEM, "allocating the probe's output");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 0.0f;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
        cudaEventRecord(e0, st);
        nlse::fp64_fma_chains<<<blocks, nlse::kThreads, 0, st>>>(out, 0.999999999, 1e-9);
        cudaEventRecord(e1, st);
        err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaGetLastError();
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.0f || ms < best)) best = ms;      // launch 0 warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return nlse::report_error(NLSE_ECUDA, cudaGetErrorString(err));
    const double flops = 2.0 * nlse::kChains * (double)nlse::kIters * blocks * nlse::kThreads;
    *flops_per_s = flops / (best * 1e-3);
    return NLSE_OK;
}
