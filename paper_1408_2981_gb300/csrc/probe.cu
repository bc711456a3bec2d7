// FP64 FMA throughput of the current GPU, measured by a kernel of independent
// dependent-FMA chains on every SM (the denominator of the FP64-pipe roofline of
// the line relaxation and the outer operator).  The paper has no counterpart.
#include <cuda_runtime.h>

#include <algorithm>

#include "tpmg_internal.h"

namespace tpmg {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;   // independent FMA chains per thread

// Each thread runs kProbeChains chains x = x * b + c (b = 1 - 2^-20, c = 2^-30 per
// chain, values stay near 1: no overflow, no subnormals) for `iters` steps and
// writes their sum, so that no FMA can be removed.
__global__ void __launch_bounds__(kProbeThreads) k_fp64_probe(int iters, double *out)
{
    double x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = 1.0 + c * 1e-3 + threadIdx.x * 1e-9;
    const double b = 1.0 - 0x1p-20, d = 0x1p-30;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) x[c] = fma(x[c], b, d);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    out[blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace

}  // namespace tpmg

extern "C" tpmg_status tpmg_fp64_peak(void *cuda_stream, double *tflops)
{
    using namespace tpmg;
    if (!tflops) return TPMG_ERR_INVALID_ARG;
    *tflops = 0.0;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_probe, kProbeThreads, 0) != cudaSuccess)
        return TPMG_ERR_CUDA;
    const int blocks = sms * std::max(per_sm, 1);
    const int iters = 1 << 12;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    tpmg_status st = TPMG_OK;
    float best = 0.f;
    if (cudaMalloc(&out, sizeof(double) * blocks * kProbeThreads) != cudaSuccess) return TPMG_ERR_OOM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = TPMG_ERR_CUDA;
    for (int rep = 0; st == TPMG_OK && rep < 4; ++rep) {   // one warm-up, then the best of three
        k_fp64_probe<<<blocks, kProbeThreads, 0, s>>>(iters, out);
        if (cudaEventRecord(e0, s) != cudaSuccess) st = TPMG_ERR_CUDA;
        k_fp64_probe<<<blocks, kProbeThreads, 0, s>>>(iters, out);
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess)
            st = TPMG_ERR_CUDA;
        float ms = 0.f;
        if (st == TPMG_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = TPMG_ERR_CUDA;
        if (st == TPMG_OK && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (st != TPMG_OK) return st;
    if (!(best > 0.f)) return TPMG_ERR_CUDA;
    const double fma_count = (double)blocks * kProbeThreads * kProbeChains * iters;
    *tflops = 2.0 * fma_count / (best * 1e-3) / 1e12;
    return TPMG_OK;
}
