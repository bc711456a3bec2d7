// FP64 FMA throughput of the current GPU, measured by kernels of independent
// dependent-FMA chains on every SM (the denominator of the FP64-pipe roofline of
// the line relaxation and the outer operator).  The paper has no counterpart.
#include <cuda_runtime.h>

#include <algorithm>

#include "tpmg_internal.h"

namespace tpmg {

namespace {

constexpr int kProbeThreads = 256;

// Each thread runs C chains x = x * b + d (b = 1 - 2^-20, d = 2^-30, values stay near
// 1: no overflow, no subnormals) for `iters` steps and writes their sum, so that no
// FMA can be removed.
template <int C>
__global__ void __launch_bounds__(kProbeThreads) k_fp64_probe(int iters, double *out)
{
    double x[C];
#pragma unroll
    for (int c = 0; c < C; ++c) x[c] = 1.0 + c * 1e-3 + threadIdx.x * 1e-9;
    const double b = 1.0 - 0x1p-20, d = 0x1p-30;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < C; ++c) x[c] = fma(x[c], b, d);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < C; ++c) s += x[c];
    out[blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

// Best FMA rate (FMA per second) of one chain count over 1, 2, 4 and the most
// resident blocks per SM: one warm-up launch, then the best of three timed ones.
template <int C>
tpmg_status probe_chains(cudaStream_t s, int sms, double *out, cudaEvent_t e0, cudaEvent_t e1, double *best)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_probe<C>, kProbeThreads, 0) != cudaSuccess)
        return TPMG_ERR_CUDA;
    const int iters = (1 << 15) / C;   // the same FMA count per thread for every C
    for (int bps : {1, 2, 4, std::min(std::max(per_sm, 1), 32)}) {
        if (bps > per_sm) continue;
        const int blocks = sms * bps;
        for (int rep = 0; rep < 4; ++rep) {
            k_fp64_probe<C><<<blocks, kProbeThreads, 0, s>>>(iters, out);
            if (cudaEventRecord(e0, s) != cudaSuccess) return TPMG_ERR_CUDA;
            k_fp64_probe<C><<<blocks, kProbeThreads, 0, s>>>(iters, out);
            float ms = 0.f;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaGetLastError() != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                return TPMG_ERR_CUDA;
            if (rep > 0 && ms > 0.f)
                *best = std::max(*best, (double)blocks * kProbeThreads * C * iters / (ms * 1e-3));
        }
    }
    return TPMG_OK;
}

}  // namespace

}  // namespace tpmg

extern "C" tpmg_status tpmg_fp64_peak(void *cuda_stream, double *tflops)
{
    using namespace tpmg;
    if (!tflops) return TPMG_ERR_INVALID_ARG;
    *tflops = 0.0;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return TPMG_ERR_CUDA;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // one double per thread of the largest grid: 32 blocks per SM at most on this architecture
    if (cudaMalloc(&out, sizeof(double) * sms * 32 * kProbeThreads) != cudaSuccess) return TPMG_ERR_OOM;
    tpmg_status st = TPMG_OK;
    double best = 0.0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = TPMG_ERR_CUDA;
    if (st == TPMG_OK) st = probe_chains<2>(s, sms, out, e0, e1, &best);
    if (st == TPMG_OK) st = probe_chains<4>(s, sms, out, e0, e1, &best);
    if (st == TPMG_OK) st = probe_chains<8>(s, sms, out, e0, e1, &best);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (st != TPMG_OK) return st;
    if (!(best > 0.0)) return TPMG_ERR_CUDA;
    *tflops = 2.0 * best / 1e12;
    return TPMG_OK;
}
