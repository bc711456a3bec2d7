// Fixed device scratch for tpmg_vcycle_noalloc.
//
// The coarse-level work vectors of that entry point live in one file-scope
// device array instead of memory from cudaMalloc.  The array belongs to the
// library's device image, so every GPU that loads the library holds its
// TPMG_VCYCLE_NOALLOC_MAX_DOUBLES doubles until the process exits.
//
// In host code the array's name is only a host-side stand-in, not a device
// address: handing it to a kernel would fault (or, where the GPU can reach
// host memory, silently use the wrong memory).  Host code therefore asks the
// runtime for the real device address once per device, with that device
// current, and passes that pointer on.
#include <cuda_runtime.h>

#include <mutex>

#include "tpmg_internal.h"

namespace tpmg {

static __device__ __align__(256) double g_vcycle_scratch[TPMG_VCYCLE_NOALLOC_MAX_DOUBLES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_addr[kMaxDevices] = {};

}  // namespace

cudaError_t noalloc_scratch(int device, double **ptr)
{
    if (!ptr) return cudaErrorInvalidValue;
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return e;
    if (device != cur || device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[device]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_vcycle_scratch);
        if (e != cudaSuccess) return e;
        g_addr[device] = static_cast<double *>(p);
    }
    *ptr = g_addr[device];
    return cudaSuccess;
}

}  // namespace tpmg
