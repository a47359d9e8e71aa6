// pod_cg_gram_noalloc: the split-K Gram G = X^T Y with no device allocation at all.
//
// Some callers cannot allocate device memory when they need this product: latency-bound
// loops where cudaMalloc/cudaFree may synchronise the whole device, and host applications
// that hand out every byte of device memory themselves under a fixed budget. This entry
// point takes its scratch (one partial 8x8 tile per row split and output tile) from a
// fixed array compiled into the library instead of a caller workspace.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "common.cuh"
#include "launch.h"
#include "pod_cg.h"

namespace {

// Scratch of the allocation-free Gram: 65,536 doubles (512 KiB). Every GPU that loads the
// library holds it until the process exits. On a 152-SM GB300 every product with
// p, q <= 65 needs at most 41,472 of them.
constexpr size_t kNoAllocScratchDoubles = 65536;
static __device__ __align__(256) double g_gram_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_dev[kMaxDevices] = {nullptr};   // device address of g_gram_scratch per device

}  // namespace

extern "C" pod_cg_status pod_cg_gram_noalloc(int n, const double* X, int p, const double* Y, int q, double* G,
                                             void* cuda_stream)
{
    if (n < 1 || p < 1 || q < 1 || p > podcg::kWMax + 1 || q > podcg::kWMax + 1 || !X || !Y || !G) {
        podcg::set_last_error("pod_cg_gram_noalloc: bad arguments (need n >= 1, 1 <= p, q <= 65, non-NULL pointers)");
        return POD_CG_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        podcg::set_last_error("pod_cg_gram_noalloc: no usable current device");
        return POD_CG_ERR_CUDA;
    }
    if (cuda_stream) {
        // the scratch used is the current device's, so the stream must run on that device
        int sdev = -1;
        e = cudaStreamGetDevice((cudaStream_t)cuda_stream, &sdev);
        if (e != cudaSuccess || sdev != dev) {
            podcg::set_last_error("pod_cg_gram_noalloc: the stream does not belong to the current device (" +
                                  std::to_string(sdev) + " vs " + std::to_string(dev) + ")");
            return e != cudaSuccess ? POD_CG_ERR_CUDA : POD_CG_ERR_ARG;
        }
    }
    double* scratch = nullptr;
    {
        // once per device, with that device current: the host-side name of the array is
        // only a stand-in, so the kernel gets the device address resolved here.
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_dev[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_gram_scratch);
            if (e != cudaSuccess) {
                podcg::set_last_error(std::string("pod_cg_gram_noalloc: cudaGetSymbolAddress: ") +
                                      cudaGetErrorString(e));
                return POD_CG_ERR_CUDA;
            }
            g_scratch_dev[dev] = static_cast<double*>(ptr);
        }
        scratch = g_scratch_dev[dev];
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms < 1) {
        podcg::set_last_error("pod_cg_gram_noalloc: cannot query the SM count");
        return POD_CG_ERR_CUDA;
    }
    const size_t need = podcg::gram_workspace_bytes(n, p, q, sms);
    const size_t have = kNoAllocScratchDoubles * sizeof(double);
    if (need > have) {
        podcg::set_last_error("pod_cg_gram_noalloc: this product needs " + std::to_string(need) +
                              " bytes of scratch; the fixed scratch holds " + std::to_string(have) +
                              " bytes (use pod_cg_gram with a caller workspace)");
        return POD_CG_ERR_ARG;
    }
    // The partials are fully overwritten by each call, so nothing has to be cleared.
    e = podcg::launch_gram(n, X, n, p, Y, n, q, nullptr, G, q, 0, scratch, have, sms, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        podcg::set_last_error(std::string("pod_cg_gram_noalloc: ") + cudaGetErrorString(e));
        return POD_CG_ERR_CUDA;
    }
    return POD_CG_OK;
}
