// Phase volume without any device allocation.
//
// Some callers of this library cannot call cudaMalloc: code that runs while a
// CUDA stream is being captured into a graph (allocation calls are not
// permitted during capture), and hosts that hand the GPU a fixed memory
// budget up front and forbid allocation afterwards. For them this file
// provides oscar_phase_volume_noalloc, which sums alpha * V over the fluid
// cells of caller-owned device arrays using only a scratch array that is part
// of the library image: a file-scope static __device__ array of block
// partials plus a block counter. Every GPU that loads the library holds this
// scratch (512 KiB + 256 bytes) until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "../../include/oscar.h"
#include "oscar_internal.h"

namespace {

constexpr int kNaBlock = 256;                         // cells per block (one per thread)
constexpr int kNaMaxBlocks = 65536;                   // partials held by the scratch
constexpr long long kNaMaxCells = (long long)kNaBlock * kNaMaxBlocks;   // 16,777,216

// partials[0 .. kNaMaxBlocks) then the block counter in the next slot
static __device__ __align__(256) double g_na_scratch[kNaMaxBlocks + 32];

// device addresses of the scratch, one per device (host code cannot use the
// symbol itself: on the host it only names a stand-in, not device memory).
// Published once per device under g_na_mu; read without the lock afterwards.
// A cudaDeviceReset destroys the context that the address belongs to, so the
// entry point must not be called again in a process after a device reset.
constexpr int kNaMaxDevices = 64;
static std::atomic<double *> g_na_ptr[kNaMaxDevices];
static std::mutex g_na_mu;

__global__ void k_na_phase_volume(const double *__restrict__ alpha, const uint8_t *__restrict__ solid, int ncell,
                                  double V, double *__restrict__ scratch, double *__restrict__ out) {
    __shared__ double sh[kNaBlock / 32];
    __shared__ int last;
    unsigned *ticket = reinterpret_cast<unsigned *>(scratch + kNaMaxBlocks);
    int c = blockIdx.x * kNaBlock + threadIdx.x;
    double v = (c < ncell && !solid[c]) ? alpha[c] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kNaBlock / 32; ++w) s += sh[w];
        scratch[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // the block that finishes last sums the partials in a fixed order (each
    // thread a fixed strided subset, then a fixed shuffle and warp order), so
    // the result does not depend on which block finished last
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kNaBlock) s += __ldcg(scratch + b);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kNaBlock / 32; ++w) t += sh[w];
        *out = t * V;
        *ticket = 0u;   // the scratch keeps the last call's contents: leave the counter cleared
    }
}

}  // namespace

extern "C" int oscar_phase_volume_noalloc(const double *alpha_dev, const uint8_t *solid_dev, long long ncell,
                                          double cell_volume, double *result_dev, void *stream) {
    if (!alpha_dev || !solid_dev || !result_dev || ncell < 1) return OSCAR_E_INVALID_ARG;
    if (ncell > kNaMaxCells) return OSCAR_E_INVALID_ARG;   // beyond the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return OSCAR_E_CUDA;
    double *scratch = g_na_ptr[dev].load(std::memory_order_acquire);
    if (!scratch) {
        // one-time set-up on this device (must not run under stream capture):
        // look the scratch up, clear it and wait for the clear, so that no call
        // from any thread or stream can see an uncleared block counter
        std::lock_guard<std::mutex> lock(g_na_mu);
        scratch = g_na_ptr[dev].load(std::memory_order_acquire);
        if (!scratch) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return OSCAR_E_CUDA;
            }
            if (cudaMemsetAsync(p, 0, sizeof(g_na_scratch), (cudaStream_t)stream) != cudaSuccess ||
                cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
                cudaGetLastError();
                return OSCAR_E_CUDA;
            }
            scratch = static_cast<double *>(p);
            g_na_ptr[dev].store(scratch, std::memory_order_release);
        }
    }
    int nb = (int)((ncell + kNaBlock - 1) / kNaBlock);
    k_na_phase_volume<<<nb, kNaBlock, 0, (cudaStream_t)stream>>>(alpha_dev, solid_dev, (int)ncell, cell_volume,
                                                                 scratch, result_dev);
    return cudaGetLastError() == cudaSuccess ? 0 : OSCAR_E_CUDA;
}
