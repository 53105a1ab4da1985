// noalloc.cu -- permeability of a caller-held velocity field without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a result: code that runs
// while a CUDA stream is being captured into a graph (cudaMalloc is not a stream operation and is
// not allowed in every capture mode), code inside a framework or plugin whose caching allocator
// must own every byte of device memory, and allocation-free steady-state loops with a fixed memory
// budget.  dvm_permeability_noalloc serves them: it reduces a device array u1 to the permeability
// k = (2/sqrt(pi)) Kn G_p and G_p (the mean of u1) with a fixed-order FP64 two-stage reduction
// (block sums of 256 points, then the block sums in block order), and keeps its scratch (one FP64
// partial sum per block and a done-counter) in a file-scope device array instead of allocated
// memory.  The solver's finalize step has the same two stages with another block grouping (1024
// points per block), so the two results agree to FP64 rounding, not bit for bit.
//
// The scratch array holds kMaxBlocks block sums, so one call accepts at most
// kMaxBlocks * kBlock = 2,097,152 points (a 128^3 grid).  Every GPU that loads the library keeps
// the array until the process exits.  All calls share it: calls whose kernels may overlap on the
// GPU (different streams without ordering, or different host threads) race on it.  Each call
// clears the done-counter on its stream before its kernel runs; the partial sums are written
// before they are read, so nothing else needs clearing.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/dvm.h"

namespace {

constexpr int kBlock = 256;
constexpr int kMaxBlocks = 8192;
constexpr long long kMaxPoints = (long long)kBlock * kMaxBlocks;
constexpr int kMaxDevices = 64;

// [0, kMaxBlocks): block partial sums; element kMaxBlocks: the done-counter (as unsigned)
static __device__ __align__(256) double g_noalloc_scratch[kMaxBlocks + 32];

struct DeviceScratch {
    double* partials = nullptr;
    unsigned* counter = nullptr;
};

std::mutex g_mutex;
DeviceScratch g_addr[kMaxDevices];
thread_local std::string g_noalloc_err;

__global__ void __launch_bounds__(kBlock) permeability_noalloc_kernel(const double* __restrict__ u1, long long n,
                                                                      double kn, double* __restrict__ out,
                                                                      double* __restrict__ partials,
                                                                      unsigned* __restrict__ counter) {
    __shared__ double s_red[kBlock / 32];
    __shared__ int s_last;
    const long long id = (long long)blockIdx.x * kBlock + threadIdx.x;
    double v = (id < n) ? u1[id] : 0.0;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) tot += s_red[w];
        partials[blockIdx.x] = tot;
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        s_last = (prev == gridDim.x - 1u);
    }
    __syncthreads();
    if (!s_last) return;
    // last block: strided sums in a fixed order, then a fixed tree
    __threadfence();
    double acc = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += kBlock) acc += __ldcg(partials + k);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) tot += s_red[w];
        const double gp = tot / (double)n;
        out[0] = 2.0 / sqrt(3.14159265358979323846) * kn * gp;
        out[1] = gp;
        *counter = 0u;
    }
}

// Device addresses of the scratch array for the current device, looked up once per device.
cudaError_t scratch_for_current_device(DeviceScratch* s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev].partials) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev].partials = static_cast<double*>(p);
        g_addr[dev].counter = reinterpret_cast<unsigned*>(static_cast<double*>(p) + kMaxBlocks);
    }
    *s = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" dvm_status dvm_permeability_noalloc(const double* u1_dev, int64_t n, double kn, double* out_dev,
                                               void* stream) {
    g_noalloc_err.clear();
    if (!u1_dev || !out_dev) {
        g_noalloc_err = "dvm_permeability_noalloc: null device pointer";
        return DVM_EINVAL;
    }
    if (n < 1 || n > kMaxPoints) {
        g_noalloc_err = "dvm_permeability_noalloc: n = " + std::to_string((long long)n) +
                        " is outside 1.." + std::to_string(kMaxPoints) + " (size of the static scratch)";
        return DVM_EINVAL;
    }
    if (!(kn > 0.0) || !std::isfinite(kn)) {
        g_noalloc_err = "dvm_permeability_noalloc: Knudsen number must be positive";
        return DVM_EINVAL;
    }
    DeviceScratch s;
    cudaError_t e = scratch_for_current_device(&s);
    if (e != cudaSuccess) {
        g_noalloc_err = std::string("dvm_permeability_noalloc: scratch lookup: ") + cudaGetErrorString(e);
        return DVM_ECUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(s.counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) {
        g_noalloc_err = std::string("dvm_permeability_noalloc: ") + cudaGetErrorString(e);
        return DVM_ECUDA;
    }
    const int blocks = (int)((n + kBlock - 1) / kBlock);
    permeability_noalloc_kernel<<<blocks, kBlock, 0, st>>>(u1_dev, n, kn, out_dev, s.partials, s.counter);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_noalloc_err = std::string("dvm_permeability_noalloc: ") + cudaGetErrorString(e);
        return DVM_ECUDA;
    }
    return DVM_OK;
}

extern "C" const char* dvm_noalloc_last_error(void) { return g_noalloc_err.c_str(); }
