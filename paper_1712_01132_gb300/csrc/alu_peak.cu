// alu_peak.cu -- measured FMA throughput of the device (measurement support for the sweep
// kernels' roofline, which is FP32 (or FP64) ALU issue, not a paper routine).
//
// Every thread runs eight independent FMA chains; FP32 uses the packed fma.rn.f32x2 form the sweep
// kernels use (two FMAs per instruction), FP64 plain fma.rn.f64.  The grid holds eight CTAs of 256
// threads per SM, enough warps to hide the FMA latency.  The chains' final values are stored so the
// compiler keeps them.
#include <cuda_runtime.h>

#include "../../include/dvm.h"

namespace {

__global__ void __launch_bounds__(256) fma_f32x2_kernel(float* out, int iters, float a, float b) {
    float x[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 16; k += 2) {
            asm volatile("{.reg .b64 r, m, c;\n\tmov.b64 r, {%0, %1};\n\tmov.b64 m, {%2, %2};\n\tmov.b64 c, {%3, %3};\n\t"
                         "fma.rn.f32x2 r, r, m, c;\n\tmov.b64 {%0, %1}, r;}"
                         : "+f"(x[k]), "+f"(x[k + 1])
                         : "f"(a), "f"(b));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) fma_f64_kernel(double* out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" dvm_status dvm_alu_peak(int precision, void* scratch, int64_t scratch_bytes, void* stream, double* tflops) {
    if (!tflops || !scratch || (precision != DVM_FP32 && precision != DVM_FP64)) return DVM_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DVM_ECUDA;
    const int blocks = sms * 8, threads = 256;
    const size_t need = (size_t)blocks * threads * (precision == DVM_FP32 ? sizeof(float) : sizeof(double));
    if ((size_t)scratch_bytes < need) return DVM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int iters = precision == DVM_FP32 ? 8192 : 256;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return DVM_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return DVM_ECUDA;
    }
    float ms = 0.f;
    cudaError_t e = cudaSuccess;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first launch warms up
        cudaEventRecord(e0, st);
        if (precision == DVM_FP32) fma_f32x2_kernel<<<blocks, threads, 0, st>>>((float*)scratch, iters, 0.999f, 1e-4f);
        else fma_f64_kernel<<<blocks, threads, 0, st>>>((double*)scratch, iters, 0.999, 1e-4);
        cudaEventRecord(e1, st);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || ms <= 0.f) return DVM_ECUDA;
    const double chains = precision == DVM_FP32 ? 16.0 : 8.0;   // FMAs per thread and iteration
    *tflops = 2.0 * chains * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
    return DVM_OK;
}
