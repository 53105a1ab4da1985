// nn3d.cu -- kernels of the learned warm start: a small 3D convolutional network that predicts the
// initial density and velocity fields (the input of dvm_set_initial) from the solid mask, a signed
// distance and log Kn.  The paper has no such network; it only changes where the source iteration of
// Sec. 3.1 starts, never the fixed point it converges to.
//
// Tensors are single samples, channel-major: x[c][z][y][x] with D x H x W voxels (x fastest), FP32.
// Convolutions are 3 x 3 x 3 with periodic padding (the media are periodic), weights w[co][ci][27]
// (tap index (kz * 3 + ky) * 3 + kx, offsets -1..1).  The network keeps FP32 master weights and
// runs forward and backward on their BF16 roundings (see dvm_nn_adam).  The convolutions and their
// data gradients are implicit GEMMs on the fifth-generation tensor cores (conv_umma.cu: tcgen05.mma
// with BF16 operands brought in by the tensor memory accelerator, FP32 accumulators in tensor
// memory; the input activations or gradients are rounded to BF16 once, into a padded copy); the
// weight gradients are tensor-core GEMMs over the voxels as well (BF16 operands, FP32 accumulation,
// split over the voxels and summed in a fixed order); the bias gradients are FP32 channel sums.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/dvm.h"

long long conv_umma_scratch_bytes(int nin, int nout, int d, int h, int w);
cudaError_t conv_umma(const float* x, const float* w, const float* bias, float* y, int nin, int nout, int d, int h,
                      int w_, int flip, int accumulate, void* scratch, long long scratch_bytes, cudaStream_t st);
int conv_umma_status(cudaStream_t st);
long long wgrad_umma_scratch_bytes(int cin, int cout, int d, int h, int w);
cudaError_t wgrad_umma(const float* x, const float* dy, float* dw, int cin, int cout, int d, int h, int w, int accumulate,
                       void* scratch, long long scratch_bytes, cudaStream_t st);

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// db[c] (+)= sum_v dy[c][v]; one block per channel, fixed-order tree
__global__ void __launch_bounds__(kBlock) channel_sum_kernel(const float* __restrict__ dy, float* __restrict__ db,
                                                             long long V, int accumulate) {
    __shared__ float s_red[kBlock / 32];
    const float* g = dy + (long long)blockIdx.x * V;
    float a = 0.f;
    for (long long v = threadIdx.x; v < V; v += kBlock) a += g[v];
    for (int off = 16; off >= 1; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int i = 0; i < kBlock / 32; ++i) s += s_red[i];
        db[blockIdx.x] = accumulate ? db[blockIdx.x] + s : s;
    }
}

__global__ void relu_kernel(float* __restrict__ y, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = fmaxf(y[i], 0.f);
}

// dx = dy where y > 0, else 0 (in place on dy)
__global__ void relu_bwd_kernel(const float* __restrict__ y, float* __restrict__ dy, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(y[i] > 0.f)) dy[i] = 0.f;
}

// 2 x 2 x 2 average pooling: y[c][Z][Y][X] = mean of x[c][2Z..2Z+1][2Y..][2X..]
__global__ void pool_kernel(const float* __restrict__ x, float* __restrict__ y, int C, int D, int H, int W) {
    const int d = D / 2, h = H / 2, w = W / 2;
    const long long n = (long long)C * d * h * w;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int X = (int)(i % w), Y = (int)((i / w) % h), Z = (int)((i / ((long long)w * h)) % d);
    const long long c = i / ((long long)w * h * d);
    const float* xc = x + c * (long long)D * H * W;
    float s = 0.f;
    for (int a = 0; a < 2; ++a)
        for (int bb = 0; bb < 2; ++bb)
            for (int e = 0; e < 2; ++e) s += xc[((long long)(2 * Z + a) * H + 2 * Y + bb) * W + 2 * X + e];
    y[i] = 0.125f * s;
}

// gradient of the pooling: dx[c][z][y][x] (+)= dy[c][z/2][y/2][x/2] / 8
__global__ void pool_bwd_kernel(const float* __restrict__ dy, float* __restrict__ dx, int C, int D, int H, int W,
                                int accumulate) {
    const long long n = (long long)C * D * H * W;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int xx = (int)(i % W), yy = (int)((i / W) % H), zz = (int)((i / ((long long)W * H)) % D);
    const long long c = i / ((long long)W * H * D);
    const float g = 0.125f * dy[((c * (D / 2) + zz / 2) * (H / 2) + yy / 2) * (W / 2) + xx / 2];
    dx[i] = accumulate ? dx[i] + g : g;
}

// nearest-neighbour 2x upsampling: y[c][z][y][x] = x[c][z/2][y/2][x/2] (y has D x H x W voxels)
__global__ void up_kernel(const float* __restrict__ x, float* __restrict__ y, int C, int D, int H, int W) {
    const long long n = (long long)C * D * H * W;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int xx = (int)(i % W), yy = (int)((i / W) % H), zz = (int)((i / ((long long)W * H)) % D);
    const long long c = i / ((long long)W * H * D);
    y[i] = x[((c * (D / 2) + zz / 2) * (H / 2) + yy / 2) * (W / 2) + xx / 2];
}

// gradient of the upsampling: dx[c][Z][Y][X] = sum of the 8 children of dy
__global__ void up_bwd_kernel(const float* __restrict__ dy, float* __restrict__ dx, int C, int D, int H, int W) {
    const int d = D / 2, h = H / 2, w = W / 2;
    const long long n = (long long)C * d * h * w;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int X = (int)(i % w), Y = (int)((i / w) % h), Z = (int)((i / ((long long)w * h)) % d);
    const long long c = i / ((long long)w * h * d);
    const float* g = dy + c * (long long)D * H * W;
    float s = 0.f;
    for (int a = 0; a < 2; ++a)
        for (int bb = 0; bb < 2; ++bb)
            for (int e = 0; e < 2; ++e) s += g[((long long)(2 * Z + a) * H + 2 * Y + bb) * W + 2 * X + e];
    dx[i] = s;
}

// masked mean squared error over the fluid voxels: per-block partial sums of m (y - t)^2 and the
// gradient dy = 2 m (y - t) / count, where m = mask[v] for every channel
__global__ void __launch_bounds__(kBlock) mse_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                                     const float* __restrict__ mask, float* __restrict__ dy,
                                                     float* __restrict__ part, int C, long long V, float inv_count) {
    __shared__ float s_red[kBlock / 32];
    const long long n = (long long)C * V;
    const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
    float e = 0.f;
    if (i < n) {
        const float m = mask[i % V];
        const float r = m * (y[i] - t[i]);
        e = r * r;
        if (dy) dy[i] = 2.f * r * inv_count;
    }
    for (int off = 16; off >= 1; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int k = 0; k < kBlock / 32; ++k) s += s_red[k];
        part[blockIdx.x] = s;
    }
}

// Adam on FP32 master weights; wq receives the BF16 rounding (as float) used by forward and backward
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ wq, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2, float gscale) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i] * gscale;
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wq[i] = __bfloat162float(__float2bfloat16_rn(wi));
}

__global__ void round_bf16_kernel(const float* __restrict__ w, float* __restrict__ wq, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wq[i] = __bfloat162float(__float2bfloat16_rn(w[i]));
}

thread_local cudaError_t g_nn_err = cudaSuccess;

dvm_status status_of(cudaError_t e) {
    g_nn_err = e;
    return e == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

inline unsigned nblk(long long n, int b = kBlock) { return (unsigned)((n + b - 1) / b); }

}  // namespace

extern "C" {

int64_t dvm_nn_conv3d_scratch_bytes(int cin, int cout, int d, int h, int w_) {
    if (cin < 1 || cout < 1 || d < 1 || h < 1 || w_ < 1) return 0;
    const long long f = conv_umma_scratch_bytes(cin, cout, d, h, w_);     // forward: cin -> cout
    const long long g = conv_umma_scratch_bytes(cout, cin, d, h, w_);     // data gradient: cout -> cin
    return f > g ? f : g;
}

dvm_status dvm_nn_conv3d(const float* x, const float* w, const float* b, float* y, int cin, int cout, int d, int h,
                         int w_, int accumulate, void* scratch, int64_t scratch_bytes, void* stream) {
    if (!x || !w || !y || !scratch || cin < 1 || cout < 1 || d < 1 || h < 1 || w_ < 1 || w_ > 128) return DVM_EINVAL;
    if (scratch_bytes < conv_umma_scratch_bytes(cin, cout, d, h, w_)) return DVM_EINVAL;
    return status_of(conv_umma(x, w, b, y, cin, cout, d, h, w_, 0, accumulate, scratch, scratch_bytes,
                               (cudaStream_t)stream));
}

dvm_status dvm_nn_conv3d_dgrad(const float* dy, const float* w, float* dx, int cin, int cout, int d, int h, int w_,
                               int accumulate, void* scratch, int64_t scratch_bytes, void* stream) {
    if (!dy || !w || !dx || !scratch || cin < 1 || cout < 1 || d < 1 || h < 1 || w_ < 1 || w_ > 128) return DVM_EINVAL;
    // dx[ci][v] = sum_co sum_k w[co][ci][k] dy[co][v - off(k)]: a convolution of dy with the
    // transposed channel roles and mirrored taps
    if (scratch_bytes < conv_umma_scratch_bytes(cout, cin, d, h, w_)) return DVM_EINVAL;
    return status_of(conv_umma(dy, w, nullptr, dx, cout, cin, d, h, w_, 1, accumulate, scratch, scratch_bytes,
                               (cudaStream_t)stream));
}

int dvm_nn_status(void* stream) { return conv_umma_status((cudaStream_t)stream); }

dvm_status dvm_nn_conv3d_wgrad(const float* x, const float* dy, float* dw, float* db, float* scratch,
                               int64_t scratch_floats, int cin, int cout, int d, int h, int w_, int accumulate,
                               void* stream) {
    if (!x || !dy || !dw || !scratch || cin < 1 || cout < 1 || d < 1 || h < 1 || w_ < 1) return DVM_EINVAL;
    if (scratch_floats * 4 < wgrad_umma_scratch_bytes(cin, cout, d, h, w_)) return DVM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const cudaError_t e = wgrad_umma(x, dy, dw, cin, cout, d, h, w_, accumulate, scratch, scratch_floats * 4, st);
    if (e != cudaSuccess) return status_of(e);
    const long long V = (long long)d * h * w_;
    if (db) channel_sum_kernel<<<cout, kBlock, 0, st>>>(dy, db, V, accumulate);
    return status_of(cudaGetLastError());
}

int64_t dvm_nn_wgrad_scratch_floats(int cin, int cout, int d, int h, int w_) {
    if (cin < 1 || cout < 1 || d < 1 || h < 1 || w_ < 1) return 0;
    return (wgrad_umma_scratch_bytes(cin, cout, d, h, w_) + 3) / 4;
}

dvm_status dvm_nn_relu(float* y, int64_t n, void* stream) {
    if (!y || n < 0) return DVM_EINVAL;
    if (n) relu_kernel<<<nblk(n), kBlock, 0, (cudaStream_t)stream>>>(y, n);
    return status_of(cudaGetLastError());
}

dvm_status dvm_nn_relu_bwd(const float* y, float* dy, int64_t n, void* stream) {
    if (!y || !dy || n < 0) return DVM_EINVAL;
    if (n) relu_bwd_kernel<<<nblk(n), kBlock, 0, (cudaStream_t)stream>>>(y, dy, n);
    return status_of(cudaGetLastError());
}

dvm_status dvm_nn_pool2(const float* x, float* y, int c, int d, int h, int w_, void* stream) {
    if (!x || !y || (d | h | w_) & 1) return DVM_EINVAL;
    pool_kernel<<<nblk((long long)c * d * h * w_ / 8), kBlock, 0, (cudaStream_t)stream>>>(x, y, c, d, h, w_);
    return status_of(cudaGetLastError());
}

dvm_status dvm_nn_pool2_bwd(const float* dy, float* dx, int c, int d, int h, int w_, int accumulate, void* stream) {
    if (!dy || !dx || (d | h | w_) & 1) return DVM_EINVAL;
    pool_bwd_kernel<<<nblk((long long)c * d * h * w_), kBlock, 0, (cudaStream_t)stream>>>(dy, dx, c, d, h, w_, accumulate);
    return status_of(cudaGetLastError());
}

dvm_status dvm_nn_up2(const float* x, float* y, int c, int d, int h, int w_, void* stream) {
    if (!x || !y || (d | h | w_) & 1) return DVM_EINVAL;
    up_kernel<<<nblk((long long)c * d * h * w_), kBlock, 0, (cudaStream_t)stream>>>(x, y, c, d, h, w_);
    return status_of(cudaGetLastError());
}

dvm_status dvm_nn_up2_bwd(const float* dy, float* dx, int c, int d, int h, int w_, void* stream) {
    if (!dy || !dx || (d | h | w_) & 1) return DVM_EINVAL;
    up_bwd_kernel<<<nblk((long long)c * d * h * w_ / 8), kBlock, 0, (cudaStream_t)stream>>>(dy, dx, c, d, h, w_);
    return status_of(cudaGetLastError());
}

dvm_status dvm_nn_mse(const float* y, const float* t, const float* mask, float* dy, float* partial, int c, int64_t v,
                      float inv_count, void* stream) {
    if (!y || !t || !mask || !partial || c < 1 || v < 1) return DVM_EINVAL;
    mse_kernel<<<nblk((long long)c * v), kBlock, 0, (cudaStream_t)stream>>>(y, t, mask, dy, partial, c, v, inv_count);
    return status_of(cudaGetLastError());
}

int64_t dvm_nn_mse_partials(int c, int64_t v) { return (int64_t)nblk((long long)c * v); }

dvm_status dvm_nn_adam(float* w, float* wq, const float* g, float* m, float* v, int64_t n, float lr, float beta1,
                       float beta2, float eps, int64_t step, float grad_scale, void* stream) {
    if (!w || !wq || !g || !m || !v || n < 0 || step < 1) return DVM_EINVAL;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    if (n) adam_kernel<<<nblk(n), kBlock, 0, (cudaStream_t)stream>>>(w, wq, g, m, v, n, lr, beta1, beta2, eps, c1, c2, grad_scale);
    return status_of(cudaGetLastError());
}

dvm_status dvm_nn_round_bf16(const float* w, float* wq, int64_t n, void* stream) {
    if (!w || !wq || n < 0) return DVM_EINVAL;
    if (n) round_bf16_kernel<<<nblk(n), kBlock, 0, (cudaStream_t)stream>>>(w, wq, n);
    return status_of(cudaGetLastError());
}

}  // extern "C"
