// dvm_device.cuh -- device helpers shared by the kernels: acquire/release flags, the bounded
// spin wait, vector types and the lane reduce-scatter used by the fused quadrature.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace dvm {

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Publish a progress value after a __syncthreads() of the writing CTA: a release store at GPU
// scope, cumulative over the CTA's writes that the barrier ordered before it.  (Measured slightly
// faster than an acq_rel fence followed by a relaxed store, the other PTX release pattern.)
__device__ __forceinline__ void publish_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// Bounded wait for *flag >= target.  On expiry the kernel's status word is set to
// DVM_ETIMEOUT (-4) and false is returned; a status already set by another CTA also ends it.
static __device__ bool wait_geq(const int* flag, int target, int* status, long long timeout_ns) {
    if (ld_acquire_gpu(flag) >= target) return true;
    const unsigned long long t0 = global_ns();
    // tight acquire spin (a flag normally flips within microseconds); the status word and the
    // clock are read every 64 polls, and long waits back off
    for (unsigned it = 1;; ++it) {
        if (ld_acquire_gpu(flag) >= target) return true;
        if ((it & 63u) == 0u) {
            if (ld_volatile(status) != 0) return false;
            if ((long long)(global_ns() - t0) > timeout_ns) {
                atomicCAS(status, 0, -4);
                return false;
            }
            if (it >= 4096u) __nanosleep(256);
        }
    }
}

// The same wait, returning the flag value it observed (>= target), or -1 when it gave up.  A caller
// that keeps the value can skip the next waits for targets up to it: the acquire that read it
// already ordered everything the writer published before.
static __device__ int wait_geq_value(const int* flag, int target, int* status, long long timeout_ns) {
    int v = ld_acquire_gpu(flag);
    if (v >= target) return v;
    if (!wait_geq(flag, target, status, timeout_ns)) return -1;
    return target;
}

// Sign bits of the two axes other than j of octant q, packed (lower axis first): the slot of a wall
// face store that the octant moving into a face and its mirror image in axis j share.
__device__ __forceinline__ int other_bits3(int q, int j) {
    return j == 0 ? (q >> 1) : (j == 1 ? ((q & 1) | ((q >> 1) & 2)) : (q & 3));
}

template <typename T> struct Vec4;
template <> struct Vec4<float> {
    using type = float4;
    static __device__ __forceinline__ float4 make(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
};
struct alignas(32) dbl4 { double x, y, z, w; };
template <> struct Vec4<double> {
    using type = dbl4;
    static __device__ __forceinline__ dbl4 make(double a, double b, double c, double d) { return dbl4{a, b, c, d}; }
};

__device__ __forceinline__ float bits_as(float, int v) { return __int_as_float(v); }
__device__ __forceinline__ double bits_as(double, int v) { return __longlong_as_double((long long)v); }
__device__ __forceinline__ int as_bits(float v) { return __float_as_int(v); }
__device__ __forceinline__ int as_bits(double v) { return (int)__double_as_longlong(v); }

// Sum over the 32 lanes of v[p] for NP (8 or 16) points at once.  Lane l ends up holding the
// sum of point p = l >> (5 - log2 NP).  The combination tree (lane offsets 16, 8, 4, 2, 1) is the
// same for every point, so the result does not depend on the point's slot.
template <typename T, int NP>
__device__ __forceinline__ T reduce_scatter(T (&v)[NP], int lane) {
    constexpr int LOG = (NP == 16) ? 4 : (NP == 8 ? 3 : (NP == 4 ? 2 : 1));
#pragma unroll
    for (int s = 0; s < LOG; ++s) {
        const int off = 16 >> s;
        const int cnt = NP >> s;
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int k = 0; k < cnt / 2; ++k) {
            const T send = up ? v[k] : v[k + cnt / 2];
            const T keep = up ? v[k + cnt / 2] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    T r = v[0];
#pragma unroll
    for (int off = 16 >> LOG; off >= 1; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
    return r;
}


// Packed FP32 pair arithmetic (sm_100-family f32x2 instructions): one instruction updates the two
// discrete velocities a lane carries.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// reduce_scatter for pairs of values (two moments per element): the same lane tree, each level's
// two additions done by one packed instruction.
template <int NP>
__device__ __forceinline__ float2 reduce_scatter2(float2 (&v)[NP], int lane) {
    constexpr int LOG = (NP == 16) ? 4 : (NP == 8 ? 3 : (NP == 4 ? 2 : 1));
#pragma unroll
    for (int s = 0; s < LOG; ++s) {
        const int off = 16 >> s;
        const int cnt = NP >> s;
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int k = 0; k < cnt / 2; ++k) {
            const float2 send = up ? v[k] : v[k + cnt / 2];
            const float2 keep = up ? v[k + cnt / 2] : v[k];
            const float2 recv = make_float2(__shfl_xor_sync(0xffffffffu, send.x, off), __shfl_xor_sync(0xffffffffu, send.y, off));
            v[k] = add2(keep, recv);
        }
    }
    float2 r = v[0];
#pragma unroll
    for (int off = 16 >> LOG; off >= 1; off >>= 1)
        r = add2(r, make_float2(__shfl_xor_sync(0xffffffffu, r.x, off), __shfl_xor_sync(0xffffffffu, r.y, off)));
    return r;
}

}  // namespace dvm
