// conv_umma.cu -- the warm-start network's 3 x 3 x 3 periodic convolutions as implicit GEMMs on the
// fifth-generation tensor cores (tcgen05.mma, BF16 operands, FP32 accumulators in tensor memory).
//
//   y[co][v] (+)= b[co] + sum_ci sum_k w[co][ci][k] x[ci][v + off(k)]
//
// GEMM view: M = voxels (a tile of `by` whole x rows of one z plane, at most 128 voxels, one per
// TMEM lane), N = output channels (a tile of BN), K = 27 taps x input channels (chunks of 32).
// Before the GEMM the input is written once as a BF16, channels-last copy with a one-voxel
// periodic halo, xp[z + 1][y + 1][x + 1][c] (channels padded to a multiple of 32 with zeros), and
// the weights as BF16 wb[tap][co][ci] (padded likewise): the A operand of a tap and channel chunk
// is then one box of xp (32 channels x W x by x 1) and the B operand one box of wb (32 x BN x 1),
// both brought to shared memory by the tensor memory accelerator (cp.async.bulk.tensor, 64-byte
// swizzle, the K-major layout tcgen05.mma reads).  One thread streams the boxes through a ring of
// stages, one thread issues the MMAs (K = 16 each, accumulating in TMEM) and releases a stage when
// its MMAs complete (tcgen05.commit); the four warps then read the accumulators back (tcgen05.ld,
// each warp its 32 lanes) and write y channel-major.  Every wait is bounded (a device status word
// records an expiry and the CTA returns after releasing its tensor memory).
//
// The data gradient is the same convolution of dy with the transposed channel roles and mirrored
// taps (wb[tap][ci][co] = w[co][ci][26 - tap]).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

namespace dvm_nn {

constexpr int kBM = 128;       // GEMM rows per tile (TMEM lanes)
constexpr int kBK = 32;        // input channels per K chunk: 64-byte rows
constexpr int kStages = 4;
constexpr int kThreads = 128;
constexpr long long kTimeoutNs = 2000000000LL;

struct ConvGeom {
    int cin, cout;        // channels of this convolution's input and output
    int D, H, W;
    int cinp, coutp;      // padded to multiples of kBK and of BN
    int by, ytiles;       // x rows per tile, tiles per z plane
    int nk;               // K chunks per tap
    int accumulate;
};

__device__ int g_conv_status;   // nonzero after a bounded wait expired

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bounded wait for the phase with the given parity to complete; false on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    const unsigned a = smem_u32(bar);
    unsigned long long t0 = 0;
    for (unsigned it = 0;; ++it) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
        if ((it & 255u) == 0u) {
            const unsigned long long t = gtime();
            if (it == 0) t0 = t;
            else if ((long long)(t - t0) > kTimeoutNs) return false;
            if (*reinterpret_cast<volatile int*>(&g_conv_status) != 0 && it > 0) return false;
        }
    }
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5}], [%6];"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
                   "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2),
                   "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar) {
    asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
                   "r"(smem_u32(bar))
                 : "memory");
}

// shared-memory matrix descriptor of a K-major operand in the 64-byte swizzled layout: rows of 64
// bytes, eight-row groups 512 bytes apart (stride byte offset), descriptor version 1
__device__ __forceinline__ uint64_t smem_desc_sw64(const void* p) {
    const uint64_t addr = (smem_u32(p) >> 4) & 0x3FFFu;
    return addr | (1ull << 16) | ((uint64_t)(512 >> 4) << 32) | (1ull << 46) | (4ull << 61);
}

// instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M = 128, N = BN
template <int BN>
__device__ __forceinline__ unsigned idesc_bf16() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(BN >> 3) << 17) | ((unsigned)(kBM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(unsigned tmem_d, uint64_t adesc, uint64_t bdesc, unsigned idesc, int acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
                 : "memory");
}

// the mbarrier completes one phase when every MMA this thread issued so far has finished
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// MT row tiles per CTA share every B box and write MT accumulators (TMEM columns t BN .. t BN + BN - 1)
template <int BN, int MT>
__global__ void __launch_bounds__(kThreads) conv3d_umma_kernel(const __grid_constant__ CUtensorMap tmA,
                                                               const __grid_constant__ CUtensorMap tmB,
                                                               const float* __restrict__ bias, float* __restrict__ y,
                                                               const ConvGeom g) {
    constexpr int kABytes = kBM * kBK * 2;            // 8 KB per row tile
    constexpr int kBBytes = BN * kBK * 2;
    constexpr int kStageBytes = MT * kABytes + kBBytes;   // a multiple of 1024 (BN multiple of 16)
    constexpr unsigned kTmemCols = MT * BN <= 32 ? 32u : (MT * BN <= 64 ? 64u : (MT * BN <= 128 ? 128u : 256u));
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sbase = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
    __shared__ unsigned s_tmem;
    __shared__ int s_fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.y * BN;
    const int rows = g.by * g.W;                      // valid GEMM rows of a tile (<= 128)
    int tz[MT], ty0[MT];                              // row tile t: z plane and first y row
#pragma unroll
    for (int t = 0; t < MT; ++t) {
        const int tile = blockIdx.x * MT + t;         // beyond the grid: z >= D, never written
        tz[t] = tile / g.ytiles;
        ty0[t] = (tile - tz[t] * g.ytiles) * g.by;
    }

    if (rows < kBM) {   // rows beyond the boxes stay zero in every stage (the boxes never write them)
        for (int i = threadIdx.x * 16; i < kStages * kStageBytes; i += kThreads * 16)
            *reinterpret_cast<uint4*>(sbase + i) = make_uint4(0u, 0u, 0u, 0u);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // before the tensor cores read them
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem_d = s_tmem;
    const int niter = 27 * g.nk;
    const unsigned box_bytes = (unsigned)(MT * kBK * 2 * g.W * g.by + kBBytes);

    if (warp == 0 && lane == 0) {
        // producer: the A box of (tap, chunk) and the B box of the same (tap, chunk) per stage
        for (int i = 0; i < niter; ++i) {
            const int s = i % kStages;
            if (i >= kStages && !mbar_wait(&empty[s], ((i / kStages) - 1) & 1)) {
                s_fail = 1;
                break;
            }
            const int tap = i / g.nk, kc = i - tap * g.nk;
            const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
            unsigned char* st = sbase + (size_t)s * kStageBytes;
            mbar_expect_tx(&full[s], box_bytes);
#pragma unroll
            for (int t = 0; t < MT; ++t)
                tma_load_4d(st + t * kABytes, &tmA, kc * kBK, 1 + dx, ty0[t] + 1 + dy, tz[t] + 1 + dz, &full[s]);
            tma_load_3d(st + MT * kABytes, &tmB, kc * kBK, n0, tap, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: K = 16 per instruction, two per chunk; the first one overwrites the accumulator
        const unsigned idesc = idesc_bf16<BN>();
        for (int i = 0; i < niter; ++i) {
            const int s = i % kStages;
            if (!mbar_wait(&full[s], (i / kStages) & 1)) {
                s_fail = 1;
                break;
            }
            tc_fence_after();
            const unsigned char* st = sbase + (size_t)s * kStageBytes;
            const uint64_t bd = smem_desc_sw64(st + MT * kABytes);
#pragma unroll
            for (int t = 0; t < MT; ++t) {
                const uint64_t ad = smem_desc_sw64(st + t * kABytes);
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk)    // 32 bytes of K per step: +2 in the 16-byte address field
                    umma_bf16(tmem_d + t * BN, ad + 2 * kk, bd + 2 * kk, idesc, (i > 0 || kk > 0) ? 1 : 0);
            }
            umma_commit(&empty[s]);
        }
        umma_commit(&done);
    }
    __syncwarp();
    const bool ok = mbar_wait(&done, 0);
    tc_fence_after();
    if (!ok || s_fail) {
        if (threadIdx.x == 0) atomicCAS(&g_conv_status, 0, -4);
    } else {
        // accumulator row r of tile t = voxel r of the tile (TMEM lane r), column t BN + j = output
        // channel n0 + j
        const int r = warp * 32 + lane;
        const long long V = (long long)g.D * g.H * g.W;
#pragma unroll
        for (int t = 0; t < MT; ++t) {
        const int yy = ty0[t] + r / g.W, xx = r % g.W;
        const bool valid = r < rows && yy < g.H && tz[t] < g.D;
        const long long v = ((long long)tz[t] * g.H + yy) * g.W + xx;
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            unsigned a[16];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                         "%13, %14, %15}, [%16];"
                         : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]),
                           "=r"(a[7]), "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]),
                           "=r"(a[14]), "=r"(a[15])
                         : "r"(tmem_d + ((unsigned)(32 * warp) << 16) + (unsigned)(t * BN + c0))
                         : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (valid) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int co = n0 + c0 + j;
                    if (co < g.cout) {
                        const float val = __uint_as_float(a[j]) + (bias ? bias[co] : 0.f);
                        float* d = y + (long long)co * V + v;
                        *d = g.accumulate ? *d + val : val;
                    }
                }
            }
        }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_d), "r"(kTmemCols) : "memory");
}

// The same convolution with the A operand shared by the three y taps: when a tile is whole x rows
// (W a multiple of 8 dividing 128, by = 128 / W rows) and a CTA's MT tiles are consecutive rows of
// one z plane, one box of MT by + 2 rows (the tiles' rows and a halo row on each side) per (dz, dx,
// channel chunk) holds the A rows of all three dy taps: tap dy of tile t starts (t by + dy + 1) W
// rows into the box, a multiple of eight 64-byte rows, so it is a plain shift of the swizzled
// operand's start address.  A stage is that box and the three dy taps' B boxes: 9 stages per chunk
// instead of 27, and a third of the A bytes per tap.
template <int BN, int MT, int NST>
__global__ void __launch_bounds__(kThreads) conv3d_umma_dy_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                  const __grid_constant__ CUtensorMap tmB,
                                                                  const float* __restrict__ bias, float* __restrict__ y,
                                                                  const ConvGeom g, int abox_bytes, int stage_bytes) {
    constexpr int kBBytes = BN * kBK * 2;
    constexpr unsigned kTmemCols = MT * BN <= 32 ? 32u : (MT * BN <= 64 ? 64u : (MT * BN <= 128 ? 128u : 256u));
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sbase = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[NST], empty[NST], done;
    __shared__ unsigned s_tmem;
    __shared__ int s_fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.y * BN;
    const int tile0 = blockIdx.x * MT;                // first tile: z plane, first y row
    const int z = tile0 / g.ytiles;
    const int yb = (tile0 - z * g.ytiles) * g.by;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem_d = s_tmem;
    const int niter = 9 * g.nk;                       // (dz, dx) x channel chunks
    const unsigned box_bytes = (unsigned)(abox_bytes + 3 * kBBytes);

    if (warp == 0 && lane == 0) {
        // producer: the A box of (dz, dx, chunk) and the B boxes of its three dy taps per stage
        for (int i = 0; i < niter; ++i) {
            const int s = i % NST;
            if (i >= NST && !mbar_wait(&empty[s], ((i / NST) - 1) & 1)) {
                s_fail = 1;
                break;
            }
            const int zx = i / g.nk, kc = i - zx * g.nk;
            const int dz = zx / 3 - 1, dx = zx % 3 - 1;
            unsigned char* st = sbase + (size_t)s * stage_bytes;
            mbar_expect_tx(&full[s], box_bytes);
            tma_load_4d(st, &tmA, kc * kBK, 1 + dx, yb, z + 1 + dz, &full[s]);   // padded rows yb .. yb + MT by + 1
#pragma unroll
            for (int j = 0; j < 3; ++j)
                tma_load_3d(st + abox_bytes + j * kBBytes, &tmB, kc * kBK, n0, (dz + 1) * 9 + j * 3 + (dx + 1), &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: per stage, for each dy tap and row tile two K = 16 steps
        const unsigned idesc = idesc_bf16<BN>();
        for (int i = 0; i < niter; ++i) {
            const int s = i % NST;
            if (!mbar_wait(&full[s], (i / NST) & 1)) {
                s_fail = 1;
                break;
            }
            tc_fence_after();
            const unsigned char* st = sbase + (size_t)s * stage_bytes;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const uint64_t bd = smem_desc_sw64(st + abox_bytes + j * kBBytes);
#pragma unroll
                for (int t = 0; t < MT; ++t) {
                    const uint64_t ad = smem_desc_sw64(st + (size_t)((t * g.by + j) * g.W) * (kBK * 2));
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk)
                        umma_bf16(tmem_d + t * BN, ad + 2 * kk, bd + 2 * kk, idesc, (i > 0 || j > 0 || kk > 0) ? 1 : 0);
                }
            }
            umma_commit(&empty[s]);
        }
        umma_commit(&done);
    }
    __syncwarp();
    const bool ok = mbar_wait(&done, 0);
    tc_fence_after();
    if (!ok || s_fail) {
        if (threadIdx.x == 0) atomicCAS(&g_conv_status, 0, -4);
    } else {
        // accumulator row r of tile t = voxel r of the tile (TMEM lane r), column t BN + j = output
        // channel n0 + j; every row of every tile is a voxel (by W = 128, whole tiles)
        const int r = warp * 32 + lane;
        const long long V = (long long)g.D * g.H * g.W;
#pragma unroll
        for (int t = 0; t < MT; ++t) {
            const int yy = yb + t * g.by + r / g.W, xx = r % g.W;
            const long long v = ((long long)z * g.H + yy) * g.W + xx;
#pragma unroll
            for (int c0 = 0; c0 < BN; c0 += 16) {
                unsigned a[16];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                             "%13, %14, %15}, [%16];"
                             : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]),
                               "=r"(a[7]), "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]),
                               "=r"(a[14]), "=r"(a[15])
                             : "r"(tmem_d + ((unsigned)(32 * warp) << 16) + (unsigned)(t * BN + c0))
                             : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (yy < g.H) {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        const int co = n0 + c0 + jj;
                        if (co < g.cout) {
                            const float val = __uint_as_float(a[jj]) + (bias ? bias[co] : 0.f);
                            float* d = y + (long long)co * V + v;
                            *d = g.accumulate ? *d + val : val;
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_d), "r"(kTmemCols) : "memory");
}

// xp[pz][py][px][c] = bf16(x[c][pz - 1][py - 1][px - 1]) with periodic wrap, zero for c >= cin.  A
// block transposes 32 padded voxels of one x row by 32 channels through shared memory, so that both
// the channel-major reads and the channels-last writes are coalesced.
__global__ void __launch_bounds__(256) pad_bf16_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ xp,
                                                       int cin, int cinp, int D, int H, int W) {
    __shared__ float t[32][33];
    const int px0 = blockIdx.x * 32;
    const int prow = blockIdx.y;                        // padded (pz, py)
    const int py = prow % (H + 2), pz = prow / (H + 2);
    const int c0 = blockIdx.z * 32;
    const int sy = py == 0 ? H - 1 : (py == H + 1 ? 0 : py - 1);
    const int sz = pz == 0 ? D - 1 : (pz == D + 1 ? 0 : pz - 1);
    const long long V = (long long)D * H * W;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    {
        const int px = px0 + tx;
        const int sx = px == 0 ? W - 1 : (px == W + 1 ? 0 : px - 1);
        for (int cc = ty; cc < 32; cc += 8) {
            const int c = c0 + cc;
            t[cc][tx] = (c < cin && px < W + 2) ? x[(long long)c * V + ((long long)sz * H + sy) * W + sx] : 0.f;
        }
    }
    __syncthreads();
    for (int vv = ty; vv < 32; vv += 8) {
        const int px = px0 + vv;
        if (px < W + 2)
            xp[(((long long)pz * (H + 2) + py) * (W + 2) + px) * cinp + c0 + tx] = __float2bfloat16_rn(t[tx][vv]);
    }
}

// wb[tap][n][c] = bf16(w[n sn + c sc + (flip ? 26 - tap : tap)]) for n < nout, c < nin, else 0
__global__ void weights_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int nout, int nin,
                                    int noutp, int ninp, int sn, int sc, int flip) {
    const long long total = 27LL * noutp * ninp;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int c = (int)(i % ninp);
    const int n = (int)((i / ninp) % noutp);
    const int tap = (int)(i / ((long long)ninp * noutp));
    float val = 0.f;
    if (n < nout && c < nin) val = w[(long long)n * sn + (long long)c * sc + (flip ? 26 - tap : tap)];
    wb[i] = __float2bfloat16_rn(val);
}

using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    });
    return fn;
}

inline int bn_for(int cout) { return cout <= 32 ? 32 : (cout <= 64 ? 64 : 128); }
inline long long align1k(long long b) { return (b + 1023) & ~1023LL; }

template <int BN, int MT>
cudaError_t launch_bn(const CUtensorMap& ta, const CUtensorMap& tb, const float* bias, float* y, const ConvGeom& g,
                      cudaStream_t st) {
    constexpr int kStageBytes = MT * kBM * kBK * 2 + BN * kBK * 2;
    const int smem = kStages * kStageBytes + 1024;
    auto kern = conv3d_umma_kernel<BN, MT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int tiles = g.D * g.ytiles;
    dim3 grid((unsigned)((tiles + MT - 1) / MT), (unsigned)(g.coutp / BN));
    kern<<<grid, kThreads, smem, st>>>(ta, tb, bias, y, g);
    return cudaGetLastError();
}

template <int BN, int MT, int NST>
cudaError_t launch_dy(const CUtensorMap& ta, const CUtensorMap& tb, const float* bias, float* y, const ConvGeom& g,
                      cudaStream_t st) {
    const int abox = (MT * g.by + 2) * g.W * kBK * 2;
    const int stage = (abox + 3 * BN * kBK * 2 + 1023) / 1024 * 1024;
    const int smem = NST * stage + 1024;
    auto kern = conv3d_umma_dy_kernel<BN, MT, NST>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(g.D * g.ytiles / MT), (unsigned)(g.coutp / BN));
    kern<<<grid, kThreads, smem, st>>>(ta, tb, bias, y, g, abox, stage);
    return cudaGetLastError();
}

}  // namespace dvm_nn

// Scratch bytes of one convolution with nin input and nout output channels on a d x h x w grid: the
// padded BF16 input copy and the BF16 weights, each 1 KB aligned.
long long conv_umma_scratch_bytes(int nin, int nout, int d, int h, int w) {
    using namespace dvm_nn;
    const int cinp = (nin + kBK - 1) / kBK * kBK;
    const int bn = bn_for(nout);
    const int coutp = (nout + bn - 1) / bn * bn;
    return align1k((long long)(d + 2) * (h + 2) * (w + 2) * cinp * 2) + align1k(27LL * coutp * cinp * 2) + 1024;
}

// One convolution (flip = 0: y = conv(x, w) + b with w[nout][nin][27]; flip = 1: the data gradient,
// nout = the forward input channels, w[nin][nout][27] read with mirrored taps).  Returns a CUDA error,
// cudaErrorInvalidValue for a grid wider than 128 voxels, or cudaErrorNotSupported when the driver
// lacks the tensor-map encoder.
cudaError_t conv_umma(const float* x, const float* w, const float* bias, float* y, int nin, int nout, int d, int h,
                      int w_, int flip, int accumulate, void* scratch, long long scratch_bytes, cudaStream_t st) {
    using namespace dvm_nn;
    if (w_ > kBM || scratch_bytes < conv_umma_scratch_bytes(nin, nout, d, h, w_)) return cudaErrorInvalidValue;
    EncodeFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    ConvGeom g;
    g.cin = nin;
    g.cout = nout;
    g.D = d;
    g.H = h;
    g.W = w_;
    g.cinp = (nin + kBK - 1) / kBK * kBK;
    const int bn = bn_for(nout);
    g.coutp = (nout + bn - 1) / bn * bn;
    g.by = kBM / w_ < h ? kBM / w_ : h;
    g.ytiles = (h + g.by - 1) / g.by;
    g.nk = g.cinp / kBK;
    g.accumulate = accumulate;
    const uintptr_t base = (reinterpret_cast<uintptr_t>(scratch) + 1023) & ~uintptr_t(1023);
    __nv_bfloat16* xp = reinterpret_cast<__nv_bfloat16*>(base);
    __nv_bfloat16* wb =
        reinterpret_cast<__nv_bfloat16*>(base + align1k((long long)(d + 2) * (h + 2) * (w_ + 2) * g.cinp * 2));
    pad_bf16_kernel<<<dim3((unsigned)((w_ + 2 + 31) / 32), (unsigned)((d + 2) * (h + 2)), (unsigned)(g.cinp / 32)), 256, 0,
                      st>>>(x, xp, nin, g.cinp, d, h, w_);
    const int sn = flip ? 27 : nin * 27;     // forward: w[n][c][k]; gradient: w[c][n][26 - k]
    const int sc = flip ? nout * 27 : 27;
    weights_bf16_kernel<<<(unsigned)((27LL * g.coutp * g.cinp + 255) / 256), 256, 0, st>>>(w, wb, nout, nin, g.coutp,
                                                                                          g.cinp, sn, sc, flip);
    CUtensorMap ta, tb;
    {
        const cuuint64_t dims[4] = {(cuuint64_t)g.cinp, (cuuint64_t)(w_ + 2), (cuuint64_t)(h + 2), (cuuint64_t)(d + 2)};
        const cuuint64_t strides[3] = {(cuuint64_t)g.cinp * 2, (cuuint64_t)g.cinp * 2 * (w_ + 2),
                                       (cuuint64_t)g.cinp * 2 * (w_ + 2) * (h + 2)};
        const cuuint32_t box[4] = {(cuuint32_t)kBK, (cuuint32_t)w_, (cuuint32_t)g.by, 1u};
        const cuuint32_t es[4] = {1u, 1u, 1u, 1u};
        if (enc(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, xp, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const cuuint64_t dims[3] = {(cuuint64_t)g.cinp, (cuuint64_t)g.coutp, 27u};
        const cuuint64_t strides[2] = {(cuuint64_t)g.cinp * 2, (cuuint64_t)g.cinp * 2 * g.coutp};
        const cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)bn, 1u};
        const cuuint32_t es[3] = {1u, 1u, 1u};
        if (enc(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, wb, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    // whole-row tiles of 128 voxels, two per CTA in one z plane: the A box shared by the dy taps
    const int mt = bn == 128 ? 1 : 2;
    if (w_ % 8 == 0 && kBM % w_ == 0 && g.by * w_ == kBM && h % g.by == 0 && g.ytiles % mt == 0) {
        CUtensorMap td;
        const cuuint64_t dims[4] = {(cuuint64_t)g.cinp, (cuuint64_t)(w_ + 2), (cuuint64_t)(h + 2), (cuuint64_t)(d + 2)};
        const cuuint64_t strides[3] = {(cuuint64_t)g.cinp * 2, (cuuint64_t)g.cinp * 2 * (w_ + 2),
                                       (cuuint64_t)g.cinp * 2 * (w_ + 2) * (h + 2)};
        const cuuint32_t box[4] = {(cuuint32_t)kBK, (cuuint32_t)w_, (cuuint32_t)(mt * g.by + 2), 1u};
        const cuuint32_t es[4] = {1u, 1u, 1u, 1u};
        if (enc(&td, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, xp, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        if (bn == 32) return launch_dy<32, 2, 3>(td, tb, bias, y, g, st);
        if (bn == 64) return launch_dy<64, 2, 3>(td, tb, bias, y, g, st);
        return launch_dy<128, 1, 3>(td, tb, bias, y, g, st);
    }
    if (bn == 32) return launch_bn<32, 2>(ta, tb, bias, y, g, st);
    if (bn == 64) return launch_bn<64, 2>(ta, tb, bias, y, g, st);
    return launch_bn<128, 1>(ta, tb, bias, y, g, st);
}

namespace dvm_nn {

// ---------------------------------------------------------------------------- weight gradients
//
//   dw[co][ci][k] (+)= sum_v dy[co][v] x[ci][v + off(k)]
//
// GEMM view: M = (tap, input channel) rows in sub-blocks of 32 (sub-block sb = tap * cinp / 32 +
// channel chunk, four per 128-row tile), N = output channels (BN), K = voxels (chunks of 32 along
// x of one (z, y) row; x padded to a multiple of 32 with zeros).  The A rows of a sub-block are x
// shifted by the tap's offset: three BF16 copies of x (one per x offset dx = -1, 0, 1, already
// shifted along x, with a periodic one-row halo in y and z) make every box start at an x that is a
// multiple of 32; B is a BF16 copy of dy.  Every CTA sums its own range of K chunks (split K) into a
// partial [32 sb rows][coutp] block per sub-block; a second kernel adds the partials of the splits
// in split order (deterministic) into dw.

struct WgradGeom {
    int cin, cout, D, H, W, Wp;      // Wp: x extent padded to a multiple of 32
    int cinp, coutp;
    int nsb;                         // sub-blocks = 27 * cinp / 32
    int nchunks, chunks_per_split;   // K chunks (D * H * Wp / 32) and chunks per CTA
};

template <int BN>
__global__ void __launch_bounds__(kThreads) wgrad_umma_kernel(const __grid_constant__ CUtensorMap tmX,
                                                              const __grid_constant__ CUtensorMap tmG,
                                                              float* __restrict__ part, const WgradGeom g) {
    constexpr int kABytes = kBM * kBK * 2;            // four 32-row sub-blocks of 64-byte rows
    constexpr int kBBytes = BN * kBK * 2;
    constexpr int kStageBytes = kABytes + kBBytes;
    constexpr unsigned kTmemCols = BN < 32 ? 32u : (unsigned)BN;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sbase = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
    __shared__ unsigned s_tmem;
    __shared__ int s_fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = blockIdx.x, n0 = blockIdx.y * BN, split = blockIdx.z;
    const int c_begin = split * g.chunks_per_split;
    const int c_end = min(g.nchunks, c_begin + g.chunks_per_split);
    const int nsub = min(4, g.nsb - mt * 4);          // sub-blocks of this tile
    const int ncc = g.cinp / 32;
    const int xchunks = g.Wp / 32;

    if (nsub < 4) {   // rows of missing sub-blocks stay zero (their boxes are never loaded)
        for (int i = threadIdx.x * 16; i < kStages * kStageBytes; i += kThreads * 16)
            *reinterpret_cast<uint4*>(sbase + i) = make_uint4(0u, 0u, 0u, 0u);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem_d = s_tmem;
    const int niter = c_end - c_begin;
    const unsigned box_bytes = (unsigned)(nsub * 32 * kBK * 2 + kBBytes);

    if (warp == 0 && lane == 0) {
        for (int i = 0; i < niter; ++i) {
            const int s = i % kStages;
            if (i >= kStages && !mbar_wait(&empty[s], ((i / kStages) - 1) & 1)) {
                s_fail = 1;
                break;
            }
            const int ch = c_begin + i;                 // K chunk: 32 voxels of the (z, y) row
            const int x0 = (ch % xchunks) * 32;
            const int row = ch / xchunks;
            const int y = row % g.H, z = row / g.H;
            unsigned char* st = sbase + (size_t)s * kStageBytes;
            mbar_expect_tx(&full[s], box_bytes);
            for (int j = 0; j < nsub; ++j) {
                const int sb = mt * 4 + j;
                const int tap = sb / ncc, cc = sb - tap * ncc;
                const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                tma_load_5d(st + j * 32 * kBK * 2, &tmX, x0, y + 1 + dy, z + 1 + dz, cc * 32, dx + 1, &full[s]);
            }
            tma_load_4d(st + kABytes, &tmG, x0, y, z, n0, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        const unsigned idesc = idesc_bf16<BN>();
        for (int i = 0; i < niter; ++i) {
            const int s = i % kStages;
            if (!mbar_wait(&full[s], (i / kStages) & 1)) {
                s_fail = 1;
                break;
            }
            tc_fence_after();
            const unsigned char* st = sbase + (size_t)s * kStageBytes;
            const uint64_t ad = smem_desc_sw64(st), bd = smem_desc_sw64(st + kABytes);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)
                umma_bf16(tmem_d, ad + 2 * kk, bd + 2 * kk, idesc, (i > 0 || kk > 0) ? 1 : 0);
            umma_commit(&empty[s]);
        }
        umma_commit(&done);
    }
    __syncwarp();
    const bool ok = mbar_wait(&done, 0);
    tc_fence_after();
    if (!ok || s_fail) {
        if (threadIdx.x == 0) atomicCAS(&g_conv_status, 0, -4);
    } else {
        // accumulator row r = (sub-block mt * 4 + r / 32, row r % 32), column j = output channel n0 + j
        const int r = warp * 32 + lane;
        const int sb = mt * 4 + r / 32;
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            unsigned a[16];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                         "%13, %14, %15}, [%16];"
                         : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]),
                           "=r"(a[7]), "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]),
                           "=r"(a[14]), "=r"(a[15])
                         : "r"(tmem_d + ((unsigned)(32 * warp) << 16) + (unsigned)c0)
                         : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (sb < g.nsb) {
                float* d = part + (((size_t)split * g.nsb + sb) * 32 + (r & 31)) * g.coutp + n0 + c0;
#pragma unroll
                for (int j = 0; j < 16; ++j) d[j] = niter > 0 ? __uint_as_float(a[j]) : 0.f;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_d), "r"(kTmemCols) : "memory");
}

// xs[dx + 1][c][pz][py][x] = bf16(x[c][pz - 1][py - 1][x + dx]) (periodic in every axis), zero for
// c >= cin or x >= W; one warp per (dx, c, pz, py) row, lanes along x
__global__ void __launch_bounds__(256) shift_bf16_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ xs,
                                                         int cin, int cinp, int D, int H, int W, int Wp) {
    const long long nrows = 3LL * cinp * (D + 2) * (H + 2);
    const long long row = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= nrows) return;
    const int lane = threadIdx.x & 31;
    const int py = (int)(row % (H + 2));
    const long long r2 = row / (H + 2);
    const int pz = (int)(r2 % (D + 2));
    const long long r3 = r2 / (D + 2);
    const int c = (int)(r3 % cinp);
    const int dx = (int)(r3 / cinp) - 1;
    const int sy = py == 0 ? H - 1 : (py == H + 1 ? 0 : py - 1);
    const int sz = pz == 0 ? D - 1 : (pz == D + 1 ? 0 : pz - 1);
    const float* src = x + (long long)c * D * H * W + ((long long)sz * H + sy) * W;
    __nv_bfloat16* dst = xs + row * Wp;
    for (int xx = lane; xx < Wp; xx += 32) {
        float val = 0.f;
        if (c < cin && xx < W) {
            int sx = xx + dx;
            sx = sx < 0 ? sx + W : (sx >= W ? sx - W : sx);
            val = src[sx];
        }
        dst[xx] = __float2bfloat16_rn(val);
    }
}

// gb[co][z][y][x] = bf16(dy[co][z][y][x]), zero for co >= cout or x >= W
__global__ void grad_bf16_kernel(const float* __restrict__ dy, __nv_bfloat16* __restrict__ gb, int cout, int coutp,
                                 int D, int H, int W, int Wp) {
    const long long total = (long long)coutp * D * H * Wp;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int xx = (int)(i % Wp);
    const long long rest = i / Wp;                      // (co, z, y)
    const long long row = rest % ((long long)D * H);
    const int co = (int)(rest / ((long long)D * H));
    float val = 0.f;
    if (co < cout && xx < W) val = dy[(long long)co * D * H * W + row * W + xx];
    gb[i] = __float2bfloat16_rn(val);
}

// dw[co][ci][k] (+)= sum over splits, in split order, of part[split][sb(k, ci)][ci % 32][co]
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, float* __restrict__ dw, int cin, int cout,
                                    int cinp, int coutp, int nsb, int nsplit, int accumulate) {
    const long long total = (long long)cout * cin * 27;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int k = (int)(i % 27);
    const int ci = (int)((i / 27) % cin);
    const int co = (int)(i / (27LL * cin));
    const int sb = k * (cinp / 32) + ci / 32;
    const size_t off = ((size_t)sb * 32 + (ci & 31)) * coutp + co;
    const size_t stride = (size_t)nsb * 32 * coutp;
    float s = 0.f;
    for (int sp = 0; sp < nsplit; ++sp) s += part[off + (size_t)sp * stride];
    dw[i] = accumulate ? dw[i] + s : s;
}

constexpr int kWgradChunksPerSplit = 64;   // 2048 voxels of K per CTA

template <int BN>
cudaError_t launch_wgrad_bn(const CUtensorMap& tx, const CUtensorMap& tg, float* part, const WgradGeom& g,
                            int nsplit, cudaStream_t st) {
    constexpr int kStageBytes = kBM * kBK * 2 + BN * kBK * 2;
    const int smem = kStages * kStageBytes + 1024;
    auto kern = wgrad_umma_kernel<BN>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g.nsb + 3) / 4), (unsigned)(g.coutp / BN), (unsigned)nsplit);
    kern<<<grid, kThreads, smem, st>>>(tx, tg, part, g);
    return cudaGetLastError();
}

WgradGeom wgrad_geom(int cin, int cout, int d, int h, int w) {
    WgradGeom g;
    g.cin = cin;
    g.cout = cout;
    g.D = d;
    g.H = h;
    g.W = w;
    g.Wp = (w + 31) / 32 * 32;
    g.cinp = (cin + 31) / 32 * 32;
    const int bn = bn_for(cout);
    g.coutp = (cout + bn - 1) / bn * bn;
    g.nsb = 27 * g.cinp / 32;
    g.nchunks = d * h * (g.Wp / 32);
    g.chunks_per_split = kWgradChunksPerSplit;
    return g;
}

}  // namespace dvm_nn

// Scratch bytes of one weight gradient: the three shifted BF16 copies of x, the BF16 copy of dy and
// the split partials, each 1 KB aligned.
long long wgrad_umma_scratch_bytes(int cin, int cout, int d, int h, int w) {
    using namespace dvm_nn;
    const WgradGeom g = wgrad_geom(cin, cout, d, h, w);
    const long long nsplit = (g.nchunks + g.chunks_per_split - 1) / g.chunks_per_split;
    return align1k(3LL * g.cinp * (d + 2) * (h + 2) * g.Wp * 2) + align1k((long long)g.coutp * d * h * g.Wp * 2) +
           align1k(nsplit * g.nsb * 32 * g.coutp * 4) + 1024;
}

// dw (+)= the weight gradient of y = conv(x, w) for the output gradient dy (see above); the bias
// gradient is not formed here.
cudaError_t wgrad_umma(const float* x, const float* dy, float* dw, int cin, int cout, int d, int h, int w, int accumulate,
                       void* scratch, long long scratch_bytes, cudaStream_t st) {
    using namespace dvm_nn;
    if (scratch_bytes < wgrad_umma_scratch_bytes(cin, cout, d, h, w)) return cudaErrorInvalidValue;
    EncodeFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const WgradGeom g = wgrad_geom(cin, cout, d, h, w);
    const int bn = bn_for(cout);
    const int nsplit = (g.nchunks + g.chunks_per_split - 1) / g.chunks_per_split;
    const uintptr_t base = (reinterpret_cast<uintptr_t>(scratch) + 1023) & ~uintptr_t(1023);
    const long long xs_bytes = align1k(3LL * g.cinp * (d + 2) * (h + 2) * g.Wp * 2);
    const long long gb_bytes = align1k((long long)g.coutp * d * h * g.Wp * 2);
    __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(base);
    __nv_bfloat16* gb = reinterpret_cast<__nv_bfloat16*>(base + xs_bytes);
    float* part = reinterpret_cast<float*>(base + xs_bytes + gb_bytes);
    {
        const long long rows = 3LL * g.cinp * (d + 2) * (h + 2);
        shift_bf16_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(x, xs, cin, g.cinp, d, h, w, g.Wp);
        const long long m = (long long)g.coutp * d * h * g.Wp;
        grad_bf16_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(dy, gb, cout, g.coutp, d, h, w, g.Wp);
    }
    CUtensorMap tx, tg;
    {
        const cuuint64_t dims[5] = {(cuuint64_t)g.Wp, (cuuint64_t)(h + 2), (cuuint64_t)(d + 2), (cuuint64_t)g.cinp, 3u};
        const cuuint64_t strides[4] = {(cuuint64_t)g.Wp * 2, (cuuint64_t)g.Wp * 2 * (h + 2),
                                       (cuuint64_t)g.Wp * 2 * (h + 2) * (d + 2),
                                       (cuuint64_t)g.Wp * 2 * (h + 2) * (d + 2) * g.cinp};
        const cuuint32_t box[5] = {32u, 1u, 1u, 32u, 1u};
        const cuuint32_t es[5] = {1u, 1u, 1u, 1u, 1u};
        if (enc(&tx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, xs, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const cuuint64_t dims[4] = {(cuuint64_t)g.Wp, (cuuint64_t)h, (cuuint64_t)d, (cuuint64_t)g.coutp};
        const cuuint64_t strides[3] = {(cuuint64_t)g.Wp * 2, (cuuint64_t)g.Wp * 2 * h, (cuuint64_t)g.Wp * 2 * h * d};
        const cuuint32_t box[4] = {32u, 1u, 1u, (cuuint32_t)bn};
        const cuuint32_t es[4] = {1u, 1u, 1u, 1u};
        if (enc(&tg, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, gb, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    cudaError_t e;
    if (bn == 32) e = launch_wgrad_bn<32>(tx, tg, part, g, nsplit, st);
    else if (bn == 64) e = launch_wgrad_bn<64>(tx, tg, part, g, nsplit, st);
    else e = launch_wgrad_bn<128>(tx, tg, part, g, nsplit, st);
    if (e != cudaSuccess) return e;
    const long long total = (long long)cout * cin * 27;
    wgrad_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(part, dw, cin, cout, g.cinp, g.coutp, g.nsb,
                                                                         nsplit, accumulate);
    return cudaGetLastError();
}

// the device status word of the convolutions (nonzero after a bounded wait expired); cleared on read
int conv_umma_status(cudaStream_t st) {
    int v = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess) return -3;
    if (cudaMemcpyFromSymbol(&v, dvm_nn::g_conv_status, sizeof(int)) != cudaSuccess) return -3;
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(dvm_nn::g_conv_status, &zero, sizeof(int));
    }
    return v;
}
