// sweep2d_f32x2.cu -- FP32 transport sweep of one source iteration in 2D (arXiv:1712.01132,
// Sec. 3.1 step i with the quadrature of step iii fused), two discrete velocities per lane.
//
// Schedule: persistent CTAs take (problem, quadrant, band) items from a ticket counter in band
// order.  A CTA sweeps its band along x1 in tiles of 8 columns; band b starts tile t once band b-1
// has published it.  Inside a tile every warp walks its rows two at a time, the upper row one
// column behind the lower one, so a warp always has two independent dependency chains in flight.
// Per-point arithmetic (Eq. 10 solved for h at the point, upwind stencil of Eq. 9):
//   h = R * [ nu rho' + 2 nu u.v + v1 + a1 (K1x h(x-s1 e1) + K2x h(x-2 s1 e1) + E1)
//                                     + a2 (K1y h(x-s2 e2) + K2y h(x-2 s2 e2) + E2) ]
// with a_j = |v_j|/dx, the stencil weights (K1, K2) = (2, -1/2) (second order), wall terms E
// where an upstream point is solid, and R the reciprocal denominator of the point's stencil case.
// Each lane carries a pair of velocities and updates both with packed f32x2 FMAs; the per-point
// scalars are stored duplicated in shared memory so they load as pairs.  Solid points carry zero
// records (their h is 0 and no stencil reads it with a nonzero weight).
//
// Latency hiding: the next tile's records are loaded into registers while the current tile is
// swept; progress is published as soon as the band edge is stored, before the moment partials
// are combined.  The moment of a point is summed in a fixed order (the lane's pair, the lane
// tree, the warps, the quadrants), so results do not depend on tile shapes or scheduling.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "dvm_device.cuh"
#include "dvm_internal.h"

namespace dvm {

namespace {

constexpr int kRec2 = 20;   // floats per point record: five duplicated-pair float4s
constexpr int kT1 = 8;      // tile width along x1
constexpr int kMaxRounds = 1;   // points prefetched per thread (bounds the rows per band)

struct LaneP {
    float2 v1, v2, a1, a2, W, Wv1, Wv2;
};

struct RawPoint {           // global data of one point needed to build its record
    float4 s, e;
    int code;
};

__device__ __forceinline__ float2 dup(float x) { return make_float2(x, x); }

// one point: returns h for the lane's two velocities
__device__ __forceinline__ float2 point_update(const float* __restrict__ rp, const float* __restrict__ rtab,
                                               const LaneP& L, float2 hp1, float2 hp2, float2 up1, float2 up2) {
    const float4* R = reinterpret_cast<const float4*>(rp);
    const float4 r0 = R[0];   // a a b1 b1
    const float4 r1 = R[1];   // b2 b2 E1 E1
    const float4 r2 = R[2];   // K1x K1x K2x K2x
    const float4 r3 = R[3];   // E2 E2 K1y K1y
    const float4 r4 = R[4];   // K2y K2y rtab-offset -
    const float2 Rv = *reinterpret_cast<const float2*>(rtab + __float_as_int(r4.z));
    const float2 S = fma2(make_float2(r1.x, r1.y), L.v2, fma2(make_float2(r0.z, r0.w), L.v1, make_float2(r0.x, r0.y)));
    const float2 t2 = fma2(make_float2(r3.z, r3.w), up1, fma2(make_float2(r4.x, r4.y), up2, make_float2(r3.x, r3.y)));
    const float2 base = fma2(L.a2, t2, S);
    const float2 t1 = fma2(make_float2(r2.x, r2.y), hp1, fma2(make_float2(r2.z, r2.w), hp2, make_float2(r1.z, r1.w)));
    return mul2(fma2(L.a1, t1, base), Rv);
}

__device__ __forceinline__ void moments_of(const LaneP& L, float2 h, float& m0, float& m1, float& m2) {
    const float2 p0 = mul2(L.W, h);
    const float2 p1 = mul2(L.Wv1, h);
    const float2 p2 = mul2(L.Wv2, h);
    m0 = p0.x + p0.y;
    m1 = p1.x + p1.y;
    m2 = p2.x + p2.y;
}

}  // namespace

__global__ void __launch_bounds__(256) sweep2d_f32x2_kernel(const SweepArgs2D<float> a) {
    constexpr int T1 = kT1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    __shared__ int s_abort;
    const int NW = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int RB = a.max_rows;
    float* rec = reinterpret_cast<float*>(smem_raw);                    // [2][RB][T1][kRec2]
    float* part = rec + (size_t)2 * RB * T1 * kRec2;                     // [NW][RB][T1][3]
    float* carry = part + (size_t)NW * RB * T1 * 3;                      // [NW][RB][2][64]
    float* rtab = carry + (size_t)NW * RB * 2 * 64;                      // [NW][4][64]
    unsigned* rmask = reinterpret_cast<unsigned*>(rtab + (size_t)NW * 4 * 64);   // [2][RB]
    const int wl = warp * 32 + lane;            // lane index; velocities 2 wl, 2 wl + 1
    const size_t NL = (size_t)a.NL;
    float* my_rtab = rtab + (size_t)warp * 4 * 64;

    for (;;) {
        if (threadIdx.x == 0) {
            s_item = ld_volatile(a.status) ? a.nitems : atomicAdd(a.ticket, 1);
            s_abort = 0;
        }
        __syncthreads();
        const int it = s_item;
        if (it >= a.nitems) return;
        const SweepItem item = a.items[it];
        const Prob2D<float>* __restrict__ P = a.prob + item.prob;
        const int q = item.quad;
        const int band = item.band;
        const int n1 = P->n1, n2 = P->n2, nb = P->nbands;
        const int N = P->N;
        const int s1neg = q & 1;
        const int s2neg = (q >> 1) & 1;
        const int row0 = band * P->rows;
        const int nrows = min(P->rows, n2 - row0);
        const float K1o = P->order == 2 ? 2.f : 1.f;
        const float K2o = P->order == 2 ? -0.5f : 0.f;
        LaneP L;
        {
            const float* la = P->lanec + ((size_t)q * NL + 2 * wl) * kLaneConsts;
            const float* lb = la + kLaneConsts;
            L.v1 = make_float2(la[0], lb[0]);
            L.v2 = make_float2(la[1], lb[1]);
            L.a1 = make_float2(la[2], lb[2]);
            L.a2 = make_float2(la[3], lb[3]);
            L.W = make_float2(la[4], lb[4]);
            L.Wv1 = make_float2(la[5], lb[5]);
            L.Wv2 = make_float2(la[6], lb[6]);
#pragma unroll
            for (int rs = 0; rs < 4; ++rs)
                *reinterpret_cast<float2*>(my_rtab + rs * 64 + 2 * lane) = make_float2(la[7 + rs], lb[7 + rs]);
        }
        const int par = a.parity;
        {
            const float* g = P->gx1 + (((size_t)par * 4 + q) * n2) * 2 * NL;
            for (int r = 0; r < nrows; ++r) {
                float* cr = carry + ((size_t)(warp * RB + r) * 2) * 64 + 2 * lane;
                *reinterpret_cast<float2*>(cr) = *reinterpret_cast<const float2*>(g + ((size_t)(row0 + r) * 2 + 0) * NL + 2 * wl);
                *reinterpret_cast<float2*>(cr + 64) = *reinterpret_cast<const float2*>(g + ((size_t)(row0 + r) * 2 + 1) * NL + 2 * wl);
            }
        }
        const int ntiles = (n1 + T1 - 1) / T1;
        const int npts = nrows * T1;
        const int rounds = (npts + blockDim.x - 1) / blockDim.x;

        // global data of the points this thread turns into records, for tile tt
        auto load_raw = [&](int tt, RawPoint (&raw)[kMaxRounds]) {
#pragma unroll
            for (int k = 0; k < kMaxRounds; ++k) {
                raw[k].code = kSolidBit;
                const int idx = k * blockDim.x + threadIdx.x;
                if (k < rounds && idx < npts) {
                    const int r = idx / T1;
                    const int ic = tt * T1 + (idx - r * T1);
                    if (ic < n1) {
                        const int x = s1neg ? n1 - 1 - ic : ic;
                        const int yo = row0 + r;
                        const int y = s2neg ? n2 - 1 - yo : yo;
                        const int id = y * n1 + x;
                        raw[k].code = P->code[id];
                        if (!(raw[k].code & kSolidBit)) {
                            raw[k].s = reinterpret_cast<const float4*>(P->src)[id];
                            raw[k].e = reinterpret_cast<const float4*>(P->E)[id];
                        }
                    }
                }
            }
        };
        // records (duplicated pairs; zero for solid points) and per-row fluid masks
        auto store_rec = [&](int buf, const RawPoint (&raw)[kMaxRounds]) {
            float* rb = rec + (size_t)buf * RB * T1 * kRec2;
            unsigned* mk = rmask + buf * RB;
#pragma unroll
            for (int k = 0; k < kMaxRounds; ++k) {
                if (k >= rounds) break;
                const int idx = k * blockDim.x + threadIdx.x;
                const bool fluid = idx < npts && !(raw[k].code & kSolidBit);
                if (idx < npts) {
                    float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f), o1 = o0, o2 = o0, o3 = o0, o4 = o0;
                    if (fluid) {
                        const int code = raw[k].code;
                        const int ca = (code >> (2 * (0 + s1neg))) & 3;
                        const int cb = (code >> (2 * (2 + s2neg))) & 3;
                        const float E1 = s1neg ? raw[k].e.y : raw[k].e.x;
                        const float E2 = s2neg ? raw[k].e.w : raw[k].e.z;
                        const float K1x = ca == 2 ? 0.f : K1o, K2x = ca == 0 ? K2o : 0.f;
                        const float K1y = cb == 2 ? 0.f : K1o, K2y = cb == 0 ? K2o : 0.f;
                        const int rs = (ca == 2) | ((cb == 2) << 1);
                        o0 = make_float4(raw[k].s.x, raw[k].s.x, raw[k].s.y, raw[k].s.y);
                        o1 = make_float4(raw[k].s.z, raw[k].s.z, E1, E1);
                        o2 = make_float4(K1x, K1x, K2x, K2x);
                        o3 = make_float4(E2, E2, K1y, K1y);
                        o4 = make_float4(K2y, K2y, __int_as_float(rs * 64), 0.f);
                    }
                    float4* R = reinterpret_cast<float4*>(rb + (size_t)idx * kRec2);
                    R[0] = o0;
                    R[1] = o1;
                    R[2] = o2;
                    R[3] = o3;
                    R[4] = o4;
                }
                const unsigned bits = __ballot_sync(0xffffffffu, fluid);
                if (lane == 0) {
                    const int base = k * blockDim.x + warp * 32;
#pragma unroll
                    for (int sub = 0; sub < 32 / T1; ++sub) {
                        const int rr = (base + sub * T1) / T1;
                        if (rr < nrows) mk[rr] = (bits >> (sub * T1)) & ((1u << T1) - 1u);
                    }
                }
            }
        };

        {
            RawPoint raw[kMaxRounds];
            load_raw(0, raw);
            store_rec(0, raw);
        }
        for (int t = 0; t < ntiles; ++t) {
            const int c0 = t * T1;
            const int width = min(T1, n1 - c0);
            const int buf = t & 1;
            RawPoint nxt[kMaxRounds];
            if (t + 1 < ntiles) load_raw(t + 1, nxt);
            if (threadIdx.x == 0 && band > 0) {
                if (!wait_geq(P->prog + q * nb + band - 1, t + 1, a.status, a.timeout_ns)) s_abort = 1;
            }
            __syncthreads();
            if (s_abort) return;
            const float* rbuf = rec + (size_t)buf * RB * T1 * kRec2;
            const unsigned* mk = rmask + buf * RB;
            float2 rb1[T1], rb2[T1];
            {
                const float* eb = (band == 0)
                    ? P->glat + (((size_t)par * 4 + q) * n1) * 2 * NL
                    : P->edge + ((size_t)(q * (nb - 1) + band - 1) * n1) * 2 * NL;
#pragma unroll
                for (int i = 0; i < T1; ++i) {
                    if (i < width) {
                        rb1[i] = __ldcg(reinterpret_cast<const float2*>(eb + ((size_t)(c0 + i) * 2 + 0) * NL + 2 * wl));
                        rb2[i] = __ldcg(reinterpret_cast<const float2*>(eb + ((size_t)(c0 + i) * 2 + 1) * NL + 2 * wl));
                    } else {
                        rb1[i] = make_float2(0.f, 0.f);
                        rb2[i] = make_float2(0.f, 0.f);
                    }
                }
            }
            const float* rt = my_rtab + 2 * lane;
            // FULL: all T1 columns exist; otherwise columns >= width are skipped (uniform test) so
            // the x1 carry keeps the last two points of the row
            auto walk_rows = [&](auto full_tag) {
                constexpr bool FULL = decltype(full_tag)::value;
                int r = 0;
                for (; r + 1 < nrows; r += 2) {
                    // rows r (lower) and r+1 (upper), the upper one column behind
                    float* ca = carry + ((size_t)(warp * RB + r) * 2) * 64 + 2 * lane;
                    float* cb = ca + 2 * 64;
                    const unsigned fm = mk[r] | mk[r + 1];
                    if (fm == 0u) continue;     // both rows solid in this tile: nothing reads them
                    float2 ha1 = *reinterpret_cast<const float2*>(ca);
                    float2 ha2 = *reinterpret_cast<const float2*>(ca + 64);
                    float2 hb1 = *reinterpret_cast<const float2*>(cb);
                    float2 hb2 = *reinterpret_cast<const float2*>(cb + 64);
                    const float* ra = rbuf + (size_t)r * T1 * kRec2;
                    const float* rbr = ra + T1 * kRec2;
                    float ma0[T1], ma1[T1], ma2[T1], mb0[T1], mb1[T1], mb2[T1];
#pragma unroll
                    for (int s = 0; s <= T1; ++s) {
                        if (s < T1) {
                            if (FULL || s < width) {
                                const float2 h = point_update(ra + s * kRec2, rt, L, ha1, ha2, rb1[s], rb2[s]);
                                ha2 = ha1;
                                ha1 = h;
                                rb2[s] = rb1[s];
                                rb1[s] = h;
                                moments_of(L, h, ma0[s], ma1[s], ma2[s]);
                            } else {
                                ma0[s] = ma1[s] = ma2[s] = 0.f;
                            }
                        }
                        if (s >= 1) {
                            const int i = s - 1;
                            if (FULL || i < width) {
                                const float2 h = point_update(rbr + i * kRec2, rt, L, hb1, hb2, rb1[i], rb2[i]);
                                hb2 = hb1;
                                hb1 = h;
                                rb2[i] = rb1[i];
                                rb1[i] = h;
                                moments_of(L, h, mb0[i], mb1[i], mb2[i]);
                            } else {
                                mb0[i] = mb1[i] = mb2[i] = 0.f;
                            }
                        }
                        if (s == T1 - 1) {
                            // lower row complete: reduce it while the upper row finishes
                            const float s0 = reduce_scatter<float, T1>(ma0, lane);
                            const float s1 = reduce_scatter<float, T1>(ma1, lane);
                            const float s2 = reduce_scatter<float, T1>(ma2, lane);
                            if ((lane & 3) == 0) {
                                float* d = part + ((size_t)(warp * RB + r) * T1 + (lane >> 2)) * 3;
                                d[0] = s0;
                                d[1] = s1;
                                d[2] = s2;
                            }
                        }
                    }
                    *reinterpret_cast<float2*>(ca) = ha1;
                    *reinterpret_cast<float2*>(ca + 64) = ha2;
                    *reinterpret_cast<float2*>(cb) = hb1;
                    *reinterpret_cast<float2*>(cb + 64) = hb2;
                    const float s0 = reduce_scatter<float, T1>(mb0, lane);
                    const float s1 = reduce_scatter<float, T1>(mb1, lane);
                    const float s2 = reduce_scatter<float, T1>(mb2, lane);
                    if ((lane & 3) == 0) {
                        float* d = part + ((size_t)(warp * RB + r + 1) * T1 + (lane >> 2)) * 3;
                        d[0] = s0;
                        d[1] = s1;
                        d[2] = s2;
                    }
                }
                if (r < nrows && mk[r] != 0u) {
                    // last row of an odd band
                    float* ca = carry + ((size_t)(warp * RB + r) * 2) * 64 + 2 * lane;
                    float2 ha1 = *reinterpret_cast<const float2*>(ca);
                    float2 ha2 = *reinterpret_cast<const float2*>(ca + 64);
                    const float* ra = rbuf + (size_t)r * T1 * kRec2;
                    float m0[T1], m1[T1], m2[T1];
#pragma unroll
                    for (int s = 0; s < T1; ++s) {
                        if (FULL || s < width) {
                            const float2 h = point_update(ra + s * kRec2, rt, L, ha1, ha2, rb1[s], rb2[s]);
                            ha2 = ha1;
                            ha1 = h;
                            rb2[s] = rb1[s];
                            rb1[s] = h;
                            moments_of(L, h, m0[s], m1[s], m2[s]);
                        } else {
                            m0[s] = m1[s] = m2[s] = 0.f;
                        }
                    }
                    *reinterpret_cast<float2*>(ca) = ha1;
                    *reinterpret_cast<float2*>(ca + 64) = ha2;
                    const float s0 = reduce_scatter<float, T1>(m0, lane);
                    const float s1 = reduce_scatter<float, T1>(m1, lane);
                    const float s2 = reduce_scatter<float, T1>(m2, lane);
                    if ((lane & 3) == 0) {
                        float* d = part + ((size_t)(warp * RB + r) * T1 + (lane >> 2)) * 3;
                        d[0] = s0;
                        d[1] = s1;
                        d[2] = s2;
                    }
                }
            };
            if (width == T1) walk_rows(std::integral_constant<bool, true>{});
            else walk_rows(std::integral_constant<bool, false>{});
            // band edge for the band above, or the x2 ghost layers of the next iteration (Eq. 8 /
            // periodic: the reflected quadrant reads the same lane)
            {
                float* et;
                if (band < nb - 1) {
                    et = P->edge + ((size_t)(q * (nb - 1) + band) * n1) * 2 * NL;
                } else {
                    const int qr = (P->lateral == 1) ? q : (q ^ 2);
                    et = P->glat + (((size_t)(par ^ 1) * 4 + qr) * n1) * 2 * NL;
                }
#pragma unroll
                for (int i = 0; i < T1; ++i) {
                    if (i < width) {
                        *reinterpret_cast<float2*>(et + ((size_t)(c0 + i) * 2 + 0) * NL + 2 * wl) = rb1[i];
                        *reinterpret_cast<float2*>(et + ((size_t)(c0 + i) * 2 + 1) * NL + 2 * wl) = rb2[i];
                    }
                }
            }
            if (t == ntiles - 1) {
                // x1 ghost layers of the next iteration (periodic in x1, same quadrant)
                float* g = P->gx1 + (((size_t)(par ^ 1) * 4 + q) * n2) * 2 * NL;
                for (int rr = 0; rr < nrows; ++rr) {
                    const float* cr = carry + ((size_t)(warp * RB + rr) * 2) * 64 + 2 * lane;
                    *reinterpret_cast<float2*>(g + ((size_t)(row0 + rr) * 2 + 0) * NL + 2 * wl) = *reinterpret_cast<const float2*>(cr);
                    *reinterpret_cast<float2*>(g + ((size_t)(row0 + rr) * 2 + 1) * NL + 2 * wl) = *reinterpret_cast<const float2*>(cr + 64);
                }
            }
            if (t + 1 < ntiles) store_rec(buf ^ 1, nxt);
            __syncthreads();
            if (threadIdx.x == 0 && it != a.withhold_item) {
                __threadfence();
                st_release_gpu(P->prog + q * nb + band, t + 1);
            }
            // moment partials of this quadrant: sum of the warps' lane sums, in warp order
            for (int idx = threadIdx.x; idx < nrows * width * 3; idx += blockDim.x) {
                const int m = idx % 3;
                const int pi = idx / 3;
                const int rr = pi / width;
                const int i = pi - rr * width;
                float s = 0.f;
                if ((mk[rr] >> i) & 1u)
                    for (int w = 0; w < NW; ++w) s += part[((size_t)(w * RB + rr) * T1 + i) * 3 + m];
                const int ic = c0 + i;
                const int x = s1neg ? n1 - 1 - ic : ic;
                const int yo = row0 + rr;
                const int y = s2neg ? n2 - 1 - yo : yo;
                P->P[((size_t)q * 3 + m) * N + (size_t)y * n1 + x] = s;
            }
        }
        __syncthreads();
    }
}

size_t sweep2d_f32x2_smem(int NW, int max_rows) {
    return sizeof(float) * ((size_t)2 * max_rows * kT1 * kRec2 + (size_t)NW * max_rows * kT1 * 3 +
                            (size_t)NW * max_rows * 2 * 64 + (size_t)NW * 4 * 64) +
           sizeof(unsigned) * (size_t)2 * max_rows;
}

int sweep2d_f32x2_max_rows(int NW) { return kMaxRounds * NW * 32 / kT1; }

cudaError_t launch_sweep2d_f32x2(const SweepArgs2D<float>& a, int grid, int NW, cudaStream_t st) {
    const size_t smem = sweep2d_f32x2_smem(NW, a.max_rows);
    cudaError_t e = cudaFuncSetAttribute(sweep2d_f32x2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sweep2d_f32x2_kernel<<<grid, NW * 32, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t sweep2d_f32x2_occupancy(int NW, int max_rows, int* blocks_per_sm) {
    const size_t smem = sweep2d_f32x2_smem(NW, max_rows);
    cudaError_t e = cudaFuncSetAttribute(sweep2d_f32x2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, sweep2d_f32x2_kernel, NW * 32, smem);
}

}  // namespace dvm
