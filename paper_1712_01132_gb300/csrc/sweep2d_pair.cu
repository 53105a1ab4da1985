// sweep2d_pair.cu -- FP32 2D transport sweep (arXiv:1712.01132, Sec. 3.1 step i with the quadrature
// of step iii fused), two consecutive bands per CTA.
//
// Same arithmetic, records and lane layout as sweep2d_f32x2_kernel (four velocities per lane as two
// packed pairs), but a CTA holds two groups of warps: group 0 sweeps band 2i and group 1 band 2i + 1
// one tile behind it.  In step s group 0 sweeps tile s and group 1 tile s - 1; the top edge of
// band 2i reaches band 2i + 1 through a double-buffered shared-memory slot and the CTA barrier that
// ends the step, instead of a global store, a fence, a flag poll and an L2 load.  Only band 2i + 1
// publishes progress (band 2i + 2, in another CTA, waits for it), so half of the band hand-offs on
// the wavefront's critical path stay inside the SM.  Used without x1/x2 subdomains.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "dvm_device.cuh"
#include "dvm_internal.h"

namespace dvm {

namespace {

constexpr int kRecF = 12;   // floats per point record (10 used): {a b1 b2 roff} {E1 K1x K2x E2} {K1y K2y}
constexpr int kVL = 4;      // velocities per lane (two packed pairs)
constexpr int kMaxRounds = 2;

struct LaneQ {
    float2 v1[2], v2[2], a1[2], a2[2], W[2], Wv1[2], Wv2[2];
};

struct RawPoint {
    float4 s, e;
    int code;
};

__device__ __forceinline__ float2 dup(float x) { return make_float2(x, x); }

}  // namespace

template <int T1>
__global__ void __launch_bounds__(256) sweep2d_pair_kernel(const SweepArgs2D<float> a) {
    constexpr int kLPP = 32 / T1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    __shared__ int s_abort;
    __shared__ int s_band[2][2];                 // per group: first oriented row, rows (0: no band)
    const int NW = blockDim.x >> 5;              // all warps
    const int NWg = NW >> 1;                     // warps per group
    const int GT = NWg * 32;                     // threads per group
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int g = warp / NWg;                    // group: 0 lower band, 1 upper band
    const int gw = warp - g * NWg;               // warp within the group
    const int gt = threadIdx.x - g * GT;         // thread within the group
    const int RB = a.max_rows;
    const size_t NL = (size_t)a.NL;
    const size_t grp_floats = (size_t)2 * RB * T1 * kRecF + (size_t)NWg * RB * T1 * 3 + (size_t)NWg * RB * 2 * 128;
    float* gbase = reinterpret_cast<float*>(smem_raw) + (size_t)g * grp_floats;
    float* rec = gbase;                                                   // [2][RB][T1][kRecF]
    float* part = rec + (size_t)2 * RB * T1 * kRecF;                      // [NWg][RB][T1][3]
    float* carry = part + (size_t)NWg * RB * T1 * 3;                      // [NWg][RB][2][128]
    float* rtab = reinterpret_cast<float*>(smem_raw) + 2 * grp_floats;   // [NW][4][128]
    float* eh = rtab + (size_t)NW * 4 * 128;                              // [2][T1][2][NL] edge hand-off
    unsigned* rmask = reinterpret_cast<unsigned*>(eh + (size_t)2 * T1 * 2 * NL) + (size_t)g * 2 * RB;  // [2 groups][2][RB]
    const int wl = gw * 32 + lane;               // lane index within the quadrant's velocity set
    const float* my_rtab = rtab + (size_t)warp * 4 * 128 + 4 * lane;

    for (;;) {
        if (threadIdx.x == 0) {
            s_item = ld_volatile(a.status) ? a.nitems : atomicAdd(a.ticket, 1);
            s_abort = 0;
            if (s_item < a.nitems) {
                const SweepItem itm = a.items[s_item];
                const Prob2D<float>& Pi = a.prob[itm.prob];
                for (int gg = 0; gg < 2; ++gg) {
                    const int b = 2 * itm.band + gg;
                    int4 bi = make_int4(0, 0, 0, 0);
                    if (b < Pi.nbands) bi = Pi.bands[itm.quad * Pi.nbands + b];
                    s_band[gg][0] = bi.x;
                    s_band[gg][1] = bi.y;
                }
            }
        }
        __syncthreads();
        const int it = s_item;
        if (it >= a.nitems) return;
        const SweepItem item = a.items[it];
        const Prob2D<float>* __restrict__ P = a.prob + item.prob;
        const int q = item.quad;
        const int band = 2 * item.band + g;          // this group's band
        const int n1 = P->n1, n2 = P->n2, nb = P->nbands;
        const int N = P->N;
        const int s1neg = q & 1;
        const int s2neg = (q >> 1) & 1;
        const int row0 = s_band[g][0], nrows = s_band[g][1];
        const bool valid = nrows > 0;
        const bool partner = s_band[1][1] > 0;       // band 2i + 1 exists
        const float K1o = P->order == 2 ? 2.f : 1.f;
        const float K2o = P->order == 2 ? -0.5f : 0.f;
        LaneQ L;
        {
            const float* lc = P->lanec + ((size_t)q * NL + (size_t)kVL * wl) * kLaneConsts;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float* la = lc + (2 * k) * kLaneConsts;
                const float* lb = la + kLaneConsts;
                L.v1[k] = make_float2(la[0], lb[0]);
                L.v2[k] = make_float2(la[1], lb[1]);
                L.a1[k] = make_float2(la[2], lb[2]);
                L.a2[k] = make_float2(la[3], lb[3]);
                L.W[k] = make_float2(la[4], lb[4]);
                L.Wv1[k] = make_float2(la[5], lb[5]);
                L.Wv2[k] = make_float2(la[6], lb[6]);
            }
            float* rt = rtab + (size_t)warp * 4 * 128 + 4 * lane;
#pragma unroll
            for (int rs = 0; rs < 4; ++rs)
                *reinterpret_cast<float4*>(rt + rs * 128) =
                    make_float4(lc[7 + rs], lc[kLaneConsts + 7 + rs], lc[2 * kLaneConsts + 7 + rs], lc[3 * kLaneConsts + 7 + rs]);
        }
        const int par = a.parity;
        if (valid) {
            const float* gx = P->gx1 + (((size_t)par * 4 + q) * n2) * 2 * NL;
            for (int r = 0; r < nrows; ++r) {
                float* cr = carry + ((size_t)(gw * RB + r) * 2) * 128 + 4 * lane;
                *reinterpret_cast<float4*>(cr) = *reinterpret_cast<const float4*>(gx + ((size_t)(row0 + r) * 2 + 0) * NL + kVL * wl);
                *reinterpret_cast<float4*>(cr + 128) = *reinterpret_cast<const float4*>(gx + ((size_t)(row0 + r) * 2 + 1) * NL + kVL * wl);
            }
        }
        const int ntiles = (n1 + T1 - 1) / T1;
        const int npts = nrows * T1;
        const int rounds = (npts + GT - 1) / GT;

        auto load_raw = [&](int tt, RawPoint (&raw)[kMaxRounds]) {
#pragma unroll
            for (int k = 0; k < kMaxRounds; ++k) {
                raw[k].code = kSolidBit;
                const int idx = k * GT + gt;
                if (k < rounds && idx < npts) {
                    const int r = idx / T1;
                    const int ic = tt * T1 + (idx - r * T1);
                    if (ic < n1) {
                        const int x = s1neg ? n1 - 1 - ic : ic;
                        const int yo = row0 + r;
                        const int y = s2neg ? n2 - 1 - yo : yo;
                        const int id = y * n1 + x;
                        // issued together: no branch on the code before the other loads
                        raw[k].code = P->code[id];
                        raw[k].s = reinterpret_cast<const float4*>(P->src)[id];
                        raw[k].e = reinterpret_cast<const float4*>(P->E)[id];
                    }
                }
            }
        };
        auto store_rec = [&](int buf, const RawPoint (&raw)[kMaxRounds]) {
            float* rb = rec + (size_t)buf * RB * T1 * kRecF;
            unsigned* mk = rmask + buf * RB;
#pragma unroll
            for (int k = 0; k < kMaxRounds; ++k) {
                if (k >= rounds) break;
                const int idx = k * GT + gt;
                const bool fluid = idx < npts && !(raw[k].code & kSolidBit);
                if (idx < npts) {
                    float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f), o1 = o0, o2 = o0;
                    if (fluid) {
                        const int code = raw[k].code;
                        const int ca = (code >> (2 * (0 + s1neg))) & 3;
                        const int cb = (code >> (2 * (2 + s2neg))) & 3;
                        const float E1 = s1neg ? raw[k].e.y : raw[k].e.x;
                        const float E2 = s2neg ? raw[k].e.w : raw[k].e.z;
                        const int rs = (ca != 0) | ((cb != 0) << 1);
                        o0 = make_float4(raw[k].s.x, raw[k].s.y, raw[k].s.z, __int_as_float(rs * 128));
                        o1 = make_float4(E1, ca == 2 ? 0.f : (ca == 1 ? 1.f : K1o), ca == 0 ? K2o : 0.f, E2);
                        o2 = make_float4(cb == 2 ? 0.f : (cb == 1 ? 1.f : K1o), cb == 0 ? K2o : 0.f, 0.f, 0.f);
                    }
                    float4* R = reinterpret_cast<float4*>(rb + (size_t)idx * kRecF);
                    R[0] = o0;
                    R[1] = o1;
                    R[2] = o2;
                }
                const unsigned bits = __ballot_sync(0xffffffffu, fluid);
                if (lane == 0) {
                    const int base = k * GT + gw * 32;
#pragma unroll
                    for (int sub = 0; sub < 32 / T1; ++sub) {
                        const int rr = (base + sub * T1) / T1;
                        if (rr < nrows) mk[rr] = (bits >> (sub * T1)) & ((1u << T1) - 1u);
                    }
                }
            }
        };

        if (valid) {
            RawPoint raw[kMaxRounds];
            load_raw(0, raw);
            store_rec(0, raw);
        }
        for (int s = 0; s <= ntiles; ++s) {
            const int t = s - g;                     // this group's tile in this step
            const bool active = valid && t >= 0 && t < ntiles;
            const int c0 = t * T1;
            const int width = active ? min(T1, n1 - c0) : 0;
            const int buf = t & 1;
            RawPoint nxt[kMaxRounds];
            if (active && t + 1 < ntiles) load_raw(t + 1, nxt);
            // band 2i (group 0) waits for band 2i - 1, swept by another CTA
            if (gt == 0 && g == 0 && active && band > 0) {
                if (!wait_geq(P->prog + q * nb + band - 1, t + 1, a.status, a.timeout_ns)) s_abort = 1;
            }
            __syncthreads();
            if (s_abort) return;
            if (active) {
                const float* rbuf = rec + (size_t)buf * RB * T1 * kRecF;
                const unsigned* mk = rmask + buf * RB;
                // the two rows below: group 1 from the hand-off slot group 0 filled in the previous
                // step; group 0 from the global edge of band 2i - 1 or the x2 ghost layers
                float4 rb1[T1], rb2[T1];
                if (g == 1) {
                    const float* eb = eh + (size_t)(t & 1) * T1 * 2 * NL;     // slot of tile t
#pragma unroll
                    for (int i = 0; i < T1; ++i) {
                        if (i < width) {
                            rb1[i] = *reinterpret_cast<const float4*>(eb + ((size_t)i * 2 + 0) * NL + kVL * wl);
                            rb2[i] = *reinterpret_cast<const float4*>(eb + ((size_t)i * 2 + 1) * NL + kVL * wl);
                        } else {
                            rb1[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                            rb2[i] = rb1[i];
                        }
                    }
                } else {
                    const float* eb = band == 0
                        ? P->glat + (((size_t)(par * 4 + q) * P->nslots + 0) * n1) * 2 * NL
                        : P->edge + ((size_t)(q * 2 * P->nslots + ((band - 1) & 1)) * n1) * 2 * NL;
#pragma unroll
                    for (int i = 0; i < T1; ++i) {
                        if (i < width) {
                            rb1[i] = __ldcg(reinterpret_cast<const float4*>(eb + ((size_t)(c0 + i) * 2 + 0) * NL + kVL * wl));
                            rb2[i] = __ldcg(reinterpret_cast<const float4*>(eb + ((size_t)(c0 + i) * 2 + 1) * NL + kVL * wl));
                        } else {
                            rb1[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                            rb2[i] = rb1[i];
                        }
                    }
                }
                auto walk_rows = [&](auto full_tag) {
                    constexpr bool FULL = decltype(full_tag)::value;
                    for (int r = 0; r < nrows; ++r) {
                        const unsigned fm = mk[r];
                        if (fm == 0u) continue;
                        float* cr = carry + ((size_t)(gw * RB + r) * 2) * 128 + 4 * lane;
                        const float4 c1 = *reinterpret_cast<const float4*>(cr);
                        const float4 c2 = *reinterpret_cast<const float4*>(cr + 128);
                        float2 hp1[2] = {make_float2(c1.x, c1.y), make_float2(c1.z, c1.w)};
                        float2 hp2[2] = {make_float2(c2.x, c2.y), make_float2(c2.z, c2.w)};
                        const float* rrow = rbuf + (size_t)r * T1 * kRecF;
                        float m0[T1], m1[T1], m2[T1];
#pragma unroll
                        for (int i = 0; i < T1; ++i) {
                            if (FULL || i < width) {
                                const float4* Rp = reinterpret_cast<const float4*>(rrow + i * kRecF);
                                const float4 A = Rp[0];
                                const float4 B = Rp[1];
                                const float2 C = *reinterpret_cast<const float2*>(Rp + 2);
                                const float4 Rv = *reinterpret_cast<const float4*>(my_rtab + __float_as_int(A.w));
                                const float2 aP = dup(A.x), b1P = dup(A.y), b2P = dup(A.z);
                                const float2 E1P = dup(B.x), K1xP = dup(B.y), K2xP = dup(B.z), E2P = dup(B.w);
                                const float2 K1yP = dup(C.x), K2yP = dup(C.y);
                                const float2 rb1a = make_float2(rb1[i].x, rb1[i].y), rb1b = make_float2(rb1[i].z, rb1[i].w);
                                const float2 rb2a = make_float2(rb2[i].x, rb2[i].y), rb2b = make_float2(rb2[i].z, rb2[i].w);
                                float2 h[2];
#pragma unroll
                                for (int k = 0; k < 2; ++k) {
                                    const float2 up1 = k ? rb1b : rb1a;
                                    const float2 up2 = k ? rb2b : rb2a;
                                    const float2 S = fma2(b2P, L.v2[k], fma2(b1P, L.v1[k], aP));
                                    const float2 t2 = fma2(K1yP, up1, fma2(K2yP, up2, E2P));
                                    const float2 bse = fma2(L.a2[k], t2, S);
                                    const float2 t1 = fma2(K1xP, hp1[k], fma2(K2xP, hp2[k], E1P));
                                    const float2 Rk = k ? make_float2(Rv.z, Rv.w) : make_float2(Rv.x, Rv.y);
                                    h[k] = mul2(fma2(L.a1[k], t1, bse), Rk);
                                    hp2[k] = hp1[k];
                                    hp1[k] = h[k];
                                }
                                rb2[i] = rb1[i];
                                rb1[i] = make_float4(h[0].x, h[0].y, h[1].x, h[1].y);
                                const float2 p0 = fma2(L.W[1], h[1], mul2(L.W[0], h[0]));
                                const float2 p1 = fma2(L.Wv1[1], h[1], mul2(L.Wv1[0], h[0]));
                                const float2 p2 = fma2(L.Wv2[1], h[1], mul2(L.Wv2[0], h[0]));
                                m0[i] = p0.x + p0.y;
                                m1[i] = p1.x + p1.y;
                                m2[i] = p2.x + p2.y;
                            } else {
                                m0[i] = m1[i] = m2[i] = 0.f;
                            }
                        }
                        *reinterpret_cast<float4*>(cr) = make_float4(hp1[0].x, hp1[0].y, hp1[1].x, hp1[1].y);
                        *reinterpret_cast<float4*>(cr + 128) = make_float4(hp2[0].x, hp2[0].y, hp2[1].x, hp2[1].y);
                        const float s0 = reduce_scatter<float, T1>(m0, lane);
                        const float s1 = reduce_scatter<float, T1>(m1, lane);
                        const float s2 = reduce_scatter<float, T1>(m2, lane);
                        if ((lane & (kLPP - 1)) == 0) {
                            float* d = part + ((size_t)(gw * RB + r) * T1 + lane / kLPP) * 3;
                            d[0] = s0;
                            d[1] = s1;
                            d[2] = s2;
                        }
                    }
                };
                if (width == T1) walk_rows(std::integral_constant<bool, true>{});
                else walk_rows(std::integral_constant<bool, false>{});
                // top edge: group 0 hands it to group 1 in shared memory (or, as the last band, to
                // the x2 ghosts); group 1 writes the global edge for band 2i + 2 (or the x2 ghosts)
                {
                    float* et;
                    int cb = c0;                              // column of the tile's first point in et
                    if (g == 0 && partner) {
                        et = eh + (size_t)(t & 1) * T1 * 2 * NL;
                        cb = 0;
                    } else if (band == nb - 1) {
                        const int qr = (P->lateral == 1) ? q : (q ^ 2);
                        et = P->glat + (((size_t)((par ^ 1) * 4 + qr) * P->nslots + 0) * n1) * 2 * NL;
                    } else {
                        et = P->edge + ((size_t)(q * 2 * P->nslots + (band & 1)) * n1) * 2 * NL;
                    }
#pragma unroll
                    for (int i = 0; i < T1; ++i) {
                        if (i < width) {
                            *reinterpret_cast<float4*>(et + ((size_t)(cb + i) * 2 + 0) * NL + kVL * wl) = rb1[i];
                            *reinterpret_cast<float4*>(et + ((size_t)(cb + i) * 2 + 1) * NL + kVL * wl) = rb2[i];
                        }
                    }
                }
                if (t == ntiles - 1) {
                    float* gx = P->gx1 + (((size_t)(par ^ 1) * 4 + q) * n2) * 2 * NL;
                    for (int rr = 0; rr < nrows; ++rr) {
                        const float* cr = carry + ((size_t)(gw * RB + rr) * 2) * 128 + 4 * lane;
                        *reinterpret_cast<float4*>(gx + ((size_t)(row0 + rr) * 2 + 0) * NL + kVL * wl) = *reinterpret_cast<const float4*>(cr);
                        *reinterpret_cast<float4*>(gx + ((size_t)(row0 + rr) * 2 + 1) * NL + kVL * wl) = *reinterpret_cast<const float4*>(cr + 128);
                    }
                }
                if (t + 1 < ntiles) store_rec(buf ^ 1, nxt);
            }
            __syncthreads();
            // band 2i + 1 publishes for band 2i + 2 (another CTA)
            if (gt == 0 && g == 1 && active && it != a.withhold_item) publish_gpu(P->prog + q * nb + band, t + 1);
            if (active) {
                const unsigned* mk = rmask + buf * RB;
                for (int idx = gt; idx < nrows * width * 3; idx += GT) {
                    const int m = idx % 3;
                    const int pi = idx / 3;
                    const int rr = pi / width;
                    const int i = pi - rr * width;
                    float sm = 0.f;
                    if ((mk[rr] >> i) & 1u)
                        for (int w = 0; w < NWg; ++w) sm += part[((size_t)(w * RB + rr) * T1 + i) * 3 + m];
                    const int ic = c0 + i;
                    const int x = s1neg ? n1 - 1 - ic : ic;
                    const int yo = row0 + rr;
                    const int y = s2neg ? n2 - 1 - yo : yo;
                    P->P[((size_t)q * 3 + m) * N + (size_t)y * n1 + x] = sm;
                }
            }
        }
        __syncthreads();
    }
}

size_t sweep2d_pair_smem(int T1, int NW, int max_rows, int NL) {
    const int NWg = NW / 2;
    const size_t grp = (size_t)2 * max_rows * T1 * kRecF + (size_t)NWg * max_rows * T1 * 3 + (size_t)NWg * max_rows * 2 * 128;
    return sizeof(float) * (2 * grp + (size_t)NW * 4 * 128 + (size_t)2 * T1 * 2 * NL) +
           sizeof(unsigned) * (size_t)2 * 2 * max_rows;
}

template <int T1>
static cudaError_t launch_pair_t(const SweepArgs2D<float>& a, int grid, int NW, cudaStream_t st) {
    const size_t smem = sweep2d_pair_smem(T1, NW, a.max_rows, a.NL);
    cudaError_t e = cudaFuncSetAttribute(sweep2d_pair_kernel<T1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sweep2d_pair_kernel<T1><<<grid, NW * 32, smem, st>>>(a);
    return cudaGetLastError();
}

// NW: warps of both groups (twice the warps one band needs)
cudaError_t launch_sweep2d_pair(const SweepArgs2D<float>& a, int T1, int grid, int NW, cudaStream_t st) {
    if (T1 == 8) return launch_pair_t<8>(a, grid, NW, st);
    if (T1 == 4) return launch_pair_t<4>(a, grid, NW, st);
    return cudaErrorInvalidValue;
}

template <int T1>
static cudaError_t occ_pair_t(int NW, int max_rows, int NL, int* blocks_per_sm) {
    const size_t smem = sweep2d_pair_smem(T1, NW, max_rows, NL);
    cudaError_t e = cudaFuncSetAttribute(sweep2d_pair_kernel<T1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, sweep2d_pair_kernel<T1>, NW * 32, smem);
}

cudaError_t sweep2d_pair_occupancy(int T1, int NW, int max_rows, int NL, int* blocks_per_sm) {
    if (T1 == 8) return occ_pair_t<8>(NW, max_rows, NL, blocks_per_sm);
    if (T1 == 4) return occ_pair_t<4>(NW, max_rows, NL, blocks_per_sm);
    return cudaErrorInvalidValue;
}

}  // namespace dvm
