// sweep2d_f32x2.cu -- FP32 transport sweep of one source iteration in 2D (arXiv:1712.01132,
// Sec. 3.1 step i with the quadrature of step iii fused), four discrete velocities per lane.
//
// Schedule: persistent CTAs take (problem, quadrant, band) items from a ticket counter in band
// order.  A CTA sweeps its band along x1 in tiles of 4, 8 (the default) or 16 columns, the last as
// two 8-column sub-tiles; band b starts tile t once band b-1 has published it.  Inside a tile a warp walks its rows two at a time, the upper row one column
// behind the lower; every lane carries four velocities as two packed pairs updated with
// fma.rn.f32x2, so each step has four independent dependency chains per lane.  Per-point arithmetic (Eq. 10 solved for h at the point, upwind stencil of Eq. 9):
//   h = R * [ nu rho' + 2 nu u.v + v1 + a1 (K1x h(x-s1 e1) + K2x h(x-2 s1 e1) + E1)
//                                     + a2 (K1y h(x-s2 e2) + K2y h(x-2 s2 e2) + E2) ]
// with a_j = |v_j|/dx, stencil weights (K1, K2) = (2, -1/2) (second order), wall terms E where an
// upstream point is solid, and R the reciprocal denominator of the point's stencil case.
//
// The per-point scalars are broadcast from a 10-word shared-memory record to every lane of the
// warps of the quadrant; with four velocities per lane each broadcast serves 128 velocities.
// Solid points carry zero records; pairs of tile rows without fluid are skipped.  The next tile's records
// are loaded into registers while the current tile is swept, and progress is published as soon as
// the band edge is stored.  The moment of a point is summed in a fixed order (the lane's four
// velocities, the lane tree, the warps, the quadrants), so results do not depend on tile shapes.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "dvm_device.cuh"
#include "dvm_internal.h"

namespace dvm {

namespace {

constexpr int kRecF = 12;   // floats per point record (10 used): {a b1 b2 roff} {E1 K1x K2x E2} {K1y K2y}
// tile width along x1: 4 or 8 columns (template parameter of the kernel)
constexpr int kVL = 4;      // velocities per lane (two packed pairs)
constexpr int kMaxRounds = 2;

struct LaneQ {
    float2 v1[2], v2[2], a1[2], a2[2], W[2], Wv1[2], Wv2[2];
    float2 Wx[4];   // (W, W v1) of the lane's four velocities, for the packed (rho, u1) sums
};

struct RawPoint {           // global data of one point needed to build its record
    float4 s, e;
    int code;
    int4 f;                 // wall faces (specular parts): upstream x1, x2; downstream x1, x2
};

__device__ __forceinline__ float2 dup(float x) { return make_float2(x, x); }

}  // namespace

template <int T1, bool XS, bool SPEC>
__global__ void __launch_bounds__(256) sweep2d_f32x2_kernel(const SweepArgs2D<float> a) {
    // a tile of T1 columns (one wait, one publish, one record load) is swept as sub-tiles of SW
    // columns, whose x2 upstream values are held in registers
    constexpr int SW = T1 > 8 ? 8 : T1;
    constexpr int NSUB = T1 / SW;
    static_assert(T1 % SW == 0 && 32 % T1 == 0, "tile width: 4, 8 or 16 columns");
    constexpr int kLPP = 32 / SW;               // lanes per point after the reduce-scatter
    constexpr int RF = SPEC ? 16 : kRecF;       // record floats (face ids in the last four)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    __shared__ int s_abort;
    __shared__ int s_binfo[4];                  // band of the current item: row0, rows, below, above
    const int NW = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int RB = a.max_rows;
    float* rec = reinterpret_cast<float*>(smem_raw);                    // [2][RB][T1][RF]
    float* part = rec + (size_t)2 * RB * T1 * RF;                        // [NW][RB][T1][4]: rho u1 u2 -
    float* carry = part + (size_t)NW * RB * T1 * 4;                      // [NW][RB][2][128]
    float* rtab = carry + (size_t)NW * RB * 2 * 128;                     // [NW][4][128]
    unsigned* rmask = reinterpret_cast<unsigned*>(rtab + (size_t)NW * 4 * 128);  // [2][RB]
    const int wl = warp * 32 + lane;            // lane index; velocities 4 wl .. 4 wl + 3
    const size_t NL = (size_t)a.NL;
    const float* my_rtab = rtab + (size_t)warp * 4 * 128 + 4 * lane;

    for (;;) {
        if (threadIdx.x == 0) {
            s_item = ld_volatile(a.status) ? a.nitems : atomicAdd(a.ticket, 1);
            s_abort = 0;
            if (s_item < a.nitems) {
                const SweepItem itm = a.items[s_item];
                const Prob2D<float>& Pi = a.prob[itm.prob];
                const int4 bi = Pi.bands[itm.quad * Pi.nbands + itm.band];
                s_binfo[0] = bi.x;
                s_binfo[1] = bi.y;
                s_binfo[2] = bi.z;
                s_binfo[3] = bi.w;
            }
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
        const int row0 = s_binfo[0], nrows = s_binfo[1];
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
                L.Wx[2 * k] = make_float2(la[4], la[5]);
                L.Wx[2 * k + 1] = make_float2(lb[4], lb[5]);
            }
            float* rt = rtab + (size_t)warp * 4 * 128 + 4 * lane;
#pragma unroll
            for (int rs = 0; rs < 4; ++rs)
                *reinterpret_cast<float4*>(rt + rs * 128) =
                    make_float4(lc[7 + rs], lc[kLaneConsts + 7 + rs], lc[2 * kLaneConsts + 7 + rs], lc[3 * kLaneConsts + 7 + rs]);
        }
        const int par = a.parity;
        // specular wall parts (Eq. 5, alpha < 1): face stores of the previous iteration (read) and
        // of this one (written), at this lane's four slots; x1 faces are told apart by the
        // quadrant's x2 sign bit, x2 faces by its x1 bit
        const float* fprev1 = nullptr;
        const float* fprev2 = nullptr;
        float* fnext1 = nullptr;
        float* fnext2 = nullptr;
        float2 specP = make_float2(0.f, 0.f);
        if constexpr (SPEC) {
            const size_t plane = (size_t)P->nfaces * 2 * NL;
            fprev1 = P->F + par * plane + (size_t)s2neg * NL + kVL * wl;
            fprev2 = P->F + par * plane + (size_t)s1neg * NL + kVL * wl;
            fnext1 = P->F + (par ^ 1) * plane + (size_t)s2neg * NL + kVL * wl;
            fnext2 = P->F + (par ^ 1) * plane + (size_t)s1neg * NL + kVL * wl;
            specP = dup((float)P->spec);
        }
        // x1 carry from a lagged slot (the x1 ghosts, or with x1 subdomains a subdomain halo of the
        // previous iteration) / into a slot for the next iteration
        auto carry_in = [&](int slot) {
            const float* g = XS ? P->gx1 + (((size_t)(par * 4 + q) * P->nxslots + slot) * n2) * 2 * NL
                                : P->gx1 + (((size_t)par * 4 + q) * n2) * 2 * NL;
            for (int r = 0; r < nrows; ++r) {
                float* cr = carry + ((size_t)(warp * RB + r) * 2) * 128 + 4 * lane;
                *reinterpret_cast<float4*>(cr) = *reinterpret_cast<const float4*>(g + ((size_t)(row0 + r) * 2 + 0) * NL + kVL * wl);
                *reinterpret_cast<float4*>(cr + 128) = *reinterpret_cast<const float4*>(g + ((size_t)(row0 + r) * 2 + 1) * NL + kVL * wl);
            }
        };
        auto carry_out = [&](int slot) {
            float* g = XS ? P->gx1 + (((size_t)((par ^ 1) * 4 + q) * P->nxslots + slot) * n2) * 2 * NL
                          : P->gx1 + (((size_t)(par ^ 1) * 4 + q) * n2) * 2 * NL;
            for (int rr = 0; rr < nrows; ++rr) {
                const float* cr = carry + ((size_t)(warp * RB + rr) * 2) * 128 + 4 * lane;
                *reinterpret_cast<float4*>(g + ((size_t)(row0 + rr) * 2 + 0) * NL + kVL * wl) = *reinterpret_cast<const float4*>(cr);
                *reinterpret_cast<float4*>(g + ((size_t)(row0 + rr) * 2 + 1) * NL + kVL * wl) = *reinterpret_cast<const float4*>(cr + 128);
            }
        };
        if constexpr (!XS) carry_in(0);
        const int ntiles = XS ? P->ntq[q] : (n1 + T1 - 1) / T1;
        // with x1 subdomains, tile tt of this quadrant: {first oriented column, width, carry slot
        // in, carry slot out}; otherwise tiles are uniform
        auto tinfo = [&](int tt) -> int4 { return __ldg(P->tiles + (size_t)q * P->ntiles + tt); };
        const int npts = nrows * T1;
        const int rounds = (npts + blockDim.x - 1) / blockDim.x;

        auto load_raw = [&](int tt, RawPoint (&raw)[kMaxRounds]) {
#pragma unroll
            for (int k = 0; k < kMaxRounds; ++k) {
                raw[k].code = kSolidBit;
                const int idx = k * blockDim.x + threadIdx.x;
                if (k < rounds && idx < npts) {
                    const int r = idx / T1;
                    int ic;
                    bool inside;
                    if constexpr (XS) {
                        const int4 ti = tinfo(tt);
                        ic = ti.x + (idx - r * T1);
                        inside = idx - r * T1 < ti.y;
                    } else {
                        ic = tt * T1 + (idx - r * T1);
                        inside = ic < n1;
                    }
                    if (inside) {
                        const int x = s1neg ? n1 - 1 - ic : ic;
                        const int yo = row0 + r;
                        const int y = s2neg ? n2 - 1 - yo : yo;
                        const int id = y * n1 + x;
                        // every load is issued without waiting for the code: a branch on it would
                        // expose one more global-memory latency per tile (values of solid points
                        // are loaded and dropped)
                        raw[k].code = P->code[id];
                        raw[k].s = reinterpret_cast<const float4*>(P->src)[id];
                        raw[k].e = reinterpret_cast<const float4*>(P->E)[id];
                        if constexpr (SPEC) {
                            const int* fi = P->face_id;
                            const size_t Nn = (size_t)N;
                            raw[k].f = make_int4(fi[(0 + s1neg) * Nn + id], fi[(2 + s2neg) * Nn + id],
                                                 fi[(1 - s1neg) * Nn + id], fi[(3 - s2neg) * Nn + id]);
                        }
                    }
                }
            }
        };
        auto store_rec = [&](int buf, const RawPoint (&raw)[kMaxRounds]) {
            float* rb = rec + (size_t)buf * RB * T1 * RF;
            unsigned* mk = rmask + buf * RB;
#pragma unroll
            for (int k = 0; k < kMaxRounds; ++k) {
                if (k >= rounds) break;
                const int idx = k * blockDim.x + threadIdx.x;
                const bool fluid = idx < npts && !(raw[k].code & kSolidBit);
                if (idx < npts) {
                    float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f), o1 = o0, o2 = o0;
                    if (fluid) {
                        const int code = raw[k].code;
                        const int ca = (code >> (2 * (0 + s1neg))) & 3;
                        const int cb = (code >> (2 * (2 + s2neg))) & 3;
                        const float E1 = s1neg ? raw[k].e.y : raw[k].e.x;
                        const float E2 = s2neg ? raw[k].e.w : raw[k].e.z;
                        // first-order denominator when either upstream point is solid (cases 1, 2)
                        const int rs = (ca != 0) | ((cb != 0) << 1);
                        o0 = make_float4(raw[k].s.x, raw[k].s.y, raw[k].s.z, __int_as_float(rs * 128));
                        o1 = make_float4(E1, ca == 2 ? 0.f : (ca == 1 ? 1.f : K1o), ca == 0 ? K2o : 0.f, E2);
                        o2 = make_float4(cb == 2 ? 0.f : (cb == 1 ? 1.f : K1o), cb == 0 ? K2o : 0.f, 0.f, 0.f);
                    }
                    float4* R = reinterpret_cast<float4*>(rb + (size_t)idx * RF);
                    R[0] = o0;
                    R[1] = o1;
                    R[2] = o2;
                    if constexpr (SPEC)
                        reinterpret_cast<int4*>(R)[3] = fluid ? raw[k].f : make_int4(-1, -1, -1, -1);
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
        // progress of the band below that thread 0 has already observed with an acquire (tiles up
        // to it need no new wait)
        int seenb = -1;
        for (int t = 0; t < ntiles; ++t) {
            int c0, width, cout_slot;
            if constexpr (XS) {
                const int4 tcur = tinfo(t);
                c0 = tcur.x;
                width = tcur.y;
                cout_slot = tcur.w;
                if (tcur.z >= 0) carry_in(tcur.z);
            } else {
                c0 = t * T1;
                width = min(T1, n1 - c0);
                cout_slot = (t == ntiles - 1) ? 0 : -1;
            }
            const int buf = t & 1;
            RawPoint nxt[kMaxRounds];
            if (t + 1 < ntiles) load_raw(t + 1, nxt);
            if (threadIdx.x == 0 && s_binfo[2] < 0 && seenb < t + 1) {
                seenb = wait_geq_value(P->prog + q * nb + band - 1, t + 1, a.status, a.timeout_ns);
                if (seenb < 0) s_abort = 1;
            }
            __syncthreads();
            if (s_abort) return;
            const float* rbuf = rec + (size_t)buf * RB * T1 * RF;
            const unsigned* mk = rmask + buf * RB;
            for (int u = 0; u < NSUB; ++u) {
            const int cs = c0 + u * SW;                       // first column of the sub-tile
            const int wsub = min(SW, width - u * SW);         // its width
            if (wsub <= 0) break;
            const int us = u * SW;
            // fluid bits of row r in this sub-tile
            auto fbits = [&](int r) -> unsigned { return (mk[r] >> us) & ((1u << SW) - 1u); };
            if constexpr (NSUB > 1) {
                // a sub-tile without fluid is not swept (its edge and carries are read by no fluid
                // point: every fluid reader has a zero coefficient for them)
                unsigned any = 0u;
                for (int r = lane; r < nrows; r += 32) any |= fbits(r);
                if (!__any_sync(0xffffffffu, any != 0u)) continue;
            }
            const float* rsub = rbuf + (size_t)us * RF;       // record of (row 0, column cs)
            // the two rows below: previous band's top edge or the x2 ghost layers
            float4 rb1[SW], rb2[SW];
            {
                const int below = s_binfo[2];
                const float* eb = (below >= 0)
                    ? P->glat + (((size_t)(par * 4 + q) * P->nslots + below) * n1) * 2 * NL
                    : P->edge + ((size_t)(q * 2 * P->nslots + (-1 - below)) * n1) * 2 * NL;
#pragma unroll
                for (int i = 0; i < SW; ++i) {
                    if (i < wsub) {
                        rb1[i] = __ldcg(reinterpret_cast<const float4*>(eb + ((size_t)(cs + i) * 2 + 0) * NL + kVL * wl));
                        rb2[i] = __ldcg(reinterpret_cast<const float4*>(eb + ((size_t)(cs + i) * 2 + 1) * NL + kVL * wl));
                    } else {
                        rb1[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                        rb2[i] = rb1[i];
                    }
                }
            }
            // one point of a row: Eq. 10 for the lane's four velocities, with the x1 upstream values
            // (hp1, hp2) carried along the row and the x2 upstream values (u1, u2) of its column;
            // returns the lane's moment sums of the point: (rho, u1) and u2
            auto point = [&](const float* rrow, int i, float2 (&hp1)[2], float2 (&hp2)[2], float4& u1, float4& u2,
                             float2& M01, float& m2) {
                const float4* Rp = reinterpret_cast<const float4*>(rrow + i * RF);
                const float4 A = Rp[0];                 // a b1 b2 roff
                const float4 B = Rp[1];                 // E1 K1x K2x E2
                const float2 C = *reinterpret_cast<const float2*>(Rp + 2);   // K1y K2y
                // specular parts of the upstream wall values: (1 - alpha) h'(x, reflected v)
                int4 Fi = make_int4(-1, -1, -1, -1);
                float4 Fx = make_float4(0.f, 0.f, 0.f, 0.f), Fy = Fx;
                if constexpr (SPEC) {
                    Fi = reinterpret_cast<const int4*>(Rp)[3];
                    if (Fi.x >= 0) Fx = *reinterpret_cast<const float4*>(fprev1 + (size_t)Fi.x * 2 * NL);
                    if (Fi.y >= 0) Fy = *reinterpret_cast<const float4*>(fprev2 + (size_t)Fi.y * 2 * NL);
                }
                const float4 Rv = *reinterpret_cast<const float4*>(my_rtab + __float_as_int(A.w));
                const float2 aP = dup(A.x), b1P = dup(A.y), b2P = dup(A.z);
                const float2 E1P = dup(B.x), K1xP = dup(B.y), K2xP = dup(B.z), E2P = dup(B.w);
                const float2 K1yP = dup(C.x), K2yP = dup(C.y);
                const float2 rb1a = make_float2(u1.x, u1.y), rb1b = make_float2(u1.z, u1.w);
                const float2 rb2a = make_float2(u2.x, u2.y), rb2b = make_float2(u2.z, u2.w);
                float2 h[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float2 up1 = k ? rb1b : rb1a;
                    const float2 up2 = k ? rb2b : rb2a;
                    const float2 S = fma2(b2P, L.v2[k], fma2(b1P, L.v1[k], aP));
                    float2 t2 = fma2(K1yP, up1, fma2(K2yP, up2, E2P));
                    if constexpr (SPEC) t2 = fma2(specP, k ? make_float2(Fy.z, Fy.w) : make_float2(Fy.x, Fy.y), t2);
                    const float2 base = fma2(L.a2[k], t2, S);
                    float2 t1 = fma2(K1xP, hp1[k], fma2(K2xP, hp2[k], E1P));
                    if constexpr (SPEC) t1 = fma2(specP, k ? make_float2(Fx.z, Fx.w) : make_float2(Fx.x, Fx.y), t1);
                    const float2 Rk = k ? make_float2(Rv.z, Rv.w) : make_float2(Rv.x, Rv.y);
                    h[k] = mul2(fma2(L.a1[k], t1, base), Rk);
                    hp2[k] = hp1[k];
                    hp1[k] = h[k];
                }
                u2 = u1;
                u1 = make_float4(h[0].x, h[0].y, h[1].x, h[1].y);
                if constexpr (SPEC) {   // molecules moving into a downstream face
                    if (Fi.z >= 0) *reinterpret_cast<float4*>(fnext1 + (size_t)Fi.z * 2 * NL) = u1;
                    if (Fi.w >= 0) *reinterpret_cast<float4*>(fnext2 + (size_t)Fi.w * 2 * NL) = u1;
                }
                M01 = fma2(L.Wx[3], dup(h[1].y), fma2(L.Wx[2], dup(h[1].x), fma2(L.Wx[1], dup(h[0].y), mul2(L.Wx[0], dup(h[0].x)))));
                const float2 p2 = fma2(L.Wv2[1], h[1], mul2(L.Wv2[0], h[0]));
                m2 = p2.x + p2.y;
            };
            auto load_carry = [&](int r, float2 (&hp1)[2], float2 (&hp2)[2]) {
                const float* cr = carry + ((size_t)(warp * RB + r) * 2) * 128 + 4 * lane;
                const float4 c1 = *reinterpret_cast<const float4*>(cr);
                const float4 c2 = *reinterpret_cast<const float4*>(cr + 128);
                hp1[0] = make_float2(c1.x, c1.y);
                hp1[1] = make_float2(c1.z, c1.w);
                hp2[0] = make_float2(c2.x, c2.y);
                hp2[1] = make_float2(c2.z, c2.w);
            };
            auto store_carry = [&](int r, const float2 (&hp1)[2], const float2 (&hp2)[2]) {
                float* cr = carry + ((size_t)(warp * RB + r) * 2) * 128 + 4 * lane;
                *reinterpret_cast<float4*>(cr) = make_float4(hp1[0].x, hp1[0].y, hp1[1].x, hp1[1].y);
                *reinterpret_cast<float4*>(cr + 128) = make_float4(hp2[0].x, hp2[0].y, hp2[1].x, hp2[1].y);
            };
            // Rows are walked two at a time, the upper one a column behind the lower (it needs the
            // lower row's value of the same column), which gives every step two independent points;
            // the moments of both rows are then reduced together.  A pair is skipped when neither
            // row has fluid in the sub-tile; an empty row of a pair is swept anyway: its zero
            // records give h = 0, which no fluid point reads (its code marks that upstream point
            // solid), so the result is the same as with the row skipped.
            auto walk_rows = [&](auto full_tag) {
                constexpr bool FULL = decltype(full_tag)::value;
                int r = 0;
                for (; r + 1 < nrows; r += 2) {
                    if ((fbits(r) | fbits(r + 1)) == 0u) continue;
                    float2 hA1[2], hA2[2], hB1[2], hB2[2];
                    load_carry(r, hA1, hA2);
                    load_carry(r + 1, hB1, hB2);
                    const float* rowA = rsub + (size_t)r * T1 * RF;
                    const float* rowB = rowA + (size_t)T1 * RF;
                    float2 M01[2 * SW];
                    float m2[2 * SW];
#pragma unroll
                    for (int st = 0; st <= SW; ++st) {
                        if (st < SW) {
                            const int i = st;
                            if (FULL || i < wsub) point(rowA, i, hA1, hA2, rb1[i], rb2[i], M01[i], m2[i]);
                            else {
                                M01[i] = make_float2(0.f, 0.f);
                                m2[i] = 0.f;
                            }
                        }
                        if (st >= 1) {
                            const int i = st - 1;
                            if (FULL || i < wsub) point(rowB, i, hB1, hB2, rb1[i], rb2[i], M01[SW + i], m2[SW + i]);
                            else {
                                M01[SW + i] = make_float2(0.f, 0.f);
                                m2[SW + i] = 0.f;
                            }
                        }
                    }
                    store_carry(r, hA1, hA2);
                    store_carry(r + 1, hB1, hB2);
                    const float2 s01 = reduce_scatter2<2 * SW>(M01, lane);
                    const float s2 = reduce_scatter<float, 2 * SW>(m2, lane);
                    // value v of the 2 SW ends in the lanes v * 32 / (2 SW) onward: row r + v / SW
                    if ((lane & (kLPP / 2 - 1)) == 0) {
                        const int v = lane / (kLPP / 2);
                        float* d = part + ((size_t)(warp * RB + r + v / SW) * T1 + us + (v % SW)) * 4;
                        *reinterpret_cast<float4*>(d) = make_float4(s01.x, s01.y, s2, 0.f);
                    }
                }
                if (r < nrows && fbits(r) != 0u) {   // the last row of an odd band
                    float2 hp1[2], hp2[2];
                    load_carry(r, hp1, hp2);
                    const float* rrow = rsub + (size_t)r * T1 * RF;
                    float2 M01[SW];
                    float m2[SW];
#pragma unroll
                    for (int i = 0; i < SW; ++i) {
                        if (FULL || i < wsub) point(rrow, i, hp1, hp2, rb1[i], rb2[i], M01[i], m2[i]);
                        else {
                            M01[i] = make_float2(0.f, 0.f);
                            m2[i] = 0.f;
                        }
                    }
                    store_carry(r, hp1, hp2);
                    const float2 s01 = reduce_scatter2<SW>(M01, lane);
                    const float s2 = reduce_scatter<float, SW>(m2, lane);
                    if ((lane & (kLPP - 1)) == 0) {
                        float* d = part + ((size_t)(warp * RB + r) * T1 + us + lane / kLPP) * 4;
                        *reinterpret_cast<float4*>(d) = make_float4(s01.x, s01.y, s2, 0.f);
                    }
                }
            };
            if (wsub == SW) walk_rows(std::integral_constant<bool, true>{});
            else walk_rows(std::integral_constant<bool, false>{});
            // band edge for the band above, or the x2 ghost layers of the next iteration (Eq. 8 /
            // periodic: the reflected quadrant reads the same lane)
            {
                float* et;
                const int above = s_binfo[3];
                if (above < 0) {
                    et = P->edge + ((size_t)(q * 2 * P->nslots + (-1 - above)) * n1) * 2 * NL;
                } else {
                    const int qd = (above > 0 || P->lateral == 1) ? q : (q ^ 2);
                    et = P->glat + (((size_t)((par ^ 1) * 4 + qd) * P->nslots + above) * n1) * 2 * NL;
                }
#pragma unroll
                for (int i = 0; i < SW; ++i) {
                    if (i < wsub) {
                        *reinterpret_cast<float4*>(et + ((size_t)(cs + i) * 2 + 0) * NL + kVL * wl) = rb1[i];
                        *reinterpret_cast<float4*>(et + ((size_t)(cs + i) * 2 + 1) * NL + kVL * wl) = rb2[i];
                    }
                }
            }
            }   // sub-tiles
            // x1 ghost layers of the next iteration (periodic in x1, same quadrant) or the halo of
            // the next x1 subdomain
            if (cout_slot >= 0) carry_out(cout_slot);
            __syncthreads();
            if (threadIdx.x == 0 && it != a.withhold_item) publish_gpu(P->prog + q * nb + band, t + 1);
            // (the next tile's records after the publish: its readers are behind the next tile's
            // first barrier)
            if (t + 1 < ntiles) store_rec(buf ^ 1, nxt);
            // moment partials of this quadrant: sum of the warps' lane sums, in warp order, a thread
            // per point (pt = rr T1 + i; only fluid points have bits, and only their partials are read)
            {
                const unsigned* mk = rmask + buf * RB;
                for (int pt = threadIdx.x; pt < nrows * T1; pt += blockDim.x) {
                    const int rr = pt / T1;
                    const int i = pt % T1;
                    if (!((mk[rr] >> i) & 1u)) continue;
                    float4 sv = *reinterpret_cast<const float4*>(part + (size_t)pt * 4);
                    for (int w = 1; w < NW; ++w) {
                        const float4 o = *reinterpret_cast<const float4*>(part + ((size_t)w * RB * T1 + pt) * 4);
                        sv.x += o.x;
                        sv.y += o.y;
                        sv.z += o.z;
                    }
                    const int ic = c0 + i;
                    const int x = s1neg ? n1 - 1 - ic : ic;
                    const int yo = row0 + rr;
                    const int y = s2neg ? n2 - 1 - yo : yo;
                    float* d = P->P + (size_t)q * 3 * N + (size_t)y * n1 + x;
                    d[0] = sv.x;
                    d[N] = sv.y;
                    d[2 * (size_t)N] = sv.z;
                }
            }
        }
        __syncthreads();
    }
}

size_t sweep2d_f32x2_smem(int T1, int NW, int max_rows, int spec) {
    return sizeof(float) * ((size_t)2 * max_rows * T1 * (spec ? 16 : kRecF) + (size_t)NW * max_rows * T1 * 4 +
                            (size_t)NW * max_rows * 2 * 128 + (size_t)NW * 4 * 128) +
           sizeof(unsigned) * (size_t)2 * max_rows;
}

int sweep2d_f32x2_max_rows(int T1, int NW) { return kMaxRounds * NW * 32 / T1; }

int sweep2d_f32x2_velocities_per_lane() { return kVL; }

template <int T1, bool XS, bool SPEC>
static cudaError_t launch_f32x2_t(const SweepArgs2D<float>& a, int grid, int NW, cudaStream_t st) {
    const size_t smem = sweep2d_f32x2_smem(T1, NW, a.max_rows, SPEC);
    cudaError_t e = cudaFuncSetAttribute(sweep2d_f32x2_kernel<T1, XS, SPEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sweep2d_f32x2_kernel<T1, XS, SPEC><<<grid, NW * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int T1>
static cudaError_t launch_f32x2_tt(const SweepArgs2D<float>& a, int xs, int grid, int NW, cudaStream_t st) {
    if (a.spec) return xs ? launch_f32x2_t<T1, true, true>(a, grid, NW, st) : launch_f32x2_t<T1, false, true>(a, grid, NW, st);
    return xs ? launch_f32x2_t<T1, true, false>(a, grid, NW, st) : launch_f32x2_t<T1, false, false>(a, grid, NW, st);
}

// xs: x1 subdomains (tile tables and lagged x1 halos); a.spec: specular wall parts
cudaError_t launch_sweep2d_f32x2(const SweepArgs2D<float>& a, int T1, int xs, int grid, int NW, cudaStream_t st) {
    if (T1 == 16) return launch_f32x2_tt<16>(a, xs, grid, NW, st);
    if (T1 == 8) return launch_f32x2_tt<8>(a, xs, grid, NW, st);
    if (T1 == 4) return launch_f32x2_tt<4>(a, xs, grid, NW, st);
    return cudaErrorInvalidValue;
}

template <int T1, bool XS, bool SPEC>
static cudaError_t occupancy_f32x2_t(int NW, int max_rows, int* blocks_per_sm) {
    const size_t smem = sweep2d_f32x2_smem(T1, NW, max_rows, SPEC);
    cudaError_t e = cudaFuncSetAttribute(sweep2d_f32x2_kernel<T1, XS, SPEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, sweep2d_f32x2_kernel<T1, XS, SPEC>, NW * 32, smem);
}

template <int T1>
static cudaError_t occupancy_f32x2_tt(int xs, int spec, int NW, int max_rows, int* bps) {
    if (spec) return xs ? occupancy_f32x2_t<T1, true, true>(NW, max_rows, bps) : occupancy_f32x2_t<T1, false, true>(NW, max_rows, bps);
    return xs ? occupancy_f32x2_t<T1, true, false>(NW, max_rows, bps) : occupancy_f32x2_t<T1, false, false>(NW, max_rows, bps);
}

cudaError_t sweep2d_f32x2_occupancy(int T1, int xs, int spec, int NW, int max_rows, int* blocks_per_sm) {
    if (T1 == 16) return occupancy_f32x2_tt<16>(xs, spec, NW, max_rows, blocks_per_sm);
    if (T1 == 8) return occupancy_f32x2_tt<8>(xs, spec, NW, max_rows, blocks_per_sm);
    if (T1 == 4) return occupancy_f32x2_tt<4>(xs, spec, NW, max_rows, blocks_per_sm);
    return cudaErrorInvalidValue;
}

}  // namespace dvm
