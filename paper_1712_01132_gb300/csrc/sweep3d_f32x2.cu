// sweep3d_f32x2.cu -- FP32 transport sweep of one source iteration in 3D (arXiv:1712.01132,
// Sec. 3.1 step i with the quadrature of step iii fused), two discrete velocities per lane.
//
// Same schedule and data layout as sweep3d_kernel (work items (problem, octant, velocity group,
// pencil) in pencil-level order, pencils of R2 x R3 rows swept along x1 in tiles of T1 columns,
// waits on the x2 and x3 neighbour pencils), but every lane carries the two consecutive velocity
// slots 2 l and 2 l + 1 of its group as one packed pair, updated with fma.rn.f32x2: the per-point
// record loads and the cross-lane quadrature are shared by two velocities.  Per point and pair:
//   h = R * [ S + a1 (K1x h(x - s1 e1) + K2x h(x - 2 s1 e1) + E1)
//               + a2 (K1y ... + E2) + a3 (K1z ... + E3) ],  S = a + b1 v1 + b2 v2 + b3 v3
// (Eq. 10 solved for h with the upwind stencil of Eq. 9, source form).  The moment sums of a point
// are formed in a fixed order (pair, lane tree, warps), independent of tile and pencil shapes.
// Solid points are not swept; upstream data is staged per warp with cp.async; a tile of T1 = 4 or
// 8 columns is swept as 4-column sub-tiles (one neighbour wait, one publish, one record load and
// one pass of moment partials per tile); the rows of a plane are walked two at a time, the upper
// row a column behind the lower; the next tile's point data is loaded while the current tile is
// swept; the pencil's top two rows and planes go to the neighbours' edge rings as they are swept;
// thread 0 re-reads a neighbour's progress flag only for tiles beyond the value it last observed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "dvm_device.cuh"
#include "dvm_internal.h"

namespace dvm {

namespace {

constexpr int kRec = 16;    // record floats: {a b1 b2 b3} {E1 E2 E3 rsel} {K1x K2x K1y K2y} {K1z K2z - -}
constexpr int kPL = 64;     // velocity slots per warp (32 lanes x 2)
constexpr int kSubW = 4;    // columns of a sub-tile: the upstream staging and the skewed row-pair walk

// transient h in HBM (ghost layers, pencil edges) as float pairs, or the BF16 deviations from the
// x1 ramp (the BF16-storage ablation): h' - x1 of the point the pair belongs to
template <bool BF> struct PairStore {
    static __device__ __forceinline__ float2 ld(const float* b, size_t i, float) {
        return __ldcg(reinterpret_cast<const float2*>(b + i));
    }
    static __device__ __forceinline__ void st(float* b, size_t i, float2 v, float) {
        *reinterpret_cast<float2*>(b + i) = v;
    }
};
template <> struct PairStore<true> {
    static __device__ __forceinline__ float2 ld(const float* b, size_t i, float x1) {
        const unsigned u = __ldcg(reinterpret_cast<const unsigned*>(reinterpret_cast<const __nv_bfloat16*>(b) + i));
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
        return make_float2(f.x + x1, f.y + x1);
    }
    static __device__ __forceinline__ void st(float* b, size_t i, float2 v, float x1) {
        *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(b) + i) =
            __floats2bfloat162_rn(v.x - x1, v.y - x1);
    }
};

__device__ __forceinline__ float2 dup2(float x) { return make_float2(x, x); }

// global data of one point that its record is built from, loaded one tile ahead
struct RawPoint3 {
    int code;
    float4 s, e0, e1;
    float st;
    int4 f0, f1;
};
constexpr int kRawRounds = 1;   // points per thread held in registers across a tile

// 16-byte asynchronous copy global -> shared that bypasses L1 (pencil edges are written by other
// SMs during the launch), and its group commit / wait
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
// the same copy, or (need == false) 16 zero bytes without reading global memory
__device__ __forceinline__ void cp_async16_or_zero(void* smem_dst, const void* gmem_src, bool need) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    const unsigned n = need ? 16u : 0u;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gmem_src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace

template <int T1, bool BF, bool SUB, bool TAU, bool SPEC>
__global__ void __launch_bounds__(256) sweep3d_f32x2_kernel(const SweepArgs3D<float> a) {
    using PS = PairStore<BF>;
    constexpr int NM = TAU ? 5 : 4;         // moments per point: rho, u1..u3 (, sum W |v|^2 h)
    constexpr int RF = SPEC ? 24 : kRec;    // record floats (face ids in two more vectors)
    constexpr int SW = kSubW;               // columns of a sub-tile (staging width)
    constexpr int NSUB = T1 / SW;           // sub-tiles per tile
    static_assert(T1 % SW == 0 && T1 <= 32 && 32 % T1 == 0, "tile width: a multiple of the sub-tile width, dividing 32");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    __shared__ int s_abort;
    const int NW = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int MR2 = a.maxR2, MR3 = a.maxR3;
    const int MROWS = MR2 * MR3;
    float* rec = reinterpret_cast<float*>(smem_raw);                      // [2][MROWS][T1][RF]
    float* part = rec + (size_t)2 * MROWS * T1 * RF;                      // [NW][MROWS][T1][NM]
    float* carry = part + (size_t)NW * MROWS * T1 * NM;                   // [NW][MROWS][2][64]
    float* pb = carry + (size_t)NW * MROWS * 2 * kPL;                     // [NW][MR2][2][SW][64]
    float* eb = pb + (size_t)NW * MR2 * 2 * SW * kPL;                     // [NW][2][2][SW][64]
    float* rtab = eb + (size_t)NW * 2 * 2 * SW * kPL;                     // [NW][8][64]
    unsigned* fmask = reinterpret_cast<unsigned*>(rtab + (size_t)NW * 8 * kPL);   // [2][MROWS] fluid bits
    int* rowoff = reinterpret_cast<int*>(fmask + 2 * MROWS);   // [MROWS] first point of a row, or -1
    const size_t NL = (size_t)a.NL;
    // When the CTA has a thread for every point of a tile, a tile's fluid bits are formed by warp
    // votes and written whole (no clearing, no atomics, and no barrier between the moment partials
    // of one tile and the next tile); otherwise they are cleared and set with atomicOr.
    const bool bmask = MROWS * T1 <= (int)blockDim.x;

    for (;;) {
        if (threadIdx.x == 0) {
            s_item = ld_volatile(a.status) ? a.nitems : atomicAdd(a.ticket, 1);
            s_abort = 0;
        }
        if (!bmask)
            for (int r = threadIdx.x; r < MROWS; r += blockDim.x) fmask[r] = 0u;    // masks of tile 0
        __syncthreads();
        const int it = s_item;
        if (it >= a.nitems) return;
        const SweepItem3 item = a.items[it];
        const Prob3D<float>* __restrict__ P = a.prob + item.prob;
        const int q = item.oct, g = item.group, p2 = item.p2, p3 = item.p3;
        const int n1 = P->n1, n2 = P->n2, n3 = P->n3;
        const int N = P->N;
        const int np2 = P->np2, np3 = P->np3;
        const int s1n = q & 1, s2n = (q >> 1) & 1, s3n = (q >> 2) & 1;
        // the pencil's rows and where its upstream rows come from / its top rows go (Prob3D)
        int4 pi2, pi3;
        if constexpr (SUB) {
            pi2 = P->pen2[s2n * np2 + p2];
            pi3 = P->pen3[s3n * np3 + p3];
        } else {
            pi2 = make_int4(p2 * P->R2, min(P->R2, n2 - p2 * P->R2), p2 == 0 ? 0 : -1 - ((p2 - 1) & 1),
                            p2 == np2 - 1 ? 0 : -1 - (p2 & 1));
            pi3 = make_int4(p3 * P->R3, min(P->R3, n3 - p3 * P->R3), p3 == 0 ? 0 : -1 - ((p3 - 1) & 1),
                            p3 == np3 - 1 ? 0 : -1 - (p3 & 1));
        }
        const int j0 = pi2.x, nr2 = pi2.y, k0 = pi3.x, nr3 = pi3.y;
        // point index (z n2 + y) n1 of the first column of pencil row r = kk MR2 + jj, or -1 for a
        // row outside the pencil: per thread for the point it loads each tile (thread idx holds
        // point idx = (r, i) = (idx / T1, idx % T1)), in shared memory for the moment partials
        auto row_first = [&](int r) -> int {
            const int kk = r / MR2, jj = r - kk * MR2;
            if (kk >= nr3 || jj >= nr2) return -1;
            const int y = s2n ? n2 - 1 - (j0 + jj) : (j0 + jj);
            const int z = s3n ? n3 - 1 - (k0 + kk) : (k0 + kk);
            return (z * n2 + y) * n1;
        };
        for (int r = threadIdx.x; r < MROWS; r += blockDim.x) rowoff[r] = row_first(r);
        const int my_r = (int)threadIdx.x / T1, my_i = (int)threadIdx.x % T1;
        const int my_off = my_r < MROWS ? row_first(my_r) : -1;
        const float K1o = P->order == 2 ? 2.f : 1.f;
        const float K2o = P->order == 2 ? -0.5f : 0.f;
        const int lv = g * a.GL + kPL * warp + 2 * lane;      // first velocity slot of this lane
        const float* la = P->lanec + ((size_t)q * NL + lv) * kLaneConsts3;
        const float* lb = la + kLaneConsts3;
        const float2 v1 = make_float2(la[0], lb[0]), v2 = make_float2(la[1], lb[1]), v3 = make_float2(la[2], lb[2]);
        const float2 a1 = make_float2(la[3], lb[3]), a2 = make_float2(la[4], lb[4]), a3 = make_float2(la[5], lb[5]);
        const float2 W = make_float2(la[6], lb[6]), Wv1 = make_float2(la[7], lb[7]);
        const float2 Wv2 = make_float2(la[8], lb[8]), Wv3 = make_float2(la[9], lb[9]);
        // moment weights regrouped by velocity slot: (rho, u1) and (u2, u3) of slot 2 l and of 2 l + 1
        const float2 Wa01 = make_float2(W.x, Wv1.x), Wb01 = make_float2(W.y, Wv1.y);
        const float2 Wa23 = make_float2(Wv2.x, Wv3.x), Wb23 = make_float2(Wv2.y, Wv3.y);
        // temperature term: |v|^2 - 3/2 and W |v|^2
        const float2 vq = make_float2(la[18], lb[18]), Wvv = make_float2(la[19], lb[19]);
        float* my_rtab = rtab + (size_t)warp * 8 * kPL + 2 * lane;
#pragma unroll
        for (int rs = 0; rs < 8; ++rs)
            *reinterpret_cast<float2*>(my_rtab + rs * kPL) = make_float2(la[10 + rs], lb[10 + rs]);
        const int par = a.parity;
        const int G = P->ngroups;
        int* prog = P->prog + ((size_t)q * G + g) * np3 * np2;
        // specular wall parts (Eq. 5, alpha < 1): face stores of the previous iteration (read where
        // an upstream point is solid) and of this one (written where a downstream point is solid),
        // at this lane's two slots
        const float* fprev[3] = {nullptr, nullptr, nullptr};
        float* fnext[3] = {nullptr, nullptr, nullptr};
        const size_t fstride = 4 * NL;
        if constexpr (SPEC) {
            const size_t plane = (size_t)P->nfaces * 4 * NL;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                fprev[j] = P->F + par * plane + (size_t)other_bits3(q, j) * NL + lv;
                fnext[j] = P->F + (par ^ 1) * plane + (size_t)other_bits3(q, j) * NL + lv;
            }
        }
        const float2 specP = dup2((float)P->spec);
        const float dxf = (float)P->dx;
        auto x1of = [&](int ic) -> float { return (float)(s1n ? n1 - 1 - ic : ic) * dxf; };
        const float x1g0 = x1of(n1 - 1), x1g1 = x1of(n1 - 2);   // columns of the x1 ghost layers
        // FP32 upstream data is staged per warp with asynchronous copies: the warp's 64 slots of
        // one (row, layer, column) are 256 contiguous bytes, copied as 16 lanes x 16 bytes (two
        // such per instruction); a lane reads its own 8 bytes after the wait and a __syncwarp
        const int hl = lane & 15, half = lane >> 4;
        const size_t lw = (size_t)g * a.GL + (size_t)kPL * warp + 4 * hl;
        const int ntiles = SUB ? P->nt1 : (n1 + T1 - 1) / T1;
        // tile: first oriented column, width, x1 carry-in and carry-out ghost slots (or -1)
        auto tile_info = [&](int tt) -> int4 {
            if constexpr (SUB) return P->tiles1[s1n * ntiles + tt];
            else return make_int4(tt * T1, min(T1, n1 - tt * T1), tt == 0 ? 0 : -1, tt == ntiles - 1 ? 0 : -1);
        };
        // records of a tile's points for this octant (shared by all lanes and velocities) and the
        // fluid bits of every row.  Point idx of a tile is (plane kk, row jj, column i); a thread's
        // points are loaded for tile t + 1 while tile t is swept (all loads issued together, with
        // no branch on the code) and written to that tile's record buffer at the end of tile t.
        const int npts = nr3 * MR2 * T1;
        // the problem's per-point arrays and this octant's and group's moment partials
        const uint16_t* __restrict__ pcode = P->code;
        const float4* __restrict__ psrc = reinterpret_cast<const float4*>(P->src);
        const float4* __restrict__ pE = reinterpret_cast<const float4*>(P->E);
        float* __restrict__ Pq = P->P + ((size_t)q * G + g) * 4 * (size_t)N;
        // point (row first index off, column i) of a tile (first column, width: tj.x, tj.y)
        auto load_point = [&](const int4& tj, int off, int i, RawPoint3& r) {
            r.code = kSolidBit;
            if (off >= 0 && i < tj.y) {
                const int ic = tj.x + i;
                const int x = s1n ? n1 - 1 - ic : ic;
                const int id = off + x;
                r.code = pcode[id];
                r.s = psrc[id];
                r.e0 = pE[2 * (size_t)id];
                r.e1 = pE[2 * (size_t)id + 1];
                if constexpr (TAU) r.st = P->srct[id];
                if constexpr (SPEC) {   // faces: upstream (read) x1 x2 x3, downstream (written)
                    const int* fi = P->face_id;
                    const size_t Nn = (size_t)N;
                    r.f0 = make_int4(fi[(0 + s1n) * Nn + id], fi[(2 + s2n) * Nn + id], fi[(4 + s3n) * Nn + id],
                                     fi[(1 - s1n) * Nn + id]);
                    r.f1 = make_int4(fi[(3 - s2n) * Nn + id], fi[(5 - s3n) * Nn + id], -1, -1);
                }
            }
        };
        auto store_point = [&](int buf, int idx, const RawPoint3& r) {
            float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0, r3 = r0;
            int4 r4 = make_int4(-1, -1, -1, -1), r5 = r4;
            const int i = idx % T1;
            if (!(r.code & kSolidBit)) {
                const int code = r.code;
                const int ca = (code >> (2 * (0 + s1n))) & 3;
                const int cb = (code >> (2 * (2 + s2n))) & 3;
                const int cc = (code >> (2 * (4 + s3n))) & 3;
                // first-order denominator when either upstream point is solid (cases 1, 2)
                const int rs = (ca != 0) | ((cb != 0) << 1) | ((cc != 0) << 2);
                r0 = r.s;
                r1 = make_float4(s1n ? r.e0.y : r.e0.x, s2n ? r.e0.w : r.e0.z, s3n ? r.e1.y : r.e1.x,
                                 __int_as_float(rs * kPL));
                r2 = make_float4(ca == 2 ? 0.f : (ca == 1 ? 1.f : K1o), ca == 0 ? K2o : 0.f,
                                 cb == 2 ? 0.f : (cb == 1 ? 1.f : K1o), cb == 0 ? K2o : 0.f);
                r3 = make_float4(cc == 2 ? 0.f : (cc == 1 ? 1.f : K1o), cc == 0 ? K2o : 0.f, TAU ? r.st : 0.f, 0.f);
                if constexpr (SPEC) {
                    r4 = r.f0;
                    r5 = r.f1;
                }
                if (!bmask) atomicOr(fmask + buf * MROWS + idx / T1, 1u << i);
            }
            float4* R = reinterpret_cast<float4*>(rec + (size_t)buf * MROWS * T1 * RF + (size_t)idx * RF);
            R[0] = r0;
            R[1] = r1;
            R[2] = r2;
            R[3] = r3;
            if constexpr (SPEC) {
                reinterpret_cast<int4*>(R)[4] = r4;
                reinterpret_cast<int4*>(R)[5] = r5;
            }
        };
        static_assert(kRawRounds == 1, "one register round: the thread's own point");
        auto load_raw = [&](int tt, RawPoint3 (&raw)[kRawRounds]) {
            const int4 tj = tile_info(tt);
            raw[0].code = kSolidBit;
            if ((int)threadIdx.x < npts) load_point(tj, my_off, my_i, raw[0]);
        };
        // the held points, then the points beyond the register rounds (loaded here)
        auto store_rec = [&](int tt, int buf, const RawPoint3 (&raw)[kRawRounds]) {
#pragma unroll
            for (int k = 0; k < kRawRounds; ++k) {
                const int idx = k * blockDim.x + threadIdx.x;
                if (idx < npts) store_point(buf, idx, raw[k]);
            }
            if (bmask) {   // row my_r's bits come from lanes my_r T1 .. my_r T1 + T1 - 1 (T1 divides 32)
                const unsigned b = __ballot_sync(0xffffffffu, !(raw[0].code & kSolidBit));
                if (my_i == 0 && my_r < MROWS) fmask[buf * MROWS + my_r] = (b >> lane) & ((1u << T1) - 1u);
            }
            if (kRawRounds * (int)blockDim.x < npts) {
                const int4 tj = tile_info(tt);
                for (int idx = kRawRounds * blockDim.x + threadIdx.x; idx < npts; idx += blockDim.x) {
                    RawPoint3 r;
                    load_point(tj, row_first(idx / T1), idx % T1, r);
                    store_point(buf, idx, r);
                }
            }
        };
        {   // tile 0 (its masks were cleared before the barrier that started the item)
            RawPoint3 raw[kRawRounds];
            load_raw(0, raw);
            store_rec(0, 0, raw);
        }
        // upstream data of a tile: x3 planes of its first plane (the pencil below in x3, ring slot,
        // or ghost slot pi3.z: the x3 ghost layers, periodic or specular, Eq. 8, or the lagged halo
        // of the block below) and x2 rows of each plane (likewise with pi2.z)
        const bool zg = pi3.z >= 0, yg = pi2.z >= 0;
        const float* zb = zg ? P->gz : P->ez;
        const size_t zo = zg
            ? ((((size_t)par * 8 + q) * P->ns3 + pi3.z) * n2 * n1) * 2 * NL
            : ((((size_t)q * np2 + p2) * 2 * P->ns3 + (-1 - pi3.z)) * P->R2 * n1) * 2 * NL;
        const float* yb = yg ? P->gy : P->ey;
        const size_t yo = yg
            ? ((((size_t)par * 8 + q) * P->ns2 + pi2.z) * n3 * n1) * 2 * NL
            : ((((size_t)q * np3 + p3) * 2 * P->ns2 + (-1 - pi2.z)) * P->R3 * n1) * 2 * NL;
        auto yrow = [&](int kk) -> size_t { return yg ? (size_t)(k0 + kk) * n1 : (size_t)kk * n1; };
        // where the pencil's top layers go, computed once per pencil: the x2 edge of plane kk, column
        // c, layer l at et2[eo2 + kk rowS + c colS + l NL] (the ring slot for the pencil above in x2,
        // or ghost slot pi2.w of the next iteration: the halo of the next block, or at the domain
        // face the x2 ghost layers, periodic: same octant, specular: s2 flipped); the x3 edge of row
        // jj at et3[eo3 + jj rowS + c colS + l NL] (likewise with pi3.w and s3)
        const size_t colS = 2 * NL, rowS = (size_t)n1 * colS;
        // the copies' sources (lane offset lw included): x2 rows of plane kk at yb[yo2 + kk rowS + ...],
        // x3 planes of row jj at zb[zo2 + jj rowS + ...]
        const size_t yo2 = yo + (yg ? (size_t)k0 * rowS : 0) + lw;
        const size_t zo2 = zo + (zg ? (size_t)j0 * rowS : 0) + lw;
        float* et2;
        size_t eo2;
        if (pi2.w < 0) {
            et2 = P->ey;
            eo2 = ((((size_t)q * np3 + p3) * 2 * P->ns2 + (-1 - pi2.w)) * P->R3 * n1) * 2 * NL + lv;
        } else {
            const int qy = (pi2.w > 0 || P->lateral == 1) ? q : (q ^ 2);
            et2 = P->gy;
            eo2 = ((((size_t)(par ^ 1) * 8 + qy) * P->ns2 + pi2.w) * n3 * n1) * 2 * NL + (size_t)k0 * rowS + lv;
        }
        float* et3;
        size_t eo3;
        if (pi3.w < 0) {
            et3 = P->ez;
            eo3 = ((((size_t)q * np2 + p2) * 2 * P->ns3 + (-1 - pi3.w)) * P->R2 * n1) * 2 * NL + lv;
        } else {
            const int qz = (pi3.w > 0 || P->lateral == 1) ? q : (q ^ 4);
            et3 = P->gz;
            eo3 = ((((size_t)(par ^ 1) * 8 + qz) * P->ns3 + pi3.w) * n2 * n1) * 2 * NL + (size_t)j0 * rowS + lv;
        }
        // FP32: the x2 rows of plane kk go to slot kk & 1, copied while plane kk - 1 is swept (the
        // sub-tile's columns cc0 .. cc0 + wd - 1, records rb: its first column in row 0).  Upstream
        // values are fetched only where the stencil of the point that reads them has a nonzero
        // coefficient for them (record K1 / K2 of the first row or plane): values of solid points
        // are never used, so they are neither stored nor fetched, and the staging holds zeros there.
        // (lane half h copies both layers of columns h, h + 2, ...; columns i >= wd are not copied)
        auto issue_y = [&](int kk, int cc0, int wd, const float* rb) {
            const float* ys = yb + yo2 + (size_t)kk * rowS + (size_t)cc0 * colS;
            float* yd = eb + (((size_t)warp * 2 + (kk & 1)) * 2 * SW) * kPL + 4 * hl;
            const float* yr = rb + (size_t)kk * MR2 * T1 * RF + 10;
#pragma unroll
            for (int u = 0; u < SW / 2; ++u) {
                const int i = half + 2 * u;
                if (i < wd) {
                    const float2 K = *reinterpret_cast<const float2*>(yr + i * RF);   // K1y, K2y
                    cp_async16_or_zero(yd + (size_t)i * kPL, ys + (size_t)(i * 2) * NL, K.x != 0.f);
                    cp_async16_or_zero(yd + (size_t)(SW + i) * kPL, ys + (size_t)(i * 2 + 1) * NL, K.y != 0.f);
                }
            }
            cp_async_commit();
        };
        // the x3 planes below the tile's first plane into the plane staging (committed with y(0)):
        // the plane just below (edge layer 0) into staging layer 1 and the one below it into layer
        // 0, where plane 0 reads them (the staging layer of plane kk - 1 is (kk + 1) & 1)
        auto issue_z = [&](int cc0, int wd, const float* rb) {
            const float* zs = zb + zo2 + (size_t)cc0 * colS;
            float* zd = pb + ((size_t)warp * MR2 * 2 * SW) * kPL + 4 * hl;
            const size_t zstride = rowS;
            for (int jj = 0; jj < nr2; ++jj) {
                const float* zr = rb + (size_t)jj * T1 * RF + 12;
#pragma unroll
                for (int u = 0; u < SW / 2; ++u) {
                    const int i = half + 2 * u;
                    if (i < wd) {
                        const float2 K = *reinterpret_cast<const float2*>(zr + i * RF);   // K1z, K2z
                        cp_async16_or_zero(zd + ((size_t)(jj * 2 + 1) * SW + i) * kPL, zs + jj * zstride + (size_t)(i * 2) * NL,
                                           K.x != 0.f);
                        cp_async16_or_zero(zd + ((size_t)(jj * 2) * SW + i) * kPL, zs + jj * zstride + (size_t)(i * 2 + 1) * NL,
                                           K.y != 0.f);
                    }
                }
            }
        };
        // does sub-tile u of a tile (its fluid bits) hold a fluid point?  (the same answer in every
        // warp; u = -1: the whole tile)
        auto has_fluid = [&](const unsigned* fm, int u) -> bool {
            const unsigned sel = u < 0 ? ((T1 == 32) ? 0xffffffffu : ((1u << T1) - 1u)) : (((1u << SW) - 1u) << (u * SW));
            unsigned any = 0u;
            for (int r = lane; r < MROWS; r += 32) any |= fm[r] & sel;
            return __any_sync(0xffffffffu, any != 0u);
        };
        // neighbour progress thread 0 has already observed with an acquire (tiles up to it need no
        // new wait: the release that published it covered every earlier tile's edges)
        int seen2 = pi2.z < 0 ? -1 : ntiles, seen3 = pi3.z < 0 ? -1 : ntiles;
        for (int t = 0; t < ntiles; ++t) {
            const int4 ti = tile_info(t);
            const int c0 = ti.x;
            const int width = ti.y;
            RawPoint3 nxt[kRawRounds];
            if (t + 1 < ntiles) load_raw(t + 1, nxt);
            if (threadIdx.x == 0) {
                if (seen2 < t + 1) seen2 = wait_geq_value(prog + p3 * np2 + p2 - 1, t + 1, a.status, a.timeout_ns);
                if (seen2 >= 0 && seen3 < t + 1) seen3 = wait_geq_value(prog + (p3 - 1) * np2 + p2, t + 1, a.status, a.timeout_ns);
                if (seen2 < 0 || seen3 < 0) s_abort = 1;
            }
            // the masks of the next tile are cleared here (their last reader, the moment loop of
            // the previous tile, is behind the barrier that ended it; they are set at the end of
            // this tile, behind the barrier below)
            unsigned* fm_cur = fmask + (t & 1) * MROWS;
            const float* recb = rec + (size_t)(t & 1) * MROWS * T1 * RF;
            if (!bmask)
                for (int r = threadIdx.x; r < MROWS; r += blockDim.x) fmask[((t + 1) & 1) * MROWS + r] = 0u;
            __syncthreads();
            if (s_abort) {
                cp_async_wait<0>();
                return;
            }
            // A tile (or sub-tile) without fluid points is not swept: nothing it would compute, copy
            // or store is read (every fluid reader of one of its points has a zero coefficient for
            // it, and the carries, staging and ghosts it leaves as they were hold finite values).  A
            // tile still waits for its neighbours and publishes, which keeps the ring slots' order.
            const bool tfl = has_fluid(fm_cur, -1);
            // x1 upstream of the tile's first column when it starts a block: x1 ghost layers of
            // the previous iteration in slot ti.z (oriented rows (k, j))
            if (ti.z >= 0) {
                const size_t gxo = ((((size_t)par * 8 + q) * P->ns1 + ti.z) * n3 * n2) * 2 * NL;
                if constexpr (!BF) {
                    for (int m = half; m < nr3 * nr2 * 2; m += 2) {
                        const int kk = m / (2 * nr2);
                        const int jl = m - kk * 2 * nr2;          // jj * 2 + layer
                        const size_t row = (size_t)(k0 + kk) * n2 + (j0 + (jl >> 1));
                        cp_async16(carry + ((size_t)(warp * MROWS + kk * MR2 + (jl >> 1)) * 2 + (jl & 1)) * kPL + 4 * hl,
                                   P->gx1 + gxo + (row * 2 + (jl & 1)) * NL + lw);
                    }
                    // complete them here when no sub-tile will commit them
                    if (!tfl) {
                        cp_async_commit();
                        cp_async_wait<0>();
                    }
                } else {
                    for (int kk = 0; kk < nr3; ++kk)
                        for (int jj = 0; jj < nr2; ++jj) {
                            const size_t row = (size_t)(k0 + kk) * n2 + (j0 + jj);
                            float* cr = carry + ((size_t)(warp * MROWS + kk * MR2 + jj) * 2) * kPL + 2 * lane;
                            *reinterpret_cast<float2*>(cr) = PS::ld(P->gx1, gxo + (row * 2 + 0) * NL + lv, x1g0);
                            *reinterpret_cast<float2*>(cr + kPL) = PS::ld(P->gx1, gxo + (row * 2 + 1) * NL + lv, x1g1);
                        }
                }
            }
            // Sub-tiles of SW columns, swept one after the other with the same staging (the x1
            // carries pass between them in shared memory, as between tiles).
            for (int u = 0; u < NSUB && tfl; ++u) {
                const int cs = c0 + u * SW;                       // first column of the sub-tile
                const int wsub = min(SW, width - u * SW);         // its width
                if (wsub <= 0) break;
                // (a sub-tile 0 without fluid leaves its carry-in copies, if any, to the group of
                // sub-tile 1, which then holds fluid)
                if (NSUB > 1 && !has_fluid(fm_cur, u)) continue;
                const int us = u * SW;                            // bit / record column offset
                const float* recs = recb + (size_t)us * RF;       // record of (row 0, column cs)
                auto rbuf_rec = [&](int kk, int jj, int i) -> const float* { return recs + (size_t)((kk * MR2 + jj) * T1 + i) * RF; };
                auto fbits = [&](int r) -> unsigned { return (fm_cur[r] >> us) & ((1u << SW) - 1u); };
                if constexpr (BF) {
                    for (int jj = 0; jj < nr2; ++jj)
                        for (int i = 0; i < wsub; ++i) {
                            const size_t row = zg ? ((size_t)(j0 + jj) * n1 + (cs + i)) : ((size_t)jj * n1 + (cs + i));
                            float* d = pb + ((((size_t)warp * MR2 + jj) * 2) * SW + i) * kPL + 2 * lane;
                            const float xs = x1of(cs + i);
                            const float* rc = rbuf_rec(0, jj, i);
                            *reinterpret_cast<float2*>(d + (size_t)SW * kPL) =
                                rc[12] != 0.f ? PS::ld(zb, zo + (row * 2 + 0) * NL + lv, xs) : make_float2(0.f, 0.f);
                            *reinterpret_cast<float2*>(d) = rc[13] != 0.f ? PS::ld(zb, zo + (row * 2 + 1) * NL + lv, xs) : make_float2(0.f, 0.f);
                        }
                } else {
                    __syncwarp();                            // the staging's last readers are done
                    issue_z(cs, wsub, recs);
                    issue_y(0, cs, wsub, recs);
                }
                for (int kk = 0; kk < nr3; ++kk) {
                    // x2 upstream rows of the first row of this plane
                    float2 rb1[SW], rb2[SW];
                    if constexpr (BF) {
                        const size_t rowbase = yrow(kk);
#pragma unroll
                        for (int i = 0; i < SW; ++i) {
                            if (i < wsub) {
                                const float xs = x1of(cs + i);
                                const float* rc = rbuf_rec(kk, 0, i);
                                rb1[i] = rc[10] != 0.f ? PS::ld(yb, yo + ((rowbase + cs + i) * 2 + 0) * NL + lv, xs) : make_float2(0.f, 0.f);
                                rb2[i] = rc[11] != 0.f ? PS::ld(yb, yo + ((rowbase + cs + i) * 2 + 1) * NL + lv, xs) : make_float2(0.f, 0.f);
                            } else {
                                rb1[i] = make_float2(0.f, 0.f);
                                rb2[i] = rb1[i];
                            }
                        }
                    } else {
                        __syncwarp();                        // slot (kk + 1) & 1 was last read at plane kk - 1
                        if (kk + 1 < nr3) {
                            issue_y(kk + 1, cs, wsub, recs);
                            cp_async_wait<1>();              // all but the copies of plane kk + 1
                        } else {
                            cp_async_wait<0>();
                        }
                        __syncwarp();
                        const float* e0 = eb + ((((size_t)warp * 2 + (kk & 1)) * 2) * SW) * kPL + 2 * lane;
#pragma unroll
                        for (int i = 0; i < SW; ++i) {
                            if (i < wsub) {
                                rb1[i] = *reinterpret_cast<const float2*>(e0 + (size_t)i * kPL);
                                rb2[i] = *reinterpret_cast<const float2*>(e0 + ((size_t)SW + i) * kPL);
                            } else {
                                rb1[i] = make_float2(0.f, 0.f);
                                rb2[i] = rb1[i];
                            }
                        }
                    }
                    // plane staging of a row: [2][SW][64], plane kk - 1 in layer (kk + 1) & 1 and plane
                    // kk - 2 in layer kk & 1, which plane kk's value then replaces
                    const size_t zl1 = (size_t)(((kk + 1) & 1) * SW) * kPL, zl2 = (size_t)((kk & 1) * SW) * kPL;
                    // FP32 pencils of two or more planes store their x3 edge as the last two planes
                    // are swept (layer 0: plane nr3 - 1, layer 1: plane nr3 - 2; fluid points only)
                    const bool e3 = !BF && nr3 >= 2 && kk >= nr3 - 2;
                    const size_t e3o = eo3 + (size_t)cs * colS + (size_t)(nr3 - 1 - kk) * NL;
                    // likewise the x2 edge of this plane as rows nr2 - 2 (layer 1) and nr2 - 1 (layer 0)
                    // are swept, in pencils of two or more rows
                    const bool e2 = !BF && nr2 >= 2;
                    const size_t e2o = eo2 + (size_t)kk * rowS + (size_t)cs * colS;
                    // one point: Eq. 10 for the lane's velocity pair with the x1 upstream values (hp1,
                    // hp2) of its row, the x2 upstream values rb of its column and the x3 upstream
                    // values of its row's plane staging zr; returns the lane's moment sums of the
                    // point: (rho, u1), (u2, u3) and the temperature moment
                    auto point = [&](const float* rrow, float* zr, int i, float2& hp1, float2& hp2, float2& M01,
                                     float2& M23, float& m4, bool st3, size_t o3, bool st2, size_t o2) {
                        const float4* R = reinterpret_cast<const float4*>(rrow + i * RF);
                        const float4 A = R[0], B = R[1], C = R[2], D = R[3];
                        const float2 z1 = *reinterpret_cast<const float2*>(zr + zl1 + (size_t)i * kPL);
                        const float2 z2 = *reinterpret_cast<const float2*>(zr + zl2 + (size_t)i * kPL);
                        const float2 Rk = *reinterpret_cast<const float2*>(my_rtab + __float_as_int(B.w));
                        float2 S = fma2(dup2(A.w), v3, fma2(dup2(A.z), v2, fma2(dup2(A.y), v1, dup2(A.x))));
                        if constexpr (TAU) S = fma2(dup2(D.z), vq, S);   // nu tau (|v|^2 - 3/2)
                        float2 t1 = fma2(dup2(C.x), hp1, fma2(dup2(C.y), hp2, dup2(B.x)));
                        float2 t2 = fma2(dup2(C.z), rb1[i], fma2(dup2(C.w), rb2[i], dup2(B.y)));
                        float2 t3 = fma2(dup2(D.x), z1, fma2(dup2(D.y), z2, dup2(B.z)));
                        int4 Fa, Fb;
                        if constexpr (SPEC) {   // + (1 - alpha) h'(x, reflected v) at walls
                            Fa = reinterpret_cast<const int4*>(R)[4];
                            Fb = reinterpret_cast<const int4*>(R)[5];
                            if (Fa.x >= 0) t1 = fma2(specP, *reinterpret_cast<const float2*>(fprev[0] + (size_t)Fa.x * fstride), t1);
                            if (Fa.y >= 0) t2 = fma2(specP, *reinterpret_cast<const float2*>(fprev[1] + (size_t)Fa.y * fstride), t2);
                            if (Fa.z >= 0) t3 = fma2(specP, *reinterpret_cast<const float2*>(fprev[2] + (size_t)Fa.z * fstride), t3);
                        }
                        // the x1 term (carried from the previous point) enters last: three dependent
                        // operations per point along the x1 chain
                        const float2 num = fma2(a1, t1, fma2(a3, t3, fma2(a2, t2, S)));
                        const float2 h = mul2(num, Rk);
                        if constexpr (SPEC) {   // molecules moving into a downstream face
                            if (Fa.w >= 0) *reinterpret_cast<float2*>(fnext[0] + (size_t)Fa.w * fstride) = h;
                            if (Fb.x >= 0) *reinterpret_cast<float2*>(fnext[1] + (size_t)Fb.x * fstride) = h;
                            if (Fb.y >= 0) *reinterpret_cast<float2*>(fnext[2] + (size_t)Fb.y * fstride) = h;
                        }
                        if (st3) PS::st(et3, o3 + (size_t)i * colS, h, 0.f);
                        if (st2) PS::st(et2, o2 + (size_t)i * colS, h, 0.f);
                        hp2 = hp1;
                        hp1 = h;
                        rb2[i] = rb1[i];
                        rb1[i] = h;
                        *reinterpret_cast<float2*>(zr + zl2 + (size_t)i * kPL) = h;
                        M01 = fma2(Wb01, dup2(h.y), mul2(Wa01, dup2(h.x)));
                        M23 = fma2(Wb23, dup2(h.y), mul2(Wa23, dup2(h.x)));
                        if constexpr (TAU) {
                            const float2 p4v = mul2(Wvv, h);
                            m4 = p4v.x + p4v.y;
                        } else {
                            m4 = 0.f;
                        }
                    };
                    // the plane's row 0: x1 carries, plane staging [2][SW][64], records, partials
                    float* const cr0 = carry + ((size_t)(warp * MROWS + kk * MR2) * 2) * kPL + 2 * lane;
                    float* const zr0 = pb + ((size_t)warp * MR2 * 2 * SW) * kPL + 2 * lane;
                    const float* const rr0 = recs + (size_t)(kk * MR2 * T1) * RF;
                    float* const pr0 = part + ((size_t)(warp * MROWS + kk * MR2) * T1 + us) * NM;
                    auto row_ptrs = [&](int jj, float*& cr, float*& zr, const float*& rrow, float*& prow) {
                        cr = cr0 + jj * (2 * kPL);
                        zr = zr0 + jj * (2 * SW * kPL);
                        rrow = rr0 + jj * (T1 * RF);
                        prow = pr0 + jj * (T1 * NM);
                    };
                    // solid points are not swept: every fluid point downstream of one gives it a zero
                    // stencil coefficient (its code marks that upstream point solid), so the values
                    // left in the carries, rows and planes there are never used.
                    // Rows two at a time, the upper one a column behind the lower (it needs the lower
                    // row's value of the same column): two independent points per step.  A step with
                    // a fluid point sweeps both of its points; a solid one has a zero record and gets
                    // h = 0, which is as unused as the value a skipped point leaves.  Points beyond
                    // the sub-tile width are never swept (their staging is not filled, and the x1
                    // carries must end at the last column).
                    int jj = 0;
                    auto walk_pairs = [&](auto full_tag) {
                        constexpr bool FULL = decltype(full_tag)::value;
                        for (; jj + 1 < nr2; jj += 2) {
                            const unsigned fa = fbits(kk * MR2 + jj), fb = fbits(kk * MR2 + jj + 1);
                            if ((fa | fb) == 0u) continue;
                            float *crA, *zrA, *prA, *crB, *zrB, *prB;
                            const float *rrA, *rrB;
                            row_ptrs(jj, crA, zrA, rrA, prA);
                            row_ptrs(jj + 1, crB, zrB, rrB, prB);
                            const size_t o3A = e3o + (size_t)jj * rowS;
                            // rows nr2 - 2 and nr2 - 1 give the x2 edge's layers 1 and 0
                            const bool x2A = e2 && jj >= nr2 - 2, x2B = e2 && jj + 1 >= nr2 - 2;
                            const size_t o2A = e2o + (size_t)(nr2 - 1 - jj) * NL, o2B = e2o + (size_t)(nr2 - 2 - jj) * NL;
                            float2 hA1 = *reinterpret_cast<const float2*>(crA), hA2 = *reinterpret_cast<const float2*>(crA + kPL);
                            float2 hB1 = *reinterpret_cast<const float2*>(crB), hB2 = *reinterpret_cast<const float2*>(crB + kPL);
                            float2 M01[8], M23[8];
                            float m4[8];
                            const float2 z2 = make_float2(0.f, 0.f);
#pragma unroll
                            for (int st = 0; st <= SW; ++st) {
                                const bool onA = st < SW && ((fa >> st) & 1u);
                                const bool onB = st >= 1 && ((fb >> (st - 1)) & 1u);
                                if (onA || onB) {
                                    if (st < SW) {
                                        if (FULL || st < wsub) point(rrA, zrA, st, hA1, hA2, M01[st], M23[st], m4[st], e3 && onA, o3A, x2A && onA, o2A);
                                        else { M01[st] = M23[st] = z2; m4[st] = 0.f; }
                                    }
                                    if (st >= 1) {
                                        if (FULL || st - 1 < wsub) point(rrB, zrB, st - 1, hB1, hB2, M01[3 + st], M23[3 + st], m4[3 + st], e3 && onB, o3A + rowS, x2B && onB, o2B);
                                        else { M01[3 + st] = M23[3 + st] = z2; m4[3 + st] = 0.f; }
                                    }
                                } else {
                                    if (st < SW) { M01[st] = M23[st] = z2; m4[st] = 0.f; }
                                    if (st >= 1) { M01[3 + st] = M23[3 + st] = z2; m4[3 + st] = 0.f; }
                                }
                            }
                            *reinterpret_cast<float2*>(crA) = hA1;
                            *reinterpret_cast<float2*>(crA + kPL) = hA2;
                            *reinterpret_cast<float2*>(crB) = hB1;
                            *reinterpret_cast<float2*>(crB + kPL) = hB2;
                            const float2 r01 = reduce_scatter2<8>(M01, lane);
                            const float2 r23 = reduce_scatter2<8>(M23, lane);
                            [[maybe_unused]] float r4 = 0.f;
                            if constexpr (TAU) r4 = reduce_scatter<float, 8>(m4, lane);
                            // value v of the eight ends in lanes 4 v .. 4 v + 3: row jj + v / 4, column v % 4
                            const int v = lane >> 2;
                            if ((lane & 3) == 0 && (v & 3) < wsub) {
                                float* d = (v < 4 ? prA : prB) + (v & 3) * NM;
                                if constexpr (TAU) {
                                    d[0] = r01.x;
                                    d[1] = r01.y;
                                    d[2] = r23.x;
                                    d[3] = r23.y;
                                    d[4] = r4;
                                } else {
                                    *reinterpret_cast<float4*>(d) = make_float4(r01.x, r01.y, r23.x, r23.y);
                                }
                            }
                        }
                    };
                    if (wsub == SW) walk_pairs(std::integral_constant<bool, true>{});
                    else walk_pairs(std::integral_constant<bool, false>{});
                    if (jj < nr2) {   // the last row of an odd row count
                        const unsigned fm = fbits(kk * MR2 + jj);
                        if (fm != 0u) {
                            float *cr, *zr, *prow;
                            const float* rrow;
                            row_ptrs(jj, cr, zr, rrow, prow);
                            float2 hp1 = *reinterpret_cast<const float2*>(cr);
                            float2 hp2 = *reinterpret_cast<const float2*>(cr + kPL);
                            float2 M01[4], M23[4];
                            float m4[4];
#pragma unroll
                            for (int c = 0; c < SW; ++c) {
                                if ((fm >> c) & 1u)
                                    point(rrow, zr, c, hp1, hp2, M01[c], M23[c], m4[c], e3, e3o + (size_t)jj * rowS, e2 && jj >= nr2 - 2,
                                          e2o + (size_t)(nr2 - 1 - jj) * NL);
                                else {
                                    M01[c] = M23[c] = make_float2(0.f, 0.f);
                                    m4[c] = 0.f;
                                }
                            }
                            const float2 r01 = reduce_scatter2<4>(M01, lane);
                            const float2 r23 = reduce_scatter2<4>(M23, lane);
                            [[maybe_unused]] float r4 = 0.f;
                            if constexpr (TAU) r4 = reduce_scatter<float, 4>(m4, lane);
                            const int p = lane >> 3;
                            if ((lane & 7) == 0 && p < wsub) {
                                float* d = prow + p * NM;
                                d[0] = r01.x;
                                d[1] = r01.y;
                                d[2] = r23.x;
                                d[3] = r23.y;
                                if constexpr (TAU) d[4] = r4;
                            }
                            *reinterpret_cast<float2*>(cr) = hp1;
                            *reinterpret_cast<float2*>(cr + kPL) = hp2;
                        }
                    }
                    // x2 edge of this plane in BF16 storage or one-row pencils (FP32 pencils stored it as
                    // the rows were swept): only values of fluid points are stored (layer 1 of a one-row
                    // pencil passes the fetched upstream value through and is always stored)
                    if (!e2) {
                        const unsigned f0 = fbits(kk * MR2 + nr2 - 1);
                        const unsigned f1 = nr2 >= 2 ? fbits(kk * MR2 + nr2 - 2) : 0xffffffffu;
                        size_t o = eo2 + (size_t)kk * rowS + (size_t)cs * colS;
#pragma unroll
                        for (int i = 0; i < SW; ++i) {
                            if (i < wsub) {
                                const float xs = x1of(cs + i);
                                if ((f0 >> i) & 1u) PS::st(et2, o, rb1[i], xs);
                                if ((f1 >> i) & 1u) PS::st(et2, o + NL, rb2[i], xs);
                            }
                            o += colS;
                        }
                    }
                }
                // x3 edge of BF16 storage or one-plane pencils (FP32 pencils stored it during the last two
                // planes): the top plane nr3 - 1 in staging layer (nr3 - 1) & 1, the plane below it
                // (or, in a one-plane pencil, the fetched upstream plane) in layer nr3 & 1
                if (BF || nr3 < 2) {
                    const float* s = pb + ((size_t)warp * MR2 * 2 * SW) * kPL + 2 * lane;
                    const float* st0 = s + (size_t)(((nr3 - 1) & 1) * SW) * kPL;
                    const float* st1 = s + (size_t)((nr3 & 1) * SW) * kPL;
                    const unsigned* ft0 = fm_cur + (nr3 - 1) * MR2;
                    const unsigned* ft1 = fm_cur + (nr3 >= 2 ? (nr3 - 2) * MR2 : 0);
                    size_t ob = eo3 + (size_t)cs * colS;
                    for (int jj = 0; jj < nr2; ++jj) {
                        const unsigned f0 = (ft0[jj] >> us) & ((1u << SW) - 1u);
                        const unsigned f1 = nr3 >= 2 ? ((ft1[jj] >> us) & ((1u << SW) - 1u)) : 0xffffffffu;
                        size_t o = ob;
#pragma unroll
                        for (int i = 0; i < SW; ++i) {
                            if (i < wsub) {
                                const float xs = x1of(cs + i);
                                if ((f0 >> i) & 1u) PS::st(et3, o, *reinterpret_cast<const float2*>(st0 + (size_t)i * kPL), xs);
                                if ((f1 >> i) & 1u) PS::st(et3, o + NL, *reinterpret_cast<const float2*>(st1 + (size_t)i * kPL), xs);
                            }
                            o += colS;
                        }
                        ob += rowS;
                        st0 += (size_t)2 * SW * kPL;
                        st1 += (size_t)2 * SW * kPL;
                    }
                }
            }   // sub-tiles
            if (ti.w >= 0 && tfl) {   // x1 carry into ghost slot ti.w of the next iteration
                const size_t gxo = ((((size_t)(par ^ 1) * 8 + q) * P->ns1 + ti.w) * n3 * n2) * 2 * NL;
                for (int kk = 0; kk < nr3; ++kk)
                    for (int jj = 0; jj < nr2; ++jj) {
                        const size_t row = (size_t)(k0 + kk) * n2 + (j0 + jj);
                        const float* cr = carry + ((size_t)(warp * MROWS + kk * MR2 + jj) * 2) * kPL + 2 * lane;
                        PS::st(P->gx1, gxo + (row * 2 + 0) * NL + lv, *reinterpret_cast<const float2*>(cr), x1g0);
                        PS::st(P->gx1, gxo + (row * 2 + 1) * NL + lv, *reinterpret_cast<const float2*>(cr + kPL), x1g1);
                    }
            }
            __syncthreads();
            if (threadIdx.x == 0 && it != a.withhold_item) {
                publish_gpu(prog + p3 * np2 + p2, t + 1);
            }
            // (the next tile's records after the publish: its readers are behind the next tile's
            // first barrier)
            if (t + 1 < ntiles) store_rec(t + 1, (t + 1) & 1, nxt);
            // moment partials of this octant and group: warp sums in warp order
            // (idx = (r T1 + i) NM + mm over the pencil's row slots; only fluid points have bits)
            const int wstride = MROWS * T1 * NM;
            if constexpr (!TAU) {   // a thread per point, its four moments as one vector
                for (int pt = threadIdx.x; tfl && pt < MROWS * T1; pt += blockDim.x) {
                    const int i = pt % T1, r = pt / T1;
                    if (!((fm_cur[r] >> i) & 1u)) continue;   // solid: the start state's zeros stay
                    float4 sv = *reinterpret_cast<const float4*>(part + (size_t)pt * 4);
                    for (int w = 1; w < NW; ++w) {
                        const float4 o = *reinterpret_cast<const float4*>(part + (size_t)w * wstride + (size_t)pt * 4);
                        sv.x += o.x;
                        sv.y += o.y;
                        sv.z += o.z;
                        sv.w += o.w;
                    }
                    const int ic = c0 + i;
                    float* d = Pq + (size_t)rowoff[r] + (s1n ? n1 - 1 - ic : ic);
                    d[0] = sv.x;
                    d[N] = sv.y;
                    d[2 * (size_t)N] = sv.z;
                    d[3 * (size_t)N] = sv.w;
                }
            }
            const int tot = (tfl && TAU) ? MROWS * T1 * NM : 0;
            for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
                const int mm = idx % NM;
                const int pt = idx / NM;
                const int i = pt % T1;
                const int r = pt / T1;
                // solid points keep the zero partials of the start state (no reader uses them)
                if (!((fm_cur[r] >> i) & 1u)) continue;
                float s = 0.f;
                for (int w = 0; w < NW; ++w) s += part[(size_t)w * wstride + idx];
                const int ic = c0 + i;
                const size_t pid = (size_t)rowoff[r] + (s1n ? n1 - 1 - ic : ic);
                if (!TAU || mm < 4) Pq[(size_t)mm * N + pid] = s;
                else P->Pt[((size_t)q * G + g) * N + pid] = s;
            }
            // (with masks by vote the next writers of part and of these masks are behind the next
            // tile's first barrier; cleared masks need this one)
            if (!bmask) __syncthreads();
        }
        __syncthreads();
    }
}

size_t sweep3d_f32x2_smem(int T1, int NW, int R2, int R3, int tau, int spec) {
    const size_t rows = (size_t)R2 * R3;
    return sizeof(float) * (2 * rows * T1 * (spec ? 24 : kRec) + (size_t)NW * rows * T1 * (tau ? 5 : 4) +
                            (size_t)NW * rows * 2 * kPL + (size_t)NW * R2 * 2 * kSubW * kPL + (size_t)NW * 2 * 2 * kSubW * kPL +
                            (size_t)NW * 8 * kPL) +
           sizeof(unsigned) * 2 * rows + sizeof(int) * rows;
}

int sweep3d_f32x2_velocities_per_lane() { return 2; }

template <int T1, bool BF, bool SUB, bool TAU, bool SPEC>
static cudaError_t launch_t(const SweepArgs3D<float>& a, int grid, int NW, cudaStream_t st) {
    const size_t smem = sweep3d_f32x2_smem(T1, NW, a.maxR2, a.maxR3, TAU, SPEC);
    auto kern = sweep3d_f32x2_kernel<T1, BF, SUB, TAU, SPEC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, NW * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int T1, bool SUB, bool TAU>
static cudaError_t launch_ts(const SweepArgs3D<float>& a, int grid, int NW, cudaStream_t st) {
    return a.spec ? launch_t<T1, false, SUB, TAU, true>(a, grid, NW, st) : launch_t<T1, false, SUB, TAU, false>(a, grid, NW, st);
}

template <int T1>
static cudaError_t launch_tt(const SweepArgs3D<float>& a, int grid, int NW, cudaStream_t st) {
    if (a.bf16) return launch_t<T1, true, false, false, false>(a, grid, NW, st);
    if (a.sub) return a.tau ? launch_ts<T1, true, true>(a, grid, NW, st) : launch_ts<T1, true, false>(a, grid, NW, st);
    return a.tau ? launch_ts<T1, false, true>(a, grid, NW, st) : launch_ts<T1, false, false>(a, grid, NW, st);
}

// instantiations: FP32 with any combination of subdomains, the temperature term and specular wall
// parts; BF16 storage with none of them
cudaError_t launch_sweep3d_f32x2(const SweepArgs3D<float>& a, int grid, int NW, cudaStream_t st) {
    if (a.bf16 && (a.sub || a.tau || a.spec)) return cudaErrorInvalidValue;
    if (a.T1 == 4) return launch_tt<4>(a, grid, NW, st);
    if (a.T1 == 8) return launch_tt<8>(a, grid, NW, st);
    return cudaErrorInvalidValue;
}

template <int T1, bool BF, bool SUB, bool TAU, bool SPEC>
static cudaError_t occ_t(int NW, int R2, int R3, int* blocks_per_sm) {
    const size_t smem = sweep3d_f32x2_smem(T1, NW, R2, R3, TAU, SPEC);
    auto kern = sweep3d_f32x2_kernel<T1, BF, SUB, TAU, SPEC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, NW * 32, smem);
}

template <int T1, bool SUB, bool TAU>
static cudaError_t occ_ts(int NW, int R2, int R3, int spec, int* bps) {
    return spec ? occ_t<T1, false, SUB, TAU, true>(NW, R2, R3, bps) : occ_t<T1, false, SUB, TAU, false>(NW, R2, R3, bps);
}

template <int T1>
static cudaError_t occ_tt(int NW, int R2, int R3, int bf16, int sub, int tau, int spec, int* bps) {
    if (bf16) return occ_t<T1, true, false, false, false>(NW, R2, R3, bps);
    if (sub) return tau ? occ_ts<T1, true, true>(NW, R2, R3, spec, bps) : occ_ts<T1, true, false>(NW, R2, R3, spec, bps);
    return tau ? occ_ts<T1, false, true>(NW, R2, R3, spec, bps) : occ_ts<T1, false, false>(NW, R2, R3, spec, bps);
}

cudaError_t sweep3d_f32x2_occupancy(int T1, int NW, int R2, int R3, int bf16, int sub, int tau, int spec,
                                    int* blocks_per_sm) {
    if (bf16 && (sub || tau || spec)) return cudaErrorInvalidValue;
    if (T1 == 4) return occ_tt<4>(NW, R2, R3, bf16, sub, tau, spec, blocks_per_sm);
    if (T1 == 8) return occ_tt<8>(NW, R2, R3, bf16, sub, tau, spec, blocks_per_sm);
    return cudaErrorInvalidValue;
}

}  // namespace dvm
