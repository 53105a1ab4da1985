// kernels2d.cu -- sm_103a kernels of one source iteration (arXiv:1712.01132, Sec. 3.1) in 2D.
//
// sweep2d   : step (i) for every quadrant of discrete velocities, with the moment quadrature of
//             step (iii) fused in.  Persistent CTAs take (problem, quadrant, band) items from a
//             ticket counter in band order; a CTA sweeps its band of rows along x1 tile by tile
//             (forward substitution in the upwind order of Eq. 9-10), one discrete velocity per
//             lane, and publishes per-tile progress so the band above can follow one tile behind.
//             Every value a point reads is final when it is read, so the result is the same as
//             the paper's raster scan.  Boundary data (wall values, ghost layers) and moments are
//             those of the previous iteration (step ii), exactly as in the paper.
// finalize2d: step (iii) completion: sums the per-quadrant moment partials, forms the wall
//             densities of Eq. 6 in FP64, the source terms and wall terms of the next sweep, and
//             the FP64 sum of u1 for the permeability of Eq. 11-12.
// init2d    : the zero-perturbation start in the kernels' source-form variables.
#include <cuda_runtime.h>

#include <cstdint>

#include "dvm_internal.h"
#include "dvm_device.cuh"

namespace dvm {

// ---------------------------------------------------------------- sweep

// Per-lane state while a warp walks along one row of a tile.
template <typename T>
struct LaneK {
    T v1, v2, a1, a2, W, Wv1, Wv2, R0, R1, R2, R3;
};

// Specular wall parts (Eq. 5, alpha < 1) of one lane: face stores of the previous iteration (read
// where the upstream point of an axis is solid) and of this one (written where the downstream point
// is solid), each already offset to this lane's slot and the quadrant's other-axis sign bit; face f
// is at f * stride.
template <typename T>
struct SpecLane {
    const T* prev1;
    const T* prev2;
    T* next1;
    T* next2;
    size_t stride;
    T spec;          // 1 - alpha
};

// Processes CH consecutive points (columns i0..i0+CH-1 of the tile) of one row.
// rec: records of this row; rb1/rb2: the two rows below (updated in place); hp1/hp2: x1 upstream.
template <typename T, int T1, int CH, bool FULL, bool SPEC>
__device__ __forceinline__ void row_chunk(const T* __restrict__ rec, int i0, int width, const LaneK<T>& L,
                                          T (&rb1)[T1], T (&rb2)[T1], T& hp1, T& hp2, T (&m0)[CH],
                                          T (&m1)[CH], T (&m2)[CH], const SpecLane<T>& SL) {
    using V = typename Vec4<T>::type;
    constexpr int RW = SPEC ? 16 : kRecWords;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const int i = i0 + c;
        if (FULL || i < width) {
            const V* R = reinterpret_cast<const V*>(rec + i * RW);
            const V A = R[0];
            const V B = R[1];
            const V C = R[2];
            // numerator of Eq. 10 solved for h(x): nu (rho' + 2 u.v) + v1 plus the upwind terms
            const T S = fma(A.z, L.v2, fma(A.y, L.v1, A.x));
            T t1 = fma(B.x, hp1, fma(B.y, hp2, A.w));
            T t2 = fma(B.z, rb1[i], fma(B.w, rb2[i], C.x));
            V D;
            if constexpr (SPEC) {
                // the wall term holds alpha rho_s' (+ shift); add (1 - alpha) h'(x, reflected v)
                D = R[3];
                const int fu1 = as_bits(D.x), fu2 = as_bits(D.y);
                if (fu1 >= 0) t1 = fma(SL.spec, SL.prev1[(size_t)fu1 * SL.stride], t1);
                if (fu2 >= 0) t2 = fma(SL.spec, SL.prev2[(size_t)fu2 * SL.stride], t2);
            }
            const T num = fma(L.a2, t2, fma(L.a1, t1, S));
            const int rs = as_bits(C.y);
            const T Rv = (rs & 2) ? ((rs & 1) ? L.R3 : L.R2) : ((rs & 1) ? L.R1 : L.R0);
            const T h = num * Rv;
            if constexpr (SPEC) {   // molecules moving into a face downstream: kept for its reflection
                const int fd1 = as_bits(D.z), fd2 = as_bits(D.w);
                if (fd1 >= 0) SL.next1[(size_t)fd1 * SL.stride] = h;
                if (fd2 >= 0) SL.next2[(size_t)fd2 * SL.stride] = h;
            }
            hp2 = hp1;
            hp1 = h;
            rb2[i] = rb1[i];
            rb1[i] = h;
            m0[c] = L.W * h;
            m1[c] = L.Wv1 * h;
            m2[c] = L.Wv2 * h;
        } else {
            m0[c] = T(0);
            m1[c] = T(0);
            m2[c] = T(0);
        }
    }
}

template <typename T, int T1, bool FULL, bool SPEC>
__device__ __forceinline__ void sweep_tile_rows(const T* __restrict__ rec, T* __restrict__ part,
                                                T* __restrict__ carry, int nrows, int width, int RB,
                                                int warp, int lane, const LaneK<T>& L, T (&rb1)[T1],
                                                T (&rb2)[T1], const SpecLane<T>& SL) {
    constexpr int CH = 8;                       // points reduced together
    constexpr int RW = SPEC ? 16 : kRecWords;
    for (int r = 0; r < nrows; ++r) {
        T* cr = carry + ((size_t)(warp * RB + r) * 2) * 32 + lane;
        T hp1 = cr[0];
        T hp2 = cr[32];
        const T* rrow = rec + (size_t)r * T1 * RW;
        T* prow = part + ((size_t)(warp * RB + r) * T1) * 3;
#pragma unroll
        for (int i0 = 0; i0 < T1; i0 += CH) {
            T m0[CH], m1[CH], m2[CH];
            row_chunk<T, T1, CH, FULL, SPEC>(rrow, i0, width, L, rb1, rb2, hp1, hp2, m0, m1, m2, SL);
            const T s0 = reduce_scatter<T, CH>(m0, lane);
            const T s1 = reduce_scatter<T, CH>(m1, lane);
            const T s2 = reduce_scatter<T, CH>(m2, lane);
            const int p = lane >> 2;
            if ((lane & 3) == 0 && (FULL || i0 + p < width)) {
                T* d = prow + (i0 + p) * 3;
                d[0] = s0;
                d[1] = s1;
                d[2] = s2;
            }
        }
        cr[0] = hp1;
        cr[32] = hp2;
    }
}

template <typename T, int T1, bool XS, bool SPEC>
__global__ void __launch_bounds__(512) sweep2d_kernel(const SweepArgs2D<T> a) {
    using V = typename Vec4<T>::type;
    constexpr int RW = SPEC ? 16 : kRecWords;   // record words (face ids in a fourth vector)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    __shared__ int s_abort;
    const int NW = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int RB = a.max_rows;
    T* rec = reinterpret_cast<T*>(smem_raw);                 // [RB][T1][RW]
    T* part = rec + (size_t)RB * T1 * RW;                    // [NW][RB][T1][3]
    T* carry = part + (size_t)NW * RB * T1 * 3;              // [NW][RB][2][32]
    const int wl = warp * 32 + lane;
    const size_t NL = (size_t)a.NL;

    for (;;) {
        if (threadIdx.x == 0) {
            s_item = ld_volatile(a.status) ? a.nitems : atomicAdd(a.ticket, 1);
            s_abort = 0;
        }
        __syncthreads();
        const int it = s_item;
        if (it >= a.nitems) return;
        const SweepItem item = a.items[it];
        const Prob2D<T>* __restrict__ P = a.prob + item.prob;
        const int q = item.quad;
        const int band = item.band;
        const int n1 = P->n1, n2 = P->n2, nb = P->nbands;
        const int N = P->N;
        const int s1neg = q & 1;
        const int s2neg = (q >> 1) & 1;
        const int4 binfo = P->bands[q * nb + band];
        const int row0 = binfo.x, nrows = binfo.y, below = binfo.z, above = binfo.w;
        const T K1o = P->order == 2 ? T(2) : T(1);
        const T K2o = P->order == 2 ? T(-0.5) : T(0);
        LaneK<T> L;
        {
            const T* lc = P->lanec + ((size_t)q * NL + wl) * kLaneConsts;
            L.v1 = lc[0]; L.v2 = lc[1]; L.a1 = lc[2]; L.a2 = lc[3];
            L.W = lc[4]; L.Wv1 = lc[5]; L.Wv2 = lc[6];
            L.R0 = lc[7]; L.R1 = lc[8]; L.R2 = lc[9]; L.R3 = lc[10];
        }
        const int par = a.parity;
        SpecLane<T> SL{};
        if constexpr (SPEC) {
            // x1 faces are told apart by the x2 sign bit of the quadrant, x2 faces by the x1 bit
            const size_t plane = (size_t)P->nfaces * 2 * NL;
            SL.stride = 2 * NL;
            SL.prev1 = P->F + par * plane + (size_t)s2neg * NL + wl;
            SL.prev2 = P->F + par * plane + (size_t)s1neg * NL + wl;
            SL.next1 = P->F + (par ^ 1) * plane + (size_t)s2neg * NL + wl;
            SL.next2 = P->F + (par ^ 1) * plane + (size_t)s1neg * NL + wl;
            SL.spec = (T)P->spec;
        }
        // x1 upstream of a tile from a lagged slot: the x1 ghost layers of the previous iteration
        // (Eq. 7, source form; slot 0) or, with x1 subdomains, a subdomain halo; and the carry of the
        // last tile into the slot the next iteration reads
        auto carry_in = [&](int slot) {
            const T* g = P->gx1 + (((size_t)(par * 4 + q) * P->nxslots + slot) * n2) * 2 * NL;
            for (int r = 0; r < nrows; ++r) {
                T* cr = carry + ((size_t)(warp * RB + r) * 2) * 32 + lane;
                cr[0] = g[((size_t)(row0 + r) * 2 + 0) * NL + wl];
                cr[32] = g[((size_t)(row0 + r) * 2 + 1) * NL + wl];
            }
        };
        auto carry_out = [&](int slot) {
            T* g = P->gx1 + (((size_t)((par ^ 1) * 4 + q) * P->nxslots + slot) * n2) * 2 * NL;
            for (int r = 0; r < nrows; ++r) {
                const T* cr = carry + ((size_t)(warp * RB + r) * 2) * 32 + lane;
                g[((size_t)(row0 + r) * 2 + 0) * NL + wl] = cr[0];
                g[((size_t)(row0 + r) * 2 + 1) * NL + wl] = cr[32];
            }
        };
        if constexpr (!XS) carry_in(0);
        const int ntiles = XS ? P->ntq[q] : (n1 + T1 - 1) / T1;
        // progress of the band below that thread 0 has already observed with an acquire (tiles up
        // to it need no new wait)
        int seenb = -1;
        for (int t = 0; t < ntiles; ++t) {
            int4 tcur;
            if constexpr (XS) {
                tcur = __ldg(P->tiles + (size_t)q * P->ntiles + t);
                if (tcur.z >= 0) carry_in(tcur.z);
            } else {
                tcur = make_int4(t * T1, min(T1, n1 - t * T1), t == 0 ? 0 : -1, t == ntiles - 1 ? 0 : -1);
            }
            const int c0 = tcur.x;
            const int width = tcur.y;
            if (threadIdx.x == 0 && below < 0 && seenb < t + 1) {
                seenb = wait_geq_value(P->prog + q * nb + band - 1, t + 1, a.status, a.timeout_ns);
                if (seenb < 0) s_abort = 1;
            }
            // per-point records of this quadrant: source, stencil coefficients, wall terms
            for (int idx = threadIdx.x; idx < nrows * T1; idx += blockDim.x) {
                const int r = idx / T1;
                const int i = idx - r * T1;
                V r0 = Vec4<T>::make(0, 0, 0, 0), r1 = r0, r2 = r0;
                V r3 = Vec4<T>::make(bits_as(T(0), -1), bits_as(T(0), -1), bits_as(T(0), -1), bits_as(T(0), -1));
                if (i < width) {
                    const int ic = c0 + i;
                    const int x = s1neg ? n1 - 1 - ic : ic;
                    const int yo = row0 + r;
                    const int y = s2neg ? n2 - 1 - yo : yo;
                    const int id = y * n1 + x;
                    const uint16_t code = P->code[id];
                    if (!(code & kSolidBit)) {
                        const V s = reinterpret_cast<const V*>(P->src)[id];
                        const V e = reinterpret_cast<const V*>(P->E)[id];
                        const int ca = (code >> (2 * (0 + s1neg))) & 3;
                        const int cb = (code >> (2 * (2 + s2neg))) & 3;
                        r0 = Vec4<T>::make(s.x, s.y, s.z, s1neg ? e.y : e.x);
                        // case 1 (second upstream point solid): first order on h(x - s e_j)
                        r1 = Vec4<T>::make(ca == 2 ? T(0) : (ca == 1 ? T(1) : K1o), ca == 0 ? K2o : T(0),
                                           cb == 2 ? T(0) : (cb == 1 ? T(1) : K1o), cb == 0 ? K2o : T(0));
                        r2 = Vec4<T>::make(s2neg ? e.w : e.z, bits_as(T(0), (ca != 0) | ((cb != 0) << 1)),
                                           T(0), T(0));
                        if constexpr (SPEC) {
                            // faces: upstream (read) and downstream (written) along x1 and x2
                            const int* fi = P->face_id;
                            const size_t Nn = (size_t)N;
                            r3 = Vec4<T>::make(bits_as(T(0), fi[(0 + s1neg) * Nn + id]), bits_as(T(0), fi[(2 + s2neg) * Nn + id]),
                                               bits_as(T(0), fi[(1 - s1neg) * Nn + id]), bits_as(T(0), fi[(3 - s2neg) * Nn + id]));
                        }
                    }
                }
                V* R = reinterpret_cast<V*>(rec + (size_t)idx * RW);
                R[0] = r0;
                R[1] = r1;
                R[2] = r2;
                if constexpr (SPEC) R[3] = r3;
            }
            __syncthreads();
            if (s_abort) return;
            // the two rows below this band: the previous band's top edge, or lagged layers (the x2
            // ghosts at the domain face, the previous iteration's halo at a subdomain boundary)
            T rb1[T1], rb2[T1];
            {
                const T* eb = (below >= 0)
                    ? P->glat + (((size_t)(par * 4 + q) * P->nslots + below) * n1) * 2 * NL
                    : P->edge + ((size_t)(q * 2 * P->nslots + (-1 - below)) * n1) * 2 * NL;
#pragma unroll
                for (int i = 0; i < T1; ++i) {
                    if (i < width) {
                        rb1[i] = __ldcg(eb + ((size_t)(c0 + i) * 2 + 0) * NL + wl);
                        rb2[i] = __ldcg(eb + ((size_t)(c0 + i) * 2 + 1) * NL + wl);
                    } else {
                        rb1[i] = T(0);
                        rb2[i] = T(0);
                    }
                }
            }
            if (width == T1)
                sweep_tile_rows<T, T1, true, SPEC>(rec, part, carry, nrows, width, RB, warp, lane, L, rb1, rb2, SL);
            else
                sweep_tile_rows<T, T1, false, SPEC>(rec, part, carry, nrows, width, RB, warp, lane, L, rb1, rb2, SL);
            // top edge for the band above, or the x2 ghost layers of the next iteration (Eq. 8 /
            // periodic: the reflected quadrant reads the same lane)
            {
                T* et;
                if (above < 0) {
                    et = P->edge + ((size_t)(q * 2 * P->nslots + (-1 - above)) * n1) * 2 * NL;
                } else {
                    const int qd = (above > 0 || P->lateral == 1) ? q : (q ^ 2);
                    et = P->glat + (((size_t)((par ^ 1) * 4 + qd) * P->nslots + above) * n1) * 2 * NL;
                }
#pragma unroll
                for (int i = 0; i < T1; ++i) {
                    if (i < width) {
                        et[((size_t)(c0 + i) * 2 + 0) * NL + wl] = rb1[i];
                        et[((size_t)(c0 + i) * 2 + 1) * NL + wl] = rb2[i];
                    }
                }
            }
            // x1 ghost layers of the next iteration (periodic in x1, same quadrant) or the halo of
            // the next x1 subdomain
            if (tcur.w >= 0) carry_out(tcur.w);
            __syncthreads();
            // the band above only needs the edge: publish before combining the moment partials
            if (threadIdx.x == 0 && it != a.withhold_item) {
                publish_gpu(P->prog + q * nb + band, t + 1);
            }
            // moment partials of this quadrant: sum of the warps' lane sums, in warp order
            for (int idx = threadIdx.x; idx < nrows * width * 3; idx += blockDim.x) {
                const int m = idx % 3;
                const int pi = idx / 3;
                const int r = pi / width;
                const int i = pi - r * width;
                T s = T(0);
                for (int w = 0; w < NW; ++w) s += part[((size_t)(w * RB + r) * T1 + i) * 3 + m];
                const int ic = c0 + i;
                const int x = s1neg ? n1 - 1 - ic : ic;
                const int yo = row0 + r;
                const int y = s2neg ? n2 - 1 - yo : yo;
                P->P[((size_t)q * 3 + m) * N + (size_t)y * n1 + x] = s;
            }
            __syncthreads();
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- finalize

// rho'_s of face (y, axis j, side sigma) (Eq. 6) in FP64 from the quadrant partials of u_j at y:
// sum_{sigma v_j > 0} W |v_j| h / D = sigma * sum_{quadrants with sign(v_j) = sigma} P_uj / D.
template <typename T>
__device__ __forceinline__ double wall_density(const Prob2D<T>* P, int y, int j, int sigma, const double* dinv) {
    double num = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int neg = (q >> j) & 1;
        if (neg == (sigma < 0 ? 1 : 0)) num += (double)P->P[((size_t)q * 3 + 1 + j) * P->N + y];
    }
    return sigma * num * dinv[j];
}

// Points per finalize thread: a block of 256 threads covers 1024 consecutive points, thread t the
// points t, t + 256, t + 512 and t + 768 of its block (coalesced), with all of their loads issued
// before any store.
constexpr int kFinPPT = 4;

template <typename T>
__global__ void __launch_bounds__(256) finalize2d_kernel(const FinArgs2D<T> a) {
    using V = typename Vec4<T>::type;
    __shared__ double s_red[8];
    __shared__ int s_last;
    const int b = a.blk_prob[blockIdx.x];
    const Prob2D<T>* __restrict__ P = a.prob + b;
    const size_t N = P->N;
    double u1d = 0.0;
    int idk[kFinPPT];
    uint16_t code[kFinPPT];
    T pu[kFinPPT][4][3];     // quadrant partials (rho, u1, u2) of each point
#pragma unroll
    for (int k = 0; k < kFinPPT; ++k) {
        idk[k] = a.blk_start[blockIdx.x] + threadIdx.x + k * 256;
        code[k] = idk[k] < P->N ? P->code[idk[k]] : kSolidBit;
    }
#pragma unroll
    for (int k = 0; k < kFinPPT; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int m = 0; m < 3; ++m)
                pu[k][q][m] = idk[k] < P->N ? P->P[((size_t)q * 3 + m) * N + idk[k]] : T(0);   // zero at solid points
#pragma unroll
    for (int k = 0; k < kFinPPT; ++k) {
        const int id = idk[k];
        if (id >= P->N) continue;
        V s = Vec4<T>::make(0, 0, 0, 0), e = s;
        if (!(code[k] & kSolidBit)) {
            T rho = T(0), u1 = T(0), u2 = T(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                rho += pu[k][q][0];
                u1 += pu[k][q][1];
                u2 += pu[k][q][2];
            }
            const T nu = (T)P->nu;
            s = Vec4<T>::make(nu * rho, T(2) * nu * u1 + T(1), T(2) * nu * u2, T(0));
            u1d += (double)u1;
            T ev[4];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int c = (code[k] >> (2 * (2 * j + u))) & 3;
                    const int sigma = u ? 1 : -1;
                    double val = 0.0;
                    if (c == 2) {
                        // first-order stencil: wall value of face (x, j, sigma) (Eq. 6, rho'_s in
                        // FP64 from the partials of u_j of the quadrants moving toward the wall:
                        // sigma * sum / D), shifted by the source-form offset sigma dx on x1 faces
                        // (Eq. 5: alpha times the diffuse value, through the alpha-scaled
                        // denominators; the specular part is added per velocity by the sweep)
                        double num = 0.0;
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (((q >> j) & 1) == (sigma < 0 ? 1 : 0)) num += (double)pu[k][q][1 + j];
                        val = sigma * num * P->dinvw[j] + (j == 0 ? sigma * P->dx : 0.0);
                    }
                    // case 1 (only the second upstream point solid) is first order on the fluid
                    // neighbour: no wall term
                    ev[2 * j + u] = (T)val;
                }
            }
            e = Vec4<T>::make(ev[0], ev[1], ev[2], ev[3]);
        }
        reinterpret_cast<V*>(P->src)[id] = s;
        reinterpret_cast<V*>(P->E)[id] = e;
    }
    // FP64 block sum of u1 (fixed tree), then the last block of the problem adds the block sums in
    // block order: the permeability is independent of scheduling.
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) u1d += __shfl_xor_sync(0xffffffffu, u1d, off);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = u1d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_red[w];
        P->kpart[blockIdx.x - P->fin_block0] = tot;
        __threadfence();
        const unsigned prev = atomicAdd(P->fin_counter, 1u);
        s_last = (prev == (unsigned)P->fin_nblocks - 1u);
    }
    __syncthreads();
    if (s_last) {
        // all threads of the last block: strided partial sums in a fixed order, then a fixed tree
        __threadfence();
        double acc = 0.0;
        for (int k = threadIdx.x; k < P->fin_nblocks; k += blockDim.x) acc += __ldcg(P->kpart + k);
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_red[w];
            const double gp = tot / (double)P->N;
            P->kval[0] = 2.0 / sqrt(3.14159265358979323846) * P->kn * gp;
            P->kval[1] = gp;
            P->kval[2] = tot;
            *P->fin_counter = 0u;
        }
    }
}

// ---------------------------------------------------------------- init and readout

// Zero-perturbation start h = 0 in the paper's variables, i.e. h' = x1 in the kernels' variables:
// moment partials x1 * sum_{k in q} W_k (1, v1, v2) and ghost layers carrying x1 of their source
// points.  A finalize pass afterwards derives the source and wall terms.
template <typename T>
__global__ void init2d_kernel(const Prob2D<T>* prob, int NL, const double* qw /*[4][3]*/) {
    const Prob2D<T>* P = prob;
    const int n1 = P->n1, n2 = P->n2, N = P->N;
    const size_t nl = NL;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (size_t idx = t0; idx < (size_t)4 * 3 * N; idx += stride) {
        const int id = idx % N;
        const int qm = idx / N;
        const double x1 = (id % n1) * P->dx;
        P->P[idx] = (P->code[id] & kSolidBit) ? T(0) : (T)(x1 * qw[qm]);
    }
    const int nxs = P->nxslots;
    for (size_t idx = t0; idx < (size_t)2 * 4 * nxs * n2 * 2 * nl; idx += stride) {
        const int layer = (idx / nl) % 2;
        const int sl = (idx / (nl * 2 * n2)) % nxs;
        const int q = (idx / (nl * 2 * n2 * nxs)) % 4;
        const int ico = P->xslot_col[q * nxs + sl] - 1 - layer;     // oriented source column
        const int col = (q & 1) ? n1 - 1 - ico : ico;
        P->gx1[idx] = (T)(col * P->dx);
    }
    for (size_t idx = t0; idx < (size_t)2 * 4 * P->nslots * n1 * 2 * nl; idx += stride) {
        const int ic = (idx / (nl * 2)) % n1;
        const int q = (idx / (nl * 2 * n1 * P->nslots)) % 4;
        const int col = (q & 1) ? n1 - 1 - ic : ic;
        P->glat[idx] = (T)(col * P->dx);
    }
    if (P->spec > 0.0)   // face stores of both parities: h' = x1 at the face's fluid point
        for (size_t idx = t0; idx < (size_t)2 * P->nfaces * 2 * nl; idx += stride) {
            const int id = P->faces[(idx / (2 * nl)) % P->nfaces] >> 2;
            P->F[idx] = (T)((id % n1) * P->dx);
        }
}

// Warm start: the state an iteration leaves when it produced the local linearised equilibrium
// h0 = rho0 + 2 u0 . v at every fluid point (source form: h0' = h0 + x1).  Moment partials are the
// quadrant quadratures of h0' (closed form through qw2[q][m][n] = sum_{k in q} W phi_m psi_n with
// phi = psi = (1, v1, v2)); the lagged ghost layers read at parity `par` hold h0' at the points the
// sweep would have captured them from (same slot layout as the sweep kernels write).
template <typename T>
__global__ void warm2d_kernel(const Prob2D<T>* P, int NL, int par, const double* __restrict__ qw2,
                              const double* __restrict__ vel, const double* __restrict__ rho0,
                              const double* __restrict__ u0) {
    const int n1 = P->n1, n2 = P->n2, N = P->N;
    const size_t nl = NL;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    auto h0 = [&](int x, int y, const double* v) -> double {
        const int id = y * n1 + x;
        if (P->code[id] & kSolidBit) return 0.0;
        return rho0[id] + x * P->dx + 2.0 * (u0[id] * v[0] + u0[N + id] * v[1]);
    };
    for (size_t idx = t0; idx < (size_t)4 * 3 * N; idx += stride) {
        const int id = idx % N;
        const int qm = idx / N;
        double val = 0.0;
        if (!(P->code[id] & kSolidBit)) {
            const double* c = qw2 + (size_t)qm * 3;
            const double r = rho0[id] + (id % n1) * P->dx;
            val = r * c[0] + 2.0 * (u0[id] * c[1] + u0[N + id] * c[2]);
        }
        P->P[idx] = (T)val;
    }
    // lagged x1 layers: slot (q, s, oriented row, layer) holds h at the oriented column
    // xslot_col[q][s] - 1 - layer (slot 0: the x1 ghosts, columns n1 - 1 - layer)
    const int nxs = P->nxslots;
    for (size_t idx = t0; idx < (size_t)4 * nxs * n2 * 2 * nl; idx += stride) {
        const int l = idx % nl;
        const int layer = (idx / nl) % 2;
        const int yo = (idx / (nl * 2)) % n2;
        const int sl = (idx / (nl * 2 * n2)) % nxs;
        const int q = idx / (nl * 2 * n2 * nxs);
        const int ico = P->xslot_col[q * nxs + sl] - 1 - layer;
        const int x = (q & 1) ? n1 - 1 - ico : ico;
        const int y = (q & 2) ? n2 - 1 - yo : yo;
        P->gx1[(size_t)par * 4 * nxs * n2 * 2 * nl + idx] = (T)h0(x, y, vel + ((size_t)q * nl + l) * 2);
    }
    // lagged x2 layers: quadrant q writes the oriented rows below slot s (slot 0: its top rows
    // n2 - 1 - layer) into the slot of the quadrant that reads them (slot 0: itself when periodic,
    // the x2-reflected quadrant when specular; subdomain slots: itself)
    const int ns = P->nslots;
    for (size_t idx = t0; idx < (size_t)4 * ns * n1 * 2 * nl; idx += stride) {
        const int l = idx % nl;
        const int layer = (idx / nl) % 2;
        const int ic = (idx / (nl * 2)) % n1;
        const int sl = (idx / (nl * 2 * n1)) % ns;
        const int q = idx / (nl * 2 * n1 * ns);
        const int x = (q & 1) ? n1 - 1 - ic : ic;
        const int yo = P->slot_row[q * ns + sl] - 1 - layer;
        const int y = (q & 2) ? n2 - 1 - yo : yo;
        const int qd = (sl > 0 || P->lateral == 1) ? q : (q ^ 2);
        P->glat[(((((size_t)par * 4 + qd) * ns + sl) * n1 + ic) * 2 + layer) * nl + l] =
            (T)h0(x, y, vel + ((size_t)q * nl + l) * 2);
    }
    // face stores (specular wall part, Eq. 5): h0' at the face's fluid point for the velocity slot
    // of the quadrant that moves into the face (s_j = the face side, other-axis sign bit o)
    if (P->spec > 0.0)
        for (size_t idx = t0; idx < (size_t)P->nfaces * 2 * nl; idx += stride) {
            const int l = idx % nl;
            const int o = (idx / nl) % 2;
            const int f = P->faces[idx / (2 * nl)];
            const int id = f >> 2, j = (f >> 1) & 1, u = f & 1;
            const int qw = (j == 0) ? ((1 - u) | (o << 1)) : (o | ((1 - u) << 1));
            P->F[(size_t)par * P->nfaces * 2 * nl + idx] = (T)h0(id % n1, id / n1, vel + ((size_t)qw * nl + l) * 2);
        }
}

// rho (paper variables, ramp restored) and u of one problem into double buffers; solid = 0.
template <typename T>
__global__ void moments2d_kernel(const Prob2D<T>* prob, double* rho, double* u) {
    const Prob2D<T>* P = prob;
    const int N = P->N;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        if (P->code[id] & kSolidBit) {
            rho[id] = 0.0;
            u[id] = 0.0;
            u[N + id] = 0.0;
            continue;
        }
        T r = T(0), u1 = T(0), u2 = T(0);
        for (int q = 0; q < 4; ++q) {
            r += P->P[((size_t)q * 3 + 0) * N + id];
            u1 += P->P[((size_t)q * 3 + 1) * N + id];
            u2 += P->P[((size_t)q * 3 + 2) * N + id];
        }
        rho[id] = (double)r - (id % P->n1) * P->dx;
        u[id] = (double)u1;
        u[N + id] = (double)u2;
    }
}

// Wall densities [2][2][N] (axis, side) in the paper's variables; 0 where there is no face.
template <typename T>
__global__ void wall2d_kernel(const Prob2D<T>* prob, double* out) {
    const Prob2D<T>* P = prob;
    const int N = P->N;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const uint16_t code = P->code[id];
        for (int j = 0; j < 2; ++j)
            for (int u = 0; u < 2; ++u) {
                double v = 0.0;
                if (!(code & kSolidBit) && ((code >> (2 * (2 * j + u))) & 3) == 2)
                    v = wall_density(P, id, j, u ? 1 : -1, P->dinv) - (id % P->n1) * P->dx;
                out[(size_t)(2 * j + u) * N + id] = v;
            }
    }
}

// ---------------------------------------------------------------- launchers

template <typename T>
size_t sweep2d_smem(int T1, int NW, int max_rows, int spec) {
    return sizeof(T) * ((size_t)max_rows * T1 * (spec ? 16 : kRecWords) + (size_t)NW * max_rows * T1 * 3 +
                        (size_t)NW * max_rows * 2 * 32);
}

template <typename T, int T1, bool XS, bool SPEC>
static cudaError_t launch_sweep_t(const SweepArgs2D<T>& a, int grid, int NW, cudaStream_t st) {
    const size_t smem = sweep2d_smem<T>(T1, NW, a.max_rows, SPEC);
    cudaError_t e = cudaFuncSetAttribute(sweep2d_kernel<T, T1, XS, SPEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sweep2d_kernel<T, T1, XS, SPEC><<<grid, NW * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int T1>
static cudaError_t launch_sweep_tt(const SweepArgs2D<T>& a, int xs, int grid, int NW, cudaStream_t st) {
    if (a.spec) return xs ? launch_sweep_t<T, T1, true, true>(a, grid, NW, st) : launch_sweep_t<T, T1, false, true>(a, grid, NW, st);
    return xs ? launch_sweep_t<T, T1, true, false>(a, grid, NW, st) : launch_sweep_t<T, T1, false, false>(a, grid, NW, st);
}

// xs: x1 subdomains (tile tables and lagged x1 halos); a.spec: specular wall parts (Eq. 5)
template <typename T>
cudaError_t launch_sweep2d(const SweepArgs2D<T>& a, int T1, int xs, int grid, int NW, cudaStream_t st) {
    if (T1 == 8) return launch_sweep_tt<T, 8>(a, xs, grid, NW, st);
    if (T1 == 16) return launch_sweep_tt<T, 16>(a, xs, grid, NW, st);
    return cudaErrorInvalidValue;
}

template <typename T, int T1, bool XS, bool SPEC>
static cudaError_t occ2(int NW, int max_rows, int* blocks_per_sm) {
    const size_t smem = sweep2d_smem<T>(T1, NW, max_rows, SPEC);
    cudaError_t e = cudaFuncSetAttribute(sweep2d_kernel<T, T1, XS, SPEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, sweep2d_kernel<T, T1, XS, SPEC>, NW * 32, smem);
}

template <typename T, int T1>
static cudaError_t occ2_t(int xs, int spec, int NW, int max_rows, int* bps) {
    if (spec) return xs ? occ2<T, T1, true, true>(NW, max_rows, bps) : occ2<T, T1, false, true>(NW, max_rows, bps);
    return xs ? occ2<T, T1, true, false>(NW, max_rows, bps) : occ2<T, T1, false, false>(NW, max_rows, bps);
}

template <typename T>
cudaError_t sweep2d_occupancy(int T1, int xs, int spec, int NW, int max_rows, int* blocks_per_sm) {
    if (T1 == 8) return occ2_t<T, 8>(xs, spec, NW, max_rows, blocks_per_sm);
    if (T1 == 16) return occ2_t<T, 16>(xs, spec, NW, max_rows, blocks_per_sm);
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_finalize2d(const FinArgs2D<T>& a, int nblocks, cudaStream_t st) {
    finalize2d_kernel<T><<<nblocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init2d(const Prob2D<T>* prob_dev, int NL, const double* qw_dev, cudaStream_t st) {
    init2d_kernel<T><<<304, 256, 0, st>>>(prob_dev, NL, qw_dev);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_warm2d(const Prob2D<T>* prob_dev, int NL, int par, const double* qw2, const double* vel,
                          const double* rho0, const double* u0, cudaStream_t st) {
    warm2d_kernel<T><<<304, 256, 0, st>>>(prob_dev, NL, par, qw2, vel, rho0, u0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_moments2d(const Prob2D<T>* prob_dev, double* rho, double* u, cudaStream_t st) {
    moments2d_kernel<T><<<304, 256, 0, st>>>(prob_dev, rho, u);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_wall2d(const Prob2D<T>* prob_dev, double* out, cudaStream_t st) {
    wall2d_kernel<T><<<304, 256, 0, st>>>(prob_dev, out);
    return cudaGetLastError();
}

#define DVM_INSTANTIATE(T)                                                                      \
    template size_t sweep2d_smem<T>(int, int, int, int);                                       \
    template cudaError_t launch_sweep2d<T>(const SweepArgs2D<T>&, int, int, int, int, cudaStream_t); \
    template cudaError_t sweep2d_occupancy<T>(int, int, int, int, int, int*);                  \
    template cudaError_t launch_finalize2d<T>(const FinArgs2D<T>&, int, cudaStream_t);          \
    template cudaError_t launch_init2d<T>(const Prob2D<T>*, int, const double*, cudaStream_t);  \
    template cudaError_t launch_warm2d<T>(const Prob2D<T>*, int, int, const double*, const double*, \
                                          const double*, const double*, cudaStream_t);            \
    template cudaError_t launch_moments2d<T>(const Prob2D<T>*, double*, double*, cudaStream_t); \
    template cudaError_t launch_wall2d<T>(const Prob2D<T>*, double*, cudaStream_t);

DVM_INSTANTIATE(float)
DVM_INSTANTIATE(double)

}  // namespace dvm
