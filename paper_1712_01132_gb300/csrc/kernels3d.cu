// kernels3d.cu -- sm_103a kernels of one source iteration (arXiv:1712.01132, Sec. 3.1) in 3D.
//
// sweep3d   : step (i) for every octant of discrete velocities (Fig. 1 generalised to octants),
//             with the quadrature of step (iii) fused in.  A work item is (problem, octant,
//             velocity group, pencil); a pencil is R2 x R3 rows (x2 x x3) swept along x1 in tiles
//             of T1 columns.  Items are ordered by pencil level p2 + p3: a pencil waits only on
//             (p2-1, p3) and (p2, p3-1), which carry lower tickets, so the persistent schedule
//             cannot deadlock.  One discrete velocity per lane.  Inside a tile the rows are walked
//             plane by plane (x3), row by row (x2), x1 fastest: every value a point reads is final,
//             so the result equals the paper's raster scan.  Serves FP64, and both precisions of
//             the Shakhov and ES-BGK model variants (NX = 3 or 6 model moments per point).
// finalize3d: sums the octant/group moment partials, forms the FP64 wall densities (Eq. 6), the
//             next sources and wall terms, and the FP64 sum of u1 for Eq. 11-12.
// init3d, warm3d, moments3d, temperature3d, modelmoments3d, wall3d: start states and readouts.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "dvm_device.cuh"
#include "dvm_internal.h"

namespace dvm {

namespace {

constexpr int kRec3 = 16;    // record: {a b1 b2 b3} {E1 E2 E3 rsel} {K1x K2x K1y K2y} {K1z K2z - -}

template <typename T> struct V4t;
template <> struct V4t<float> {
    using type = float4;
    static __device__ __forceinline__ float4 make(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
};
struct alignas(32) d4 { double x, y, z, w; };
template <> struct V4t<double> {
    using type = d4;
    static __device__ __forceinline__ d4 make(double a, double b, double c, double d) { return d4{a, b, c, d}; }
};

__device__ __forceinline__ float ibits(float, int v) { return __int_as_float(v); }
__device__ __forceinline__ double ibits(double, int v) { return __longlong_as_double((long long)v); }
__device__ __forceinline__ int tbits(float v) { return __float_as_int(v); }
__device__ __forceinline__ int tbits(double v) { return (int)__double_as_longlong(v); }

// Transient h kept in HBM between pencils and iterations (ghost layers, pencil edges): stored as T,
// or (BF16 storage ablation) as the BF16 rounding (round to nearest even) of the deviation from the
// x1 ramp, h' - x1 with x1 the coordinate of the point the value belongs to, which keeps the
// stored numbers at the size of the perturbation instead of the O(1) ramp.
template <typename T, bool BF> struct HStore {
    static __device__ __forceinline__ T ld(const T* b, size_t i, T) { return __ldcg(b + i); }
    static __device__ __forceinline__ void st(T* b, size_t i, T v, T) { b[i] = v; }
};
template <> struct HStore<float, true> {
    static __device__ __forceinline__ float ld(const float* b, size_t i, float x1) {
        const unsigned short u = __ldcg(reinterpret_cast<const unsigned short*>(b) + i);
        return __bfloat162float(__ushort_as_bfloat16(u)) + x1;
    }
    static __device__ __forceinline__ void st(float* b, size_t i, float v, float x1) {
        reinterpret_cast<__nv_bfloat16*>(b)[i] = __float2bfloat16_rn(v - x1);
    }
};

}  // namespace

template <typename T, int T1, bool BF, bool SUB, bool TAU, bool SPEC, int NX>
__global__ void __launch_bounds__(256) sweep3d_kernel(const SweepArgs3D<T> a) {
    using V = typename V4t<T>::type;
    using HS = HStore<T, BF>;
    static_assert(NX == 0 || ((NX == 3 || NX == 6) && TAU && !SPEC),
                  "model moments (Shakhov 3, ES-BGK 6) go with the temperature term, without specular parts");
    // moments per point: rho, u1..u3 (, sum W |v|^2 h) (, the NX model moments sum W psi_a h)
    constexpr int NM = NX > 0 ? 5 + NX : (TAU ? 5 : 4);
    // record words: face ids (specular parts) or nu xcoef m_a (model moments) in more vectors
    constexpr int RW = SPEC ? 24 : (NX == 3 ? 20 : (NX == 6 ? 24 : kRec3));
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    __shared__ int s_abort;
    const int NW = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int MR2 = a.maxR2, MR3 = a.maxR3;
    const int MROWS = MR2 * MR3;
    T* rec = reinterpret_cast<T*>(smem_raw);                         // [MROWS][T1][RW]
    T* part = rec + (size_t)MROWS * T1 * RW;                         // [NW][MROWS][T1][NM]
    T* carry = part + (size_t)NW * MROWS * T1 * NM;                  // [NW][MROWS][2][32]
    T* pb = carry + (size_t)NW * MROWS * 2 * 32;                     // [NW][MR2][2][T1][32]
    T* rtab = pb + (size_t)NW * MR2 * 2 * T1 * 32;                   // [NW][8][32]
    const size_t NL = (size_t)a.NL;

    for (;;) {
        if (threadIdx.x == 0) {
            s_item = ld_volatile(a.status) ? a.nitems : atomicAdd(a.ticket, 1);
            s_abort = 0;
        }
        __syncthreads();
        const int it = s_item;
        if (it >= a.nitems) return;
        const SweepItem3 item = a.items[it];
        const Prob3D<T>* __restrict__ P = a.prob + item.prob;
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
        const T K1o = P->order == 2 ? T(2) : T(1);
        const T K2o = P->order == 2 ? T(-0.5) : T(0);
        const int lv = g * a.GL + warp * 32 + lane;      // velocity lane within the octant
        const T* lcp = P->lanec + ((size_t)q * NL + lv) * kLaneConsts3;
        const T v1 = lcp[0], v2 = lcp[1], v3 = lcp[2], a1 = lcp[3], a2 = lcp[4], a3 = lcp[5];
        const T W = lcp[6], Wv1 = lcp[7], Wv2 = lcp[8], Wv3 = lcp[9];
        const T vq = lcp[18], Wvv = lcp[19];             // |v|^2 - 3/2 and W |v|^2 (temperature term)
        // model moments: source factors phi_a and quadrature weights W psi_a
        T xf[NX > 0 ? NX : 1], xw[NX > 0 ? NX : 1];
#pragma unroll
        for (int m = 0; m < NX; ++m) {
            xf[m] = lcp[20 + m];
            xw[m] = lcp[26 + m];
        }
        T* my_rtab = rtab + (size_t)warp * 8 * 32 + lane;
#pragma unroll
        for (int rs = 0; rs < 8; ++rs) my_rtab[rs * 32] = lcp[10 + rs];
        const int par = a.parity;
        const int G = P->ngroups;
        int* prog = P->prog + ((size_t)q * G + g) * np3 * np2;
        // specular wall parts (Eq. 5, alpha < 1): face stores of the previous iteration (read where
        // an upstream point is solid) and of this one (written where a downstream point is solid)
        const T* fprev[3] = {nullptr, nullptr, nullptr};
        T* fnext[3] = {nullptr, nullptr, nullptr};
        const size_t fstride = 4 * NL;
        if constexpr (SPEC) {
            const size_t plane = (size_t)P->nfaces * 4 * NL;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                fprev[j] = P->F + par * plane + (size_t)other_bits3(q, j) * NL + lv;
                fnext[j] = P->F + (par ^ 1) * plane + (size_t)other_bits3(q, j) * NL + lv;
            }
        }
        const T specT = (T)P->spec;
        // x1 coordinate of oriented column ic (the shift of the BF16 storage)
        const T dxT = (T)P->dx;
        auto x1of = [&](int ic) -> T { return (T)(s1n ? n1 - 1 - ic : ic) * dxT; };
        const T x1g0 = x1of(n1 - 1), x1g1 = x1of(n1 - 2);   // columns of the x1 ghost layers
        const int ntiles = SUB ? P->nt1 : (n1 + T1 - 1) / T1;
        // neighbour progress thread 0 has already observed with an acquire (tiles up to it need no
        // new wait)
        int seen2 = pi2.z < 0 ? -1 : ntiles, seen3 = pi3.z < 0 ? -1 : ntiles;
        for (int t = 0; t < ntiles; ++t) {
            // tile: first oriented column, width, x1 carry-in and carry-out ghost slots (or -1)
            int4 ti;
            if constexpr (SUB) ti = P->tiles1[s1n * ntiles + t];
            else ti = make_int4(t * T1, min(T1, n1 - t * T1), t == 0 ? 0 : -1, t == ntiles - 1 ? 0 : -1);
            const int c0 = ti.x;
            const int width = ti.y;
            if (threadIdx.x == 0) {
                if (seen2 < t + 1) seen2 = wait_geq_value(prog + p3 * np2 + p2 - 1, t + 1, a.status, a.timeout_ns);
                if (seen2 >= 0 && seen3 < t + 1) seen3 = wait_geq_value(prog + (p3 - 1) * np2 + p2, t + 1, a.status, a.timeout_ns);
                if (seen2 < 0 || seen3 < 0) s_abort = 1;
            }
            // records of the tile's points for this octant
            const int npts = nr3 * MR2 * T1;
            int anyf = 0;                         // a fluid point among this thread's
            for (int idx = threadIdx.x; idx < npts; idx += blockDim.x) {
                const int kk = idx / (MR2 * T1);
                const int rem = idx - kk * MR2 * T1;
                const int jj = rem / T1;
                const int i = rem - jj * T1;
                V r0 = V4t<T>::make(0, 0, 0, 0), r1 = r0, r2 = r0, r3 = r0;
                V r4 = V4t<T>::make(ibits(T(0), -1), ibits(T(0), -1), ibits(T(0), -1), ibits(T(0), -1)), r5 = r4;
                if constexpr (NX > 0) r4 = r5 = V4t<T>::make(0, 0, 0, 0);   // no model source off the fluid
                if (jj < nr2 && i < width) {
                    const int ic = c0 + i;
                    const int x = s1n ? n1 - 1 - ic : ic;
                    const int y = s2n ? n2 - 1 - (j0 + jj) : (j0 + jj);
                    const int z = s3n ? n3 - 1 - (k0 + kk) : (k0 + kk);
                    const int id = (z * n2 + y) * n1 + x;
                    const uint16_t code = P->code[id];
                    if (!(code & kSolidBit)) {
                        anyf = 1;
                        const V s = reinterpret_cast<const V*>(P->src)[id];
                        const V e0 = reinterpret_cast<const V*>(P->E)[2 * (size_t)id];
                        const V e1 = reinterpret_cast<const V*>(P->E)[2 * (size_t)id + 1];
                        const int ca = (code >> (2 * (0 + s1n))) & 3;
                        const int cb = (code >> (2 * (2 + s2n))) & 3;
                        const int cc = (code >> (2 * (4 + s3n))) & 3;
                        const T E1 = s1n ? e0.y : e0.x;
                        const T E2 = s2n ? e0.w : e0.z;
                        const T E3 = s3n ? e1.y : e1.x;
                        // first-order denominator when either upstream point is solid (cases 1, 2)
                        const int rs = (ca != 0) | ((cb != 0) << 1) | ((cc != 0) << 2);
                        r0 = V4t<T>::make(s.x, s.y, s.z, s.w);
                        r1 = V4t<T>::make(E1, E2, E3, ibits(T(0), rs));
                        r2 = V4t<T>::make(ca == 2 ? T(0) : (ca == 1 ? T(1) : K1o), ca == 0 ? K2o : T(0),
                                          cb == 2 ? T(0) : (cb == 1 ? T(1) : K1o), cb == 0 ? K2o : T(0));
                        r3 = V4t<T>::make(cc == 2 ? T(0) : (cc == 1 ? T(1) : K1o), cc == 0 ? K2o : T(0),
                                          TAU ? P->srct[id] : T(0), T(0));
                        if constexpr (SPEC) {   // faces: upstream (read) x1 x2 x3, downstream (written)
                            const int* fi = P->face_id;
                            const size_t Nn = (size_t)N;
                            r4 = V4t<T>::make(ibits(T(0), fi[(0 + s1n) * Nn + id]), ibits(T(0), fi[(2 + s2n) * Nn + id]),
                                              ibits(T(0), fi[(4 + s3n) * Nn + id]), ibits(T(0), fi[(1 - s1n) * Nn + id]));
                            r5 = V4t<T>::make(ibits(T(0), fi[(3 - s2n) * Nn + id]), ibits(T(0), fi[(5 - s3n) * Nn + id]),
                                              ibits(T(0), -1), ibits(T(0), -1));
                        }
                        if constexpr (NX > 0) {   // nu xcoef m_a
                            r4 = reinterpret_cast<const V*>(P->srcx)[2 * (size_t)id];
                            r5 = reinterpret_cast<const V*>(P->srcx)[2 * (size_t)id + 1];
                        }
                    }
                }
                V* R = reinterpret_cast<V*>(rec + (size_t)((kk * MR2 + jj) * T1 + i) * RW);
                R[0] = r0;
                R[1] = r1;
                R[2] = r2;
                R[3] = r3;
                if constexpr (SPEC) {
                    R[4] = r4;
                    R[5] = r5;
                }
                if constexpr (NX > 0) R[4] = r4;
                if constexpr (NX > 4) R[5] = r5;
            }
            // A tile without fluid points is not swept: nothing it would compute or store is read
            // (every fluid reader of one of its points has a zero coefficient for it, and the
            // carries, planes, edges and ghost layers it leaves as they were hold finite values).
            // It still waits for its neighbours and publishes, which keeps the ring slots' order.
            const bool tfl = __syncthreads_or(anyf) != 0;
            if (s_abort) return;
            // x1 upstream of the tile's first column when it starts a block: x1 ghost layers of
            // the previous iteration in slot ti.z (oriented rows (k, j))
            if (ti.z >= 0) {
                const size_t gxo = ((((size_t)par * 8 + q) * P->ns1 + ti.z) * n3 * n2) * 2 * NL;
                for (int kk = 0; kk < nr3; ++kk)
                    for (int jj = 0; jj < nr2; ++jj) {
                        const size_t row = (size_t)(k0 + kk) * n2 + (j0 + jj);
                        T* cr = carry + ((size_t)(warp * MROWS + kk * MR2 + jj) * 2) * 32 + lane;
                        cr[0] = HS::ld(P->gx1, gxo + (row * 2 + 0) * NL + lv, x1g0);
                        cr[32] = HS::ld(P->gx1, gxo + (row * 2 + 1) * NL + lv, x1g1);
                    }
            }
            if (tfl) {
            // x3 upstream planes of the first plane of the pencil: the pencil below in x3 (ring
            // slot) or ghost slot pi3.z (x3 ghost layers, periodic or specular, Eq. 8, or the
            // lagged halo of the block below)
            {
                const bool zg = pi3.z >= 0;
                const T* zb = zg ? P->gz : P->ez;
                const size_t zo = zg
                    ? ((((size_t)par * 8 + q) * P->ns3 + pi3.z) * n2 * n1) * 2 * NL
                    : ((((size_t)q * np2 + p2) * 2 * P->ns3 + (-1 - pi3.z)) * P->R2 * n1) * 2 * NL;
                for (int jj = 0; jj < nr2; ++jj)
                    for (int i = 0; i < width; ++i) {
                        const size_t row = zg ? ((size_t)(j0 + jj) * n1 + (c0 + i)) : ((size_t)jj * n1 + (c0 + i));
                        T* d = pb + ((((size_t)warp * MR2 + jj) * 2) * T1 + i) * 32 + lane;
                        const T xs = x1of(c0 + i);
                        d[0] = HS::ld(zb, zo + (row * 2 + 0) * NL + lv, xs);
                        d[(size_t)T1 * 32] = HS::ld(zb, zo + (row * 2 + 1) * NL + lv, xs);
                    }
            }
            for (int kk = 0; kk < nr3; ++kk) {
                // x2 upstream rows of the first row of this plane
                T rb1[T1], rb2[T1];
                {
                    const bool yg = pi2.z >= 0;
                    const T* yb = yg ? P->gy : P->ey;
                    const size_t yo = yg
                        ? ((((size_t)par * 8 + q) * P->ns2 + pi2.z) * n3 * n1) * 2 * NL
                        : ((((size_t)q * np3 + p3) * 2 * P->ns2 + (-1 - pi2.z)) * P->R3 * n1) * 2 * NL;
                    const size_t rowbase = yg ? (size_t)(k0 + kk) * n1 : (size_t)kk * n1;
#pragma unroll
                    for (int i = 0; i < T1; ++i) {
                        if (i < width) {
                            const T xs = x1of(c0 + i);
                            rb1[i] = HS::ld(yb, yo + ((rowbase + c0 + i) * 2 + 0) * NL + lv, xs);
                            rb2[i] = HS::ld(yb, yo + ((rowbase + c0 + i) * 2 + 1) * NL + lv, xs);
                        } else {
                            rb1[i] = T(0);
                            rb2[i] = T(0);
                        }
                    }
                }
                for (int jj = 0; jj < nr2; ++jj) {
                    T* cr = carry + ((size_t)(warp * MROWS + kk * MR2 + jj) * 2) * 32 + lane;
                    T hp1 = cr[0], hp2 = cr[32];
                    T* zr = pb + ((((size_t)warp * MR2 + jj) * 2) * T1) * 32 + lane;   // [2][T1][32]
                    const T* rrow = rec + (size_t)((kk * MR2 + jj) * T1) * RW;
                    T* prow = part + ((size_t)(warp * MROWS + kk * MR2 + jj) * T1) * NM;
#pragma unroll
                    for (int i0 = 0; i0 < T1; i0 += 4) {
                        T m0[4], m1[4], m2[4], m3[4], m4[4], mx[NX > 0 ? NX : 1][4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int i = i0 + c;
                            if (i < width) {
                                const V* R = reinterpret_cast<const V*>(rrow + i * RW);
                                const V A = R[0], B = R[1], C = R[2], D = R[3];
                                const T z1 = zr[(size_t)i * 32];
                                const T z2 = zr[((size_t)T1 + i) * 32];
                                T S = fma(A.w, v3, fma(A.z, v2, fma(A.y, v1, A.x)));
                                if constexpr (TAU) S = fma(D.z, vq, S);   // nu tau (|v|^2 - 3/2)
                                if constexpr (NX > 0) {   // nu xcoef sum_a m_a phi_a(v)
                                    const V X0 = R[4];
                                    S = fma(X0.z, xf[2], fma(X0.y, xf[1], fma(X0.x, xf[0], S)));
                                    if constexpr (NX == 6) {
                                        const V X1 = R[5];
                                        S = fma(X1.y, xf[5], fma(X1.x, xf[4], fma(X0.w, xf[3], S)));
                                    }
                                }
                                T t1 = fma(C.x, hp1, fma(C.y, hp2, B.x));
                                T t2 = fma(C.z, rb1[i], fma(C.w, rb2[i], B.y));
                                T t3 = fma(D.x, z1, fma(D.y, z2, B.z));
                                V Fa, Fb;
                                if constexpr (SPEC) {   // + (1 - alpha) h'(x, reflected v) at walls
                                    Fa = R[4];
                                    Fb = R[5];
                                    const int fu1 = tbits(Fa.x), fu2 = tbits(Fa.y), fu3 = tbits(Fa.z);
                                    if (fu1 >= 0) t1 = fma(specT, fprev[0][(size_t)fu1 * fstride], t1);
                                    if (fu2 >= 0) t2 = fma(specT, fprev[1][(size_t)fu2 * fstride], t2);
                                    if (fu3 >= 0) t3 = fma(specT, fprev[2][(size_t)fu3 * fstride], t3);
                                }
                                const T num = fma(a3, t3, fma(a2, t2, fma(a1, t1, S)));
                                const T h = num * my_rtab[tbits(B.w) * 32];
                                if constexpr (SPEC) {   // molecules moving into a downstream face
                                    const int fd1 = tbits(Fa.w), fd2 = tbits(Fb.x), fd3 = tbits(Fb.y);
                                    if (fd1 >= 0) fnext[0][(size_t)fd1 * fstride] = h;
                                    if (fd2 >= 0) fnext[1][(size_t)fd2 * fstride] = h;
                                    if (fd3 >= 0) fnext[2][(size_t)fd3 * fstride] = h;
                                }
                                hp2 = hp1;
                                hp1 = h;
                                rb2[i] = rb1[i];
                                rb1[i] = h;
                                zr[((size_t)T1 + i) * 32] = z1;
                                zr[(size_t)i * 32] = h;
                                m0[c] = W * h;
                                m1[c] = Wv1 * h;
                                m2[c] = Wv2 * h;
                                m3[c] = Wv3 * h;
                                m4[c] = Wvv * h;
#pragma unroll
                                for (int m = 0; m < NX; ++m) mx[m][c] = xw[m] * h;
                            } else {
                                m0[c] = m1[c] = m2[c] = m3[c] = m4[c] = T(0);
#pragma unroll
                                for (int m = 0; m < NX; ++m) mx[m][c] = T(0);
                            }
                        }
                        const T r0 = reduce_scatter<T, 4>(m0, lane);
                        const T r1 = reduce_scatter<T, 4>(m1, lane);
                        const T r2 = reduce_scatter<T, 4>(m2, lane);
                        const T r3 = reduce_scatter<T, 4>(m3, lane);
                        T r4 = T(0), rx[NX > 0 ? NX : 1];
                        if constexpr (TAU) r4 = reduce_scatter<T, 4>(m4, lane);
#pragma unroll
                        for (int m = 0; m < NX; ++m) rx[m] = reduce_scatter<T, 4>(mx[m], lane);
                        const int p = lane >> 3;
                        if ((lane & 7) == 0 && i0 + p < width) {
                            T* d = prow + (i0 + p) * NM;
                            d[0] = r0;
                            d[1] = r1;
                            d[2] = r2;
                            d[3] = r3;
                            if constexpr (TAU) d[4] = r4;
#pragma unroll
                            for (int m = 0; m < NX; ++m) d[5 + m] = rx[m];
                        }
                    }
                    cr[0] = hp1;
                    cr[32] = hp2;
                }
                // x2 edge of this plane for the pencil above in x2 (ring slot), or ghost slot pi2.w
                // of the next iteration: the halo of the next block, or at the domain face the x2
                // ghost layers (periodic: same octant; specular: octant with s2 flipped)
                {
                    T* et;
                    size_t eo, rowbase;
                    if (pi2.w < 0) {
                        et = P->ey;
                        eo = ((((size_t)q * np3 + p3) * 2 * P->ns2 + (-1 - pi2.w)) * P->R3 * n1) * 2 * NL;
                        rowbase = (size_t)kk * n1;
                    } else {
                        const int qy = (pi2.w > 0 || P->lateral == 1) ? q : (q ^ 2);
                        et = P->gy;
                        eo = ((((size_t)(par ^ 1) * 8 + qy) * P->ns2 + pi2.w) * n3 * n1) * 2 * NL;
                        rowbase = (size_t)(k0 + kk) * n1;
                    }
#pragma unroll
                    for (int i = 0; i < T1; ++i) {
                        if (i < width) {
                            const T xs = x1of(c0 + i);
                            HS::st(et, eo + ((rowbase + c0 + i) * 2 + 0) * NL + lv, rb1[i], xs);
                            HS::st(et, eo + ((rowbase + c0 + i) * 2 + 1) * NL + lv, rb2[i], xs);
                        }
                    }
                }
            }
            // x3 edge for the pencil above in x3 (ring slot), or ghost slot pi3.w of the next
            // iteration
            {
                T* et;
                size_t eo;
                const bool last = pi3.w >= 0;
                if (!last) {
                    et = P->ez;
                    eo = ((((size_t)q * np2 + p2) * 2 * P->ns3 + (-1 - pi3.w)) * P->R2 * n1) * 2 * NL;
                } else {
                    const int qz = (pi3.w > 0 || P->lateral == 1) ? q : (q ^ 4);
                    et = P->gz;
                    eo = ((((size_t)(par ^ 1) * 8 + qz) * P->ns3 + pi3.w) * n2 * n1) * 2 * NL;
                }
                for (int jj = 0; jj < nr2; ++jj)
                    for (int i = 0; i < width; ++i) {
                        const size_t row = last ? ((size_t)(j0 + jj) * n1 + (c0 + i)) : ((size_t)jj * n1 + (c0 + i));
                        const T* s = pb + ((((size_t)warp * MR2 + jj) * 2) * T1 + i) * 32 + lane;
                        const T xs = x1of(c0 + i);
                        HS::st(et, eo + (row * 2 + 0) * NL + lv, s[0], xs);
                        HS::st(et, eo + (row * 2 + 1) * NL + lv, s[(size_t)T1 * 32], xs);
                    }
            }
            }   // tfl
            if (ti.w >= 0 && tfl) {   // x1 carry into ghost slot ti.w of the next iteration
                const size_t gxo = ((((size_t)(par ^ 1) * 8 + q) * P->ns1 + ti.w) * n3 * n2) * 2 * NL;
                for (int kk = 0; kk < nr3; ++kk)
                    for (int jj = 0; jj < nr2; ++jj) {
                        const size_t row = (size_t)(k0 + kk) * n2 + (j0 + jj);
                        const T* cr = carry + ((size_t)(warp * MROWS + kk * MR2 + jj) * 2) * 32 + lane;
                        HS::st(P->gx1, gxo + (row * 2 + 0) * NL + lv, cr[0], x1g0);
                        HS::st(P->gx1, gxo + (row * 2 + 1) * NL + lv, cr[32], x1g1);
                    }
            }
            __syncthreads();
            if (threadIdx.x == 0 && it != a.withhold_item) {
                publish_gpu(prog + p3 * np2 + p2, t + 1);
            }
            // moment partials of this octant and group: warp sums in warp order (a tile without
            // fluid keeps the zero partials of its solid points)
            const int tot = tfl ? nr3 * nr2 * width * NM : 0;
            for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
                const int mm = idx % NM;
                const int pi = idx / NM;
                const int i = pi % width;
                const int r = pi / width;
                const int jj = r % nr2;
                const int kk = r / nr2;
                T s = T(0);
                for (int w = 0; w < NW; ++w) s += part[((size_t)(w * MROWS + kk * MR2 + jj) * T1 + i) * NM + mm];
                const int ic = c0 + i;
                const int x = s1n ? n1 - 1 - ic : ic;
                const int y = s2n ? n2 - 1 - (j0 + jj) : (j0 + jj);
                const int z = s3n ? n3 - 1 - (k0 + kk) : (k0 + kk);
                const size_t pid = ((size_t)z * n2 + y) * n1 + x;
                if (mm < 4) P->P[(((size_t)q * G + g) * 4 + mm) * N + pid] = s;
                else if (mm == 4) P->Pt[((size_t)q * G + g) * N + pid] = s;
                else P->Px[(((size_t)q * G + g) * NX + (mm - 5)) * N + pid] = s;
            }
            __syncthreads();
        }
    }
}

// rho'_s of face (y, axis j, side sigma) in FP64 from the octant/group partials of u_j at y
template <typename T>
__device__ __forceinline__ double wall_density3(const Prob3D<T>* P, int y, int j, int sigma, const double* dinv) {
    double num = 0.0;
    const int G = P->ngroups;
    for (int q = 0; q < 8; ++q) {
        if (((q >> j) & 1) != (sigma < 0 ? 1 : 0)) continue;
        for (int g = 0; g < G; ++g) num += (double)P->P[(((size_t)q * G + g) * 4 + 1 + j) * P->N + y];
    }
    return sigma * num * dinv[j];
}

constexpr int kFinPPT3 = 4;   // points per finalize thread in 3D

template <typename T>
__global__ void __launch_bounds__(256) finalize3d_kernel(const FinArgs3D<T> a) {
    using V = typename V4t<T>::type;
    __shared__ double s_red[8];
    __shared__ int s_last;
    const int b = a.blk_prob[blockIdx.x];
    const Prob3D<T>* __restrict__ P = a.prob + b;
    // kFinPPT3 points per thread (threadIdx.x + k 256 of the block's points): the FP64 work of
    // the block sums, a large part of this kernel on GB300's FP64 unit, is shared by four points
    double u1d = 0.0;
#pragma unroll 1
    for (int kq = 0; kq < kFinPPT3; ++kq) {
        const int id = a.blk_start[blockIdx.x] + threadIdx.x + kq * 256;
        if (id < P->N) {
            const uint16_t code = P->code[id];
            // the moment partials are loaded before the code is known (a solid point's partials are
            // the start state's zeros), so both loads overlap
            const size_t N = P->N;
            const int G = P->ngroups;
            T mo[4] = {T(0), T(0), T(0), T(0)};
    #pragma unroll
            for (int q = 0; q < 8; ++q)
    #pragma unroll 2
                for (int g = 0; g < G; ++g)
    #pragma unroll
                    for (int mm = 0; mm < 4; ++mm) mo[mm] += P->P[(((size_t)q * G + g) * 4 + mm) * N + id];
            V s = V4t<T>::make(0, 0, 0, 0), e0 = s, e1 = s;
            if (!(code & kSolidBit)) {
                const T nu = (T)P->nu;
                s = V4t<T>::make(nu * mo[0], T(2) * nu * mo[1] + T(1), T(2) * nu * mo[2], T(2) * nu * mo[3]);
                u1d += (double)mo[1];
                if (P->tau) {
                    // tau = (2/3) e - rho (Eq. 4) from the shifted moments e' = sum W |v|^2 h' and rho':
                    // tau = (2/3) e' - rho' + x1 (1 - (2/3) sum W |v|^2), the same in both forms
                    T e = T(0);
                    for (int q = 0; q < 8; ++q)
                        for (int g = 0; g < G; ++g) e += P->Pt[((size_t)q * G + g) * N + id];
                    const T x1 = (T)((id % P->n1) * P->dx);
                    const T tau = T(2.0 / 3.0) * e - mo[0] + x1 * (T)(1.0 - 2.0 / 3.0 * P->sw2);
                    P->srct[id] = nu * tau;
                    if (P->nx) {
                        // model moments m_a = sum W psi_a h = m'_a - x1 sx_a (heat flux, stress); the
                        // source carries nu xcoef m_a
                        const int nx = P->nx;
                        T xv[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
                        for (int m = 0; m < nx; ++m) {
                            T xs = T(0);
                            for (int q = 0; q < 8; ++q)
                                for (int g = 0; g < G; ++g) xs += P->Px[(((size_t)q * G + g) * nx + m) * N + id];
                            xv[m] = nu * (T)P->xcoef * (xs - x1 * (T)P->sx[m]);
                        }
                        reinterpret_cast<V*>(P->srcx)[2 * (size_t)id] = V4t<T>::make(xv[0], xv[1], xv[2], xv[3]);
                        reinterpret_cast<V*>(P->srcx)[2 * (size_t)id + 1] = V4t<T>::make(xv[4], xv[5], T(0), T(0));
                    }
                }
                T ev[6];
    #pragma unroll
                for (int j = 0; j < 3; ++j) {
    #pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int cs = (code >> (2 * (2 * j + u))) & 3;
                        const int sigma = u ? 1 : -1;
                        double val = 0.0;
                        if (cs == 2) {
                            // Eq. 5: alpha times the diffuse value (the specular part is added per velocity)
                            // (Eq. 5: alpha times the diffuse value, through the alpha-scaled denominators)
                            val = wall_density3(P, id, j, sigma, P->dinvw) + (j == 0 ? sigma * P->dx : 0.0);
                        }
                        // case 1 (only the second upstream point solid) is first order on the fluid
                        // neighbour: no wall term
                        ev[2 * j + u] = (T)val;
                    }
                }
                e0 = V4t<T>::make(ev[0], ev[1], ev[2], ev[3]);
                e1 = V4t<T>::make(ev[4], ev[5], T(0), T(0));
            }
            reinterpret_cast<V*>(P->src)[id] = s;
            reinterpret_cast<V*>(P->E)[2 * (size_t)id] = e0;
            reinterpret_cast<V*>(P->E)[2 * (size_t)id + 1] = e1;
    
        }
    }
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

// Store h' (source form) of a point with x1 coordinate x1 into a ghost or edge array, in the
// array's storage form (T, or the BF16 deviation from the ramp).
template <typename T>
__device__ __forceinline__ void put_h(const Prob3D<T>* P, T* base, size_t i, double hp, double x1) {
    if (P->bf16) reinterpret_cast<__nv_bfloat16*>(base)[i] = __float2bfloat16_rn((float)(hp - x1));
    else base[i] = (T)hp;
}

// Zero-perturbation start in the kernels' source-form variables (h' = x1).  Arrays of per-point values
// are filled point-major within each (octant, group, moment) plane; ghost layers row by row, one warp
// per row of nl velocity slots that all hold the same value (the row's x1), with no per-element index
// division.
template <typename T>
__device__ __forceinline__ void fill_row(const Prob3D<T>* P, T* base, size_t row, size_t nl, int lane, double x1) {
    T* d = base + row * nl;
    if (P->bf16) {
        for (size_t l = lane; l < nl; l += 32) put_h(P, base, row * nl + l, x1, x1);
    } else {
        for (size_t l = lane; l < nl; l += 32) d[l] = (T)x1;
    }
}

template <typename T>
__global__ void init3d_kernel(const Prob3D<T>* P, int NL, const double* qw /*[8][G][4]*/,
                              const double* qwt /*[8][G][4]: sum W |v|^2 (1, v)*/,
                              const double* qwx /*[8][G][nx][4]: sum W psi_a (1, v)*/) {
    const int n1 = P->n1, n2 = P->n2, n3 = P->n3, N = P->N, G = P->ngroups;
    const size_t nl = NL;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    for (int qgm = 0; qgm < 8 * G * 4; ++qgm)
        for (int id = tid; id < N; id += nth) {
            const double x1 = (id % n1) * P->dx;
            P->P[(size_t)qgm * N + id] = (P->code[id] & kSolidBit) ? T(0) : (T)(x1 * qw[qgm]);
        }
    if (P->spec > 0.0)   // face stores of both parities: h' = x1 at the face's fluid point
        for (size_t idx = tid; idx < (size_t)2 * P->nfaces * 4 * nl; idx += nth) {
            const int id = P->faces[(idx / (4 * nl)) % P->nfaces] >> 3;
            P->F[idx] = (T)((id % n1) * P->dx);
        }
    if (P->tau)   // sum W |v|^2 h' of h' = x1
        for (int qg = 0; qg < 8 * G; ++qg)
            for (int id = tid; id < N; id += nth) {
                const double x1 = (id % n1) * P->dx;
                P->Pt[(size_t)qg * N + id] = (P->code[id] & kSolidBit) ? T(0) : (T)(x1 * qwt[qg * 4]);
            }
    if (P->nx)   // model moments sum W psi_a h' of h' = x1
        for (int qgx = 0; qgx < 8 * G * P->nx; ++qgx)
            for (int id = tid; id < N; id += nth) {
                const double x1 = (id % n1) * P->dx;
                P->Px[(size_t)qgx * N + id] = (P->code[id] & kSolidBit) ? T(0) : (T)(x1 * qwx[qgx * 4]);
            }
    // ghost rows: one warp per row of nl slots
    const int lane = threadIdx.x & 31;
    const size_t gw = (size_t)tid >> 5, nw = (size_t)nth >> 5;
    const int ns1 = P->ns1, ns2 = P->ns2, ns3 = P->ns3;
    // x1 ghosts, rows (par, q, slot, k, j, layer): slot s holds the two columns before oriented
    // column slot_col1[s]
    for (size_t row = gw; row < (size_t)2 * 8 * ns1 * n3 * n2 * 2; row += nw) {
        const int layer = (int)(row % 2);
        const int slot = (int)((row / ((size_t)2 * n3 * n2)) % ns1);
        const int q = (int)((row / ((size_t)2 * n3 * n2 * ns1)) % 8);
        const int ico = P->slot_col1[(q & 1) * ns1 + slot] - 1 - layer;
        const int col = (q & 1) ? n1 - 1 - ico : ico;
        fill_row(P, P->gx1, row, nl, lane, col * P->dx);
    }
    // x2 ghosts, rows (par, q, slot, k, i, layer); x3 ghosts, rows (par, q, slot, j, i, layer)
    for (size_t row = gw; row < (size_t)2 * 8 * ns2 * n3 * n1 * 2; row += nw) {
        const int ic = (int)((row / 2) % n1);
        const int q = (int)((row / ((size_t)2 * n3 * n1 * ns2)) % 8);
        const int col = (q & 1) ? n1 - 1 - ic : ic;
        fill_row(P, P->gy, row, nl, lane, col * P->dx);
    }
    for (size_t row = gw; row < (size_t)2 * 8 * ns3 * n2 * n1 * 2; row += nw) {
        const int ic = (int)((row / 2) % n1);
        const int q = (int)((row / ((size_t)2 * n2 * n1 * ns3)) % 8);
        const int col = (q & 1) ? n1 - 1 - ic : ic;
        fill_row(P, P->gz, row, nl, lane, col * P->dx);
    }
}

// Warm start (3D): the state an iteration leaves when it produced h0 = rho0 + 2 u0 . v at every
// fluid point (source form h0' = h0 + x1).  Partials per octant and velocity group through
// qw2[q][g][m][n] = sum W phi_m psi_n with phi = psi = (1, v1, v2, v3); ghost layers read at parity
// `par` hold h0' where the sweep would have captured them (same slot layout as the sweep writes).
template <typename T>
__global__ void warm3d_kernel(const Prob3D<T>* P, int NL, int par, const double* __restrict__ qw2,
                              const double* __restrict__ qwt, const double* __restrict__ qwx,
                              const double* __restrict__ vel,
                              const double* __restrict__ rho0, const double* __restrict__ u0) {
    const int n1 = P->n1, n2 = P->n2, n3 = P->n3, N = P->N, G = P->ngroups;
    const size_t nl = NL;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    // h0' at the oriented point (io, jo, ko) of octant q; x1 receives the point's x1 coordinate
    auto h0 = [&](int q, int io, int jo, int ko, const double* v, double& x1) -> double {
        const int x = (q & 1) ? n1 - 1 - io : io;
        const int y = (q & 2) ? n2 - 1 - jo : jo;
        const int z = (q & 4) ? n3 - 1 - ko : ko;
        const size_t id = ((size_t)z * n2 + y) * n1 + x;
        x1 = x * P->dx;
        if (P->code[id] & kSolidBit) return 0.0;
        return rho0[id] + x1 + 2.0 * (u0[id] * v[0] + u0[N + id] * v[1] + u0[2 * (size_t)N + id] * v[2]);
    };
    for (size_t idx = t0; idx < (size_t)8 * G * 4 * N; idx += stride) {
        const size_t id = idx % N;
        const size_t qgm = idx / N;
        double val = 0.0;
        if (!(P->code[id] & kSolidBit)) {
            const double* c = qw2 + qgm * 4;
            const double r = rho0[id] + (id % n1) * P->dx;
            val = r * c[0] + 2.0 * (u0[id] * c[1] + u0[N + id] * c[2] + u0[2 * (size_t)N + id] * c[3]);
        }
        P->P[idx] = (T)val;
    }
    // face stores (specular wall parts, Eq. 5): h0' at the face's fluid point for the velocity slot
    // of the octant moving into the face (s_j = the face side, the other two axes' bits o)
    if (P->spec > 0.0)
        for (size_t idx = t0; idx < (size_t)P->nfaces * 4 * nl; idx += stride) {
            const int l = idx % nl;
            const int o = (idx / nl) % 4;
            const int f = P->faces[idx / (4 * nl)];
            const int id = f >> 3, j = (f >> 1) & 3, u = f & 1;
            const int qj = (1 - u) << j;
            const int qw = j == 0 ? (qj | (o << 1)) : (j == 1 ? (qj | (o & 1) | ((o & 2) << 1)) : (qj | o));
            double x1;
            const double hv = h0(qw, (qw & 1) ? n1 - 1 - id % n1 : id % n1, (qw & 2) ? n2 - 1 - (id / n1) % n2 : (id / n1) % n2,
                                 (qw & 4) ? n3 - 1 - id / (n1 * n2) : id / (n1 * n2), vel + ((size_t)qw * nl + l) * 3, x1);
            P->F[(size_t)par * P->nfaces * 4 * nl + idx] = (T)hv;
        }
    // temperature term: sum W |v|^2 h0' through qwt[q][g][n] = sum W |v|^2 psi_n, psi = (1, v)
    if (P->tau)
        for (size_t idx = t0; idx < (size_t)8 * G * N; idx += stride) {
            const size_t id = idx % N;
            double val = 0.0;
            if (!(P->code[id] & kSolidBit)) {
                const double* c = qwt + (idx / N) * 4;
                const double r = rho0[id] + (id % n1) * P->dx;
                val = r * c[0] + 2.0 * (u0[id] * c[1] + u0[N + id] * c[2] + u0[2 * (size_t)N + id] * c[3]);
            }
            P->Pt[idx] = (T)val;
        }
    // model moments: sum W psi_a h0' through qwx[q][g][a][n]
    if (P->nx)
        for (size_t idx = t0; idx < (size_t)8 * G * P->nx * N; idx += stride) {
            const size_t id = idx % N;
            double val = 0.0;
            if (!(P->code[id] & kSolidBit)) {
                const double* c = qwx + (idx / N) * 4;
                const double r = rho0[id] + (id % n1) * P->dx;
                val = r * c[0] + 2.0 * (u0[id] * c[1] + u0[N + id] * c[2] + u0[2 * (size_t)N + id] * c[3]);
            }
            P->Px[idx] = (T)val;
        }
    const int ns1 = P->ns1, ns2 = P->ns2, ns3 = P->ns3;
    // x1 ghosts: (q, slot s, oriented row (k, j), layer) holds h at oriented column
    // slot_col1[s] - 1 - layer (slot 0: n1 - 1 - layer, the periodic wrap)
    for (size_t idx = t0; idx < (size_t)8 * ns1 * n3 * n2 * 2 * nl; idx += stride) {
        const int l = idx % nl;
        const int layer = (idx / nl) % 2;
        const int row = (idx / (nl * 2)) % ((size_t)n3 * n2);
        const int slot = (idx / (nl * 2 * n3 * n2)) % ns1;
        const int q = idx / (nl * 2 * n3 * n2 * ns1);
        const int ico = P->slot_col1[(q & 1) * ns1 + slot] - 1 - layer;
        double x1;
        const double hv = h0(q, ico, row % n2, row / n2, vel + ((size_t)q * nl + l) * 3, x1);
        put_h(P, P->gx1, (size_t)par * 8 * ns1 * n3 * n2 * 2 * nl + idx, hv, x1);
    }
    // x2 ghosts: octant q writes its oriented rows slot_row2[s] - 1 - layer into slot s of the
    // octant that reads them (slot 0 at the domain face: periodic same octant, specular s2 flipped)
    for (size_t idx = t0; idx < (size_t)8 * ns2 * n3 * n1 * 2 * nl; idx += stride) {
        const int l = idx % nl;
        const int layer = (idx / nl) % 2;
        const int row = (idx / (nl * 2)) % ((size_t)n3 * n1);
        const int slot = (idx / (nl * 2 * n3 * n1)) % ns2;
        const int q = idx / (nl * 2 * n3 * n1 * ns2);
        const int qy = (slot > 0 || P->lateral == 1) ? q : (q ^ 2);
        const int jo = P->slot_row2[((q >> 1) & 1) * ns2 + slot] - 1 - layer;
        double x1;
        const double hv = h0(q, row % n1, jo, row / n1, vel + ((size_t)q * nl + l) * 3, x1);
        put_h(P, P->gy, (((((size_t)par * 8 + qy) * ns2 + slot) * n3 * n1 + row) * 2 + layer) * nl + l, hv, x1);
    }
    // x3 ghosts: the same with oriented planes slot_row3[s] - 1 - layer
    for (size_t idx = t0; idx < (size_t)8 * ns3 * n2 * n1 * 2 * nl; idx += stride) {
        const int l = idx % nl;
        const int layer = (idx / nl) % 2;
        const int row = (idx / (nl * 2)) % ((size_t)n2 * n1);
        const int slot = (idx / (nl * 2 * n2 * n1)) % ns3;
        const int q = idx / (nl * 2 * n2 * n1 * ns3);
        const int qz = (slot > 0 || P->lateral == 1) ? q : (q ^ 4);
        const int ko = P->slot_row3[((q >> 2) & 1) * ns3 + slot] - 1 - layer;
        double x1;
        const double hv = h0(q, row % n1, row / n1, ko, vel + ((size_t)q * nl + l) * 3, x1);
        put_h(P, P->gz, (((((size_t)par * 8 + qz) * ns3 + slot) * n2 * n1 + row) * 2 + layer) * nl + l, hv, x1);
    }
}

template <typename T>
__global__ void moments3d_kernel(const Prob3D<T>* P, double* rho, double* u) {
    const int N = P->N, G = P->ngroups;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        if (P->code[id] & kSolidBit) {
            rho[id] = 0.0;
            for (int j = 0; j < 3; ++j) u[(size_t)j * N + id] = 0.0;
            continue;
        }
        T mo[4] = {T(0), T(0), T(0), T(0)};
        for (int q = 0; q < 8; ++q)
            for (int g = 0; g < G; ++g)
                for (int mm = 0; mm < 4; ++mm) mo[mm] += P->P[(((size_t)q * G + g) * 4 + mm) * N + id];
        rho[id] = (double)mo[0] - (id % P->n1) * P->dx;
        for (int j = 0; j < 3; ++j) u[(size_t)j * N + id] = (double)mo[1 + j];
    }
}

// Temperature of Eq. 4 per point (FP64 sums of the partials): tau = (2/3) e' - rho' +
// x1 (1 - (2/3) sum W |v|^2), the paper's tau (solid points 0).
template <typename T>
__global__ void temperature3d_kernel(const Prob3D<T>* P, double* tau) {
    const int N = P->N, G = P->ngroups;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        if (P->code[id] & kSolidBit) {
            tau[id] = 0.0;
            continue;
        }
        double e = 0.0, r = 0.0;
        for (int q = 0; q < 8; ++q)
            for (int g = 0; g < G; ++g) {
                e += (double)P->Pt[((size_t)q * G + g) * N + id];
                r += (double)P->P[(((size_t)q * G + g) * 4) * N + id];
            }
        const double x1 = (id % P->n1) * P->dx;
        tau[id] = 2.0 / 3.0 * e - r + x1 * (1.0 - 2.0 / 3.0 * P->sw2);
    }
}

// Model moments per point (FP64 sums of the partials): m_a = m'_a - x1 sx_a (solid points 0),
// [nx][N]: the heat flux of the Shakhov model, the traceless stress of the ES-BGK model.
template <typename T>
__global__ void modelmoments3d_kernel(const Prob3D<T>* P, double* out) {
    const int N = P->N, G = P->ngroups, nx = P->nx;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const bool solid = (P->code[id] & kSolidBit) != 0;
        const double x1 = (id % P->n1) * P->dx;
        for (int m = 0; m < nx; ++m) {
            double xs = 0.0;
            if (!solid)
                for (int q = 0; q < 8; ++q)
                    for (int g = 0; g < G; ++g) xs += (double)P->Px[(((size_t)q * G + g) * nx + m) * N + id];
            out[(size_t)m * N + id] = solid ? 0.0 : xs - x1 * P->sx[m];
        }
    }
}

template <typename T>
__global__ void wall3d_kernel(const Prob3D<T>* P, double* out) {
    const int N = P->N;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const uint16_t code = P->code[id];
        for (int j = 0; j < 3; ++j)
            for (int u = 0; u < 2; ++u) {
                double v = 0.0;
                if (!(code & kSolidBit) && ((code >> (2 * (2 * j + u))) & 3) == 2)
                    v = wall_density3(P, id, j, u ? 1 : -1, P->dinv) - (id % P->n1) * P->dx;
                out[(size_t)(2 * j + u) * N + id] = v;
            }
    }
}

template <typename T>
size_t sweep3d_smem(int T1, int NW, int R2, int R3, int tau, int spec, int nx) {
    const size_t rows = (size_t)R2 * R3;
    const size_t rw = spec ? 24 : (nx == 3 ? 20 : (nx == 6 ? 24 : kRec3));
    return sizeof(T) * (rows * T1 * rw + (size_t)NW * rows * T1 * (nx ? 5 + nx : (tau ? 5 : 4)) +
                        (size_t)NW * rows * 2 * 32 + (size_t)NW * R2 * 2 * T1 * 32 + (size_t)NW * 8 * 32);
}

template <typename T, int T1, bool SUB, bool TAU, bool SPEC, int NX = 0>
static cudaError_t occ3(int NW, int R2, int R3, int* blocks_per_sm) {
    const size_t smem = sweep3d_smem<T>(T1, NW, R2, R3, TAU, SPEC, NX);
    auto kern = sweep3d_kernel<T, T1, false, SUB, TAU, SPEC, NX>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, NW * 32, smem);
}

template <typename T, int T1, bool SUB, bool TAU>
static cudaError_t occ3_s(int NW, int R2, int R3, int spec, int* bps) {
    return spec ? occ3<T, T1, SUB, TAU, true>(NW, R2, R3, bps) : occ3<T, T1, SUB, TAU, false>(NW, R2, R3, bps);
}

template <typename T, int T1>
static cudaError_t occ3_t(int NW, int R2, int R3, int sub, int tau, int spec, int* bps) {
    if (sub) return tau ? occ3_s<T, T1, true, true>(NW, R2, R3, spec, bps) : occ3_s<T, T1, true, false>(NW, R2, R3, spec, bps);
    return tau ? occ3_s<T, T1, false, true>(NW, R2, R3, spec, bps) : occ3_s<T, T1, false, false>(NW, R2, R3, spec, bps);
}

// model-moment kernels (Shakhov nx = 3, ES-BGK nx = 6): with tau, without sub and spec
template <typename T>
static cudaError_t occ3_x(int T1, int NW, int R2, int R3, int nx, int* bps) {
    if (T1 == 4) return nx == 3 ? occ3<T, 4, false, true, false, 3>(NW, R2, R3, bps) : occ3<T, 4, false, true, false, 6>(NW, R2, R3, bps);
    if (T1 == 8) return nx == 3 ? occ3<T, 8, false, true, false, 3>(NW, R2, R3, bps) : occ3<T, 8, false, true, false, 6>(NW, R2, R3, bps);
    return cudaErrorInvalidValue;
}

// The scalar kernel serves the FP64 path and the Shakhov and ES-BGK models in both precisions
// (FP32 and its BF16-storage ablation otherwise use the packed kernel of sweep3d_f32x2.cu); its
// BF16 flag stays false.  sub: lagged-halo subdomains (table-driven pencils and tiles); tau: the
// temperature term; spec: specular wall parts; nx: model moments (3 or 6; with tau, without sub
// and spec).
template <typename T>
cudaError_t sweep3d_occupancy(int T1, int NW, int R2, int R3, int bf16, int sub, int tau, int spec, int nx,
                              int* blocks_per_sm) {
    if (bf16) return cudaErrorInvalidValue;
    if (nx) {
        if (sub || !tau || spec || (nx != 3 && nx != 6)) return cudaErrorInvalidValue;
        return occ3_x<T>(T1, NW, R2, R3, nx, blocks_per_sm);
    }
    if (T1 == 4) return occ3_t<T, 4>(NW, R2, R3, sub, tau, spec, blocks_per_sm);
    if (T1 == 8) return occ3_t<T, 8>(NW, R2, R3, sub, tau, spec, blocks_per_sm);
    return cudaErrorInvalidValue;
}

template <typename T, int T1, bool SUB, bool TAU, bool SPEC, int NX = 0>
static cudaError_t launch3(const SweepArgs3D<T>& a, int grid, int NW, cudaStream_t st) {
    const size_t smem = sweep3d_smem<T>(T1, NW, a.maxR2, a.maxR3, TAU, SPEC, NX);
    auto kern = sweep3d_kernel<T, T1, false, SUB, TAU, SPEC, NX>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, NW * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int T1, bool SUB, bool TAU>
static cudaError_t launch3_s(const SweepArgs3D<T>& a, int grid, int NW, cudaStream_t st) {
    return a.spec ? launch3<T, T1, SUB, TAU, true>(a, grid, NW, st) : launch3<T, T1, SUB, TAU, false>(a, grid, NW, st);
}

template <typename T, int T1>
static cudaError_t launch3_t(const SweepArgs3D<T>& a, int grid, int NW, cudaStream_t st) {
    if (a.sub) return a.tau ? launch3_s<T, T1, true, true>(a, grid, NW, st) : launch3_s<T, T1, true, false>(a, grid, NW, st);
    return a.tau ? launch3_s<T, T1, false, true>(a, grid, NW, st) : launch3_s<T, T1, false, false>(a, grid, NW, st);
}

template <typename T>
static cudaError_t launch3_x(const SweepArgs3D<T>& a, int grid, int NW, cudaStream_t st) {
    if (a.sub || !a.tau || a.spec) return cudaErrorInvalidValue;
    if (a.T1 == 4 && a.nx == 3) return launch3<T, 4, false, true, false, 3>(a, grid, NW, st);
    if (a.T1 == 4 && a.nx == 6) return launch3<T, 4, false, true, false, 6>(a, grid, NW, st);
    if (a.T1 == 8 && a.nx == 3) return launch3<T, 8, false, true, false, 3>(a, grid, NW, st);
    if (a.T1 == 8 && a.nx == 6) return launch3<T, 8, false, true, false, 6>(a, grid, NW, st);
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_sweep3d(const SweepArgs3D<T>& a, int grid, int NW, cudaStream_t st) {
    if (a.bf16) return cudaErrorInvalidValue;
    if (a.nx) return launch3_x<T>(a, grid, NW, st);
    if (a.T1 == 4) return launch3_t<T, 4>(a, grid, NW, st);
    if (a.T1 == 8) return launch3_t<T, 8>(a, grid, NW, st);
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_finalize3d(const FinArgs3D<T>& a, int nblocks, cudaStream_t st) {
    finalize3d_kernel<T><<<nblocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init3d(const Prob3D<T>* p, int NL, const double* qw, const double* qwt, const double* qwx,
                          cudaStream_t st) {
    init3d_kernel<T><<<608, 256, 0, st>>>(p, NL, qw, qwt, qwx);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_warm3d(const Prob3D<T>* p, int NL, int par, const double* qw2, const double* qwt,
                          const double* qwx, const double* vel, const double* rho0, const double* u0,
                          cudaStream_t st) {
    warm3d_kernel<T><<<608, 256, 0, st>>>(p, NL, par, qw2, qwt, qwx, vel, rho0, u0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_moments3d(const Prob3D<T>* p, double* rho, double* u, cudaStream_t st) {
    moments3d_kernel<T><<<608, 256, 0, st>>>(p, rho, u);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_temperature3d(const Prob3D<T>* p, double* tau, cudaStream_t st) {
    temperature3d_kernel<T><<<608, 256, 0, st>>>(p, tau);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_modelmoments3d(const Prob3D<T>* p, double* out, cudaStream_t st) {
    modelmoments3d_kernel<T><<<608, 256, 0, st>>>(p, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_wall3d(const Prob3D<T>* p, double* out, cudaStream_t st) {
    wall3d_kernel<T><<<608, 256, 0, st>>>(p, out);
    return cudaGetLastError();
}

template size_t sweep3d_smem<double>(int, int, int, int, int, int, int);
template size_t sweep3d_smem<float>(int, int, int, int, int, int, int);
template cudaError_t sweep3d_occupancy<double>(int, int, int, int, int, int, int, int, int, int*);
template cudaError_t launch_sweep3d<double>(const SweepArgs3D<double>&, int, int, cudaStream_t);
// FP32 with the Shakhov or ES-BGK model (the scalar kernel's only FP32 use)
template <>
cudaError_t sweep3d_occupancy<float>(int T1, int NW, int R2, int R3, int bf16, int sub, int tau, int spec, int nx,
                                     int* blocks_per_sm) {
    if (bf16 || (nx != 3 && nx != 6) || sub || !tau || spec) return cudaErrorInvalidValue;
    return occ3_x<float>(T1, NW, R2, R3, nx, blocks_per_sm);
}
template <>
cudaError_t launch_sweep3d<float>(const SweepArgs3D<float>& a, int grid, int NW, cudaStream_t st) {
    if (a.bf16 || !a.nx) return cudaErrorInvalidValue;
    return launch3_x<float>(a, grid, NW, st);
}

#define DVM_INSTANTIATE3(T)                                                                                  \
    template cudaError_t launch_finalize3d<T>(const FinArgs3D<T>&, int, cudaStream_t);                      \
    template cudaError_t launch_init3d<T>(const Prob3D<T>*, int, const double*, const double*, const double*, \
                                          cudaStream_t);                                                     \
    template cudaError_t launch_warm3d<T>(const Prob3D<T>*, int, int, const double*, const double*,          \
                                          const double*, const double*, const double*, const double*,        \
                                          cudaStream_t);                                                     \
    template cudaError_t launch_modelmoments3d<T>(const Prob3D<T>*, double*, cudaStream_t);                  \
    template cudaError_t launch_moments3d<T>(const Prob3D<T>*, double*, double*, cudaStream_t);              \
    template cudaError_t launch_temperature3d<T>(const Prob3D<T>*, double*, cudaStream_t);                   \
    template cudaError_t launch_wall3d<T>(const Prob3D<T>*, double*, cudaStream_t);

DVM_INSTANTIATE3(float)
DVM_INSTANTIATE3(double)

}  // namespace dvm
