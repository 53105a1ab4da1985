// dvm_api.cpp -- host side of the C ABI declared in include/dvm.h.
//
// Responsibilities: argument validation, per-problem preprocessing (the per-point stencil cases
// that the paper fixes in preprocessing "to avoid IF-THEN at every iteration", Sec. 2.3; the
// grouping of the discrete velocities into quadrants whose lanes line up under reflection; the
// per-lane reciprocal denominators of the point update), device memory layout, and the iteration
// driver (sweep + finalize per iteration, permeability and Err every check interval, Eq. 15).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/dvm.h"
#include "dvm_internal.h"

namespace dvm {
bool half_range_gh(int m, double* c, double* a);
template <typename T> size_t sweep2d_smem(int T1, int NW, int max_rows, int spec);
template <typename T> cudaError_t launch_sweep2d(const SweepArgs2D<T>&, int T1, int xs, int grid, int NW, cudaStream_t);
template <typename T> cudaError_t sweep2d_occupancy(int T1, int xs, int spec, int NW, int max_rows, int* blocks_per_sm);
template <typename T> cudaError_t launch_finalize2d(const FinArgs2D<T>&, int nblocks, cudaStream_t);
template <typename T> cudaError_t launch_init2d(const Prob2D<T>*, int NL, const double* qw, cudaStream_t);
template <typename T> cudaError_t launch_moments2d(const Prob2D<T>*, double* rho, double* u, cudaStream_t);
template <typename T> cudaError_t launch_wall2d(const Prob2D<T>*, double* out, cudaStream_t);
template <typename T>
cudaError_t launch_warm2d(const Prob2D<T>*, int NL, int par, const double* qw2, const double* vel, const double* rho0,
                          const double* u0, cudaStream_t);
cudaError_t launch_sweep2d_f32x2(const SweepArgs2D<float>&, int T1, int xs, int grid, int NW, cudaStream_t);
cudaError_t sweep2d_f32x2_occupancy(int T1, int xs, int spec, int NW, int max_rows, int* blocks_per_sm);
int sweep2d_f32x2_max_rows(int T1, int NW);
int sweep2d_f32x2_velocities_per_lane();
template <typename T> size_t sweep3d_smem(int T1, int NW, int R2, int R3, int tau, int spec, int shk);
size_t sweep3d_f32x2_smem(int T1, int NW, int R2, int R3, int tau, int spec);
int sweep3d_f32x2_velocities_per_lane();
cudaError_t launch_sweep3d_f32x2(const SweepArgs3D<float>&, int grid, int NW, cudaStream_t);
cudaError_t sweep3d_f32x2_occupancy(int T1, int NW, int R2, int R3, int bf16, int sub, int tau, int spec, int* blocks_per_sm);
template <typename T>
cudaError_t sweep3d_occupancy(int T1, int NW, int R2, int R3, int bf16, int sub, int tau, int spec, int shk,
                              int* blocks_per_sm);
template <typename T> cudaError_t launch_sweep3d(const SweepArgs3D<T>&, int grid, int NW, cudaStream_t);
template <typename T> cudaError_t launch_finalize3d(const FinArgs3D<T>&, int nblocks, cudaStream_t);
template <typename T>
cudaError_t launch_init3d(const Prob3D<T>*, int NL, const double* qw, const double* qwt, const double* qwx, cudaStream_t);
template <typename T> cudaError_t launch_modelmoments3d(const Prob3D<T>*, double* out, cudaStream_t);
template <typename T> cudaError_t launch_moments3d(const Prob3D<T>*, double* rho, double* u, cudaStream_t);
template <typename T> cudaError_t launch_temperature3d(const Prob3D<T>*, double* tau, cudaStream_t);
template <typename T> cudaError_t launch_wall3d(const Prob3D<T>*, double* out, cudaStream_t);
template <typename T>
cudaError_t launch_warm3d(const Prob3D<T>*, int NL, int par, const double* qw2, const double* qwt, const double* qwx,
                          const double* vel, const double* rho0, const double* u0, cudaStream_t);
}  // namespace dvm

using namespace dvm;

namespace {

constexpr int kFinBlock2 = 1024;  // points per finalize block in 2D (256 threads x 4 points)
constexpr int kFinBlock3 = 1024;  // points per finalize block in 3D (256 threads x 4 points)

struct Buf {
    void* p;
    size_t bytes;
};

struct HostProb {
    int n[3];
    int N;
    double kn, nu, dx;
    int nbands;
    std::vector<int> qbands;     // 2D: bands of every quadrant
    std::vector<uint16_t> code;
};

}  // namespace

struct dvm_ctx {
    std::string err;
    dvm_options opt;
    cudaStream_t stream = nullptr;
    int dims = 2, nprob = 0, nv = 0, nvq = 0, NQ = 4, NL = 32, NW = 1;
    int prec = DVM_FP64;             // arithmetic precision (BF16 storage computes in FP32)
    bool bf16 = false;               // 3D ghosts and pencil edges stored as BF16
    bool xsub = false;               // 2D x1 subdomains (tile tables, lagged x1 halos)
    bool sub3 = false;               // 3D lagged-halo subdomains (pencil and tile tables)
    bool tau3 = false;               // 3D temperature term of Eq. 2
    int nx3 = 0;                     // 3D model moments: 3 Shakhov, 6 ES-BGK (scalar sweep kernel)
    bool packed3 = false;            // 3D FP32 sweep on the packed kernel (FP32 without Shakhov)
    bool spec2 = false;              // Maxwell walls with alpha < 1 (Eq. 5)
    double* qwt_dev = nullptr;       // 3D: [octant][group][4] sums of W |v|^2 (1, v)
    double* qwx_dev = nullptr;       // 3D model moments: [octant][group][nx][4] sums of W psi_a (1, v)
    int T1 = 8, rows = 8, max_rows = 8;
    std::vector<HostProb> hp;
    std::vector<Buf> bufs;
    // device objects
    void* probs_dev = nullptr;       // Prob2D<T>[nprob]
    std::vector<char> probs_host;    // host copy of the Prob2D array
    SweepItem* items_dev = nullptr;
    int nitems = 0;
    int* counters_dev = nullptr;     // [ticket][prog flags...]
    size_t counters_bytes = 0;
    int* status_dev = nullptr;
    int* blk_prob_dev = nullptr;
    int* blk_start_dev = nullptr;
    int fin_blocks = 0;
    double* qw_dev = nullptr;        // [nprob][4][3]
    double* qw2_dev = nullptr;       // warm start: [octant][group][d+1][d+1] sums of W phi_m psi_n
    double* vel_dev = nullptr;       // warm start: [octant][NL][dims] velocity of every lane (FP64)
    double* scratch_dev = nullptr;   // readout scratch (max N * 4 doubles)
    size_t scratch_bytes = 0;
    // pinned host mirrors
    double* kval_host = nullptr;     // [nprob][3]
    int* status_host = nullptr;
    // iteration state
    long long iters = 0;
    std::vector<double> k_check;     // k at the last check (or at the start state), per problem
    std::vector<long long> it_check; // iteration count of that k, per problem
    double last_err = HUGE_VAL;
    int sweep_grid = 1;
    long long timeout_ns = kDefaultTimeoutNs;
    int withhold_item = -1;
    std::vector<int> prog_offset;    // per problem, offset of its progress flags in counters
    std::vector<double*> kval_dev;   // per problem, device address of (k, G_p, sum u1)
    int GL = 32, G = 1;              // 3D: lanes per velocity group, groups per octant
    int R2 = 4, R3 = 4;              // 3D pencil rows
    // measurement support
    bool profile = false;
    std::vector<cudaEvent_t> ev_pool;      // events owned by the context
    std::vector<cudaEvent_t> ev_marks;     // [3 per profiled iteration] before sweep, after sweep, after finalize
    long long h2d_bytes = 0, d2h_bytes = 0;
    // CUDA graphs of runs of iterations, keyed by run length, starting ghost parity and whether
    // kernel timing was on at capture (then the graph records its own events, 3 per iteration)
    struct Graph {
        int n, parity;
        bool prof;
        cudaGraphExec_t exec;
        std::vector<cudaEvent_t> marks;
    };
    std::vector<Graph> graphs;
    bool capturing = false;                  // inside the stream capture of a profiled graph
    std::vector<cudaEvent_t> capture_marks;  // events recorded into the graph being captured
    const std::vector<cudaEvent_t>* graph_pending = nullptr;   // marks of a replay not yet read
    double acc_sweep_ms = 0.0, acc_fin_ms = 0.0;                 // timings read from graph replays
    int64_t acc_sweep_n = 0, acc_fin_n = 0;
};

namespace {

thread_local std::string g_create_err;   // message of the last failed creation on this thread

dvm_status fail(dvm_ctx* c, dvm_status s, const std::string& msg) {
    if (c) c->err = msg;
    g_create_err = msg;
    return s;
}

dvm_status cuda_fail(dvm_ctx* c, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(c, DVM_ENOMEM, m);
    return fail(c, DVM_ECUDA, m);
}

void* dev_alloc(dvm_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (c->opt.alloc) {
        p = c->opt.alloc(bytes, c->opt.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->bufs.push_back({p, bytes});
    return p;
}

void free_all(dvm_ctx* c) {
    for (auto& b : c->bufs) {
        if (c->opt.alloc) {
            if (c->opt.free) c->opt.free(b.p, b.bytes, c->opt.alloc_user);
        } else {
            cudaFree(b.p);
        }
    }
    c->bufs.clear();
    if (c->kval_host) cudaFreeHost(c->kval_host);
    if (c->status_host) cudaFreeHost(c->status_host);
    c->kval_host = nullptr;
    c->status_host = nullptr;
}

// periodic along x1 always; lateral axes periodic or mirrored (specular, Eq. 8)
int map_coord(int l, int n, bool periodic) {
    if (l >= 0 && l < n) return l;
    if (periodic) return ((l % n) + n) % n;
    return l < 0 ? -1 - l : 2 * n - 1 - l;
}

// Stencil cases (Eq. 9 with the first-order switch of Sec. 3.1: first order when either upstream
// point of the second-order stencil is solid) of every fluid point.
void classify(HostProb& P, int dims, const uint8_t* solid, int lateral, int order) {
    const int n1 = P.n[0], n2 = P.n[1], n3 = dims == 3 ? P.n[2] : 1;
    P.code.assign(P.N, 0);
    for (int z = 0; z < n3; ++z)
        for (int y = 0; y < n2; ++y)
            for (int x = 0; x < n1; ++x) {
                const int id = (z * n2 + y) * n1 + x;
                if (solid[id]) {
                    P.code[id] = kSolidBit;
                    continue;
                }
                uint16_t code = 0;
                const int c[3] = {x, y, z};
                for (int j = 0; j < dims; ++j)
                    for (int u = 0; u < 2; ++u) {
                        const int sigma = u ? 1 : -1;       // direction of the upstream points
                        const bool per = (j == 0) || lateral == DVM_LATERAL_PERIODIC;
                        int c1[3] = {c[0], c[1], c[2]}, c2[3] = {c[0], c[1], c[2]};
                        c1[j] = map_coord(c[j] + sigma, P.n[j], per);
                        c2[j] = map_coord(c[j] + 2 * sigma, P.n[j], per);
                        const bool s1 = solid[(c1[2] * n2 + c1[1]) * n1 + c1[0]] != 0;
                        const bool s2 = solid[(c2[2] * n2 + c2[1]) * n1 + c2[0]] != 0;
                        int cs = 0;
                        if (s1) cs = 2;
                        else if (order == 2 && s2) cs = 1;
                        code |= (uint16_t)(cs << (2 * (2 * j + u)));
                    }
                P.code[id] = code;
            }
}

template <typename T>
dvm_status build_2d(dvm_ctx* c, const dvm_geometry* geoms, const dvm_velocity_grid* grid) {
    const int NQ = 4;
    // ---- velocity groups: quadrant q (bit j set when v_j < 0), lanes ordered by (|v1|, |v2|)
    std::vector<std::vector<int>> group(NQ);
    for (int k = 0; k < grid->nv; ++k) {
        const double* v = grid->v + 2 * k;
        group[(v[0] < 0 ? 1 : 0) | (v[1] < 0 ? 2 : 0)].push_back(k);
    }
    auto key_less = [&](int a, int b) {
        const double* va = grid->v + 2 * a;
        const double* vb = grid->v + 2 * b;
        if (std::fabs(va[0]) != std::fabs(vb[0])) return std::fabs(va[0]) < std::fabs(vb[0]);
        return std::fabs(va[1]) < std::fabs(vb[1]);
    };
    for (auto& g : group) std::sort(g.begin(), g.end(), key_less);
    const int nvq = (int)group[0].size();
    for (int q = 1; q < NQ; ++q)
        if ((int)group[q].size() != nvq) return fail(c, DVM_EINVAL, "velocity grid is not symmetric under sign changes");
    for (int m = 0; m < nvq; ++m) {
        const double* v0 = grid->v + 2 * group[0][m];
        for (int q = 1; q < NQ; ++q) {
            const double* vq = grid->v + 2 * group[q][m];
            if (std::fabs(vq[0]) != std::fabs(v0[0]) || std::fabs(vq[1]) != std::fabs(v0[1]) ||
                grid->w[group[q][m]] != grid->w[group[0][m]])
                return fail(c, DVM_EINVAL, "velocity grid is not symmetric under sign changes");
        }
    }
    c->nvq = nvq;
    // FP32 lanes carry two velocities (packed f32x2 arithmetic), FP64 lanes one
    const int vpl = (c->prec == DVM_FP32) ? sweep2d_f32x2_velocities_per_lane() : 1;
    c->NW = (nvq + 32 * vpl - 1) / (32 * vpl);
    c->NL = 32 * vpl * c->NW;
    const int NL = c->NL;
    if (c->NW > 16) return fail(c, DVM_EINVAL, "too many velocities per quadrant");
    // ---- tiles
    c->T1 = c->opt.tile_x1 ? c->opt.tile_x1 : 8;
    if (c->prec == DVM_FP32) {               // the packed FP32 kernel: 4-, 8- and 16-column tiles
        if (c->T1 != 4 && c->T1 != 8 && c->T1 != 16) return fail(c, DVM_EINVAL, "tile_x1 must be 4, 8 or 16 for FP32");
    } else if (c->T1 != 8 && c->T1 != 16) {
        return fail(c, DVM_EINVAL, "tile_x1 must be 8 or 16 for FP64");
    }
    int rows = c->opt.band_rows ? c->opt.band_rows : 8;
    if (rows < 1) return fail(c, DVM_EINVAL, "band_rows must be positive");
    if (c->prec == DVM_FP32) rows = std::min(rows, sweep2d_f32x2_max_rows(c->T1, c->NW));
    c->rows = rows;
    int max_rows = 1;
    for (int b = 0; b < c->nprob; ++b) max_rows = std::max(max_rows, std::min(rows, c->hp[b].n[1]));
    c->max_rows = max_rows;
    // ---- wall denominators (Eq. 6) and quadrant weight sums
    double dwall[2] = {0, 0};
    for (int k = 0; k < grid->nv; ++k)
        for (int j = 0; j < 2; ++j)
            if (grid->v[2 * k + j] > 0) dwall[j] += grid->w[k] * grid->v[2 * k + j];
    const double dinv[2] = {1.0 / dwall[0], 1.0 / dwall[1]};
    std::vector<double> qw((size_t)c->nprob * NQ * 3, 0.0);
    for (int b = 0; b < c->nprob; ++b)
        for (int q = 0; q < NQ; ++q)
            for (int k : group[q]) {
                qw[((size_t)b * NQ + q) * 3 + 0] += grid->w[k];
                qw[((size_t)b * NQ + q) * 3 + 1] += grid->w[k] * grid->v[2 * k];
                qw[((size_t)b * NQ + q) * 3 + 2] += grid->w[k] * grid->v[2 * k + 1];
            }
    // ---- warm-start tables: lane velocities and quadrant sums of W phi_m psi_n, phi = psi = (1, v)
    std::vector<double> qw2((size_t)NQ * 3 * 3, 0.0), vel((size_t)NQ * NL * 2, 0.0);
    for (int q = 0; q < NQ; ++q)
        for (int l = 0; l < nvq; ++l) {
            const int k = group[q][l];
            const double ph[3] = {1.0, grid->v[2 * k], grid->v[2 * k + 1]};
            vel[((size_t)q * NL + l) * 2 + 0] = ph[1];
            vel[((size_t)q * NL + l) * 2 + 1] = ph[2];
            for (int m = 0; m < 3; ++m)
                for (int n = 0; n < 3; ++n) qw2[((size_t)q * 3 + m) * 3 + n] += grid->w[k] * ph[m] * ph[n];
        }
    c->qw2_dev = (double*)dev_alloc(c, qw2.size() * sizeof(double));
    c->vel_dev = (double*)dev_alloc(c, vel.size() * sizeof(double));
    if (!c->qw2_dev || !c->vel_dev) return fail(c, DVM_ENOMEM, "device allocation failed");
    {
        cudaError_t e;
        if ((e = cudaMemcpyAsync(c->qw2_dev, qw2.data(), qw2.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream)) ||
            (e = cudaMemcpyAsync(c->vel_dev, vel.data(), vel.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream)) ||
            (e = cudaStreamSynchronize(c->stream)))
            return cuda_fail(c, e, "upload warm-start tables");
        c->h2d_bytes += (qw2.size() + vel.size()) * sizeof(double);
    }
    // ---- per problem device buffers
    std::vector<Prob2D<T>> probs(c->nprob);
    std::vector<SweepItem> items;
    std::vector<int> blk_prob, blk_start;
    int prog_total = 0;
    c->prog_offset.assign(c->nprob, 0);
    for (int b = 0; b < c->nprob; ++b) {
        HostProb& H = c->hp[b];
        Prob2D<T>& P = probs[b];
        std::memset(&P, 0, sizeof(P));
        P.n1 = H.n[0];
        P.n2 = H.n[1];
        P.N = H.N;
        P.rows = std::min(rows, P.n2);
        // ---- bands per quadrant in oriented rows; with c2 x2 subdomains (lagged-halo
        // decomposition, Sec. 3.2) no band straddles a subdomain boundary
        const int c2 = std::max(1, c->opt.subdomains[1]);
        std::vector<int> Y(c2 + 1);
        for (int s = 0; s <= c2; ++s) Y[s] = (s * P.n2 + c2 - 1) / c2;    // subdomain s: [Y_s, Y_s+1)
        std::vector<std::vector<int4>> qb(NQ);
        std::vector<int> slot_row((size_t)NQ * c2);
        for (int q = 0; q < NQ; ++q) {
            const bool s2neg = (q >> 1) & 1;
            for (int sp = 0; sp < c2; ++sp) {            // oriented subdomain order
                const int lo = s2neg ? P.n2 - Y[c2 - sp] : Y[sp];
                const int hi = s2neg ? P.n2 - Y[c2 - 1 - sp] : Y[sp + 1];
                slot_row[(size_t)q * c2 + sp] = sp == 0 ? P.n2 : lo;
                // live edges use ring slots 2 sp + (local band & 1): two suffice, since band j + 2
                // of a subdomain reaches tile t only after band j + 1 consumed band j's edge of
                // tile t; every subdomain has its own pair because its first band does not wait
                int j = 0;
                for (int r0 = lo; r0 < hi; r0 += P.rows, ++j) {
                    const int nr = std::min(P.rows, hi - r0);
                    const int below = r0 == lo ? sp : -1 - (2 * sp + ((j - 1) & 1));
                    const int above = r0 + nr == hi ? (sp + 1) % c2 : -1 - (2 * sp + (j & 1));
                    qb[q].push_back(make_int4(r0, nr, below, above));
                }
            }
        }
        P.nbands = 0;
        for (int q = 0; q < NQ; ++q) P.nbands = std::max(P.nbands, (int)qb[q].size());
        P.nslots = c2;
        H.nbands = P.nbands;
        H.qbands.assign(NQ, 0);
        std::vector<int4> btab((size_t)NQ * P.nbands, make_int4(0, 0, -1, -1));
        for (int q = 0; q < NQ; ++q) {
            H.qbands[q] = (int)qb[q].size();
            for (size_t k = 0; k < qb[q].size(); ++k) btab[(size_t)q * P.nbands + k] = qb[q][k];
        }
        int4* bands_dev = (int4*)dev_alloc(c, btab.size() * sizeof(int4));
        int* slot_dev = (int*)dev_alloc(c, slot_row.size() * sizeof(int));
        if (!bands_dev || !slot_dev) return fail(c, DVM_ENOMEM, "device allocation failed");
        {
            cudaError_t e;
            if ((e = cudaMemcpyAsync(bands_dev, btab.data(), btab.size() * sizeof(int4), cudaMemcpyHostToDevice, c->stream)) ||
                (e = cudaMemcpyAsync(slot_dev, slot_row.data(), slot_row.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream)) ||
                (e = cudaStreamSynchronize(c->stream)))
                return cuda_fail(c, e, "upload band tables");
            c->h2d_bytes += btab.size() * sizeof(int4) + slot_row.size() * sizeof(int);
        }
        P.bands = bands_dev;
        P.slot_row = slot_dev;
        // ---- x1 tiles per quadrant; with c1 x1 subdomains no tile straddles a subdomain boundary,
        // the first tile of a subdomain takes its x1 carry from lagged slot sp (slot 0: the x1
        // ghosts) and the last one writes the carry into the slot of the next subdomain
        const int c1 = std::max(1, c->opt.subdomains[0]);
        std::vector<int> xslot((size_t)NQ * c1);
        std::vector<std::vector<int4>> qt(NQ);
        {
            std::vector<int> X(c1 + 1);
            for (int s = 0; s <= c1; ++s) X[s] = (s * P.n1 + c1 - 1) / c1;
            for (int q = 0; q < NQ; ++q) {
                const bool s1neg = q & 1;
                for (int sp = 0; sp < c1; ++sp) {
                    const int lo = s1neg ? P.n1 - X[c1 - sp] : X[sp];
                    const int hi = s1neg ? P.n1 - X[c1 - 1 - sp] : X[sp + 1];
                    xslot[(size_t)q * c1 + sp] = sp == 0 ? P.n1 : lo;
                    for (int cc = lo; cc < hi; cc += c->T1) {
                        const int wd = std::min(c->T1, hi - cc);
                        qt[q].push_back(make_int4(cc, wd, cc == lo ? sp : -1, cc + wd == hi ? (sp + 1) % c1 : -1));
                    }
                }
            }
        }
        P.nxslots = c1;
        P.ntiles = 0;
        for (int q = 0; q < NQ; ++q) {
            P.ntq[q] = (int)qt[q].size();
            P.ntiles = std::max(P.ntiles, P.ntq[q]);
        }
        {
            int* xs_dev = (int*)dev_alloc(c, xslot.size() * sizeof(int));
            if (!xs_dev) return fail(c, DVM_ENOMEM, "device allocation failed");
            cudaError_t e = cudaMemcpyAsync(xs_dev, xslot.data(), xslot.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream);
            P.xslot_col = xs_dev;
            P.tiles = nullptr;
            if (e == cudaSuccess && c->xsub) {
                std::vector<int4> ttab((size_t)NQ * P.ntiles, make_int4(0, 0, -1, -1));
                for (int q = 0; q < NQ; ++q)
                    for (size_t k = 0; k < qt[q].size(); ++k) ttab[(size_t)q * P.ntiles + k] = qt[q][k];
                int4* t_dev = (int4*)dev_alloc(c, ttab.size() * sizeof(int4));
                if (!t_dev) return fail(c, DVM_ENOMEM, "device allocation failed");
                e = cudaMemcpyAsync(t_dev, ttab.data(), ttab.size() * sizeof(int4), cudaMemcpyHostToDevice, c->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
                P.tiles = t_dev;
                c->h2d_bytes += ttab.size() * sizeof(int4);
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "upload tile tables");
            c->h2d_bytes += xslot.size() * sizeof(int);
        }
        P.lateral = c->opt.lateral_bc;
        P.order = c->opt.stencil_order;
        P.kn = H.kn;
        P.nu = H.nu;
        P.dx = H.dx;
        P.dinv[0] = dinv[0];
        P.dinv[1] = dinv[1];
        for (int j = 0; j < 2; ++j) P.dinvw[j] = (1.0 - c->opt.specular_fraction) * dinv[j];
        const size_t N = H.N;
        uint16_t* code = (uint16_t*)dev_alloc(c, N * sizeof(uint16_t));
        P.src = (T*)dev_alloc(c, N * 4 * sizeof(T));
        P.E = (T*)dev_alloc(c, N * 4 * sizeof(T));
        P.P = (T*)dev_alloc(c, (size_t)NQ * 3 * N * sizeof(T));
        P.gx1 = (T*)dev_alloc(c, (size_t)2 * NQ * P.nxslots * P.n2 * 2 * NL * sizeof(T));
        P.glat = (T*)dev_alloc(c, (size_t)2 * NQ * P.nslots * P.n1 * 2 * NL * sizeof(T));
        P.edge = (T*)dev_alloc(c, (size_t)NQ * 2 * P.nslots * P.n1 * 2 * NL * sizeof(T));
        T* lanec = (T*)dev_alloc(c, (size_t)NQ * NL * kLaneConsts * sizeof(T));
        P.fin_nblocks = (int)((N + kFinBlock2 - 1) / kFinBlock2);
        P.fin_block0 = (int)blk_prob.size();
        P.kpart = (double*)dev_alloc(c, (size_t)P.fin_nblocks * sizeof(double));
        P.kval = (double*)dev_alloc(c, 3 * sizeof(double));
        P.fin_counter = (unsigned int*)dev_alloc(c, sizeof(unsigned int));
        if (!code || !P.src || !P.E || !P.P || !P.gx1 || !P.glat || !P.edge || !lanec || !P.kpart || !P.kval ||
            !P.fin_counter)
            return fail(c, DVM_ENOMEM, "device allocation failed");
        P.code = code;
        P.lanec = lanec;
        // Maxwell walls with alpha < 1 (Eq. 5): wall faces (fluid point, axis, side) where the
        // point's code marks the neighbour solid, and the store of their specular parts
        P.spec = c->opt.specular_fraction;
        if (c->spec2) {
            std::vector<int> fid((size_t)4 * N, -1), faces;
            for (size_t id = 0; id < N; ++id) {
                if (H.code[id] & kSolidBit) continue;
                for (int ju = 0; ju < 4; ++ju)
                    if (((H.code[id] >> (2 * ju)) & 3) == 2) {
                        fid[(size_t)ju * N + id] = (int)faces.size();
                        faces.push_back((int)(id * 4 + ju));
                    }
            }
            P.nfaces = (int)faces.size();
            int* fid_dev = (int*)dev_alloc(c, fid.size() * sizeof(int));
            int* faces_dev = (int*)dev_alloc(c, std::max<size_t>(1, faces.size()) * sizeof(int));
            P.F = (T*)dev_alloc(c, std::max<size_t>(1, (size_t)2 * P.nfaces * 2 * NL) * sizeof(T));
            if (!fid_dev || !faces_dev || !P.F) return fail(c, DVM_ENOMEM, "device allocation failed");
            cudaError_t e2;
            if ((e2 = cudaMemcpyAsync(fid_dev, fid.data(), fid.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream)) ||
                (!faces.empty() && (e2 = cudaMemcpyAsync(faces_dev, faces.data(), faces.size() * sizeof(int),
                                                         cudaMemcpyHostToDevice, c->stream))) ||
                (e2 = cudaStreamSynchronize(c->stream)))
                return cuda_fail(c, e2, "upload face tables");
            c->h2d_bytes += (fid.size() + faces.size()) * sizeof(int);
            P.face_id = fid_dev;
            P.faces = faces_dev;
        }
        cudaError_t e = cudaMemcpyAsync(code, H.code.data(), N * sizeof(uint16_t), cudaMemcpyHostToDevice, c->stream);
        c->h2d_bytes += N * sizeof(uint16_t);
        if (e != cudaSuccess) return cuda_fail(c, e, "copy code");
        e = cudaMemsetAsync(P.fin_counter, 0, sizeof(unsigned int), c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "memset");
        e = cudaMemsetAsync(P.kval, 0, 3 * sizeof(double), c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "memset");
        e = cudaMemsetAsync(P.edge, 0, (size_t)NQ * 2 * P.nslots * P.n1 * 2 * NL * sizeof(T), c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "memset");
        // lane constants: v1, v2, |v1|/dx, |v2|/dx, W, W v1, W v2, R[0..3]
        std::vector<T> lc((size_t)NQ * NL * kLaneConsts, T(0));
        const double c0o = (P.order == 2) ? 1.5 : 1.0;
        for (int q = 0; q < NQ; ++q)
            for (int l = 0; l < NL; ++l) {
                double v1, v2, w;
                if (l < nvq) {
                    const int k = group[q][l];
                    v1 = grid->v[2 * k];
                    v2 = grid->v[2 * k + 1];
                    w = grid->w[k];
                } else {   // padding lane: finite values, zero weight
                    v1 = (q & 1) ? -1.0 : 1.0;
                    v2 = (q & 2) ? -1.0 : 1.0;
                    w = 0.0;
                }
                const double a1 = std::fabs(v1) / H.dx, a2 = std::fabs(v2) / H.dx;
                T* d = &lc[((size_t)q * NL + l) * kLaneConsts];
                d[0] = (T)v1; d[1] = (T)v2; d[2] = (T)a1; d[3] = (T)a2;
                d[4] = (T)w; d[5] = (T)(w * v1); d[6] = (T)(w * v2);
                for (int rs = 0; rs < 4; ++rs) {
                    const double c0a = (rs & 1) ? 1.0 : c0o;
                    const double c0b = (rs & 2) ? 1.0 : c0o;
                    d[7 + rs] = (T)(1.0 / (H.nu + c0a * a1 + c0b * a2));
                }
            }
        e = cudaMemcpyAsync(lanec, lc.data(), lc.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream);
        c->h2d_bytes += lc.size() * sizeof(T);
        if (e != cudaSuccess) return cuda_fail(c, e, "copy lane constants");
        e = cudaStreamSynchronize(c->stream);   // host vectors go out of scope
        if (e != cudaSuccess) return cuda_fail(c, e, "sync");
        for (int k = 0; k < P.fin_nblocks; ++k) {
            blk_prob.push_back(b);
            blk_start.push_back(k * kFinBlock2);
        }
        c->prog_offset[b] = 1 + prog_total;
        prog_total += NQ * P.nbands;
        c->kval_dev.push_back(P.kval);
    }
    // ---- work items in band order (a band only waits for lower bands: deadlock-free tickets)
    int maxb = 0;
    for (int b = 0; b < c->nprob; ++b) maxb = std::max(maxb, probs[b].nbands);
    for (int band = 0; band < maxb; ++band)
        for (int b = 0; b < c->nprob; ++b)
            for (int q = 0; q < NQ; ++q)
                if (band < c->hp[b].qbands[q]) items.push_back({b, q, band, 0});
    c->nitems = (int)items.size();
    c->counters_bytes = sizeof(int) * (size_t)(1 + prog_total);
    c->counters_dev = (int*)dev_alloc(c, c->counters_bytes);
    c->status_dev = (int*)dev_alloc(c, sizeof(int));
    c->items_dev = (SweepItem*)dev_alloc(c, items.size() * sizeof(SweepItem));
    c->fin_blocks = (int)blk_prob.size();
    c->blk_prob_dev = (int*)dev_alloc(c, blk_prob.size() * sizeof(int));
    c->blk_start_dev = (int*)dev_alloc(c, blk_start.size() * sizeof(int));
    c->qw_dev = (double*)dev_alloc(c, qw.size() * sizeof(double));
    size_t maxN = 0;
    for (auto& H : c->hp) maxN = std::max(maxN, (size_t)H.N);
    c->scratch_bytes = maxN * 4 * sizeof(double);
    c->scratch_dev = (double*)dev_alloc(c, c->scratch_bytes);
    c->probs_dev = dev_alloc(c, probs.size() * sizeof(Prob2D<T>));
    if (!c->counters_dev || !c->status_dev || !c->items_dev || !c->blk_prob_dev || !c->blk_start_dev ||
        !c->qw_dev || !c->scratch_dev || !c->probs_dev)
        return fail(c, DVM_ENOMEM, "device allocation failed");
    for (int b = 0; b < c->nprob; ++b) probs[b].prog = c->counters_dev + c->prog_offset[b];
    cudaError_t e;
    if ((e = cudaMemcpyAsync(c->items_dev, items.data(), items.size() * sizeof(SweepItem), cudaMemcpyHostToDevice, c->stream)) ||
        (e = cudaMemcpyAsync(c->blk_prob_dev, blk_prob.data(), blk_prob.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream)) ||
        (e = cudaMemcpyAsync(c->blk_start_dev, blk_start.data(), blk_start.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream)) ||
        (e = cudaMemcpyAsync(c->qw_dev, qw.data(), qw.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream)) ||
        (e = cudaMemcpyAsync(c->probs_dev, probs.data(), probs.size() * sizeof(Prob2D<T>), cudaMemcpyHostToDevice, c->stream)) ||
        (e = cudaMemsetAsync(c->status_dev, 0, sizeof(int), c->stream)) ||
        (e = cudaStreamSynchronize(c->stream)))
        return cuda_fail(c, e, "upload");
    c->h2d_bytes += items.size() * sizeof(SweepItem) + (blk_prob.size() + blk_start.size()) * sizeof(int) +
                    qw.size() * sizeof(double) + probs.size() * sizeof(Prob2D<T>);
    c->probs_host.assign((const char*)probs.data(), (const char*)probs.data() + probs.size() * sizeof(Prob2D<T>));
    // ---- persistent grid size
    int per_sm = 0;
    if (c->prec == DVM_FP32) e = sweep2d_f32x2_occupancy(c->T1, c->xsub, c->spec2 ? 1 : 0, c->NW, c->max_rows, &per_sm);
    else e = sweep2d_occupancy<T>(c->T1, c->xsub, c->spec2 ? 1 : 0, c->NW, c->max_rows, &per_sm);
    if (e != cudaSuccess) return cuda_fail(c, e, "occupancy");
    if (per_sm < 1) return fail(c, DVM_EINVAL, "sweep kernel does not fit on an SM with these tiles");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c->sweep_grid = std::max(1, std::min(c->nitems, per_sm * sms));
    // ---- zero-perturbation start
    for (int b = 0; b < c->nprob; ++b) {
        const Prob2D<T>* pd = (const Prob2D<T>*)c->probs_dev + b;
        e = launch_init2d<T>(pd, NL, c->qw_dev + (size_t)b * NQ * 3, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    }
    FinArgs2D<T> fa{(const Prob2D<T>*)c->probs_dev, c->blk_prob_dev, c->blk_start_dev, c->status_dev};
    e = launch_finalize2d<T>(fa, c->fin_blocks, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "finalize kernel");
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "init");
    return DVM_OK;
}


// Blocks of the lagged-halo decomposition along one axis of n points (Sec. 3.2: block s holds the
// points l with floor(l c / n) = s), split into pieces of at most R points, for both orientations
// (o = 1: the axis is swept from its high end).  Entry {first oriented index, count, below, above}:
// below = s (ghost slot of block s) for the first piece of oriented block s, else -1 - ring slot;
// above = (s + 1) mod c for its last piece, else -1 - ring slot; ring slots 2 s + (piece & 1).
// slot[o][s] = the oriented index that follows the two layers held in ghost slot s.
static void axis_blocks(int n, int c, int R, std::vector<int4> (&tab)[2], std::vector<int>& slot) {
    std::vector<int> Y(c + 1);
    for (int s = 0; s <= c; ++s) Y[s] = (int)(((long long)s * n + c - 1) / c);
    slot.assign((size_t)2 * c, 0);
    for (int o = 0; o < 2; ++o) {
        tab[o].clear();
        for (int sp = 0; sp < c; ++sp) {
            const int lo = o ? n - Y[c - sp] : Y[sp];
            const int hi = o ? n - Y[c - 1 - sp] : Y[sp + 1];
            slot[(size_t)o * c + sp] = sp == 0 ? n : lo;
            int jl = 0;
            for (int r0 = lo; r0 < hi; r0 += R, ++jl) {
                const int nr = std::min(R, hi - r0);
                tab[o].push_back(make_int4(r0, nr, r0 == lo ? sp : -1 - (2 * sp + ((jl - 1) & 1)),
                                           r0 + nr == hi ? (sp + 1) % c : -1 - (2 * sp + (jl & 1))));
            }
        }
    }
}

template <typename T>
dvm_status build_3d(dvm_ctx* c, const dvm_geometry* geoms, const dvm_velocity_grid* grid) {
    const int NO = 8;
    // ---- velocity groups: octant q (bit j set when v_j < 0), lanes ordered by (|v1|, |v2|, |v3|)
    std::vector<std::vector<int>> group(NO);
    for (int k = 0; k < grid->nv; ++k) {
        const double* v = grid->v + 3 * k;
        group[(v[0] < 0 ? 1 : 0) | (v[1] < 0 ? 2 : 0) | (v[2] < 0 ? 4 : 0)].push_back(k);
    }
    auto key_less = [&](int a, int b) {
        const double* va = grid->v + 3 * a;
        const double* vb = grid->v + 3 * b;
        for (int j = 0; j < 3; ++j)
            if (std::fabs(va[j]) != std::fabs(vb[j])) return std::fabs(va[j]) < std::fabs(vb[j]);
        return false;
    };
    for (auto& g : group) std::sort(g.begin(), g.end(), key_less);
    const int nvo = (int)group[0].size();
    for (int q = 1; q < NO; ++q)
        if ((int)group[q].size() != nvo) return fail(c, DVM_EINVAL, "velocity grid is not symmetric under sign changes");
    for (int m = 0; m < nvo; ++m) {
        const double* v0 = grid->v + 3 * group[0][m];
        for (int q = 1; q < NO; ++q) {
            const double* vq = grid->v + 3 * group[q][m];
            for (int j = 0; j < 3; ++j)
                if (std::fabs(vq[j]) != std::fabs(v0[j])) return fail(c, DVM_EINVAL, "velocity grid is not symmetric under sign changes");
            if (grid->w[group[q][m]] != grid->w[group[0][m]]) return fail(c, DVM_EINVAL, "velocity grid is not symmetric under sign changes");
        }
    }
    c->nvq = nvo;
    // FP32 lanes carry two velocity slots (packed f32x2 kernel), FP64 lanes and the Shakhov model's
    // scalar kernel one
    c->packed3 = c->prec == DVM_FP32 && c->nx3 == 0;
    const int vpl = c->packed3 ? sweep3d_f32x2_velocities_per_lane() : 1;
    const int warps_total = (nvo + 32 * vpl - 1) / (32 * vpl);
    // at most 8 warps per CTA (group_warps: fewer warps per CTA, more velocity groups)
    // (FP64 default: 4 warps per CTA, with the 2 x 2 pencils below 1.24x faster than 8 warps and
    // 4 x 4 pencils on a 128^3 rock with 16^3 velocities)
    const int wmax = (c->opt.group_warps > 0) ? std::min(8, c->opt.group_warps) : (c->prec == DVM_FP64 ? 4 : 8);
    c->G = (warps_total + wmax - 1) / wmax;
    c->NW = (warps_total + c->G - 1) / c->G;
    c->GL = 32 * vpl * c->NW;                             // velocity slots per group
    c->NL = c->GL * c->G;
    const int NL = c->NL, G = c->G;
    // default tiles: FP32 (packed kernel) 8 columns, swept as two 4-column sub-tiles (one wait and
    // one publish per 8 columns: 1.12x faster than 4-column tiles on a 128^3 rock with 16^3
    // velocities); FP64 4 columns.  Default pencils 4 x 4 rows, FP64 2 x 2.
    c->T1 = c->opt.tile_x1 == 8 ? 8 : (c->opt.tile_x1 == 4 ? 4 : (c->packed3 ? 8 : 4));
    const int R = c->opt.band_rows ? c->opt.band_rows : (c->prec == DVM_FP64 ? 2 : 4);
    c->R2 = c->R3 = std::max(1, R);
    {
        // shrink the tile, then the pencil, until the CTA's shared memory fits the device limit
        int dev = 0, smem_max = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (smem_max <= 0) smem_max = 227 * 1024;
        const size_t lim = (size_t)smem_max - 1024;
        auto smem_of = [&]() -> size_t {
            if (c->packed3) return sweep3d_f32x2_smem(c->T1, c->NW, c->R2, c->R3, c->tau3, c->spec2);
            return sweep3d_smem<T>(c->T1, c->NW, c->R2, c->R3, c->tau3, c->spec2, c->nx3);
        };
        while (smem_of() > lim) {
            if (c->T1 > 4) c->T1 = 4;
            else if (c->R2 > 1) { c->R2--; c->R3 = c->R2; }
            else return fail(c, DVM_EINVAL, "3D sweep does not fit in shared memory");
        }
    }
    int mr2 = 1, mr3 = 1;
    for (int b = 0; b < c->nprob; ++b) {
        mr2 = std::max(mr2, std::min(c->R2, c->hp[b].n[1]));
        mr3 = std::max(mr3, std::min(c->R3, c->hp[b].n[2]));
    }
    c->max_rows = mr2 * 1000 + mr3;   // packed (R2, R3) maxima
    double dwall[3] = {0, 0, 0};
    for (int k = 0; k < grid->nv; ++k)
        for (int j = 0; j < 3; ++j)
            if (grid->v[3 * k + j] > 0) dwall[j] += grid->w[k] * grid->v[3 * k + j];
    const double dinv[3] = {1.0 / dwall[0], 1.0 / dwall[1], 1.0 / dwall[2]};
    // group weight sums for the start state: [nprob][8][G][4]
    std::vector<double> qw((size_t)c->nprob * NO * G * 4, 0.0);
    for (int b = 0; b < c->nprob; ++b)
        for (int q = 0; q < NO; ++q)
            for (int m = 0; m < nvo; ++m) {
                const int k = group[q][m];
                const int gg = m / c->GL;
                double* d = &qw[(((size_t)b * NO + q) * G + gg) * 4];
                d[0] += grid->w[k];
                for (int j = 0; j < 3; ++j) d[1 + j] += grid->w[k] * grid->v[3 * k + j];
            }
    // ---- warm-start tables: lane velocities and group sums of W phi_m psi_n, phi = psi = (1, v)
    // (qwt: the same with phi = |v|^2, for the temperature term; sw2 = sum of W |v|^2 over the grid)
    std::vector<double> qw2((size_t)NO * G * 4 * 4, 0.0), vel((size_t)NO * NL * 3, 0.0), qwt((size_t)NO * G * 4, 0.0);
    // model moments: source factors phi_a and moment functions psi_a of a velocity (Shakhov: the
    // heat flux, ES-BGK: the traceless stress), the group sums of W psi_a (1, v) and the grid sums
    // of W psi_a (the source-form shift)
    const int nx = c->nx3;
    auto model_fns = [nx](const double* v, double* phi, double* psi) {
        const double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        if (nx == 3)
            for (int j = 0; j < 3; ++j) phi[j] = psi[j] = v[j] * (vv - 2.5);
        if (nx == 6) {
            const int I[6] = {0, 1, 2, 0, 0, 1}, J[6] = {0, 1, 2, 1, 2, 2};
            for (int m = 0; m < 6; ++m) {
                phi[m] = (m < 3 ? 1.0 : 2.0) * v[I[m]] * v[J[m]];
                psi[m] = 2.0 * (v[I[m]] * v[J[m]] - (m < 3 ? vv / 3.0 : 0.0));
            }
        }
    };
    std::vector<double> qwx((size_t)NO * G * std::max(nx, 1) * 4, 0.0);
    double sx[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q < NO; ++q)
        for (int m = 0; m < nvo; ++m) {
            const int k = group[q][m];
            const int gg = m / c->GL;
            const double ph[4] = {1.0, grid->v[3 * k], grid->v[3 * k + 1], grid->v[3 * k + 2]};
            for (int j = 0; j < 3; ++j) vel[((size_t)q * NL + m) * 3 + j] = ph[1 + j];
            for (int a = 0; a < 4; ++a)
                for (int b2 = 0; b2 < 4; ++b2)
                    qw2[(((size_t)q * G + gg) * 4 + a) * 4 + b2] += grid->w[k] * ph[a] * ph[b2];
            const double vv = ph[1] * ph[1] + ph[2] * ph[2] + ph[3] * ph[3];
            for (int b2 = 0; b2 < 4; ++b2) qwt[((size_t)q * G + gg) * 4 + b2] += grid->w[k] * vv * ph[b2];
            if (nx) {
                double phi[6], psi[6];
                model_fns(grid->v + 3 * k, phi, psi);
                for (int m = 0; m < nx; ++m)
                    for (int b2 = 0; b2 < 4; ++b2)
                        qwx[(((size_t)q * G + gg) * nx + m) * 4 + b2] += grid->w[k] * psi[m] * ph[b2];
            }
        }
    if (nx)
        for (int k = 0; k < grid->nv; ++k) {
            double phi[6], psi[6];
            model_fns(grid->v + 3 * k, phi, psi);
            for (int m = 0; m < nx; ++m) sx[m] += grid->w[k] * psi[m];
        }
    double sw2 = 0.0;
    for (int k = 0; k < grid->nv; ++k)
        for (int j = 0; j < 3; ++j) sw2 += grid->w[k] * grid->v[3 * k + j] * grid->v[3 * k + j];
    c->qw2_dev = (double*)dev_alloc(c, qw2.size() * sizeof(double));
    c->vel_dev = (double*)dev_alloc(c, vel.size() * sizeof(double));
    c->qwt_dev = (double*)dev_alloc(c, qwt.size() * sizeof(double));
    c->qwx_dev = (double*)dev_alloc(c, qwx.size() * sizeof(double));
    if (!c->qw2_dev || !c->vel_dev || !c->qwt_dev || !c->qwx_dev) return fail(c, DVM_ENOMEM, "device allocation failed");
    {
        cudaError_t e;
        if ((e = cudaMemcpyAsync(c->qw2_dev, qw2.data(), qw2.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream)) ||
            (e = cudaMemcpyAsync(c->vel_dev, vel.data(), vel.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream)) ||
            (e = cudaMemcpyAsync(c->qwt_dev, qwt.data(), qwt.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream)) ||
            (e = cudaMemcpyAsync(c->qwx_dev, qwx.data(), qwx.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream)) ||
            (e = cudaStreamSynchronize(c->stream)))
            return cuda_fail(c, e, "upload warm-start tables");
        c->h2d_bytes += (qw2.size() + vel.size() + qwt.size() + qwx.size()) * sizeof(double);
    }
    std::vector<Prob3D<T>> probs(c->nprob);
    std::vector<SweepItem3> items;
    std::vector<int> blk_prob, blk_start;
    int prog_total = 0;
    c->prog_offset.assign(c->nprob, 0);
    for (int b = 0; b < c->nprob; ++b) {
        HostProb& H = c->hp[b];
        Prob3D<T>& P = probs[b];
        std::memset(&P, 0, sizeof(P));
        P.n1 = H.n[0];
        P.n2 = H.n[1];
        P.n3 = H.n[2];
        P.N = H.N;
        P.R2 = std::min(c->R2, P.n2);
        P.R3 = std::min(c->R3, P.n3);
        // pencils along x2 and x3 and tiles along x1, per orientation; with c_j lagged-halo blocks
        // (Sec. 3.2) no pencil or tile straddles a block boundary
        P.ns1 = std::max(1, c->opt.subdomains[0]);
        P.ns2 = std::max(1, c->opt.subdomains[1]);
        P.ns3 = std::max(1, c->opt.subdomains[2]);
        std::vector<int4> t1[2], t2[2], t3[2];
        std::vector<int> sc1, sr2, sr3;
        axis_blocks(P.n1, P.ns1, c->T1, t1, sc1);
        axis_blocks(P.n2, P.ns2, P.R2, t2, sr2);
        axis_blocks(P.n3, P.ns3, P.R3, t3, sr3);
        for (auto& tab : t1)
            for (auto& e : tab) {   // tiles: carry-in / carry-out ghost slot or -1
                e.z = e.z >= 0 ? e.z : -1;
                e.w = e.w >= 0 ? e.w : -1;
            }
        P.nt1 = (int)t1[0].size();
        P.np2 = (int)t2[0].size();
        P.np3 = (int)t3[0].size();
        {
            std::vector<int4> tabs;
            for (auto* t : {&t2[0], &t2[1], &t3[0], &t3[1], &t1[0], &t1[1]}) tabs.insert(tabs.end(), t->begin(), t->end());
            std::vector<int> slots;
            for (auto* t : {&sr2, &sr3, &sc1}) slots.insert(slots.end(), t->begin(), t->end());
            int4* tabs_dev = (int4*)dev_alloc(c, tabs.size() * sizeof(int4));
            int* slots_dev = (int*)dev_alloc(c, slots.size() * sizeof(int));
            if (!tabs_dev || !slots_dev) return fail(c, DVM_ENOMEM, "device allocation failed");
            cudaError_t e;
            if ((e = cudaMemcpyAsync(tabs_dev, tabs.data(), tabs.size() * sizeof(int4), cudaMemcpyHostToDevice, c->stream)) ||
                (e = cudaMemcpyAsync(slots_dev, slots.data(), slots.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream)) ||
                (e = cudaStreamSynchronize(c->stream)))
                return cuda_fail(c, e, "upload pencil tables");
            c->h2d_bytes += tabs.size() * sizeof(int4) + slots.size() * sizeof(int);
            P.pen2 = tabs_dev;
            P.pen3 = tabs_dev + 2 * P.np2;
            P.tiles1 = tabs_dev + 2 * P.np2 + 2 * P.np3;
            P.slot_row2 = slots_dev;
            P.slot_row3 = slots_dev + 2 * P.ns2;
            P.slot_col1 = slots_dev + 2 * P.ns2 + 2 * P.ns3;
        }
        P.ngroups = G;
        P.lateral = c->opt.lateral_bc;
        P.order = c->opt.stencil_order;
        P.kn = H.kn;
        P.nu = H.nu;
        P.dx = H.dx;
        for (int j = 0; j < 3; ++j) P.dinv[j] = dinv[j];
        for (int j = 0; j < 3; ++j) P.dinvw[j] = (1.0 - c->opt.specular_fraction) * dinv[j];
        const size_t N = H.N;
        const size_t n1 = P.n1, n2 = P.n2, n3 = P.n3;
        uint16_t* code = (uint16_t*)dev_alloc(c, N * sizeof(uint16_t));
        P.src = (T*)dev_alloc(c, N * 4 * sizeof(T));
        P.E = (T*)dev_alloc(c, N * 8 * sizeof(T));
        P.P = (T*)dev_alloc(c, (size_t)NO * G * 4 * N * sizeof(T));
        P.tau = c->tau3 ? 1 : 0;
        P.sw2 = sw2;
        if (P.tau) {
            P.Pt = (T*)dev_alloc(c, (size_t)NO * G * N * sizeof(T));
            P.srct = (T*)dev_alloc(c, N * sizeof(T));
            if (!P.Pt || !P.srct) return fail(c, DVM_ENOMEM, "device allocation failed");
        }
        // model moments: Shakhov A = (4/5)(1 - Pr), the coefficient for which the heat flux relaxes
        // at Pr times the collision frequency; ES-BGK 1 - 1/Pr, with the collision frequency Pr nu
        // (set with the problem's nu) so that the stress relaxes at the BGK rate
        P.nx = nx;
        P.xcoef = nx == 3 ? 0.8 * (1.0 - c->opt.shakhov_prandtl) : (nx == 6 ? 1.0 - 1.0 / c->opt.es_prandtl : 0.0);
        for (int m = 0; m < 6; ++m) P.sx[m] = sx[m];
        if (nx) {
            P.Px = (T*)dev_alloc(c, (size_t)NO * G * nx * N * sizeof(T));
            P.srcx = (T*)dev_alloc(c, N * 8 * sizeof(T));
            if (!P.Px || !P.srcx) return fail(c, DVM_ENOMEM, "device allocation failed");
        }
        // Maxwell walls with alpha < 1 (Eq. 5): wall faces from the point codes and their store
        P.spec = c->opt.specular_fraction;
        if (c->spec2) {
            std::vector<int> fid((size_t)6 * N, -1), faces;
            for (size_t id = 0; id < N; ++id) {
                if (H.code[id] & kSolidBit) continue;
                for (int ju = 0; ju < 6; ++ju)
                    if (((H.code[id] >> (2 * ju)) & 3) == 2) {
                        fid[(size_t)ju * N + id] = (int)faces.size();
                        faces.push_back((int)(id * 8 + ju));
                    }
            }
            P.nfaces = (int)faces.size();
            int* fid_dev = (int*)dev_alloc(c, fid.size() * sizeof(int));
            int* faces_dev = (int*)dev_alloc(c, std::max<size_t>(1, faces.size()) * sizeof(int));
            P.F = (T*)dev_alloc(c, std::max<size_t>(1, (size_t)2 * P.nfaces * 4 * NL) * sizeof(T));
            if (!fid_dev || !faces_dev || !P.F) return fail(c, DVM_ENOMEM, "device allocation failed");
            cudaError_t e2;
            if ((e2 = cudaMemcpyAsync(fid_dev, fid.data(), fid.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream)) ||
                (!faces.empty() && (e2 = cudaMemcpyAsync(faces_dev, faces.data(), faces.size() * sizeof(int),
                                                         cudaMemcpyHostToDevice, c->stream))) ||
                (e2 = cudaStreamSynchronize(c->stream)))
                return cuda_fail(c, e2, "upload face tables");
            c->h2d_bytes += (fid.size() + faces.size()) * sizeof(int);
            P.face_id = fid_dev;
            P.faces = faces_dev;
        }
        P.bf16 = c->bf16 ? 1 : 0;
        const size_t es = c->bf16 ? 2 : sizeof(T);     // bytes per stored ghost / edge value
        P.gx1 = (T*)dev_alloc(c, (size_t)2 * NO * P.ns1 * n3 * n2 * 2 * NL * es);
        P.gy = (T*)dev_alloc(c, (size_t)2 * NO * P.ns2 * n3 * n1 * 2 * NL * es);
        P.gz = (T*)dev_alloc(c, (size_t)2 * NO * P.ns3 * n2 * n1 * 2 * NL * es);
        // pencil edges: two slots per pencil column and block suffice (pencil p + 2 reaches tile t
        // only after pencil p + 1 has consumed pencil p's edge of tile t; the first pencil of a block
        // does not wait, so every block has its own pair)
        const size_t ey_sz = (size_t)NO * P.np3 * 2 * P.ns2 * P.R3 * n1 * 2 * NL;
        const size_t ez_sz = (size_t)NO * P.np2 * 2 * P.ns3 * P.R2 * n1 * 2 * NL;
        P.ey = (T*)dev_alloc(c, ey_sz * es);
        P.ez = (T*)dev_alloc(c, ez_sz * es);
        T* lanec = (T*)dev_alloc(c, (size_t)NO * NL * kLaneConsts3 * sizeof(T));
        P.fin_nblocks = (int)((N + kFinBlock3 - 1) / kFinBlock3);
        P.fin_block0 = (int)blk_prob.size();
        P.kpart = (double*)dev_alloc(c, (size_t)P.fin_nblocks * sizeof(double));
        P.kval = (double*)dev_alloc(c, 3 * sizeof(double));
        P.fin_counter = (unsigned int*)dev_alloc(c, sizeof(unsigned int));
        if (!code || !P.src || !P.E || !P.P || !P.gx1 || !P.gy || !P.gz || !P.ey || !P.ez || !lanec || !P.kpart ||
            !P.kval || !P.fin_counter)
            return fail(c, DVM_ENOMEM, "device allocation failed");
        P.code = code;
        P.lanec = lanec;
        cudaError_t e;
        if ((e = cudaMemcpyAsync(code, H.code.data(), N * sizeof(uint16_t), cudaMemcpyHostToDevice, c->stream)) ||
            (e = cudaMemsetAsync(P.fin_counter, 0, sizeof(unsigned int), c->stream)) ||
            (e = cudaMemsetAsync(P.kval, 0, 3 * sizeof(double), c->stream)) ||
            (e = cudaMemsetAsync(P.ey, 0, ey_sz * es, c->stream)) ||
            (e = cudaMemsetAsync(P.ez, 0, ez_sz * es, c->stream)))
            return cuda_fail(c, e, "upload");
        c->h2d_bytes += N * sizeof(uint16_t);
        std::vector<T> lc((size_t)NO * NL * kLaneConsts3, T(0));
        const double c0o = (P.order == 2) ? 1.5 : 1.0;
        for (int q = 0; q < NO; ++q)
            for (int l = 0; l < NL; ++l) {
                double v[3], w;
                if (l < nvo) {
                    const int k = group[q][l];
                    for (int j = 0; j < 3; ++j) v[j] = grid->v[3 * k + j];
                    w = grid->w[k];
                } else {   // padding lane: finite values, zero weight
                    for (int j = 0; j < 3; ++j) v[j] = ((q >> j) & 1) ? -1.0 : 1.0;
                    w = 0.0;
                }
                T* d = &lc[((size_t)q * NL + l) * kLaneConsts3];
                double av[3];
                for (int j = 0; j < 3; ++j) {
                    av[j] = std::fabs(v[j]) / H.dx;
                    d[j] = (T)v[j];
                    d[3 + j] = (T)av[j];
                    d[7 + j] = (T)(w * v[j]);
                }
                d[6] = (T)w;
                const double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
                d[18] = (T)(vv - 1.5);    // temperature term: |v|^2 - 3/2 and W |v|^2
                d[19] = (T)(w * vv);
                if (nx) {   // model moments: phi_a and W psi_a
                    double phi[6], psi[6];
                    model_fns(v, phi, psi);
                    for (int m = 0; m < nx; ++m) {
                        d[20 + m] = (T)phi[m];
                        d[26 + m] = (T)(w * psi[m]);
                    }
                }
                for (int rs = 0; rs < 8; ++rs) {
                    double den = H.nu;
                    for (int j = 0; j < 3; ++j) den += (((rs >> j) & 1) ? 1.0 : c0o) * av[j];
                    d[10 + rs] = (T)(1.0 / den);
                }
            }
        if ((e = cudaMemcpyAsync(lanec, lc.data(), lc.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream)) ||
            (e = cudaStreamSynchronize(c->stream)))
            return cuda_fail(c, e, "upload lane constants");
        c->h2d_bytes += lc.size() * sizeof(T);
        for (int k = 0; k < P.fin_nblocks; ++k) {
            blk_prob.push_back(b);
            blk_start.push_back(k * kFinBlock3);
        }
        c->prog_offset[b] = 1 + prog_total;
        prog_total += NO * G * P.np3 * P.np2;
        c->kval_dev.push_back(P.kval);
    }
    // ---- items ordered by pencil level (a pencil waits only on lower levels)
    int maxlevel = 0;
    for (int b = 0; b < c->nprob; ++b) maxlevel = std::max(maxlevel, probs[b].np2 + probs[b].np3 - 2);
    for (int lev = 0; lev <= maxlevel; ++lev)
        for (int b = 0; b < c->nprob; ++b)
            for (int p3 = 0; p3 < probs[b].np3; ++p3) {
                const int p2 = lev - p3;
                if (p2 < 0 || p2 >= probs[b].np2) continue;
                for (int q = 0; q < NO; ++q)
                    for (int gg = 0; gg < G; ++gg) items.push_back({b, q, p2, p3, gg, 0, 0, 0});
            }
    c->nitems = (int)items.size();
    c->counters_bytes = sizeof(int) * (size_t)(1 + prog_total);
    c->counters_dev = (int*)dev_alloc(c, c->counters_bytes);
    c->status_dev = (int*)dev_alloc(c, sizeof(int));
    c->items_dev = (SweepItem*)dev_alloc(c, items.size() * sizeof(SweepItem3));
    c->fin_blocks = (int)blk_prob.size();
    c->blk_prob_dev = (int*)dev_alloc(c, blk_prob.size() * sizeof(int));
    c->blk_start_dev = (int*)dev_alloc(c, blk_start.size() * sizeof(int));
    c->qw_dev = (double*)dev_alloc(c, qw.size() * sizeof(double));
    size_t maxN = 0;
    for (auto& H : c->hp) maxN = std::max(maxN, (size_t)H.N);
    c->scratch_bytes = maxN * 6 * sizeof(double);
    c->scratch_dev = (double*)dev_alloc(c, c->scratch_bytes);
    c->probs_dev = dev_alloc(c, probs.size() * sizeof(Prob3D<T>));
    if (!c->counters_dev || !c->status_dev || !c->items_dev || !c->blk_prob_dev || !c->blk_start_dev ||
        !c->qw_dev || !c->scratch_dev || !c->probs_dev)
        return fail(c, DVM_ENOMEM, "device allocation failed");
    for (int b = 0; b < c->nprob; ++b) probs[b].prog = c->counters_dev + c->prog_offset[b];
    cudaError_t e;
    if ((e = cudaMemcpyAsync(c->items_dev, items.data(), items.size() * sizeof(SweepItem3), cudaMemcpyHostToDevice, c->stream)) ||
        (e = cudaMemcpyAsync(c->blk_prob_dev, blk_prob.data(), blk_prob.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream)) ||
        (e = cudaMemcpyAsync(c->blk_start_dev, blk_start.data(), blk_start.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream)) ||
        (e = cudaMemcpyAsync(c->qw_dev, qw.data(), qw.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream)) ||
        (e = cudaMemcpyAsync(c->probs_dev, probs.data(), probs.size() * sizeof(Prob3D<T>), cudaMemcpyHostToDevice, c->stream)) ||
        (e = cudaMemsetAsync(c->status_dev, 0, sizeof(int), c->stream)) ||
        (e = cudaStreamSynchronize(c->stream)))
        return cuda_fail(c, e, "upload");
    c->h2d_bytes += items.size() * sizeof(SweepItem3) + (blk_prob.size() + blk_start.size()) * sizeof(int) +
                    qw.size() * sizeof(double) + probs.size() * sizeof(Prob3D<T>);
    c->probs_host.assign((const char*)probs.data(), (const char*)probs.data() + probs.size() * sizeof(Prob3D<T>));
    int per_sm = 0;
    if (c->packed3)
        e = sweep3d_f32x2_occupancy(c->T1, c->NW, mr2, mr3, c->bf16 ? 1 : 0, c->sub3 ? 1 : 0, c->tau3 ? 1 : 0,
                                    c->spec2 ? 1 : 0, &per_sm);
    else e = sweep3d_occupancy<T>(c->T1, c->NW, mr2, mr3, 0, c->sub3 ? 1 : 0, c->tau3 ? 1 : 0, c->spec2 ? 1 : 0,
                                  c->nx3, &per_sm);
    if (e != cudaSuccess) return cuda_fail(c, e, "occupancy");
    if (per_sm < 1) return fail(c, DVM_EINVAL, "3D sweep kernel does not fit on an SM with these pencils");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c->sweep_grid = std::max(1, std::min(c->nitems, per_sm * sms));
    for (int b = 0; b < c->nprob; ++b) {
        const Prob3D<T>* pd = (const Prob3D<T>*)c->probs_dev + b;
        e = launch_init3d<T>(pd, NL, c->qw_dev + (size_t)b * NO * G * 4, c->qwt_dev, c->qwx_dev, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    }
    FinArgs3D<T> fa{(const Prob3D<T>*)c->probs_dev, c->blk_prob_dev, c->blk_start_dev, c->status_dev};
    e = launch_finalize3d<T>(fa, c->fin_blocks, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "finalize kernel");
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "init");
    return DVM_OK;
}

template <typename T>
dvm_status enqueue_iter_3d(dvm_ctx* c);

cudaEvent_t take_event(dvm_ctx* c) {
    const size_t used = c->ev_marks.size();
    if (used < c->ev_pool.size()) return c->ev_pool[used];
    cudaEvent_t ev = nullptr;
    if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
    c->ev_pool.push_back(ev);
    return ev;
}

cudaError_t mark(dvm_ctx* c) {
    if (!c->profile) return cudaSuccess;
    if (c->capturing) {   // an event record node of the graph: recorded at every replay
        cudaEvent_t ev = nullptr;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return e;
        c->capture_marks.push_back(ev);
        return cudaEventRecordWithFlags(ev, c->stream, cudaEventRecordExternal);
    }
    cudaEvent_t ev = take_event(c);
    if (!ev) return cudaErrorMemoryAllocation;
    c->ev_marks.push_back(ev);
    return cudaEventRecord(ev, c->stream);
}

cudaError_t sweep_launch(const SweepArgs2D<float>& a, dvm_ctx* c) {
    return launch_sweep2d_f32x2(a, c->T1, c->xsub, c->sweep_grid, c->NW, c->stream);
}

cudaError_t sweep_launch(const SweepArgs2D<double>& a, dvm_ctx* c) {
    return launch_sweep2d<double>(a, c->T1, c->xsub, c->sweep_grid, c->NW, c->stream);
}

template <typename T>
dvm_status enqueue_iter_2d(dvm_ctx* c) {
    cudaError_t e = cudaMemsetAsync(c->counters_dev, 0, c->counters_bytes, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset counters");
    SweepArgs2D<T> a;
    a.spec = c->spec2 ? 1 : 0;
    a.prob = (const Prob2D<T>*)c->probs_dev;
    a.items = c->items_dev;
    a.nitems = c->nitems;
    a.NL = c->NL;
    a.max_rows = c->max_rows;
    a.parity = (int)(c->iters & 1);
    a.ticket = c->counters_dev;
    a.status = c->status_dev;
    a.timeout_ns = c->timeout_ns;
    a.withhold_item = c->withhold_item;
    if ((e = mark(c)) != cudaSuccess) return cuda_fail(c, e, "event");
    e = sweep_launch(a, c);
    if (e != cudaSuccess) return cuda_fail(c, e, "sweep kernel");
    if ((e = mark(c)) != cudaSuccess) return cuda_fail(c, e, "event");
    FinArgs2D<T> fa{(const Prob2D<T>*)c->probs_dev, c->blk_prob_dev, c->blk_start_dev, c->status_dev};
    e = launch_finalize2d<T>(fa, c->fin_blocks, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "finalize kernel");
    if ((e = mark(c)) != cudaSuccess) return cuda_fail(c, e, "event");
    c->iters++;
    return DVM_OK;
}

cudaError_t sweep3d_launch(const SweepArgs3D<float>& a, dvm_ctx* c) {
    if (!c->packed3) return launch_sweep3d<float>(a, c->sweep_grid, c->NW, c->stream);   // Shakhov
    return launch_sweep3d_f32x2(a, c->sweep_grid, c->NW, c->stream);
}

cudaError_t sweep3d_launch(const SweepArgs3D<double>& a, dvm_ctx* c) {
    return launch_sweep3d<double>(a, c->sweep_grid, c->NW, c->stream);
}

template <typename T>
dvm_status enqueue_iter_3d(dvm_ctx* c) {
    cudaError_t e = cudaMemsetAsync(c->counters_dev, 0, c->counters_bytes, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset counters");
    SweepArgs3D<T> a;
    a.prob = (const Prob3D<T>*)c->probs_dev;
    a.items = (const SweepItem3*)c->items_dev;
    a.nitems = c->nitems;
    a.NL = c->NL;
    a.GL = c->GL;
    a.T1 = c->T1;
    a.maxR2 = c->max_rows / 1000;
    a.maxR3 = c->max_rows % 1000;
    a.bf16 = c->bf16 ? 1 : 0;
    a.sub = c->sub3 ? 1 : 0;
    a.tau = c->tau3 ? 1 : 0;
    a.nx = c->nx3;
    a.spec = c->spec2 ? 1 : 0;
    a.parity = (int)(c->iters & 1);
    a.ticket = c->counters_dev;
    a.status = c->status_dev;
    a.timeout_ns = c->timeout_ns;
    a.withhold_item = c->withhold_item;
    if ((e = mark(c)) != cudaSuccess) return cuda_fail(c, e, "event");
    e = sweep3d_launch(a, c);
    if (e != cudaSuccess) return cuda_fail(c, e, "sweep kernel");
    if ((e = mark(c)) != cudaSuccess) return cuda_fail(c, e, "event");
    FinArgs3D<T> fa{(const Prob3D<T>*)c->probs_dev, c->blk_prob_dev, c->blk_start_dev, c->status_dev};
    e = launch_finalize3d<T>(fa, c->fin_blocks, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "finalize kernel");
    if ((e = mark(c)) != cudaSuccess) return cuda_fail(c, e, "event");
    c->iters++;
    return DVM_OK;
}

dvm_status enqueue_iter(dvm_ctx* c) {
    if (c->dims == 3) return c->prec == DVM_FP32 ? enqueue_iter_3d<float>(c) : enqueue_iter_3d<double>(c);
    return c->prec == DVM_FP32 ? enqueue_iter_2d<float>(c) : enqueue_iter_2d<double>(c);
}

// add the kernel times of the last profiled graph replay (its stream work must be complete)
cudaError_t drain_graph_marks(dvm_ctx* c) {
    if (!c->graph_pending) return cudaSuccess;
    const std::vector<cudaEvent_t>& m = *c->graph_pending;
    c->graph_pending = nullptr;
    for (size_t i = 0; i + 2 < m.size(); i += 3) {
        float a = 0.f, b = 0.f;
        cudaError_t e;
        if ((e = cudaEventElapsedTime(&a, m[i], m[i + 1])) != cudaSuccess ||
            (e = cudaEventElapsedTime(&b, m[i + 1], m[i + 2])) != cudaSuccess)
            return e;
        c->acc_sweep_ms += a;
        c->acc_fin_ms += b;
        ++c->acc_sweep_n;
        ++c->acc_fin_n;
    }
    return cudaSuccess;
}

void drop_graphs(dvm_ctx* c) {
    c->graph_pending = nullptr;
    for (auto& g : c->graphs) {
        cudaGraphExecDestroy(g.exec);
        for (cudaEvent_t ev : g.marks) cudaEventDestroy(ev);
    }
    c->graphs.clear();
}

// n iterations: one by one, or through a captured CUDA graph (same launches, same bits)
dvm_status run_iterations(dvm_ctx* c, int n) {
    if (n <= 0) return DVM_OK;
    if (!c->opt.use_graph || c->stream == nullptr) {
        for (int i = 0; i < n; ++i) {
            dvm_status s = enqueue_iter(c);
            if (s != DVM_OK) return s;
        }
        return DVM_OK;
    }
    const int par = (int)(c->iters & 1);
    cudaError_t e;
    // a profiled graph re-records its own events: read the previous replay's first
    if (c->graph_pending) {
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "stream");
        if ((e = drain_graph_marks(c)) != cudaSuccess) return cuda_fail(c, e, "event timing");
    }
    for (auto& g : c->graphs)
        if (g.n == n && g.parity == par && g.prof == c->profile) {
            if ((e = cudaGraphLaunch(g.exec, c->stream)) != cudaSuccess) return cuda_fail(c, e, "graph launch");
            if (g.prof) c->graph_pending = &g.marks;
            c->iters += n;
            return DVM_OK;
        }
    const long long it0 = c->iters;
    if ((e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
        return cuda_fail(c, e, "begin capture");
    c->capturing = c->profile;
    c->capture_marks.clear();
    dvm_status s = DVM_OK;
    for (int i = 0; i < n && s == DVM_OK; ++i) s = enqueue_iter(c);
    c->capturing = false;
    std::vector<cudaEvent_t> marks;
    marks.swap(c->capture_marks);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(c->stream, &graph);
    c->iters = it0;     // the captured launches have not run yet
    cudaGraphExec_t exec = nullptr;
    if (s == DVM_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (s != DVM_OK || e != cudaSuccess) {
        for (cudaEvent_t ev : marks) cudaEventDestroy(ev);
        if (s != DVM_OK) return s;
        return cuda_fail(c, e, "graph capture");
    }
    c->graphs.push_back({n, par, c->profile, exec, std::move(marks)});
    if ((e = cudaGraphLaunch(exec, c->stream)) != cudaSuccess) return cuda_fail(c, e, "graph launch");
    if (c->profile) c->graph_pending = &c->graphs.back().marks;
    c->iters += n;
    return DVM_OK;
}

// wait for the stream, fetch k of every problem and the device status word
dvm_status collect(dvm_ctx* c) {
    cudaError_t e;
    for (int b = 0; b < c->nprob; ++b) {
        const double* kv = c->kval_dev[b];
        e = cudaMemcpyAsync(c->kval_host + 3 * b, kv, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "read permeability");
    }
    e = cudaMemcpyAsync(c->status_host, c->status_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "read status");
    c->d2h_bytes += (long long)c->nprob * 3 * sizeof(double) + sizeof(int);
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream");
    if ((e = drain_graph_marks(c)) != cudaSuccess) return cuda_fail(c, e, "event timing");
    if (*c->status_host != 0) {
        const int st = *c->status_host;
        cudaMemsetAsync(c->status_dev, 0, sizeof(int), c->stream);
        cudaStreamSynchronize(c->stream);
        if (st == DVM_ETIMEOUT) return fail(c, DVM_ETIMEOUT, "a bounded wait in the sweep kernel expired");
        return fail(c, DVM_ECUDA, "device status " + std::to_string(st));
    }
    return DVM_OK;
}

// Rebuild sources, wall terms and permeability of every problem from the moment partials.
dvm_status run_finalize(dvm_ctx* c) {
    cudaError_t e;
    if (c->dims == 3) {
        if (c->prec == DVM_FP32) {
            FinArgs3D<float> fa{(const Prob3D<float>*)c->probs_dev, c->blk_prob_dev, c->blk_start_dev, c->status_dev};
            e = launch_finalize3d<float>(fa, c->fin_blocks, c->stream);
        } else {
            FinArgs3D<double> fa{(const Prob3D<double>*)c->probs_dev, c->blk_prob_dev, c->blk_start_dev, c->status_dev};
            e = launch_finalize3d<double>(fa, c->fin_blocks, c->stream);
        }
    } else if (c->prec == DVM_FP32) {
        FinArgs2D<float> fa{(const Prob2D<float>*)c->probs_dev, c->blk_prob_dev, c->blk_start_dev, c->status_dev};
        e = launch_finalize2d<float>(fa, c->fin_blocks, c->stream);
    } else {
        FinArgs2D<double> fa{(const Prob2D<double>*)c->probs_dev, c->blk_prob_dev, c->blk_start_dev, c->status_dev};
        e = launch_finalize2d<double>(fa, c->fin_blocks, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "finalize kernel");
    return DVM_OK;
}

// ---- iteration state (checkpoint / resume): moment partials + ghost layers of the read parity

struct Seg {
    void* p;
    size_t bytes;
};

template <typename T>
void state_segs_2d(const Prob2D<T>& P, size_t NL, int par, std::vector<Seg>& out) {
    const size_t gx = (size_t)4 * P.nxslots * P.n2 * 2 * NL, gl = (size_t)4 * P.nslots * P.n1 * 2 * NL;
    out.push_back({P.P, (size_t)4 * 3 * P.N * sizeof(T)});
    out.push_back({P.gx1 + par * gx, gx * sizeof(T)});
    out.push_back({P.glat + par * gl, gl * sizeof(T)});
    if (P.spec > 0.0 && P.nfaces > 0) {
        const size_t fs = (size_t)P.nfaces * 2 * NL;
        out.push_back({P.F + par * fs, fs * sizeof(T)});
    }
}

template <typename T>
void state_segs_3d(const Prob3D<T>& P, size_t NL, int par, std::vector<Seg>& out) {
    const size_t gx = (size_t)8 * P.ns1 * P.n3 * P.n2 * 2 * NL;
    const size_t gy = (size_t)8 * P.ns2 * P.n3 * P.n1 * 2 * NL;
    const size_t gz = (size_t)8 * P.ns3 * P.n2 * P.n1 * 2 * NL;
    const size_t es = P.bf16 ? 2 : sizeof(T);
    out.push_back({P.P, (size_t)8 * P.ngroups * 4 * P.N * sizeof(T)});
    if (P.tau) out.push_back({P.Pt, (size_t)8 * P.ngroups * P.N * sizeof(T)});
    if (P.nx) out.push_back({P.Px, (size_t)8 * P.ngroups * P.nx * P.N * sizeof(T)});
    if (P.spec > 0.0 && P.nfaces > 0) {
        const size_t fs = (size_t)P.nfaces * 4 * NL;
        out.push_back({P.F + par * fs, fs * sizeof(T)});
    }
    out.push_back({(char*)P.gx1 + par * gx * es, gx * es});
    out.push_back({(char*)P.gy + par * gy * es, gy * es});
    out.push_back({(char*)P.gz + par * gz * es, gz * es});
}

std::vector<Seg> state_segments(const dvm_ctx* c, int par) {
    std::vector<Seg> out;
    for (int b = 0; b < c->nprob; ++b) {
        if (c->dims == 3) {
            if (c->prec == DVM_FP32) state_segs_3d(((const Prob3D<float>*)c->probs_host.data())[b], c->NL, par, out);
            else state_segs_3d(((const Prob3D<double>*)c->probs_host.data())[b], c->NL, par, out);
        } else {
            if (c->prec == DVM_FP32) state_segs_2d(((const Prob2D<float>*)c->probs_host.data())[b], c->NL, par, out);
            else state_segs_2d(((const Prob2D<double>*)c->probs_host.data())[b], c->NL, par, out);
        }
    }
    return out;
}

struct StateHeader {
    char magic[8];
    int32_t version, dims, precision, nprob, nv, NL, G, order, lateral, pad;
    int64_t iters;
    double last_err;
};

struct StateProb {
    int64_t n[3];
    double kn, k_check;
    int64_t it_check;
};

constexpr char kStateMagic[8] = {'D', 'V', 'M', 'S', 'T', 'A', 'T', 'E'};

StateHeader state_header(const dvm_ctx* c) {
    StateHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kStateMagic, 8);
    h.version = 2;
    h.dims = c->dims;
    h.precision = c->opt.precision;
    h.nprob = c->nprob;
    h.nv = c->nv;
    h.NL = c->NL;
    h.G = c->G;
    h.order = c->opt.stencil_order;
    h.lateral = c->opt.lateral_bc;
    h.iters = c->iters;
    h.last_err = c->last_err;
    return h;
}

size_t state_bytes(const dvm_ctx* c) {
    size_t n = sizeof(StateHeader) + (size_t)c->nprob * sizeof(StateProb);
    for (const Seg& sg : state_segments(c, 0)) n += sg.bytes;
    return n;
}

dvm_status validate_grid(dvm_ctx* c, int dims, const dvm_velocity_grid* g) {
    if (!g || g->nv <= 0 || !g->v || !g->w) return fail(c, DVM_EINVAL, "velocity grid is empty");
    double s = 0.0;
    for (int k = 0; k < g->nv; ++k) {
        for (int j = 0; j < dims; ++j) {
            const double vj = g->v[(size_t)k * dims + j];
            if (!(vj != 0.0) || !std::isfinite(vj)) return fail(c, DVM_EINVAL, "velocity component zero or not finite");
        }
        if (!(g->w[k] > 0.0) || !std::isfinite(g->w[k])) return fail(c, DVM_EINVAL, "weight not positive");
        s += g->w[k];
    }
    if (std::fabs(s - 1.0) > 1e-12) return fail(c, DVM_EINVAL, "weights do not sum to 1");
    return DVM_OK;
}

}  // namespace

extern "C" {

void dvm_default_options(dvm_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = DVM_FP64;
    o->stencil_order = 2;
    o->lateral_bc = DVM_LATERAL_SPECULAR;
    o->check_interval = 100;
}

dvm_status dvm_effective_pore_size(int dims, double k_inf, double porosity, double* ratio) {
    if (!ratio || (dims != 2 && dims != 3) || !(k_inf > 0.0) || !std::isfinite(k_inf) || !(porosity > 0.0) ||
        !(porosity <= 1.0))
        return DVM_EINVAL;
    *ratio = dims == 2 ? std::sqrt(12.0 * k_inf / porosity) : std::sqrt(8.0 * k_inf / (3.14159265358979323846 * porosity));
    return DVM_OK;
}

dvm_status dvm_gh_velocity_grid(int dims, int n, double* v, double* w) {
    if ((dims != 2 && dims != 3) || n < 2 || n > 128 || (n & 1) || !v || !w) return DVM_EINVAL;
    const int m = n / 2;
    std::vector<double> cc(m), aa(m);
    if (!half_range_gh(m, cc.data(), aa.data())) return DVM_EINVAL;
    std::vector<double> v1(n), w1(n);
    const double isqpi = 1.0 / std::sqrt(3.14159265358979323846);
    for (int i = 0; i < m; ++i) {
        v1[m - 1 - i] = -cc[i];
        w1[m - 1 - i] = aa[i] * isqpi;
        v1[m + i] = cc[i];
        w1[m + i] = aa[i] * isqpi;
    }
    const int nv = dims == 2 ? n * n : n * n * n;
    for (int k = 0; k < nv; ++k) {
        int idx[3];
        int r = k;
        for (int j = dims - 1; j >= 0; --j) {   // axis 0 slowest
            idx[j] = r % n;
            r /= n;
        }
        double wk = 1.0;
        for (int j = 0; j < dims; ++j) {
            v[(size_t)k * dims + j] = v1[idx[j]];
            wk *= w1[idx[j]];
        }
        w[k] = wk;
    }
    return DVM_OK;
}

dvm_status dvm_create_batch(int nprob, const dvm_geometry* geoms, const double* kn, const dvm_velocity_grid* grid,
                            const dvm_options* opt, dvm_ctx** out) {
    if (!out) return DVM_EINVAL;
    *out = nullptr;
    dvm_ctx* c = new (std::nothrow) dvm_ctx();
    if (!c) return DVM_ENOMEM;
    if (opt) c->opt = *opt;
    else dvm_default_options(&c->opt);
    g_create_err.clear();
    auto reject = [&](dvm_status s, const char* m) {
        // creation failed before any device work: the message stays readable through
        // dvm_last_error(NULL) on this thread
        g_create_err = m;
        delete c;
        return s;
    };
    if (nprob < 1 || !geoms || !kn) return reject(DVM_EINVAL, "no problems");
    const int dims = geoms[0].dims;
    if (dims != 2 && dims != 3) return reject(DVM_EINVAL, "dims must be 2 or 3");
    if (c->opt.precision != DVM_FP64 && c->opt.precision != DVM_FP32 && c->opt.precision != DVM_BF16_STORE)
        return reject(DVM_EINVAL, "precision");
    if (c->opt.precision == DVM_BF16_STORE && dims != 3)
        return reject(DVM_EINVAL, "BF16 storage is implemented for 3D problems only");
    if (c->opt.stencil_order != 1 && c->opt.stencil_order != 2) return reject(DVM_EINVAL, "stencil_order");
    if (c->opt.lateral_bc != 0 && c->opt.lateral_bc != 1) return reject(DVM_EINVAL, "lateral_bc");
    if (c->opt.check_interval < 1) return reject(DVM_EINVAL, "check_interval");
    for (int j = 0; j < 3; ++j)
        if (c->opt.subdomains[j] < 0) return reject(DVM_EINVAL, "subdomain counts must not be negative");
    if (dims == 2 && c->opt.subdomains[2] > 1) return reject(DVM_EINVAL, "a 2D problem has no x3 subdomains");
    c->xsub = dims == 2 && c->opt.subdomains[0] > 1;
    c->sub3 = dims == 3 && (c->opt.subdomains[0] > 1 || c->opt.subdomains[1] > 1 || c->opt.subdomains[2] > 1);
    if (c->sub3 && c->opt.precision == DVM_BF16_STORE)
        return reject(DVM_EINVAL, "BF16 storage is not implemented with subdomains");
    if (c->opt.temperature_term && dims != 3)
        return reject(DVM_EINVAL, "the temperature term is implemented for 3D problems (Eq. 2 has three velocity components)");
    if (c->opt.temperature_term && c->opt.precision == DVM_BF16_STORE)
        return reject(DVM_EINVAL, "BF16 storage is not implemented with the temperature term");
    c->tau3 = dims == 3 && c->opt.temperature_term != 0;
    if (!(c->opt.specular_fraction >= 0.0 && c->opt.specular_fraction <= 1.0))
        return reject(DVM_EINVAL, "specular_fraction (1 - alpha of Eq. 5) must lie in [0, 1]");
    if (c->opt.specular_fraction > 0.0 && c->opt.precision == DVM_BF16_STORE)
        return reject(DVM_EINVAL, "BF16 storage is not implemented with alpha < 1");
    c->spec2 = c->opt.specular_fraction > 0.0;
    if (!(c->opt.shakhov_prandtl >= 0.0) || !std::isfinite(c->opt.shakhov_prandtl))
        return reject(DVM_EINVAL, "shakhov_prandtl must be 0 (BGK) or a positive Prandtl number");
    if (c->opt.shakhov_prandtl > 0.0 && (dims != 3 || !c->opt.temperature_term))
        return reject(DVM_EINVAL, "the Shakhov model is implemented for 3D problems with the temperature term");
    if (c->opt.shakhov_prandtl > 0.0 && (c->sub3 || c->spec2 || c->opt.precision == DVM_BF16_STORE))
        return reject(DVM_EINVAL, "the Shakhov model is not implemented with subdomains, alpha < 1 or BF16 storage");
    if (!(c->opt.es_prandtl >= 0.0) || !std::isfinite(c->opt.es_prandtl))
        return reject(DVM_EINVAL, "es_prandtl must be 0 (BGK) or a positive Prandtl number");
    if (c->opt.es_prandtl > 0.0 && (dims != 3 || !c->opt.temperature_term))
        return reject(DVM_EINVAL, "the ES-BGK model is implemented for 3D problems with the temperature term");
    if (c->opt.es_prandtl > 0.0 && (c->sub3 || c->spec2 || c->opt.precision == DVM_BF16_STORE))
        return reject(DVM_EINVAL, "the ES-BGK model is not implemented with subdomains, alpha < 1 or BF16 storage");
    if (c->opt.es_prandtl > 0.0 && c->opt.shakhov_prandtl > 0.0)
        return reject(DVM_EINVAL, "choose one model: Shakhov or ES-BGK");
    c->nx3 = c->opt.shakhov_prandtl > 0.0 ? 3 : (c->opt.es_prandtl > 0.0 ? 6 : 0);
    if (c->opt.group_warps < 0) return reject(DVM_EINVAL, "group_warps must not be negative");
    c->dims = dims;
    c->nprob = nprob;
    c->prec = c->opt.precision == DVM_BF16_STORE ? DVM_FP32 : c->opt.precision;
    c->bf16 = c->opt.precision == DVM_BF16_STORE;
    c->stream = (cudaStream_t)c->opt.stream;
    if (validate_grid(c, dims, grid) != DVM_OK) {
        const std::string m = c->err;
        return reject(DVM_EINVAL, m.c_str());
    }
    c->nv = grid->nv;
    c->hp.resize(nprob);
    for (int b = 0; b < nprob; ++b) {
        const dvm_geometry& g = geoms[b];
        if (g.dims != dims || !g.solid) return reject(DVM_EINVAL, "geometry");
        if (!(kn[b] > 0.0) || !std::isfinite(kn[b])) return reject(DVM_EINVAL, "Knudsen number must be positive");
        HostProb& H = c->hp[b];
        long long N = 1;
        for (int j = 0; j < 3; ++j) {
            H.n[j] = (j < dims) ? (int)g.n[j] : 1;
            if (j < dims && (g.n[j] < 3 || g.n[j] > (1 << 20))) return reject(DVM_EINVAL, "every extent must be >= 3");
            N *= H.n[j];
        }
        if (N > (1LL << 30)) return reject(DVM_EINVAL, "geometry too large");
        if (c->opt.subdomains[1] > 1 && g.n[1] < 2LL * c->opt.subdomains[1])
            return reject(DVM_EINVAL, "every x2 subdomain needs at least two rows");
        if (c->opt.subdomains[0] > 1 && g.n[0] < 2LL * c->opt.subdomains[0])
            return reject(DVM_EINVAL, "every x1 subdomain needs at least two columns");
        if (dims == 3 && c->opt.subdomains[2] > 1 && g.n[2] < 2LL * c->opt.subdomains[2])
            return reject(DVM_EINVAL, "every x3 subdomain needs at least two planes");
        H.N = (int)N;
        H.kn = kn[b];
        H.nu = std::sqrt(3.14159265358979323846) / (2.0 * kn[b]);
        // ES-BGK: the collision frequency Pr nu keeps the BGK viscosity (the Kn of Eq. 1)
        if (c->nx3 == 6) H.nu *= c->opt.es_prandtl;
        H.dx = 1.0 / H.n[0];
        classify(H, dims, g.solid, c->opt.lateral_bc, c->opt.stencil_order);
        long long fluid = 0, faces = 0;
        for (int id = 0; id < H.N; ++id) {
            if (H.code[id] & kSolidBit) continue;
            ++fluid;
            for (int s = 0; s < 2 * dims; ++s)
                if (((H.code[id] >> (2 * s)) & 3) == 2) ++faces;
        }
        if (fluid == 0) return reject(DVM_EINVAL, "no fluid voxel");
        if (faces == 0) return reject(DVM_EINVAL, "no solid/fluid interface: the steady problem has no solution");
    }
    cudaError_t e;
    if ((e = cudaMallocHost(&c->kval_host, sizeof(double) * 3 * nprob)) != cudaSuccess ||
        (e = cudaMallocHost(&c->status_host, sizeof(int))) != cudaSuccess) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return e == cudaErrorMemoryAllocation ? DVM_ENOMEM : DVM_ECUDA;
    }
    dvm_status s;
    if (dims == 3) s = (c->prec == DVM_FP32) ? build_3d<float>(c, geoms, grid) : build_3d<double>(c, geoms, grid);
    else s = (c->prec == DVM_FP32) ? build_2d<float>(c, geoms, grid) : build_2d<double>(c, geoms, grid);
    if (s != DVM_OK) {
        cudaStreamSynchronize(c->stream);
        free_all(c);
        delete c;
        return s;
    }
    c->k_check.assign(nprob, 0.0);   // k of the zero start h = 0
    c->it_check.assign(nprob, 0);
    *out = c;
    return DVM_OK;
}

dvm_status dvm_create(const dvm_geometry* geometry, double kn, const dvm_velocity_grid* grid, const dvm_options* opt,
                      dvm_ctx** out) {
    return dvm_create_batch(1, geometry, &kn, grid, opt, out);
}

dvm_status dvm_step(dvm_ctx* c, int n) {
    if (!c || n < 0) return DVM_EINVAL;
    return run_iterations(c, n);
}

dvm_status dvm_sync(dvm_ctx* c) {
    if (!c) return DVM_EINVAL;
    return collect(c);
}

dvm_status dvm_iterate(dvm_ctx* c, int max_iter, double tol, int* iters_done, double* err_out) {
    if (!c || max_iter < 0 || !(tol >= 0.0)) return DVM_EINVAL;
    const int ci = c->opt.check_interval;
    int done = 0;
    dvm_status result = DVM_NOT_CONVERGED;
    while (done < max_iter) {
        const int to_check = ci - (int)(c->iters % ci);
        const int n = std::min(to_check, max_iter - done);
        {
            dvm_status s = run_iterations(c, n);
            if (s != DVM_OK) return s;
        }
        done += n;
        if (c->iters % ci != 0) continue;
        dvm_status s = collect(c);
        if (s != DVM_OK) {
            if (iters_done) *iters_done = done;
            return s;
        }
        double worst = 0.0;
        for (int b = 0; b < c->nprob; ++b) {
            const double k = c->kval_host[3 * b];
            if (!std::isfinite(k)) {
                if (iters_done) *iters_done = done;
                return fail(c, DVM_ENUMERIC, "permeability is not finite");
            }
            // Eq. 15: Err = |k(l) - k(l - ci)| / (ci |k(l)|), k(l - ci) the k of the previous check
            // (of the start state at the first one).  Checks fall on multiples of ci; when
            // dvm_step or a warm start moved the previous one, ci becomes the actual gap.
            const double gap = (double)std::max(1LL, c->iters - c->it_check[b]);
            const double err = (k != 0.0) ? std::fabs((k - c->k_check[b]) / k) / gap : (c->k_check[b] == 0.0 ? 0.0 : HUGE_VAL);
            worst = std::max(worst, err);
            c->k_check[b] = k;
            c->it_check[b] = c->iters;
        }
        c->last_err = worst;
        if (worst < tol) {
            result = DVM_OK;
            break;
        }
    }
    if (iters_done) *iters_done = done;
    if (err_out) *err_out = c->last_err;
    return result;
}

dvm_status dvm_moments_at(dvm_ctx* c, int prob, double* rho, double* u, int on_device) {
    if (!c || prob < 0 || prob >= c->nprob || !rho || !u) return DVM_EINVAL;
    const size_t N = c->hp[prob].N;
    double* drho = on_device ? rho : c->scratch_dev;
    double* du = on_device ? u : c->scratch_dev + N;
    cudaError_t e;
    if (c->dims == 3) {
        if (c->prec == DVM_FP32) e = launch_moments3d<float>((const Prob3D<float>*)c->probs_dev + prob, drho, du, c->stream);
        else e = launch_moments3d<double>((const Prob3D<double>*)c->probs_dev + prob, drho, du, c->stream);
    } else if (c->prec == DVM_FP32) {
        e = launch_moments2d<float>((const Prob2D<float>*)c->probs_dev + prob, drho, du, c->stream);
    } else {
        e = launch_moments2d<double>((const Prob2D<double>*)c->probs_dev + prob, drho, du, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "moments kernel");
    if (!on_device) {
        if ((e = cudaMemcpyAsync(rho, drho, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream)) ||
            (e = cudaMemcpyAsync(u, du, N * c->dims * sizeof(double), cudaMemcpyDeviceToHost, c->stream)))
            return cuda_fail(c, e, "read moments");
        c->d2h_bytes += (long long)N * (1 + c->dims) * sizeof(double);
    }
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "moments");
    return DVM_OK;
}

dvm_status dvm_moments(dvm_ctx* c, double* rho, double* u, int on_device) {
    return dvm_moments_at(c, 0, rho, u, on_device);
}

dvm_status dvm_temperature_at(dvm_ctx* c, int prob, double* tau, int on_device) {
    if (!c || prob < 0 || prob >= c->nprob || !tau) return DVM_EINVAL;
    if (!c->tau3) return fail(c, DVM_EINVAL, "the temperature term is not enabled");
    const size_t N = c->hp[prob].N;
    double* dt = on_device ? tau : c->scratch_dev;
    cudaError_t e;
    if (c->prec == DVM_FP32) e = launch_temperature3d<float>((const Prob3D<float>*)c->probs_dev + prob, dt, c->stream);
    else e = launch_temperature3d<double>((const Prob3D<double>*)c->probs_dev + prob, dt, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "temperature kernel");
    if (!on_device) {
        if ((e = cudaMemcpyAsync(tau, dt, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
            return cuda_fail(c, e, "read temperature");
        c->d2h_bytes += (long long)N * sizeof(double);
    }
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "temperature");
    return DVM_OK;
}

// model moments [nx][N] of problem prob (heat flux of the Shakhov model, stress of ES-BGK)
static dvm_status model_moments_at(dvm_ctx* c, int prob, double* out, int on_device, int want_nx, const char* what) {
    if (!c || prob < 0 || prob >= c->nprob || !out) return DVM_EINVAL;
    if (c->nx3 != want_nx) return fail(c, DVM_EINVAL, what);
    const size_t N = c->hp[prob].N;
    double* d = on_device ? out : c->scratch_dev;
    cudaError_t e;
    if (c->prec == DVM_FP32) e = launch_modelmoments3d<float>((const Prob3D<float>*)c->probs_dev + prob, d, c->stream);
    else e = launch_modelmoments3d<double>((const Prob3D<double>*)c->probs_dev + prob, d, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "model-moment kernel");
    if (!on_device) {
        if ((e = cudaMemcpyAsync(out, d, (size_t)want_nx * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
            return cuda_fail(c, e, "read model moments");
        c->d2h_bytes += (long long)((size_t)want_nx * N * sizeof(double));
    }
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "model moments");
    return DVM_OK;
}

dvm_status dvm_heat_flux_at(dvm_ctx* c, int prob, double* q, int on_device) {
    return model_moments_at(c, prob, q, on_device, 3, "the Shakhov model is not enabled");
}

dvm_status dvm_stress_at(dvm_ctx* c, int prob, double* p, int on_device) {
    return model_moments_at(c, prob, p, on_device, 6, "the ES-BGK model is not enabled");
}

dvm_status dvm_wall_density_at(dvm_ctx* c, int prob, double* rhos) {
    if (!c || prob < 0 || prob >= c->nprob || !rhos) return DVM_EINVAL;
    const size_t N = c->hp[prob].N;
    cudaError_t e;
    if (c->dims == 3) {
        if (c->prec == DVM_FP32) e = launch_wall3d<float>((const Prob3D<float>*)c->probs_dev + prob, c->scratch_dev, c->stream);
        else e = launch_wall3d<double>((const Prob3D<double>*)c->probs_dev + prob, c->scratch_dev, c->stream);
    } else if (c->prec == DVM_FP32) {
        e = launch_wall2d<float>((const Prob2D<float>*)c->probs_dev + prob, c->scratch_dev, c->stream);
    } else {
        e = launch_wall2d<double>((const Prob2D<double>*)c->probs_dev + prob, c->scratch_dev, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "wall kernel");
    if ((e = cudaMemcpyAsync(rhos, c->scratch_dev, N * 2 * c->dims * sizeof(double), cudaMemcpyDeviceToHost, c->stream)) ||
        (e = cudaStreamSynchronize(c->stream)))
        return cuda_fail(c, e, "read wall densities");
    c->d2h_bytes += (long long)N * 2 * c->dims * sizeof(double);
    return DVM_OK;
}

dvm_status dvm_permeability_at(dvm_ctx* c, int prob, double* k, double* gp) {
    if (!c || prob < 0 || prob >= c->nprob) return DVM_EINVAL;
    dvm_status s = collect(c);
    if (s != DVM_OK) return s;
    if (k) *k = c->kval_host[3 * prob];
    if (gp) *gp = c->kval_host[3 * prob + 1];
    return DVM_OK;
}

dvm_status dvm_permeability(dvm_ctx* c, double* k, double* gp) { return dvm_permeability_at(c, 0, k, gp); }

dvm_status dvm_autotune(int nprob, const dvm_geometry* geoms, const double* kn, const dvm_velocity_grid* grid,
                        dvm_options* opt, int iters, double* best_ms) {
    if (!opt || iters < 1 || nprob < 1 || !geoms) return DVM_EINVAL;
    const int dims = geoms[0].dims;
    std::vector<std::array<int, 3>> cand;    // (tile_x1, band_rows, group_warps)
    const int gw0 = opt->group_warps;
    if (dims == 3) {
        for (int w : {8, 4}) {
            if (gw0 > 0 && w != 8) break;        // warps per CTA fixed by the caller
            for (int t : {4, 8})
                for (int r : {2, 3, 4, 5, 6}) cand.push_back({t, r, gw0 > 0 ? gw0 : w});
        }
    } else if (opt->precision == DVM_FP32) {
        for (int t : {16, 8, 4})
            for (int r : {4, 8, 12, 16}) cand.push_back({t, r, gw0});
    } else {
        for (int t : {8, 16})
            for (int r : {4, 8, 12, 16}) cand.push_back({t, r, gw0});
    }
    cudaStream_t st = (cudaStream_t)opt->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        g_create_err = "autotune: event creation failed";
        return DVM_ECUDA;
    }
    double best = HUGE_VAL;
    int best_t = 0, best_r = 0, best_w = gw0;
    std::vector<std::array<int, 3>> seen;     // effective shapes after the library's clamping
    std::string last_reject;
    dvm_status result = DVM_OK;
    for (auto [t, r, w] : cand) {
        dvm_options o = *opt;
        o.tile_x1 = t;
        o.band_rows = r;
        o.group_warps = w;
        o.use_graph = 0;                     // time the launches, not a first capture
        dvm_ctx* c = nullptr;
        dvm_status s = dvm_create_batch(nprob, geoms, kn, grid, &o, &c);
        if (s == DVM_EINVAL) {               // does not fit (or invalid input: reported below)
            last_reject = g_create_err;
            continue;
        }
        if (s != DVM_OK) { result = s; break; }
        const std::array<int, 3> eff{c->T1, dims == 3 ? c->R2 : c->rows, c->NW};
        bool dup = false;
        for (auto& x : seen) dup = dup || (x == eff);
        if (dup) { dvm_destroy(c); continue; }
        seen.push_back(eff);
        float ms = 0.f;
        s = dvm_step(c, 2);
        if (s == DVM_OK) s = dvm_sync(c);
        if (s == DVM_OK && cudaEventRecord(e0, st) != cudaSuccess) s = DVM_ECUDA;
        if (s == DVM_OK) s = dvm_step(c, iters);
        if (s == DVM_OK && cudaEventRecord(e1, st) != cudaSuccess) s = DVM_ECUDA;
        if (s == DVM_OK) s = dvm_sync(c);
        if (s == DVM_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) s = DVM_ECUDA;
        if (s != DVM_OK) g_create_err = std::string("autotune: ") + c->err;
        dvm_destroy(c);
        if (s != DVM_OK) { result = s; break; }
        const double per = ms / iters;
        if (per < best) { best = per; best_t = t; best_r = r; best_w = w; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != DVM_OK) return result;
    if (!(best < HUGE_VAL)) {
        g_create_err = "autotune: no candidate tile shape was accepted (last reason: " + last_reject + ")";
        return DVM_EINVAL;
    }
    opt->tile_x1 = best_t;
    opt->band_rows = best_r;
    opt->group_warps = best_w;
    if (best_ms) *best_ms = best;
    return DVM_OK;
}

dvm_status dvm_set_initial_at(dvm_ctx* c, int prob, const double* rho0, const double* u0) {
    if (!c || prob < 0 || prob >= c->nprob || !rho0 || !u0) return DVM_EINVAL;
    const HostProb& H = c->hp[prob];
    const size_t N = H.N;
    for (size_t i = 0; i < N; ++i) {
        if (H.code[i] & kSolidBit) continue;
        bool ok = std::isfinite(rho0[i]);
        for (int j = 0; j < c->dims; ++j) ok = ok && std::isfinite(u0[(size_t)j * N + i]);
        if (!ok) return fail(c, DVM_EINVAL, "warm start: value not finite at a fluid point");
    }
    double* d_rho = c->scratch_dev;
    double* d_u = c->scratch_dev + N;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d_rho, rho0, N * sizeof(double), cudaMemcpyHostToDevice, c->stream)) ||
        (e = cudaMemcpyAsync(d_u, u0, N * c->dims * sizeof(double), cudaMemcpyHostToDevice, c->stream)))
        return cuda_fail(c, e, "upload warm start");
    c->h2d_bytes += (long long)N * (1 + c->dims) * sizeof(double);
    const int par = (int)(c->iters & 1);
    if (c->dims == 3) {
        if (c->prec == DVM_FP32)
            e = launch_warm3d<float>((const Prob3D<float>*)c->probs_dev + prob, c->NL, par, c->qw2_dev, c->qwt_dev, c->qwx_dev, c->vel_dev, d_rho, d_u, c->stream);
        else
            e = launch_warm3d<double>((const Prob3D<double>*)c->probs_dev + prob, c->NL, par, c->qw2_dev, c->qwt_dev, c->qwx_dev, c->vel_dev, d_rho, d_u, c->stream);
    } else if (c->prec == DVM_FP32) {
        e = launch_warm2d<float>((const Prob2D<float>*)c->probs_dev + prob, c->NL, par, c->qw2_dev, c->vel_dev, d_rho, d_u, c->stream);
    } else {
        e = launch_warm2d<double>((const Prob2D<double>*)c->probs_dev + prob, c->NL, par, c->qw2_dev, c->vel_dev, d_rho, d_u, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "warm-start kernel");
    dvm_status s = run_finalize(c);
    if (s != DVM_OK) return s;
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "warm start");
    // the next Eq. 15 check compares with the k of the warm-start state
    s = collect(c);
    if (s != DVM_OK) return s;
    c->k_check[prob] = c->kval_host[3 * prob];
    c->it_check[prob] = c->iters;
    return DVM_OK;
}

dvm_status dvm_set_initial(dvm_ctx* c, const double* rho0, const double* u0) {
    return dvm_set_initial_at(c, 0, rho0, u0);
}

dvm_status dvm_get_state(dvm_ctx* c, void* buf, size_t* bytes) {
    if (!c || !bytes) return DVM_EINVAL;
    const size_t need = state_bytes(c);
    if (!buf) {
        *bytes = need;
        return DVM_OK;
    }
    if (*bytes < need) {
        *bytes = need;
        return fail(c, DVM_EINVAL, "state buffer too small");
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "get state");
    char* out = static_cast<char*>(buf);
    const StateHeader h = state_header(c);
    std::memcpy(out, &h, sizeof(h));
    out += sizeof(h);
    for (int b = 0; b < c->nprob; ++b) {
        StateProb sp;
        for (int j = 0; j < 3; ++j) sp.n[j] = c->hp[b].n[j];
        sp.kn = c->hp[b].kn;
        sp.k_check = c->k_check[b];
        sp.it_check = c->it_check[b];
        std::memcpy(out, &sp, sizeof(sp));
        out += sizeof(sp);
    }
    for (const Seg& sg : state_segments(c, (int)(c->iters & 1))) {
        if ((e = cudaMemcpyAsync(out, sg.p, sg.bytes, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
            return cuda_fail(c, e, "read state");
        out += sg.bytes;
        c->d2h_bytes += (long long)sg.bytes;
    }
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "read state");
    *bytes = need;
    return DVM_OK;
}

dvm_status dvm_set_state(dvm_ctx* c, const void* buf, size_t bytes) {
    if (!c || !buf) return DVM_EINVAL;
    if (bytes != state_bytes(c)) return fail(c, DVM_EINVAL, "state size does not match this context");
    const char* in = static_cast<const char*>(buf);
    StateHeader h;
    std::memcpy(&h, in, sizeof(h));
    in += sizeof(h);
    const StateHeader mine = state_header(c);
    if (std::memcmp(h.magic, kStateMagic, 8) != 0 || h.version != 2)
        return fail(c, DVM_EINVAL, "not a state written by dvm_get_state");
    if (h.dims != mine.dims || h.precision != mine.precision || h.nprob != mine.nprob || h.nv != mine.nv ||
        h.NL != mine.NL || h.G != mine.G || h.order != mine.order || h.lateral != mine.lateral || h.iters < 0)
        return fail(c, DVM_EINVAL, "state was written by a context with other options or velocity grid");
    std::vector<double> kc(c->nprob);
    std::vector<long long> ic(c->nprob);
    for (int b = 0; b < c->nprob; ++b) {
        StateProb sp;
        std::memcpy(&sp, in, sizeof(sp));
        in += sizeof(sp);
        for (int j = 0; j < 3; ++j)
            if (sp.n[j] != c->hp[b].n[j]) return fail(c, DVM_EINVAL, "state was written for other geometries");
        if (sp.kn != c->hp[b].kn) return fail(c, DVM_EINVAL, "state was written for other Knudsen numbers");
        if (sp.it_check < 0 || sp.it_check > h.iters) return fail(c, DVM_EINVAL, "corrupt state (check iteration)");
        kc[b] = sp.k_check;
        ic[b] = sp.it_check;
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "set state");
    for (const Seg& sg : state_segments(c, (int)(h.iters & 1))) {
        if ((e = cudaMemcpyAsync(sg.p, in, sg.bytes, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
            return cuda_fail(c, e, "write state");
        in += sg.bytes;
        c->h2d_bytes += (long long)sg.bytes;
    }
    dvm_status s = run_finalize(c);
    if (s != DVM_OK) return s;
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "write state");
    c->iters = h.iters;
    c->last_err = h.last_err;
    c->k_check = kc;
    c->it_check = ic;
    return DVM_OK;
}

dvm_status dvm_info(const dvm_ctx* c, int64_t* iterations, int* nprob) {
    if (!c) return DVM_EINVAL;
    if (iterations) *iterations = c->iters;
    if (nprob) *nprob = c->nprob;
    return DVM_OK;
}

const char* dvm_last_error(const dvm_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

dvm_status dvm_profile_enable(dvm_ctx* c, int on) {
    if (!c) return DVM_EINVAL;
    c->profile = on != 0;
    return DVM_OK;
}

dvm_status dvm_profile_read(dvm_ctx* c, double* sweep_ms, int64_t* sweep_n, double* fin_ms, int64_t* fin_n) {
    if (!c) return DVM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "profile sync");
    if ((e = drain_graph_marks(c)) != cudaSuccess) return cuda_fail(c, e, "event timing");
    double ts = c->acc_sweep_ms, tf = c->acc_fin_ms;
    int64_t ns = c->acc_sweep_n, nf = c->acc_fin_n;
    c->acc_sweep_ms = c->acc_fin_ms = 0.0;
    c->acc_sweep_n = c->acc_fin_n = 0;
    for (size_t i = 0; i + 2 < c->ev_marks.size(); i += 3) {
        float a = 0.f, b = 0.f;
        if ((e = cudaEventElapsedTime(&a, c->ev_marks[i], c->ev_marks[i + 1])) != cudaSuccess ||
            (e = cudaEventElapsedTime(&b, c->ev_marks[i + 1], c->ev_marks[i + 2])) != cudaSuccess)
            return cuda_fail(c, e, "event timing");
        ts += a;
        tf += b;
        ++ns;
        ++nf;
    }
    c->ev_marks.clear();
    if (sweep_ms) *sweep_ms = ts;
    if (sweep_n) *sweep_n = ns;
    if (fin_ms) *fin_ms = tf;
    if (fin_n) *fin_n = nf;
    return DVM_OK;
}

dvm_status dvm_transfer_bytes(const dvm_ctx* c, int64_t* h2d, int64_t* d2h) {
    if (!c) return DVM_EINVAL;
    if (h2d) *h2d = c->h2d_bytes;
    if (d2h) *d2h = c->d2h_bytes;
    return DVM_OK;
}

void dvm_destroy(dvm_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    for (cudaEvent_t ev : c->ev_pool) cudaEventDestroy(ev);
    free_all(c);
    delete c;
}

// Test hooks (not part of the documented ABI): shorten the wait bound and withhold the progress
// flag of one work item so that the waits of the band above it expire.
dvm_status dvm_debug_set_wait(dvm_ctx* c, long long timeout_ns, int withhold_item) {
    if (!c || timeout_ns <= 0) return DVM_EINVAL;
    c->timeout_ns = timeout_ns;
    c->withhold_item = withhold_item;
    drop_graphs(c);     // the captured launches carry the old settings
    return DVM_OK;
}

}  // extern "C"
