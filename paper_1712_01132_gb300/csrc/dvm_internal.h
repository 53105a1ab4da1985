// dvm_internal.h -- structures shared by the host side of the library and its CUDA kernels.
//
// Terminology (all from arXiv:1712.01132):
//   octant/quadrant q : the 2^d groups of discrete velocities with equal component signs; every
//                       group is swept from its own upstream corner (Sec. 3.1, Fig. 1).  Bit j of
//                       q is set when s_j = sign(v_j) < 0.
//   lane               : one discrete velocity of a group; a group is padded to a multiple of 32
//                       lanes with zero-weight velocities.
//   band               : a block of consecutive x2 rows (2D) swept by one CTA along x1 in tiles of
//                       T1 columns; band b+1 follows band b one tile behind (wavefront over
//                       tiles, dependency-identical to the raster scan of the paper).
//   source form        : the kernels carry h' = h + x1 (the unit pressure jump of Eq. 7 becomes a
//                       plain periodic wrap plus a source term v1), which keeps the unknowns free of
//                       the O(1) ramp; outputs are converted back to the paper's variables.
#pragma once

#include <cstdint>

namespace dvm {

constexpr int kLaneConsts = 12;     // per-lane constants, see LaneConst
constexpr int kRecWords = 12;       // per-point record words (three 4-vectors)
constexpr long long kDefaultTimeoutNs = 2000000000LL;   // 2 s bound on every spin wait

// Per-lane constants of velocity lane l of group q of a problem, in the working precision:
//   [0] v1  [1] v2  [2] v3 (3D)  [3] |v1|/dx  [4] |v2|/dx  [5] |v3|/dx (3D)
//   [6] W   [7] W v1  [8] W v2  [9] W v3 (3D)  [10..] reciprocal denominators R[rsel], see below.
// 2D uses the layout of LaneConst2D.
// 2D layout: v1, v2, a1, a2, W, Wv1, Wv2, R0, R1, R2, R3, pad.
//   R[rsel] = 1 / (nu + C0(axis1) a1 + C0(axis2) a2) with C0 = 1 (first order) when bit j of rsel is
//   set and C0 = 1.5 (order 2) or 1 (order 1) otherwise.

template <typename T>
struct Prob2D {
    int n1, n2, N;
    int nbands;          // bands per quadrant (the largest count over the quadrants)
    int rows;            // rows per band (bands at subdomain ends may be shorter)
    int nslots;          // lagged x2 slots per quadrant: slot 0 is the domain face, slot s >= 1 the
                         // bottom of the s-th x2 subdomain (lagged-halo decomposition, Sec. 3.2)
    const int4* bands;   // [4][nbands] per quadrant, in oriented rows: {first row, rows, below,
                         // above}; below/above = s >= 0: lagged slot s; -1 - e: live band edge in
                         // ring slot e (two slots per subdomain, alternating between its bands)
    const int* slot_row; // [4][nslots] oriented row just above the layers a slot holds (slot 0: n2)
    int nxslots;         // lagged x1 slots per quadrant: slot 0 is the periodic x1 face, slot s >= 1
                         // the start of the s-th x1 subdomain (1 without x1 subdomains)
    int ntiles;          // x1 tiles per quadrant (largest count) when x1 subdomains are used
    int ntq[4];          // x1 tiles of each quadrant
    const int4* tiles;   // [4][ntiles] with x1 subdomains: {first oriented column, width, lagged
                         // slot the carry is read from before the tile or -1, slot written after it
                         // or -1}; NULL without x1 subdomains (uniform tiles)
    const int* xslot_col;  // [4][nxslots] oriented column just after the layers a slot holds
    int lateral;         // 0 specular, 1 periodic
    int order;           // 2 or 1
    double kn, nu, dx;
    double dinv[2];      // reciprocals of the Eq. 6 denominators per axis
    double dinvw[2];     // alpha dinv: the diffuse part of a wall value (Eq. 5; = dinv for alpha = 1)
    const uint16_t* code;   // [N] stencil cases, see kernels
    T* src;              // [N][4]  (nu rho', 2 nu u1 + 1, 2 nu u2, 0)
    T* E;                // [N][4]  wall terms per (axis j, upstream side u): index 2 j + u
    T* P;                // [4][3][N] moment partials per quadrant (rho', u1, u2)
    // Maxwell diffuse-specular walls (Eq. 5) with accommodation alpha < 1: the wall value of a
    // molecule leaving a wall is alpha rho_s + (1 - alpha) h(x_f, reflected v), the second part
    // from the previous iteration, kept per wall face (fluid point, axis j, side u with a solid
    // neighbour at x + (2u - 1) e_j).  spec = 1 - alpha (0: fully diffuse, the paper's setting).
    double spec;
    int nfaces;
    const int* face_id;  // [4][N] face of (axis j, side u) at a point, index 2 j + u, or -1
    const int* faces;    // [nfaces] point id * 4 + 2 j + u
    T* F;                // [2][nfaces][2][NL] h' of the molecules moving into each face (parity,
                         // face, sign bit of the other axis, velocity slot), written by the sweep
                         // moving into the face, read by the reflected quadrant next iteration
    T* gx1;              // [2][4][nxslots][n2][2][NL] lagged x1 layers (parity, quadrant, slot, row,
                         // layer, lane): the x1 ghosts (slot 0) and the x1 subdomain halos
    T* glat;             // [2][4][nslots][n1][2][NL] lagged x2 layers (parity, quadrant, slot, col,
                         // layer, lane): the x2 ghosts (slot 0) and the subdomain halos
    T* edge;             // [4][2 nslots][n1][2][NL] band-to-band edges (ring slots, see bands)
    int* prog;           // [4][nbands] tiles completed per band in this iteration
    const T* lanec;      // [4][NL][kLaneConsts]
    double* kpart;       // [nfinblocks] partial sums of u1 (FP64)
    double* kval;        // [3]: k, G_p, sum u1 of the last finalize
    int fin_block0;      // first finalize block of this problem
    int fin_nblocks;     // finalize blocks of this problem
    unsigned int* fin_counter;   // blocks of this problem done (last-block reduction)
};

struct SweepItem { int prob, quad, band, pad; };

template <typename T>
struct SweepArgs2D {
    const Prob2D<T>* prob;      // device array [nprob]
    const SweepItem* items;     // device array [nitems], ordered by band index
    int nitems;
    int NL;                     // lanes per quadrant (multiple of 32)
    int max_rows;               // rows per band used to size shared memory
    int parity;                 // ghost buffers: read [parity], write [parity ^ 1]
    int spec;                   // specular wall parts (Prob2D::spec > 0)
    int* ticket;                // work counter (zeroed before every launch)
    int* status;                // device error word (0 = ok)
    long long timeout_ns;
    int withhold_item;          // test hook: this item never publishes progress (-1 = none)
};

template <typename T>
struct FinArgs2D {
    const Prob2D<T>* prob;
    const int* blk_prob;        // [nblocks] problem of each block
    const int* blk_start;       // [nblocks] first point of each block
    int* status;
};

// 3D problem.  Octant q has bit j set when s_j < 0.  A pencil is R2 x R3 rows (x2 x x3) swept
// along x1 in tiles of T1 columns; the velocities of an octant may be split into groups (each
// group is an independent sweep with its own moment partials).
template <typename T>
struct Prob3D {
    int n1, n2, n3, N;
    int R2, R3, np2, np3;   // pencil rows and pencil counts
    int ngroups;            // velocity groups per octant
    int lateral, order;
    int bf16;               // 1: ghosts and pencil edges hold BF16 deviations from the x1 ramp
                            //    (h' - x1 of the point the value belongs to), 2 bytes each
    double kn, nu, dx;
    double dinv[3];
    double dinvw[3];        // alpha dinv (Eq. 5; = dinv for alpha = 1)
    const uint16_t* code;   // [N]
    T* src;                 // [N][4]  (nu rho', 2 nu u1 + 1, 2 nu u2, 2 nu u3)
    T* E;                   // [N][8]  wall terms, index 2 j + u (6 used)
    T* P;                   // [8][G][4][N] moment partials per octant and velocity group
    // temperature term of Eq. 2 (option; 3D): tau = (2/3) sum W |v|^2 h - rho (Eq. 4)
    int tau;                // 1: the source carries tau (|v|^2 - 3/2)
    double sw2;             // sum over the grid of W |v|^2 (3/2 for a rule exact on v^2)
    T* Pt;                  // [8][G][N] partials of sum W |v|^2 h' (with tau)
    T* srct;                // [N] nu tau of the last iteration, read by the sweep (with tau)
    // model moments of the linearised Shakhov (nx = 3) and ES-BGK (nx = 6) models (with tau): the
    // source adds xcoef sum_a m_a phi_a(v) with the point's moments m_a = sum W psi_a(v) h;
    // Shakhov: phi_j = psi_j = v_j (|v|^2 - 5/2) (the heat flux), xcoef = (4/5)(1 - Pr); ES:
    // phi = (v1^2, v2^2, v3^2, 2 v1 v2, 2 v1 v3, 2 v2 v3), psi_a = 2 (v_i v_j - delta_ij |v|^2 / 3)
    // (the traceless stress), xcoef = 1 - 1/Pr and the collision frequency Pr nu
    int nx;                 // 0 (BGK), 3 (Shakhov) or 6 (ES-BGK)
    double xcoef;
    double sx[6];           // sum over the grid of W psi_a: m'_a = m_a + x1 sx_a
    T* Px;                  // [8][G][nx][N] partials of sum W psi_a h'
    T* srcx;                // [N][8] nu xcoef m_a of the last iteration, read by the sweep
    // Maxwell walls with alpha < 1 (Eq. 5), as in Prob2D: spec = 1 - alpha; faces are (fluid
    // point, axis j, side u) with a solid neighbour at x + (2u - 1) e_j
    double spec;
    int nfaces;
    const int* face_id;     // [6][N] face of (axis j, side u) at a point, index 2 j + u, or -1
    const int* faces;       // [nfaces] point id * 8 + 2 j + u
    T* F;                   // [2][nfaces][4][NL] h' of the molecules moving into each face (parity,
                            // face, sign bits of the two other axes, velocity slot)
    // Lagged-halo subdomains (Sec. 3.2): ns_j = c_j blocks along axis j (1: none).  Slot s of a
    // ghost array holds the two layers upstream of oriented block s from the previous iteration
    // (slot 0: the domain's own ghost layers); the last pencil / tile of block s writes slot
    // (s + 1) mod ns_j for the next iteration.
    int ns1, ns2, ns3;
    T* gx1;                 // [2][8][ns1][n3 * n2][2][NL] x1 ghosts (parity, octant, slot, row (k, j), layer,
                            // lane); ghosts and edges are T, or BF16 when bf16 is set (element
                            // offsets are the same, the pointers are reinterpreted)
    T* gy;                  // [2][8][ns2][n3 * n1][2][NL] x2 ghosts (row (k, i))
    T* gz;                  // [2][8][ns3][n2 * n1][2][NL] x3 ghosts (row (j, i))
    T* ey;                  // [8][np3][2 ns2][R3][n1][2][NL] x2 edges between pencils: two ring slots per
                            // x2 block (slot 2 s + (local pencil index & 1))
    T* ez;                  // [8][np2][2 ns3][R2][n1][2][NL] x3 edges between pencils
    // Pencils per orientation (s_j < 0 or not): {first oriented row, rows, below, above}; below >= 0:
    // the pencil's upstream rows come from ghost slot `below` (previous iteration), below < 0: from
    // ring slot -1 - below, written by the pencil before it in this sweep; above likewise for the
    // rows it writes (>= 0: ghost slot of the next iteration).  x1 tiles per orientation: {first
    // oriented column, width, carry-in slot or -1, carry-out slot or -1}.  Read by the kernels only
    // with subdomains; without them the same values follow from p * R and t * T1.
    int nt1;                // x1 tiles of a pencil
    const int4* pen2;       // [2][np2]
    const int4* pen3;       // [2][np3]
    const int4* tiles1;     // [2][nt1]
    const int* slot_row2;   // [2][ns2] oriented row that follows the layers held in slot s
    const int* slot_row3;   // [2][ns3]
    const int* slot_col1;   // [2][ns1] oriented column that follows the layers held in slot s
    int* prog;              // [8][G][np3][np2] tiles completed
    const T* lanec;         // [8][NL][kLaneConsts3]
    double* kpart;
    double* kval;
    int fin_block0;
    int fin_nblocks;
    unsigned int* fin_counter;
};

// v1 v2 v3 a1 a2 a3 W Wv1 Wv2 Wv3 R[8] |v|^2-3/2 W|v|^2, then the model moments' phi_a [20..25]
// and W psi_a [26..31] (Shakhov, ES-BGK)
constexpr int kLaneConsts3 = 32;

struct SweepItem3 { int prob, oct, p2, p3, group, pad0, pad1, pad2; };

template <typename T>
struct SweepArgs3D {
    const Prob3D<T>* prob;
    const SweepItem3* items;
    int nitems;
    int NL;                     // lanes per octant (all groups)
    int GL;                     // lanes per velocity group (= 32 x warps per CTA)
    int T1;
    int maxR2, maxR3;
    int bf16;                   // ghosts and pencil edges stored as BF16 (see Prob3D::bf16)
    int sub;                    // lagged-halo subdomains: pencils and tiles from the Prob3D tables
    int tau;                    // temperature term (Prob3D::tau)
    int nx;                     // model moments (Prob3D::nx: Shakhov 3, ES-BGK 6; scalar kernel only)
    int spec;                   // specular wall parts (Prob3D::spec > 0)
    int parity;
    int* ticket;
    int* status;
    long long timeout_ns;
    int withhold_item;
};

template <typename T>
struct FinArgs3D {
    const Prob3D<T>* prob;
    const int* blk_prob;
    const int* blk_start;
    int* status;
};

// Stencil-case encoding of code[x] (2D uses axes 0,1; 3D axes 0..2):
//   bits 2*(2 j + u) .. +1 : case for axis j with upstream side u (u = 0: upstream is -e_j, i.e.
//   the sweep sign s_j > 0; u = 1: upstream is +e_j):
//     0 both upstream points fluid (second-order stencil of Eq. 9),
//     1 only the second one solid (first-order stencil on the fluid neighbour),
//     2 the first upstream point solid (first-order stencil on the wall value of that face)
//   bit 15 : solid voxel
constexpr uint16_t kSolidBit = 0x8000u;

}  // namespace dvm
