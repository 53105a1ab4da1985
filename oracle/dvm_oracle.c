/*
 * dvm_oracle.c -- plain, slow, FP64 CPU oracle of the discrete-velocity solver for steady,
 * pressure-driven rarefied flow through a voxelised porous medium (Ho, Zhu, Wu, Wang, Guo, Li,
 * Zhang, "A multi-level parallel solver for rarefied gas flows in porous media", arXiv:1712.01132).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call this file; only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark use it.  It shares no
 * code with the CUDA library.
 *
 * What it computes (one iteration of the source iteration of Sec. 3.1, steps (i)-(v)):
 *   (i)   for every discrete velocity v_k, a forward-substitution ("raster scan") sweep over the
 *         fluid points starting at the upstream corner of v_k's octant, solving the discretised
 *         linearised BGK equation (Eq. 10, the discretised form of Eq. 3) at each point with the
 *         upwind stencil of Eq. 9: (C0,C1,C2) = (1.5,-2,0.5)/dx by default, (1,-1,0)/dx when
 *         either upstream point of that stencil along the axis is solid;
 *   (ii)  boundary data for the next iteration: Maxwell diffuse-specular walls (Eq. 5; alpha = 1,
 *         fully diffuse, is the paper's setting and the default), the pressure jump periodic
 *         condition in x1 (Eq. 7), specular (Eq. 8) or periodic lateral faces;
 *   (iii) moments rho, u (Eq. 4) and wall densities (Eq. 6); the temperature tau of Eq. 4 and its
 *         source term tau (|v|^2 - 3/2) in Eq. 2 / Eq. 10 are dropped as in Sec. 4 unless the tau
 *         option is set (3D only: Eq. 2 and Eq. 4 are written for three velocity components);
 *         with the Shakhov option the source also carries the heat-flux term of the linearised
 *         S model, (4/5)(1 - Pr) q.v (|v|^2 - 5/2) with q = sum W v (|v|^2 - 5/2) h (an
 *         extension the paper names in Sec. 1 and Sec. 6 without writing it out; it needs tau);
 *         with the ES option (the ellipsoidal-statistical BGK model, named in the same places)
 *         the collision frequency becomes Pr nu and the source carries (1 - 1/Pr) sum_ij P_ij
 *         v_i v_j with the traceless stress P_ij = 2 sum W (v_i v_j - delta_ij |v|^2 / 3) h;
 *   (iv)  permeability k = (2/sqrt(pi)) Kn G_p (Eq. 11-12);
 *   (v)   Err of Eq. 15 is formed by the caller from the k history.
 * Moments, wall densities and all boundary (ghost) data used in a sweep are those of the previous
 * iteration; values at upstream fluid points inside the domain are those of the current sweep.
 *
 * Readings of points the paper leaves open (each is listed with its reason in the design notes):
 *   - Eq. 10 sums over the axis index j (Einstein convention).
 *   - First order is used along axis j iff one of the two upstream points of the second-order
 *     stencil, x - s_j e_j or x - 2 s_j e_j, is solid ("the upstream grid point is located on the
 *     boundary surfaces").  When x - s_j e_j is solid the upstream value is the wall value of that
 *     face; when only x - 2 s_j e_j is solid it is h(x - s_j e_j).  (Keeping the second-order
 *     stencil with a wall value at x - 2 s_j e_j makes the iteration diverge on two-voxel
 *     channels.)
 *   - A wall value belongs to a face (fluid point y, axis j, side sigma) whose solid neighbour is
 *     y + sigma e_j; its density (Eq. 6) is evaluated from h at the fluid point y.  A solid corner
 *     therefore carries one value per normal, as Sec. 3.1 requires.
 *   - Voxels are cell-centred; dx = 1/n1; the x1 period is 1, so the jump of Eq. 7 is 1 (the
 *     amplitude J is a parameter so linearity can be tested).  Specular faces mirror at the
 *     image face (ghost -1 <-> 0, -2 <-> 1).
 *   - The initial state is h = 0 in the bulk with boundary data obtained from it through the
 *     boundary conditions (so the first inflow ghost of Eq. 7 carries +J).
 *   - G_p is the mean of u1 over all points (solid = 0): the cross-section mean averaged over every
 *     x1 cross-section.
 *
 * Two algebraically identical formulations are provided: the paper's jump form (h carries the
 * -J x1 ramp, ghosts add the jump) and the source form h' = h + J x1 (plain periodic wrap, an
 * extra source term J v1, wall values shifted by J sigma dx on x1 faces).  Outputs are always in
 * jump-form variables.  An optional lagged-halo domain decomposition reproduces the paper's MPI
 * subdomain semantics (Sec. 3.2): upstream values that lie in another subdomain are taken from the
 * previous iteration.
 *
 * Determinism: velocities are swept in parallel in groups of a fixed size; the moments of a group
 * are then accumulated point by point in ascending velocity order, so results do not depend on
 * the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_GROUP 64

typedef struct {
    int dims;              /* 2 or 3 */
    int n[3];              /* n1, n2, n3 (n3 = 1 for dims = 2) */
    const uint8_t* solid;  /* [n3][n2][n1], x1 fastest; nonzero = solid */
    double kn;             /* Knudsen number, Eq. 1 */
    double jump;           /* pressure-jump amplitude J of Eq. 7 (1 for the paper's problem) */
    int nv;                /* number of discrete velocities */
    const double* v;       /* [nv][dims] */
    const double* w;       /* [nv] quadrature weights including the f_eq factor, sum = 1 */
    int order;             /* 2 (paper default) or 1 (first order everywhere) */
    int lateral;           /* 0 specular (Eq. 8), 1 periodic */
    int form;              /* 0 jump form (paper), 1 source form */
    int traversal;         /* 0 raster scan (paper), 1 wavefront over hyperplanes */
    int dec[3];            /* subdomain counts c1, c2, c3 of the lagged-halo decomposition */
    int tau;               /* 1: keep the temperature term of Eq. 2 (3D only); 0: drop it (Sec. 4) */
    double alpha;          /* tangential momentum accommodation coefficient of Eq. 5 (1: diffuse) */
    double shakhov_pr;     /* 0: BGK; > 0: linearised Shakhov model with this Prandtl number */
    double es_pr;          /* 0: BGK; > 0: linearised ES-BGK model with this Prandtl number */
} ora_cfg;

typedef struct {
    ora_cfg c;
    int d, n1, n2, n3, N, nv;
    uint8_t* solid;
    double *v, *w;
    double nu, dx, J;
    int* refl;             /* [3][nv] index of the velocity reflected in axis j */
    double dface[3][2];    /* Eq. 6 denominator per (axis, side) */
    double *rho, *u;       /* [N], [d][N] (stored in the working form's variables) */
    double* tau;           /* [N] temperature of Eq. 4 (the same in both forms), with the tau option */
    double sw2;            /* sum_k W_k |v_k|^2 (3/2 when the rule integrates v^2 exactly) */
    double* q;             /* [3][N] heat flux sum W v (|v|^2 - 5/2) h (paper's variables), Shakhov */
    double sq[3];          /* sum_k W_k v_jk (|v_k|^2 - 5/2) (0 on a symmetric grid, up to rounding) */
    double shk;            /* Shakhov coefficient (4/5)(1 - Pr), 0 for BGK */
    double* pi;            /* [6][N] traceless stress, components 11 22 33 12 13 23 (ES model) */
    double spi[6];         /* sum_k 2 W_k (v_i v_j - delta_ij |v|^2 / 3) (0 for an isotropic rule) */
    double esb;            /* ES coefficient 1 - 1/Pr, 0 for BGK */
    double* rhos;          /* [d][2][N] wall density of face (x, j, side) ; side 0: -1, 1: +1 */
    int area[3];           /* transverse face area per axis */
    double* lag[2];        /* [nv][d][2 layers][area] lagged ghost values, current / next */
    double* full[2];       /* [nv][N] lagged h, only with a decomposition */
    int* sub[3];           /* [n_j] subdomain index of each coordinate */
    int decomposed;
    int keep_full;         /* lagged h of every velocity kept: decomposition or alpha < 1 */
    double* H;             /* [ORA_GROUP][N] scratch */
    double* flux;          /* [n1] x1 face flux of the last iteration (jump-form variables) */
    uint8_t* facemask;     /* [N] bit (2 j + side) set when face (x, j, side) exists */
    long iter;
} ora;

static int sgnd(double a) { return a > 0 ? 1 : -1; }

static int idx3(const ora* o, const int c[3]) { return c[0] + o->n1 * (c[1] + o->n2 * c[2]); }

static int nax(const ora* o, int j) { return j == 0 ? o->n1 : (j == 1 ? o->n2 : o->n3); }

/* periodic on axis 0 always, on lateral axes when lateral == 1; specular mirror otherwise */
static int periodic_axis(const ora* o, int j) { return j == 0 || o->c.lateral == 1; }

/* map a coordinate that may lie outside [0, n) back into the domain */
static int base_coord(const ora* o, int j, int l) {
    int n = nax(o, j);
    if (l >= 0 && l < n) return l;
    if (periodic_axis(o, j)) { int r = l % n; return r < 0 ? r + n : r; }
    /* specular: mirror plane at the image face */
    if (l < 0) return -1 - l;
    return 2 * n - 1 - l;
}

/* x1 replica index of a coordinate (0 inside, -1 upstream of x1min, +1 downstream of x1max) */
static int replica(const ora* o, int j, int l) {
    if (j != 0) return 0;
    if (l < 0) return -1;
    if (l >= o->n1) return 1;
    return 0;
}

static int transverse(const ora* o, int j, const int c[3]) {
    if (j == 0) return c[1] + o->n2 * c[2];
    if (j == 1) return c[0] + o->n1 * c[2];
    return c[0] + o->n1 * c[1];
}

static int is_solid_at(const ora* o, int j, const int c[3], int l) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[j] = base_coord(o, j, l);
    return o->solid[idx3(o, cc)] != 0;
}

static double* lagp(const ora* o, double* lag, int k, int j, int layer) {
    return lag + (((size_t)k * o->d + j) * 2 + layer) * (size_t)o->area[j];
}

/* source-form shift of a wall value on a face (.., j, side s) of an x1 face */
static double wall_shift(const ora* o, int j, int side) {
    return (o->c.form == 1 && j == 0) ? o->J * side * o->dx : 0.0;
}

/* wall value seen at a solid point adjacent, along axis j, to the fluid point at coordinate
 * l (possibly outside the domain) of the line through c; side is the direction from the fluid
 * point to the solid. */
static double wall_value(const ora* o, int j, const int c[3], int l, int side) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[j] = base_coord(o, j, l);
    int sd = side;
    if (!periodic_axis(o, j) && (l < 0 || l >= nax(o, j))) sd = -side; /* mirrored face */
    double val = o->rhos[((size_t)j * 2 + (sd > 0)) * o->N + idx3(o, cc)];
    if (o->c.form == 0) val -= replica(o, j, l) * o->J;  /* gas in another x1 replica */
    return val + wall_shift(o, j, side);
}

/* upstream h value of velocity k at coordinate l along axis j of the line through c, which is a
 * fluid point: the current sweep inside the domain (same subdomain), lagged data otherwise. */
static double h_value(const ora* o, int k, int j, const int c[3], int l, const double* h,
                      const int xc[3]) {
    int n = nax(o, j);
    if (l >= 0 && l < n) {
        int cc[3] = {c[0], c[1], c[2]};
        cc[j] = l;
        int id = idx3(o, cc);
        if (o->decomposed && o->sub[j][l] != o->sub[j][xc[j]])
            return o->full[0][(size_t)k * o->N + id];
        return h[id];
    }
    int layer = (l < 0) ? (-1 - l) : (l - n);    /* 0 for distance 1, 1 for distance 2 */
    double val = lagp(o, o->lag[0], k, j, layer)[transverse(o, j, c)];
    if (o->c.form == 0) val -= replica(o, j, l) * o->J;
    return val;
}

static void point_update(const ora* o, int k, const int c[3], double* h) {
    int id = idx3(o, c);
    if (o->solid[id]) { h[id] = 0.0; return; }
    const double* vk = o->v + (size_t)k * o->d;
    double dot = 0.0;
    for (int j = 0; j < o->d; ++j) dot += o->u[(size_t)j * o->N + id] * vk[j];
    double num = o->nu * (o->rho[id] + 2.0 * dot);
    if (o->c.tau) {
        double vv = 0.0;
        for (int j = 0; j < o->d; ++j) vv += vk[j] * vk[j];
        num += o->nu * o->tau[id] * (vv - 1.5);
        if (o->c.shakhov_pr > 0.0) {
            double qv = 0.0;
            for (int j = 0; j < o->d; ++j) qv += o->q[(size_t)j * o->N + id] * vk[j];
            num += o->nu * o->shk * qv * (vv - 2.5);
        }
        if (o->c.es_pr > 0.0) {
            const double* P = o->pi;
            const size_t Nn = o->N;
            double pv = P[0 * Nn + id] * vk[0] * vk[0] + P[1 * Nn + id] * vk[1] * vk[1] + P[2 * Nn + id] * vk[2] * vk[2] +
                        2.0 * (P[3 * Nn + id] * vk[0] * vk[1] + P[4 * Nn + id] * vk[0] * vk[2] + P[5 * Nn + id] * vk[1] * vk[2]);
            num += o->nu * o->esb * pv;
        }
    }
    if (o->c.form == 1) num += o->J * vk[0];
    double den = o->nu;
    for (int j = 0; j < o->d; ++j) {
        int s = sgnd(vk[j]);
        double av = fabs(vk[j]);
        int l0 = c[j];
        int l1 = l0 - s, l2 = l0 - 2 * s;
        if (is_solid_at(o, j, c, l1)) {
            /* first-order stencil, upstream value = wall value of face (x, j, -s): Eq. 5, the
             * diffuse part alpha rho_s plus, for alpha < 1, the specular part (1 - alpha)
             * h(v - 2 n (v.n)) of the molecules reaching the face, taken (like rho_s) at the
             * fluid point of the face and from the previous iteration, with the same source-form
             * shift */
            double C0 = 1.0 / o->dx, C1 = -1.0 / o->dx;
            double U1 = wall_value(o, j, c, l0, -s);
            if (o->c.alpha < 1.0) {
                double hr = o->full[0][(size_t)o->refl[j * o->nv + k] * o->N + id];
                U1 = o->c.alpha * U1 + (1.0 - o->c.alpha) * (hr + wall_shift(o, j, -s));
            }
            num -= av * C1 * U1;
            den += av * C0;
        } else {
            double U1 = h_value(o, k, j, c, l1, h, c);
            if (o->c.order == 1 || is_solid_at(o, j, c, l2)) {
                /* first order: everywhere, or because the second upstream point of the
                 * second-order stencil lies in the solid */
                double C0 = 1.0 / o->dx, C1 = -1.0 / o->dx;
                num -= av * C1 * U1;
                den += av * C0;
            } else {
                double C0 = 1.5 / o->dx, C1 = -2.0 / o->dx, C2 = 0.5 / o->dx;
                double U2 = h_value(o, k, j, c, l2, h, c);
                num -= av * (C1 * U1 + C2 * U2);
                den += av * C0;
            }
        }
    }
    h[id] = num / den;
}

static void sweep(const ora* o, int k, double* h) {
    const double* vk = o->v + (size_t)k * o->d;
    int s[3] = {1, 1, 1};
    for (int j = 0; j < o->d; ++j) s[j] = sgnd(vk[j]);
    int n[3] = {o->n1, o->n2, o->n3};
    if (o->c.traversal == 0) {
        /* raster scan from the upstream corner, x1 fastest (Sec. 3.1, Fig. 1) */
        for (int l3 = 0; l3 < n[2]; ++l3)
            for (int l2 = 0; l2 < n[1]; ++l2)
                for (int l1 = 0; l1 < n[0]; ++l1) {
                    int c[3] = {s[0] > 0 ? l1 : n[0] - 1 - l1, s[1] > 0 ? l2 : n[1] - 1 - l2,
                                s[2] > 0 ? l3 : n[2] - 1 - l3};
                    point_update(o, k, c, h);
                }
    } else {
        /* hyperplanes l1 + l2 + l3 = const in octant-oriented coordinates */
        int dmax = n[0] + n[1] + n[2] - 3;
        for (int ds = 0; ds <= dmax; ++ds)
            for (int l3 = 0; l3 < n[2]; ++l3)
                for (int l2 = 0; l2 < n[1]; ++l2) {
                    int l1 = ds - l2 - l3;
                    if (l1 < 0 || l1 >= n[0]) continue;
                    int c[3] = {s[0] > 0 ? l1 : n[0] - 1 - l1, s[1] > 0 ? l2 : n[1] - 1 - l2,
                                s[2] > 0 ? l3 : n[2] - 1 - l3};
                    point_update(o, k, c, h);
                }
    }
}

/* Step (ii) for velocity k: record the h values that the next iteration reads as ghost data.
 * The reader of axis j is k itself (periodic) or its reflection (specular); it reads, at its
 * upstream face, layers at distance 1 and 2 whose in-domain images are stored here. */
static void capture_ghosts(const ora* o, int k, const double* h) {
    for (int j = 0; j < o->d; ++j) {
        int r = periodic_axis(o, j) ? k : o->refl[j * o->nv + k];
        int sr = sgnd(o->v[(size_t)r * o->d + j]);
        int n = nax(o, j);
        for (int layer = 0; layer < 2; ++layer) {
            int l = (sr > 0) ? (-1 - layer) : (n + layer);   /* reader's ghost coordinate */
            int lb = base_coord(o, j, l);
            double* dst = lagp(o, o->lag[1], r, j, layer);
            int c[3];
            int nt[3] = {o->n1, o->n2, o->n3};
            nt[j] = 1;
            for (c[2] = 0; c[2] < nt[2]; ++c[2])
                for (c[1] = 0; c[1] < nt[1]; ++c[1])
                    for (c[0] = 0; c[0] < nt[0]; ++c[0]) {
                        int cc[3] = {c[0], c[1], c[2]};
                        cc[j] = lb;
                        int id = idx3(o, cc);
                        dst[transverse(o, j, cc)] = o->solid[id] ? 0.0 : h[id];
                    }
        }
    }
}

static void init_state(ora* o) {
    /* h = 0 (jump form) everywhere; in the source form h' = J x1 */
    size_t N = o->N;
    memset(o->u, 0, sizeof(double) * N * o->d);
    memset(o->tau, 0, sizeof(double) * N);   /* tau of h = 0 */
    memset(o->q, 0, sizeof(double) * 3 * N);  /* heat flux of h = 0 */
    memset(o->pi, 0, sizeof(double) * 6 * N); /* stress of h = 0 */
    for (int id = 0; id < o->N; ++id) {
        int i1 = id % o->n1;
        double x1 = (o->c.form == 1) ? o->J * i1 * o->dx : 0.0;
        o->rho[id] = o->solid[id] ? 0.0 : x1;
        for (int j = 0; j < o->d; ++j)
            for (int sd = 0; sd < 2; ++sd) o->rhos[((size_t)j * 2 + sd) * N + id] = 0.0;
    }
    /* wall densities of existing faces: derived from h = 0, i.e. 0 (jump) / J x1(y) (source) */
    for (int id = 0; id < o->N; ++id)
        for (int j = 0; j < o->d; ++j)
            for (int sd = 0; sd < 2; ++sd)
                if (o->facemask[id] >> (2 * j + sd) & 1)
                    o->rhos[((size_t)j * 2 + sd) * N + id] = (o->c.form == 1) ? o->J * (id % o->n1) * o->dx : 0.0;
    for (int k = 0; k < o->nv; ++k)
        for (int j = 0; j < o->d; ++j)
            for (int layer = 0; layer < 2; ++layer) {
                double* dst = lagp(o, o->lag[0], k, j, layer);
                int n = nax(o, j);
                int sr = sgnd(o->v[(size_t)k * o->d + j]);
                int l = (sr > 0) ? (-1 - layer) : (n + layer);
                int lb = base_coord(o, j, l);
                int nt[3] = {o->n1, o->n2, o->n3};
                nt[j] = 1;
                int c[3];
                for (c[2] = 0; c[2] < nt[2]; ++c[2])
                    for (c[1] = 0; c[1] < nt[1]; ++c[1])
                        for (c[0] = 0; c[0] < nt[0]; ++c[0]) {
                            int cc[3] = {c[0], c[1], c[2]};
                            cc[j] = lb;
                            double x1 = (o->c.form == 1) ? o->J * cc[0] * o->dx : 0.0;
                            dst[transverse(o, j, cc)] = x1;
                        }
            }
    if (o->keep_full) {
        for (int k = 0; k < o->nv; ++k)
            for (int id = 0; id < o->N; ++id)
                o->full[0][(size_t)k * N + id] =
                    (o->c.form == 1 && !o->solid[id]) ? o->J * (id % o->n1) * o->dx : 0.0;
    }
    o->iter = 0;
}

ora* ora_create(const ora_cfg* cfg) {
    if (!cfg || (cfg->dims != 2 && cfg->dims != 3) || cfg->nv <= 0 || cfg->kn <= 0) return NULL;
    if (!(cfg->alpha >= 0.0 && cfg->alpha <= 1.0)) return NULL;
    if (cfg->tau && cfg->dims != 3) return NULL;
    if (cfg->shakhov_pr < 0.0 || (cfg->shakhov_pr > 0.0 && !cfg->tau)) return NULL;
    if (cfg->es_pr < 0.0 || (cfg->es_pr > 0.0 && (!cfg->tau || cfg->shakhov_pr > 0.0))) return NULL;
    ora* o = (ora*)calloc(1, sizeof(ora));
    o->c = *cfg;
    o->d = cfg->dims;
    o->n1 = cfg->n[0];
    o->n2 = cfg->n[1];
    o->n3 = cfg->dims == 3 ? cfg->n[2] : 1;
    o->N = o->n1 * o->n2 * o->n3;
    o->nv = cfg->nv;
    o->solid = (uint8_t*)malloc(o->N);
    memcpy(o->solid, cfg->solid, o->N);
    o->v = (double*)malloc(sizeof(double) * o->nv * o->d);
    memcpy(o->v, cfg->v, sizeof(double) * o->nv * o->d);
    o->w = (double*)malloc(sizeof(double) * o->nv);
    memcpy(o->w, cfg->w, sizeof(double) * o->nv);
    o->c.solid = o->solid;
    o->c.v = o->v;
    o->c.w = o->w;
    o->nu = sqrt(M_PI) / (2.0 * cfg->kn);     /* collision frequency of Eq. 3 */
    /* ES model: the stress relaxes at nu_ES (1 - (1 - 1/Pr)) = nu_ES / Pr, so the same viscosity
     * (the Kn of Eq. 1) needs the collision frequency nu_ES = Pr nu */
    if (cfg->es_pr > 0.0) o->nu *= cfg->es_pr;
    o->esb = cfg->es_pr > 0.0 ? 1.0 - 1.0 / cfg->es_pr : 0.0;
    o->dx = 1.0 / o->n1;                       /* L = x1 extent (Sec. 2.1) */
    o->J = cfg->jump;
    o->sw2 = 0.0;
    for (int k = 0; k < o->nv; ++k)
        for (int j = 0; j < o->d; ++j) o->sw2 += o->w[k] * o->v[(size_t)k * o->d + j] * o->v[(size_t)k * o->d + j];
    /* S model: the heat-flux moment of the extra term, sum W v_i (|v|^2 - 5/2) A q.v (|v|^2 - 5/2),
     * is A (5/4) q_i for an exact rule, so q relaxes at the rate nu (1 - 5 A / 4) = Pr nu when
     * A = (4/5)(1 - Pr) */
    o->shk = cfg->shakhov_pr > 0.0 ? 0.8 * (1.0 - cfg->shakhov_pr) : 0.0;
    for (int j = 0; j < 3; ++j) o->sq[j] = 0.0;
    for (int k = 0; k < o->nv; ++k) {
        double vv = 0.0;
        for (int j = 0; j < o->d; ++j) vv += o->v[(size_t)k * o->d + j] * o->v[(size_t)k * o->d + j];
        for (int j = 0; j < o->d; ++j) o->sq[j] += o->w[k] * o->v[(size_t)k * o->d + j] * (vv - 2.5);
    }
    for (int a = 0; a < 6; ++a) o->spi[a] = 0.0;
    if (o->d == 3)
        for (int k = 0; k < o->nv; ++k) {
            const double* vk = o->v + (size_t)k * 3;
            const double vv = vk[0] * vk[0] + vk[1] * vk[1] + vk[2] * vk[2];
            const double wk = o->w[k];
            o->spi[0] += 2.0 * wk * (vk[0] * vk[0] - vv / 3.0);
            o->spi[1] += 2.0 * wk * (vk[1] * vk[1] - vv / 3.0);
            o->spi[2] += 2.0 * wk * (vk[2] * vk[2] - vv / 3.0);
            o->spi[3] += 2.0 * wk * vk[0] * vk[1];
            o->spi[4] += 2.0 * wk * vk[0] * vk[2];
            o->spi[5] += 2.0 * wk * vk[1] * vk[2];
        }
    o->refl = (int*)malloc(sizeof(int) * 3 * o->nv);
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < o->nv; ++k) {
            o->refl[j * o->nv + k] = -1;
            if (j >= o->d) continue;
            for (int q = 0; q < o->nv; ++q) {
                int ok = 1;
                for (int a = 0; a < o->d; ++a) {
                    double want = (a == j) ? -o->v[(size_t)k * o->d + a] : o->v[(size_t)k * o->d + a];
                    if (o->v[(size_t)q * o->d + a] != want) { ok = 0; break; }
                }
                if (ok) { o->refl[j * o->nv + k] = q; break; }
            }
        }
    for (int j = 0; j < o->d; ++j)
        for (int sd = 0; sd < 2; ++sd) {
            int side = sd ? 1 : -1;
            double D = 0.0;
            /* Eq. 6 denominator: velocities leaving the wall, sigma v_j < 0 */
            for (int k = 0; k < o->nv; ++k) {
                double vj = o->v[(size_t)k * o->d + j];
                if (side * vj < 0) D += o->w[k] * fabs(vj);
            }
            o->dface[j][sd] = D;
        }
    o->rho = (double*)calloc(o->N, sizeof(double));
    o->u = (double*)calloc((size_t)o->N * o->d, sizeof(double));
    o->tau = (double*)calloc(o->N, sizeof(double));
    o->q = (double*)calloc((size_t)3 * o->N, sizeof(double));
    o->pi = (double*)calloc((size_t)6 * o->N, sizeof(double));
    o->rhos = (double*)calloc((size_t)o->N * o->d * 2, sizeof(double));
    o->area[0] = o->n2 * o->n3;
    o->area[1] = o->n1 * o->n3;
    o->area[2] = o->n1 * o->n2;
    size_t lagsz = 0;
    for (int j = 0; j < o->d; ++j) lagsz += (size_t)2 * o->area[j];
    /* per velocity the layout is [d][2][area_j]; use the max area for simple indexing */
    int amax = o->area[0];
    for (int j = 1; j < o->d; ++j) if (o->area[j] > amax) amax = o->area[j];
    for (int j = 0; j < o->d; ++j) o->area[j] = amax;
    lagsz = (size_t)o->nv * o->d * 2 * amax;
    o->lag[0] = (double*)calloc(lagsz, sizeof(double));
    o->lag[1] = (double*)calloc(lagsz, sizeof(double));
    o->decomposed = 0;
    for (int j = 0; j < 3; ++j) {
        int cj = cfg->dec[j] > 0 ? cfg->dec[j] : 1;
        if (j < o->d && cj > 1) o->decomposed = 1;
        int n = nax(o, j);
        o->sub[j] = (int*)malloc(sizeof(int) * n);
        for (int l = 0; l < n; ++l) o->sub[j][l] = (j < o->d) ? (int)(((long)l * cj) / n) : 0;
    }
    o->keep_full = o->decomposed || cfg->alpha < 1.0;
    if (o->keep_full) {
        o->full[0] = (double*)calloc((size_t)o->nv * o->N, sizeof(double));
        o->full[1] = (double*)calloc((size_t)o->nv * o->N, sizeof(double));
    }
    o->facemask = (uint8_t*)calloc(o->N, 1);
    for (int id = 0; id < o->N; ++id) {
        if (o->solid[id]) continue;
        int c[3] = {id % o->n1, (id / o->n1) % o->n2, id / (o->n1 * o->n2)};
        for (int j = 0; j < o->d; ++j)
            for (int sd = 0; sd < 2; ++sd)
                if (is_solid_at(o, j, c, c[j] + (sd ? 1 : -1))) o->facemask[id] |= (uint8_t)(1u << (2 * j + sd));
    }
    o->H = (double*)malloc(sizeof(double) * ORA_GROUP * (size_t)o->N);
    o->flux = (double*)calloc(o->n1, sizeof(double));
    init_state(o);
    return o;
}

void ora_destroy(ora* o) {
    if (!o) return;
    free(o->solid); free(o->v); free(o->w); free(o->refl);
    free(o->rho); free(o->u); free(o->tau); free(o->q); free(o->pi); free(o->rhos);
    free(o->lag[0]); free(o->lag[1]);
    free(o->full[0]); free(o->full[1]);
    for (int j = 0; j < 3; ++j) free(o->sub[j]);
    free(o->H); free(o->flux); free(o->facemask);
    free(o);
}

/* upwind x1 face value, in jump-form variables, of velocity k on the face between coordinates
 * i and i+1 of the x1 line through c (i = n1 - 1 is the periodic face) */
static double upwind_face_value(const ora* o, int k, const int c[3], int i, const double* h) {
    int s = sgnd(o->v[(size_t)k * o->d]);
    int lup = (s > 0) ? i : i + 1;      /* upwind coordinate (continued) */
    int loth = (s > 0) ? i + 1 : i;     /* the other side of the face */
    int cu[3] = {base_coord(o, 0, lup), c[1], c[2]};
    int co[3] = {base_coord(o, 0, loth), c[1], c[2]};
    double val;
    if (o->solid[idx3(o, cu)]) {
        if (o->solid[idx3(o, co)]) return 0.0;       /* no gas on either side */
        val = wall_value(o, 0, c, loth, -s);        /* wall face attached to the fluid side */
    } else {
        val = h[idx3(o, cu)];
        if (o->c.form == 0) val -= replica(o, 0, lup) * o->J;
    }
    if (o->c.form == 1) val -= o->J * lup * o->dx;  /* h = h' - J x1, x1 continued */
    return val;
}

/* One iteration (steps i-iii).  Returns 0. */
/* tau = (2/3) sum W |v|^2 h - rho (Eq. 4) at every fluid point from e = sum W |v|^2 h and the new
 * rho, both in the working variables.  In the source form h' = h + J x1, so
 * tau = (2/3) e' - rho' + J x1 (1 - (2/3) sum W |v|^2): the paper's tau in either form. */
static void update_tau(ora* o, const double* e) {
    for (int id = 0; id < o->N; ++id) {
        if (o->solid[id]) { o->tau[id] = 0.0; continue; }
        double x1 = (o->c.form == 1) ? o->J * (id % o->n1) * o->dx : 0.0;
        o->tau[id] = 2.0 / 3.0 * e[id] - o->rho[id] + x1 * (1.0 - 2.0 / 3.0 * o->sw2);
    }
}

/* q_j = sum W v_j (|v|^2 - 5/2) h from the working-variable sum qn; in the source form
 * h' = h + J x1, so q_j = qn_j - J x1 sq_j: the paper's q in either form. */
static void update_q(ora* o, const double* qn) {
    for (int j = 0; j < o->d; ++j)
        for (int id = 0; id < o->N; ++id) {
            double x1 = (o->c.form == 1) ? o->J * (id % o->n1) * o->dx : 0.0;
            o->q[(size_t)j * o->N + id] = o->solid[id] ? 0.0 : qn[(size_t)j * o->N + id] - x1 * o->sq[j];
        }
}

/* the six stress components 2 W (v_i v_j - delta_ij |v|^2 / 3) h of velocity k, added to pn at id */
static void add_stress(const ora* o, int k, double wh, double* pn, size_t id) {
    const double* vk = o->v + (size_t)k * 3;
    const double vv = vk[0] * vk[0] + vk[1] * vk[1] + vk[2] * vk[2];
    const size_t N = o->N;
    pn[0 * N + id] += 2.0 * wh * (vk[0] * vk[0] - vv / 3.0);
    pn[1 * N + id] += 2.0 * wh * (vk[1] * vk[1] - vv / 3.0);
    pn[2 * N + id] += 2.0 * wh * (vk[2] * vk[2] - vv / 3.0);
    pn[3 * N + id] += 2.0 * wh * vk[0] * vk[1];
    pn[4 * N + id] += 2.0 * wh * vk[0] * vk[2];
    pn[5 * N + id] += 2.0 * wh * vk[1] * vk[2];
}

/* P_ij from the working-variable sums pn; in the source form h' = h + J x1, so P = pn - J x1 spi:
 * the paper's stress in either form. */
static void update_pi(ora* o, const double* pn) {
    for (int a = 0; a < 6; ++a)
        for (int id = 0; id < o->N; ++id) {
            double x1 = (o->c.form == 1) ? o->J * (id % o->n1) * o->dx : 0.0;
            o->pi[(size_t)a * o->N + id] = o->solid[id] ? 0.0 : pn[(size_t)a * o->N + id] - x1 * o->spi[a];
        }
}

static void iterate_once(ora* o) {
    const size_t N = o->N;
    const int d = o->d;
    double* rho_n = (double*)calloc(N, sizeof(double));
    double* u_n = (double*)calloc(N * d, sizeof(double));
    double* num_n = (double*)calloc(N * d * 2, sizeof(double));
    double* e_n = (double*)calloc(N, sizeof(double));          /* sum W |v|^2 h (tau option) */
    double* q_n = (double*)calloc(N * 3, sizeof(double));      /* heat-flux sums (Shakhov) */
    double* p_n = (double*)calloc(N * 6, sizeof(double));      /* stress sums (ES) */
    memset(o->flux, 0, sizeof(double) * o->n1);
    for (int g0 = 0; g0 < o->nv; g0 += ORA_GROUP) {
        int gn = o->nv - g0 < ORA_GROUP ? o->nv - g0 : ORA_GROUP;
#pragma omp parallel for schedule(dynamic, 1)
        for (int kk = 0; kk < gn; ++kk) {
            int k = g0 + kk;
            double* h = o->H + (size_t)kk * N;
            sweep(o, k, h);
            capture_ghosts(o, k, h);
            if (o->keep_full) memcpy(o->full[1] + (size_t)k * N, h, sizeof(double) * N);
        }
        /* step (iii): quadrature, accumulated in ascending velocity order at every point */
#pragma omp parallel for schedule(static)
        for (long id = 0; id < (long)N; ++id) {
            if (o->solid[id]) continue;
            for (int kk = 0; kk < gn; ++kk) {
                int k = g0 + kk;
                double hk = o->H[(size_t)kk * N + id];
                double wk = o->w[k];
                rho_n[id] += wk * hk;
                if (o->c.tau) {
                    double vv = 0.0;
                    for (int j = 0; j < d; ++j) vv += o->v[(size_t)k * d + j] * o->v[(size_t)k * d + j];
                    e_n[id] += wk * vv * hk;
                    if (o->c.shakhov_pr > 0.0)
                        for (int j = 0; j < d; ++j) q_n[(size_t)j * N + id] += wk * o->v[(size_t)k * d + j] * (vv - 2.5) * hk;
                    if (o->c.es_pr > 0.0) add_stress(o, k, wk * hk, p_n, (size_t)id);
                }
                for (int j = 0; j < d; ++j) {
                    double vj = o->v[(size_t)k * d + j];
                    u_n[(size_t)j * N + id] += wk * vj * hk;
                }
                for (int j = 0; j < d; ++j)
                    for (int sd = 0; sd < 2; ++sd) {
                        int side = sd ? 1 : -1;
                        double vj = o->v[(size_t)k * d + j];
                        if (side * vj > 0 && (o->facemask[id] >> (2 * j + sd) & 1))
                            num_n[((size_t)j * 2 + sd) * N + id] += wk * fabs(vj) * hk;
                    }
            }
        }
        /* x1 face fluxes (diagnostic): face i is between i and i+1 (i = n1-1 wraps) */
#pragma omp parallel for schedule(static)
        for (int i = 0; i < o->n1; ++i) {
            double acc = 0.0;
            int c[3];
            for (c[2] = 0; c[2] < o->n3; ++c[2])
                for (c[1] = 0; c[1] < o->n2; ++c[1])
                    for (int kk = 0; kk < gn; ++kk) {
                        int k = g0 + kk;
                        c[0] = i;
                        acc += o->w[k] * o->v[(size_t)k * d] *
                               upwind_face_value(o, k, c, i, o->H + (size_t)kk * N);
                    }
            o->flux[i] += acc;
        }
    }
    /* wall densities, Eq. 6 */
    for (int j = 0; j < d; ++j)
        for (int sd = 0; sd < 2; ++sd)
            for (size_t id = 0; id < N; ++id)
                o->rhos[((size_t)j * 2 + sd) * N + id] = num_n[((size_t)j * 2 + sd) * N + id] / o->dface[j][sd];
    memcpy(o->rho, rho_n, sizeof(double) * N);
    memcpy(o->u, u_n, sizeof(double) * N * d);
    if (o->c.tau) update_tau(o, e_n);
    if (o->c.shakhov_pr > 0.0) update_q(o, q_n);
    if (o->c.es_pr > 0.0) update_pi(o, p_n);
    double* t = o->lag[0]; o->lag[0] = o->lag[1]; o->lag[1] = t;
    if (o->keep_full) { t = o->full[0]; o->full[0] = o->full[1]; o->full[1] = t; }
    free(rho_n); free(u_n); free(num_n); free(e_n); free(q_n); free(p_n);
    o->iter++;
}

/* Run n iterations.  k_out (may be NULL) receives k after each iteration. */
int ora_iterate(ora* o, int n, double* k_out, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int it = 0; it < n; ++it) {
        iterate_once(o);
        if (k_out) {
            double gp = 0.0;
            for (int id = 0; id < o->N; ++id) gp += o->u[id];
            gp /= (double)o->N;
            k_out[it] = 2.0 / sqrt(M_PI) * o->c.kn * gp;   /* Eq. 11 */
        }
    }
    return 0;
}

long ora_iter(const ora* o) { return o->iter; }

/* Moments in jump-form variables: rho [N], u [d][N]. */
void ora_get_moments(const ora* o, double* rho, double* u) {
    for (int id = 0; id < o->N; ++id) {
        double x1 = (o->c.form == 1 && !o->solid[id]) ? o->J * (id % o->n1) * o->dx : 0.0;
        rho[id] = o->rho[id] - x1;
    }
    memcpy(u, o->u, sizeof(double) * o->N * o->d);
}

/* Wall densities [d][2][N] in jump-form variables (0 where there is no face). */
void ora_get_wall(const ora* o, double* rhos) {
    for (int j = 0; j < o->d; ++j)
        for (int sd = 0; sd < 2; ++sd)
            for (int id = 0; id < o->N; ++id) {
                double v = o->rhos[((size_t)j * 2 + sd) * o->N + id];
                if (o->c.form == 1 && (o->facemask[id] >> (2 * j + sd) & 1)) v -= o->J * (id % o->n1) * o->dx;
                rhos[((size_t)j * 2 + sd) * o->N + id] = v;
            }
}

void ora_get_flux(const ora* o, double* flux) { memcpy(flux, o->flux, sizeof(double) * o->n1); }

/* Temperature tau of Eq. 4 [N] (zero without the tau option and at solid points). */
void ora_get_tau(const ora* o, double* tau) { memcpy(tau, o->tau, sizeof(double) * o->N); }

/* Heat flux q [d][N] of the Shakhov option (zero otherwise and at solid points). */
void ora_get_q(const ora* o, double* q) { memcpy(q, o->q, sizeof(double) * o->N * o->d); }

/* Traceless stress [6][N] (11 22 33 12 13 23) of the ES option (zero otherwise and at solid points). */
void ora_get_pi(const ora* o, double* p) { memcpy(p, o->pi, sizeof(double) * o->N * 6); }

/* Overwrite the state with a uniform value c in the working variables (jump = 0 tests). */
void ora_set_uniform(ora* o, double c) {
    for (int id = 0; id < o->N; ++id) {
        o->rho[id] = o->solid[id] ? 0.0 : c;
        for (int j = 0; j < o->d; ++j) o->u[(size_t)j * o->N + id] = 0.0;
        for (int j = 0; j < o->d; ++j)
            for (int sd = 0; sd < 2; ++sd)
                o->rhos[((size_t)j * 2 + sd) * o->N + id] = (o->facemask[id] >> (2 * j + sd) & 1) ? c : 0.0;
    }
    for (int id = 0; id < o->N; ++id) o->tau[id] = o->solid[id] ? 0.0 : c * (2.0 / 3.0 * o->sw2 - 1.0);
    if (o->c.shakhov_pr > 0.0)
        for (int j = 0; j < o->d; ++j)
            for (int id = 0; id < o->N; ++id) o->q[(size_t)j * o->N + id] = o->solid[id] ? 0.0 : c * o->sq[j];
    if (o->c.es_pr > 0.0)
        for (int a = 0; a < 6; ++a)
            for (int id = 0; id < o->N; ++id) o->pi[(size_t)a * o->N + id] = o->solid[id] ? 0.0 : c * o->spi[a];
    size_t lagsz = (size_t)o->nv * o->d * 2 * o->area[0];
    for (size_t i = 0; i < lagsz; ++i) o->lag[0][i] = c;
    if (o->keep_full)
        for (size_t i = 0; i < (size_t)o->nv * o->N; ++i) o->full[0][i] = c;
}

/* Warm start (the paper always starts from h = 0; this is an extension whose fixed point is the
 * same): replace the state by the one an iteration leaves when it has produced
 *     h0(x, v_k) = rho0(x) + 2 u0(x) . v_k     (jump-form variables; + J x1 in the source form)
 * at every fluid point, i.e. the source term of Eq. 10 evaluated at (rho0, u0).  Exactly the
 * post-sweep steps of an iteration are applied to h0: the quadrature of Eq. 4 (ascending velocity
 * order at every point), the wall numerators and densities of Eq. 6 at the faces, and the ghost
 * capture of step (ii) for the boundary conditions of Eq. 7 and Eq. 8.  rho0 is [N], u0 [d][N];
 * values at solid points are ignored.  The iteration counter is not changed. */
void ora_set_initial(ora* o, const double* rho0, const double* u0) {
    const size_t N = o->N;
    const int d = o->d;
    double* h = (double*)malloc(sizeof(double) * N);
    double* rho_n = (double*)calloc(N, sizeof(double));
    double* u_n = (double*)calloc(N * d, sizeof(double));
    double* num_n = (double*)calloc(N * d * 2, sizeof(double));
    double* e_n = (double*)calloc(N, sizeof(double));
    double* q_n = (double*)calloc(N * 3, sizeof(double));
    double* p_n = (double*)calloc(N * 6, sizeof(double));
    for (int k = 0; k < o->nv; ++k) {
        const double* vk = o->v + (size_t)k * d;
        double vv = 0.0;
        for (int j = 0; j < d; ++j) vv += vk[j] * vk[j];
        for (size_t id = 0; id < N; ++id) {
            if (o->solid[id]) { h[id] = 0.0; continue; }
            double dot = 0.0;
            for (int j = 0; j < d; ++j) dot += u0[(size_t)j * N + id] * vk[j];
            double x1 = (o->c.form == 1) ? o->J * (double)(id % o->n1) * o->dx : 0.0;
            h[id] = rho0[id] + 2.0 * dot + x1;
        }
        capture_ghosts(o, k, h);
        if (o->keep_full) memcpy(o->full[1] + (size_t)k * N, h, sizeof(double) * N);
        for (size_t id = 0; id < N; ++id) {
            if (o->solid[id]) continue;
            double wk = o->w[k];
            rho_n[id] += wk * h[id];
            e_n[id] += wk * vv * h[id];
            for (int j = 0; j < d; ++j) q_n[(size_t)j * N + id] += wk * vk[j] * (vv - 2.5) * h[id];
            if (o->c.es_pr > 0.0) add_stress(o, k, wk * h[id], p_n, id);
            for (int j = 0; j < d; ++j) u_n[(size_t)j * N + id] += wk * vk[j] * h[id];
            for (int j = 0; j < d; ++j)
                for (int sd = 0; sd < 2; ++sd) {
                    int side = sd ? 1 : -1;
                    if (side * vk[j] > 0 && (o->facemask[id] >> (2 * j + sd) & 1))
                        num_n[((size_t)j * 2 + sd) * N + id] += wk * fabs(vk[j]) * h[id];
                }
        }
    }
    for (int j = 0; j < d; ++j)
        for (int sd = 0; sd < 2; ++sd)
            for (size_t id = 0; id < N; ++id)
                o->rhos[((size_t)j * 2 + sd) * N + id] = num_n[((size_t)j * 2 + sd) * N + id] / o->dface[j][sd];
    memcpy(o->rho, rho_n, sizeof(double) * N);
    memcpy(o->u, u_n, sizeof(double) * N * d);
    if (o->c.tau) update_tau(o, e_n);
    if (o->c.shakhov_pr > 0.0) update_q(o, q_n);
    if (o->c.es_pr > 0.0) update_pi(o, p_n);
    double* t = o->lag[0]; o->lag[0] = o->lag[1]; o->lag[1] = t;
    if (o->keep_full) { t = o->full[0]; o->full[0] = o->full[1]; o->full[1] = t; }
    free(h); free(rho_n); free(u_n); free(num_n); free(e_n); free(q_n); free(p_n);
}

/* One sweep of velocity k from the current state, without updating the state (point-update
 * tests): h receives [N] values in the working variables. */
void ora_sweep_one(const ora* o, int k, double* h) { sweep(o, k, h); }

int ora_dims(const ora* o) { return o->d; }
int ora_npoints(const ora* o) { return o->N; }
