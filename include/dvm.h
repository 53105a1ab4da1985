/*
 * dvm.h -- C ABI of the GB300 discrete-velocity solver for steady, pressure-driven rarefied gas
 * flow through voxelised porous media (linearised BGK model, Ho, Zhu, Wu, Wang, Guo, Li, Zhang,
 * "A multi-level parallel solver for rarefied gas flows in porous media", arXiv:1712.01132).
 *
 * One iteration (Sec. 3.1, steps i-iii) runs on the GPU as a transport sweep of every discrete
 * velocity over the fluid voxels (Eq. 9-10, forward substitution in upwind order) fused with the
 * velocity quadrature of the moments (Eq. 4), followed by a finalize pass that forms the wall
 * densities (Eq. 6), the source terms of the next iteration and, every check interval, the
 * permeability (Eq. 11-12) and the convergence measure (Eq. 15).
 *
 * Conventions
 *  - Plain C types only.  Every pointer argument is a HOST pointer unless the argument says
 *    otherwise.  Inputs are copied during the call; the caller keeps ownership of everything it
 *    passes in and owns every output buffer.
 *  - Masks are uint8 arrays laid out [n3][n2][n1] (x1 fastest; x1 is the flow direction), nonzero
 *    = solid voxel.  Fields are double arrays in the same layout; vector fields are [dims][...].
 *  - Every call returns a dvm_status.  Negative values are errors; dvm_last_error() gives a
 *    message.  No C++ exception crosses this boundary.  A context is used by one host thread at a
 *    time.
 *  - A context holds one or more problems (a batch) that share a velocity grid and options; every
 *    problem has its own geometry and Knudsen number.  Work is issued on the CUDA stream given in
 *    the options (the legacy default stream when NULL).
 */
#ifndef DVM_H
#define DVM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dvm_ctx dvm_ctx;   /* opaque, owned by the library */

typedef enum {
    DVM_OK = 0,              /* success; from dvm_iterate: converged (Err < tol) */
    DVM_NOT_CONVERGED = 1,   /* dvm_iterate reached its iteration cap (informational) */
    DVM_EINVAL = -1,         /* invalid argument (message in dvm_last_error) */
    DVM_ENOMEM = -2,         /* device allocation failed */
    DVM_ECUDA = -3,          /* a CUDA call or kernel failed */
    DVM_ETIMEOUT = -4,       /* a bounded wait inside the sweep kernel expired */
    DVM_ENUMERIC = -5        /* non-finite permeability detected */
} dvm_status;

/* Solid mask of one problem. dims = 2 (n[2] ignored) or 3; every n[j] >= 3. */
typedef struct {
    int dims;
    int64_t n[3];
    const uint8_t* solid;    /* host, [n3][n2][n1], nonzero = solid */
} dvm_geometry;

/* Discrete velocity set (Sec. 2.2): nv velocities v [nv][dims] (units of the most probable speed)
 * with quadrature weights w [nv] that include the equilibrium factor pi^(-dims/2) exp(-|v|^2), so
 * that sum(w) = 1 and sum(w g(v)) approximates int f_eq g dv.  Requirements: no zero component,
 * the set is symmetric under the sign change of each component separately, sum(w) = 1 +- 1e-12. */
typedef struct {
    int nv;
    const double* v;
    const double* w;
} dvm_velocity_grid;

/* precision of h, moments and sweeps.  DVM_BF16_STORE (3D only) is the BF16-storage ablation:
 * FP32 arithmetic and FP32 moments, but the transient h kept in HBM between pencils and between
 * iterations (pencil edges and ghost layers) is stored as BF16 (round to nearest even) deviations
 * from the x1 ramp of the source form; its errors are reported, not gated. */
enum { DVM_FP64 = 0, DVM_FP32 = 1, DVM_BF16_STORE = 2 };
enum { DVM_LATERAL_SPECULAR = 0, DVM_LATERAL_PERIODIC = 1 };

typedef struct {
    int precision;       /* DVM_FP64, DVM_FP32 or DVM_BF16_STORE; wall sums, G_p and Err are always FP64 */
    int stencil_order;   /* 2: Eq. 9 second order with the first-order switch at walls; 1: first order */
    int lateral_bc;      /* DVM_LATERAL_SPECULAR (Eq. 8) or DVM_LATERAL_PERIODIC */
    int check_interval;  /* iterations between permeability/Err evaluations (Sec. 3.1: 100) */
    void* stream;        /* cudaStream_t, or NULL for the legacy default stream */
    int tile_x1;         /* sweep tile width along x1: 2D FP64 8 or 16, 2D FP32 4, 8 or 16, 3D 4
                            or 8 (FP32 sweeps a 16-column 2D tile as two 8-column sub-tiles and an
                            8-column 3D tile as two 4-column sub-tiles, between one neighbour wait
                            and one publish); 0 = automatic (8 in 2D; in 3D 8 for FP32 and BF16 storage, 4 for FP64 and
                            for the Shakhov and ES-BGK models) */
    int band_rows;       /* rows per sweep band in 2D, pencil rows R2 = R3 in 3D (0 = automatic:
                            8 in 2D, 4 in 3D FP32, 2 in 3D FP64; in 3D the tile width, then the
                            rows, are reduced until the CTA fits shared memory) */
    /* Optional device allocator (e.g. the caller's caching allocator).  When alloc is NULL the
     * library uses cudaMalloc/cudaFree.  alloc returns NULL on failure. */
    void* (*alloc)(size_t bytes, void* user);
    void (*free)(void* ptr, size_t bytes, void* user);
    void* alloc_user;
    /* Nonzero: dvm_iterate and dvm_step capture each run of iterations between two convergence
     * checks (memset, sweep and finalize launches) into a CUDA graph once and replay it (one graph
     * per run length, starting ghost parity and kernel-timing state, kept until the context is
     * destroyed).  Needs a non-NULL stream (the legacy default stream cannot be captured; with
     * NULL the launches are issued one by one).  With kernel timing enabled (dvm_profile_enable)
     * the captured graph also records its own timing events around every sweep and finalize
     * launch.  The results are the same bits either way. */
    int use_graph;
    /* Lagged-halo domain decomposition of Sec. 3.2 (the paper's MPI subdomains, emulated): the
     * domain is cut into c1 x c2 x c3 blocks (block s along axis j holds the points l with
     * floor(l c_j / n_j) = s); an upstream point in another block takes its value from the previous
     * iteration instead of the current sweep, so blocks sweep independently.  This changes the
     * iteration history (more iterations to converge) but not the fixed point.  0 or 1 = no cut
     * (the exact serial iteration, the default).  Implemented: c1 x c2 in 2D and c1 x c2 x c3 in 3D,
     * each block at least two points wide along every cut axis (DVM_EINVAL otherwise); 2D problems
     * reject c3 > 1, and BF16 storage and the Shakhov / ES-BGK models reject any cut. */
    int subdomains[3];
    /* 3D: at most this many warps per sweep CTA (1..8; 0 = automatic: 8, or 4 for FP64).  The
     * velocities of an octant are split into groups of 64 (FP32) or 32 (FP64) slots per warp, one
     * CTA per group and pencil, so fewer warps per CTA mean more, smaller CTAs per SM (more pencils
     * in flight) at the price of building every point's record once per group.  The moments are summed per group and
     * then over groups, so this choice changes their summation order (results agree to rounding,
     * and for a fixed choice they are the same bits for every tile and pencil shape).  Ignored in
     * 2D. */
    int group_warps;
    /* Nonzero (3D only): keep the temperature term of the linearised BGK equation (Eq. 2): the
     * source gains tau (|v|^2 - 3/2) with the temperature perturbation tau = (2/3) sum_k W_k
     * |v_k|^2 h - rho (Eq. 4).  The paper drops it (Sec. 4: no influence on the permeability of its
     * isothermal flows); the walls re-emit at the wall temperature either way (Eq. 5).  0 (default):
     * dropped.  2D problems and BF16 storage reject it with DVM_EINVAL. */
    int temperature_term;
    /* Maxwell diffuse-specular walls (Eq. 5): 1 - alpha, the specular fraction of the molecules
     * leaving a wall, whose h is h(v - 2 n (v.n)) of the molecules reaching it (taken, like the
     * wall density, at the wall's fluid point from the previous iteration).  0 (default): fully
     * diffuse, the paper's setting (alpha = 1).  Values outside [0, 1] and BF16 storage reject it
     * with DVM_EINVAL. */
    double specular_fraction;
    /* 0 (default): the BGK model of Eq. 2, the paper's.  A Prandtl number Pr > 0 selects the
     * linearised Shakhov (S) model, which the paper names as an extension of its solver (Sec. 1,
     * Sec. 6): the source also carries (4/5)(1 - Pr) q.v (|v|^2 - 5/2) with the heat flux
     * q = sum_k W_k v_k (|v_k|^2 - 5/2) h (the coefficient for which q relaxes at Pr times the
     * collision frequency).  3D with temperature_term only; it runs on the one-velocity-per-lane
     * sweep kernel in FP32 too.  Negative or non-finite values, 2D, no temperature term,
     * subdomains, specular_fraction > 0 or BF16 storage: DVM_EINVAL. */
    double shakhov_prandtl;
    /* 0 (default): BGK.  A Prandtl number Pr > 0 selects the linearised ES-BGK model, the other
     * extension the paper names: the collision frequency becomes Pr nu (the BGK viscosity, so the
     * Kn of Eq. 1 keeps its meaning) and the source also carries (1 - 1/Pr) sum_ij P_ij v_i v_j
     * with the traceless stress P_ij = 2 sum_k W_k (v_ki v_kj - delta_ij |v_k|^2 / 3) h.  The same
     * restrictions as shakhov_prandtl, and not together with it. */
    double es_prandtl;
} dvm_options;

/* Fill *opt with the defaults: FP64, second order, specular lateral faces, check interval 100,
 * NULL stream, automatic tiles, cudaMalloc. */
void dvm_default_options(dvm_options* opt);

/* Half-range Gauss-Hermite velocity grid (Sec. 2.2, Gautschi's half-range rule): n_per_axis
 * (even, 2..128) points per axis, n_per_axis/2 positive nodes of the rule for
 * int_0^inf exp(-v^2) g(v) dv mirrored to negative values, tensor product over dims (2 or 3)
 * axes.  v receives [n^dims][dims] doubles, w receives [n^dims] doubles (weights as described for
 * dvm_velocity_grid, sum = 1).  Host only; needs no GPU.  EINVAL on bad arguments. */
dvm_status dvm_gh_velocity_grid(int dims, int n_per_axis, double* v, double* w);

/* Effective pore size of a medium (Eq. 14, Sec. 4): the ratio r = Lstar / L is sqrt(12 k_inf / eps)
 * in 2D (the channel with the medium's continuum permeability) and sqrt(8 k_inf / (pi eps)) in 3D
 * (the tube), from the continuum-limit permeability k_inf (in units of L^2) and the porosity eps;
 * the effective Knudsen number is Kn / r.  *ratio receives r.  Host only; needs no GPU.  EINVAL
 * when dims is not 2 or 3, k_inf <= 0 or eps is outside (0, 1]. */
dvm_status dvm_effective_pore_size(int dims, double k_inf, double porosity, double* ratio);

/* Create a context for one problem (Sec. 2.1): geometry, Knudsen number kn > 0 (Eq. 1, reference
 * length = x1 extent, so dx = 1/n1 and nu = sqrt(pi)/(2 kn) in Eq. 3) and velocity grid.  The
 * state is the zero perturbation h = 0 with boundary data derived from it (the inflow ghosts of
 * Eq. 7 carry the unit pressure jump).  opt may be NULL (defaults).  Errors: EINVAL (bad kn, dims,
 * sizes < 3, no fluid, no solid/fluid interface, invalid velocity grid), ENOMEM, ECUDA.  On error
 * *out is set to NULL. */
dvm_status dvm_create(const dvm_geometry* geometry, double kn, const dvm_velocity_grid* grid,
                      const dvm_options* opt, dvm_ctx** out);

/* Create a context for a batch of nprob problems (same dims, own geometry and Knudsen number
 * each) that iterate together: every sweep and finalize launch covers all of them. */
dvm_status dvm_create_batch(int nprob, const dvm_geometry* geometries, const double* kn,
                            const dvm_velocity_grid* grid, const dvm_options* opt, dvm_ctx** out);

/* Run iterations (Sec. 3.1) until every problem satisfies Err < tol at a check (Eq. 15 with the
 * check interval ci of the options) or max_iter iterations have run in this call.  Checks fall on
 * the iteration counts that are multiples of ci (counted from context creation).  At a check of
 * iteration l, Err = |k(l) - k(l')| / ((l - l') |k(l)|) with l' the previous check of the problem,
 * so l - l' = ci as in Eq. 15, except after dvm_step moved the count past a multiple of ci without
 * a check or after a warm start (then l' is the iteration of that event).  k(l') at the first
 * check is the k of the start state: 0 for the zero start h = 0 (so the first Err is exactly 1/ci:
 * a tolerance >= 1/ci stops at the first check), the warm start's own k after
 * dvm_set_initial_at.  A problem with k(l) = 0 has Err = 0 if k(l') = 0 too (no flow path).
 * iters_done (may be NULL) receives the iterations run by this call, err_out (may be NULL) the
 * largest Err at the last check (HUGE_VAL before the first).  Returns DVM_OK when converged,
 * DVM_NOT_CONVERGED at the cap, ETIMEOUT/ECUDA/ENUMERIC on failure.  Synchronises the stream at
 * every check. */
dvm_status dvm_iterate(dvm_ctx* ctx, int max_iter, double tol, int* iters_done, double* err_out);

/* Enqueue n iterations on the stream without convergence checks or host synchronisation (the
 * permeability of the last iteration is still computed).  Use dvm_sync to wait and collect
 * errors. */
dvm_status dvm_step(dvm_ctx* ctx, int n);

/* Wait for the stream and report a pending device error (ETIMEOUT/ECUDA). */
dvm_status dvm_sync(dvm_ctx* ctx);

/* Moments of problem 0 after the last iteration (Eq. 4): rho [N] and u [dims][N] in the paper's
 * variables (the density carries the -x1 ramp of the unit pressure gradient); solid points are 0.
 * on_device != 0 means rho and u are device pointers. */
dvm_status dvm_moments(dvm_ctx* ctx, double* rho, double* u, int on_device);
dvm_status dvm_moments_at(dvm_ctx* ctx, int prob, double* rho, double* u, int on_device);

/* Temperature perturbation tau of Eq. 4 of problem prob after the last iteration, [N] doubles (solid
 * points 0), with the temperature term enabled (dvm_options.temperature_term); on_device != 0 means
 * tau is a device pointer.  EINVAL when the term is off. */
dvm_status dvm_temperature_at(dvm_ctx* ctx, int prob, double* tau, int on_device);

/* Heat flux q = sum_k W_k v_k (|v_k|^2 - 5/2) h of problem prob after the last iteration, [3][N]
 * doubles (solid points 0), with the Shakhov model enabled (dvm_options.shakhov_prandtl > 0);
 * on_device != 0 means q is a device pointer.  EINVAL when the model is off. */
dvm_status dvm_heat_flux_at(dvm_ctx* ctx, int prob, double* q, int on_device);

/* Traceless stress P_ij = 2 sum_k W_k (v_ki v_kj - delta_ij |v_k|^2 / 3) h of problem prob after the
 * last iteration, [6][N] doubles in the order 11 22 33 12 13 23 (solid points 0), with the ES-BGK
 * model enabled (dvm_options.es_prandtl > 0); on_device != 0 means p is a device pointer.  EINVAL
 * when the model is off. */
dvm_status dvm_stress_at(dvm_ctx* ctx, int prob, double* p, int on_device);

/* Permeability k = (2/sqrt(pi)) Kn G_p (Eq. 11) and G_p, the mean of u1 over all points (Eq. 12:
 * the cross-section mean, averaged over every x1 cross-section), of the last iteration. */
dvm_status dvm_permeability(dvm_ctx* ctx, double* k, double* gp);
dvm_status dvm_permeability_at(dvm_ctx* ctx, int prob, double* k, double* gp);

/* Wall densities of problem prob (Eq. 6) as [dims][2][N]: face (x, axis j, side -1/+1) whose
 * solid neighbour is x -/+ e_j; 0 where there is no such face. */
dvm_status dvm_wall_density_at(dvm_ctx* ctx, int prob, double* rhos);

/* Tile autotuner (no counterpart in the paper, whose kernel has no tiles): times `iters`
 * iterations (after two untimed ones) of every candidate sweep tile shape on the given problems,
 * with the options in *opt otherwise, and writes the fastest into opt->tile_x1 and
 * opt->band_rows (and, in 3D, opt->group_warps).  Candidates: 2D FP32 x1 tile {16, 8, 4} x band rows
 * {4, 8, 12, 16}; 2D FP64 x1 tile {8, 16} x band rows {4, 8, 12, 16}; 3D x1 tile {4, 8} x pencil
 * rows {2, 3, 4, 5, 6} x warps per CTA {8, 4} (only the caller's value when opt->group_warps is
 * nonzero); shapes that do not fit the device are skipped.  Because every tile shape runs the same dependency-exact
 * wavefront, the tile choice changes the speed and never the result (warps per CTA change the
 * summation order of the moments, see group_warps).  Each candidate context is created
 * and destroyed in turn (device memory of one context at a time); kernels run on opt->stream.
 * best_ms (may be NULL) receives the fastest time per iteration.  Errors: those of dvm_create_batch
 * and dvm_iterate; EINVAL when no candidate fits. */
dvm_status dvm_autotune(int nprob, const dvm_geometry* geometries, const double* kn,
                        const dvm_velocity_grid* grid, dvm_options* opt, int iters, double* best_ms);

/* Warm start of problem prob (0 for dvm_set_initial).  The paper always starts from h = 0
 * (Sec. 3.1); a warm start changes only the iteration count, never the converged answer, because
 * the steady solution is the unique fixed point of the iteration (up to the constant density of
 * each closed fluid region).  The new state is the one an iteration leaves when it has produced
 * the local linearised equilibrium h0(x, v) = rho0(x) + 2 u0(x) . v at every fluid point (the
 * source term of Eq. 10 evaluated at rho0, u0): the moments are the quadrature (Eq. 4) of h0, the
 * wall densities follow from h0 by Eq. 6, and the lagged boundary data of Eq. 7 (x1, periodic
 * with the unit jump) and Eq. 8 (specular) or periodic lateral faces are h0 at the image points.
 * rho0: HOST pointer to [N] doubles, u0: HOST pointer to [dims][N] doubles, both in the paper's
 * variables (the layout dvm_moments returns; values at solid points are ignored).  The
 * caller keeps both buffers.  The context's iteration count keeps running; the next convergence
 * check of this problem compares with the k of the warm-start state, over the iterations run
 * since (a restart of the Eq. 15 history).  Synchronises the stream.  EINVAL (bad prob, NULL,
 * non-finite value at a fluid point), ECUDA. */
dvm_status dvm_set_initial(dvm_ctx* ctx, const double* rho0, const double* u0);
dvm_status dvm_set_initial_at(dvm_ctx* ctx, int prob, const double* rho0, const double* u0);

/* Checkpoint / resume (no counterpart in the paper).  The iteration state is everything the next
 * iteration reads from the previous one (Sec. 3.1): the per-octant moment partials (from which the
 * moments, the wall densities of Eq. 6 and the permeability are rebuilt) and the lagged ghost
 * layers of Eq. 7/8, plus the iteration count and the Eq. 15 history.  dvm_get_state writes it to
 * the HOST buffer buf: with buf == NULL it only stores the required size in *bytes; with a buffer
 * smaller than that it stores the size and returns EINVAL.  dvm_set_state loads a state written by
 * a context with the same geometries, Knudsen numbers, velocity grid, precision, stencil order and
 * lateral condition (EINVAL otherwise) and rebuilds the derived quantities, so that the following
 * iterations are bit-for-bit those the saved context would have run.  Both synchronise the
 * stream; the caller owns buf.  The blob is native-endian and not meant as an archive format. */
dvm_status dvm_get_state(dvm_ctx* ctx, void* buf, size_t* bytes);
dvm_status dvm_set_state(dvm_ctx* ctx, const void* buf, size_t bytes);

/* Number of iterations run since creation, problems in the batch, points of problem prob. */
dvm_status dvm_info(const dvm_ctx* ctx, int64_t* iterations, int* nprob);

/* Message of the last error on this context ("" if none); valid until the next call.  With
 * ctx == NULL: the message of the last failed dvm_create/dvm_create_batch on this thread. */
const char* dvm_last_error(const dvm_ctx* ctx);

/* Release the context and its device memory (synchronises its stream). NULL is a no-op. */
void dvm_destroy(dvm_ctx* ctx);

/* Kernel timing (measurement support, not part of the method).  When enabled, every iteration
 * records CUDA events on the context's stream around its sweep and finalize launches (with
 * use_graph, as event-record nodes of the captured graph: the graph path stays the one that runs;
 * a replay's events are read at the next convergence check, dvm_sync or dvm_profile_read, and
 * before the next replay of a timed graph, which then waits for the stream).
 * dvm_profile_read synchronises the stream, returns the summed event durations (milliseconds) and
 * launch counts since the last read (any pointer may be NULL) and restarts the accumulation. */
dvm_status dvm_profile_enable(dvm_ctx* ctx, int on);
dvm_status dvm_profile_read(dvm_ctx* ctx, double* sweep_ms, int64_t* sweep_launches,
                            double* finalize_ms, int64_t* finalize_launches);

/* Measured FMA throughput of the current device in TFLOP/s (measurement support for the sweep
 * kernels' roofline, which is ALU issue; not part of the method): every thread of eight 256-thread
 * CTAs per SM runs independent FMA chains, packed fma.rn.f32x2 for DVM_FP32 (the sweep kernels'
 * instruction) or fma.rn.f64 for DVM_FP64, timed with CUDA events on `stream` after one warm-up
 * launch.  scratch: DEVICE buffer of at least 8 x SMs x 256 x 8 bytes for the chains' results.
 * Synchronises the stream.  Errors: EINVAL (NULL, other precision, scratch too small), ECUDA. */
dvm_status dvm_alu_peak(int precision, void* scratch, int64_t scratch_bytes, void* stream, double* tflops);

/* Bytes copied host->device and device->host by this context since creation (inputs, setup
 * tables, readouts, permeability and status words). */
dvm_status dvm_transfer_bytes(const dvm_ctx* ctx, int64_t* h2d, int64_t* d2h);

/* Permeability of a caller-held velocity field, without allocating device memory.  The paper has
 * no counterpart: this is a service for callers that cannot allocate at the moment they need the
 * result, e.g. code running while a stream is captured into a CUDA graph, plugins whose host
 * framework owns all device memory, or allocation-free steady-state loops.
 * u1_dev: DEVICE pointer to n doubles (the x1 velocity of every point, solid points 0, any layout);
 * kn > 0; out_dev: DEVICE pointer to 2 doubles receiving k = (2/sqrt(pi)) kn mean(u1) and mean(u1),
 * written asynchronously on `stream` (cudaStream_t, NULL = legacy default stream).
 * Scratch: a file-scope device array sized for at most 2,097,152 points (8192 blocks of 256); larger
 * n returns DVM_EINVAL.  Each GPU that loads the library holds the array until the process exits.
 * The first call on a device looks up the array's address (cudaGetSymbolAddress) and caches it;
 * make that first call before any stream capture.  The cached address belongs to the device's
 * current context: after cudaDeviceReset (or any other re-creation of the primary context) it is
 * stale, so do not call this function again in that process.  The result agrees with the k of the
 * solver's own reduction to FP64 rounding (other block grouping).  Calls share the array: calls whose kernels can
 * overlap on the GPU race, so order them on one stream.  Calls no cudaMalloc/cudaFree.  Errors:
 * DVM_EINVAL (null pointer, n out of range, bad kn), DVM_ECUDA; message in
 * dvm_noalloc_last_error(). */
dvm_status dvm_permeability_noalloc(const double* u1_dev, int64_t n, double kn, double* out_dev, void* stream);
const char* dvm_noalloc_last_error(void);

/* ---- Learned warm start: kernels of a small 3D convolutional network -------------------------
 * The paper has no counterpart.  A network predicts the initial density and velocity fields
 * (the input of dvm_set_initial) from the solid mask, a signed distance and log Kn; it changes
 * only where the source iteration of Sec. 3.1 starts, never its fixed point.  All pointers are
 * DEVICE pointers to FP32 single-sample tensors in channel-major layout t[c][z][y][x] (x fastest,
 * d x h x w voxels); work is enqueued on `stream` (cudaStream_t, NULL = legacy default stream) and
 * nothing is allocated (the callers pass scratch buffers).  Convolutions are 3 x 3 x 3 with periodic padding, weights w[co][ci][27]
 * with tap index (kz * 3 + ky) * 3 + kx for offsets kz, ky, kx in -1..1, biases b[co] (may be
 * NULL), FP32 accumulation.  accumulate != 0 adds into the output instead of overwriting it.
 * Errors: DVM_EINVAL (NULL pointer, non-positive size, odd extent for the 2x resampling, scratch
 * too small), DVM_ECUDA (launch failure). */
/* y = conv(x, w) + b: y[co][v] = b[co] + sum_ci sum_k w[co][ci][k] x[ci][v + off(k)].  Runs on the
 * tcgen05 tensor cores with BF16 operands (x and w rounded to nearest even) and FP32 accumulation.
 * scratch: DEVICE buffer of at least dvm_nn_conv3d_scratch_bytes(cin, cout, d, h, w_) bytes (the
 * padded BF16 copy of x and the BF16 weights; any alignment), reused by the next call on the same
 * stream.  w_ (the x extent) must be at most 128 (DVM_EINVAL otherwise). */
dvm_status dvm_nn_conv3d(const float* x, const float* w, const float* b, float* y, int cin, int cout,
                         int d, int h, int w_, int accumulate, void* scratch, int64_t scratch_bytes,
                         void* stream);
/* data gradient: dx[ci][v] (+)= sum_co sum_k w[co][ci][k] dy[co][v - off(k)], the same tensor-core
 * convolution of dy with the channel roles transposed and the taps mirrored; scratch as above. */
dvm_status dvm_nn_conv3d_dgrad(const float* dy, const float* w, float* dx, int cin, int cout, int d,
                               int h, int w_, int accumulate, void* scratch, int64_t scratch_bytes,
                               void* stream);
/* scratch bytes that serve both dvm_nn_conv3d and dvm_nn_conv3d_dgrad of this shape (0 for a
 * non-positive size) */
int64_t dvm_nn_conv3d_scratch_bytes(int cin, int cout, int d, int h, int w_);
/* Synchronises the stream and returns the convolutions' device status word: 0, or DVM_ETIMEOUT when
 * a bounded wait inside a convolution expired (its output is then not written).  Clears it. */
int dvm_nn_status(void* stream);
/* weight and bias gradients: dw[co][ci][k] (+)= sum_v dy[co][v] x[ci][v + off(k)] on the tcgen05
 * tensor cores (x and dy rounded to BF16, FP32 accumulation, the voxel sum split over CTAs and the
 * splits added in a fixed order), db[co] (+)= sum_v dy[co][v] in FP32 (db may be NULL).  scratch:
 * DEVICE buffer of at least dvm_nn_wgrad_scratch_floats(...) floats (BF16 copies of x and dy and the
 * split partials). */
dvm_status dvm_nn_conv3d_wgrad(const float* x, const float* dy, float* dw, float* db, float* scratch,
                               int64_t scratch_floats, int cin, int cout, int d, int h, int w_,
                               int accumulate, void* stream);
int64_t dvm_nn_wgrad_scratch_floats(int cin, int cout, int d, int h, int w_);
/* y = max(y, 0) in place; relu_bwd: dy = 0 where y <= 0 (in place on dy) */
dvm_status dvm_nn_relu(float* y, int64_t n, void* stream);
dvm_status dvm_nn_relu_bwd(const float* y, float* dy, int64_t n, void* stream);
/* 2 x 2 x 2 mean pooling of x (c channels, d x h x w, all even) into y (d/2 x h/2 x w/2) and its
 * gradient; nearest-neighbour 2x upsampling of x (d/2 x h/2 x w/2) into y (d x h x w) and its
 * gradient (the sum over the 8 children) */
dvm_status dvm_nn_pool2(const float* x, float* y, int c, int d, int h, int w_, void* stream);
dvm_status dvm_nn_pool2_bwd(const float* dy, float* dx, int c, int d, int h, int w_, int accumulate,
                            void* stream);
dvm_status dvm_nn_up2(const float* x, float* y, int c, int d, int h, int w_, void* stream);
dvm_status dvm_nn_up2_bwd(const float* dy, float* dx, int c, int d, int h, int w_, void* stream);
/* masked squared error: partial[b] = block sums of (mask[v] (y - t))^2 over the c x v values
 * (dvm_nn_mse_partials(c, v) blocks) and, when dy is not NULL, dy = 2 mask (y - t) inv_count */
dvm_status dvm_nn_mse(const float* y, const float* t, const float* mask, float* dy, float* partial,
                      int c, int64_t v, float inv_count, void* stream);
int64_t dvm_nn_mse_partials(int c, int64_t v);
/* Adam step (bias-corrected, step >= 1) on FP32 master weights w with moments m, v and gradient
 * g * grad_scale; wq receives the BF16 rounding of w (as FP32), the weights forward and backward
 * use.  round_bf16: wq = BF16 rounding of w. */
dvm_status dvm_nn_adam(float* w, float* wq, const float* g, float* m, float* v, int64_t n, float lr,
                       float beta1, float beta2, float eps, int64_t step, float grad_scale, void* stream);
dvm_status dvm_nn_round_bf16(const float* w, float* wq, int64_t n, void* stream);

/* Test hook (fault-handling tests; not needed in normal use): set the bound of every spin wait
 * of the sweep kernel to timeout_ns and make work item withhold_item (-1: none) never publish its
 * progress, so that the band waiting on it gives up, the kernel records DVM_ETIMEOUT in its status
 * word and every CTA returns.  The next dvm_iterate/dvm_sync reports DVM_ETIMEOUT; the context and
 * the CUDA context stay usable (the solution state of that iteration is not meaningful). */
dvm_status dvm_debug_set_wait(dvm_ctx* ctx, long long timeout_ns, int withhold_item);

#ifdef __cplusplus
}
#endif

#endif /* DVM_H */
