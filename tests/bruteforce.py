"""Brute-force dense solve of the discrete steady problem on tiny grids (test helper).

Independent of the C oracle: this assembles, as one dense linear system, the discretised
linearised BGK equations of every (fluid point, velocity) pair -- Eq. 10 with the upwind stencil
of Eq. 9, diffuse walls of Eq. 5-6, the pressure jump of Eq. 7 and specular (Eq. 8) or periodic
lateral faces -- with the moments of Eq. 4 written as linear functionals of the unknowns, and
solves it with a least-squares solver plus the gauge condition mean(rho) = 0 (the problem fixes rho
only up to a constant).

The iteration lags some couplings (moments, wall densities and ghost data come from the previous
iteration) while upstream fluid values inside the domain come from the current sweep.  Where the
stencil is not in conservative form (the second-order stencil next to walls), the steady system is
not consistent: the iteration's limit is h^n = h* + n delta (a uniform drift of the constant mode)
with A h* + delta A_cur 1 = b, where A = A_cur + A_lag.  The solve below includes delta as an
unknown, so it reproduces the limit of the iteration exactly in both cases (delta = 0 when the
system is consistent, e.g. with the first-order stencil).
"""
import math

import numpy as np


def solve_dense(solid, kn, v, w, jump=1.0, order=2, lateral="specular", tau=False, alpha=1.0, shakhov_pr=0.0,
                es_pr=0.0):
    """tau: keep the temperature term tau (|v|^2 - 3/2) of Eq. 2 with tau = (2/3) sum W |v|^2 h - rho
    (Eq. 4), a linear functional of the unknowns at the same point like rho and u.
    alpha: Maxwell accommodation of Eq. 5; the wall value of velocity k is alpha rho_s + (1 - alpha)
    h(x_f, reflected k) with h at the wall's fluid point x_f (lagged, like rho_s).
    shakhov_pr > 0 (with tau): linearised Shakhov model, the source adds
    (4/5)(1 - Pr) q.v_k (|v_k|^2 - 5/2) with q = sum W v (|v|^2 - 5/2) h at the same point.
    es_pr > 0 (with tau): linearised ES-BGK model, collision frequency Pr nu and the source adds
    (1 - 1/Pr) sum_ij P_ij v_i v_j with P_ij = 2 sum W (v_i v_j - delta_ij |v|^2 / 3) h."""
    assert shakhov_pr == 0.0 or tau
    assert es_pr == 0.0 or (tau and shakhov_pr == 0.0)
    solid = np.asarray(solid, dtype=bool)
    dims = solid.ndim
    shape = solid.shape
    n = shape[::-1]                      # (n1, n2[, n3])
    v = np.asarray(v, dtype=float).reshape(-1, dims)
    w = np.asarray(w, dtype=float)
    nv = len(w)
    nu = math.sqrt(math.pi) / (2.0 * kn)
    if es_pr > 0.0:
        nu *= es_pr                      # the same viscosity with the ES model's stress relaxation
    dx = 1.0 / n[0]

    def arr_index(c):                    # coordinate tuple (x1, x2, ...) -> numpy index
        return tuple(c[::-1])

    fluid_coords = [tuple(int(t) for t in np.unravel_index(i, shape)[::-1])
                    for i in range(solid.size) if not solid.flat[i]]
    fid = {c: f for f, c in enumerate(fluid_coords)}
    nf = len(fluid_coords)

    refl = np.zeros((dims, nv), dtype=int)
    for j in range(dims):
        for k in range(nv):
            target = v[k].copy()
            target[j] = -target[j]
            match = np.where(np.all(v == target, axis=1))[0]
            refl[j, k] = match[0]

    denom = np.zeros((dims, 2))
    for j in range(dims):
        for sd, side in enumerate((-1, 1)):
            denom[j, sd] = sum(w[k] * abs(v[k, j]) for k in range(nv) if side * v[k, j] < 0)

    def periodic(j):
        return j == 0 or lateral == "periodic"

    def map_coord(j, l):
        """-> (in-domain coordinate, x1 replica index, mirrored?)"""
        nj = n[j]
        if 0 <= l < nj:
            return l, 0, False
        if periodic(j):
            return l % nj, (-1 if l < 0 else 1) if j == 0 else 0, False
        return (-1 - l if l < 0 else 2 * nj - 1 - l), 0, True

    def moved(c, j, l):
        cc = list(c)
        cc[j] = l
        return tuple(cc)

    def is_solid(c, j, l):
        lb, _, _ = map_coord(j, l)
        return bool(solid[arr_index(moved(c, j, lb))])

    def col(f, k):
        return f * nv + k

    def h_term(c, j, l, k):
        """(coefficients, constant, lagged?) of an upstream fluid value"""
        lb, r, mir = map_coord(j, l)
        kk = refl[j, k] if mir else k
        f = fid[moved(c, j, lb)]
        return {col(f, kk): 1.0}, -r * jump, lb != l

    def wall_term(c, j, l, side, k0):
        lb, r, mir = map_coord(j, l)
        sd = -side if mir else side
        f = fid[moved(c, j, lb)]
        sdi = 1 if sd > 0 else 0
        coefs = {}
        for k in range(nv):
            if sd * v[k, j] > 0:
                coefs[col(f, k)] = alpha * w[k] * abs(v[k, j]) / denom[j, sdi]
        if alpha < 1.0:
            kr = refl[j, k0] if not mir else k0
            coefs[col(f, kr)] = coefs.get(col(f, kr), 0.0) + (1.0 - alpha)
        return coefs, -r * jump, True

    U = nf * nv
    A = np.zeros((U + 1, U + 1))     # last column: drift delta ; last row: gauge
    lag1 = np.zeros(U)                # A_lag applied to the constant vector 1
    b = np.zeros(U + 1)
    for f, c in enumerate(fluid_coords):
        for k in range(nv):
            row = col(f, k)
            # -nu (rho + 2 u.v_k [+ tau (|v_k|^2 - 3/2)])
            vk2 = float(np.dot(v[k], v[k]))
            for kk in range(nv):
                cv = nu * w[kk] * (1.0 + 2.0 * float(np.dot(v[kk], v[k])))
                if tau:
                    cv += nu * w[kk] * (2.0 / 3.0 * float(np.dot(v[kk], v[kk])) - 1.0) * (vk2 - 1.5)
                if shakhov_pr > 0.0:
                    vkk2 = float(np.dot(v[kk], v[kk]))
                    cv += (nu * 0.8 * (1.0 - shakhov_pr) * w[kk] * float(np.dot(v[kk], v[k]))
                           * (vkk2 - 2.5) * (vk2 - 2.5))
                if es_pr > 0.0:
                    vkk2 = float(np.dot(v[kk], v[kk]))
                    # sum_ij P_ij v_ki v_kj with P_ij = 2 W (v_kk,i v_kk,j - delta_ij |v_kk|^2 / 3)
                    pv = 2.0 * (float(np.dot(v[kk], v[k])) ** 2 - vkk2 * vk2 / 3.0)
                    cv += nu * (1.0 - 1.0 / es_pr) * w[kk] * pv
                A[row, col(f, kk)] -= cv
                lag1[row] -= cv
            diag = nu
            for j in range(dims):
                s = 1 if v[k, j] > 0 else -1
                a = abs(v[k, j])
                terms = []
                if is_solid(c, j, c[j] - s):
                    C0, C1 = 1.0 / dx, -1.0 / dx
                    terms.append((a * C1, wall_term(c, j, c[j], -s, k)))
                elif order == 1 or is_solid(c, j, c[j] - 2 * s):
                    C0, C1 = 1.0 / dx, -1.0 / dx
                    terms.append((a * C1, h_term(c, j, c[j] - s, k)))
                else:
                    C0, C1, C2 = 1.5 / dx, -2.0 / dx, 0.5 / dx
                    terms.append((a * C1, h_term(c, j, c[j] - s, k)))
                    terms.append((a * C2, h_term(c, j, c[j] - 2 * s, k)))
                diag += a * C0
                for coef, (lin, const, lagged) in terms:
                    for cidx, cv in lin.items():
                        A[row, cidx] += coef * cv
                        if lagged:
                            lag1[row] += coef * cv
                    b[row] -= coef * const
            A[row, row] += diag
    # gauge: sum of rho over fluid points = 0
    for f in range(nf):
        for k in range(nv):
            A[U, col(f, k)] = w[k]
    A[:U, U] = -lag1                  # A h* - delta A_lag 1 = b
    sol, *_ = np.linalg.lstsq(A, b, rcond=None)
    delta = float(sol[U])
    H = sol[:U].reshape(nf, nv)
    rho = np.zeros(shape)
    u = np.zeros((dims,) + shape)
    temp = np.zeros(shape)
    heat = np.zeros((dims,) + shape)
    stress = np.zeros((6,) + shape)
    vv = (v * v).sum(axis=1)
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    for f, c in enumerate(fluid_coords):
        rho[arr_index(c)] = float(np.dot(w, H[f]))
        temp[arr_index(c)] = 2.0 / 3.0 * float(np.dot(w * vv, H[f])) - rho[arr_index(c)]
        for j in range(dims):
            u[(j,) + arr_index(c)] = float(np.dot(w * v[:, j], H[f]))
            heat[(j,) + arr_index(c)] = float(np.dot(w * v[:, j] * (vv - 2.5), H[f]))
        if dims == 3:
            for a, (i, j) in enumerate(pairs):
                stress[(a,) + arr_index(c)] = float(np.dot(2.0 * w * (v[:, i] * v[:, j] - (vv / 3.0 if i == j else 0.0)),
                                                           H[f]))
    k_perm = 2.0 / math.sqrt(math.pi) * kn * float(u[0].sum() / u[0].size)
    resid = float(np.abs(A[:U] @ sol - b[:U]).max())
    if shakhov_pr > 0.0:
        return rho, u, k_perm, resid, delta, temp, heat
    if es_pr > 0.0:
        return rho, u, k_perm, resid, delta, temp, stress
    if tau:
        return rho, u, k_perm, resid, delta, temp
    return rho, u, k_perm, resid, delta
