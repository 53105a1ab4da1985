"""Half-range Gauss-Hermite quadrature for the oracle (Sec. 2.2: the Cartesian velocity grid is
built from the half-range Gauss-Hermite rule of Gautschi).

TEST INFRASTRUCTURE ONLY: used by the test suite, the smoke check and the CPU-baseline leg of the
benchmark; the CUDA library has its own, independently written generator.

Route (chosen to be independent of the library's discretised-Stieltjes route):
  1. exact moments mu_m = int_0^inf v^m exp(-v^2) dv = Gamma((m+1)/2) / 2, evaluated in
     60-digit decimal arithmetic (sqrt(pi) from a fixed digit string of pi);
  2. Chebyshev's algorithm (moments -> three-term recurrence coefficients alpha_k, beta_k) in the
     same precision, which tolerates the ill-conditioning of the moment map;
  3. nodes: eigenvalues of the Jacobi matrix in double precision as starting values, polished by
     Newton's method on the monic orthogonal polynomial pi_M evaluated by the recurrence;
  4. weights: Christoffel numbers 1 / sum_k p_k(x_i)^2 with the orthonormal p_k.
"""
from decimal import Decimal, getcontext
import math

import numpy as np

_PI_DIGITS = ("3.14159265358979323846264338327950288419716939937510"
              "58209749445923078164062862089986280348253421170679")

_DPS = 60


def _ctx():
    getcontext().prec = _DPS + 20


def _moments(nmom):
    """mu_m = Gamma((m+1)/2)/2 for m = 0..nmom-1 in Decimal."""
    _ctx()
    sqrt_pi = Decimal(_PI_DIGITS).sqrt()
    mu = []
    for m in range(nmom):
        if m % 2 == 1:          # Gamma(k+1) = k!, k = (m-1)/2
            k = (m - 1) // 2
            g = Decimal(math.factorial(k))
        else:                   # Gamma(k + 1/2) = (2k)! sqrt(pi) / (4^k k!), k = m/2
            k = m // 2
            g = Decimal(math.factorial(2 * k)) * sqrt_pi / (Decimal(4) ** k * Decimal(math.factorial(k)))
        mu.append(g / 2)
    return mu


def _chebyshev(mu, n):
    """Chebyshev algorithm: recurrence coefficients alpha[0..n-1], beta[0..n-1] of the monic
    orthogonal polynomials of the measure with moments mu[0..2n-1] (beta[0] = mu[0])."""
    sig_prev = [Decimal(0)] * (2 * n)
    sig = list(mu[: 2 * n])
    alpha = [mu[1] / mu[0]]
    beta = [mu[0]]
    for k in range(1, n):
        sig_new = [Decimal(0)] * (2 * n)
        for l in range(k, 2 * n - k):
            sig_new[l] = sig[l + 1] - alpha[k - 1] * sig[l] - beta[k - 1] * sig_prev[l]
        alpha.append(sig_new[k + 1] / sig_new[k] - sig[k] / sig[k - 1])
        beta.append(sig_new[k] / sig[k - 1])
        sig_prev, sig = sig, sig_new
    return alpha, beta


def _orthopoly(x, alpha, beta, n):
    """Monic pi_n(x) and its derivative by the three-term recurrence."""
    p0, p1 = Decimal(0), Decimal(1)
    d0, d1 = Decimal(0), Decimal(0)
    for k in range(n):
        p2 = (x - alpha[k]) * p1 - (beta[k] * p0 if k > 0 else Decimal(0))
        d2 = p1 + (x - alpha[k]) * d1 - (beta[k] * d0 if k > 0 else Decimal(0))
        p0, p1 = p1, p2
        d0, d1 = d1, d2
    return p1, d1


def half_range_gauss_hermite(m):
    """Nodes c_i > 0 and weights a_i of the m-point rule for int_0^inf exp(-v^2) g(v) dv."""
    if m < 1:
        raise ValueError("m >= 1")
    _ctx()
    mu = _moments(2 * m)
    alpha, beta = _chebyshev(mu, m)
    jac = np.zeros((m, m))
    for k in range(m):
        jac[k, k] = float(alpha[k])
        if k + 1 < m:
            jac[k, k + 1] = jac[k + 1, k] = math.sqrt(float(beta[k + 1]))
    x0 = np.sort(np.linalg.eigvalsh(jac))
    nodes, weights = [], []
    for xi in x0:
        x = Decimal(repr(float(xi)))
        for _ in range(60):
            p, dp = _orthopoly(x, alpha, beta, m)
            step = p / dp
            x -= step
            if abs(step) < Decimal(10) ** (-_DPS + 5):
                break
        # Christoffel number with orthonormal polynomials p_k = pi_k / sqrt(beta_0 ... beta_k)
        s = Decimal(0)
        pm1, pk = Decimal(0), Decimal(1)
        norm = beta[0]
        s += pk * pk / norm
        for k in range(m - 1):
            pn = (x - alpha[k]) * pk - (beta[k] * pm1 if k > 0 else Decimal(0))
            pm1, pk = pk, pn
            norm = norm * beta[k + 1]
            s += pk * pk / norm
        nodes.append(float(x))
        weights.append(float(1 / s))
    return np.array(nodes), np.array(weights)


def velocity_grid(dims, n_per_axis):
    """Tensor-product velocity grid of n_per_axis points per axis (n_per_axis/2 half-range nodes
    mirrored to both signs).  Returns v [nv, dims] and weights W [nv] normalised with the
    dimensionless equilibrium f_eq = pi^(-d/2) exp(-|v|^2), so sum(W) = 1 and
    sum(W g(v)) approximates int f_eq g dv."""
    if n_per_axis % 2:
        raise ValueError("n_per_axis must be even")
    c, a = half_range_gauss_hermite(n_per_axis // 2)
    v1 = np.concatenate([-c[::-1], c])
    w1 = np.concatenate([a[::-1], a]) / math.sqrt(math.pi)
    grids = np.meshgrid(*([v1] * dims), indexing="ij")
    wgrids = np.meshgrid(*([w1] * dims), indexing="ij")
    v = np.stack([g.reshape(-1) for g in grids], axis=1)
    w = np.prod(np.stack([g.reshape(-1) for g in wgrids], axis=1), axis=1)
    return np.ascontiguousarray(v), np.ascontiguousarray(w)
