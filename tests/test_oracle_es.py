"""Pins of the oracle's ES-BGK (ellipsoidal-statistical) model option.  The paper names the ES-BGK
model next to the Shakhov model as an extension of its BGK solver (Sec. 1, Sec. 6) without writing
it out.  Linearised about the equilibrium, the anisotropic Gaussian of the model adds
(1 - 1/Pr) sum_ij P_ij v_i v_j to the source of Eq. 2, with the traceless stress
P_ij = 2 sum W (v_i v_j - delta_ij |v|^2 / 3) h, and the collision frequency becomes Pr nu so
that the viscosity (and the Kn of Eq. 1) stays that of the BGK model.

Pinned to: the stress and heat-flux relaxation rates of the model through exact Gauss-Hermite
moments (which fix both the coefficient and the collision frequency); an independent dense solve
of the discrete steady system; Pr = 1 reducing to the BGK model with the temperature term; and the
exact invariants (jump form = source form, raster = wavefront, linearity)."""
import numpy as np
import pytest

from bruteforce import solve_dense
from oracle import Oracle, velocity_grid

PR = 2.0 / 3.0
PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def _tiny_3d():
    solid = np.zeros((3, 4, 4), bool)
    solid[1, 1:3, 1:3] = True
    return solid


def test_relaxation_rates_fix_the_coefficient_and_the_collision_frequency():
    """For a rule exact to degree 6, sum W 2 (v_k v_l - delta |v|^2 / 3) v_i v_j contracts a
    traceless symmetric P to P_kl (Gaussian moments E[v_k v_l v_i v_j] = (d_kl d_ij + d_ki d_lj +
    d_kj d_li) / 4), and the term carries no mass, momentum, energy or heat flux.  With collision
    frequency nu_ES the stress then relaxes at nu_ES (1 - b) for the coefficient b, i.e. at
    nu_ES / Pr for b = 1 - 1/Pr: the BGK viscosity needs nu_ES = Pr nu, and the heat flux relaxes
    at nu_ES = Pr nu (the model's Prandtl number)."""
    v, w = velocity_grid(3, 8)
    vv = (v * v).sum(axis=1)
    rng = np.random.default_rng(1)
    A = rng.standard_normal((3, 3))
    P = A + A.T
    P -= np.trace(P) / 3.0 * np.eye(3)
    term = np.einsum("ij,ki,kj->k", P, v, v)             # sum_ij P_ij v_i v_j at every velocity
    stress = np.array([[float((2.0 * w * (v[:, a] * v[:, b] - (vv / 3.0 if a == b else 0.0))) @ term)
                        for b in range(3)] for a in range(3)])
    assert np.abs(stress - P).max() < 1e-13
    assert abs(float(w @ term)) < 1e-14                                          # mass
    assert np.abs((w[:, None] * v * term[:, None]).sum(axis=0)).max() < 1e-14      # momentum
    assert abs(float((w * vv) @ term)) < 1e-13                                   # energy
    assert np.abs((w[:, None] * v * (vv - 2.5)[:, None] * term[:, None]).sum(axis=0)).max() < 1e-13   # heat flux
    for pr in (2.0 / 3.0, 0.5, 1.0):
        b = 1.0 - 1.0 / pr
        nu_es = pr * 1.0
        assert abs(nu_es * (1.0 - b) - 1.0) < 1e-15          # stress relaxes at the BGK rate nu = 1


@pytest.mark.parametrize("lateral", ["specular", "periodic"])
@pytest.mark.parametrize("order", [2, 1])
def test_es_fixed_point_matches_dense_solve(lateral, order):
    solid = _tiny_3d()
    v, w = velocity_grid(3, 4)
    rho, u, k, resid, delta, tau, stress = solve_dense(solid, 1.0, v, w, lateral=lateral, order=order, tau=True,
                                                       es_pr=PR)
    assert resid < 1e-11
    o = Oracle(solid, 1.0, v, w, lateral=lateral, order=order, threads=1, tau=True, es_pr=PR)
    o.iterate(3000)
    _, u2 = o.moments()
    assert np.abs(u - u2).max() < 1e-12
    assert np.abs(tau - o.temperature()).max() < 1e-12
    assert np.abs(stress - o.stress()).max() < 1e-12
    assert o.permeability() == pytest.approx(k, rel=1e-11)
    assert np.abs(stress).max() > 1e-3             # the stress is active
    _, u_bgk, *_ = solve_dense(solid, 1.0, v, w, lateral=lateral, order=order, tau=True)
    assert np.abs(u - u_bgk).max() > 1e-6


def test_prandtl_one_is_the_bgk_model_bitwise():
    solid = _tiny_3d()
    v, w = velocity_grid(3, 4)
    a = Oracle(solid, 0.4, v, w, threads=1, tau=True)
    b = Oracle(solid, 0.4, v, w, threads=1, tau=True, es_pr=1.0)
    a.iterate(15)
    b.iterate(15)
    assert np.array_equal(a.moments()[1], b.moments()[1])
    assert np.array_equal(a.temperature(), b.temperature())
    assert np.abs(b.stress()).max() > 0.0


@pytest.mark.parametrize("nper", [4, 2])
def test_es_jump_form_equals_source_form(nper):
    solid = np.zeros((4, 5, 6), bool)
    solid[1:3, 2, 2:4] = True
    v, w = velocity_grid(3, nper)
    a = Oracle(solid, 0.3, v, w, form="jump", threads=1, tau=True, es_pr=PR)
    b = Oracle(solid, 0.3, v, w, form="source", threads=1, tau=True, es_pr=PR)
    a.iterate(30)
    b.iterate(30)
    assert np.abs(a.moments()[1] - b.moments()[1]).max() < 1e-13
    assert np.abs(a.stress() - b.stress()).max() < 1e-12
    assert np.abs(a.temperature() - b.temperature()).max() < 1e-12


def test_es_linear_in_jump_and_raster_equals_wavefront():
    solid = np.zeros((4, 5, 6), bool)
    solid[1:3, 2, 2:4] = True
    v, w = velocity_grid(3, 4)
    a = Oracle(solid, 0.5, v, w, jump=1.0, threads=1, tau=True, es_pr=PR)
    b = Oracle(solid, 0.5, v, w, jump=2.5, threads=1, tau=True, es_pr=PR)
    c = Oracle(solid, 0.5, v, w, jump=1.0, threads=1, tau=True, es_pr=PR, traversal="wavefront")
    a.iterate(20)
    b.iterate(20)
    c.iterate(20)
    assert np.abs(b.stress() - 2.5 * a.stress()).max() < 1e-13
    assert np.abs(b.moments()[1] - 2.5 * a.moments()[1]).max() < 1e-13
    assert np.array_equal(a.moments()[1], c.moments()[1])
    assert np.array_equal(a.stress(), c.stress())


def test_es_option_is_validated():
    v, w = velocity_grid(3, 4)
    with pytest.raises(ValueError):
        Oracle(_tiny_3d(), 0.4, v, w, tau=False, es_pr=PR)
    with pytest.raises(ValueError):
        Oracle(_tiny_3d(), 0.4, v, w, tau=True, es_pr=PR, shakhov_pr=PR)
