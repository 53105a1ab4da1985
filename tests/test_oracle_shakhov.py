"""Pins of the oracle's Shakhov (S) model option.  The paper solves the BGK equation and names the
ES-BGK and Shakhov models as extensions of the same solver (Sec. 1, Sec. 6) without writing them
out; the linearised S model adds (4/5)(1 - Pr) q.v (|v|^2 - 5/2) to the source of Eq. 2, with the
heat flux q = sum W v (|v|^2 - 5/2) h, next to the temperature term.

Pinned to: the defining property of the S model (the heat flux relaxes at Pr times the collision
frequency, which fixes the coefficient) through exact Gauss-Hermite moments; an independent dense
solve of the discrete steady system; Pr = 1 reducing to the BGK model with the temperature term;
and the exact invariants (jump form = source form, raster = wavefront, linearity)."""
import math

import numpy as np
import pytest

from bruteforce import solve_dense
from oracle import Oracle, velocity_grid


def _tiny_3d():
    solid = np.zeros((3, 4, 4), bool)
    solid[1, 1:3, 1:3] = True
    return solid


def test_heat_flux_moment_of_the_s_term_fixes_the_coefficient():
    """For a rule exact to degree 6 (8 nodes per axis), sum W v_i (|v|^2 - 5/2) v_j (|v|^2 - 5/2)
    = (5/4) delta_ij (Gaussian moments: E[v1^2 |v|^4] = 35/8, E[v1^2 |v|^2] = 5/4, E[v1^2] = 1/2),
    while the mass, momentum and energy moments of the term vanish.  The BGK part relaxes q at the
    collision frequency, so the S term with coefficient A leaves nu (1 - 5 A / 4) = Pr nu exactly
    when A = (4/5)(1 - Pr)."""
    v, w = velocity_grid(3, 8)
    vv = (v * v).sum(axis=1)
    g = v * (vv - 2.5)[:, None]                       # v (|v|^2 - 5/2)
    M = (w[:, None, None] * g[:, :, None] * g[:, None, :]).sum(axis=0)
    assert np.abs(M - 1.25 * np.eye(3)).max() < 1e-13
    q = np.array([0.3, -0.2, 0.7])
    for pr in (2.0 / 3.0, 0.5, 1.0):
        A = 0.8 * (1.0 - pr)
        term = A * (g @ q)                            # the S term at every velocity, per unit nu
        assert abs(float(w @ term)) < 1e-14                                     # mass
        assert np.abs((w[:, None] * v * term[:, None]).sum(axis=0)).max() < 1e-14   # momentum
        assert abs(float((w * vv) @ term)) < 1e-14                              # energy
        relax = q - (w[:, None] * g * term[:, None]).sum(axis=0)               # BGK part minus S part
        assert np.abs(relax - pr * q).max() < 1e-13


@pytest.mark.parametrize("lateral", ["specular", "periodic"])
@pytest.mark.parametrize("order", [2, 1])
def test_shakhov_fixed_point_matches_dense_solve(lateral, order):
    solid = _tiny_3d()
    v, w = velocity_grid(3, 4)
    rho, u, k, resid, delta, tau, heat = solve_dense(solid, 1.0, v, w, lateral=lateral, order=order, tau=True,
                                                     shakhov_pr=2.0 / 3.0)
    assert resid < 1e-11
    o = Oracle(solid, 1.0, v, w, lateral=lateral, order=order, threads=1, tau=True, shakhov_pr=2.0 / 3.0)
    o.iterate(2000)
    _, u2 = o.moments()
    assert np.abs(u - u2).max() < 1e-12
    assert np.abs(tau - o.temperature()).max() < 1e-12
    assert np.abs(heat - o.heat_flux()).max() < 1e-12
    assert o.permeability() == pytest.approx(k, rel=1e-11)
    assert np.abs(heat).max() > 1e-3               # the heat flux is active
    # and it changes the flow: the BGK fixed point with the temperature term differs
    _, u_bgk, *_ = solve_dense(solid, 1.0, v, w, lateral=lateral, order=order, tau=True)
    assert np.abs(u - u_bgk).max() > 1e-6


def test_prandtl_one_is_the_bgk_model_bitwise():
    solid = _tiny_3d()
    v, w = velocity_grid(3, 4)
    a = Oracle(solid, 0.4, v, w, threads=1, tau=True)
    b = Oracle(solid, 0.4, v, w, threads=1, tau=True, shakhov_pr=1.0)
    a.iterate(15)
    b.iterate(15)
    assert np.array_equal(a.moments()[1], b.moments()[1])
    assert np.array_equal(a.temperature(), b.temperature())
    assert np.abs(b.heat_flux()).max() > 0.0       # q is still formed


@pytest.mark.parametrize("nper", [4, 2])
def test_shakhov_jump_form_equals_source_form(nper):
    solid = np.zeros((4, 5, 6), bool)
    solid[1:3, 2, 2:4] = True
    v, w = velocity_grid(3, nper)
    a = Oracle(solid, 0.3, v, w, form="jump", threads=1, tau=True, shakhov_pr=2.0 / 3.0)
    b = Oracle(solid, 0.3, v, w, form="source", threads=1, tau=True, shakhov_pr=2.0 / 3.0)
    a.iterate(30)
    b.iterate(30)
    assert np.abs(a.moments()[1] - b.moments()[1]).max() < 1e-13
    assert np.abs(a.heat_flux() - b.heat_flux()).max() < 1e-12
    assert np.abs(a.temperature() - b.temperature()).max() < 1e-12


def test_shakhov_linear_in_jump_and_raster_equals_wavefront():
    solid = np.zeros((4, 5, 6), bool)
    solid[1:3, 2, 2:4] = True
    v, w = velocity_grid(3, 4)
    a = Oracle(solid, 0.5, v, w, jump=1.0, threads=1, tau=True, shakhov_pr=2.0 / 3.0)
    b = Oracle(solid, 0.5, v, w, jump=2.5, threads=1, tau=True, shakhov_pr=2.0 / 3.0)
    c = Oracle(solid, 0.5, v, w, jump=1.0, threads=1, tau=True, shakhov_pr=2.0 / 3.0, traversal="wavefront")
    a.iterate(20)
    b.iterate(20)
    c.iterate(20)
    assert np.abs(b.heat_flux() - 2.5 * a.heat_flux()).max() < 1e-13
    assert np.abs(b.moments()[1] - 2.5 * a.moments()[1]).max() < 1e-13
    assert np.array_equal(a.moments()[1], c.moments()[1])
    assert np.array_equal(a.heat_flux(), c.heat_flux())


def test_shakhov_warm_start_state_has_no_heat_flux_for_an_exact_rule():
    """h0 = rho0 + 2 u0.v has q = 2 u0 sum W v1^2 (|v|^2 - 5/2) = 0 for a rule exact to degree 4."""
    solid = _tiny_3d()
    v, w = velocity_grid(3, 6)
    rng = np.random.default_rng(3)
    o = Oracle(solid, 0.4, v, w, threads=1, tau=True, shakhov_pr=2.0 / 3.0)
    o.set_initial(rng.standard_normal(solid.shape), rng.standard_normal((3,) + solid.shape))
    assert np.abs(o.heat_flux()).max() < 1e-13


def test_shakhov_needs_the_temperature_term():
    with pytest.raises(ValueError):
        Oracle(_tiny_3d(), 0.4, *velocity_grid(3, 4), tau=False, shakhov_pr=2.0 / 3.0)
    assert math.isclose(0.8 * (1.0 - 2.0 / 3.0), 4.0 / 15.0)
