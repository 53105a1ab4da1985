"""Pins of the oracle's temperature-term option: the source of Eq. 2 keeps tau (|v|^2 - 3/2) with
tau = (2/3) sum W |v|^2 h - rho (Eq. 4), which the paper drops for its isothermal flows (Sec. 4).
Pinned to an independent dense solve of the discrete steady system, to exact invariants (uniform
state, linearity, jump form = source form, raster = wavefront) and to the warm-start closed form."""
import numpy as np
import pytest

from bruteforce import solve_dense
from oracle import Oracle, velocity_grid
from paper_1712_01132_gb300 import inputs


def _tiny_3d():
    solid = np.zeros((3, 4, 4), bool)
    solid[1, 1:3, 1:3] = True
    return solid


@pytest.mark.parametrize("lateral", ["specular", "periodic"])
@pytest.mark.parametrize("order", [2, 1])
def test_tau_fixed_point_matches_dense_solve(lateral, order):
    solid = _tiny_3d()
    v, w = velocity_grid(3, 4)
    rho, u, k, resid, delta, tau = solve_dense(solid, 1.0, v, w, lateral=lateral, order=order, tau=True)
    assert resid < 1e-11
    o = Oracle(solid, 1.0, v, w, lateral=lateral, order=order, threads=1, tau=True)
    o.iterate(2000)
    _, u2 = o.moments()
    assert np.abs(u - u2).max() < 1e-12
    assert np.abs(tau - o.temperature()).max() < 1e-12
    assert o.permeability() == pytest.approx(k, rel=1e-11)
    assert np.abs(tau).max() > 1e-3          # the term is active


def test_tau_uniform_state_is_a_fixed_point():
    """h = c: rho = c and tau = c ((2/3) sum W |v|^2 - 1) = 0 (the rule integrates v^2 exactly)."""
    solid = _tiny_3d()
    v, w = velocity_grid(3, 4)
    o = Oracle(solid, 0.2, v, w, jump=0.0, threads=1, tau=True)
    o.set_uniform(1.75)
    o.iterate(3)
    rho, u = o.moments()
    assert np.abs(rho[~solid] - 1.75).max() < 1e-13
    assert np.abs(u).max() < 1e-13
    assert np.abs(o.temperature()).max() < 1e-13


@pytest.mark.parametrize("nper", [4, 2])
def test_tau_jump_form_equals_source_form(nper):
    """Also with two nodes per axis, whose rule does not integrate v^2 exactly: the source form
    forms the paper's tau through the exact correction of the x1 ramp."""
    solid = np.zeros((4, 5, 6), bool)
    solid[1:3, 2, 2:4] = True
    v, w = velocity_grid(3, nper)
    a = Oracle(solid, 0.3, v, w, form="jump", threads=1, tau=True)
    b = Oracle(solid, 0.3, v, w, form="source", threads=1, tau=True)
    a.iterate(30)
    b.iterate(30)
    assert np.abs(a.moments()[1] - b.moments()[1]).max() < 1e-13
    assert np.abs(a.moments()[0] - b.moments()[0]).max() < 1e-12
    assert np.abs(a.temperature() - b.temperature()).max() < 1e-12


def test_tau_linear_in_jump_amplitude():
    solid = _tiny_3d()
    v, w = velocity_grid(3, 4)
    a = Oracle(solid, 0.5, v, w, jump=1.0, threads=1, tau=True)
    b = Oracle(solid, 0.5, v, w, jump=2.5, threads=1, tau=True)
    a.iterate(20)
    b.iterate(20)
    assert np.abs(b.temperature() - 2.5 * a.temperature()).max() < 1e-13
    assert np.abs(b.moments()[1] - 2.5 * a.moments()[1]).max() < 1e-13


def test_tau_raster_equals_wavefront_bitwise():
    solid = np.zeros((4, 5, 6), bool)
    solid[1:3, 2, 2:4] = True
    v, w = velocity_grid(3, 4)
    a = Oracle(solid, 0.3, v, w, traversal="raster", threads=1, tau=True)
    b = Oracle(solid, 0.3, v, w, traversal="wavefront", threads=1, tau=True)
    a.iterate(5)
    b.iterate(5)
    assert np.array_equal(a.temperature(), b.temperature())
    assert np.array_equal(a.moments()[1], b.moments()[1])


def test_tau_warm_start_closed_form():
    """set_initial: h0 = rho0 + 2 u0.v gives tau = rho0 ((2/3) sum W |v|^2 - 1) (the odd moments
    of the symmetric grid vanish): zero with four nodes per axis, nonzero with two."""
    solid = _tiny_3d()
    rng = np.random.default_rng(3)
    r0 = rng.standard_normal(solid.shape)
    u0 = 0.1 * rng.standard_normal((3,) + solid.shape)
    for nper in (4, 2):
        v, w = velocity_grid(3, nper)
        sw2 = float((w[:, None] * v * v).sum())
        o = Oracle(solid, 0.3, v, w, threads=1, tau=True)
        o.set_initial(r0, u0)
        assert np.abs(o.temperature() - r0 * (2.0 / 3.0 * sw2 - 1.0) * ~solid).max() < 1e-13


def test_tau_moves_permeability_only_slightly():
    """The paper's remark that tau has no influence on the permeability of its isothermal flows:
    on a 3D sphere-array quadrant the converged k moves by far less than 1e-3 relative."""
    solid = inputs.sphere_quadrant(8, 4, 4, porosity=0.75)
    v, w = velocity_grid(3, 4)
    k = {}
    for tau in (False, True):
        o = Oracle(solid, 0.5, v, w, threads=1, tau=tau)
        o.iterate(400)
        k[tau] = o.permeability()
    assert abs(k[True] / k[False] - 1) < 1e-3


def test_tau_is_rejected_in_2d():
    v, w = velocity_grid(2, 4)
    with pytest.raises(ValueError):
        Oracle(np.zeros((6, 6), bool), 0.3, v, w, tau=True)
