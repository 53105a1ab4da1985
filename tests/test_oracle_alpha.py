"""Pins of the oracle's Maxwell accommodation option (Eq. 5): the wall value of a molecule leaving a
wall is alpha rho_s + (1 - alpha) h(v - 2 n (v.n)), the specular part taken at the wall's fluid
point from the previous iteration like rho_s; alpha = 1 (fully diffuse) is the paper's setting.
Pinned to an independent dense solve, to exact invariants, and to the monotone growth of the
permeability as the walls become more specular (more slip)."""
import numpy as np
import pytest

from bruteforce import solve_dense
from oracle import Oracle, velocity_grid
from paper_1712_01132_gb300 import inputs


def _tiny_2d():
    solid = np.zeros((7, 8), bool)
    solid[2:4, 2:5] = True
    solid[5, 6] = True
    return solid


@pytest.mark.parametrize("alpha", [0.8, 0.4])
@pytest.mark.parametrize("lateral", ["specular", "periodic"])
def test_alpha_fixed_point_matches_dense_solve_2d(alpha, lateral):
    solid = _tiny_2d()
    v, w = velocity_grid(2, 4)
    rho, u, k, resid, delta = solve_dense(solid, 1.0, v, w, lateral=lateral, order=2, alpha=alpha)
    assert resid < 1e-11
    o = Oracle(solid, 1.0, v, w, lateral=lateral, order=2, threads=1, alpha=alpha)
    o.iterate(4000)
    _, u2 = o.moments()
    assert np.abs(u - u2).max() < 1e-12
    assert o.permeability() == pytest.approx(k, rel=1e-12)


def test_alpha_fixed_point_matches_dense_solve_3d():
    solid = np.zeros((3, 4, 4), bool)
    solid[1, 1:3, 1:3] = True
    v, w = velocity_grid(3, 4)
    rho, u, k, resid, delta = solve_dense(solid, 1.0, v, w, lateral="specular", order=2, alpha=0.6)
    assert resid < 1e-11
    o = Oracle(solid, 1.0, v, w, lateral="specular", order=2, threads=1, alpha=0.6)
    o.iterate(2000)
    _, u2 = o.moments()
    assert np.abs(u - u2).max() < 1e-12
    assert o.permeability() == pytest.approx(k, rel=1e-11)


def test_alpha_uniform_state_is_a_fixed_point():
    solid = inputs.cylinder_cell(16, 0.7)
    v, w = velocity_grid(2, 8)
    o = Oracle(solid, 0.2, v, w, jump=0.0, threads=1, alpha=0.5)
    o.set_uniform(1.75)
    o.iterate(3)
    rho, u = o.moments()
    assert np.abs(rho[~solid] - 1.75).max() < 1e-13
    assert np.abs(u).max() < 1e-13


@pytest.mark.parametrize("lateral", ["specular", "periodic"])
def test_alpha_jump_form_equals_source_form(lateral):
    solid = inputs.random_discs(24, 16, seed=1, rmin=2, rmax=4, solid_fraction=0.35)
    v, w = velocity_grid(2, 8)
    a = Oracle(solid, 0.3, v, w, lateral=lateral, form="jump", threads=1, alpha=0.6)
    b = Oracle(solid, 0.3, v, w, lateral=lateral, form="source", threads=1, alpha=0.6)
    a.iterate(40)
    b.iterate(40)
    assert np.abs(a.moments()[1] - b.moments()[1]).max() < 1e-13
    assert np.abs(a.moments()[0] - b.moments()[0]).max() < 1e-12
    assert np.abs(a.wall() - b.wall()).max() < 1e-12


def test_alpha_linear_in_jump_and_raster_equals_wavefront():
    solid = inputs.random_discs(20, 12, seed=5, rmin=2, rmax=3, solid_fraction=0.3)
    v, w = velocity_grid(2, 8)
    a = Oracle(solid, 0.5, v, w, jump=1.0, threads=1, alpha=0.7)
    b = Oracle(solid, 0.5, v, w, jump=2.5, threads=1, alpha=0.7)
    c = Oracle(solid, 0.5, v, w, jump=1.0, threads=1, alpha=0.7, traversal="wavefront")
    for o in (a, b, c):
        o.iterate(25)
    assert np.abs(b.moments()[1] - 2.5 * a.moments()[1]).max() < 1e-13 * np.abs(b.moments()[1]).max() + 1e-15
    assert np.array_equal(a.moments()[1], c.moments()[1])


def test_permeability_grows_as_walls_become_specular():
    solid = inputs.random_discs(24, 16, seed=1, rmin=2, rmax=4, solid_fraction=0.35)
    v, w = velocity_grid(2, 8)
    ks = []
    for alpha in (1.0, 0.8, 0.5):
        o = Oracle(solid, 0.3, v, w, alpha=alpha)
        o.run(1e-9, 20000)
        ks.append(o.permeability())
    assert ks[0] < ks[1] < ks[2]


def test_alpha_one_is_the_default_bitwise_and_bad_alpha_is_rejected():
    solid = inputs.cylinder_cell(16, 0.7)
    v, w = velocity_grid(2, 8)
    a = Oracle(solid, 0.2, v, w, threads=1)
    b = Oracle(solid, 0.2, v, w, threads=1, alpha=1.0)
    a.iterate(5)
    b.iterate(5)
    assert np.array_equal(a.moments()[1], b.moments()[1])
    for bad in (1.5, -0.1):
        with pytest.raises(ValueError):
            Oracle(solid, 0.2, v, w, alpha=bad)
