"""Pins of the oracle's warm start (CPU only).

The paper starts every run from h = 0 (Sec. 3.1).  A warm start replaces that state by the one an
iteration leaves after producing the local linearised equilibrium h0 = rho0 + 2 u0 . v; it must not
change the fixed point.  The pins below use only facts of the discretised equations: equilibria
that are exact fixed points, the zero start, affinity of the iteration map and uniqueness of the
steady solution.  A reflected velocity taken where the same one is needed (or the converse), a
wrong wall-density normalisation, a wrong quadrature of h0 or a missing x1 ramp in the source form
fails at least one of them.  The ghost layers are stored by the iteration's own capture step
(step ii), which the fixed-point pins of the oracle already cover.
"""
import numpy as np
import pytest

from oracle import Oracle, velocity_grid
from paper_1712_01132_gb300 import inputs


def _state(o):
    rho, u = o.moments()
    return rho, u, o.wall()


@pytest.mark.parametrize("form", ["jump", "source"])
@pytest.mark.parametrize("lateral", ["specular", "periodic"])
def test_zero_warm_start_is_the_zero_start(form, lateral):
    solid = inputs.cylinder_cell(12)
    v, w = velocity_grid(2, 4)
    a = Oracle(solid, 0.3, v, w, form=form, lateral=lateral, threads=1)
    b = Oracle(solid, 0.3, v, w, form=form, lateral=lateral, threads=1)
    b.set_initial(np.zeros(solid.shape), np.zeros((2,) + solid.shape))
    a.iterate(4)
    b.iterate(4)
    for x, y in zip(_state(a), _state(b)):
        if form == "jump":
            assert np.array_equal(x, y)
        else:    # the source-form quadrature of h0' = x1 rounds differently from the exact ramp
            assert np.abs(x - y).max() < 1e-13


@pytest.mark.parametrize("lateral", ["specular", "periodic"])
def test_uniform_density_with_walls_is_a_fixed_point(lateral):
    """Zero jump: h = c is an exact solution; walls (Eq. 6) must give rho_s = c."""
    solid = inputs.cylinder_cell(14)
    v, w = velocity_grid(2, 6)
    o = Oracle(solid, 0.2, v, w, jump=0.0, lateral=lateral, threads=1)
    c = 0.37
    o.set_initial(np.full(solid.shape, c), np.zeros((2,) + solid.shape))
    rho, u, wall = _state(o)
    assert np.abs(rho[~solid] - c).max() < 1e-14
    faces = wall != 0
    assert faces.any() and np.abs(wall[faces] - c).max() < 1e-14
    o.iterate(3)
    rho, u, wall = _state(o)
    assert np.abs(rho[~solid] - c).max() < 1e-13
    assert np.abs(u).max() < 1e-13
    assert np.abs(wall[wall != 0] - c).max() < 1e-13


@pytest.mark.parametrize("lateral,U", [("periodic", (0.3, -0.2)), ("specular", (0.3, 0.0))])
def test_uniform_flow_without_walls_is_a_fixed_point(lateral, U):
    """Zero jump, no solid: h = 2 U . v is exact (uniform, so v . grad h = 0; the quadrature gives
    back u = U because sum W v_i v_j = delta_ij / 2).  Periodic lateral faces keep any U; specular
    faces keep U only when U has no normal component."""
    solid = np.zeros((9, 11), dtype=bool)
    v, w = velocity_grid(2, 8)
    o = Oracle(solid, 0.5, v, w, jump=0.0, lateral=lateral, threads=1)
    u0 = np.stack([np.full(solid.shape, U[0]), np.full(solid.shape, U[1])])
    o.set_initial(np.zeros(solid.shape), u0)
    o.iterate(3)
    rho, u = o.moments()
    assert np.abs(rho).max() < 1e-13
    assert np.abs(u - u0).max() < 1e-13


def test_specular_faces_stop_normal_flow():
    """Negative control for the test above: with specular x2 faces a uniform x2 flow is not an
    equilibrium (the reflected velocity is read), so it must change."""
    solid = np.zeros((9, 11), dtype=bool)
    v, w = velocity_grid(2, 8)
    o = Oracle(solid, 0.5, v, w, jump=0.0, lateral="specular", threads=1)
    u0 = np.stack([np.zeros(solid.shape), np.full(solid.shape, 0.2)])
    o.set_initial(np.zeros(solid.shape), u0)
    o.iterate(2)
    _, u = o.moments()
    assert np.abs(u[1] - 0.2).max() > 1e-2


def test_uniform_flow_3d_periodic_is_a_fixed_point():
    solid = np.zeros((5, 6, 7), dtype=bool)
    v, w = velocity_grid(3, 4)
    o = Oracle(solid, 0.5, v, w, jump=0.0, lateral="periodic", threads=1)
    U = (0.1, -0.25, 0.4)
    u0 = np.stack([np.full(solid.shape, x) for x in U])
    o.set_initial(np.zeros(solid.shape), u0)
    o.iterate(2)
    rho, u = o.moments()
    assert np.abs(rho).max() < 1e-13
    assert np.abs(u - u0).max() < 1e-13


@pytest.mark.parametrize("form", ["jump", "source"])
def test_iteration_is_affine_in_the_warm_start(form):
    """The iteration map is affine in the state and h0 is linear in (rho0, u0), so
    S_n(x) + S_n(y) = S_n(x + y) + S_n(0) for every iteration count n."""
    solid = inputs.random_discs(17, 13, seed=4, rmin=2.0, rmax=4.0, solid_fraction=0.35)
    v, w = velocity_grid(2, 4)
    rng = np.random.default_rng(11)
    x = (rng.standard_normal(solid.shape), rng.standard_normal((2,) + solid.shape))
    y = (rng.standard_normal(solid.shape), rng.standard_normal((2,) + solid.shape))
    starts = {"x": x, "y": y, "xy": (x[0] + y[0], x[1] + y[1]),
              "0": (np.zeros(solid.shape), np.zeros((2,) + solid.shape))}
    res = {}
    for name, (r0, u0) in starts.items():
        o = Oracle(solid, 0.4, v, w, form=form, lateral="periodic", threads=1)
        o.set_initial(r0, u0)
        o.iterate(3)
        res[name] = _state(o)
    for i in range(3):
        lhs = res["x"][i] + res["y"][i]
        rhs = res["xy"][i] + res["0"][i]
        assert np.abs(lhs - rhs).max() < 1e-12 * (1 + np.abs(lhs).max())


@pytest.mark.parametrize("lateral", ["specular", "periodic"])
def test_warm_start_does_not_move_the_fixed_point(lateral):
    solid = inputs.cylinder_cell(16)
    v, w = velocity_grid(2, 8)
    a = Oracle(solid, 0.5, v, w, lateral=lateral, threads=1)
    a.run(1e-12, 20000, check_interval=50)
    k0 = a.permeability()
    rho_c, u_c = a.moments()
    b = Oracle(solid, 0.5, v, w, lateral=lateral, threads=1)
    rng = np.random.default_rng(3)
    b.set_initial(0.7 * rho_c + 0.05 * rng.standard_normal(solid.shape),
                  0.7 * u_c + 0.01 * rng.standard_normal(u_c.shape))
    b.run(1e-12, 20000, check_interval=50)
    k1 = b.permeability()
    _, u1 = b.moments()
    assert abs(k1 - k0) <= 1e-8 * abs(k0)
    assert np.abs(u1 - u_c).max() <= 1e-7 * np.abs(u_c).max()

