"""GPU tests of the lagged-halo subdomains in 3D (the paper's MPI c1 x c2 x c3 decomposition,
Sec. 3.2, emulated on one GPU) against the oracle's decomposition at equal iteration counts, and the
invariances the decomposition must keep: results independent of tile, pencil and warp shapes, the
checkpoint round trip, the same fixed point with more iterations."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
from paper_1712_01132_gb300 import dvm, inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def _grid(n):
    return dvm.dvm_gh_velocity_grid(3, n), oracle.velocity_grid(3, n)


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _rock(n3, n2, n1, seed, frac=0.25):
    rng = np.random.default_rng(seed)
    solid = rng.random((n3, n2, n1)) < frac
    solid[:, :, 0] = False          # keep an open x1 path so the problem has flow
    return solid


def _compare(s, o, tol=FP64_TOL):
    rho, u = s.moments()
    rho_o, u_o = o.moments()
    assert _rel(u, u_o) < tol
    assert np.abs(rho - rho_o).max() < tol * max(1.0, np.abs(rho_o).max())
    k, _ = s.permeability()
    assert abs(k - o.permeability()) <= tol * abs(o.permeability())
    wall, wall_o = s.wall(), o.wall()
    assert np.abs(wall - wall_o).max() < tol * max(1.0, np.abs(wall_o).max())


@pytest.mark.parametrize("dec", [(1, 2, 1), (1, 1, 3), (2, 1, 1), (2, 2, 2), (3, 2, 4)])
@pytest.mark.parametrize("lateral", ["periodic", "specular"])
@pytest.mark.parametrize("t1,rows", [(4, 2), (8, 4)])
def test_3d_subdomains_fp64_match_oracle(dec, lateral, t1, rows):
    mask = _rock(9, 10, 11, seed=3)
    (v, w), (vo, wo) = _grid(8)
    s = dvm.Solver(mask, 0.4, v, w, precision="fp64", lateral=lateral, tile_x1=t1, band_rows=rows, subdomains=dec)
    o = oracle.Oracle(mask, 0.4, vo, wo, lateral=lateral, decomposition=dec)
    for n in (1, 2, 4):
        s.step(n)
        s.sync()
        o.iterate(n)
        _compare(s, o)


def test_3d_subdomains_velocity_groups_fp64():
    """16^3 velocities: two velocity groups per octant, each with the decomposition."""
    mask = _rock(7, 8, 9, seed=5, frac=0.2)
    (v, w), (vo, wo) = _grid(16)
    s = dvm.Solver(mask, 0.8, v, w, precision="fp64", lateral="periodic", band_rows=3, subdomains=(2, 2, 3))
    o = oracle.Oracle(mask, 0.8, vo, wo, lateral="periodic", decomposition=(2, 2, 3))
    s.step(3)
    s.sync()
    o.iterate(3)
    _compare(s, o)


def test_3d_subdomains_warm_start_and_checkpoint_fp64():
    mask = _rock(8, 9, 10, seed=7)
    (v, w), (vo, wo) = _grid(8)
    rng = np.random.default_rng(4)
    r0 = 0.2 * rng.standard_normal(mask.shape)
    u0 = 0.05 * rng.standard_normal((3,) + mask.shape)
    dec = (2, 3, 2)
    s = dvm.Solver(mask, 0.3, v, w, precision="fp64", lateral="specular", band_rows=2, subdomains=dec)
    o = oracle.Oracle(mask, 0.3, vo, wo, lateral="specular", decomposition=dec)
    s.step(1)
    s.set_initial(r0, u0)
    o.set_initial(r0, u0)
    _compare(s, o)
    s.step(2)
    s.sync()
    o.iterate(2)
    _compare(s, o)
    blob = s.get_state()
    s.step(3)
    s.sync()
    ref = s.moments()
    t = dvm.Solver(mask, 0.3, v, w, precision="fp64", lateral="specular", band_rows=2, subdomains=dec)
    t.set_state(blob)
    t.step(3)
    t.sync()
    got = t.moments()
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])


def test_3d_subdomains_fp32_match_oracle_first_iterations():
    mask = _rock(10, 12, 13, seed=11, frac=0.3)
    (v, w), (vo, wo) = _grid(8)
    s = dvm.Solver(mask, 0.2, v, w, precision="fp32", lateral="periodic", band_rows=3, subdomains=(2, 2, 2))
    o = oracle.Oracle(mask, 0.2, vo, wo, lateral="periodic", decomposition=(2, 2, 2))
    s.step(3)
    s.sync()
    o.iterate(3)
    rho, u = s.moments()
    rho_o, u_o = o.moments()
    assert _rel(u, u_o) < 1e-4
    assert np.abs(rho - rho_o).max() < 1e-5 * max(1.0, np.abs(rho_o).max())
    k, _ = s.permeability()
    assert abs(k - o.permeability()) <= 1e-4 * abs(o.permeability())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_3d_subdomains_independent_of_tiles_and_pencils(precision):
    mask = _rock(11, 10, 13, seed=8)
    (v, w), _ = _grid(8)
    ref = None
    for t1, rows in ((8, 4), (4, 2), (8, 3), (4, 10), (8, 1)):
        s = dvm.Solver(mask, 0.3, v, w, precision=precision, tile_x1=t1, band_rows=rows, subdomains=(3, 2, 2))
        s.step(5)
        s.sync()
        got = s.moments()
        if ref is None:
            ref = got
        else:
            assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])


def test_3d_subdomains_keep_the_fixed_point_and_slow_convergence():
    """First-order stencil (consistent discrete system): every lag pattern has the same fixed point;
    more blocks need at least as many iterations."""
    mask = inputs.gaussian_rock(12, seed=2, corr_len=2.0, porosity=0.6)
    (v, w), _ = _grid(8)
    res = {}
    for dec in ((1, 1, 1), (2, 2, 2), (3, 3, 3)):
        s = dvm.Solver(mask, 0.1, v, w, precision="fp64", lateral="periodic", check_interval=10,
                       stencil_order=1, subdomains=dec)
        st, it, err = s.iterate(20000, 1e-10)
        assert st == dvm.DVM_OK
        res[dec] = (it, s.permeability()[0])
    k1 = res[(1, 1, 1)][1]
    for dec in ((2, 2, 2), (3, 3, 3)):
        assert abs(res[dec][1] - k1) <= 1e-8 * abs(k1)
    assert res[(1, 1, 1)][0] <= res[(2, 2, 2)][0] <= res[(3, 3, 3)][0]


def test_3d_subdomain_options_are_validated():
    rock = inputs.gaussian_rock(8, seed=1, corr_len=1.5, porosity=0.6)
    v3, w3 = dvm.dvm_gh_velocity_grid(3, 4)
    for sub in ((5, 1, 1), (1, 5, 1), (1, 1, 5), (1, -1, 1)):
        with pytest.raises(dvm.DvmError):
            dvm.Solver(rock, 0.2, v3, w3, subdomains=sub)
    with pytest.raises(dvm.DvmError):
        dvm.Solver(rock, 0.2, v3, w3, precision="bf16_store", subdomains=(1, 2, 1))
