"""GPU parity of Maxwell diffuse-specular walls with accommodation alpha < 1 (Eq. 5, 2D): the wall
value of molecules leaving a wall is alpha rho_s + (1 - alpha) h(x_f, reflected v) of the previous
iteration.  Compared with the oracle's alpha option element by element at equal iteration counts
(FP64 1e-10, FP32 1e-4), with subdomains, a warm start, a checkpoint and a batch; tile shapes do not
change the bits; invalid uses are rejected."""
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
    return dvm.dvm_gh_velocity_grid(2, n), oracle.velocity_grid(2, n)


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _compare(s, o, prob=0, tol=FP64_TOL):
    rho, u = s.moments(prob)
    rho_o, u_o = o.moments()
    assert _rel(u, u_o) < tol
    assert np.abs(rho - rho_o).max() < tol * max(1.0, np.abs(rho_o).max())
    k, _ = s.permeability(prob)
    assert abs(k - o.permeability()) <= tol * abs(o.permeability())
    wall, wall_o = s.wall(prob), o.wall()
    assert np.abs(wall - wall_o).max() < tol * max(1.0, np.abs(wall_o).max())


@pytest.mark.parametrize("alpha", [0.6, 0.3])
@pytest.mark.parametrize("lateral", ["periodic", "specular"])
@pytest.mark.parametrize("t1,rows", [(8, 4), (16, 3)])
def test_alpha_fp64_matches_oracle(alpha, lateral, t1, rows):
    mask = inputs.random_discs(37, 29, seed=1, rmin=1.5, rmax=4, solid_fraction=0.35)
    (v, w), (vo, wo) = _grid(8)
    s = dvm.Solver(mask, 0.3, v, w, precision="fp64", lateral=lateral, tile_x1=t1, band_rows=rows,
                   specular_fraction=1 - alpha)
    o = oracle.Oracle(mask, 0.3, vo, wo, lateral=lateral, alpha=alpha)
    for n in (1, 2, 5):
        s.step(n)
        s.sync()
        o.iterate(n)
        _compare(s, o)


def test_alpha_with_subdomains_fp64():
    mask = inputs.random_discs(33, 28, seed=6, rmin=1.5, rmax=4, solid_fraction=0.35)
    (v, w), (vo, wo) = _grid(8)
    s = dvm.Solver(mask, 0.2, v, w, precision="fp64", lateral="specular", band_rows=3, subdomains=(3, 2, 1),
                   specular_fraction=0.5)
    o = oracle.Oracle(mask, 0.2, vo, wo, lateral="specular", decomposition=(3, 2), alpha=0.5)
    s.step(4)
    s.sync()
    o.iterate(4)
    _compare(s, o)


def test_alpha_warm_start_and_checkpoint_fp64():
    mask = inputs.random_discs(30, 22, seed=11, rmin=2, rmax=4, solid_fraction=0.3)
    (v, w), (vo, wo) = _grid(8)
    rng = np.random.default_rng(2)
    r0 = 0.2 * rng.standard_normal(mask.shape)
    u0 = 0.05 * rng.standard_normal((2,) + mask.shape)
    s = dvm.Solver(mask, 0.2, v, w, precision="fp64", lateral="periodic", specular_fraction=0.4)
    o = oracle.Oracle(mask, 0.2, vo, wo, lateral="periodic", alpha=0.6)
    s.step(1)
    s.set_initial(r0, u0)
    o.set_initial(r0, u0)
    _compare(s, o)
    s.step(3)
    s.sync()
    o.iterate(3)
    _compare(s, o)
    blob = s.get_state()
    s.step(3)
    s.sync()
    ref = s.moments()
    t = dvm.Solver(mask, 0.2, v, w, precision="fp64", lateral="periodic", specular_fraction=0.4)
    t.set_state(blob)
    t.step(3)
    t.sync()
    assert np.array_equal(ref[1], t.moments()[1])


def test_alpha_batch_fp32_first_iterations():
    masks = [inputs.random_discs(30, 22, seed=11, rmin=2, rmax=4, solid_fraction=0.3),
             inputs.cylinder_cell(32, 0.7),
             inputs.random_discs(47, 19, seed=12, rmin=2, rmax=3, solid_fraction=0.35)]
    kns = [0.05, 0.1, 1.0]
    (v, w), (vo, wo) = _grid(16)
    s = dvm.Solver(masks, kns, v, w, precision="fp32", lateral="periodic", specular_fraction=0.3)
    s.step(4)
    s.sync()
    for b, (m, kn) in enumerate(zip(masks, kns)):
        o = oracle.Oracle(m, kn, vo, wo, lateral="periodic", alpha=0.7)
        o.iterate(4)
        rho, u = s.moments(b)
        rho_o, u_o = o.moments()
        assert _rel(u, u_o) < 1e-4
        assert np.abs(rho - rho_o).max() < 1e-5 * max(1.0, np.abs(rho_o).max())
        k, _ = s.permeability(b)
        assert abs(k - o.permeability()) <= 1e-4 * abs(o.permeability())


@pytest.mark.parametrize("precision,shapes", [("fp64", ((8, 8), (16, 3), (8, 35))), ("fp32", ((8, 8), (4, 3), (8, 17)))])
def test_alpha_bits_independent_of_tiles(precision, shapes):
    mask = inputs.random_discs(53, 35, seed=7, rmin=2, rmax=5, solid_fraction=0.4)
    (v, w), _ = _grid(16)
    ref = None
    for t1, rows in shapes:
        s = dvm.Solver(mask, 0.2, v, w, precision=precision, tile_x1=t1, band_rows=rows, specular_fraction=0.5)
        s.step(6)
        s.sync()
        got = s.moments()
        if ref is None:
            ref = got
        else:
            assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])


def test_alpha_options_are_validated():
    mask = inputs.cylinder_cell(16, 0.7)
    (v, w), _ = _grid(8)
    for bad in (-0.1, 1.5, float("nan")):
        with pytest.raises(dvm.DvmError):
            dvm.Solver(mask, 0.2, v, w, specular_fraction=bad)
    rock = inputs.gaussian_rock(8, seed=1, corr_len=1.5, porosity=0.6)
    v3, w3 = dvm.dvm_gh_velocity_grid(3, 4)
    with pytest.raises(dvm.DvmError):
        dvm.Solver(rock, 0.2, v3, w3, precision="bf16_store", specular_fraction=0.5)


# ----------------------------------------------------------------------------------------- 3D

def _rock(n3, n2, n1, seed, frac=0.25):
    rng = np.random.default_rng(seed)
    solid = rng.random((n3, n2, n1)) < frac
    solid[:, :, 0] = False
    return solid


def _grid3(n):
    return dvm.dvm_gh_velocity_grid(3, n), oracle.velocity_grid(3, n)


@pytest.mark.parametrize("lateral", ["periodic", "specular"])
@pytest.mark.parametrize("t1,rows", [(4, 2), (8, 4)])
def test_alpha_3d_fp64_matches_oracle(lateral, t1, rows):
    mask = _rock(9, 10, 11, seed=3)
    (v, w), (vo, wo) = _grid3(8)
    s = dvm.Solver(mask, 0.4, v, w, precision="fp64", lateral=lateral, tile_x1=t1, band_rows=rows,
                   specular_fraction=0.4)
    o = oracle.Oracle(mask, 0.4, vo, wo, lateral=lateral, alpha=0.6)
    for n in (1, 3):
        s.step(n)
        s.sync()
        o.iterate(n)
        _compare(s, o)


def test_alpha_3d_with_subdomains_tau_and_groups_fp64():
    """alpha < 1 together with lagged-halo subdomains, the temperature term and two velocity groups
    per octant."""
    mask = _rock(7, 8, 9, seed=5, frac=0.2)
    (v, w), (vo, wo) = _grid3(16)
    s = dvm.Solver(mask, 0.8, v, w, precision="fp64", lateral="periodic", band_rows=3, subdomains=(2, 1, 2),
                   temperature_term=True, specular_fraction=0.3)
    o = oracle.Oracle(mask, 0.8, vo, wo, lateral="periodic", decomposition=(2, 1, 2), tau=True, alpha=0.7)
    s.step(3)
    s.sync()
    o.iterate(3)
    _compare(s, o)
    assert np.abs(s.temperature() - o.temperature()).max() < FP64_TOL * max(1.0, np.abs(o.temperature()).max())


def test_alpha_3d_warm_start_and_checkpoint_fp64():
    mask = _rock(8, 9, 10, seed=7)
    (v, w), (vo, wo) = _grid3(8)
    rng = np.random.default_rng(4)
    r0 = 0.2 * rng.standard_normal(mask.shape)
    u0 = 0.05 * rng.standard_normal((3,) + mask.shape)
    s = dvm.Solver(mask, 0.3, v, w, precision="fp64", lateral="specular", band_rows=2, specular_fraction=0.5)
    o = oracle.Oracle(mask, 0.3, vo, wo, lateral="specular", alpha=0.5)
    s.step(1)
    s.set_initial(r0, u0)
    o.set_initial(r0, u0)
    _compare(s, o)
    s.step(2)
    s.sync()
    o.iterate(2)
    _compare(s, o)
    blob = s.get_state()
    s.step(2)
    s.sync()
    ref = s.moments()
    t = dvm.Solver(mask, 0.3, v, w, precision="fp64", lateral="specular", band_rows=2, specular_fraction=0.5)
    t.set_state(blob)
    t.step(2)
    t.sync()
    assert np.array_equal(ref[1], t.moments()[1])


def test_alpha_3d_fp32_matches_oracle_and_keeps_bits_across_shapes():
    mask = _rock(10, 12, 13, seed=11, frac=0.3)
    (v, w), (vo, wo) = _grid3(8)
    o = oracle.Oracle(mask, 0.2, vo, wo, lateral="periodic", alpha=0.6)
    o.iterate(3)
    ref = None
    for t1, rows, gw in ((4, 3, 0), (8, 2, 0), (4, 5, 4)):
        s = dvm.Solver(mask, 0.2, v, w, precision="fp32", lateral="periodic", tile_x1=t1, band_rows=rows,
                       group_warps=gw, specular_fraction=0.4)
        s.step(3)
        s.sync()
        rho, u = s.moments()
        rho_o, u_o = o.moments()
        assert _rel(u, u_o) < 1e-4
        assert np.abs(rho - rho_o).max() < 1e-5 * max(1.0, np.abs(rho_o).max())
        if ref is None:
            ref = (rho, u)
        else:
            assert np.array_equal(ref[1], u)
