"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

FP64 path: element-wise agreement at equal iteration counts, tolerance 1e-10 relative (fields to
their max-norm, permeability to itself).  FP32 path: at convergence, permeability within 1e-4
relative and fields within 1e-3 of their max-norm (density compared after removing its fluid mean,
the iteration fixes it only up to a constant).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
from paper_1712_01132_gb300 import dvm, inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def _grid(dims, n):
    return dvm.dvm_gh_velocity_grid(dims, n), oracle.velocity_grid(dims, n)


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _compare_fp64(s, o, prob=0, tol=FP64_TOL):
    rho, u = s.moments(prob)
    rho_o, u_o = o.moments()
    k, _ = s.permeability(prob)
    assert _rel(u, u_o) < tol
    assert np.abs(rho - rho_o).max() < tol * max(1.0, np.abs(rho_o).max())
    assert abs(k - o.permeability()) <= tol * abs(o.permeability())
    wall = s.wall(prob)
    wall_o = o.wall()
    assert np.abs(wall - wall_o).max() < tol * max(1.0, np.abs(wall_o).max())


@pytest.mark.parametrize("lateral", ["periodic", "specular"])
def test_cylinder_cell_fp64_matches_oracle(lateral):
    """32x32 periodic cell with a centred cylinder (porosity 0.7), 16x16 velocities, Kn = 0.1."""
    mask = inputs.cylinder_cell(32, 0.7)
    (v, w), (vo, wo) = _grid(2, 16)
    s = dvm.Solver(mask, 0.1, v, w, precision="fp64", lateral=lateral)
    o = oracle.Oracle(mask, 0.1, vo, wo, lateral=lateral)
    for n in (1, 2, 37):
        s.step(n)
        s.sync()
        o.iterate(n)
        _compare_fp64(s, o)


def test_cylinder_cell_fp64_to_convergence():
    """The configuration's stopping rule: Err < 1e-8 or 2000 iterations."""
    mask = inputs.cylinder_cell(32, 0.7)
    (v, w), (vo, wo) = _grid(2, 16)
    s = dvm.Solver(mask, 0.1, v, w, precision="fp64", lateral="periodic")
    st, it, err = s.iterate(2000, 1e-8)
    assert st == dvm.DVM_OK and err < 1e-8
    o = oracle.Oracle(mask, 0.1, vo, wo, lateral="periodic")
    it_o, k_o, err_o = o.run(1e-8, 2000)
    assert it == it_o
    _compare_fp64(s, o)


@pytest.mark.parametrize("shape,seed", [((29, 37), 1), ((20, 45), 2), ((41, 23), 3)])
@pytest.mark.parametrize("lateral", ["periodic", "specular"])
def test_ragged_random_media_fp64(shape, seed, lateral):
    """Sizes that are not multiples of the tiles, thin walls, corners; several tiles and bands."""
    n2, n1 = shape
    mask = inputs.random_discs(n1, n2, seed=seed, rmin=1.5, rmax=4, solid_fraction=0.35)
    (v, w), (vo, wo) = _grid(2, 8)
    s = dvm.Solver(mask, 0.3, v, w, precision="fp64", lateral=lateral, band_rows=5)
    o = oracle.Oracle(mask, 0.3, vo, wo, lateral=lateral)
    s.step(25)
    s.sync()
    o.iterate(25)
    _compare_fp64(s, o)


def test_first_order_stencil_fp64():
    mask = inputs.random_discs(40, 24, seed=4, rmin=2, rmax=4, solid_fraction=0.3)
    (v, w), (vo, wo) = _grid(2, 8)
    s = dvm.Solver(mask, 0.2, v, w, precision="fp64", stencil_order=1, lateral="specular")
    o = oracle.Oracle(mask, 0.2, vo, wo, order=1, lateral="specular")
    s.step(30)
    s.sync()
    o.iterate(30)
    _compare_fp64(s, o)


def test_thin_walls_and_single_voxels_fp64():
    """One-voxel solid lines and isolated solid voxels: first-order switches on both sides."""
    mask = np.zeros((18, 21), bool)
    mask[4, 2:15] = True        # thin horizontal wall
    mask[6:14, 10] = True       # thin vertical wall
    mask[15, 3] = True          # isolated voxel
    mask[1, 19] = True
    (v, w), (vo, wo) = _grid(2, 8)
    for lateral in ("specular", "periodic"):
        s = dvm.Solver(mask, 0.5, v, w, precision="fp64", lateral=lateral, band_rows=3)
        o = oracle.Oracle(mask, 0.5, vo, wo, lateral=lateral)
        s.step(20)
        s.sync()
        o.iterate(20)
        _compare_fp64(s, o)


def test_tile_and_band_shapes_give_identical_bits():
    """The wavefront partition of the sweep does not change any result bit."""
    mask = inputs.random_discs(53, 35, seed=7, rmin=2, rmax=5, solid_fraction=0.4)
    (v, w), _ = _grid(2, 16)
    ref = None
    shapes = {"fp64": ((8, 8), (16, 3), (8, 35), (16, 1), (8, 17)),
              "fp32": ((8, 8), (4, 3), (8, 35), (4, 1), (8, 17), (4, 32), (16, 8), (16, 3), (16, 1))}
    for prec in ("fp64", "fp32"):
        ref = None
        for t1, rows in shapes[prec]:
            s = dvm.Solver(mask, 0.2, v, w, precision=prec, tile_x1=t1, band_rows=rows)
            s.step(9)
            s.sync()
            rho, u = s.moments()
            wall = s.wall()
            if ref is None:
                ref = (rho, u, wall)
            else:
                assert np.array_equal(ref[0], rho) and np.array_equal(ref[1], u) and np.array_equal(ref[2], wall)
            s.close()


def test_batch_of_uneven_problems_fp64():
    """One context, three geometries of different sizes and Knudsen numbers."""
    masks = [inputs.random_discs(30, 22, seed=11, rmin=2, rmax=4, solid_fraction=0.3),
             inputs.cylinder_cell(32, 0.7),
             inputs.random_discs(47, 19, seed=12, rmin=2, rmax=3, solid_fraction=0.35)]
    kns = [0.05, 0.1, 1.0]
    (v, w), (vo, wo) = _grid(2, 8)
    s = dvm.Solver(masks, kns, v, w, precision="fp64", lateral="periodic")
    s.step(15)
    s.sync()
    for b, (m, kn) in enumerate(zip(masks, kns)):
        o = oracle.Oracle(m, kn, vo, wo, lateral="periodic")
        o.iterate(15)
        _compare_fp64(s, o, prob=b)


@pytest.mark.parametrize("kn", [0.1, 1.0])
def test_fp32_at_convergence(kn):
    """Reduced precision: converged permeability within 1e-4 and fields within 1e-3."""
    mask = inputs.random_discs(96, 80, seed=21, rmin=6, rmax=12, solid_fraction=0.5)
    (v, w), (vo, wo) = _grid(2, 16)
    s = dvm.Solver(mask, kn, v, w, precision="fp32", lateral="periodic")
    st, it, err = s.iterate(6000, 1e-7)
    assert st == dvm.DVM_OK
    o = oracle.Oracle(mask, kn, vo, wo, lateral="periodic")
    o.run(1e-10, 20000)
    k, _ = s.permeability()
    assert abs(k - o.permeability()) <= 1e-4 * abs(o.permeability())
    rho, u = s.moments()
    rho_o, u_o = o.moments()
    fl = ~mask
    assert _rel(u, u_o) < 1e-3
    d = (rho - rho[fl].mean()) * fl
    d_o = (rho_o - rho_o[fl].mean()) * fl
    assert _rel(d, d_o) < 1e-3


def test_full_size_kn_sweep_fp32_first_iterations():
    """512x512 overlapping-disc medium, 32x32 velocities, Kn in {0.01, 0.1, 1, 10}, one batched
    context as the benchmark runs it: the first iterations agree element-wise with the oracle."""
    mask = inputs.random_discs(512, 512, seed=0)
    kns = [0.01, 0.1, 1.0, 10.0]
    (v, w), (vo, wo) = _grid(2, 32)
    s = dvm.Solver([mask] * 4, kns, v, w, precision="fp32", lateral="periodic")
    s.step(2)
    s.sync()
    for b, kn in enumerate(kns):
        o = oracle.Oracle(mask, kn, vo, wo, lateral="periodic")
        o.iterate(2)
        rho, u = s.moments(b)
        rho_o, u_o = o.moments()
        assert _rel(u, u_o) < 1e-4
        assert np.abs(rho - rho_o).max() < 1e-5
        k, _ = s.permeability(b)
        assert abs(k - o.permeability()) <= 1e-4 * abs(o.permeability())


def test_blocked_geometry_has_zero_permeability():
    """A solid wall across the whole x1 period stops the flow: k -> 0."""
    mask = np.zeros((16, 20), bool)
    mask[:, 9] = True
    (v, w), _ = _grid(2, 8)
    s = dvm.Solver(mask, 0.5, v, w, precision="fp64")
    s.iterate(3000, 1e-12)
    _, u = s.moments()
    assert abs(s.permeability()[0]) < 1e-9
    assert np.abs(u[0]).max() < 1e-8


def test_bounded_wait_expires_with_status_and_context_survives():
    """A progress flag that nothing sets: the waiting band gives up after the bound, the call
    reports DVM_ETIMEOUT, and the same context iterates normally afterwards."""
    mask = inputs.cylinder_cell(32, 0.7)
    (v, w), _ = _grid(2, 8)
    s = dvm.Solver(mask, 0.1, v, w, precision="fp64", band_rows=8)
    s.debug_set_wait(50_000_000, withhold_item=0)        # 50 ms; item 0 = band 0 of quadrant 0
    s.step(1)
    with pytest.raises(dvm.DvmError) as ei:
        s.sync()
    assert ei.value.status == dvm.DVM_ETIMEOUT
    s.debug_set_wait(2_000_000_000, withhold_item=-1)
    s.step(3)
    s.sync()
    rho, u = s.moments()
    assert np.isfinite(u).all()


# ----------------------------------------------------------------------------------------- 3D

def _rock3d(n3, n2, n1, seed, frac=0.25):
    rng = np.random.default_rng(seed)
    solid = rng.random((n3, n2, n1)) < frac
    solid[:, :, 0] = False          # keep an open x1 path so the problem has flow
    return solid


@pytest.mark.parametrize("lateral", ["periodic", "specular"])
def test_3d_fp64_matches_oracle(lateral):
    """Octant sweeps, x2/x3 pencil edges and ghosts: 3D random medium, 8^3 velocities."""
    mask = _rock3d(9, 10, 11, seed=3)
    (v, w), (vo, wo) = _grid(3, 8)
    s = dvm.Solver(mask, 0.4, v, w, precision="fp64", lateral=lateral, band_rows=3)
    o = oracle.Oracle(mask, 0.4, vo, wo, lateral=lateral)
    for n in (1, 6):
        s.step(n)
        s.sync()
        o.iterate(n)
        _compare_fp64(s, o)


def test_3d_velocity_groups_fp64():
    """16^3 velocities: 512 per octant are split into two independent velocity groups."""
    mask = _rock3d(6, 7, 8, seed=5, frac=0.2)
    (v, w), (vo, wo) = _grid(3, 16)
    s = dvm.Solver(mask, 0.8, v, w, precision="fp64", lateral="periodic", band_rows=4)
    o = oracle.Oracle(mask, 0.8, vo, wo, lateral="periodic")
    s.step(4)
    s.sync()
    o.iterate(4)
    _compare_fp64(s, o)


def test_3d_pencil_shapes_give_identical_bits():
    mask = _rock3d(10, 9, 13, seed=8)
    (v, w), _ = _grid(3, 8)
    for prec in ("fp64", "fp32"):
        ref = None
        for t1, rows in ((8, 4), (4, 2), (8, 3), (4, 10), (8, 1)):
            s = dvm.Solver(mask, 0.3, v, w, precision=prec, tile_x1=t1, band_rows=rows)
            s.step(5)
            s.sync()
            rho, u = s.moments()
            if ref is None:
                ref = (rho, u)
            else:
                assert np.array_equal(ref[0], rho) and np.array_equal(ref[1], u)
            s.close()


def test_3d_fp32_at_convergence():
    mask = inputs.gaussian_rock(16, seed=2, corr_len=2.0, porosity=0.5)
    (v, w), (vo, wo) = _grid(3, 8)
    s = dvm.Solver(mask, 0.5, v, w, precision="fp32", lateral="periodic")
    st, it, err = s.iterate(4000, 1e-7)
    assert st == dvm.DVM_OK
    o = oracle.Oracle(mask, 0.5, vo, wo, lateral="periodic")
    o.run(1e-10, 20000)
    k, _ = s.permeability()
    assert abs(k - o.permeability()) <= 1e-4 * abs(o.permeability())
    _, u = s.moments()
    _, u_o = o.moments()
    assert _rel(u, u_o) < 1e-3


def test_full_size_3d_rock_fp32_first_iterations():
    """128^3 Gaussian-field rock (correlation length 8, porosity 0.35, percolating cluster kept),
    16^3 = 4096 velocities, Kn = 0.5: the first iterations agree element-wise with the oracle."""
    mask = inputs.gaussian_rock(128, seed=0, corr_len=8.0, porosity=0.35)
    (v, w), (vo, wo) = _grid(3, 16)
    s = dvm.Solver(mask, 0.5, v, w, precision="fp32", lateral="periodic")
    s.step(2)
    s.sync()
    o = oracle.Oracle(mask, 0.5, vo, wo, lateral="periodic")
    o.iterate(2)
    rho, u = s.moments()
    rho_o, u_o = o.moments()
    assert _rel(u, u_o) < 1e-4
    assert np.abs(rho - rho_o).max() < 1e-5
    k, _ = s.permeability()
    assert abs(k - o.permeability()) <= 1e-4 * abs(o.permeability())
