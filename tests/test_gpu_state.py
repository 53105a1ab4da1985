"""GPU tests of the warm start and of checkpoint / resume, through the C ABI.

Warm start: the CUDA path's state after dvm_set_initial matches the oracle's ora_set_initial
element-wise (FP64: 1e-10 relative; FP32: the reduced-precision bounds), before and after
iterations.  Checkpoint: a state written by dvm_get_state and loaded by dvm_set_state into a fresh
context continues bit for bit.
"""
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


def _compare(s, o, tol, prob=0):
    rho, u = s.moments(prob)
    rho_o, u_o = o.moments()
    assert _rel(u, u_o) < tol
    assert np.abs(rho - rho_o).max() < tol * max(1.0, np.abs(rho_o).max())
    k, _ = s.permeability(prob)
    assert abs(k - o.permeability()) <= tol * abs(o.permeability())
    wall, wall_o = s.wall(prob), o.wall()
    assert np.abs(wall - wall_o).max() < tol * max(1.0, np.abs(wall_o).max())


def _smooth_start(shape, dims, seed, amp_rho=0.3, amp_u=0.05):
    """Seeded smooth fields (a few Fourier modes) for rho0 and u0."""
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[np.arange(n) / n for n in shape], indexing="ij")
    def field(amp):
        f = np.zeros(shape)
        for _ in range(4):
            kv = rng.integers(1, 3, size=len(shape))
            ph = rng.uniform(0, 2 * np.pi)
            f += np.cos(2 * np.pi * sum(k * g for k, g in zip(kv, grids)) + ph)
        return amp * f / 4
    return field(amp_rho), np.stack([field(amp_u) for _ in range(dims)])


@pytest.mark.parametrize("lateral", ["periodic", "specular"])
@pytest.mark.parametrize("shape,seed", [((32, 32), None), ((37, 45), 5)])
def test_warm_start_2d_fp64_matches_oracle(lateral, shape, seed):
    if seed is None:
        mask = inputs.cylinder_cell(32, 0.7)
    else:
        mask = inputs.random_discs(shape[1], shape[0], seed=seed, rmin=1.5, rmax=4, solid_fraction=0.35)
    (v, w), (vo, wo) = _grid(2, 8)
    rho0, u0 = _smooth_start(mask.shape, 2, seed=17)
    s = dvm.Solver(mask, 0.2, v, w, precision="fp64", lateral=lateral, band_rows=5)
    o = oracle.Oracle(mask, 0.2, vo, wo, lateral=lateral)
    s.set_initial(rho0, u0)
    o.set_initial(rho0, u0)
    _compare(s, o, FP64_TOL)
    for n in (1, 4):
        s.step(n)
        s.sync()
        o.iterate(n)
        _compare(s, o, FP64_TOL)


def test_warm_start_after_iterations_uses_the_current_parity():
    """A warm start in the middle of a run (odd iteration count) writes the ghost layers the next
    sweep reads."""
    mask = inputs.cylinder_cell(24, 0.7)
    (v, w), (vo, wo) = _grid(2, 8)
    rho0, u0 = _smooth_start(mask.shape, 2, seed=3)
    s = dvm.Solver(mask, 0.4, v, w, precision="fp64", lateral="specular")
    s.step(3)
    s.set_initial(rho0, u0)
    o = oracle.Oracle(mask, 0.4, vo, wo, lateral="specular")
    o.set_initial(rho0, u0)
    s.step(2)
    s.sync()
    o.iterate(2)
    _compare(s, o, FP64_TOL)


@pytest.mark.parametrize("lateral", ["periodic", "specular"])
@pytest.mark.parametrize("n", [4, 16])
def test_warm_start_3d_fp64_matches_oracle(lateral, n):
    """n = 16 puts 512 velocities in an octant: two velocity groups per octant."""
    mask = inputs.gaussian_rock(9, seed=4, corr_len=1.5, porosity=0.55) if n == 4 else \
        inputs.gaussian_rock(6, seed=1, corr_len=1.2, porosity=0.6)
    (v, w), (vo, wo) = _grid(3, n)
    rho0, u0 = _smooth_start(mask.shape, 3, seed=9)
    s = dvm.Solver(mask, 0.3, v, w, precision="fp64", lateral=lateral, band_rows=2)
    o = oracle.Oracle(mask, 0.3, vo, wo, lateral=lateral)
    s.set_initial(rho0, u0)
    o.set_initial(rho0, u0)
    _compare(s, o, FP64_TOL)
    s.step(2)
    s.sync()
    o.iterate(2)
    _compare(s, o, FP64_TOL)


def test_warm_start_fp32_first_iterations():
    mask = inputs.random_discs(96, 80, seed=21, rmin=6, rmax=12, solid_fraction=0.5)
    (v, w), (vo, wo) = _grid(2, 16)
    rho0, u0 = _smooth_start(mask.shape, 2, seed=8)
    s = dvm.Solver(mask, 0.1, v, w, precision="fp32", lateral="periodic")
    o = oracle.Oracle(mask, 0.1, vo, wo, lateral="periodic")
    s.set_initial(rho0, u0)
    o.set_initial(rho0, u0)
    s.step(3)
    s.sync()
    o.iterate(3)
    rho, u = s.moments()
    rho_o, u_o = o.moments()
    assert _rel(u, u_o) < 1e-4
    assert np.abs(rho - rho_o).max() < 1e-5 * max(1.0, np.abs(rho_o).max())


def test_warm_start_fp32_converges_to_the_same_permeability():
    mask = inputs.random_discs(64, 48, seed=12, rmin=4, rmax=8, solid_fraction=0.45)
    (v, w), (vo, wo) = _grid(2, 16)
    o = oracle.Oracle(mask, 0.5, vo, wo, lateral="periodic")
    o.run(1e-11, 20000)
    rho_c, u_c = o.moments()
    s = dvm.Solver(mask, 0.5, v, w, precision="fp32", lateral="periodic")
    s.set_initial(0.8 * rho_c, 0.8 * u_c)
    st, it, err = s.iterate(6000, 1e-8)
    assert st == dvm.DVM_OK
    k, _ = s.permeability()
    assert abs(k - o.permeability()) <= 1e-4 * abs(o.permeability())
    _, u = s.moments()
    assert _rel(u, u_c) < 1e-3


def test_warm_start_touches_only_its_problem():
    masks = [inputs.cylinder_cell(24, 0.7), inputs.random_discs(30, 20, seed=2, rmin=2, rmax=4, solid_fraction=0.4)]
    (v, w), _ = _grid(2, 8)
    a = dvm.Solver(masks, [0.2, 0.7], v, w, precision="fp64", lateral="periodic")
    b = dvm.Solver(masks, [0.2, 0.7], v, w, precision="fp64", lateral="periodic")
    rho0, u0 = _smooth_start(masks[1].shape, 2, seed=1)
    b.set_initial(rho0, u0, prob=1)
    a.step(5)
    b.step(5)
    ra, ua = a.moments(0)
    rb, ub = b.moments(0)
    assert np.array_equal(ra, rb) and np.array_equal(ua, ub)
    assert not np.array_equal(a.moments(1)[1], b.moments(1)[1])


def test_warm_start_rejects_non_finite_values():
    mask = inputs.cylinder_cell(16, 0.7)
    (v, w), _ = _grid(2, 4)
    s = dvm.Solver(mask, 0.2, v, w, precision="fp64")
    rho0 = np.zeros(mask.shape)
    rho0[~mask] = np.nan
    with pytest.raises(dvm.DvmError):
        s.set_initial(rho0, np.zeros((2,) + mask.shape))


@pytest.mark.parametrize("dims,precision", [(2, "fp64"), (2, "fp32"), (3, "fp32"), (3, "fp64")])
def test_checkpoint_resume_is_bitwise(dims, precision):
    if dims == 2:
        masks = [inputs.random_discs(45, 37, seed=3, rmin=2, rmax=5, solid_fraction=0.4),
                 inputs.cylinder_cell(32, 0.7)]
        (v, w), _ = _grid(2, 16)
    else:
        masks = [inputs.gaussian_rock(10, seed=2, corr_len=1.5, porosity=0.55)]
        (v, w), _ = _grid(3, 8)
    kns = [0.3, 0.05][:len(masks)]
    a = dvm.Solver(masks, kns, v, w, precision=precision, lateral="specular")
    a.iterate(7, 0.0)                      # odd count: the state's ghosts sit at parity 1
    blob = a.get_state()
    a.iterate(5, 0.0)
    b = dvm.Solver(masks, kns, v, w, precision=precision, lateral="specular")
    b.set_state(blob)
    assert b.iterations == 7
    b.iterate(5, 0.0)
    assert b.iterations == a.iterations
    for p in range(len(masks)):
        ra, ua = a.moments(p)
        rb, ub = b.moments(p)
        assert np.array_equal(ra, rb) and np.array_equal(ua, ub)
        assert a.permeability(p) == b.permeability(p)
        assert np.array_equal(a.wall(p), b.wall(p))


def test_set_state_rejects_other_contexts():
    mask = inputs.cylinder_cell(16, 0.7)
    (v, w), _ = _grid(2, 8)
    a = dvm.Solver(mask, 0.2, v, w, precision="fp64")
    a.step(2)
    blob = a.get_state()
    for other in (dict(kn=0.3), dict(precision="fp32"), dict(lateral="periodic")):
        kw = dict(kn=0.2, precision="fp64", lateral="specular")
        kw.update(other)
        kn = kw.pop("kn")
        b = dvm.Solver(mask, kn, v, w, **kw)
        with pytest.raises(dvm.DvmError):
            b.set_state(blob)
    c = dvm.Solver(mask, 0.2, v, w, precision="fp64")
    with pytest.raises(dvm.DvmError):
        c.set_state(blob[:-8])
    bad = bytearray(blob)
    bad[0:8] = b"XXXXXXXX"
    with pytest.raises(dvm.DvmError):
        c.set_state(bytes(bad))
