"""GPU parity of the temperature-term option (3D): the source of Eq. 2 keeps tau (|v|^2 - 3/2)
with tau from Eq. 4.  Compared with the oracle's tau option element by element at equal iteration
counts (FP64 1e-10, FP32 1e-4), with lagged-halo subdomains, velocity groups, a warm start and a
checkpoint round trip; tile and pencil shapes do not change the bits; invalid uses are rejected."""
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
    solid[:, :, 0] = False
    return solid


def _compare(s, o, tol=FP64_TOL):
    rho, u = s.moments()
    rho_o, u_o = o.moments()
    assert _rel(u, u_o) < tol
    assert np.abs(rho - rho_o).max() < tol * max(1.0, np.abs(rho_o).max())
    tau, tau_o = s.temperature(), o.temperature()
    assert np.abs(tau - tau_o).max() < tol * max(1.0, np.abs(tau_o).max())
    k, _ = s.permeability()
    assert abs(k - o.permeability()) <= tol * abs(o.permeability())
    wall, wall_o = s.wall(), o.wall()
    assert np.abs(wall - wall_o).max() < tol * max(1.0, np.abs(wall_o).max())


@pytest.mark.parametrize("lateral", ["periodic", "specular"])
@pytest.mark.parametrize("t1,rows", [(4, 2), (8, 4)])
def test_tau_fp64_matches_oracle(lateral, t1, rows):
    mask = _rock(9, 10, 11, seed=3)
    (v, w), (vo, wo) = _grid(8)
    s = dvm.Solver(mask, 0.4, v, w, precision="fp64", lateral=lateral, tile_x1=t1, band_rows=rows,
                   temperature_term=True)
    o = oracle.Oracle(mask, 0.4, vo, wo, lateral=lateral, tau=True)
    for n in (1, 3):
        s.step(n)
        s.sync()
        o.iterate(n)
        _compare(s, o)
    assert np.abs(o.temperature()).max() > 1e-4       # the term is active


def test_tau_with_subdomains_and_velocity_groups_fp64():
    mask = _rock(7, 8, 9, seed=5, frac=0.2)
    (v, w), (vo, wo) = _grid(16)
    s = dvm.Solver(mask, 0.8, v, w, precision="fp64", lateral="periodic", band_rows=3, subdomains=(2, 1, 2),
                   temperature_term=True)
    o = oracle.Oracle(mask, 0.8, vo, wo, lateral="periodic", decomposition=(2, 1, 2), tau=True)
    s.step(3)
    s.sync()
    o.iterate(3)
    _compare(s, o)


def test_tau_warm_start_and_checkpoint_fp64():
    mask = _rock(8, 9, 10, seed=7)
    (v, w), (vo, wo) = _grid(8)
    rng = np.random.default_rng(4)
    r0 = 0.2 * rng.standard_normal(mask.shape)
    u0 = 0.05 * rng.standard_normal((3,) + mask.shape)
    s = dvm.Solver(mask, 0.3, v, w, precision="fp64", lateral="specular", band_rows=2, temperature_term=True)
    o = oracle.Oracle(mask, 0.3, vo, wo, lateral="specular", tau=True)
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
    ref = (s.moments(), s.temperature())
    t = dvm.Solver(mask, 0.3, v, w, precision="fp64", lateral="specular", band_rows=2, temperature_term=True)
    t.set_state(blob)
    t.step(3)
    t.sync()
    assert np.array_equal(ref[0][1], t.moments()[1]) and np.array_equal(ref[1], t.temperature())


def test_tau_fp32_matches_oracle_first_iterations():
    mask = _rock(10, 12, 13, seed=11, frac=0.3)
    (v, w), (vo, wo) = _grid(8)
    s = dvm.Solver(mask, 0.2, v, w, precision="fp32", lateral="periodic", band_rows=3, temperature_term=True)
    o = oracle.Oracle(mask, 0.2, vo, wo, lateral="periodic", tau=True)
    s.step(3)
    s.sync()
    o.iterate(3)
    rho, u = s.moments()
    rho_o, u_o = o.moments()
    assert _rel(u, u_o) < 1e-4
    assert np.abs(rho - rho_o).max() < 1e-5 * max(1.0, np.abs(rho_o).max())
    assert np.abs(s.temperature() - o.temperature()).max() < 1e-5
    k, _ = s.permeability()
    assert abs(k - o.permeability()) <= 1e-4 * abs(o.permeability())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tau_bits_independent_of_tiles_and_pencils(precision):
    mask = _rock(11, 10, 13, seed=8)
    (v, w), _ = _grid(8)
    ref = None
    for t1, rows in ((8, 4), (4, 2), (8, 3), (4, 10)):
        s = dvm.Solver(mask, 0.3, v, w, precision=precision, tile_x1=t1, band_rows=rows, temperature_term=True)
        s.step(5)
        s.sync()
        got = (s.moments()[1], s.temperature())
        if ref is None:
            ref = got
        else:
            assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])


def test_tau_option_is_validated():
    (v2, w2) = dvm.dvm_gh_velocity_grid(2, 8)
    with pytest.raises(dvm.DvmError):
        dvm.Solver(inputs.cylinder_cell(16, 0.7), 0.2, v2, w2, temperature_term=True)
    rock = inputs.gaussian_rock(8, seed=1, corr_len=1.5, porosity=0.6)
    v3, w3 = dvm.dvm_gh_velocity_grid(3, 4)
    with pytest.raises(dvm.DvmError):
        dvm.Solver(rock, 0.2, v3, w3, precision="bf16_store", temperature_term=True)
    s = dvm.Solver(rock, 0.2, v3, w3, precision="fp32")
    with pytest.raises(dvm.DvmError):
        s.temperature()
