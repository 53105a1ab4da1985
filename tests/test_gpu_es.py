"""GPU parity of the ES-BGK model option (3D, with the temperature term): the collision frequency
becomes Pr nu and the source also carries (1 - 1/Pr) sum_ij P_ij v_i v_j with the traceless stress
P_ij = 2 sum W (v_i v_j - delta_ij |v|^2 / 3) h.  Compared with the oracle's ES option element by
element at equal iteration counts (FP64 1e-10, FP32 1e-4 on u and k), with velocity groups, a warm
start and a checkpoint round trip; tile and pencil shapes do not change the bits; Pr = 1 gives the
BGK model's bits; invalid uses are rejected."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
from paper_1712_01132_gb300 import dvm, inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
PR = 2.0 / 3.0


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
    q, q_o = s.stress(), o.stress()
    assert np.abs(q - q_o).max() < tol * max(1.0, np.abs(q_o).max())
    k, _ = s.permeability()
    assert abs(k - o.permeability()) <= tol * abs(o.permeability())


@pytest.mark.parametrize("lateral", ["periodic", "specular"])
@pytest.mark.parametrize("t1,rows", [(4, 2), (8, 4)])
def test_es_fp64_matches_oracle(lateral, t1, rows):
    mask = _rock(9, 10, 11, seed=3)
    (v, w), (vo, wo) = _grid(8)
    s = dvm.Solver(mask, 0.4, v, w, precision="fp64", lateral=lateral, tile_x1=t1, band_rows=rows,
                   temperature_term=True, es_prandtl=PR)
    o = oracle.Oracle(mask, 0.4, vo, wo, lateral=lateral, tau=True, es_pr=PR)
    for n in (1, 3):
        s.step(n)
        s.sync()
        o.iterate(n)
        _compare(s, o)
    assert np.abs(o.stress()).max() > 1e-4       # the stress is active


def test_es_velocity_groups_warm_start_and_checkpoint_fp64():
    mask = _rock(7, 8, 9, seed=5, frac=0.2)
    (v, w), (vo, wo) = _grid(16)                     # 512 velocities per octant: 16 groups of 32
    rng = np.random.default_rng(4)
    r0 = 0.2 * rng.standard_normal(mask.shape)
    u0 = 0.05 * rng.standard_normal((3,) + mask.shape)
    s = dvm.Solver(mask, 0.8, v, w, precision="fp64", lateral="specular", band_rows=3, temperature_term=True,
                   es_prandtl=PR)
    o = oracle.Oracle(mask, 0.8, vo, wo, lateral="specular", tau=True, es_pr=PR)
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
    ref = (s.moments()[1], s.stress())
    t = dvm.Solver(mask, 0.8, v, w, precision="fp64", lateral="specular", band_rows=3, temperature_term=True,
                   es_prandtl=PR)
    t.set_state(blob)
    t.step(2)
    t.sync()
    assert np.array_equal(ref[0], t.moments()[1]) and np.array_equal(ref[1], t.stress())


def test_es_fp32_matches_oracle_first_iterations():
    mask = _rock(10, 12, 13, seed=11, frac=0.3)
    (v, w), (vo, wo) = _grid(8)
    s = dvm.Solver(mask, 0.2, v, w, precision="fp32", lateral="periodic", band_rows=3, temperature_term=True,
                   es_prandtl=PR)
    o = oracle.Oracle(mask, 0.2, vo, wo, lateral="periodic", tau=True, es_pr=PR)
    s.step(3)
    s.sync()
    o.iterate(3)
    rho, u = s.moments()
    rho_o, u_o = o.moments()
    assert _rel(u, u_o) < 1e-4
    assert np.abs(rho - rho_o).max() < 1e-5 * max(1.0, np.abs(rho_o).max())
    assert np.abs(s.temperature() - o.temperature()).max() < 1e-5
    assert np.abs(s.stress() - o.stress()).max() < 1e-4 * max(1.0, np.abs(o.stress()).max())
    k, _ = s.permeability()
    assert abs(k - o.permeability()) <= 1e-4 * abs(o.permeability())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_es_bits_independent_of_tiles_and_pencils(precision):
    mask = _rock(11, 10, 13, seed=8)
    (v, w), _ = _grid(8)
    ref = None
    for t1, rows in ((8, 4), (4, 2), (8, 3), (4, 10)):
        s = dvm.Solver(mask, 0.3, v, w, precision=precision, tile_x1=t1, band_rows=rows, temperature_term=True,
                       es_prandtl=PR)
        s.step(5)
        s.sync()
        got = (s.moments()[1], s.stress())
        if ref is None:
            ref = got
        else:
            assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])


def test_es_prandtl_one_gives_the_bgk_bits_fp64():
    """1 - 1/Pr = 0 and nu unchanged: the same arithmetic up to added zeros, on the same kernel."""
    mask = _rock(9, 10, 11, seed=2)
    (v, w), _ = _grid(8)
    a = dvm.Solver(mask, 0.5, v, w, precision="fp64", temperature_term=True)
    b = dvm.Solver(mask, 0.5, v, w, precision="fp64", temperature_term=True, es_prandtl=1.0)
    a.step(4)
    b.step(4)
    a.sync()
    b.sync()
    assert np.array_equal(a.moments()[1], b.moments()[1])
    assert np.array_equal(a.temperature(), b.temperature())


def test_es_converged_k_differs_from_bgk_and_matches_oracle():
    """Run both to Err < 1e-8: the ES model's k agrees with the oracle's and differs from BGK's."""
    mask = _rock(8, 8, 10, seed=9, frac=0.2)
    (v, w), (vo, wo) = _grid(8)
    s = dvm.Solver(mask, 0.3, v, w, precision="fp64", lateral="periodic", temperature_term=True,
                   es_prandtl=PR, check_interval=10)
    st, it, err = s.iterate(3000, 1e-9)
    o = oracle.Oracle(mask, 0.3, vo, wo, lateral="periodic", tau=True, es_pr=PR)
    o.iterate(it)
    k, _ = s.permeability()
    assert abs(k - o.permeability()) <= FP64_TOL * abs(o.permeability())
    b = dvm.Solver(mask, 0.3, v, w, precision="fp64", lateral="periodic", temperature_term=True, check_interval=10)
    b.iterate(3000, 1e-9)
    kb, _ = b.permeability()
    assert abs(k - kb) > 1e-6 * abs(kb)


def test_es_option_is_validated():
    rock = inputs.gaussian_rock(8, seed=1, corr_len=1.5, porosity=0.6)
    v3, w3 = dvm.dvm_gh_velocity_grid(3, 4)
    for kw in (dict(es_prandtl=PR),                                   # no temperature term
               dict(es_prandtl=-0.5, temperature_term=True),
               dict(es_prandtl=PR, temperature_term=True, specular_fraction=0.3),
               dict(es_prandtl=PR, temperature_term=True, subdomains=(2, 1, 1)),
               dict(es_prandtl=PR, temperature_term=True, precision="bf16_store")):
        with pytest.raises(dvm.DvmError):
            dvm.Solver(rock, 0.2, v3, w3, **kw)
    (v2, w2) = dvm.dvm_gh_velocity_grid(2, 8)
    with pytest.raises(dvm.DvmError):
        dvm.Solver(inputs.cylinder_cell(16, 0.7), 0.2, v2, w2, es_prandtl=PR)
    with pytest.raises(dvm.DvmError):
        dvm.Solver(rock, 0.2, v3, w3, temperature_term=True, es_prandtl=PR, shakhov_prandtl=PR)
    s = dvm.Solver(rock, 0.2, v3, w3, precision="fp32", temperature_term=True)
    with pytest.raises(dvm.DvmError):
        s.stress()
