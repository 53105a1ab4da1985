"""The paired-band FP32 2D sweep (two consecutive bands per CTA, the lower band's top edge handed
to the upper band in shared memory) against the one-band kernel and the FP64 oracle.  Both kernels
do the same arithmetic in the same order, so every result bit must agree; odd band counts (a last
pair with one band), single-band problems, ragged x1 tails and batches whose problems have
different band counts are covered."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
from paper_1712_01132_gb300 import dvm, inputs

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _fields(s, nprob):
    out = []
    for b in range(nprob):
        rho, u = s.moments(b)
        out.append((rho, u, s.wall(b), s.permeability(b)[0]))
    return out


def _run(masks, kns, v, w, steps, **opt):
    s = dvm.Solver(masks, kns, v, w, precision="fp32", **opt)
    s.step(steps)
    s.sync()
    f = _fields(s, len(kns) if isinstance(kns, (list, tuple)) else 1)
    s.close()
    return f


@pytest.mark.parametrize("lateral", ["periodic", "specular"])
@pytest.mark.parametrize("nv", [16, 32])
@pytest.mark.parametrize("t1,rows", [(8, 8), (4, 3), (8, 35), (4, 1), (8, 17), (4, 12)])
def test_pairs_give_the_one_band_bits(lateral, nv, t1, rows):
    mask = inputs.random_discs(53, 35, seed=7, rmin=2, rmax=5, solid_fraction=0.4)
    v, w = dvm.dvm_gh_velocity_grid(2, nv)
    ref = _run(mask, 0.2, v, w, 9, lateral=lateral, tile_x1=t1, band_rows=rows)
    got = _run(mask, 0.2, v, w, 9, lateral=lateral, tile_x1=t1, band_rows=rows, band_pairs=True)
    for (r0, u0, w0, k0), (r1, u1, w1, k1) in zip(ref, got):
        assert np.array_equal(r0, r1) and np.array_equal(u0, u1) and np.array_equal(w0, w1) and k0 == k1


def test_pairs_batch_of_uneven_problems_with_graphs():
    masks = [inputs.random_discs(30, 22, seed=11, rmin=2, rmax=4, solid_fraction=0.3),
             inputs.cylinder_cell(32, 0.7),
             inputs.random_discs(47, 19, seed=12, rmin=2, rmax=3, solid_fraction=0.35),
             inputs.random_discs(21, 41, seed=13, rmin=2, rmax=4, solid_fraction=0.3)]
    kns = [0.05, 0.1, 1.0, 0.3]
    v, w = dvm.dvm_gh_velocity_grid(2, 16)
    ref = _run(masks, kns, v, w, 23, lateral="periodic", band_rows=4, check_interval=10)
    got = _run(masks, kns, v, w, 23, lateral="periodic", band_rows=4, check_interval=10,
               band_pairs=True, use_graph=True)
    for (r0, u0, w0, k0), (r1, u1, w1, k1) in zip(ref, got):
        assert np.array_equal(r0, r1) and np.array_equal(u0, u1) and np.array_equal(w0, w1) and k0 == k1


@pytest.mark.parametrize("shape,seed", [((29, 37), 1), ((41, 23), 3)])
def test_pairs_match_oracle_first_iterations(shape, seed):
    mask = inputs.random_discs(shape[0], shape[1], seed=seed, rmin=2, rmax=5, solid_fraction=0.35)
    v, w = dvm.dvm_gh_velocity_grid(2, 16)
    vo, wo = oracle.velocity_grid(2, 16)
    s = dvm.Solver(mask, 0.1, v, w, precision="fp32", lateral="specular", band_rows=5, band_pairs=True)
    s.step(6)
    s.sync()
    o = oracle.Oracle(mask, 0.1, vo, wo, lateral="specular")
    o.iterate(6)
    rho, u = s.moments()
    rho_o, u_o = o.moments()
    assert _rel(u, u_o) < 1e-4
    assert np.abs(rho - rho_o).max() < 1e-5 * max(1.0, np.abs(rho_o).max())
    k, _ = s.permeability()
    assert abs(k - o.permeability()) <= 1e-4 * abs(o.permeability())


def test_pairs_full_size_kn_sweep_first_iteration_bits():
    """The 512 x 512, 32 x 32 velocity, four-Knudsen batch of the throughput measurement."""
    mask = inputs.random_discs(512, 512, seed=0)
    v, w = dvm.dvm_gh_velocity_grid(2, 32)
    kns = [0.01, 0.1, 1.0, 10.0]
    ref = _run([mask] * 4, kns, v, w, 3, lateral="periodic")
    got = _run([mask] * 4, kns, v, w, 3, lateral="periodic", band_pairs=True)
    for (r0, u0, w0, k0), (r1, u1, w1, k1) in zip(ref, got):
        assert np.array_equal(r0, r1) and np.array_equal(u0, u1) and np.array_equal(w0, w1) and k0 == k1


def test_pairs_reject_too_many_velocities():
    mask = inputs.cylinder_cell(16, 0.5)
    v, w = dvm.dvm_gh_velocity_grid(2, 64)               # 1024 velocities per quadrant
    with pytest.raises(dvm.DvmError) as ei:
        dvm.Solver(mask, 0.1, v, w, precision="fp32", band_pairs=True)
    assert ei.value.status == dvm.DVM_EINVAL
