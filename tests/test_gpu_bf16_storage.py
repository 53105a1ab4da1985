"""The BF16-storage ablation (3D): FP32 arithmetic with the transient h held in HBM (pencil edges,
ghost layers) stored as BF16 deviations from the x1 ramp.  Its error against the oracle is
reported, not gated; these tests check that the mode works end to end and that its error stays at
the BF16 level (loose bounds), and they print the measured errors."""
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


@pytest.mark.parametrize("lateral", ["periodic", "specular"])
def test_bf16_storage_first_iterations(lateral):
    mask = inputs.gaussian_rock(12, seed=3, corr_len=1.5, porosity=0.55)
    v, w = dvm.dvm_gh_velocity_grid(3, 8)
    vo, wo = oracle.velocity_grid(3, 8)
    o = oracle.Oracle(mask, 0.5, vo, wo, lateral=lateral)
    o.iterate(3)
    _, u_o = o.moments()
    errs = {}
    for prec in ("fp32", "bf16_store"):
        s = dvm.Solver(mask, 0.5, v, w, precision=prec, lateral=lateral, band_rows=3)
        s.step(3)
        s.sync()
        _, u = s.moments()
        errs[prec] = (_rel(u, u_o), abs(s.permeability()[0] / o.permeability() - 1.0))
    print("first 3 iterations, max|du|/max|u| and |dk|/k:", errs)
    assert errs["fp32"][0] < 1e-4
    assert errs["bf16_store"][0] < 2e-2 and errs["bf16_store"][1] < 2e-2


def test_bf16_storage_converged_permeability():
    mask = inputs.gaussian_rock(16, seed=2, corr_len=2.0, porosity=0.5)
    v, w = dvm.dvm_gh_velocity_grid(3, 8)
    vo, wo = oracle.velocity_grid(3, 8)
    o = oracle.Oracle(mask, 0.5, vo, wo, lateral="periodic")
    o.run(1e-10, 20000)
    s = dvm.Solver(mask, 0.5, v, w, precision="bf16_store", lateral="periodic")
    st, it, err = s.iterate(4000, 1e-6)
    k = s.permeability()[0]
    _, u = s.moments()
    _, u_o = o.moments()
    print("converged: |dk|/k = %.3e, max|du|/max|u| = %.3e, iterations %d, status %d"
          % (abs(k / o.permeability() - 1), _rel(u, u_o), it, st))
    assert np.isfinite(k)
    assert abs(k / o.permeability() - 1) < 5e-2


def test_bf16_storage_checkpoint_and_warm_start():
    mask = inputs.gaussian_rock(10, seed=4, corr_len=1.5, porosity=0.55)
    v, w = dvm.dvm_gh_velocity_grid(3, 8)
    a = dvm.Solver(mask, 0.3, v, w, precision="bf16_store", lateral="specular")
    rng = np.random.default_rng(1)
    a.set_initial(0.1 * rng.standard_normal(mask.shape), 0.01 * rng.standard_normal((3,) + mask.shape))
    a.step(5)
    blob = a.get_state()
    a.step(4)
    b = dvm.Solver(mask, 0.3, v, w, precision="bf16_store", lateral="specular")
    b.set_state(blob)
    b.step(4)
    assert np.array_equal(a.moments()[1], b.moments()[1])
    c = dvm.Solver(mask, 0.3, v, w, precision="fp32", lateral="specular")
    with pytest.raises(dvm.DvmError):          # an FP32 context does not accept a BF16 state
        c.set_state(blob)


def test_bf16_storage_is_3d_only():
    mask = inputs.cylinder_cell(16, 0.7)
    v, w = dvm.dvm_gh_velocity_grid(2, 4)
    with pytest.raises(dvm.DvmError):
        dvm.Solver(mask, 0.2, v, w, precision="bf16_store")
