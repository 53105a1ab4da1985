"""The allocation-free permeability entry point (collected last on purpose).

Callers that cannot allocate device memory when they need a result -- code running during CUDA
graph capture, plugins whose host framework owns all device memory, allocation-free steady-state
loops -- can compute the permeability of a velocity field they hold with
dvm_permeability_noalloc; its scratch is a static device array of fixed size.  This test checks
it against the solver's own permeability (dvm_permeability) on two calls in a row, and that a
field larger than the scratch allows is rejected.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1712_01132_gb300 import dvm, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_permeability_matches_solver(precision):
    mask = inputs.random_discs(96, 64, seed=31, rmin=3, rmax=8, solid_fraction=0.4)
    v, w = dvm.dvm_gh_velocity_grid(2, 16)
    s = dvm.Solver(mask, 0.3, v, w, precision=precision, lateral="periodic")
    n = mask.size
    rho = torch.empty(n, dtype=torch.float64, device="cuda")
    u = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for it in (25, 40):                      # two calls in a row, on different fields
        s.step(it)
        s.sync()
        k_ref, gp_ref = s.permeability()
        s.moments_device(0, rho.data_ptr(), u.data_ptr())
        torch.cuda.synchronize()
        for _ in range(2):
            out.zero_()
            dvm.dvm_permeability_noalloc(u.data_ptr(), n, 0.3, out.data_ptr(), stream)
            torch.cuda.synchronize()
            k, gp = out.cpu().numpy()
            assert k == pytest.approx(k_ref, rel=1e-10)
            assert gp == pytest.approx(gp_ref, rel=1e-10)
    s.close()


def test_noalloc_rejects_fields_beyond_its_scratch():
    big = 8192 * 256 + 1
    buf = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(dvm.DvmError) as ei:
        dvm.dvm_permeability_noalloc(buf.data_ptr(), big, 0.3, buf.data_ptr())
    assert ei.value.status == dvm.DVM_EINVAL and "outside" in str(ei.value)
