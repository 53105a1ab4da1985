"""The convergence measure of the CUDA path (Eq. 15, Sec. 3.1 steps iv-v) against its definition and
against the oracle, through the C ABI.

dvm_iterate evaluates Err(l) = |k(l) - k(l')| / ((l - l') |k(l)|) at the iteration counts that are
multiples of the check interval, with l' the previous check (l - l' = 100 in the paper), the start
state at the first check (k = 0 for h = 0), or the iteration of a warm start.  The FP64 path is
compared with the FP64 oracle at equal iteration counts, so both Err sequences must agree to the
rounding of a difference of two nearly equal permeabilities.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
from paper_1712_01132_gb300 import dvm, inputs

pytestmark = pytest.mark.gpu


def test_err_follows_eq15_across_steps_and_a_warm_start():
    mask = inputs.cylinder_cell(32, 0.7)
    v, w = dvm.dvm_gh_velocity_grid(2, 16)
    vo, wo = oracle.velocity_grid(2, 16)
    s = dvm.Solver(mask, 0.1, v, w, precision="fp64", lateral="periodic")
    o = oracle.Oracle(mask, 0.1, vo, wo, lateral="periodic")

    st, it, err = s.iterate(100, 0.0)              # first check: compared with the zero start
    k1 = s.permeability()[0]
    _, _, err_o = o.run(0.0, 100)
    assert it == 100 and o.iterations == 100
    assert err == 1.0 / 100.0                      # |k1 - 0| / (100 |k1|), exactly
    assert err_o == 1.0 / 100.0

    st, it, err = s.iterate(100, 0.0)
    k2 = s.permeability()[0]
    _, _, err_o = o.run(0.0, 200)
    assert err == pytest.approx(abs(k2 - k1) / (100 * abs(k2)), rel=1e-12)
    assert err == pytest.approx(err_o, rel=1e-6)

    s.step(30)                                     # no check at 230: the next one is at 300
    s.sync()
    st, it, err = s.iterate(1000, 1e300)     # any Err stops at the first check
    k3 = s.permeability()[0]
    assert it == 70 and s.iterations == 300
    assert err == pytest.approx(abs(k3 - k2) / (100 * abs(k3)), rel=1e-12)
    o.iterate(30)
    _, _, err_o = o.run(0.0, 300)
    assert err == pytest.approx(err_o, rel=1e-6)

    s.step(30)                                     # warm start at 330 from the current fields
    s.sync()
    o.iterate(30)
    rho, u = s.moments()
    s.set_initial(rho, u)
    rho_o, u_o = o.moments()
    o.set_initial(rho_o, u_o)
    kw = s.permeability()[0]
    assert kw == pytest.approx(o.permeability(), rel=1e-10)
    st, it, err = s.iterate(1000, 1e300)           # check at 400, 70 iterations after the warm start
    k4 = s.permeability()[0]
    assert it == 70
    assert err == pytest.approx(abs(k4 - kw) / (70 * abs(k4)), rel=1e-12)
    _, _, err_o = o.run(0.0, 400)
    assert err == pytest.approx(err_o, rel=1e-6)
    s.close()


def test_err_survives_a_checkpoint():
    mask = inputs.cylinder_cell(32, 0.7)
    v, w = dvm.dvm_gh_velocity_grid(2, 16)
    a = dvm.Solver(mask, 0.1, v, w, precision="fp64", lateral="periodic")
    a.iterate(100, 0.0)
    a.step(50)
    a.sync()
    blob = a.get_state()
    _, _, err_a = a.iterate(1000, 1e300)
    b = dvm.Solver(mask, 0.1, v, w, precision="fp64", lateral="periodic")
    b.set_state(blob)
    _, it_b, err_b = b.iterate(1000, 1e300)
    assert it_b == 50 and err_b == err_a
    a.close()
    b.close()
