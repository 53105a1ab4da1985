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


# ------------------------------------------------------------------ reduced precision at convergence
#
# The FP32 path (FP32 h and moments, FP64 wall sums, G_p and Err) run to Err < 1e-8, against the
# FP64 oracle converged to Err < 1e-10 (tests/golden, written by make_convergence_golden.py, which
# calls only the oracle): permeability within 1e-4 relative, u within 1e-3 of its max-norm, and rho
# (fluid mean removed: the iteration fixes it only up to a constant) within 1e-3 of its max-norm.
# The cases cover the ends of the benchmark's Kn sweep (0.01 and 10) on a 192^2 disc medium with
# 32^2 velocities, two problems of the batched generator (24^2 velocities) in one context, and a
# Gaussian-field rock with the 3D workload's 16^3 velocities.

import json
import os
import sys

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
if GOLD not in sys.path:
    sys.path.insert(0, GOLD)

FP32_TOL = 1e-8


def _golden(name):
    with open(os.path.join(GOLD, "convergence_%s.json" % name)) as f:
        meta = json.load(f)
    d = np.load(os.path.join(GOLD, "convergence_%s.npz" % name))
    return meta, d["rho"].astype(np.float64), d["u"].astype(np.float64)


def _cases():
    import make_convergence_golden
    return make_convergence_golden.cases()


def _check(mask, s, prob, meta, rho_o, u_o):
    k, _ = s.permeability(prob)
    rho, u = s.moments(prob)
    fl = ~mask
    d = (rho - rho[fl].mean()) * fl
    true_err = abs(k - meta["k"]) / abs(meta["k"])
    print("%s: k %.10e oracle %.10e, |dk|/k %.2e" % (meta["case"], k, meta["k"], true_err))
    assert true_err <= 1e-4
    assert np.abs(u - u_o).max() <= 1e-3 * np.abs(u_o).max()
    assert np.abs(d - rho_o).max() <= 1e-3 * np.abs(rho_o).max()


@pytest.mark.parametrize("name", ["discs192_kn0.01", "discs192_kn10", "rock24_kn0.5"])
def test_fp32_converged_matches_converged_oracle(name):
    meta, rho_o, u_o = _golden(name)
    mask, kn, n_axis, _ = _cases()[name]
    v, w = dvm.dvm_gh_velocity_grid(mask.ndim, n_axis)
    s = dvm.Solver(mask, kn, v, w, precision="fp32", lateral="periodic", use_graph=True)
    st, it, err = s.iterate(100000, FP32_TOL)
    assert st == dvm.DVM_OK and err < FP32_TOL
    _check(mask, s, 0, meta, rho_o, u_o)
    s.close()


def test_fp32_batch_of_generated_problems_converges_to_the_oracle():
    names = ["c3_seed1000", "c3_seed1004"]
    gold = [_golden(n) for n in names]
    cs = _cases()
    masks = [cs[n][0] for n in names]
    kns = [cs[n][1] for n in names]
    v, w = dvm.dvm_gh_velocity_grid(2, 24)
    s = dvm.Solver(masks, kns, v, w, precision="fp32", lateral="periodic", use_graph=True)
    st, it, err = s.iterate(100000, FP32_TOL)       # every problem of the batch below tol
    assert st == dvm.DVM_OK and err < FP32_TOL
    for b, (meta, rho_o, u_o) in enumerate(gold):
        _check(masks[b], s, b, meta, rho_o, u_o)
    s.close()
