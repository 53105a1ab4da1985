"""What the learned warm start gains: a small network trained on converged solutions of the solver
(3D rocks near the continuum limit, Knudsen numbers log-uniform in [0.02, 0.2], where the source
iteration converges slowly) starts held-out problems closer to their solution, so they reach the
Err < 1e-6 test of Eq. 15 in fewer iterations, and to the same permeability as the plain zero start
(the fixed point does not depend on the start)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1712_01132_gb300 import dvm, inputs, warmstart

pytestmark = pytest.mark.gpu

SIDE, NV = 24, 8
OPTS = dict(precision="fp32", lateral="periodic", check_interval=10)


def _sample(seed, kn, v, w):
    mask = inputs.gaussian_rock(SIDE, seed=seed, corr_len=3.0, porosity=0.5)
    it, dt, k, rho, u, st = warmstart.solve_to(mask, kn, v, w, 1e-6, 20000, **OPTS)
    assert st == dvm.DVM_OK
    return mask, kn, rho, u, it, k


def test_trained_network_reduces_iterations_and_keeps_the_answer():
    v, w = dvm.dvm_gh_velocity_grid(3, NV)
    rng = np.random.default_rng(0)
    train = []
    for i in range(12):
        kn = float(10 ** rng.uniform(np.log10(0.02), np.log10(0.2)))
        mask, kn, rho, u, it, k = _sample(100 + i, kn, v, w)
        x = torch.from_numpy(warmstart.features(mask, kn)).cuda()
        t = torch.from_numpy(warmstart.targets(mask, kn, rho, u)).cuda()
        m = torch.from_numpy((~mask).astype(np.float32).ravel()).cuda()
        train.append((x, t, m))
    net = warmstart.UNet(levels=2, base=8, seed=1)
    net.set_standardisation([(t.cpu().numpy(), m.cpu().numpy()) for _, t, m in train])
    train = [(x, net.standardise(t), m) for x, t, m in train]
    losses = []
    for step in range(900):
        x, t, m = train[step % len(train)]
        net.zero_grad()
        y = net.forward(x)
        loss, dy = net.loss_and_grad(y, t, m)
        net.backward(dy)
        net.step(lr=2e-3)
        losses.append(loss)
    first, last = float(np.mean(losses[:len(train)])), float(np.mean(losses[-len(train):]))
    assert last < 0.5 * first
    plain_total = warm_total = 0
    for seed, kn in ((900, 0.03), (901, 0.05), (902, 0.1)):
        mask = inputs.gaussian_rock(SIDE, seed=seed, corr_len=3.0, porosity=0.5)
        it0, _, k0, _, _, st0 = warmstart.solve_to(mask, kn, v, w, 1e-6, 20000, **OPTS)
        pred = warmstart.predict(net, mask, kn)
        it1, _, k1, _, _, st1 = warmstart.solve_to(mask, kn, v, w, 1e-6, 20000,
                                                   initial=warmstart.to_initial(mask, kn, pred), **OPTS)
        print("held-out seed %d Kn %.2f: iterations plain %d, warm %d; k %.6e vs %.6e" % (seed, kn, it0, it1, k0, k1))
        assert st0 == dvm.DVM_OK and st1 == dvm.DVM_OK
        assert abs(k1 - k0) <= 1e-3 * abs(k0)
        plain_total += it0
        warm_total += it1
    print("training loss %.4e -> %.4e; iterations plain %d, warm %d" % (first, last, plain_total, warm_total))
    assert warm_total < plain_total
