"""GPU parity of the warm-start network kernels (through the C ABI) with the FP64 reference
`oracle.nn_reference`: each kernel, then the whole U-Net forward and backward pass with the same
(BF16-rounded) parameters.  The convolutions and data gradients run on the BF16 tensor cores, so
the reference rounds their operands to BF16 the same way; products are then exact and only the
FP32 accumulation differs: 1e-5 relative per kernel.  Through the whole network the GPU's FP32
activations and the reference's FP64 ones can round to neighbouring BF16 values at a rare element,
which the looser whole-network bounds (1e-3 outputs, 1e-2 gradients) allow for."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import nn_reference as ref
from paper_1712_01132_gb300 import dvm, warmstart

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def _s():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("cin,cout,dims", [(5, 7, (6, 8, 10)), (3, 16, (4, 4, 4)), (17, 9, (8, 2, 6)),
                                           # channel counts of the warm-start network (base 32): full
                                           # 128-voxel x 32-channel tiles, many CTAs per channel block
                                           (32, 32, (16, 16, 16)), (64, 64, (16, 16, 16)),
                                           (96, 32, (16, 16, 16)), (32, 96, (8, 16, 32))])
def test_conv_kernels_match_reference(cin, cout, dims):
    lib = dvm.load()
    rng = np.random.default_rng(cin * 100 + cout)
    x = rng.standard_normal((cin,) + dims).astype(np.float32)
    w = (rng.standard_normal((cout, cin, 27)) / np.sqrt(cin * 27)).astype(np.float32)
    b = rng.standard_normal(cout).astype(np.float32)
    g = rng.standard_normal((cout,) + dims).astype(np.float32)
    xd, wd, bd, gd = _dev(x), _dev(w), _dev(b), _dev(g)
    y = torch.empty((cout,) + dims, device="cuda")
    nsc = lib.dvm_nn_conv3d_scratch_bytes(cin, cout, *dims)
    sc = torch.empty(nsc + 3, dtype=torch.uint8, device="cuda")[3:]     # any alignment
    assert lib.dvm_nn_conv3d(_p(xd), _p(wd), _p(bd), _p(y), cin, cout, *dims, 0, _p(sc), nsc, _s()) == 0
    assert lib.dvm_nn_status(_s()) == 0
    xr, wr, gr = ref.round_bf16(x), ref.round_bf16(w), ref.round_bf16(g)     # tensor-core operands
    assert _rel(y.cpu().numpy(), ref.conv3d(xr, wr, b.astype(np.float64))) < 1e-5
    dx = torch.empty((cin,) + dims, device="cuda")
    assert lib.dvm_nn_conv3d_dgrad(_p(gd), _p(wd), _p(dx), cin, cout, *dims, 0, _p(sc), nsc, _s()) == 0
    assert lib.dvm_nn_status(_s()) == 0
    assert _rel(dx.cpu().numpy(), ref.conv3d_dgrad(gr, wr)) < 1e-5
    y2 = y.clone()                                   # accumulate = 1 adds to the old values
    assert lib.dvm_nn_conv3d(_p(xd), _p(wd), _p(bd), _p(y2), cin, cout, *dims, 1, _p(sc), nsc, _s()) == 0
    assert lib.dvm_nn_conv3d(_p(xd), _p(wd), _p(bd), _p(y2), cin, cout, *dims, 1, _p(sc), 1024, _s()) != 0   # too small
    assert _rel(y2.cpu().numpy(), 2.0 * y.cpu().numpy()) < 1e-6
    n = lib.dvm_nn_wgrad_scratch_floats(cin, cout, *dims)
    scratch = torch.empty(n, device="cuda")
    dw = torch.full((cout, cin, 27), 0.5, device="cuda")
    db = torch.full((cout,), 0.25, device="cuda")
    assert lib.dvm_nn_conv3d_wgrad(_p(xd), _p(gd), _p(dw), _p(db), _p(scratch), n, cin, cout, *dims, 1, _s()) == 0
    rdw, _ = ref.conv3d_wgrad(xr, gr)                    # tensor-core operands (BF16-rounded)
    _, rdb = ref.conv3d_wgrad(x.astype(np.float64), g.astype(np.float64))
    assert _rel(dw.cpu().numpy(), rdw + 0.5) < 1e-5      # accumulate = 1 adds to the old values
    assert _rel(db.cpu().numpy(), rdb + 0.25) < 1e-5
    assert lib.dvm_nn_conv3d_wgrad(_p(xd), _p(gd), _p(dw), None, _p(scratch), n - 1, cin, cout, *dims, 0, _s()) != 0


def test_resampling_relu_and_loss_kernels():
    lib = dvm.load()
    rng = np.random.default_rng(5)
    c, dims = 3, (4, 6, 8)
    x = rng.standard_normal((c,) + dims).astype(np.float32)
    xd = _dev(x)
    y = torch.empty((c, 2, 3, 4), device="cuda")
    assert lib.dvm_nn_pool2(_p(xd), _p(y), c, *dims, _s()) == 0
    assert _rel(y.cpu().numpy(), ref.pool2(x.astype(np.float64))) < 1e-6
    gy = rng.standard_normal((c, 2, 3, 4)).astype(np.float32)
    gx = torch.zeros((c,) + dims, device="cuda")
    assert lib.dvm_nn_pool2_bwd(_p(_dev(gy)), _p(gx), c, *dims, 1, _s()) == 0
    assert _rel(gx.cpu().numpy(), ref.pool2_bwd(gy.astype(np.float64))) < 1e-6
    up = torch.empty((c,) + dims, device="cuda")
    assert lib.dvm_nn_up2(_p(_dev(gy)), _p(up), c, *dims, _s()) == 0
    assert _rel(up.cpu().numpy(), ref.up2(gy.astype(np.float64))) < 1e-7
    gu = torch.empty((c, 2, 3, 4), device="cuda")
    assert lib.dvm_nn_up2_bwd(_p(xd), _p(gu), c, *dims, _s()) == 0
    assert _rel(gu.cpu().numpy(), ref.up2_bwd(x.astype(np.float64))) < 1e-6
    assert lib.dvm_nn_pool2(_p(xd), _p(y), c, 5, 6, 8, _s()) != 0          # odd extent
    r = xd.clone()
    assert lib.dvm_nn_relu(_p(r), r.numel(), _s()) == 0
    assert np.array_equal(r.cpu().numpy(), np.maximum(x, 0))
    g = _dev(np.ones_like(x))
    assert lib.dvm_nn_relu_bwd(_p(r), _p(g), g.numel(), _s()) == 0
    assert np.array_equal(g.cpu().numpy(), (x > 0).astype(np.float32))
    t = rng.standard_normal((c,) + dims).astype(np.float32)
    mask = rng.random(dims) > 0.4
    net = warmstart.UNet(levels=1, base=2)
    loss, dy = net.loss_and_grad(xd, _dev(t), _dev(mask.astype(np.float32).ravel()))
    rl, rdy = ref.masked_mse(x.astype(np.float64), t.astype(np.float64), mask)
    assert loss == pytest.approx(rl, rel=1e-5)
    assert _rel(dy.cpu().numpy(), rdy) < 1e-5


@pytest.mark.parametrize("levels,base,n", [(2, 4, 8), (3, 3, 8), (4, 2, 16)])
def test_unet_forward_and_backward_match_reference(levels, base, n):
    net = warmstart.UNet(levels=levels, base=base, seed=levels)
    rng = np.random.default_rng(levels)
    for b in net.b:                                  # non-zero biases exercise the bias paths
        b.copy_(torch.tensor(rng.standard_normal(b.shape[0]) * 0.1, dtype=torch.float32, device="cuda"))
    net._requantize()
    x = rng.standard_normal((3, n, n, n)).astype(np.float32)
    t = rng.standard_normal((4, n, n, n)).astype(np.float32)
    mask = rng.random((n, n, n)) > 0.3
    y = net.forward(_dev(x))
    loss, dy = net.loss_and_grad(y, _dev(t), _dev(mask.astype(np.float32).ravel()))
    net.zero_grad()
    net.backward(dy)
    params = net.parameters_for_reference()
    ry, cache = ref.forward(params, x.astype(np.float64), levels, bf16_operands=True)
    rloss, rdy = ref.masked_mse(ry, t.astype(np.float64), mask)
    grads = ref.backward(params, cache, rdy, levels, bf16_operands=True)
    ey = _rel(y.cpu().numpy(), ry)
    eg = max(max(_rel(net.dw[i].cpu().numpy(), gw), _rel(net.db[i].cpu().numpy(), gb)) for i, (gw, gb) in enumerate(grads))
    print("U-Net levels %d base %d n %d: output rel err %.2e, worst gradient rel err %.2e" % (levels, base, n, ey, eg))
    assert ey < 1e-3
    assert loss == pytest.approx(rloss, rel=1e-3)
    assert eg < 1e-2


def test_adam_step_and_bf16_rounding():
    lib = dvm.load()
    rng = np.random.default_rng(9)
    n = 1000
    w = rng.standard_normal(n).astype(np.float32)
    g = rng.standard_normal(n).astype(np.float32)
    wd, gd = _dev(w), _dev(g)
    wq = torch.empty(n, device="cuda")
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    assert lib.dvm_nn_adam(_p(wd), _p(wq), _p(gd), _p(m), _p(v), n, 1e-2, 0.9, 0.999, 1e-8, 1, 1.0, _s()) == 0
    # first bias-corrected Adam step: w - lr * g / (|g| + eps)
    ref_w = w - 1e-2 * g / (np.abs(g) + 1e-8)
    assert np.abs(wd.cpu().numpy() - ref_w).max() < 1e-6
    q = wq.cpu().numpy()
    bits = q.view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)                       # a BF16 value
    assert np.abs(q - wd.cpu().numpy()).max() <= np.abs(wd.cpu().numpy()).max() * 2 ** -8
