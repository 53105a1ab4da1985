"""Pins of the FP64 network reference used to check the warm-start kernels (CPU only).

Each part is pinned by something other than itself: the convolution by scipy's correlate with
periodic wrap, every linear piece by its adjoint identity, the whole backward pass by central
finite differences of the loss, and the BF16 rounding of tensor-core operands by torch's
conversion."""
import numpy as np
import pytest

scipy_ndimage = pytest.importorskip("scipy.ndimage")

from oracle import nn_reference as nn


def test_conv_matches_scipy_correlate_with_wrap():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 5, 6, 7))
    w = rng.standard_normal((1, 1, 27))
    y = nn.conv3d(x, w)
    kern = w[0, 0].reshape(3, 3, 3)          # [kz][ky][kx], offsets -1..1
    ref = scipy_ndimage.correlate(x[0], kern, mode="wrap")
    assert np.abs(y[0] - ref).max() < 1e-12


def test_multichannel_conv_is_a_sum_of_single_channel_correlations():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 4, 5, 6))
    w = rng.standard_normal((2, 3, 27))
    b = rng.standard_normal(2)
    y = nn.conv3d(x, w, b)
    for o in range(2):
        ref = b[o] + sum(scipy_ndimage.correlate(x[c], w[o, c].reshape(3, 3, 3), mode="wrap") for c in range(3))
        assert np.abs(y[o] - ref).max() < 1e-12


def test_adjoint_identities():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 4, 6, 8))
    w = rng.standard_normal((5, 3, 27))
    g = rng.standard_normal((5, 4, 6, 8))
    lhs = float((nn.conv3d(x, w) * g).sum())
    assert lhs == pytest.approx(float((x * nn.conv3d_dgrad(g, w)).sum()), rel=1e-12)
    dw, db = nn.conv3d_wgrad(x, g)
    assert lhs == pytest.approx(float((w * dw).sum()), rel=1e-12)
    assert np.allclose(db, g.sum(axis=(1, 2, 3)), rtol=1e-12)
    p = rng.standard_normal((3, 2, 3, 4))
    assert float((nn.pool2(x) * p).sum()) == pytest.approx(float((x * nn.pool2_bwd(p)).sum()), rel=1e-12)
    q = rng.standard_normal((3, 8, 12, 16))
    assert float((nn.up2(x) * q).sum()) == pytest.approx(float((x * nn.up2_bwd(q)).sum()), rel=1e-12)


@pytest.mark.parametrize("levels", [2, 3])
def test_network_gradients_match_finite_differences(levels):
    rng = np.random.default_rng(3 + levels)
    n = 4 * 2 ** (levels - 1)
    shapes = nn.layer_shapes(levels, 2, 3, 4)
    params = [(0.4 * rng.standard_normal((co, ci, 27)) / np.sqrt(ci * 27), 0.1 * rng.standard_normal(co))
              for ci, co in shapes]
    x = rng.standard_normal((3, n, n, n))
    t = rng.standard_normal((4, n, n, n))
    mask = rng.random((n, n, n)) > 0.3

    def loss(ps):
        y, _ = nn.forward(ps, x, levels)
        return nn.masked_mse(y, t, mask)[0]

    y, cache = nn.forward(params, x, levels)
    _, dy = nn.masked_mse(y, t, mask)
    grads = nn.backward(params, cache, dy, levels)
    h = 1e-6
    for li in range(len(params)):
        for which in (0, 1):
            arr = params[li][which]
            for _ in range(3):
                idx = tuple(rng.integers(0, s) for s in arr.shape)
                orig = arr[idx]
                arr[idx] = orig + h
                lp = loss(params)
                arr[idx] = orig - h
                lm = loss(params)
                arr[idx] = orig
                fd = (lp - lm) / (2 * h)
                an = grads[li][which][idx]
                assert abs(fd - an) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (li, which, idx, fd, an)


def test_bf16_rounding_matches_torch():
    """The reference's BF16 rounding (round to nearest even, on the float32 value) is torch's."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    a = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 0.0, -0.0])])
    want = torch.tensor(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(nn.round_bf16(a), want)
