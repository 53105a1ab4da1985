"""Host-side pieces of the learned warm start, on the CPU: the network's input features, its
training targets and their inverse, and the U-Net's layer bookkeeping."""
import math

import numpy as np
import pytest

pytest.importorskip("scipy")
from paper_1712_01132_gb300 import inputs, warmstart as ws


def _periodic_sdf_brute_force(mask, cap):
    """Distance to the nearest voxel of the other phase under the minimum-image convention
    (per axis min(|d|, n - |d|)), positive in the fluid, negative in the solid, clipped to +-cap."""
    shape = np.array(mask.shape)
    solid, fluid = np.argwhere(mask), np.argwhere(~mask)
    out = np.zeros(mask.shape)
    for p in np.ndindex(mask.shape):
        other = fluid if mask[p] else solid
        d = np.abs(other - np.array(p))
        d = np.minimum(d, shape - d)
        r = math.sqrt(float((d * d).sum(axis=1).min()))
        out[p] = -r if mask[p] else r
    return np.clip(out, -cap, cap)


@pytest.mark.parametrize("seed", [0, 1])
def test_signed_distance_is_the_periodic_distance_to_the_other_phase(seed):
    rng = np.random.default_rng(seed)
    mask = rng.random((10, 9, 11)) < 0.3
    got = ws.signed_distance(mask, cap=4)
    np.testing.assert_allclose(got, _periodic_sdf_brute_force(mask, 4), rtol=0, atol=1e-12)


def test_signed_distance_of_a_slab_crossing_the_seam():
    # a solid slab of three planes that wraps across the periodic seam along x: planes 9, 0, 1
    mask = np.zeros((4, 5, 10), bool)
    mask[..., [9, 0, 1]] = True
    got = ws.signed_distance(mask, cap=8)
    want = np.array([-1, -1, 1, 2, 3, 4, 3, 2, 1, -1], float)   # |distance| to the other phase along x
    want[0] = -2                                                # the slab's middle plane
    np.testing.assert_array_equal(got[0, 0], want)
    assert (got == got[:1, :1]).all()                           # uniform across y and z


def test_features_channels():
    mask = inputs.gaussian_rock(12, seed=3, corr_len=3.0, porosity=0.4)
    f = ws.features(mask, 0.5)
    assert f.shape == (3,) + mask.shape and f.dtype == np.float32
    np.testing.assert_array_equal(f[0], mask.astype(np.float32))
    np.testing.assert_allclose(f[1], ws.signed_distance(mask) / ws.SDF_SCALE, rtol=1e-6)
    np.testing.assert_allclose(f[2], math.log10(0.5 * mask.shape[-1]), rtol=1e-6)


def test_targets_and_initial_state_are_inverse_on_the_fluid():
    rng = np.random.default_rng(7)
    mask = rng.random((6, 7, 8)) < 0.35
    fl = ~mask
    n1 = mask.shape[-1]
    x1 = np.broadcast_to(np.arange(n1) / n1, mask.shape)
    rho = (rng.standard_normal(mask.shape) * 0.01 - x1) * fl
    u = rng.standard_normal((3,) + mask.shape) * 1e-3 * fl[None]
    t = ws.targets(mask, 0.5, rho, u)
    assert t.shape == (4,) + mask.shape
    assert (t[:, mask] == 0).all()
    # the density target is the source-form density with its fluid mean removed
    assert abs(t[0][fl].mean()) < 1e-6
    rho0, u0 = ws.to_initial(mask, 0.5, t)
    shift = (rho + x1)[fl].mean()
    np.testing.assert_allclose(rho0[fl], rho[fl] - shift, rtol=0, atol=1e-8)
    np.testing.assert_allclose(u0[:, fl], u[:, fl], rtol=1e-6, atol=1e-12)
    assert (rho0[mask] == 0).all() and (u0[:, mask] == 0).all()


def test_unet_layer_shapes_chain():
    levels, base, cin, cout = 4, 32, 3, 4
    shapes = ws.layer_shapes(levels, base, cin, cout)
    assert len(shapes) == 2 * levels + 2 * (levels - 1) + 1
    ch = [base * 2 ** l for l in range(levels)]
    assert shapes[0] == (cin, ch[0]) and shapes[-1] == (ch[0], cout)
    # encoder: each convolution takes what the previous one gave
    for l in range(levels):
        a, b = shapes[2 * l], shapes[2 * l + 1]
        assert a[1] == b[0] == b[1] == ch[l]
    # decoder: the first convolution of a level takes the skip plus the upsampled level below
    dec = shapes[2 * levels:-1]
    for i, l in enumerate(reversed(range(levels - 1))):
        assert dec[2 * i] == (ch[l] + ch[l + 1], ch[l]) and dec[2 * i + 1] == (ch[l], ch[l])
