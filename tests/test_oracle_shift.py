"""Periodic-shift equivariance of the oracle's converged state (CPU only).

On the periodic grid, shifting the geometry by s voxels along an axis shifts the converged velocity
field by s and leaves the permeability unchanged: along x1 the shift moves solid across the seam
where the unit pressure jump of Eq. 7 enters, laterally across the periodic faces.  The iteration
history is not equivariant (which couplings cross a seam, and so are lagged one iteration, moves
with the geometry), but the fixed point of the first-order scheme, whose steady system is
consistent, is.  A ghost layer mapped to the wrong column or row, a jump applied at the wrong face
or with the wrong sign, or a wrap that skips a point breaks the equality.  (With the second-order
stencil the steady system is inconsistent next to walls and the limit depends on the lag pattern,
so there a shift moves the converged k by about 1e-3 on such a coarse medium.)
"""
import numpy as np
import pytest

from oracle import Oracle, velocity_grid
from paper_1712_01132_gb300 import inputs


def _converged(mask, kn, v, w):
    o = Oracle(mask, kn, v, w, lateral="periodic", order=1, threads=1)
    o.run(1e-13, 8000)
    _, u = o.moments()
    return u, o.permeability()


@pytest.mark.parametrize("axis,shift", [(0, 5), (1, 7)])
def test_2d_shift_moves_the_converged_field(axis, shift):
    g = inputs.random_discs(20, 18, seed=5, rmin=2, rmax=4, solid_fraction=0.3)
    v, w = velocity_grid(2, 8)
    ua, ka = _converged(g, 0.3, v, w)
    ub, kb = _converged(np.roll(g, shift, axis=axis), 0.3, v, w)
    assert np.abs(np.roll(ua, shift, axis=axis + 1) - ub).max() < 1e-12 * np.abs(ua).max()
    assert kb == pytest.approx(ka, rel=1e-12)
    # the shift is not a symmetry of this medium: the fields themselves differ
    assert np.abs(ua - ub).max() > 1e-3 * np.abs(ua).max()


@pytest.mark.parametrize("axis,shift", [(0, 2), (2, 3)])
def test_3d_shift_moves_the_converged_field(axis, shift):
    rng = np.random.default_rng(4)
    g = rng.random((6, 7, 8)) < 0.2
    g[:, :, 0] = False                     # an open x1 path
    v, w = velocity_grid(3, 4)
    ua, ka = _converged(g, 0.5, v, w)
    ub, kb = _converged(np.roll(g, shift, axis=axis), 0.5, v, w)
    assert np.abs(np.roll(ua, shift, axis=axis + 1) - ub).max() < 1e-12 * np.abs(ua).max()
    assert kb == pytest.approx(ka, rel=1e-12)
    assert np.abs(ua - ub).max() > 1e-3 * np.abs(ua).max()
