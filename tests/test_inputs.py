"""Seeded geometry generators (CPU)."""
import numpy as np
import pytest

from paper_1712_01132_gb300 import inputs


def test_cylinder_cell_porosity():
    s = inputs.cylinder_cell(32, 0.7)
    assert s.shape == (32, 32)
    assert 1 - s.mean() == pytest.approx(0.7, abs=0.01)
    assert np.array_equal(s, s[::-1, :]) and np.array_equal(s, s[:, ::-1])


def test_random_discs_seeded_and_filled():
    a = inputs.random_discs(128, 96, seed=7)
    b = inputs.random_discs(128, 96, seed=7)
    assert np.array_equal(a, b)
    raw = inputs.random_discs(128, 96, seed=7, percolating=False)
    assert raw.mean() >= 0.5
    assert np.all(a >= raw)          # the filter only adds solid


def test_keep_percolating_fills_pockets_and_blocked_channels():
    s = np.ones((8, 10), bool)
    s[2, :] = False                  # a channel through the whole x1 period
    s[5, 3:6] = False                # an isolated pocket
    out = inputs.keep_percolating(s)
    assert not out[2].any()
    assert out[5].all()
    blocked = s.copy()
    blocked[2, 4] = True             # interrupt the channel: nothing percolates
    assert inputs.keep_percolating(blocked).all()


def test_keep_percolating_follows_periodic_wrap():
    s = np.ones((6, 8), bool)
    # a path that closes an x1 period only through the lateral periodic face:
    # row 5 col 7 -> (x1 wrap) row 5 col 0 -> (lateral wrap) row 0 col 0 -> row 0 col 4
    # -> (lateral wrap) row 5 col 4 -> row 5 col 7
    s[0, 0:5] = False
    s[5, 4:8] = False
    s[5, 0] = False
    out_periodic = inputs.keep_percolating(s, lateral_periodic=True)
    assert not out_periodic[0, 0:5].any() and not out_periodic[5, 4:8].any()
    out_closed = inputs.keep_percolating(s, lateral_periodic=False)
    assert out_closed.all()


def test_gaussian_rock_porosity_and_percolation():
    raw = inputs.gaussian_rock(32, seed=0, corr_len=4.0, porosity=0.35, percolating=False)
    assert 1 - raw.mean() == pytest.approx(0.35, abs=1e-3)
    kept = inputs.gaussian_rock(32, seed=0, corr_len=4.0, porosity=0.35)
    assert kept.shape == (32, 32, 32)
    assert np.all(kept >= raw) and (1 - kept.mean()) > 0.2


def test_sphere_quadrant_porosity():
    s = inputs.sphere_quadrant(40, 20, 20, porosity=0.75)
    assert 1 - s.mean() == pytest.approx(0.75, abs=0.01)


def test_disc_batch_recipe():
    """Sides in [64, 512], porosity at most the drawn target (filling non-percolating pockets only
    lowers it), Kn in [0.01, 10], no geometry without a fluid path, deterministic."""
    a = inputs.disc_batch(6, seed0=1000)
    b = inputs.disc_batch(6, seed0=1000)
    assert len(a) == 6
    for (m, kn, seed), (m2, kn2, seed2) in zip(a, b):
        assert np.array_equal(m, m2) and kn == kn2 and seed == seed2
        assert 64 <= m.shape[0] <= 512 and 64 <= m.shape[1] <= 512
        assert 0.01 <= kn <= 10.0
        assert (~m).any() and 1.0 - m.mean() <= 0.7 + 1e-9
    seeds = [s for _, _, s in a]
    assert seeds == sorted(seeds) and seeds[0] == 1000
