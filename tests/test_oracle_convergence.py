"""Pins of the oracle's convergence measure, Eq. 15 (Sec. 3.1, steps iv-v).

Err(l) = |k(l) - k(l - 100)| / (100 |k(l)|), evaluated every 100 iterations; the iteration stops at
the first check with Err below the tolerance.  The solver is replaced by a hand-written
permeability history, so these tests fix the bookkeeping of ``Oracle.run`` alone: the divisor, the
check that is compared with (the previous check, not the previous iteration), where checks fall,
and the stopping iteration.  Every expected number below is worked out by hand from the history.
"""
import math

import pytest

import oracle


class _History(oracle.Oracle):
    """An Oracle whose iterations only advance a counter and report k(l) from a given function."""

    def __init__(self, k_of_l, k0=0.0):   # no C solver behind it
        self._h = None
        self._l = 0
        self._k = k_of_l
        self._k0 = k0
        self.k_history = []
        self.k_check = 0.0
        self.it_check = 0
        self.err = math.inf
        self.calls = []

    @property
    def iterations(self):
        return self._l

    def iterate(self, n):
        self.calls.append(n)
        ks = [self._k(self._l + i + 1) for i in range(n)]
        self._l += n
        self.k_history.extend(ks)
        return ks

    def permeability(self):
        return self._k(self._l) if self._l else self._k0


def _geometric(l):
    # k(l) = 1 - 10^(-l/100): 0.9, 0.99, 0.999, 0.9999, 0.99999 at l = 100 ... 500
    return 1.0 - 10.0 ** (-l / 100.0)


def test_eq15_every_100_iterations_stops_at_the_first_check_below_tol():
    o = _History(_geometric)
    it, k, err = o.run(1e-6, 10000)
    # Err(100) = 1/100 (start state k = 0); Err(200) = 0.09/(100*0.99) = 9.09e-4;
    # Err(300) = 0.009/99.9 = 9.009e-5; Err(400) = 0.0009/99.99 = 9.0009e-6;
    # Err(500) = 0.00009/99.999 = 9.00009e-7 < 1e-6: stop at 500
    assert it == 500
    assert o.calls == [100] * 5
    assert k == pytest.approx(0.99999, rel=1e-14)
    assert err == pytest.approx(0.00009 / 99.999, rel=1e-9)


def test_eq15_first_check_compares_with_the_zero_start():
    o = _History(_geometric)
    it, _, err = o.run(0.011, 10000)       # Err(100) = 0.9 / (100 * 0.9) = 0.01 < 0.011
    assert it == 100
    assert err == pytest.approx(0.01, rel=1e-14)


def test_eq15_tolerance_between_two_checks():
    o = _History(_geometric)
    it, _, err = o.run(1e-5, 10000)        # Err(400) = 9.0009e-6 is the first below 1e-5
    assert it == 400
    assert err == pytest.approx(0.0009 / 99.99, rel=1e-9)
    o = _History(_geometric)
    it, _, err = o.run(9.0e-6, 10000)      # 9.0009e-6 is not below 9.0e-6; Err(500) is
    assert it == 500


def test_eq15_with_check_interval_50():
    # k(l) = l / (l + 50): at the m-th check k(50 m) = m / (m + 1), so
    # k(50 m) - k(50 (m - 1)) = m/(m + 1) - (m - 1)/m = 1 / (m (m + 1)), and dividing by
    # 50 k(50 m) = 50 m / (m + 1) gives Err(50 m) = 1 / (50 m^2) (m = 1: 1/50, the zero start)
    o = _History(lambda l: l / (l + 50.0))
    it, _, err = o.run(1e-4, 10000, check_interval=50)
    # 1/(50 m^2) < 1e-4  <=>  m^2 > 200  <=>  m >= 15: stop at l = 750 with Err = 1/11250
    assert it == 750
    assert o.calls == [50] * 15
    assert err == pytest.approx(1.0 / 11250.0, rel=1e-12)


def test_eq15_is_not_the_change_over_one_iteration():
    # a history that is flat between checks except for one jump just before the check: the
    # change over the last iteration is 0 at every check but the change over 100 iterations is not
    def k(l):
        return 1.0 + (0.5 if l >= 150 else 0.0)
    o = _History(k)
    it, _, err = o.run(1e-3, 300)
    # Err(100) = 1/100; Err(200) = 0.5 / (100 * 1.5) = 3.33e-3 (not 0); Err(300) = 0 < 1e-3
    assert it == 300
    assert err == 0.0
    assert o.calls == [100, 100, 100]


def test_eq15_checks_fall_on_multiples_of_the_interval_across_calls():
    o = _History(_geometric)
    it, _, err = o.run(0.0, 130)           # one check at 100, then 30 iterations without a check
    assert it == 130 and o.calls == [100, 30]
    assert err == pytest.approx(0.01, rel=1e-14)
    it, _, err = o.run(0.0, 200)           # 70 more iterations to the check at 200
    assert it == 200 and o.calls == [100, 30, 70]
    assert err == pytest.approx(0.09 / 99.0, rel=1e-12)


def test_eq15_after_a_warm_start_compares_with_the_warm_state():
    o = _History(_geometric, k0=0.5)
    o.k_check, o.it_check = o.permeability(), o.iterations    # what set_initial records
    it, _, err = o.run(0.5, 10000)
    # Err(100) = |0.9 - 0.5| / (100 * 0.9) = 4.44e-3, not 1/100
    assert it == 100
    assert err == pytest.approx(0.4 / 90.0, rel=1e-12)


def test_eq15_divides_by_the_iterations_since_a_moved_check():
    o = _History(_geometric)
    o.run(0.0, 100)
    o._l = 130                              # a warm start at iteration 130 with k(130) recorded
    o.k_check, o.it_check = _geometric(130), 130
    it, _, err = o.run(0.0, 200)            # next check at 200, 70 iterations after the warm start
    assert it == 200
    assert err == pytest.approx((_geometric(200) - _geometric(130)) / (70 * _geometric(200)), rel=1e-12)


def test_zero_permeability_has_zero_error():
    o = _History(lambda l: 0.0)
    it, _, err = o.run(1e-6, 1000)
    assert it == 100 and err == 0.0
