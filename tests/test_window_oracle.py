"""Pins of the eclipse-window detection-efficiency oracle (``oracle/window_oracle.c``).

The efficiency follows the paper's definition (Sec. 5, detection-efficiency figure): the
probability, over the unknown eclipse phase, that at least two eclipses contain
observations.  The oracle folds every time at each (frequency, phase); the pins below
reach the same numbers another way: by enumerating the eclipse intervals in time, by
closed forms for dense and for one-per-night cadences, and by invariants."""
import math

import numpy as np
import pytest

import oracle


def _intervals_count(t, f, phi, D, min_points=1):
    """Independent formulation: eclipse n spans [c_n - D/2, c_n + D/2] with
    c_n = t_0 + (phi + n)/f; count the intervals holding >= min_points times."""
    P = 1.0 / f
    t0 = t[0]
    nlo = math.floor((t[0] - t0) / P - phi) - 2
    nhi = math.ceil((t[-1] - t0) / P - phi) + 2
    seen = 0
    for n in range(nlo, nhi + 1):
        c = t0 + (phi + n) * P
        k = sum(1 for ti in t if abs(ti - c) <= D / 2)
        if k >= min_points:
            seen += 1
    return seen


@pytest.mark.parametrize("seed", range(12))
def test_counts_match_interval_enumeration(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 40))
    t = np.sort(rng.uniform(0.0, 30.0, n)) + 2455000.0
    nphi = 16
    freqs = rng.uniform(0.05, 3.0, 7)
    D = float(rng.uniform(0.02, 0.3))
    mp = int(rng.integers(1, 3))
    _, counts = oracle.window(t, nphi, freqs=freqs, duration=D, min_points=mp,
                              want_counts=True)
    for k, f in enumerate(freqs):
        for m in range(nphi):
            phi = (2 * m + 1) / (2 * nphi)
            assert counts[k, m] == _intervals_count(list(t), f, phi, D, mp), (k, m)


def test_dense_cadence_closed_forms():
    """Observations every 0.01 d for 30 d, eclipses 0.05 d long: every eclipse whose
    window lies inside the span is observed.  Periods below 10 d always show >= 2
    eclipses (efficiency 1); periods above the span plus a duration show at most one
    (efficiency 0)."""
    t = 2455000.0 + np.arange(3001) * 0.01
    freqs = np.array([1 / 0.5, 1 / 3.3, 1 / 9.9, 1 / 31.0, 1 / 80.0])
    eff, _ = oracle.window(t, 64, freqs=freqs, duration=0.05)
    assert eff[:3].tolist() == [1.0, 1.0, 1.0]
    assert eff[3:].tolist() == [0.0, 0.0]


def test_integer_day_alias_closed_form():
    """One observation per night at the same clock time, P = 1 d: every night sees the
    same phase, so either every night is in eclipse or none is.  The phases in eclipse
    are those within h = D/2 cycles of 0 (or 1): (2m+1)/(2 nphi) <= h or >= 1 - h."""
    nights = 40
    t = 2455000.0 + np.arange(nights, dtype=np.float64)
    nphi, D = 100, 0.105                   # h = 0.0525 cycle at f = 1 (no phase on the edge)
    eff, counts = oracle.window(t, nphi, freqs=np.array([1.0]), duration=D, want_counts=True)
    phis = (2 * np.arange(nphi) + 1) / (2 * nphi)
    inside = (phis <= 0.0525) | (phis >= 0.9475)
    assert eff[0] == inside.mean() == 0.10
    assert np.array_equal(counts[0], np.where(inside, nights, 0))


def test_alias_drifts_off_integer_period():
    """A period slightly off one day walks the eclipse through the nightly windows, so
    the efficiency rises well above the integer-day value."""
    t = np.sort(np.concatenate([2455000.0 + d + np.linspace(0.1, 0.3, 13) for d in range(60)]))
    eff, _ = oracle.window(t, 200, freqs=np.array([1.0, 1 / 1.07]), duration=0.04)
    assert eff[0] < 0.35 < 0.9 < eff[1]


def test_min_eclipses_and_min_points_monotone():
    rng = np.random.default_rng(7)
    t = np.sort(rng.uniform(0, 20, 200))
    freqs = rng.uniform(0.1, 2.0, 11)
    e0, _ = oracle.window(t, 32, freqs=freqs, duration=0.1, min_eclipses=0)
    e1, _ = oracle.window(t, 32, freqs=freqs, duration=0.1, min_eclipses=1)
    e2, _ = oracle.window(t, 32, freqs=freqs, duration=0.1, min_eclipses=2)
    e2p, _ = oracle.window(t, 32, freqs=freqs, duration=0.1, min_eclipses=2, min_points=3)
    assert np.all(e0 == 1.0)
    assert np.all(e1 >= e2) and np.all(e2 >= e2p)


def test_single_point():
    t = np.array([5.0])
    e2, _ = oracle.window(t, 50, freqs=np.array([0.5]), qfrac=0.11)
    e1, c = oracle.window(t, 50, freqs=np.array([0.5]), qfrac=0.11, min_eclipses=1,
                          want_counts=True)
    assert e2[0] == 0.0
    # dt = 0: u = -phi, in eclipse iff min(phi, 1 - phi) <= 0.055
    phis = (2 * np.arange(50) + 1) / 100
    assert np.array_equal(c[0], ((phis <= 0.055) | (phis >= 0.945)).astype(np.int32))
    assert e1[0] == 0.12


def test_uniform_grid_and_fraction_of_period():
    """The uniform grid is RN(fmin + RN(k df)) (the search's grid), and a duration given
    as a fraction q of the period means h = q/2 at every frequency."""
    rng = np.random.default_rng(3)
    t = np.sort(rng.uniform(0, 50, 120))
    fmin, df, nf = 0.2, 0.013, 40
    eu, cu = oracle.window(t, 24, fmin=fmin, df=df, nf=nf, qfrac=0.06, want_counts=True)
    grid = np.array([oracle.freq(k, fmin, df) for k in range(nf)])
    ee, ce = oracle.window(t, 24, freqs=grid, qfrac=0.06, want_counts=True)
    assert np.array_equal(eu, ee) and np.array_equal(cu, ce)
    for k in (0, 17, 39):
        for m in (0, 11):
            phi = (2 * m + 1) / 48
            assert cu[k, m] == _intervals_count(list(t), grid[k], phi, 0.06 / grid[k])


def test_time_offset_invariance_exact():
    """dt = t - t_0 is exact for dyadic times, so an offset by an integer changes nothing."""
    rng = np.random.default_rng(11)
    t = np.sort(np.round(rng.uniform(0, 25, 80) * 1024) / 1024)
    f = rng.uniform(0.1, 2, 9)
    _, c1 = oracle.window(t, 20, freqs=f, duration=0.07, want_counts=True)
    _, c2 = oracle.window(t + 2455000.0, 20, freqs=f, duration=0.07, want_counts=True)
    assert np.array_equal(c1, c2)


def test_bad_arguments_rejected():
    with pytest.raises(ValueError):
        oracle.window(np.array([2.0, 1.0]), 4, freqs=np.array([1.0]), duration=0.1)
    with pytest.raises(ValueError):
        oracle.window(np.array([1.0, 2.0]), 4, freqs=np.array([1.0]))
    with pytest.raises(ValueError):
        oracle.window(np.array([1.0, np.nan]), 4, freqs=np.array([1.0]), duration=0.1)
