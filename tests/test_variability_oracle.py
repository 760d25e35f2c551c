"""Pins of the high-variability pre-filter oracle (``oracle/variability_oracle.c``).

Sec. 2.2.1 of the paper: the expected photometric stability per 0.1-mag bin comes from a
sigma-clipped average over each chip's stars, and stars more than 2 sigma above it are
flagged.  The pins check each step another way: closed-form light curves, SciPy's own
sigma clipping, and catalogs whose answer is known by construction."""
import numpy as np
import pytest

import oracle
from paper_1112_1701_b300 import synth


def test_star_stats_closed_forms():
    m = np.array([15.0, 15.5] * 50, np.float32)             # +-0.25 about 15.25
    mag, rms = oracle.star_stats(m)
    assert mag == 15.25 and rms == 0.25
    mag, rms = oracle.star_stats(np.full(17, 18.125, np.float32))
    assert mag == 18.125 and rms == 0.0


@pytest.mark.parametrize("seed", range(4))
def test_star_stats_against_exact_rationals(seed):
    """Mean magnitude and population RMS against exact rational arithmetic on the FP32
    magnitudes: each within the FP64 bound of a plain n-term sum (n 2^-53 of the sum of
    magnitudes, plus the roundings of the division and the square root).  A sample sd
    (n - 1), a dropped square or a shifted mean would miss by far more."""
    from fractions import Fraction
    rng = np.random.default_rng(40 + seed)
    n = int(rng.integers(5, 400))
    m = (rng.uniform(14, 20) + rng.normal(0, 10 ** rng.uniform(-3, -1), n)).astype(np.float32)
    mag, rms = oracle.star_stats(m)
    q = [Fraction(float(v)) for v in m]
    mean = sum(q) / n
    var = sum((v - mean) ** 2 for v in q) / n
    u = 2.0 ** -53
    M = float(np.max(np.abs(m)))
    assert abs(Fraction(mag) - mean) <= (n + 1) * u * M
    exact_rms = float(var) ** 0.5
    assert abs(rms - exact_rms) <= (n + 1) * u * M + (n + 4) * u * exact_rms


def test_clip_margin_is_the_closest_decision():
    """The clip margin is the smallest | |v - mu| - clip sd | over the decisions of every
    round, recomputed here round by round in plain Python."""
    rng = np.random.default_rng(9)
    v = np.concatenate([rng.normal(0.02, 0.003, 60), [0.05, 0.2]])
    keep = np.ones(len(v), bool)
    best = np.inf
    for _ in range(5):
        kv = v[keep]
        mu = sum(kv.tolist()) / len(kv)
        sd = (sum(((x - mu) ** 2 for x in kv.tolist())) / len(kv)) ** 0.5
        gap = np.abs(np.abs(v - mu) - 3.0 * sd)
        best = min(best, float(gap.min()))
        nk = np.abs(v - mu) <= 3.0 * sd
        if np.array_equal(nk, keep):
            break
        keep = nk
    mu, sd, kept, mg = oracle.clip(v, 3.0, 5, with_margin=True)
    assert kept == int(keep.sum())
    assert mg == pytest.approx(best, rel=1e-9, abs=1e-15)


@pytest.mark.parametrize("seed", range(6))
def test_clip_equals_scipy_sigmaclip(seed):
    """With enough rounds to converge, the clipping is SciPy's sigmaclip (3 sigma both
    sides, population sd, inclusive bounds), whose result mean and sd must agree."""
    from scipy import stats
    rng = np.random.default_rng(seed)
    v = np.concatenate([rng.normal(0.02, 0.003, 200), rng.uniform(0.05, 0.3, 7)])
    mu, sd, kept = oracle.clip(v, 3.0, 100)
    c, lo, hi = stats.sigmaclip(v, 3.0, 3.0)
    assert kept == len(c)
    assert mu == pytest.approx(c.mean(), rel=1e-12)
    assert sd == pytest.approx(c.std(), rel=1e-12)


def test_clip_known_outlier():
    """Twenty ones and a ten: the ten lies 4.47 sd out and is dropped, after which the
    ones alone remain (mu = 1, sd = 0)."""
    mu, sd, kept = oracle.clip([1.0] * 20 + [10.0], 3.0, 5)
    assert (mu, sd, kept) == (1.0, 0.0, 20)
    mu, sd, kept = oracle.clip([1.0] * 20 + [10.0], 3.0, 0)     # no clipping rounds
    assert kept == 21 and mu == pytest.approx(30 / 21)


def _catalog(curves, chips):
    off = np.concatenate([[0], np.cumsum([len(c) for c in curves])]).astype(np.int64)
    return off, np.concatenate(curves).astype(np.float32), np.asarray(chips, np.int32)


def test_flags_by_construction():
    """One bin of 12 stars of identical RMS 0.01 and one of RMS 0.05: the loud star is
    clipped, the bin's sd is 0, so exactly the loud star is flagged.  A second chip with
    the same stars but only 3 of them (below min_stars) flags nothing."""
    base = np.array([17.03, 17.05] * 100, np.float32)        # mean 17.04, rms 0.01
    loud = np.array([17.00, 17.10] * 100, np.float32)        # mean 17.05, rms 0.05
    curves = [base] * 12 + [loud] + [base] * 2 + [loud]
    chips = [0] * 13 + [1] * 3
    off, m, chip = _catalog(curves, chips)
    o = oracle.variability(off, m, chip, 2, min_stars=5)
    assert o["flag"].tolist() == [0] * 12 + [1] + [0, 0, 0]
    assert np.all(o["bin"] == 170)
    assert o["mu"][0] == pytest.approx(0.01, abs=1e-6) and o["sd"][0] == pytest.approx(0.0, abs=1e-6)


def test_bins_follow_the_magnitude_grid():
    """0.1-mag bins on a fixed grid: floor(mag * 10); stars in different bins or chips are
    estimated separately."""
    curves = [np.full(10, v, np.float32) for v in (15.01, 15.09, 15.11, 15.19, 15.21)]
    off, m, chip = _catalog(curves, [0, 0, 0, 1, 0])
    o = oracle.variability(off, m, chip, 2, min_stars=1)
    assert o["bin"].tolist() == [150, 150, 151, 151, 152]
    assert o["flag"].sum() == 0          # constant curves: rms 0, nothing above 0


def test_injected_variables_are_flagged():
    """Synthetic chips with 1% eclipsing variables (0.1-0.4 mag dips on 10-20% of the
    epochs): nearly all variables are flagged, and the false-alarm rate of the quiet stars
    stays near the 2-sigma tail."""
    c = synth.chip_catalog(nchips=2, stars_per_chip=1500, npts=300, seed=21)
    o = oracle.variability(c.off, c.m, c.chip, c.nchips)
    f = o["flag"].astype(bool)
    assert f[c.variable].mean() > 0.85
    assert f[~c.variable].mean() < 0.05


def test_bad_arguments():
    off, m, chip = _catalog([np.ones(3, np.float32)], [5])
    with pytest.raises(ValueError):
        oracle.variability(off, m, chip, 2)
