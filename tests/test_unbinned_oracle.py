"""Pins of the unbinned (edge-to-edge) BLS oracle (``oracle/unbinned_oracle.c``).

Boxes are cyclic runs of consecutive points in (phase, index) order whose phase extent lies
in [qmin, qmax]; phases are the binned search's FP64 fold frac(RN(dt f)).  The pins check
the phases against exact rational arithmetic, the order against a plain sort, enumerate
every run on tiny inputs with an explicit least-squares fit, and check the relation to the
binned search and a noise-free box."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1112_1701_b300 import synth


@pytest.mark.parametrize("seed", range(5))
def test_phases_within_one_rounding_of_exact(seed):
    """phi = frac(RN(dt f)): the product rounds once (relative 2^-53) and the fraction is
    exact, so phi is within 2^-53 dt f of the exact frac(dt f), modulo one cycle (a product
    that rounds up to an integer gives phase 0 for an exact fraction just below 1)."""
    rng = np.random.default_rng(seed)
    dt = np.concatenate([[0.0], np.sort(rng.uniform(0, 10 ** rng.uniform(-1, 3.5), 50))])
    for f in rng.uniform(0.05, 20.0, 5):
        phi = oracle.ubls_phases(dt, f)
        assert np.all((phi >= 0.0) & (phi < 1.0))
        for d, ph in zip(dt, phi):
            ex = Fraction(float(d)) * Fraction(float(f))
            fr = ex - math.floor(ex)
            err = min(abs(Fraction(float(ph)) - fr), abs(Fraction(float(ph)) + 1 - fr))
            assert err <= Fraction(2) ** -53 * ex + Fraction(2) ** -80


def test_order_is_phase_then_index():
    """Equal phases (repeated times, and times a whole number of periods apart) keep their
    index order; otherwise ascending phase."""
    dt = np.array([3.0, 0.5, 3.0, 1.0, 0.0, 2.5, 5.0, 0.25])
    phi = oracle.ubls_phases(dt, 1.0)
    order = oracle.ubls_order(phi)
    expect = sorted(range(len(dt)), key=lambda i: (phi[i], i))
    assert order.tolist() == expect
    assert order.tolist()[:4] == [0, 2, 3, 4]          # phase 0: indices ascending
    # extents: a run wrapping through phase 0 adds a cycle
    q = order.tolist().index(7)                        # phase 0.25, then 0.5, 0.5
    assert oracle.ubls_extent(phi, order, q, 3) == 0.25
    assert oracle.ubls_extent(phi, order, q, 6) == 0.75  # 0.25 .. 0.5, then 0 (+1)


def _brute(dt, w, x, f, qmin, qmax):
    """Every cyclic run of the (phase, index) order, its extent in FP64 from the phases,
    P from an explicit weighted least-squares fit of a two-level step."""
    n = len(dt)
    phi = [float(d) * float(f) - math.floor(float(d) * float(f)) for d in dt]
    order = sorted(range(n), key=lambda i: (phi[i], i))
    best = 0.0
    for a in range(n):
        for ln in range(1, n):
            run = [order[(a + q) % n] for q in range(ln)]
            d = phi[run[-1]] - phi[run[0]]
            E = d + 1.0 if a + ln - 1 >= n else d
            if E > qmax or E < qmin:
                continue
            s_ind = np.zeros(n)
            s_ind[run] = 1.0
            A = np.stack([np.ones(n), s_ind], axis=1) * np.sqrt(w)[:, None]
            coef, *_ = np.linalg.lstsq(A, x * np.sqrt(w), rcond=None)
            if coef[1] >= 0:          # dips only
                continue
            chi2 = float(np.sum((x * np.sqrt(w) - A @ coef) ** 2))
            best = max(best, float(np.sum(w * x * x)) - chi2)
    return best


@pytest.mark.parametrize("seed", range(10))
def test_best_box_equals_brute_force(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(3, 11))
    t = synth.T0 + np.sort(rng.uniform(0, 20, n))
    y = (1 + rng.normal(0, 0.01, n)).astype(np.float32)
    dy = rng.uniform(0.005, 0.02, n).astype(np.float32)
    dt, w, x, _ = oracle.prep(t, y, dy)
    for f in rng.uniform(0.1, 3.0, 3):
        for qmin, qmax in ((0.0, 0.3), (0.02, 0.5)):
            P, a, ln, r, s, order = oracle.ubls_power(dt, w, x, f, qmin, qmax)
            assert P == pytest.approx(_brute(dt, w, x, f, qmin, qmax), rel=1e-9, abs=1e-15)


def test_unbinned_at_least_binned_when_qmin_is_zero():
    """Every binned box (k bins, k/nb <= qmax) holds points spanning at most k/nb of phase,
    so with qmin = 0 its point set is also an unbinned box: the unbinned maximum is at
    least the binned one."""
    b = synth.config1()
    c, g = b.curves[0], b.grids[0]
    kmin, kmax = oracle.kminmax(100, b.qmin, b.qmax)
    dt, w, x, _ = oracle.prep(c.t, c.y, c.dy)
    for j in (0, 250, 1000, 1876):
        f = oracle.freq(j, g.fmin, g.df)
        Pb, *_ = oracle.power(dt, w, x, f, 100, kmin, kmax)
        # (a hair above kmax/nb: the box's FP64 extent may exceed k/nb by an ulp)
        Pu, *_ = oracle.ubls_power(dt, w, x, f, 0.0, kmax / 100 + 1e-12)
        assert Pu >= Pb * (1 - 1e-12)


def test_noise_free_box_fits_perfectly():
    rng = np.random.default_rng(8)
    n = 400
    t = synth.T0 + np.sort(rng.uniform(0, 30, n))
    P0, dur = 1.7, 0.12
    y = np.where(np.mod(t - synth.T0 - 0.3, P0) < dur, 0.97, 1.0).astype(np.float32)
    Pspec, pk = oracle.ubls(t, y, None, 0.01, 0.2, freqs=np.array([1 / P0 * 0.97, 1 / P0]))
    dt, w, x, scal = oracle.prep(t, y, None)
    assert pk.j == 1
    assert pk.power == pytest.approx(scal[3], rel=1e-9)       # chi2 = 0
    assert pk.depth == pytest.approx(0.03, rel=1e-5)
    assert pk.duration <= dur
    inbox = np.mod(t - synth.T0 - 0.3, P0) < dur
    assert pk.len == int(inbox.sum())


def test_bad_arguments():
    t = synth.T0 + np.arange(5.0)
    with pytest.raises(ValueError):
        oracle.ubls(t, np.ones(5, np.float32), None, 0.3, 0.2, freqs=np.array([1.0]))
