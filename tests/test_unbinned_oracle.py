"""Pins of the unbinned (edge-to-edge) BLS oracle (``oracle/unbinned_oracle.c``).

Boxes are cyclic runs of consecutive points in phase order whose phase extent lies in
[qmin, qmax]; phases are 64-bit fixed-point fractions (so ordering and extents are exact
integer decisions).  The pins recompute the phase keys with Python integers, enumerate every
run on tiny inputs with an explicit least-squares fit, and check the relation to the binned
search and a noise-free box."""
import math

import numpy as np
import pytest

import oracle
from paper_1112_1701_b300 import synth


def _keys_py(dt, f):
    dtmax = float(np.max(dt))
    L = (math.frexp(dtmax)[1]) if dtmax > 0 else 0      # dtmax < 2^L
    s = 34 - int((L + 1) / 2)
    s = max(1, min(s, 62 - L))
    F = round(math.ldexp(f, 64 - s))
    return np.array([((round(math.ldexp(float(d), s)) * F) % 2 ** 64) >> 32 for d in dt],
                    dtype=np.uint64), s


@pytest.mark.parametrize("seed", range(5))
def test_phase_keys_match_integer_arithmetic(seed):
    rng = np.random.default_rng(seed)
    dt = np.concatenate([[0.0], np.sort(rng.uniform(0, 10 ** rng.uniform(-1, 3.5), 50))])
    dtmax = float(dt.max())
    for f in rng.uniform(0.05, 20.0, 5):
        kc = oracle.ubls_keys(dt, dtmax, f)
        kp, s = _keys_py(dt, f)
        assert oracle.fx_shift(dtmax) == s
        assert np.array_equal(kc.astype(np.uint64), kp)


def _brute(dt, w, x, f, qmin, qmax):
    """Every cyclic run of the phase order, its extent from the keys, P from an explicit
    weighted least-squares fit of a two-level step."""
    n = len(dt)
    key, _ = _keys_py(dt, f)
    order = sorted(range(n), key=lambda i: (int(key[i]), i))
    QMIN = math.ceil(qmin * 2 ** 32)
    QMAX = math.floor(qmax * 2 ** 32)
    best = 0.0
    for a in range(n):
        for ln in range(1, n):
            run = [order[(a + q) % n] for q in range(ln)]
            E = (int(key[run[-1]]) - int(key[run[0]])) % 2 ** 32
            if E > QMAX:
                break
            if E < QMIN:
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
            P, a, ln, r, s, order = oracle.ubls_power(dt, w, x, float(dt.max()), f, qmin, qmax)
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
        Pu, *_ = oracle.ubls_power(dt, w, x, float(dt.max()), f, 0.0, kmax / 100)
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
