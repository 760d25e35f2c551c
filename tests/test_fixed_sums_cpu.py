"""CPU model of the fixed-point sum mode's quantisation and its error bound (no GPU).

In the fixed-point sum mode the prep kernel rounds each point's weight and weighted flux once
to integers, W_i = RN(w_i Sw) with Sw = 2^32 - 2n - 16 and X_i = RN(w_i x_i Sx) with
Sx = (2^31 - n - 16) / sum|w x|; the binning kernels add them exactly (32-bit integer
reductions) and the sweep reads r = fl(fl(sum W) fl(1/sum_all W)) and
s = fl(fl(sum X) fl(1/Sx)).  This test models that arithmetic in numpy (FP64 products rounded
to integers half to even, FP32 conversions) on the oracle's FP64 weights and checks:

  * no overflow: sum W < 2^32 and sum |X| < 2^31 for every curve, so no bin's integer sums
    can wrap, whatever points it holds;
  * the derived bound on every box's r and s against exact FP64 sums of the definition:
        |r_fix - r| <= (m/2 + r n/2) / sum W + 3.01 * 2^-24 r
        |s_fix - s| <= m / (2 Sx) + 3.01 * 2^-24 |s|          (m points in the box);
  * the bound's margin in Sw is needed: with Sw = 2^32 equal weights can round the total
    past 2^32 (seven points).
"""
import math

import numpy as np

import oracle
from paper_1112_1701_b300 import synth

U = 2.0 ** -24


def _quantise(w, wx, sw_margin=True):
    n = len(w)
    Sw = 2.0 ** 32 - (2 * n + 16 if sw_margin else 0)
    ax = math.fsum(np.abs(wx))
    Sx = (2.0 ** 31 - n - 16) / ax if ax > 0 else 1.0
    W = np.rint(w * Sw).astype(np.int64)
    X = np.rint(wx * Sx).astype(np.int64)
    return W, X, Sw, Sx


def _boxes(t, nb, rng, nfreq=6):
    """Point sets of cyclic runs of phase bins at a few frequencies (the oracle's bins)."""
    f = rng.uniform(0.2, 5.0, nfreq)
    B = oracle.bins(t, f, nb)
    out = []
    for row in B:
        for _ in range(40):
            i1, k = int(rng.integers(nb)), int(rng.integers(1, nb // 2))
            sel = ((row - i1) % nb) < k
            if sel.any():
                out.append(sel)
    return out


def _check_curve(t, y, dy, nb, rng):
    dt, w, x, scal = oracle.prep(t, y, dy)
    wx = w * x
    W, X, Sw, Sx = _quantise(w, wx)
    n = len(t)
    assert int(W.sum()) < 2 ** 32 and int(np.abs(X).sum()) < 2 ** 31
    Wtot = int(W.sum())
    wq = np.float32(1.0 / Wtot)
    xq = np.float32(1.0 / Sx)
    worst = 0.0
    for sel in _boxes(t, nb, rng):
        m = int(sel.sum())
        r = math.fsum(w[sel])
        s = math.fsum(wx[sel])
        r_fix = float(np.float32(np.float32(int(W[sel].sum())) * wq))
        s_fix = float(np.float32(np.float32(int(X[sel].sum())) * xq))
        br = (m / 2 + r * n / 2) / Wtot * (1 + 1e-9) + 3.01 * U * r
        bs = m / (2 * Sx) * (1 + 1e-9) + 3.01 * U * abs(s)
        assert abs(r_fix - r) <= br, (m, r, r_fix - r, br)
        assert abs(s_fix - s) <= bs, (m, s, s_fix - s, bs)
        worst = max(worst, abs(r_fix - r) / br, abs(s_fix - s) / bs)
    return worst


def test_bound_holds_on_batched_curves():
    b = synth.config2(ncurves=6, nf=10)
    rng = np.random.default_rng(11)
    for c in b.curves:
        assert _check_curve(c.t, c.y, c.dy, 200, rng) <= 1.0


def test_bound_holds_on_long_curve_with_mixed_errors():
    rng = np.random.default_rng(12)
    n = 20000
    t = synth.T0 + np.sort(rng.uniform(0, 90, n))
    y = (1 + rng.normal(0, 0.02, n)).astype(np.float32)
    dy = rng.uniform(0.002, 0.1, n).astype(np.float32)   # weights spread over 2500x
    assert _check_curve(t, y, dy, 256, rng) <= 1.0


def test_equal_weights_need_the_total_margin():
    w = np.full(7, 1.0 / 7.0)
    W, _, _, _ = _quantise(w, np.zeros(7), sw_margin=False)
    assert int(W.sum()) > 2 ** 32 - 1          # 2^32 / 7 rounds up: the total would wrap
    W, _, _, _ = _quantise(w, np.zeros(7))
    assert int(W.sum()) < 2 ** 32
