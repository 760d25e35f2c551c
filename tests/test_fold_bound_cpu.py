"""Integer-exact CPU model of the fixed-point folds' edge windows (no GPU).

The fold-sweep kernels take a point's bin from a 32-bit fixed-point phase word q and re-fold
in FP64 only the points whose in-bin place r = q nb mod 2^32 lies within `tol` of a bin edge.
That is sound only if the derived bound on |q 2^-32 - frac(dt f)| is right.  This test models
the two integer folds exactly (Python integers; the same words, products and roundings) and
checks, against the oracle's FP64 bins, that no point outside the window has another bin:

  * direct: q = floor(DT F / 2^32) mod 2^32 with DT = RN_int(dt 2^s), F = RN_int(f 2^(64-s));
  * incremental (uniform grids): q = Q + tau D mod 2^32 with Q the direct word at the tile's
    reference column jc, D = RN(DT dF / 2^64) mod 2^32, dF = RN_int(df 2^(96-s)),
    tau = j - jc, and the window widened by |tau| times D's error, the grid's two FP64
    roundings and the FP64 definition's own rounding.

Inputs: long baselines at high frequencies, and points on exact bin edges.  Dropping the
dominant term of the incremental window (|tau| times D's rounding) makes the exact-edge case
fail; the smaller terms (the floor's one-sided nb, the grid roundings) are margins these
inputs do not resolve.  The CUDA arithmetic itself is checked against the oracle by the GPU
bin tests (`bls_debug_fold` runs both folds).
"""
import math

import numpy as np

import oracle
from paper_1112_1701_b300 import synth

M32 = (1 << 32) - 1


def _shift(dtmax):
    L = math.frexp(dtmax)[1] if dtmax > 0 else 0
    s = 34 - (L + 1) // 2
    s = min(s, 62 - L)
    return max(s, 1)


def _rn(x):
    return int(round(x))   # round half to even, as the device conversion


def _window(E, nb):
    tol = math.ceil(E * nb * 4294967296.0 * 1.01 + 4.0)
    return tol, int(4294967296.0 - 2.0 * tol - nb)


def _model_bins(dt, s, q_of_DT, E, nb):
    """(bins, in-window flags) of the points for phase words q_of_DT(DT)."""
    tol, fspan = _window(E, nb)
    b = np.empty(len(dt), np.int64)
    edge = np.empty(len(dt), bool)
    for i, v in enumerate(dt):
        q = q_of_DT(_rn(math.ldexp(float(v), s)))
        b[i] = (q * nb) >> 32
        r = (q * nb) & M32
        edge[i] = ((r - tol) & M32) >= fspan
    return b, edge


def _direct(dt, f, nb):
    dtmax = float(dt.max())
    s = _shift(dtmax)
    F = _rn(math.ldexp(f, 64 - s))
    E = (f * 2.0 ** -(s + 1) + dtmax * 2.0 ** (s - 65) + 2.0 ** -66
         + 2.0 ** -52 * (dtmax * f + 1.0))
    return _model_bins(dt, s, lambda DT: ((DT * F) >> 32) & M32, E, nb)


def _incremental(dt, fmin, df, nf, j, nb, T=128):
    dtmax = float(dt.max())
    s = _shift(dtmax)
    jc = min(j // T * T + T // 2, nf - 1)
    f, fc = oracle.freq(j, fmin, df), oracle.freq(jc, fmin, df)
    Fc = _rn(math.ldexp(fc, 64 - s))
    dF = _rn(math.ldexp(df, 96 - s))
    assert Fc < 2 ** 64 and dF < 2 ** 63
    tau = (j - jc) & M32

    def q_of(DT):
        Q = ((DT * Fc) >> 32) & M32
        D = ((DT * dF + (1 << 63)) >> 64) & M32
        return (Q + tau * D) & M32

    at = abs(j - jc)
    E = (fc * 2.0 ** -(s + 1) + dtmax * 2.0 ** (s - 65) + 2.0 ** -66
         + at * (2.0 ** -33 + df * 2.0 ** -(s + 1) + dtmax * 2.0 ** (s - 97) + 2.0 ** -98)
         + dtmax * max(f, fc) * 2.0 ** -51 * 1.01 + 2.0 ** -52 * (dtmax * f + 1.0))
    return _model_bins(dt, s, q_of, E, nb)


def _check(t, fmin, df, nf, nb, js):
    t = np.asarray(t, np.float64)
    dt = t - t.min()
    bo = oracle.bins(t, [oracle.freq(j, fmin, df) for j in js], nb)
    nedge = 0
    for q, j in enumerate(js):
        for b, edge in (_direct(dt, oracle.freq(j, fmin, df), nb),
                        _incremental(dt, fmin, df, nf, j, nb)):
            wrong = (b != bo[q]) & ~edge
            assert not wrong.any(), (j, int(wrong.sum()))
            nedge += int(edge.sum())
    return nedge / (2 * len(js) * len(t))


def test_windows_hold_three_year_baseline_high_frequencies():
    b = synth.config3(ncurves=1, nf=200000)
    c, g = b.curves[0], b.grids[0]
    js = [0, 1, 63, 64, 127, 128, 100031, 199871, 199935, 199936, 199999]
    rate = _check(c.t, g.fmin, g.df, g.nf, 200, js)
    assert rate < 2e-3        # the reference point (dt = 0) is always in the window


def test_windows_hold_on_exact_bin_edges():
    nb, f0, df, nf = 64, 0.5, 0.001, 1000
    js = [0, 2, 63, 64, 65, 127, 998, 999]
    rng = np.random.default_rng(5)
    dts = [np.array([0.0])]
    for j in js:
        f = oracle.freq(j, f0, df)
        dts.append((rng.integers(0, 200, 24) + rng.integers(0, nb, 24) / nb) / f)
    t = synth.T0 + np.sort(np.concatenate(dts))
    _check(t, f0, df, nf, nb, js)


def test_incremental_window_is_small_on_the_batched_workload():
    b = synth.config2(ncurves=2, nf=50000)
    for c, g in zip(b.curves, b.grids):
        js = [0, 64, 127, 25000, 49983, 49999]
        assert _check(c.t, g.fmin, g.df, g.nf, 200, js) < 2e-3
