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

The kernels evaluate the incremental window in FP32 with upward rounding from per-curve
coefficients (prep kernel); a model of that evaluation is checked never to give a narrower
window than the FP64 bound (dropping the tile-offset term makes it fail).

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


def _up32(x):
    """The smallest FP32 number >= the exact rational x (upward rounding)."""
    from fractions import Fraction
    v = np.float32(float(x))
    while Fraction(float(v)) < x:
        v = np.nextafter(v, np.float32(np.inf))
    while True:
        w = np.nextafter(v, np.float32(-np.inf))
        if Fraction(float(w)) >= x:
            v = w
        else:
            return v


def _window_fp32(dtm, df, s, f, fc, tau, nb):
    """The kernels' per-column window: per-curve coefficients formed in FP64 and rounded up
    to FP32, then the column's bound with every FP32 operation rounded up."""
    from fractions import Fraction as Fr
    ewc = _up32(Fr(2.0 ** -(s + 1)))
    ew0 = _up32(Fr(dtm * 2.0 ** (s - 65) + 2.0 ** -66 + 2.0 ** -52))
    ewt = _up32(Fr(2.0 ** -33 + df * 2.0 ** -(s + 1) + dtm * 2.0 ** (s - 97) + 2.0 ** -98))
    ewh = _up32(Fr(dtm * 2.0 ** -51 * 1.0101))
    ewf = _up32(Fr(dtm * 2.0 ** -52))
    ff, fcf = _up32(Fr(f)), _up32(Fr(fc))
    at = np.float32(abs(tau))

    def fma(a, b, c):
        return _up32(Fr(float(a)) * Fr(float(b)) + Fr(float(c)))

    E = fma(fcf, ewc, ew0)
    E = fma(at, ewt, E)
    E = fma(max(ff, fcf), ewh, E)
    E = fma(ff, ewf, E)
    t = _up32(Fr(float(E)) * nb)
    t = _up32(Fr(float(t)) * 2 ** 32)
    t = _up32(Fr(float(t)) * Fr(float(np.float32(1.0101))))
    t = _up32(Fr(float(t)) + 4)
    return float(t)


def test_fp32_windows_never_narrower_than_the_fp64_bound():
    """The incremental fold's window is computed in FP32 with upward rounding from per-curve
    coefficients; over baselines of days to years, grids up to 20 cycles per day, tile
    offsets up to 64 and bin counts 2-4096, it is never below the FP64 bound's window."""
    rng = np.random.default_rng(21)
    checked = 0
    for _ in range(300):
        dtm = float(10.0 ** rng.uniform(0, 3.1))
        s = _shift(dtm)
        df = float(10.0 ** rng.uniform(-7, -2))
        f = float(rng.uniform(0.01, 20.0))
        tau = int(rng.integers(-64, 65))
        fc = f - tau * df
        if fc <= 0:
            continue
        nb = int(rng.choice([2, 7, 100, 200, 256, 400, 4096]))
        E64 = (fc * 2.0 ** -(s + 1) + dtm * 2.0 ** (s - 65) + 2.0 ** -66
               + abs(tau) * (2.0 ** -33 + df * 2.0 ** -(s + 1) + dtm * 2.0 ** (s - 97) + 2.0 ** -98)
               + dtm * max(f, fc) * 2.0 ** -51 * 1.01 + 2.0 ** -52 * (dtm * f + 1.0))
        tol64 = math.ceil(E64 * nb * 4294967296.0 * 1.01 + 4.0)
        tolu = _window_fp32(dtm, df, s, f, fc, tau, nb)
        if tolu >= 1.0e9:
            continue   # the fold falls back to FP64 for the tile
        assert math.ceil(tolu) >= tol64, (dtm, df, f, tau, nb, tolu, tol64)
        checked += 1
    assert checked > 200
