"""Pins of the trapezoid-refit oracle (``oracle/shape_oracle.c``).

The refit is a weighted least-squares fit of a trapezoid (flat bottom, linear ingress and
egress) to the folded flux at a peak's frequency; the paper's discussion (Sec. 5) names the
eclipse duration and the flat-bottomed shape as discriminators.  The pins reach the same
numbers by other routes: an explicit least-squares solve, the BLS box power, and exactly
known injected shapes."""
import numpy as np
import pytest

import oracle
from paper_1112_1701_b300 import synth


def _lstsq_power(phi, w, x, c, T, tau):
    """Independent route: shape values by explicit geometry, then a weighted linear fit of
    x on [1, s] with numpy; Q = sum w x^2 - chi2."""
    D = (phi - c + 0.5) % 1.0 - 0.5
    a = np.abs(D)
    if tau > 0:
        s = np.clip((T / 2 - a) / tau, 0.0, 1.0)
    else:
        s = (a < T / 2).astype(np.float64)
    A = np.stack([np.ones_like(s), s], axis=1) * np.sqrt(w)[:, None]
    b = x * np.sqrt(w)
    coef, *_ = np.linalg.lstsq(A, b, rcond=None)
    chi2 = float(np.sum((b - A @ coef) ** 2))
    return float(np.sum(w * x * x)) - chi2, -coef[1]


@pytest.mark.parametrize("seed", range(8))
def test_point_power_equals_least_squares(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(8, 60))
    phi = rng.random(n)
    dy = rng.uniform(0.5, 2.0, n)
    w = dy ** -2 / np.sum(dy ** -2)
    y = rng.normal(0, 1, n)
    x = y - np.sum(w * y)
    for c, T, tau in ((0.3, 0.2, 0.0), (0.95, 0.3, 0.05), (0.5, 0.1, 0.05), (0.02, 0.4, 0.2)):
        Q, d, ok = oracle.shape_point(phi, w, x, c, T, tau)
        Ql, dl = _lstsq_power(phi, w, x, c, T, tau)
        if ok:
            assert Q == pytest.approx(Ql, rel=1e-9, abs=1e-12)
            assert d == pytest.approx(dl, rel=1e-9, abs=1e-12)
        else:
            assert dl <= 1e-12 or Ql <= 1e-12    # a bump (or nothing) is not counted


def test_box_grid_point_is_the_bls_box():
    """With one grid point at the box's own centre and width and no ingress, the trapezoid
    holds the box's points and Q equals the BLS power of that box."""
    b = synth.config1()
    c, g = b.curves[0], b.grids[0]
    dt, w, x, _ = oracle.prep(c.t, c.y, c.dy)
    kmin, kmax = oracle.kminmax(100, b.qmin, b.qmax)
    for j in (0, 137, 1543):
        f = oracle.freq(j, g.fmin, g.df)
        P, i1, k, r, s = oracle.power(dt, w, x, f, 100, kmin, kmax)
        fit, _ = oracle.shape(dt, w, x, f, 100, i1, k, nc=1, nw=1, na=1, wlo=1.0, whi=1.0)
        assert fit.index == 0
        assert fit.power == pytest.approx(P, rel=1e-11)
        assert fit.depth == pytest.approx(-s / (r * (1 - r)), rel=1e-11)


def test_noise_free_trapezoid_is_recovered_exactly():
    """A noiseless trapezoid placed exactly on a grid point: that point fits with chi2 = 0,
    so it wins with Q = sum w x^2 and the injected depth."""
    rng = np.random.default_rng(9)
    n = 3000
    f, nb, i1, k = 1.0 / 0.7, 100, 31, 6
    dt = np.sort(rng.uniform(0, 40, n))
    phi = dt * f - np.floor(dt * f)
    q = k / nb
    pb = (i1 + k / 2) / nb
    m, u, v = 12, 5, 3                        # centre, width, ingress indices of the grid
    nc, nw, na, wlo, whi, amax = 17, 13, 6, 0.5, 2.0, 0.5
    cc = pb + q * (m / (nc - 1) - 0.5)
    T = q * (wlo + u / (nw - 1) * (whi - wlo))
    tau = T * (amax * v / (na - 1))
    D = (phi - cc + 0.5) % 1.0 - 0.5
    shape = np.clip((T / 2 - np.abs(D)) / tau, 0, 1)
    y = 1.0 - 0.05 * shape
    w = np.full(n, 1.0 / n)
    x = y - np.sum(w * y)
    fit, _ = oracle.shape(dt, w, x, f, nb, i1, k)
    assert fit.index == (m * nw + u) * na + v
    assert fit.depth == pytest.approx(0.05, rel=1e-9)
    assert fit.power == pytest.approx(float(np.sum(w * x * x)), rel=1e-9)
    assert fit.width == pytest.approx(T, rel=1e-12) and fit.ingress == pytest.approx(tau, rel=1e-12)


def test_bumps_do_not_count_and_grid_shape():
    rng = np.random.default_rng(4)
    n = 500
    dt = np.sort(rng.uniform(0, 10, n))
    f = 1.3
    phi = dt * f - np.floor(dt * f)
    y = 1.0 + 0.1 * ((phi > 0.4) & (phi < 0.5))        # a bump, no dip
    w = np.full(n, 1.0 / n)
    x = y - np.sum(w * y)
    fit, Q = oracle.shape(dt, w, x, f, 50, 21, 4, nc=5, nw=3, na=2, want_grid=True)
    assert Q.shape == (30,)
    assert fit.index == -1 or fit.power < 1e-4          # only noise-free flat parts remain
    with pytest.raises(ValueError):
        oracle.shape(dt, w, x, f, 50, 21, 4, amax=0.7)
