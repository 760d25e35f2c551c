"""Seeded synthetic light curves shaped like the PTF/M-dwarfs survey.

The survey's real light curves are not available, so every input in this project is
synthetic, with the cadence and noise the paper describes:

* nightly windows of a few hours, 15-25 min cadence, fields followed for 1-3 months,
  interleaved with a 1-3 day supernova cadence, so sampling is irregular
  (Sec. 2 and Table 1);
* photometric precision from a few mmag to 10% per point (Table 1, Fig. 2);
* eclipses of 5-20% depth with periods near 0.35-0.46 d for the systems found
  (Sec. 3, Table 3); injected boxes span wider ranges around those.

Times are emitted as HJD-like FP64 values (``T0 + days``) so that the caller's
subtraction of a reference time is exercised. Flux and errors are FP32.

This module holds no box-least-squares arithmetic (no folding, binning or box
statistics). It only draws sampling times, noise and injected box eclipses. The
same arrays are handed both to the CUDA path and to the FP64 oracle.

Seeding: curve ``c`` of configuration ``s`` draws from ``numpy.random.Generator(
PCG64(s * 10**6 + c))``, so any curve can be regenerated alone.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
from scipy.signal import lfilter

T0 = 2455000.0          # HJD-like origin of every synthetic time axis
WINDOW = (0.10, 0.35)   # nightly observing window inside each day [d] (6 h)


@dataclass
class Curve:
    t: np.ndarray               # FP64 times [d]
    y: np.ndarray               # FP32 flux (normalised to ~1)
    dy: np.ndarray              # FP32 1-sigma errors
    truth: Optional[dict] = None  # injected box (period, epoch, duration, depth) or None


@dataclass
class Grid:
    """A uniform trial-frequency grid f_j = fmin + j*df, j < nf [1/d]."""
    fmin: float
    df: float
    nf: int

    @staticmethod
    def span(fmin: float, fmax: float, nf: int) -> "Grid":
        return Grid(float(fmin), float((fmax - fmin) / (nf - 1)) if nf > 1 else 0.0, int(nf))


@dataclass
class Batch:
    """Curves plus the search settings they share (or carry per curve)."""
    curves: List[Curve]
    grids: List[Grid]
    nb: List[int]
    qmin: float
    qmax: float
    name: str = ""
    extra: dict = field(default_factory=dict)

    def __len__(self) -> int:
        return len(self.curves)

    def subset(self, idx: Sequence[int]) -> "Batch":
        idx = list(idx)
        return Batch([self.curves[i] for i in idx], [self.grids[i] for i in idx],
                     [self.nb[i] for i in idx], self.qmin, self.qmax,
                     self.name + "[subset]", dict(self.extra))

    def point_freqs(self) -> int:
        """Sum over curves of N_c * nf_c: the number of point x frequency evaluations."""
        return int(sum(len(c.t) * g.nf for c, g in zip(self.curves, self.grids)))


def curve_rng(seed: int, c: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed * 10**6 + c))


def nightly_times(rng: np.random.Generator, n: int, nights: np.ndarray,
                  window=WINDOW) -> np.ndarray:
    """n sorted times, uniform over the union of equal-length nightly windows."""
    if len(nights) == 0:
        raise ValueError("no observable nights")
    which = rng.integers(0, len(nights), size=n)
    off = rng.uniform(window[0], window[1], size=n)
    t = np.sort(nights[which].astype(np.float64) + off)
    return T0 + t


def red_white_noise(rng: np.random.Generator, t: np.ndarray, sigma: float,
                    rho: float = 0.9, red_frac: float = 0.5) -> np.ndarray:
    """White N(0, sigma) plus AR(1) noise (coefficient rho, marginal std red_frac*sigma)
    run in sample order and restarted at every night gap (> 0.5 d)."""
    n = len(t)
    white = rng.normal(0.0, sigma, size=n)
    s = red_frac * sigma
    z = rng.normal(0.0, 1.0, size=n)
    red = np.empty(n)
    starts = np.flatnonzero(np.diff(t, prepend=-np.inf) > 0.5)
    ends = np.append(starts[1:], n)
    for a, b in zip(starts, ends):
        u = s * np.sqrt(1.0 - rho * rho) * z[a:b]
        u[0] = s * z[a]  # stationary start of each night
        red[a:b] = lfilter([1.0], [1.0, -rho], u)
    return white + red


def inject_box(t: np.ndarray, y: np.ndarray, period: float, epoch: float,
               duration: float, depth: float) -> np.ndarray:
    """Subtract a box eclipse of the given depth: in eclipse while
    (t - T0 - epoch) mod period < duration."""
    ph = np.mod(t - T0 - epoch, period)
    out = y.copy()
    out[ph < duration] -= depth
    return out


def _loguniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=size))


def _survey_curve(rng: np.random.Generator, n: int, span_nights: int, p_weather: float,
                  inject: bool, depth_range, period_range, q_range, seasons=False,
                  depth_log=True) -> Curve:
    nights = np.arange(span_nights, dtype=np.float64)
    if seasons:  # observable 8 of every 12 months
        nights = nights[np.mod(nights, 365.25) < 365.25 * 8.0 / 12.0]
    keep = rng.random(len(nights)) >= p_weather
    if not keep.any():
        keep[rng.integers(0, len(nights))] = True
    t = nightly_times(rng, n, nights[keep])
    sigma = rng.uniform(0.005, 0.03)
    y = 1.0 + red_white_noise(rng, t, sigma)
    truth = None
    if inject:
        depth = (_loguniform(rng, *depth_range) if depth_log
                 else rng.uniform(*depth_range))
        period = _loguniform(rng, *period_range)
        q = _loguniform(rng, *q_range)
        epoch = rng.uniform(0.0, period)
        y = inject_box(t, y, period, epoch, q * period, depth)
        truth = dict(period=period, epoch=T0 + epoch, duration=q * period, depth=depth)
    return Curve(t, y.astype(np.float32), np.full(n, sigma, dtype=np.float32), truth)


# ----------------------------------------------------------------------------------
# Workloads. Settings not printed in the paper (bin counts, duration ranges, grids)
# follow the readings stated in the design notes.
# ----------------------------------------------------------------------------------

def config1(seed: int = 1) -> Batch:
    """Plain search, one curve: 500 times in 20 of 30 nights, y = 1 + N(0, 0.01),
    dy = 0.01, box depth 0.02, P = 0.40 d, duration 0.04 d, random epoch;
    2000 frequencies uniform in [0.2, 5] 1/d, nb = 100, q in [0.01, 0.10]."""
    rng = curve_rng(seed, 0)
    nights = np.sort(rng.choice(30, size=20, replace=False)).astype(np.float64)
    t = nightly_times(rng, 500, nights)
    y = 1.0 + rng.normal(0.0, 0.01, size=500)
    epoch = rng.uniform(0.0, 0.40)
    y = inject_box(t, y, 0.40, epoch, 0.04, 0.02)
    c = Curve(t, y.astype(np.float32), np.full(500, 0.01, dtype=np.float32),
              dict(period=0.40, epoch=T0 + epoch, duration=0.04, depth=0.02))
    return Batch([c], [Grid.span(0.2, 5.0, 2000)], [100], 0.01, 0.10, "cfg1-plain")


def config2(ncurves: int = 1024, seed: int = 2, nf: int = 50000, first: int = 0) -> Batch:
    """Batched search: N log-uniform in [500, 5000], nightly 6-h windows over 60 days
    with 30% of nights lost to weather; 70% noise-only (white sigma U[0.005, 0.03]
    plus AR(1) rho = 0.9), 30% with boxes of depth log-U[0.5%, 5%] and period
    log-U[0.3, 10] d; nf frequencies uniform in [0.1, 5] 1/d; nb = 200;
    q in [0.005, 0.15]."""
    curves = []
    for c in range(first, first + ncurves):
        rng = curve_rng(seed, c)
        n = int(round(_loguniform(rng, 500, 5000)))
        inject = rng.random() < 0.30
        curves.append(_survey_curve(rng, n, 60, 0.30, inject, (0.005, 0.05),
                                    (0.3, 10.0), (0.01, 0.08)))
    g = Grid.span(0.1, 5.0, nf)
    return Batch(curves, [g] * ncurves, [200] * ncurves, 0.005, 0.15, "cfg2-batched")


def config3(ncurves: int = 256, seed: int = 3, nf: int = 200000, n: int = 3000,
            first: int = 0) -> Batch:
    """Precision study: 3000 points over a 3-year baseline with seasonal gaps and
    nightly windows, boxes with period log-U[0.2, 20] d; nf frequencies uniform in
    [0.05, 5] 1/d; nb = 200; q in [0.005, 0.15]."""
    curves = []
    for c in range(first, first + ncurves):
        rng = curve_rng(seed, c)
        curves.append(_survey_curve(rng, n, 1095, 0.30, True, (0.005, 0.05),
                                    (0.2, 20.0), (0.01, 0.08), seasons=True))
    g = Grid.span(0.05, 5.0, nf)
    return Batch(curves, [g] * ncurves, [200] * ncurves, 0.005, 0.15, "cfg3-precision")


def config4_requests(nreq: int, seed: int = 4, first: int = 0,
                     n_range=(200, 20000), nf_range=(10000, 100000),
                     nb_range=(100, 400)) -> Batch:
    """Serving stream: each request one curve with N log-U[200, 20000], its own grid
    of U-int[10k, 100k] frequencies in [0.1, 5] 1/d and nb U-int[100, 400]; noise as
    in the batched workload over 60 nights; 30% carry boxes."""
    curves, grids, nbs = [], [], []
    for c in range(first, first + nreq):
        rng = curve_rng(seed, c)
        n = int(round(_loguniform(rng, *n_range)))
        nf = int(rng.integers(nf_range[0], nf_range[1] + 1))
        nb = int(rng.integers(nb_range[0], nb_range[1] + 1))
        inject = rng.random() < 0.30
        curves.append(_survey_curve(rng, n, 60, 0.30, inject, (0.005, 0.05),
                                    (0.3, 10.0), (0.01, 0.08)))
        grids.append(Grid.span(0.1, 5.0, nf))
        nbs.append(nb)
    return Batch(curves, grids, nbs, 0.005, 0.15, "cfg4-serving")


def poisson_arrivals(nreq: int, rate_hz: float, seed: int = 4) -> np.ndarray:
    """Arrival offsets [s] of a Poisson stream at the given offered rate."""
    rng = np.random.Generator(np.random.PCG64(seed * 10**6 + 999_999))
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=nreq))


def config5(ncurves: int = 100000, seed: int = 5, nf: int = 200000, first: int = 0) -> Batch:
    """Survey-scale sweep: 2000 points per curve over 90 nights, FP32 flux, 5% with
    boxes of depth U[1%, 3%] and period log-U[0.3, 10] d; nf frequencies in
    [0.1, 5] 1/d; nb = 256; q in [0.005, 0.15]; top-5 peaks per curve."""
    curves = []
    for c in range(first, first + ncurves):
        rng = curve_rng(seed, c)
        inject = rng.random() < 0.05
        curves.append(_survey_curve(rng, 2000, 90, 0.30, inject, (0.01, 0.03),
                                    (0.3, 10.0), (0.01, 0.08), depth_log=False))
    g = Grid.span(0.1, 5.0, nf)
    return Batch(curves, [g] * ncurves, [256] * ncurves, 0.005, 0.15, "cfg5-survey",
                 dict(topk=5))


# ----------------------------------------------------------------------------------
# Detection-efficiency workloads: survey cadences and injected eclipses.
# ----------------------------------------------------------------------------------

def survey_cadence(seed: int = 6, nights: int = 60, p_weather: float = 0.3,
                   cadence_min: float = 20.0, window=(0.10, 0.30), jitter_min: float = 1.0,
                   field: int = 0) -> np.ndarray:
    """Exposure times of one survey field: an exposure every cadence_min minutes through
    each night's window (about 5 h), each shifted by a uniform jitter of +-jitter_min
    minutes, on the nights the weather leaves (each lost with probability p_weather).
    Sorted, HJD-like."""
    rng = curve_rng(seed, field)
    step = cadence_min / 1440.0
    per_night = np.arange(window[0], window[1], step)
    keep = np.flatnonzero(rng.random(nights) >= p_weather)
    if len(keep) == 0:
        keep = np.array([0])
    t = (keep[:, None].astype(np.float64) + per_night[None, :]).ravel()
    t = t + rng.uniform(-jitter_min, jitter_min, size=t.size) / 1440.0
    return T0 + np.sort(t)


def eclipse_injections(t: np.ndarray, periods: Sequence[float], per_period: int,
                       duration: float, depth: float, sigma: float, seed: int = 7,
                       nf: int = 20000, fmin: float = 0.1, fmax: float = 5.0,
                       nb: int = 200) -> Batch:
    """Injection set for the recovery harness: for each period, per_period copies of the
    cadence t with white noise N(0, sigma) and a box eclipse of the given depth and
    duration at a random epoch (truth in Curve.truth, the epoch in [0, period))."""
    curves, grids = [], []
    g = Grid.span(fmin, fmax, nf)
    c = 0
    for P in periods:
        for _ in range(per_period):
            rng = curve_rng(seed, c)
            c += 1
            epoch = rng.uniform(0.0, P)
            y = 1.0 + rng.normal(0.0, sigma, size=len(t))
            y = inject_box(t, y, P, epoch, duration, depth)
            curves.append(Curve(t.copy(), y.astype(np.float32),
                                np.full(len(t), sigma, dtype=np.float32),
                                dict(period=P, epoch=T0 + epoch, duration=duration,
                                     depth=depth)))
            grids.append(g)
    return Batch(curves, grids, [nb] * len(curves), 0.005, 0.15, "injection-recovery")


# ----------------------------------------------------------------------------------
# High-variability pre-filter workload: chip catalogs of light curves in magnitudes.
# ----------------------------------------------------------------------------------

@dataclass
class Catalog:
    """Light curves of the stars of several chips, concatenated: star s has magnitudes
    m[off[s]:off[s+1]] and lies on chip[s]; variable[s] marks the injected variables."""
    off: np.ndarray
    m: np.ndarray
    chip: np.ndarray
    variable: np.ndarray
    nchips: int


def chip_catalog(seed: int = 12, nchips: int = 11, stars_per_chip: int = 3000,
                 npts: int = 600, var_frac: float = 0.01, mag_range=(14.0, 20.5)) -> Catalog:
    """Stars with magnitudes rising in number towards the faint end (log N ~ 0.3 m), a
    noise floor of 3 mmag plus photon noise growing with magnitude (about 1% at 18.5,
    ~10% at 20.5), npts epochs each; a fraction var_frac are eclipsing-binary-like
    variables with box dips of depth U[0.1, 0.4] mag over 10-20% of their epochs."""
    rng = np.random.Generator(np.random.PCG64(seed * 10**6))
    n = nchips * stars_per_chip
    lo, hi = mag_range
    a = 0.3 * np.log(10.0)
    u = rng.random(n)
    mag = lo + np.log1p(u * (np.exp(a * (hi - lo)) - 1.0)) / a
    sigma = np.sqrt(0.003 ** 2 + (0.01 * 10 ** (0.4 * (mag - 18.5))) ** 2)
    variable = rng.random(n) < var_frac
    m = mag[:, None] + sigma[:, None] * rng.normal(0.0, 1.0, (n, npts))
    for s in np.flatnonzero(variable):
        frac = rng.uniform(0.1, 0.2)
        dip = rng.random(npts) < frac
        m[s, dip] += rng.uniform(0.1, 0.4)
    off = np.arange(n + 1, dtype=np.int64) * npts
    chip = np.repeat(np.arange(nchips, dtype=np.int32), stars_per_chip)
    return Catalog(off, m.astype(np.float32).ravel(), chip, variable, nchips)
