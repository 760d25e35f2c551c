"""Detection-efficiency harness (Sec. 5 of the paper, detection-efficiency figure).

Two measures per trial period, both on a survey cadence with its observing windows and
weather losses:

* the window efficiency: the fraction of eclipse phases at which at least two eclipses
  contain observations (``bls_window_efficiency``, the paper's definition);
* the recovery efficiency: the fraction of injected eclipsing curves (random epoch, given
  depth, duration and noise) on that cadence whose batched BLS search (``bls_search``)
  puts its best peak on the injected period or a low-order harmonic of it.

Everything on the GPU goes through the C ABI; this module only builds arguments, calls
the library and applies the recovery criterion to the returned peaks.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np

from . import bls

HARMONICS = (1.0, 2.0, 0.5)   # f_best / f_true ratios that count as a recovery


def recovered(f_best: np.ndarray, f_true: np.ndarray, df: float, steps: float = 2.0,
              harmonics: Sequence[float] = HARMONICS) -> np.ndarray:
    """True where the best frequency lies within `steps` grid steps of f_true times one
    of the harmonic ratios (the search cannot do better than its grid spacing)."""
    f_best = np.asarray(f_best, np.float64)
    f_true = np.asarray(f_true, np.float64)
    ok = np.zeros(f_best.shape, dtype=bool)
    for h in harmonics:
        ok |= np.abs(f_best - h * f_true) <= steps * df
    return ok


@dataclass
class EfficiencyCurve:
    periods: np.ndarray        # trial periods
    window: np.ndarray         # P(>= min_eclipses eclipses observed), per period
    recovery: np.ndarray       # fraction of injections recovered by the search, per period
    per_period: int            # injections per period
    best_freq: np.ndarray      # [n_periods, per_period] best frequency of every injection


def window_efficiency_at_periods(t: np.ndarray, periods: Sequence[float], duration: float,
                                 nphi: int = 256, min_eclipses: int = 2, min_points: int = 1,
                                 stream=None) -> np.ndarray:
    """Window efficiency at the given periods (explicit frequency grid 1/P)."""
    freqs = 1.0 / np.asarray(periods, np.float64)
    eff, _ = bls.window_efficiency(t, nphi, freqs=freqs, duration=duration,
                                   min_eclipses=min_eclipses, min_points=min_points,
                                   stream=stream)
    return eff


def injection_recovery(batch, plan: Optional[bls.Plan] = None, steps: float = 2.0,
                       **plan_kw) -> Tuple[np.ndarray, np.ndarray]:
    """Best frequency of every curve of an injection batch (synth.eclipse_injections) and
    whether it recovers the injected period: returns (best_freq[n], recovered[n])."""
    cis = bls.curves_from_batch(batch)
    own = plan is None
    if own:
        plan = bls.Plan(nb=batch.nb[0], qmin=batch.qmin, qmax=batch.qmax, **plan_kw)
    try:
        pk = plan.search(cis)
    finally:
        if own:
            plan.close()
    f_best = pk[:, 0]["freq"].astype(np.float64)
    f_true = np.array([1.0 / c.truth["period"] for c in batch.curves])
    df = batch.grids[0].df
    return f_best, recovered(f_best, f_true, df, steps)


def detection_efficiency(t: np.ndarray, periods: Sequence[float], per_period: int,
                         duration: float, depth: float, sigma: float, seed: int = 7,
                         nf: int = 20000, nphi: int = 256, plan: Optional[bls.Plan] = None,
                         **plan_kw) -> EfficiencyCurve:
    """Window and recovery efficiency per period on one cadence."""
    from . import synth
    periods = np.asarray(periods, np.float64)
    win = window_efficiency_at_periods(t, periods, duration, nphi=nphi)
    batch = synth.eclipse_injections(t, periods, per_period, duration, depth, sigma,
                                     seed=seed, nf=nf)
    f_best, ok = injection_recovery(batch, plan=plan, **plan_kw)
    shape = (len(periods), per_period)
    return EfficiencyCurve(periods, win, ok.reshape(shape).mean(axis=1), per_period,
                           f_best.reshape(shape))
