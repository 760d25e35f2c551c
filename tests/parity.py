"""Shared helpers of the GPU parity tests: oracle runs and the stated tolerance.

Tolerance (per frequency, on SR = sqrt(P)):

    |SR_gpu - SR_oracle| <= 1e-5 * SR_oracle + 1e-6 * sqrt(sum w x^2)

The relative term is the 1e-5 bar on SR; the absolute floor covers frequencies where SR is
pure noise: the histograms and box sums are FP32, so a box sum s carries an absolute
rounding error of a few FP32 ulps of sum|w x| over the box, which is below
1e-6 * sqrt(sum w x^2) for the box widths and curve lengths used here.
"""
import numpy as np

import oracle
from paper_1112_1701_b300 import bls

REL, ABS = 1e-5, 1e-6


def sr_tol(sr_oracle, sumwx2):
    return REL * np.asarray(sr_oracle) + ABS * np.sqrt(sumwx2)


def host(a, dtype=None):
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.asarray(a, dtype=dtype) if dtype else np.asarray(a)


def grid_of(ci: bls.CurveInput):
    if ci.freqs is not None:
        return host(ci.freqs, np.float64)
    return np.array([oracle.freq(j, ci.fmin, ci.df) for j in range(ci.nf)])


def oracle_run(ci: bls.CurveInput, nb, kmin, kmax, sign=0, topk=1):
    t, y = host(ci.t, np.float64), host(ci.y, np.float32)
    dy = None if ci.dy is None else host(ci.dy, np.float32)
    if ci.freqs is not None:
        return oracle.bls(t, y, dy, nb, kmin, kmax, freqs=host(ci.freqs, np.float64),
                          sign=sign, topk=topk)
    return oracle.bls(t, y, dy, nb, kmin, kmax, fmin=ci.fmin, df=ci.df, nf=ci.nf, sign=sign,
                      topk=topk)


def prep_of(ci: bls.CurveInput):
    dy = None if ci.dy is None else host(ci.dy, np.float32)
    return oracle.prep(host(ci.t, np.float64), host(ci.y, np.float32), dy)


def check_powers(ci, Pg, I1g, Kg, nb, kmin, kmax, sign=0, Po=None, I1o=None, Ko=None,
                 label=""):
    """Per-frequency parity: SR within tolerance everywhere; where the chosen box differs,
    the oracle's power of the GPU's box must itself be within tolerance of the maximum."""
    if Po is None:
        Po, I1o, Ko, _ = oracle_run(ci, nb, kmin, kmax, sign)
    dt, w, x, scal = prep_of(ci)
    sro, srg = np.sqrt(Po), np.sqrt(np.asarray(Pg, np.float64))
    tol = sr_tol(sro, scal[3])
    err = np.abs(srg - sro)
    worst = int(np.argmax(err - tol))
    assert np.all(err <= tol), (
        f"{label}: SR mismatch at j={worst}: gpu {srg[worst]:.9g} oracle {sro[worst]:.9g} "
        f"tol {tol[worst]:.3g}; {int(np.sum(err > tol))} of {len(err)} over")
    fr = grid_of(ci)
    diff = np.flatnonzero((I1g != I1o) | (Kg != Ko))
    for j in diff[:200]:
        Pb, _, _ = oracle.box(dt, w, x, fr[j], nb, int(I1g[j]), int(Kg[j]), sign)
        assert abs(np.sqrt(Pb) - sro[j]) <= tol[j], (
            f"{label}: j={j} gpu box ({I1g[j]},{Kg[j]}) has oracle SR {np.sqrt(Pb):.9g}, "
            f"max {sro[j]:.9g} at ({I1o[j]},{Ko[j]})")
    return Po, I1o, Ko, scal


def separated_best(P, sumwx2):
    """(j*, separated): the oracle's best index and whether the best two local maxima of
    SR differ by more than twice the tolerance (each may be off by one tolerance)."""
    sr = np.sqrt(P)
    j = int(np.argmax(sr))
    nf = len(sr)
    lm = [i for i in range(nf) if (i == 0 or sr[i] > sr[i - 1]) and
          (i == nf - 1 or sr[i] >= sr[i + 1])]
    vals = sorted((sr[i] for i in lm), reverse=True)
    sep = len(vals) < 2 or (vals[0] - vals[1]) > 2 * sr_tol(vals[0], sumwx2)
    return j, sep


def check_sde(pg, po, P_oracle, sumwx2):
    """SDE = (SR_peak - mean SR) / sd SR: the GPU's spectrum may differ from the oracle's
    by T = max_j tol(SR_j) at every frequency, which moves the mean and the standard
    deviation by at most T each; the peak SR itself is an FP64 refit (equal to 1e-9).
    So |dSDE| <= (T + |SDE| T) / sd, doubled for the second-order terms."""
    sr = np.sqrt(np.asarray(P_oracle, np.float64))
    T = float(np.max(sr_tol(sr, sumwx2)))
    sd = float(sr.std())
    if sd == 0.0:
        assert pg["sde"] == 0.0
        return
    bound = 2.0 * (1.0 + abs(po.sde)) * T / sd + 1e-9 * abs(po.sde)
    assert abs(pg["sde"] - po.sde) <= bound, (pg["sde"], po.sde, bound)


def check_peak(pg, po, rel=1e-9):
    """A GPU peak record against the oracle's for the same (j, i1, k)."""
    assert pg["j"] == po.j and pg["i1"] == po.i1 and pg["k"] == po.k, (pg, po)
    for f in ("freq", "period", "duration"):
        assert abs(pg[f] - getattr(po, f)) <= 1e-13 * abs(getattr(po, f)), f
    assert abs(pg["epoch"] - po.epoch) <= 1e-9
    for f in ("depth", "sr", "snr", "power"):
        a, b = pg[f], getattr(po, f)
        assert abs(a - b) <= rel * abs(b) + 1e-15, (f, a, b)
