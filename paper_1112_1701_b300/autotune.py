"""Autotuner of the tiled search's launch parameters, driving the C ABI.

The tiled search has three launch parameters that change its speed and not its bins or
boxes: the frequencies per block (tile width T: one histogram column per frequency, so T x
nb x 8 B of shared memory), the points staged per chunk, and the fold-sweep kernel
(warp-specialised or one-group, ``BLS_FOLD_*`` in ``include/bls.h``).  The library's
defaults come from fixed rules (the widest tile that fits, 512-point chunks, the
warp-specialised kernel where its TMEM copy fits); this module measures instead.

For a batch of curves that share nb and the duration range it:
  * draws a sample of the curves spread over their length distribution (curve lengths set
    the balance between binning and sweeping) and truncates their grids so that the sample
    still spreads several tiles over every SM;
  * times the fold-sweep kernel (CUDA events, ``bls_profile_get``) for every feasible
    candidate, repeating each and keeping the median;
  * returns the fastest, and caches it per (device, nb, kmin, kmax, phase mode, sums, sign,
    curve-length class) in memory and, when a path is given, in a JSON file.

A second stage tunes the curves per launch: with the best of the above, the sample is
searched in one, two and four launches (max_curves_per_launch), and the fastest split
(ties to fewer launches) is applied to the whole batch.  Mixed-nb workloads (serving) keep
the per-class rules, since a plan's tile width applies to all its curves.
"""
from __future__ import annotations

import dataclasses
import json
import math
import os
import threading
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

from . import bls

CHUNKS = (512, 256)
MAX_T = 256          # fold_sweep_max_threads()
SPLITS = (2, 4)      # launches per batch tried by the second stage (besides one)


@dataclass(frozen=True)
class Candidate:
    freqs_per_block: int   # 0 = the library's rule
    point_chunk: int       # 0 = the library's rule
    fold_kernel: str       # key of bls.FOLD
    curves_per_launch: int = 0   # 0 = every curve of a class in one launch

    def plan_kwargs(self) -> dict:
        return dict(freqs_per_block=self.freqs_per_block, point_chunk=self.point_chunk,
                    fold_kernel=self.fold_kernel, max_curves_per_launch=self.curves_per_launch)


DEFAULT = Candidate(0, 0, "auto")


@dataclass
class TuneResult:
    best: Candidate
    best_ms: float                  # fold-sweep ms per sample search
    default_ms: float               # the library's rules on the same sample
    table: List[tuple] = field(default_factory=list)   # (Candidate, ms or None if infeasible)
    key: str = ""
    sample: str = ""
    cached: bool = False
    splits: int = 1                 # launches the batch is split into

    def to_json(self) -> dict:
        return {"freqs_per_block": self.best.freqs_per_block,
                "point_chunk": self.best.point_chunk, "fold_kernel": self.best.fold_kernel,
                "launch_splits": self.splits,
                "curves_per_launch": self.best.curves_per_launch,
                "best_ms": self.best_ms, "default_ms": self.default_ms, "key": self.key,
                "sample": self.sample, "candidates": len(self.table)}


def candidates(nb: int, kmin: int, kmax: int, sums: str = "fixed",
               smem_optin: int = 231424, reserve: int = 2048) -> List[Candidate]:
    """Feasible candidates for one nb: for each chunk size, the tile widths (multiples of 16)
    from the widest that fits shared memory down to half of it (at least 32), in both kernels
    where the warp-specialised one can take the width (a multiple of 8, at most 128); then
    the widest warp-specialised width that is not a multiple of 16 (its histograms packed at
    that stride) with the largest chunk of 256..512 points that fits it; plus the library's
    own choice.  smem_optin is the dynamic shared memory a block may use (the device's
    opt-in limit less the kernels' static shared memory)."""
    esz = 16 if sums == "kahan" else 8

    def fits(T, stride, chunk):
        return 2 * chunk * 24 + nb * stride * esz + reserve <= smem_optin

    out = [DEFAULT]
    for chunk in CHUNKS:
        tmax = min((smem_optin - 2 * chunk * 24 - reserve) // (nb * esz), MAX_T) & ~15
        if tmax < 16:
            continue
        lo = max(16, (tmax // 2) & ~15)
        widths = sorted(set(list(range(lo, tmax + 1, 16)) + [w for w in (32, 64, 96, 128) if w <= tmax]),
                        reverse=True)
        for T in widths:
            out.append(Candidate(T, chunk, "one_group"))
            if T % 8 == 0 and T <= 128:
                out.append(Candidate(T, chunk, "ws"))
    for T in range(120, 7, -16):   # 120, 104, ..., 8
        ch = next((c for c in range(max(CHUNKS), min(CHUNKS) - 1, -16) if fits(T, T, c)), None)
        if ch is not None:
            out.append(Candidate(T, ch, "ws"))
            break
    return out


def length_class(curves: Sequence[bls.CurveInput]) -> int:
    """log2 of the median curve length, rounded: the cache's curve-length class."""
    n = np.median([len(c.t) for c in curves]) if len(curves) else 2
    return int(round(math.log2(max(2.0, float(n)))))


def sample_curves(curves: Sequence[bls.CurveInput], count: int, tiles_needed: int,
                  widest: int) -> List[bls.CurveInput]:
    """`count` curves at evenly spaced quantiles of length, grids truncated (uniform grids to
    their first nf frequencies, explicit grids to their first entries) so that the sample
    holds about `tiles_needed` tiles of `widest` frequencies."""
    order = sorted(range(len(curves)), key=lambda i: len(curves[i].t))
    count = max(1, min(count, len(order)))
    idx = [order[int(round(q * (len(order) - 1)))] for q in np.linspace(0.0, 1.0, count)]
    nf_keep = max(widest, int(math.ceil(tiles_needed * widest / count)))
    out = []
    for i in idx:
        c = curves[i]
        if c.freqs is not None:
            fr = c.freqs[:nf_keep]
            out.append(bls.CurveInput(c.t, c.y, c.dy, freqs=fr, nb=c.nb, qmin=c.qmin, qmax=c.qmax))
        else:
            out.append(bls.CurveInput(c.t, c.y, c.dy, nf=min(c.nf, nf_keep), fmin=c.fmin,
                                      df=c.df, nb=c.nb, qmin=c.qmin, qmax=c.qmax))
    return out


class TuneCache:
    """Tuned parameters per key, in memory and optionally in a JSON file."""

    def __init__(self, path: Optional[str] = None):
        self.path = path
        self._lock = threading.Lock()
        self._d: Dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self._d = json.load(f)

    def get(self, key: str) -> Optional[tuple]:
        """(Candidate without the batch's curves per launch, launch splits) or None."""
        with self._lock:
            v = self._d.get(key)
        if v is None:
            return None
        return (Candidate(int(v["freqs_per_block"]), int(v["point_chunk"]), str(v["fold_kernel"])),
                int(v.get("launch_splits", 1)))

    def put(self, key: str, res: TuneResult):
        with self._lock:
            self._d[key] = res.to_json()
            if self.path:
                tmp = self.path + f".tmp{os.getpid()}"
                with open(tmp, "w") as f:
                    json.dump(self._d, f, indent=1, sort_keys=True)
                os.replace(tmp, self.path)


_CACHE = TuneCache(os.environ.get("BLS_TUNE_CACHE") or None)


def cache_key(device: str, sms: int, nb: int, kmin: int, kmax: int, phase: str, sums: str,
              sign: str, lclass: int) -> str:
    return f"{device}|sm{sms}|nb{nb}|k{kmin}-{kmax}|{phase}|{sums}|{sign}|n2^{lclass}"


def time_candidate(cand: Candidate, sample: Sequence[bls.CurveInput], nb: int, qmin: float,
                   qmax: float, phase: str, sums: str, sign: str, reps: int,
                   stream=None) -> Optional[float]:
    """Median fold-sweep ms of `reps` searches of the sample (after one warm-up), or None when
    the candidate does not fit the device."""
    try:
        with bls.Plan(nb=nb, qmin=qmin, qmax=qmax, phase=phase, sum=sums, sign=sign,
                      stream=stream, **cand.plan_kwargs()) as p:
            p.search(sample)
            ms = []
            for _ in range(reps):
                p.profile(reset=True)
                p.search(sample)
                pr = p.profile()
                ms.append(pr["fold_ms"])
    except bls.BLSError as e:
        if "shared memory" in str(e):
            return None
        raise
    return float(np.median(ms))


def tune(curves: Sequence[bls.CurveInput], nb: int, qmin: float, qmax: float, *,
         phase: str = "fx64", sums: str = "fixed", sign: str = "dips", sample: int = 32,
         tiles_per_sm: int = 16, reps: int = 3, cache: Optional[TuneCache] = None,
         use_cache: bool = True, stream=None,
         timer: Optional[Callable[..., Optional[float]]] = None,
         device: Optional[tuple] = None) -> TuneResult:
    """Fastest candidate for this batch (see the module docstring).  `timer` replaces the
    GPU timing (same signature as time_candidate) and `device` = (name, SM count) replaces
    the device query: both for tests without a GPU."""
    cache = _CACHE if cache is None else cache
    if device is None:
        import torch
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        device = (props.name, props.multi_processor_count)
    name, sms = device
    kmin, kmax = bls.kminmax(nb, qmin, qmax)
    key = cache_key(name, sms, nb, kmin, kmax, phase, sums, sign, length_class(curves))
    def for_batch(c: Candidate, splits: int) -> Candidate:
        return dataclasses.replace(
            c, curves_per_launch=0 if splits == 1 else int(math.ceil(len(curves) / splits)))

    if use_cache:
        hit = cache.get(key)
        if hit is not None:
            c, splits = hit
            return TuneResult(for_batch(c, splits), float("nan"), float("nan"), [], key, "cache",
                              True, splits)
    cands = candidates(nb, kmin, kmax, sums)
    widest = max(c.freqs_per_block for c in cands if c.freqs_per_block) if len(cands) > 1 else 128
    smp = sample_curves(curves, sample, tiles_per_sm * sms, widest)
    timer = timer or time_candidate
    table = []
    for c in cands:
        table.append((c, timer(c, smp, nb, qmin, qmax, phase, sums, sign, reps, stream=stream)))
    ok = [(c, ms) for c, ms in table if ms is not None]
    if not ok:
        raise RuntimeError("no feasible launch configuration for nb = %d" % nb)
    best, best_ms = min(ok, key=lambda x: (x[1], x[0] != DEFAULT))
    default_ms = dict(table).get(DEFAULT) or float("nan")
    # second stage: the sample in 1, 2 or 4 launches
    splits = 1
    for sp in SPLITS:
        if len(smp) < sp:
            break
        c2 = dataclasses.replace(best, curves_per_launch=int(math.ceil(len(smp) / sp)))
        ms = timer(c2, smp, nb, qmin, qmax, phase, sums, sign, reps, stream=stream)
        table.append((c2, ms))
        if ms is not None and ms < best_ms:
            best_ms, splits = ms, sp
    nfs = [len(c.freqs) if c.freqs is not None else c.nf for c in smp]
    res = TuneResult(for_batch(best, splits), best_ms, default_ms, table, key,
                     f"{len(smp)} curves (length quantiles), {min(nfs)}-{max(nfs)} frequencies "
                     f"each, {reps} timed searches per candidate", False, splits)
    cache.put(key, res)
    return res


def tuned_plan(curves: Sequence[bls.CurveInput], nb: int, qmin: float, qmax: float,
               **plan_kwargs) -> tuple:
    """A Plan with the tuned launch parameters for this batch, and the TuneResult."""
    tkw = {k: plan_kwargs[k] for k in ("phase", "sign") if k in plan_kwargs}
    if "sum" in plan_kwargs:
        tkw["sums"] = plan_kwargs["sum"]
    res = tune(curves, nb, qmin, qmax, stream=plan_kwargs.get("stream"), **tkw)
    kw = dict(plan_kwargs)
    kw.update(res.best.plan_kwargs())
    return bls.Plan(nb=nb, qmin=qmin, qmax=qmax, **kw), res
