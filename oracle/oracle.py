"""ctypes binding of ``bls_oracle.c``, ``window_oracle.c``, ``shape_oracle.c``,
``variability_oracle.c`` and ``unbinned_oracle.c``, the plain FP64 oracles (test
infrastructure).

Every function mirrors one C function; see that file for the definition each one
follows (Sec. 2.2.2 of the paper and the BLS method it cites).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bls_oracle.c")
_SRCS = [_SRC] + [os.path.join(_HERE, f) for f in ("window_oracle.c", "shape_oracle.c",
                                                  "variability_oracle.c", "unbinned_oracle.c")]
_LIB = os.path.join(_HERE, "libbls_oracle.so")
_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: -O2, no FMA contraction, no fast-math."""
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(s)
                                                  for s in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-Wall", "-o", tmp, *_SRCS, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Peak(C.Structure):
    _fields_ = [("j", C.c_int), ("freq", C.c_double), ("period", C.c_double),
                ("epoch", C.c_double), ("duration", C.c_double), ("depth", C.c_double),
                ("snr", C.c_double), ("sr", C.c_double), ("power", C.c_double),
                ("i1", C.c_int), ("k", C.c_int), ("sde", C.c_double)]


class _Shape(C.Structure):
    _fields_ = [("index", C.c_int), ("power", C.c_double), ("centre", C.c_double),
                ("width", C.c_double), ("ingress", C.c_double), ("depth", C.c_double)]


class _UPeak(C.Structure):
    _fields_ = [("j", C.c_int), ("first", C.c_int), ("len", C.c_int), ("first_point", C.c_int),
                ("freq", C.c_double), ("power", C.c_double), ("sr", C.c_double),
                ("depth", C.c_double), ("epoch", C.c_double), ("duration", C.c_double),
                ("snr", C.c_double)]


class _Curve(C.Structure):
    _fields_ = [("t", C.c_void_p), ("y", C.c_void_p), ("dy", C.c_void_p), ("n", C.c_int),
                ("freqs", C.c_void_p), ("nf", C.c_int), ("fmin", C.c_double),
                ("df", C.c_double), ("nb", C.c_int), ("kmin", C.c_int), ("kmax", C.c_int)]


@dataclass
class OraclePeak:
    j: int
    freq: float
    period: float
    epoch: float
    duration: float
    depth: float
    snr: float
    sr: float
    power: float
    i1: int
    k: int
    sde: float


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            D, I, P = C.c_double, C.c_int, C.c_void_p
            lib.oracle_kminmax.argtypes = [I, D, D, C.POINTER(I), C.POINTER(I)]
            lib.oracle_freq.argtypes = [I, D, D]
            lib.oracle_freq.restype = D
            lib.oracle_fold.argtypes = [D, D, I]
            lib.oracle_prep.argtypes = [I, P, P, P, P, P, P, P]
            lib.oracle_bins.argtypes = [I, P, I, P, I, P]
            lib.oracle_power.argtypes = [I, P, P, P, D, I, I, I, I, C.POINTER(D),
                                         C.POINTER(I), C.POINTER(I), C.POINTER(D),
                                         C.POINTER(D)]
            lib.oracle_box.argtypes = [I, P, P, P, D, I, I, I, I, C.POINTER(D), C.POINTER(D),
                                       C.POINTER(D)]
            lib.oracle_bls.argtypes = [C.POINTER(_Curve), I, P, P, P, I, P]
            lib.oracle_bls_many.argtypes = [I, C.POINTER(_Curve), I, I, P, I, P]
            lib.oracle_window_count.argtypes = [I, P, D, D, D, I]
            lib.oracle_window.argtypes = [I, P, I, P, D, D, I, D, D, I, I, P, P]
            lib.oracle_shape_point.argtypes = [I, P, P, P, D, D, D, C.POINTER(D), C.POINTER(I)]
            lib.oracle_shape_point.restype = D
            lib.oracle_shape.argtypes = [I, P, P, P, D, I, I, I, I, I, I, D, D, D,
                                         C.POINTER(_Shape), P]
            lib.oracle_star_stats.argtypes = [I, P, C.POINTER(D), C.POINTER(D)]
            lib.oracle_clip.argtypes = [I, P, D, I, C.POINTER(D), C.POINTER(D), P]
            lib.oracle_variability.argtypes = [I, P, P, P, I, D, I, D, I, P, P, P, P, P, P, P]
            lib.oracle_ubls_phases.argtypes = [I, P, D, P]
            lib.oracle_ubls_order.argtypes = [I, P, P]
            lib.oracle_ubls_extent.argtypes = [I, P, P, I, I]
            lib.oracle_ubls_extent.restype = D
            lib.oracle_ubls_power.argtypes = [I, P, P, P, D, D, D, I, C.POINTER(I), C.POINTER(I),
                                              C.POINTER(D), C.POINTER(D), P]
            lib.oracle_ubls_power.restype = D
            lib.oracle_ubls.argtypes = [I, P, P, P, I, P, D, D, D, D, I, P, C.POINTER(_UPeak)]
            _lib = lib
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def kminmax(nb: int, qmin: float, qmax: float):
    lo, hi = C.c_int(), C.c_int()
    if _load().oracle_kminmax(nb, qmin, qmax, C.byref(lo), C.byref(hi)) != 0:
        raise ValueError("invalid nb/q range")
    return lo.value, hi.value


def freq(j: int, fmin: float, df: float) -> float:
    return _load().oracle_freq(int(j), float(fmin), float(df))


def fold(dt: float, f: float, nb: int) -> int:
    return _load().oracle_fold(float(dt), float(f), int(nb))


def _arrays(t, y, dy):
    t = np.ascontiguousarray(t, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float32)
    dy = None if dy is None else np.ascontiguousarray(dy, dtype=np.float32)
    return t, y, dy


def prep(t, y, dy):
    """Returns dt, w, x (FP64) and (t_ref, W, ybar, sum w x^2)."""
    t, y, dy = _arrays(t, y, dy)
    n = len(t)
    dt, w, x = np.empty(n), np.empty(n), np.empty(n)
    scal = np.empty(4)
    if _load().oracle_prep(n, _p(t), _p(y), _p(dy), _p(dt), _p(w), _p(x), _p(scal)) != 0:
        raise ValueError("invalid curve")
    return dt, w, x, tuple(scal)


def bins(t, freqs: Sequence[float], nb: int) -> np.ndarray:
    """Per-point phase bins, shape (len(freqs), n)."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    out = np.empty((len(f), len(t)), dtype=np.int32)
    if _load().oracle_bins(len(t), _p(t), len(f), _p(f), nb, _p(out)) != 0:
        raise ValueError("invalid input")
    return out


def power(dt, w, x, f: float, nb: int, kmin: int, kmax: int, sign: int = 0):
    """Best box at one frequency: (P, i1, k, r, s)."""
    dt = np.ascontiguousarray(dt, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    P, r, s = C.c_double(), C.c_double(), C.c_double()
    i1, k = C.c_int(), C.c_int()
    rc = _load().oracle_power(len(dt), _p(dt), _p(w), _p(x), float(f), nb, kmin, kmax, sign,
                              C.byref(P), C.byref(i1), C.byref(k), C.byref(r), C.byref(s))
    if rc != 0:
        raise ValueError("invalid input")
    return P.value, i1.value, k.value, r.value, s.value


def box(dt, w, x, f: float, nb: int, i1: int, k: int, sign: int = 0):
    """Power of the given box at one frequency: (P, r, s)."""
    dt = np.ascontiguousarray(dt, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    P, r, s = C.c_double(), C.c_double(), C.c_double()
    if _load().oracle_box(len(dt), _p(dt), _p(w), _p(x), float(f), nb, int(i1), int(k), sign,
                          C.byref(P), C.byref(r), C.byref(s)) != 0:
        raise ValueError("invalid input")
    return P.value, r.value, s.value


def _curve_struct(t, y, dy, nb, kmin, kmax, freqs=None, fmin=0.0, df=0.0, nf=None):
    keep = [t, y, dy, freqs]
    cs = _Curve(_p(t), _p(y), _p(dy), len(t), _p(freqs),
                int(len(freqs) if freqs is not None else nf), float(fmin), float(df),
                int(nb), int(kmin), int(kmax))
    return cs, keep


def _peaks(arr) -> List[OraclePeak]:
    return [OraclePeak(p.j, p.freq, p.period, p.epoch, p.duration, p.depth, p.snr, p.sr,
                       p.power, p.i1, p.k, p.sde) for p in arr]


def bls(t, y, dy, nb: int, kmin: int, kmax: int, *, freqs=None, fmin=0.0, df=0.0,
        nf: Optional[int] = None, sign: int = 0, topk: int = 1):
    """Full periodogram of one curve: (P[nf], i1[nf], k[nf], peaks[topk])."""
    t, y, dy = _arrays(t, y, dy)
    if freqs is not None:
        freqs = np.ascontiguousarray(freqs, dtype=np.float64)
        nf = len(freqs)
    cs, keep = _curve_struct(t, y, dy, nb, kmin, kmax, freqs, fmin, df, nf)
    P = np.empty(nf)
    i1 = np.empty(nf, dtype=np.int32)
    k = np.empty(nf, dtype=np.int32)
    pk = (_Peak * max(topk, 1))()
    rc = _load().oracle_bls(C.byref(cs), sign, _p(P), _p(i1), _p(k), topk, pk)
    if rc != 0:
        raise ValueError(f"oracle_bls failed ({rc})")
    del keep
    return P, i1, k, _peaks(pk[:topk])


def bls_many(curves, nthreads: int = 1, sign: int = 0, topk: int = 1,
             want_power: bool = False):
    """Periodograms of many curves on POSIX threads.

    ``curves`` is a sequence of dicts with keys t, y, dy, nb, kmin, kmax and either
    freqs or (fmin, df, nf).  Returns (peaks per curve, concatenated powers or None).
    """
    structs = (_Curve * len(curves))()
    keep = []
    total_nf = 0
    for i, c in enumerate(curves):
        t, y, dy = _arrays(c["t"], c["y"], c.get("dy"))
        fr = c.get("freqs")
        if fr is not None:
            fr = np.ascontiguousarray(fr, dtype=np.float64)
        cs, kp = _curve_struct(t, y, dy, c["nb"], c["kmin"], c["kmax"], fr,
                               c.get("fmin", 0.0), c.get("df", 0.0), c.get("nf"))
        structs[i] = cs
        keep.append(kp)
        total_nf += cs.nf
    P = np.empty(total_nf) if want_power else None
    pk = (_Peak * (len(curves) * max(topk, 1)))()
    rc = _load().oracle_bls_many(len(curves), structs, sign, nthreads, _p(P), topk, pk)
    if rc != 0:
        raise ValueError(f"oracle_bls_many failed ({rc})")
    del keep
    out = _peaks(pk)
    return [out[i * topk:(i + 1) * topk] for i in range(len(curves))], P


def window(t, nphi: int, *, freqs=None, fmin=0.0, df=0.0, nf: Optional[int] = None,
           duration: float = 0.0, qfrac: float = 0.0, min_eclipses: int = 2,
           min_points: int = 1, want_counts: bool = False):
    """Eclipse-window detection efficiency per frequency (``oracle_window``):
    (eff[nf], counts[nf, nphi] or None)."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    if freqs is not None:
        freqs = np.ascontiguousarray(freqs, dtype=np.float64)
        nf = len(freqs)
    eff = np.empty(nf)
    counts = np.empty((nf, nphi), dtype=np.int32) if want_counts else None
    rc = _load().oracle_window(len(t), _p(t), nf, _p(freqs), fmin, df, nphi, duration, qfrac,
                               min_eclipses, min_points, _p(eff), _p(counts))
    if rc != 0:
        raise ValueError("oracle_window: bad arguments")
    return eff, counts


def window_count(t, f: float, phi: float, h: float, min_points: int = 1) -> int:
    """Observed eclipses of one (frequency, phase) pair (``oracle_window_count``)."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    return _load().oracle_window_count(len(t), _p(t), f, phi, h, min_points)


@dataclass
class OracleShape:
    index: int
    power: float
    centre: float
    width: float
    ingress: float
    depth: float


def shape(dt, w, x, f: float, nb: int, i1: int, k: int, nc: int = 17, nw: int = 13,
          na: int = 6, wlo: float = 0.5, whi: float = 2.0, amax: float = 0.5,
          want_grid: bool = False):
    """Trapezoid refit of one peak (``oracle_shape``): (OracleShape, Q[grid] or None)."""
    dt, w, x = (np.ascontiguousarray(a, dtype=np.float64) for a in (dt, w, x))
    out = _Shape()
    Q = np.zeros(nc * nw * na) if want_grid else None
    rc = _load().oracle_shape(len(dt), _p(dt), _p(w), _p(x), f, nb, i1, k, nc, nw, na, wlo, whi,
                              amax, C.byref(out), _p(Q))
    if rc != 0:
        raise ValueError(f"oracle_shape failed ({rc})")
    return OracleShape(out.index, out.power, out.centre, out.width, out.ingress, out.depth), Q


def shape_point(phi, w, x, c: float, T: float, tau: float):
    """Q and depth of one trapezoid on folded phases (``oracle_shape_point``)."""
    phi, w, x = (np.ascontiguousarray(a, dtype=np.float64) for a in (phi, w, x))
    d = C.c_double()
    ok = C.c_int()
    Q = _load().oracle_shape_point(len(phi), _p(phi), _p(w), _p(x), c, T, tau, C.byref(d),
                                   C.byref(ok))
    return Q, d.value, bool(ok.value)


def star_stats(m):
    """Mean magnitude and population RMS of one light curve (``oracle_star_stats``)."""
    m = np.ascontiguousarray(m, dtype=np.float32)
    mag, rms = C.c_double(), C.c_double()
    _load().oracle_star_stats(len(m), _p(m), C.byref(mag), C.byref(rms))
    return mag.value, rms.value


def clip(vals, clip: float = 3.0, iters: int = 5, with_margin: bool = False):
    """Sigma-clipped (mu, sd, kept) of a set of values (``oracle_clip``); with_margin adds
    the smallest distance of any keep-or-drop decision from its threshold."""
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    mu, sd, mg = C.c_double(), C.c_double(), C.c_double()
    kept = _load().oracle_clip(len(vals), _p(vals), clip, iters, C.byref(mu), C.byref(sd),
                               C.addressof(mg))
    if with_margin:
        return mu.value, sd.value, kept, mg.value
    return mu.value, sd.value, kept


def variability(off, m, chip, nchips: int, clip: float = 3.0, iters: int = 5,
                nsig: float = 2.0, min_stars: int = 5):
    """High-variability flags (``oracle_variability``): dict of per-star arrays mag, rms,
    bin, mu, sd, flag, and margin (the clip margin of the star's (chip, bin) group: the
    smallest distance of any clipping decision from its threshold)."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    m = np.ascontiguousarray(m, dtype=np.float32)
    chip = np.ascontiguousarray(chip, dtype=np.int32)
    n = len(chip)
    out = dict(mag=np.zeros(n), rms=np.zeros(n), bin=np.zeros(n, np.int32), mu=np.zeros(n),
               sd=np.zeros(n), flag=np.zeros(n, np.uint8), margin=np.zeros(n))
    rc = _load().oracle_variability(n, _p(off), _p(m), _p(chip), nchips, clip, iters, nsig,
                                    min_stars, _p(out["mag"]), _p(out["rms"]), _p(out["bin"]),
                                    _p(out["mu"]), _p(out["sd"]), _p(out["flag"]),
                                    _p(out["margin"]))
    if rc != 0:
        raise ValueError("oracle_variability: bad arguments")
    return out


@dataclass
class UnbinnedPeak:
    j: int
    first: int
    len: int
    first_point: int
    freq: float
    power: float
    sr: float
    depth: float
    epoch: float
    duration: float
    snr: float


def ubls_phases(dt, f: float) -> np.ndarray:
    """FP64 phases frac(RN(dt f)) of every point (``oracle_ubls_phases``)."""
    dt = np.ascontiguousarray(dt, dtype=np.float64)
    phi = np.zeros(len(dt))
    _load().oracle_ubls_phases(len(dt), _p(dt), f, _p(phi))
    return phi


def ubls_order(phi) -> np.ndarray:
    """Points in (phase, index) order (``oracle_ubls_order``)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    ord_ = np.zeros(len(phi), np.int32)
    _load().oracle_ubls_order(len(phi), _p(phi), _p(ord_))
    return ord_


def ubls_extent(phi, order, first: int, length: int) -> float:
    """Phase extent of a run of the phase order (``oracle_ubls_extent``)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    order = np.ascontiguousarray(order, dtype=np.int32)
    return _load().oracle_ubls_extent(len(phi), _p(phi), _p(order), first, length)


def ubls_power(dt, w, x, f: float, qmin: float, qmax: float, sign: int = 0):
    """Best unbinned box of one frequency: (P, first, len, r, s, order)."""
    dt, w, x = (np.ascontiguousarray(a, dtype=np.float64) for a in (dt, w, x))
    a, l = C.c_int(), C.c_int()
    r, s = C.c_double(), C.c_double()
    order = np.zeros(len(dt), np.int32)
    P = _load().oracle_ubls_power(len(dt), _p(dt), _p(w), _p(x), f, qmin, qmax, sign,
                                  C.byref(a), C.byref(l), C.byref(r), C.byref(s), _p(order))
    return P, a.value, l.value, r.value, s.value, order


def ubls(t, y, dy, qmin: float, qmax: float, *, freqs=None, fmin=0.0, df=0.0, nf=None,
         sign: int = 0):
    """Unbinned periodogram (``oracle_ubls``): (P[nf], UnbinnedPeak)."""
    t, y, dy = _arrays(t, y, dy)
    if freqs is not None:
        freqs = np.ascontiguousarray(freqs, dtype=np.float64)
        nf = len(freqs)
    P = np.zeros(nf)
    pk = _UPeak()
    rc = _load().oracle_ubls(len(t), _p(t), _p(y), _p(dy), nf, _p(freqs), fmin, df, qmin, qmax,
                             sign, _p(P), C.byref(pk))
    if rc != 0:
        raise ValueError(f"oracle_ubls failed ({rc})")
    return P, UnbinnedPeak(pk.j, pk.first, pk.len, pk.first_point, pk.freq, pk.power, pk.sr,
                           pk.depth, pk.epoch, pk.duration, pk.snr)
