"""Python binding of ``libbls.so`` (argument marshalling only).

Every computation happens in the library's CUDA kernels; this module only builds the C
structs of ``include/bls.h`` from numpy arrays or torch tensors and converts results.
There is no CPU fallback: if the library is missing, loading it raises.

Inputs may be numpy arrays (host) or CUDA torch tensors (device); device tensors are
passed by ``data_ptr()`` and the plan can be bound to ``torch.cuda.current_stream()``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass
from typing import Iterable, List, Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# BLS_DEBUG=1 in the environment (read when the library is first loaded) selects the build
# with device-side index checks, whose failures make a call return ERR_INTERNAL.
LIB_PATH = os.path.join(_PKG, "libbls_debug.so" if os.environ.get("BLS_DEBUG") == "1" else "libbls.so")

OK, PENDING = 0, 1
ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_INTERNAL, ERR_CANCELLED = -1, -2, -3, -4, -5, -6
PHASE = {"fx64": 0, "f64": 1, "f32": 2, "df32": 3}
SUM = {"fixed": 0, "f32": 1, "kahan": 2}
SIGN = {"dips": 0, "both": 1}
ALGO = {"tiled": 0, "plain_f64": 1, "unbinned": 2}
FOLD = {"auto": 0, "ws": 1, "one_group": 2}


class BLSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"BLS status {status}: {msg}")
        self.status = status


class PlanDesc(C.Structure):
    _fields_ = [("nb", C.c_int), ("qmin", C.c_double), ("qmax", C.c_double),
                ("kmin", C.c_int), ("kmax", C.c_int), ("topk", C.c_int), ("phase", C.c_int),
                ("sum", C.c_int), ("sign", C.c_int), ("algo", C.c_int),
                ("max_device_bytes", C.c_size_t), ("max_curves_per_launch", C.c_int),
                ("freqs_per_block", C.c_int), ("point_chunk", C.c_int),
                ("max_active_requests", C.c_int), ("step_point_freqs", C.c_longlong),
                ("fold_kernel", C.c_int)]


class CurveStruct(C.Structure):
    _fields_ = [("t", C.c_void_p), ("y", C.c_void_p), ("dy", C.c_void_p), ("n", C.c_int),
                ("freqs", C.c_void_p), ("nf", C.c_int), ("fmin", C.c_double),
                ("df", C.c_double), ("nb", C.c_int), ("qmin", C.c_double),
                ("qmax", C.c_double)]


class PeakStruct(C.Structure):
    _fields_ = [("best_j", C.c_int), ("i1", C.c_int), ("k", C.c_int), ("pad_", C.c_int),
                ("freq", C.c_double), ("period", C.c_double), ("epoch", C.c_double),
                ("duration", C.c_double), ("depth", C.c_double), ("snr", C.c_double),
                ("sr", C.c_double), ("power", C.c_double), ("sde", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64),
                ("cancelled", C.c_uint64), ("failed", C.c_uint64), ("steps", C.c_uint64),
                ("active", C.c_uint64), ("queued", C.c_uint64),
                ("device_bytes_in_use", C.c_size_t), ("device_bytes_peak", C.c_size_t),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double)]


class WindowDesc(C.Structure):
    _fields_ = [("t", C.c_void_p), ("n", C.c_int), ("freqs", C.c_void_p), ("nf", C.c_int),
                ("fmin", C.c_double), ("df", C.c_double), ("nphi", C.c_int),
                ("duration", C.c_double), ("qfrac", C.c_double), ("min_eclipses", C.c_int),
                ("min_points", C.c_int)]


class ShapeGrid(C.Structure):
    _fields_ = [("ncentre", C.c_int), ("nwidth", C.c_int), ("ningress", C.c_int),
                ("width_lo", C.c_double), ("width_hi", C.c_double), ("ingress_max", C.c_double)]


SHAPE_DTYPE = np.dtype([("index", np.int32), ("box_index", np.int32), ("power", np.float64),
                        ("box_power", np.float64), ("epoch", np.float64),
                        ("duration", np.float64), ("ingress", np.float64), ("depth", np.float64)])


class VarDesc(C.Structure):
    _fields_ = [("off", C.c_void_p), ("m", C.c_void_p), ("chip", C.c_void_p),
                ("nstars", C.c_int), ("nchips", C.c_int), ("clip", C.c_double),
                ("iters", C.c_int), ("nsig", C.c_double), ("min_stars", C.c_int)]


VAR_DTYPE = np.dtype([("mag", np.float64), ("rms", np.float64), ("mu", np.float64),
                      ("sd", np.float64), ("bin", np.int32), ("flag", np.uint8),
                      ("pad_", np.uint8, 3)])


class Profile(C.Structure):
    _fields_ = [("searches", C.c_uint64), ("kernel_launches", C.c_uint64),
                ("fold_launches", C.c_uint64), ("prep_ms", C.c_double),
                ("fold_ms", C.c_double), ("reduce_ms", C.c_double),
                ("graph_captures", C.c_uint64), ("graph_replays", C.c_uint64)]


PEAK_DTYPE = np.dtype([("j", np.int32), ("i1", np.int32), ("k", np.int32), ("pad_", np.int32),
                       ("freq", np.float64), ("period", np.float64), ("epoch", np.float64),
                       ("duration", np.float64), ("depth", np.float64), ("snr", np.float64),
                       ("sr", np.float64), ("power", np.float64), ("sde", np.float64)])
assert PEAK_DTYPE.itemsize == C.sizeof(PeakStruct)

_lib = None
_lock = threading.Lock()

EXPORTS = ["bls_plan_create", "bls_plan_destroy", "bls_search", "bls_submit", "bls_poll",
           "bls_cancel", "bls_server_stats_get", "bls_kminmax", "bls_debug_fold",
           "bls_debug_powers", "bls_tile_shape", "bls_profile_get", "bls_search_static", "bls_window_efficiency", "bls_refine", "bls_search_shapes", "bls_variability",
           "bls_moments_of", "bls_moments_merge", "bls_sde", "bls_last_error"]


def lib():
    """Load ``libbls.so`` (built in-tree); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run `python -m "
                                   "paper_1112_1701_b300.build` (there is no CPU fallback)")
            L = C.CDLL(LIB_PATH)
            P, I, D = C.c_void_p, C.c_int, C.c_double
            L.bls_plan_create.argtypes = [C.POINTER(PlanDesc), P, C.POINTER(P)]
            L.bls_plan_destroy.argtypes = [P]
            L.bls_plan_destroy.restype = None
            L.bls_search.argtypes = [P, C.POINTER(CurveStruct), I, P, P]
            L.bls_submit.argtypes = [P, C.POINTER(CurveStruct), C.POINTER(C.c_uint64)]
            L.bls_poll.argtypes = [P, C.c_uint64, P, I]
            L.bls_cancel.argtypes = [P, C.c_uint64]
            L.bls_server_stats_get.argtypes = [P, C.POINTER(ServerStats)]
            L.bls_kminmax.argtypes = [I, D, D, C.POINTER(I), C.POINTER(I)]
            L.bls_tile_shape.argtypes = [P, I, C.POINTER(I), C.POINTER(I), C.POINTER(I)]
            L.bls_moments_of.argtypes = [P, C.c_longlong, C.POINTER(Moments)]
            L.bls_moments_merge.argtypes = [C.POINTER(Moments), I, C.POINTER(Moments)]
            L.bls_sde.argtypes = [D, C.POINTER(Moments), C.POINTER(D)]
            L.bls_debug_fold.argtypes = [P, C.POINTER(CurveStruct), P, I, P]
            L.bls_debug_powers.argtypes = [P, C.POINTER(CurveStruct), P, P, P]
            L.bls_profile_get.argtypes = [P, C.POINTER(Profile), I]
            L.bls_search_static.argtypes = [C.POINTER(CurveStruct), I, I, P, P, P]
            L.bls_window_efficiency.argtypes = [C.POINTER(WindowDesc), P, P, P]
            L.bls_refine.argtypes = [P, C.POINTER(CurveStruct), I, P, I, I, P]
            L.bls_search_shapes.argtypes = [P, C.POINTER(CurveStruct), I, P, P,
                                            C.POINTER(ShapeGrid), P]
            L.bls_variability.argtypes = [C.POINTER(VarDesc), P, P]
            L.bls_last_error.argtypes = []
            L.bls_last_error.restype = C.c_char_p
            _lib = L
    return _lib


def _check(st: int):
    if st not in (OK,):
        raise BLSError(st, lib().bls_last_error().decode())
    return st


def kminmax(nb: int, qmin: float, qmax: float):
    a, b = C.c_int(), C.c_int()
    _check(lib().bls_kminmax(nb, qmin, qmax, C.byref(a), C.byref(b)))
    return a.value, b.value


class Moments(C.Structure):
    _fields_ = [("count", C.c_longlong), ("mean", C.c_double), ("m2", C.c_double)]


def moments_of(sr) -> tuple:
    """``bls_moments_of``: (count, mean, M2) of an SR spectrum (FP32, host or device)."""
    a = _host(sr, np.float32, "sr")
    m = Moments()
    _check(lib().bls_moments_of(_ptr(a), _len(a), C.byref(m)))
    return m.count, m.mean, m.m2


def moments_merge(parts) -> tuple:
    """``bls_moments_merge``: moments of the union of disjoint parts' (count, mean, M2)."""
    arr = (Moments * max(1, len(parts)))(*[Moments(int(n), float(mu), float(m2))
                                             for n, mu, m2 in parts])
    m = Moments()
    _check(lib().bls_moments_merge(arr, len(parts), C.byref(m)))
    return m.count, m.mean, m.m2


def sde(sr: float, moments) -> float:
    """``bls_sde``: signal detection efficiency of a peak against merged moments."""
    n, mu, m2 = moments
    m = Moments(int(n), float(mu), float(m2))
    out = C.c_double()
    _check(lib().bls_sde(float(sr), C.byref(m), C.byref(out)))
    return out.value


def _ptr(a):
    """Address of a numpy array or a torch tensor (keeps no reference)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


_TORCH_DTYPE = {np.dtype(np.float64): "torch.float64", np.dtype(np.float32): "torch.float32",
                np.dtype(np.int64): "torch.int64", np.dtype(np.int32): "torch.int32"}


def _host(a, dtype, name="array"):
    """numpy arrays are converted (a contiguous copy of the stated dtype when needed);
    torch tensors are passed by address, so they must already have that dtype and be
    contiguous -- the library reads them as plain arrays of it."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        want = _TORCH_DTYPE[np.dtype(dtype)]
        if str(a.dtype) != want:
            raise BLSError(ERR_INVALID, f"{name}: tensor of {a.dtype}, expected {want}")
        if not a.is_contiguous():
            raise BLSError(ERR_INVALID, f"{name}: tensor is not contiguous")
        return a
    return np.ascontiguousarray(a, dtype=dtype)


def _len(a) -> int:
    return int(a.numel()) if hasattr(a, "numel") else int(a.size)


@dataclass
class CurveInput:
    """One light curve and its grid.  Arrays: numpy (host) or CUDA torch tensors."""
    t: object
    y: object
    dy: object = None
    nf: int = 0
    fmin: float = 0.0
    df: float = 0.0
    freqs: object = None
    nb: int = 0
    qmin: float = 0.0
    qmax: float = 0.0


def _struct(c: CurveInput, keep: list) -> CurveStruct:
    t = _host(c.t, np.float64, "t")
    y = _host(c.y, np.float32, "y")
    dy = _host(c.dy, np.float32, "dy")
    fr = _host(c.freqs, np.float64, "freqs")
    keep += [t, y, dy, fr]
    n = _len(t)
    for name, a in (("y", y), ("dy", dy)):
        if a is not None and _len(a) != n:
            raise BLSError(ERR_INVALID, f"{name} holds {_len(a)} values, t holds {n}")
    nf = _len(fr) if fr is not None else int(c.nf)
    return CurveStruct(_ptr(t), _ptr(y), _ptr(dy), n, _ptr(fr), nf, float(c.fmin),
                       float(c.df), int(c.nb), float(c.qmin), float(c.qmax))


class PackedCurves:
    """Many curves stored back to back in three arrays (t FP64, y and dy FP32: numpy, or
    torch tensors on the host or a CUDA device; dy may be None), each with a uniform grid.
    The bls_curve descriptors are written with vectorised numpy from the per-curve point
    counts, so a search call does no per-curve Python work.  counts, nf, fmin, df, nb, qmin
    and qmax are per-curve sequences or scalars (0 = the plan's default for nb, qmin, qmax)."""

    def __init__(self, t, y, dy, counts, nf, fmin, df, nb=0, qmin=0.0, qmax=0.0):
        counts = np.asarray(counts, np.int64)
        m = len(counts)
        self.keep = [_host(t, np.float64, "t"), _host(y, np.float32, "y"),
                     _host(dy, np.float32, "dy")]
        off = np.zeros(m, np.int64)
        np.cumsum(counts[:-1], out=off[1:])
        npts = int(counts.sum())
        for a in self.keep:
            if a is not None and _len(a) < npts:
                raise ValueError(f"packed array holds {_len(a)} points, counts sum to {npts}")
        F = CurveStruct
        dt = np.dtype({"names": [f for f, _ in F._fields_],
                       "formats": ["u8", "u8", "u8", "i4", "u8", "i4", "f8", "f8", "i4", "f8", "f8"],
                       "offsets": [getattr(F, f).offset for f, _ in F._fields_],
                       "itemsize": C.sizeof(F)})
        rec = np.zeros(m, dt)
        for name, a, w in (("t", self.keep[0], 8), ("y", self.keep[1], 4), ("dy", self.keep[2], 4)):
            rec[name] = 0 if a is None else np.uint64(_ptr(a)) + (off * w).astype(np.uint64)
        rec["n"] = counts
        rec["freqs"] = 0
        rec["nf"] = nf
        rec["fmin"] = fmin
        rec["df"] = df
        rec["nb"] = nb
        rec["qmin"] = qmin
        rec["qmax"] = qmax
        self.rec = rec
        self.arr = (F * m).from_buffer(rec)
        self.total_nf = int(np.asarray(rec["nf"], np.int64).sum())

    def __len__(self):
        return len(self.rec)


def _curve_array(curves, keep: list):
    if isinstance(curves, PackedCurves):
        return curves.arr
    return (CurveStruct * len(curves))(*[_struct(c, keep) for c in curves])


def _check_spectrum(spectrum, arr) -> None:
    """The spectrum output must hold the sum of the curves' frequency counts (the library
    writes that many floats)."""
    if spectrum is None:
        return
    need = int(np.asarray(arr.rec["nf"], np.int64).sum()) if isinstance(arr, PackedCurves) \
        else sum(int(c.nf) for c in arr)
    have = int(spectrum.numel()) if hasattr(spectrum, "numel") else int(np.asarray(spectrum).size)
    if have < need:
        raise ValueError(f"spectrum holds {have} values, the curves have {need} frequencies")


def packed_from_batch(batch, device=None, pinned: bool = False) -> PackedCurves:
    """PackedCurves of a synth.Batch (arrays placed as by curves_from_batch)."""
    ts = np.concatenate([c.t for c in batch.curves])
    ys = np.concatenate([c.y for c in batch.curves])
    dys = np.concatenate([c.dy for c in batch.curves])
    if device is not None or pinned:
        import torch
        conv = (lambda a: torch.from_numpy(a).to(device)) if device is not None else \
            (lambda a: torch.from_numpy(a).pin_memory())
        ts, ys, dys = conv(ts), conv(ys), conv(dys)
    return PackedCurves(ts, ys, dys, [len(c.t) for c in batch.curves],
                        [g.nf for g in batch.grids], [g.fmin for g in batch.grids],
                        [g.df for g in batch.grids], list(batch.nb), batch.qmin, batch.qmax)


def curves_from_batch(batch, device=None, pinned: bool = False) -> List[CurveInput]:
    """CurveInputs of a synth.Batch, packed into contiguous arrays (one copy per array
    for the whole batch).  With ``device`` (e.g. "cuda") the arrays are torch tensors
    resident there; with ``pinned`` they are page-locked host torch tensors."""
    ts = np.concatenate([c.t for c in batch.curves])
    ys = np.concatenate([c.y for c in batch.curves])
    dys = np.concatenate([c.dy for c in batch.curves])
    if device is not None or pinned:
        import torch
        conv = (lambda a: torch.from_numpy(a).to(device)) if device is not None else \
            (lambda a: torch.from_numpy(a).pin_memory())
        ts, ys, dys = conv(ts), conv(ys), conv(dys)
    out, o = [], 0
    for c, g, nb in zip(batch.curves, batch.grids, batch.nb):
        n = len(c.t)
        out.append(CurveInput(ts[o:o + n], ys[o:o + n], dys[o:o + n], nf=g.nf, fmin=g.fmin,
                              df=g.df, nb=nb, qmin=batch.qmin, qmax=batch.qmax))
        o += n
    return out


def window_efficiency(t, nphi: int, *, freqs=None, fmin: float = 0.0, df: float = 0.0,
                      nf: Optional[int] = None, duration: float = 0.0, qfrac: float = 0.0,
                      min_eclipses: int = 2, min_points: int = 1, want_counts: bool = False,
                      stream=None, eff=None, counts=None):
    """``bls_window_efficiency``: eclipse-window detection efficiency per frequency.

    ``t`` (sorted) and ``freqs`` are numpy arrays or CUDA tensors.  Returns (eff, counts):
    numpy arrays, or the given ``eff`` / ``counts`` buffers (numpy or CUDA tensors)."""
    t = _host(t, np.float64)
    if freqs is not None:
        freqs = _host(freqs, np.float64)
        nf = len(freqs)
    if nf is None:
        raise ValueError("give freqs, or fmin/df/nf")
    if eff is None:
        eff = np.zeros(nf, np.float64)
    if counts is None and want_counts:
        counts = np.zeros((nf, nphi), np.int32)
    d = WindowDesc(_ptr(t), len(t), _ptr(freqs), nf, fmin, df, nphi, duration, qfrac,
                   min_eclipses, min_points)
    _check(lib().bls_window_efficiency(C.byref(d), stream, _ptr(eff), _ptr(counts)))
    return eff, counts


def variability(off, m, chip, nchips: int, clip: float = 3.0, iters: int = 5,
                nsig: float = 2.0, min_stars: int = 5, stream=None, out=None):
    """``bls_variability``: high-variability flags of every star.  Arrays: numpy or CUDA
    tensors; returns the records (numpy structured array of VAR_DTYPE, or ``out``)."""
    off = _host(off, np.int64)
    m = _host(m, np.float32)
    chip = _host(chip, np.int32)
    n = len(chip)
    if out is None:
        out = np.zeros(n, dtype=VAR_DTYPE)
    d = VarDesc(_ptr(off), _ptr(m), _ptr(chip), n, nchips, clip, iters, nsig, min_stars)
    _check(lib().bls_variability(C.byref(d), stream, _ptr(out)))
    return out


def search_static(curve: CurveInput, topk: int = 1, sign: str = "dips", stream=None,
                  peaks=None, spectrum=None):
    """``bls_search_static``: one curve, device inputs and outputs, no allocation inside.

    ``peaks`` is a CUDA uint8 tensor of at least topk * sizeof(bls_peak) bytes; it receives
    the peak records (read them back with ``peaks_to_numpy``)."""
    keep: list = []
    cs = _struct(curve, keep)
    # the library cannot see the size of a device buffer: check the outputs here
    if peaks is None or not hasattr(peaks, "element_size"):
        raise BLSError(ERR_INVALID, "peaks must be a CUDA tensor")
    need = int(topk) * PEAK_DTYPE.itemsize
    if _len(peaks) * peaks.element_size() < need or not peaks.is_contiguous():
        raise BLSError(ERR_INVALID, f"peaks holds {_len(peaks) * peaks.element_size()} bytes, "
                                    f"topk = {int(topk)} records need {need}")
    if spectrum is not None:
        if not hasattr(spectrum, "element_size") or str(spectrum.dtype) != "torch.float32" \
                or not spectrum.is_contiguous():
            raise BLSError(ERR_INVALID, "spectrum must be a contiguous float32 CUDA tensor")
        if _len(spectrum) < cs.nf:
            raise BLSError(ERR_INVALID, f"spectrum holds {_len(spectrum)} values, the curve "
                                        f"has {cs.nf} frequencies")
    _check(lib().bls_search_static(C.byref(cs), int(topk), SIGN[sign], stream, _ptr(peaks),
                                   _ptr(spectrum)))


def peaks_to_numpy(buf, topk: int) -> np.ndarray:
    """Peak records written to a device byte buffer, as a structured numpy array."""
    raw = buf.detach().cpu().numpy().view(np.uint8)[:topk * PEAK_DTYPE.itemsize]
    return raw.view(PEAK_DTYPE).copy()


class Plan:
    """A search plan on the current CUDA device (``bls_plan_create``)."""

    def __init__(self, nb=200, qmin=0.005, qmax=0.15, kmin=0, kmax=0, topk=1, phase="fx64",
                 sum="fixed", sign="dips", algo="tiled", max_device_bytes=0,
                 max_curves_per_launch=0, freqs_per_block=0, point_chunk=0,
                 max_active_requests=0, step_point_freqs=0, fold_kernel="auto", stream=None):
        self.desc = PlanDesc(nb, qmin, qmax, kmin, kmax, topk, PHASE[phase], SUM[sum],
                             SIGN[sign], ALGO[algo], max_device_bytes, max_curves_per_launch,
                             freqs_per_block, point_chunk, max_active_requests,
                             step_point_freqs, FOLD[fold_kernel])
        self.topk = topk
        h = C.c_void_p()
        _check(lib().bls_plan_create(C.byref(self.desc), stream, C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().bls_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def search(self, curves, spectrum=None) -> np.ndarray:
        """Peaks of every curve (a sequence of CurveInput, or PackedCurves): structured array
        of shape (ncurves, topk)."""
        keep: list = []
        arr = _curve_array(curves, keep)
        _check_spectrum(spectrum, curves if isinstance(curves, PackedCurves) else arr)
        out = np.zeros((len(curves), self.topk), dtype=PEAK_DTYPE)
        _check(lib().bls_search(self._h, arr, len(curves), out.ctypes.data, _ptr(spectrum)))
        return out

    def search_shapes(self, curves: Sequence[CurveInput], ncentre: int = 0, nwidth: int = 0,
                      ningress: int = 0, width_lo: float = 0.0, width_hi: float = 0.0,
                      ingress_max: float = -1.0, spectrum=None):
        """``bls_search_shapes``: (peaks, trapezoid refits), both (ncurves, topk)."""
        keep: list = []
        arr = (CurveStruct * len(curves))(*[_struct(c, keep) for c in curves])
        out = np.zeros((len(curves), self.topk), dtype=PEAK_DTYPE)
        shapes = np.zeros((len(curves), self.topk), dtype=SHAPE_DTYPE)
        _check_spectrum(spectrum, arr)
        g = ShapeGrid(ncentre, nwidth, ningress, width_lo, width_hi, ingress_max)
        _check(lib().bls_search_shapes(self._h, arr, len(curves), out.ctypes.data,
                                       _ptr(spectrum), C.byref(g), shapes.ctypes.data))
        return out, shapes

    def refine(self, curves: Sequence[CurveInput], peaks: np.ndarray, oversample: int = 10,
               half: int = 2) -> np.ndarray:
        """``bls_refine``: fine-grid re-search around each peak of ``peaks`` (as returned by
        ``search`` for the same curves)."""
        keep: list = []
        arr = (CurveStruct * len(curves))(*[_struct(c, keep) for c in curves])
        coarse = np.ascontiguousarray(peaks, dtype=PEAK_DTYPE).reshape(len(curves), self.topk)
        out = np.zeros((len(curves), self.topk), dtype=PEAK_DTYPE)
        _check(lib().bls_refine(self._h, arr, len(curves), coarse.ctypes.data, oversample, half,
                                out.ctypes.data))
        return out

    def submit(self, curve: CurveInput) -> int:
        keep: list = []
        cs = _struct(curve, keep)
        tk = C.c_uint64()
        _check(lib().bls_submit(self._h, C.byref(cs), C.byref(tk)))
        return tk.value

    def poll(self, ticket: int, timeout_ms: int = 0):
        """(status, peaks or None); status is OK, PENDING or ERR_TIMEOUT; raises on
        other errors."""
        out = np.zeros(self.topk, dtype=PEAK_DTYPE)
        st = lib().bls_poll(self._h, ticket, out.ctypes.data, int(timeout_ms))
        if st in (PENDING, ERR_TIMEOUT):
            return st, None
        _check(st)
        return st, out

    def cancel(self, ticket: int):
        _check(lib().bls_cancel(self._h, ticket))

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().bls_server_stats_get(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def profile(self, reset: bool = False) -> dict:
        """CUDA-event kernel timings of the searches run so far (bls_profile_get)."""
        s = Profile()
        _check(lib().bls_profile_get(self._h, C.byref(s), int(reset)))
        return {k: getattr(s, k) for k, _ in Profile._fields_}

    def debug_fold(self, curve: CurveInput, js: Iterable[int]) -> np.ndarray:
        keep: list = []
        cs = _struct(curve, keep)
        js = np.ascontiguousarray(list(js), dtype=np.int32)
        n = cs.n
        out = np.empty((len(js), n), dtype=np.int32)
        _check(lib().bls_debug_fold(self._h, C.byref(cs), js.ctypes.data, len(js),
                                    out.ctypes.data))
        return out

    def tile_shape(self, nb: int = 0) -> dict:
        """The launch shape this plan's tiled search uses for curves of `nb` bins (0: the
        plan's own): frequencies per tile, points per staged chunk and the fold-sweep kernel."""
        cols, chunk, ws = C.c_int(), C.c_int(), C.c_int()
        _check(lib().bls_tile_shape(self._h, int(nb), C.byref(cols), C.byref(chunk), C.byref(ws)))
        return {"cols": cols.value, "chunk": chunk.value,
                "fold_kernel": "ws" if ws.value else "one_group"}

    def debug_powers(self, curve: CurveInput):
        keep: list = []
        cs = _struct(curve, keep)
        P = np.empty(cs.nf, dtype=np.float32)
        i1 = np.empty(cs.nf, dtype=np.int32)
        k = np.empty(cs.nf, dtype=np.int32)
        _check(lib().bls_debug_powers(self._h, C.byref(cs), P.ctypes.data, i1.ctypes.data,
                                      k.ctypes.data))
        return P, i1, k
