"""Sharding of the batched search over several GPUs, one process per GPU.

Each light curve is searched on its own (Sec. 2.2.2 runs the periodogram of every curve
independently), so a batch splits into contiguous curve ranges, one per rank.  Each rank
searches its range with no device collective, and rank 0 gathers the per-curve peak
records on the host (sizeof(bls_peak) = 80 B per peak).

A single curve with a very long frequency grid can instead be split into contiguous
frequency ranges.  Each rank searches an explicit sub-grid whose frequencies are the full
grid's, evaluated by the same formula f_j = fmin + j*df (one rounded product, one rounded
sum), so every rank sees bit-identical trial frequencies; the best peak is then one
argmax over ranks under the search's ordering key: power descending, then frequency
index, box start and box width ascending, and its signal detection efficiency is
recomputed from the merged moments of the ranks' spectra.  Only the best peak (top-1) is
merged this way: a local maximum of SR(f) at a shard boundary would need its neighbour
on the other rank.

The collectives are torch.distributed object gathers, so any backend works (gloo on CPU
hosts, NCCL between GPUs); a group of one rank needs no process group at all.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

from . import bls
from .bls import PEAK_DTYPE


def _world(group=None) -> Tuple[int, int]:
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            return dist.get_world_size(group), dist.get_rank(group)
    except ImportError:
        pass
    return 1, 0


def curve_range(ncurves: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous curve range [lo, hi) of `rank`: sizes differ by at most one, lower ranks
    take the remainder."""
    if world < 1 or not 0 <= rank < world or ncurves < 0:
        raise ValueError(f"bad shard: ncurves={ncurves} world={world} rank={rank}")
    base, rem = divmod(ncurves, world)
    lo = rank * base + min(rank, rem)
    return lo, lo + base + (1 if rank < rem else 0)


def freq_range(nf: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous frequency-index range [lo, hi) of `rank` (same split as curve_range)."""
    return curve_range(nf, world, rank)


def sub_grid(fmin: float, df: float, lo: int, hi: int) -> np.ndarray:
    """Frequencies f_j = fmin + j*df for lo <= j < hi, each evaluated as one rounded FP64
    product and one rounded FP64 sum (numpy does not contract them), so a shard's explicit
    grid equals the corresponding slice of the full uniform grid bit for bit."""
    j = np.arange(lo, hi, dtype=np.float64)
    return np.float64(fmin) + j * np.float64(df)


def _gather(obj, group=None) -> Optional[list]:
    world, rank = _world(group)
    if world == 1:
        return [obj]
    import torch.distributed as dist
    out = [None] * world if rank == 0 else None
    dst = dist.get_global_rank(group, 0) if group is not None else 0
    dist.gather_object(obj, out, dst=dst, group=group)
    return out


def search_curve_shards(ncurves: int, search: Callable[[int, int], np.ndarray],
                        group=None) -> Optional[np.ndarray]:
    """Runs `search(lo, hi)` on this rank's curve range; it returns a (hi-lo, topk) array of
    PEAK_DTYPE.  Rank 0 returns the (ncurves, topk) records of the whole batch in curve
    order; the other ranks return None."""
    world, rank = _world(group)
    lo, hi = curve_range(ncurves, world, rank)
    local = np.asarray(search(lo, hi))
    if local.dtype != PEAK_DTYPE or local.ndim != 2 or local.shape[0] != hi - lo:
        raise ValueError(f"search({lo}, {hi}) returned {local.dtype} {local.shape}")
    parts = _gather((lo, local), group)
    if rank != 0:
        return None
    parts.sort(key=lambda p: p[0])
    return np.concatenate([p[1] for p in parts], axis=0)


def better(a, b) -> bool:
    """True if peak record `a` ranks above `b`: larger power, then smaller frequency index,
    box start and box width."""
    if a["power"] != b["power"]:
        return bool(a["power"] > b["power"])
    return (int(a["j"]), int(a["i1"]), int(a["k"])) < (int(b["j"]), int(b["i1"]), int(b["k"]))


def merge_best(peaks: Sequence[np.void]) -> np.ndarray:
    """The best of several peak records of one curve under `better`, as a 1-element
    PEAK_DTYPE array."""
    if len(peaks) == 0:
        raise ValueError("no peaks to merge")
    best = peaks[0]
    for p in peaks[1:]:
        if better(p, best):
            best = p
    return np.array([best], dtype=PEAK_DTYPE)


def spectrum_moments(sr: np.ndarray) -> Tuple[int, float, float]:
    """(count, mean, sum of squared deviations) of an SR spectrum (``bls_moments_of``:
    two passes in FP64 over the FP32 values)."""
    return bls.moments_of(np.ascontiguousarray(sr, dtype=np.float32))


def merge_moments(parts) -> Tuple[int, float, float]:
    """Moments of the union of disjoint parts (``bls_moments_merge``: the pairwise update of
    Chan, Golub and LeVeque)."""
    return bls.moments_merge(list(parts))


def search_freq_shards(nf: int, fmin: float, df: float,
                       search: Callable[[np.ndarray, int], Tuple[np.void, np.ndarray]],
                       group=None) -> Optional[np.ndarray]:
    """Runs `search(freqs, lo)` on this rank's slice of a uniform grid of nf frequencies;
    it returns the best PEAK_DTYPE record over that slice (`j` local to it) and the slice's
    SR spectrum.  Rank 0 returns the best record over the whole grid with j global and its
    signal detection efficiency recomputed over the whole spectrum (the slices' moments
    merged); the other ranks return None.  A rank whose slice is empty contributes
    nothing."""
    world, rank = _world(group)
    lo, hi = freq_range(nf, world, rank)
    rec = None
    mom = (0, 0.0, 0.0)
    if hi > lo:
        r, sr = search(sub_grid(fmin, df, lo, hi), lo)
        arr = np.array(r, dtype=PEAK_DTYPE).reshape(1)
        arr["j"] += lo
        rec = arr[0]
        mom = spectrum_moments(sr)
    parts = _gather((rec, mom), group)
    if rank != 0:
        return None
    best = merge_best([p[0] for p in parts if p[0] is not None])
    best["sde"] = bls.sde(float(best["sr"][0]), merge_moments([p[1] for p in parts]))
    return best


def world_info(group=None) -> Tuple[int, int]:
    """(world size, rank) of `group`, or (1, 0) without a process group."""
    return _world(group)


__all__: List[str] = ["curve_range", "freq_range", "sub_grid", "search_curve_shards",
                      "search_freq_shards", "merge_best", "better", "world_info",
                      "spectrum_moments", "merge_moments"]
