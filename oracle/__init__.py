"""FP64 CPU oracles of the box-least-squares periodogram (binned and unbinned), the
eclipse-window detection efficiency, the trapezoid refit of a peak and the high-variability
pre-filter (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package. It shares no code with the CUDA library and never imports it.
"""
from .oracle import (  # noqa: F401
    OraclePeak, build, kminmax, freq, fold, prep, bins, power, box, bls, bls_many, lib_path,
    window, window_count, OracleShape, shape, shape_point, star_stats, clip, variability,
    UnbinnedPeak, ubls_phases, ubls_order, ubls_extent, ubls_power, ubls,
)
