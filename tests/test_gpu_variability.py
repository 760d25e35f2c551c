"""High-variability pre-filter: CUDA path vs the FP64 oracle (marked gpu).

Every statistic is summed in FP64 in the definition's order on both sides, so the
per-star magnitudes, RMS values, bins, bin expectations and flags must be identical."""
import numpy as np
import pytest

import oracle
from paper_1112_1701_b300 import bls, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    bls.lib()


def _compare(off, m, chip, nchips, **kw):
    g = bls.variability(off, m, chip, nchips, **kw)
    o = oracle.variability(off, m, chip, nchips, **kw)
    for f in ("mag", "rms", "bin", "mu", "sd", "flag"):
        assert np.array_equal(g[f], o[f]), f
    return g


def test_survey_field_catalog():
    c = synth.chip_catalog(nchips=11, stars_per_chip=1200, npts=400, seed=31)
    g = _compare(c.off, c.m, c.chip, c.nchips)
    f = g["flag"].astype(bool)
    assert f[c.variable].mean() > 0.85


def test_interleaved_chips_and_options():
    """Stars of different chips interleaved, unequal light-curve lengths, other clipping
    settings."""
    rng = np.random.default_rng(4)
    c = synth.chip_catalog(nchips=3, stars_per_chip=700, npts=150, seed=32)
    perm = rng.permutation(len(c.chip))
    lens = rng.integers(20, 300, len(perm))
    curves = [c.m[c.off[s]:c.off[s + 1]][:L] for s, L in zip(perm, lens)]
    off = np.concatenate([[0], np.cumsum([len(x) for x in curves])]).astype(np.int64)
    m = np.concatenate(curves).astype(np.float32)
    chip = c.chip[perm]
    for kw in (dict(), dict(clip=2.5, iters=10, nsig=3.0, min_stars=10), dict(iters=0)):
        _compare(off, m, chip, 3, **kw)


def test_device_inputs_and_outputs():
    torch = pytest.importorskip("torch")
    c = synth.chip_catalog(nchips=2, stars_per_chip=500, npts=100, seed=33)
    h = bls.variability(c.off, c.m, c.chip, 2)
    out = torch.zeros(len(c.chip) * bls.VAR_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    bls.variability(torch.tensor(c.off, device="cuda"), torch.tensor(c.m, device="cuda"),
                    torch.tensor(c.chip, device="cuda"), 2, out=out,
                    stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    d = out.cpu().numpy().view(bls.VAR_DTYPE)
    for f in ("mag", "rms", "bin", "mu", "sd", "flag"):
        assert np.array_equal(d[f], h[f]), f


def test_single_star_chip_and_invalid():
    off = np.array([0, 5, 9], np.int64)
    m = np.array([15.0, 15.1, 15.0, 15.1, 15.0, 17.0, 17.0, 17.2, 17.2], np.float32)
    g = _compare(off, m, np.array([0, 1], np.int32), 2, min_stars=1)
    assert g["flag"].sum() == 0          # one star per bin: sd 0, not above itself
    with pytest.raises(bls.BLSError):
        bls.variability(off, m, np.array([0, 2], np.int32), 2)       # chip out of range
    bad = m.copy()
    bad[2] = np.nan
    with pytest.raises(bls.BLSError):
        bls.variability(off, bad, np.array([0, 1], np.int32), 2)
    e = bls.variability(off, m, np.array([0, 1], np.int32), 2)       # still usable
    assert e["bin"].tolist() == [150, 171]
