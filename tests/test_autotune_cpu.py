"""Autotuner host logic (no GPU): candidate sets, sampling, selection and the cache, with a
stand-in timer in place of the CUDA-event timing."""
import json

import numpy as np
import pytest

from paper_1112_1701_b300 import autotune as at
from paper_1112_1701_b300 import bls, build, synth


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    bls.lib()


def test_candidates_fit_shared_memory_and_kernel_rules():
    cands = at.candidates(200, 1, 30)
    assert cands[0] == at.DEFAULT
    for c in cands[1:]:
        assert 8 <= c.freqs_per_block <= 256
        # the one-group kernel's histograms are strided at a multiple of 16 columns, the
        # warp-specialised kernel's at the width itself (a multiple of 8)
        stride = c.freqs_per_block if c.fold_kernel == "ws" else (c.freqs_per_block + 15) & ~15
        assert 2 * c.point_chunk * 24 + 2048 + stride * 200 * 8 <= 231424
        if c.fold_kernel == "ws":
            assert c.freqs_per_block % 8 == 0 and c.freqs_per_block <= 128
        else:
            assert c.freqs_per_block % 16 == 0
    # one warp-specialised width between the multiples of 16: the widest that fits with a
    # chunk of 256..512 points (nb = 200: 120 columns; nb = 256: 104 columns, 336 points)
    odd = [c for c in cands[1:] if c.freqs_per_block % 16]
    assert [(c.freqs_per_block, c.point_chunk, c.fold_kernel) for c in odd] == [(120, 512, "ws")]
    odd256 = [c for c in at.candidates(256, 1, 39)[1:] if c.freqs_per_block % 16]
    assert [(c.freqs_per_block, c.point_chunk) for c in odd256] == [(104, 336)]
    widths = {c.freqs_per_block for c in cands if c.point_chunk == 512}
    assert max(widths) == 128 and 96 in widths and 64 in widths
    assert any(c.fold_kernel == "ws" and c.freqs_per_block == 128 for c in cands)
    # Kahan sums: 16-byte entries (half the widths), both kernels
    kc = at.candidates(200, 1, 30, sums="kahan")
    assert any(c.fold_kernel == "ws" for c in kc)
    assert max(c.freqs_per_block for c in kc[1:]) == 64
    # small nb: widths up to 256
    assert max(c.freqs_per_block for c in at.candidates(100, 1, 15)[1:]) == 256


def test_sample_spans_lengths_and_truncates_grids():
    b = synth.config2(ncurves=40, nf=5000, seed=3)
    cis = bls.curves_from_batch(b)
    smp = at.sample_curves(cis, 8, tiles_needed=100, widest=128)
    ns = [len(c.t) for c in smp]
    all_n = sorted(len(c.t) for c in cis)
    assert ns == sorted(ns) and ns[0] == all_n[0] and ns[-1] == all_n[-1]
    assert all(c.nf == 1600 for c in smp)          # ceil(100 * 128 / 8) frequencies
    assert smp[0].fmin == cis[0].fmin and smp[0].df == cis[0].df
    freqs = np.linspace(0.2, 3.0, 900)
    ex = [bls.CurveInput(c.t, c.y, c.dy, freqs=freqs, nb=200) for c in cis[:3]]
    smp2 = at.sample_curves(ex, 2, tiles_needed=4, widest=128)
    assert all(len(c.freqs) == 256 for c in smp2)
    assert np.array_equal(smp2[0].freqs, freqs[:256])


def _fake_timer(table):
    calls = []

    def timer(c, smp, nb, qmin, qmax, phase, sums, sign, reps, stream=None):
        calls.append(c)
        return table(c)
    return timer, calls


def test_tune_picks_fastest_skips_infeasible_and_caches(tmp_path):
    b = synth.config2(ncurves=16, nf=2000, seed=4)
    cis = bls.curves_from_batch(b)

    def cost(c):
        if c.freqs_per_block == 112:
            return None                    # "does not fit"
        if c == at.DEFAULT:
            return 10.0
        return 5.0 if (c.freqs_per_block, c.point_chunk, c.fold_kernel) == (96, 512, "ws") else 20.0
    timer, calls = _fake_timer(cost)
    path = str(tmp_path / "tune.json")
    cache = at.TuneCache(path)
    res = at.tune(cis, 200, 0.005, 0.15, timer=timer, cache=cache, device=("B300", 148))
    assert res.best == at.Candidate(96, 512, "ws") and res.best_ms == 5.0
    assert res.default_ms == 10.0 and not res.cached
    assert any(ms is None for _, ms in res.table)
    # every candidate, then the best one in two and four launches (no gain: one launch kept)
    assert len(calls) == len(at.candidates(200, 1, 30)) + len(at.SPLITS)
    assert res.splits == 1 and res.best.curves_per_launch == 0
    saved = json.load(open(path))
    assert res.key in saved and saved[res.key]["freqs_per_block"] == 96
    # a second run hits the cache (in a fresh cache object reading the file)
    timer2, calls2 = _fake_timer(cost)
    res2 = at.tune(cis, 200, 0.005, 0.15, timer=timer2, cache=at.TuneCache(path),
                   device=("B300", 148))
    assert res2.cached and res2.best == res.best and not calls2
    # another length class or device is another key
    res3 = at.tune(cis, 200, 0.005, 0.15, timer=timer2, cache=at.TuneCache(path),
                   device=("B300", 132))
    assert not res3.cached


def test_second_stage_picks_the_launch_split():
    """When the sample runs faster in four launches, the whole batch is split into four:
    curves_per_launch = ceil(N / 4) for the batch (not the sample), and the cache keeps the
    split, not the count."""
    b = synth.config2(ncurves=50, nf=2000, seed=5)
    cis = bls.curves_from_batch(b)

    def cost(c):
        if c.freqs_per_block == 0:
            return 10.0
        if c.curves_per_launch:
            return 4.0 if c.curves_per_launch <= 8 else 6.0
        return 9.0 if (c.freqs_per_block, c.point_chunk) == (128, 512) else 20.0
    timer, calls = _fake_timer(cost)
    cache = at.TuneCache(None)
    res = at.tune(cis, 200, 0.005, 0.15, timer=timer, cache=cache, device=("B300", 148))
    assert res.splits == 4 and res.best_ms == 4.0
    assert res.best.curves_per_launch == 13                      # ceil(50 / 4)
    assert res.best.plan_kwargs()["max_curves_per_launch"] == 13
    hit = at.tune(cis[:20], 200, 0.005, 0.15, timer=timer, cache=cache, device=("B300", 148))
    assert hit.cached and hit.splits == 4 and hit.best.curves_per_launch == 5   # ceil(20 / 4)


def test_ties_keep_the_library_rule():
    cis = bls.curves_from_batch(synth.config2(ncurves=4, nf=500, seed=5))
    timer, _ = _fake_timer(lambda c: 7.0)
    res = at.tune(cis, 200, 0.005, 0.15, timer=timer, cache=at.TuneCache(None),
                  device=("X", 10))
    assert res.best == at.DEFAULT


def test_plan_accepts_the_fold_kernel_choice():
    assert bls.FOLD == {"auto": 0, "ws": 1, "one_group": 2}
    d = bls.PlanDesc(200, 0.005, 0.15, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, bls.FOLD["ws"])
    assert d.fold_kernel == 1
