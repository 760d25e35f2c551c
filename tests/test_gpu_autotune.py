"""Autotuner on the GPU (marked gpu): it times every feasible candidate, and the tuned
plan's search gives the default plan's peaks (bins and boxes do not depend on the launch
parameters; powers agree within the sweep approximation)."""
import numpy as np
import pytest

from paper_1112_1701_b300 import autotune as at
from paper_1112_1701_b300 import bls, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    bls.lib()


def test_tuned_plan_matches_default():
    b = synth.config2(ncurves=12, nf=3000, seed=21)
    cis = bls.curves_from_batch(b)
    cache = at.TuneCache(None)
    res = at.tune(cis, 200, b.qmin, b.qmax, sample=6, tiles_per_sm=2, reps=1, cache=cache)
    timed = [ms for _, ms in res.table if ms is not None]
    assert len(timed) >= 10 and all(ms > 0 for ms in timed)
    assert res.best_ms == min(timed) and res.default_ms > 0
    nf = sum(ci.nf for ci in cis)
    s0, s1 = np.zeros(nf, np.float32), np.zeros(nf, np.float32)
    with bls.Plan(nb=200, qmin=b.qmin, qmax=b.qmax, topk=2) as p:
        pk0 = p.search(cis, spectrum=s0)
    with bls.Plan(nb=200, qmin=b.qmin, qmax=b.qmax, topk=2, **res.best.plan_kwargs()) as p:
        pk1 = p.search(cis, spectrum=s1)
    np.testing.assert_allclose(s1, s0, rtol=1e-6, atol=0)
    for f in ("j", "i1", "k", "power"):
        assert np.array_equal(pk0[:, 0][f], pk1[:, 0][f]), f
    # the cache answers the next call; tuned_plan builds the plan from it
    assert at.tune(cis, 200, b.qmin, b.qmax, cache=cache).cached
    plan, r2 = at.tuned_plan(cis, 200, b.qmin, b.qmax, topk=2)
    with plan:
        pk2 = plan.search(cis)
    assert np.array_equal(pk2[:, 0]["j"], pk0[:, 0]["j"])


@pytest.mark.parametrize("kernel", ["ws", "one_group"])
def test_forced_kernel_choices_agree(kernel):
    b = synth.config2(ncurves=4, nf=1500, seed=22)
    cis = bls.curves_from_batch(b)
    nf = sum(ci.nf for ci in cis)
    s0, s1 = np.zeros(nf, np.float32), np.zeros(nf, np.float32)
    with bls.Plan(nb=200, qmin=b.qmin, qmax=b.qmax) as p:
        pk0 = p.search(cis, spectrum=s0)
    with bls.Plan(nb=200, qmin=b.qmin, qmax=b.qmax, fold_kernel=kernel) as p:
        pk1 = p.search(cis, spectrum=s1)
    np.testing.assert_allclose(s1, s0, rtol=1e-6, atol=0)
    assert np.array_equal(pk0["j"], pk1["j"])
    # a forced warp-specialised kernel on a class whose TMEM copy does not fit still
    # sweeps correctly (from shared memory)
    if kernel == "ws":
        for ci in cis:
            ci.nb = 300
        with bls.Plan(nb=300, qmin=b.qmin, qmax=0.1, freqs_per_block=64) as p:
            pa = p.search(cis, spectrum=s0)
        with bls.Plan(nb=300, qmin=b.qmin, qmax=0.1, freqs_per_block=64, fold_kernel="ws") as p:
            pb = p.search(cis, spectrum=s1)
        np.testing.assert_allclose(s1, s0, rtol=1e-6, atol=0)
        assert np.array_equal(pa["j"], pb["j"])
