"""Unbinned (edge-to-edge) BLS, CUDA path vs the oracle (marked gpu).

Both sides order points by the FP64 phase frac(RN(dt f)) (ties by index) and decide run
extents in FP64, so the order and the admissible runs are identical; the run sums are FP32
on the GPU's search and FP64 in the oracle, so SR per frequency must agree within the
search's tolerance, the best frequency and run must agree wherever the oracle's best is
separated, and the reported peak (refit in FP64 in run order) must then equal the
oracle's."""
import numpy as np
import pytest

import oracle
from paper_1112_1701_b300 import bls, build, synth
from tests.parity import separated_best, sr_tol

pytestmark = pytest.mark.gpu

QMIN, QMAX = 0.005, 0.15


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    bls.lib()


def _nf(ci):
    return len(ci.freqs) if ci.freqs is not None else ci.nf


def _run(cis, topk=1, sign="dips", qmin=QMIN, qmax=QMAX):
    with bls.Plan(nb=200, qmin=qmin, qmax=qmax, topk=topk, algo="unbinned", sign=sign) as p:
        spec = np.zeros(sum(_nf(ci) for ci in cis), np.float32)
        pk = p.search(cis, spectrum=spec)
    return pk, spec


def _check(ci, pk, sr_gpu, sign=0, qmin=QMIN, qmax=QMAX):
    kw = dict(freqs=ci.freqs) if ci.freqs is not None else dict(fmin=ci.fmin, df=ci.df, nf=ci.nf)
    P, opk = oracle.ubls(ci.t, ci.y, ci.dy, qmin, qmax, sign=sign, **kw)
    scal = oracle.prep(ci.t, ci.y, ci.dy)[3]
    sro = np.sqrt(P)
    tol = sr_tol(sro, scal[3])
    assert np.all(np.abs(sr_gpu.astype(np.float64) - sro) <= tol), \
        float(np.max(np.abs(sr_gpu - sro) - tol))
    jo, sep = separated_best(P, scal[3])
    if not sep:
        return False
    assert pk["j"] == opk.j
    if (pk["i1"], pk["k"]) != (opk.first, opk.len):
        return False            # an FP32 near-tie among runs of the same frequency
    for f in ("power", "depth", "sr", "snr"):
        assert pk[f] == pytest.approx(getattr(opk, f), rel=1e-9, abs=1e-15), f
    assert pk["epoch"] == pytest.approx(opk.epoch, abs=1e-9)
    assert pk["duration"] == pytest.approx(opk.duration, rel=1e-12)
    assert pk["freq"] == opk.freq
    return True


def test_batch_matches_oracle():
    b = synth.config2(ncurves=5, nf=400, seed=61)
    cis = bls.curves_from_batch(b)
    pk, spec = _run(cis)
    o = 0
    exact = 0
    for c, ci in enumerate(cis):
        exact += _check(ci, pk[c, 0], spec[o:o + _nf(ci)])
        o += _nf(ci)
    assert exact >= 2


def test_large_curve_both_signs_explicit_grid():
    """More than 4096 points (an 8192-entry sort) and both signs on an explicit grid."""
    rng = np.random.default_rng(5)
    n = 5000
    t = synth.T0 + np.sort(rng.uniform(0, 40, n))
    y = (1 + rng.normal(0, 0.01, n) - 0.02 * (np.mod(t - synth.T0, 1.3) < 0.08)).astype(np.float32)
    dy = np.full(n, 0.01, np.float32)
    freqs = np.sort(rng.uniform(0.3, 1.5, 60))
    freqs[10] = 1 / 1.3
    ci = bls.CurveInput(t, y, dy, freqs=freqs, nb=200, qmin=QMIN, qmax=QMAX)
    for sign, s in (("dips", 0), ("both", 1)):
        pk, spec = _run([ci], sign=sign)
        _check(ci, pk[0, 0], spec, sign=s)
        assert pk[0, 0]["j"] == 10


def test_equal_phases_and_extents_on_the_bounds():
    """Times on a 2^-7-day lattice, shuffled (inputs need not be sorted): at f = 1 and 0.5
    many phases are exactly equal (order by index) and many run extents equal qmin or qmax
    exactly (both bounds admit); at f = 1 +- 2^-40 phases differ by less than 2^-32 of a
    cycle, so equal 32-bit keys must be put in phase order, and at 1 - 2^-40 integer times
    fold to just below phase 1 (a wrap).  The GPU's order and bounds are the oracle's."""
    rng = np.random.default_rng(77)
    n = 700
    dt = rng.integers(0, 40 * 128, n).astype(np.float64) / 128.0
    dt[rng.choice(n, 60, replace=False)] = 7.0                 # repeated times
    t = synth.T0 + dt
    y = (1 + rng.normal(0, 0.01, n) - 0.02 * (np.mod(dt, 1.0) < 0.125)).astype(np.float32)
    dy = rng.uniform(0.008, 0.012, n).astype(np.float32)
    freqs = np.array([1.0, 1.0 + 2.0 ** -40, 1.0 - 2.0 ** -40, 0.5, 2.0, 0.75])
    qmin, qmax = 2.0 ** -6, 0.125
    ci = bls.CurveInput(t, y, dy, freqs=freqs, nb=100, qmin=qmin, qmax=qmax)
    for sign, sg in (("dips", 0), ("both", 1)):
        pk, spec = _run([ci], sign=sign, qmin=qmin, qmax=qmax)
        _check(ci, pk[0, 0], spec, sign=sg, qmin=qmin, qmax=qmax)
    # each frequency alone: the GPU's best run (a position range of its phase order) read
    # in the oracle's order must be admissible, within tolerance of the best power, and
    # carry the oracle's FP64 extent exactly (duration = E / f)
    d, w, x, scal = oracle.prep(t, y, dy)
    for f in freqs:
        one = bls.CurveInput(t, y, dy, freqs=np.array([f]), nb=100, qmin=qmin, qmax=qmax)
        pk, spec = _run([one], qmin=qmin, qmax=qmax)
        Pb, *_ = oracle.ubls_power(d, w, x, f, qmin, qmax)
        phi = oracle.ubls_phases(d, f)
        order = oracle.ubls_order(phi)
        i1, k = int(pk[0, 0]["i1"]), int(pk[0, 0]["k"])
        assert 1 <= k <= n - 1
        E = oracle.ubls_extent(phi, order, i1, k)
        assert qmin <= E <= qmax
        assert pk[0, 0]["duration"] == E / f
        run = order[(i1 + np.arange(k)) % n]
        r, sx = float(np.sum(w[run])), float(np.sum(w[run] * x[run]))
        Prun = sx * sx / (r * (1 - r))
        assert sx < 0
        tol = sr_tol(np.sqrt(Pb), scal[3])
        assert np.sqrt(Prun) >= np.sqrt(Pb) - 2 * tol
        assert pk[0, 0]["power"] == pytest.approx(Prun, rel=1e-9)


def test_tiny_and_edge_cases():
    t = synth.T0 + np.array([0.0, 0.3, 1.1])
    y = np.array([1.0, 0.9, 1.0], np.float32)
    ci = bls.CurveInput(t, y, None, nf=7, fmin=0.2, df=0.1, nb=10, qmin=0.001, qmax=0.5)
    pk, spec = _run([ci], qmin=0.001, qmax=0.5)
    _check(ci, pk[0, 0], spec, qmin=0.001, qmax=0.5)
    flat = bls.CurveInput(t, np.ones(3, np.float32), None, nf=4, fmin=0.2, df=0.1, nb=10,
                          qmin=0.001, qmax=0.5)
    pk, spec = _run([flat], qmin=0.001, qmax=0.5)
    assert np.all(spec == 0) and pk[0, 0]["power"] == 0.0


def test_long_curves_in_global_scratch():
    """Curves above the shared-memory size (a 20,000-point curve, the serving workload's
    longest, searched together with a 3000-point one): the working arrays live in a global
    scratch slice per persistent block; the search is the oracle's, as for short curves."""
    rng = np.random.default_rng(21)
    cis = []
    for n, P0 in ((20000, 1.7), (3000, 0.9)):
        t = synth.T0 + np.sort(rng.uniform(0, 60, n))
        y = (1 + rng.normal(0, 0.01, n)
             - 0.015 * (np.mod(t - synth.T0 - 0.2, P0) < 0.06)).astype(np.float32)
        dy = rng.uniform(0.008, 0.012, n).astype(np.float32)
        freqs = np.sort(np.concatenate([rng.uniform(0.3, 2.0, 23), [1 / P0]]))
        cis.append(bls.CurveInput(t, y, dy, freqs=freqs, nb=200, qmin=0.005, qmax=0.05))
    for sign, sg in (("dips", 0), ("both", 1)):
        pk, spec = _run(cis, sign=sign, qmin=0.005, qmax=0.05)
        o = 0
        for c, ci in enumerate(cis):
            _check(ci, pk[c, 0], spec[o:o + 24], sign=sg, qmin=0.005, qmax=0.05)
            o += 24


def test_limits_and_unsupported():
    rng = np.random.default_rng(1)
    n = 40000
    t = synth.T0 + np.sort(rng.uniform(0, 10, n))
    ci = bls.CurveInput(t, np.ones(n, np.float32), None, nf=3, fmin=0.5, df=0.1, nb=50,
                        qmin=QMIN, qmax=QMAX)
    with pytest.raises(bls.BLSError):
        _run([ci])
    b = synth.config1()
    c, g = b.curves[0], b.grids[0]
    ci = bls.CurveInput(c.t, c.y, c.dy, nf=50, fmin=g.fmin, df=g.df, nb=100, qmin=b.qmin,
                        qmax=b.qmax)
    with bls.Plan(nb=100, qmin=b.qmin, qmax=b.qmax, algo="unbinned") as p:
        with pytest.raises(bls.BLSError):
            p.search_shapes([ci])
