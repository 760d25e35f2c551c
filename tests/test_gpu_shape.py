"""Trapezoid refit of the peaks (bls_search_shapes), CUDA path vs the FP64 oracle (marked
gpu).  The grid search runs in FP32 on the GPU and FP64 in the oracle: the GPU's pick must
have an oracle power within the residue tolerance of the oracle's best, identical picks
must give identical records (the GPU refits its pick in FP64), and an exact noiseless
trapezoid must be found exactly."""
import numpy as np
import pytest

import oracle
from paper_1112_1701_b300 import bls, build, synth
from tests.parity import sr_tol

pytestmark = pytest.mark.gpu

GRID = dict(nc=17, nw=13, na=6, wlo=0.5, whi=2.0, amax=0.5)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    bls.lib()


def _check(sh, pk, c, nb):
    dt, w, x, scal = oracle.prep(c.t, c.y, c.dy)
    fit, Q = oracle.shape(dt, w, x, float(pk["freq"]), nb, int(pk["i1"]), int(pk["k"]),
                          want_grid=True, **GRID)
    sq = np.sqrt(Q)
    for idx, power, best in ((sh["index"], sh["power"], fit.index),
                             (sh["box_index"], sh["box_power"],
                              int(np.argmax(np.where(np.arange(len(Q)) % GRID["na"] == 0, Q, -1))))):
        if best < 0 or Q[best] <= 0:
            assert idx == -1
            continue
        tol = 2 * sr_tol(sq[best], scal[3])
        assert sq[idx] >= sq[best] - tol, (idx, best)
        # the FP64 refit of the GPU's pick is the oracle's power at that grid point
        assert power == pytest.approx(Q[idx], rel=1e-9, abs=1e-15)
    if sh["index"] == fit.index >= 0:
        assert sh["depth"] == pytest.approx(fit.depth, rel=1e-9)
        assert sh["duration"] == pytest.approx(fit.width / pk["freq"], rel=1e-12)
        assert sh["ingress"] == pytest.approx(fit.ingress / pk["freq"], rel=1e-12, abs=1e-15)
        assert sh["epoch"] == pytest.approx(scal[0] + fit.centre / pk["freq"], abs=1e-9)
        return True
    return False


def test_shapes_match_oracle_on_batch():
    b = synth.config2(ncurves=8, nf=1200, seed=51)
    cis = bls.curves_from_batch(b)
    with bls.Plan(nb=200, qmin=b.qmin, qmax=b.qmax, topk=2) as p:
        pk, sh = p.search_shapes(cis)
        pk2 = p.search(cis)
    assert np.array_equal(pk, pk2)          # the refit does not touch the peaks
    same = 0
    for c in range(8):
        for q in range(2):
            if pk[c, q]["j"] < 0:
                assert sh[c, q]["index"] == -1
                continue
            same += _check(sh[c, q], pk[c, q], b.curves[c], 200)
    assert same >= 10


def test_noiseless_trapezoid_picks_equal_oracle():
    """Noiseless flat-bottomed eclipses with linear edges: no near-ties, so the GPU's grid
    pick must be the oracle's, with the same record, and the trapezoid must fit better than
    any box (power above box power, nonzero ingress)."""
    rng = np.random.default_rng(17)
    n, nb = 3000, 100
    t = synth.T0 + np.sort(rng.uniform(0, 45, n))
    curves, cis = [], []
    for P, c0, T, tau, depth in ((0.83, 0.33, 0.06, 0.012, 0.04), (2.1, 0.7, 0.045, 0.015, 0.02),
                                 (0.41, 0.05, 0.09, 0.02, 0.1)):
        f0 = 1.0 / P
        dt = t - t[0]
        phi = dt * f0 - np.floor(dt * f0)
        D = (phi - c0 + 0.5) % 1.0 - 0.5
        s = np.clip((T / 2 - np.abs(D)) / tau, 0, 1)
        y = (1.0 - depth * s).astype(np.float32)
        dy = np.full(n, 0.01, np.float32)
        curves.append(synth.Curve(t, y, dy))
        cis.append(bls.CurveInput(t, y, dy, freqs=np.array([f0 * 0.999, f0, f0 * 1.001]),
                                  nb=nb, qmin=0.01, qmax=0.2))
    with bls.Plan(nb=nb, qmin=0.01, qmax=0.2, topk=1) as p:
        pk, sh = p.search_shapes(cis)
    for c in range(3):
        assert pk[c, 0]["j"] == 1
        assert _check(sh[c, 0], pk[c, 0], curves[c], nb)
        assert sh[c, 0]["ingress"] > 0 and sh[c, 0]["power"] > sh[c, 0]["box_power"]


def test_grid_options_and_errors():
    b = synth.config1()
    c, g = b.curves[0], b.grids[0]
    ci = bls.CurveInput(c.t, c.y, c.dy, nf=g.nf, fmin=g.fmin, df=g.df, nb=100, qmin=b.qmin,
                        qmax=b.qmax)
    with bls.Plan(nb=100, qmin=b.qmin, qmax=b.qmax, topk=1) as p:
        pk, sh = p.search_shapes([ci], ncentre=1, nwidth=1, ningress=1, width_lo=1.0,
                                 width_hi=1.0)
        # one grid point: the box itself, whose power is the peak's BLS power
        assert sh[0, 0]["index"] == 0 and sh[0, 0]["box_index"] == 0
        assert sh[0, 0]["power"] == pytest.approx(pk[0, 0]["power"], rel=1e-9)
        for bad in (dict(ncentre=-1), dict(width_lo=2.0, width_hi=1.0), dict(ingress_max=0.7)):
            with pytest.raises(bls.BLSError):
                p.search_shapes([ci], **bad)
