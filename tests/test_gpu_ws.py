"""The warp-specialised fold-sweep kernel (marked gpu).

Tiles of any multiple of 8 frequencies up to 128 (histograms strided at the width itself)
run in the warp-specialised kernel (a
binning warp group and a sweep warp group that takes each tile's histograms over through
TMEM; T/4 columns per SM sub-partition, two sweep threads per column); BLS_FOLD_WS=0 or
fold_kernel="one_group" select the one-group kernel.  Checked here:
  * the search's spectrum (SR of the kernel's per-frequency powers) against the oracle
    within the parity tolerance, over several tiles with a ragged tail, for TMEM copies with
    repeated bins and with wrapped reads, seeded sweeps (kmin > 1), tiles swept from shared
    memory by the sweep group (nb > 256) and the exact sweep;
  * identical spectra and peaks for every warp-specialised tile width (the per-frequency
    arithmetic does not depend on the tile);
  * the one-group kernel (run in a child process with BLS_FOLD_WS=0) within FP32 rounding
    of the same spectrum, with the same peaks.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1112_1701_b300 import bls, build, synth
from tests.parity import prep_of, sr_tol

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    bls.lib()


def _cases():
    """(name, curve inputs, nb, qmin, qmax) -- every curve of a case shares nb and q."""
    out = []
    b = synth.config2(ncurves=3, nf=700, seed=31)   # 700 = 5 x 128 + 60: a ragged tail
    out.append(("batch_nb200", [bls.CurveInput(c.t, c.y, c.dy, nf=g.nf, fmin=g.fmin, df=g.df,
                                               nb=200, qmin=b.qmin, qmax=b.qmax)
                                for c, g in zip(b.curves, b.grids)], 200, b.qmin, b.qmax))
    rng = np.random.default_rng(12)
    n = 400
    t = synth.T0 + np.sort(rng.integers(0, 40, n) + rng.uniform(0, 0.05, n))
    y = (1 + rng.normal(0, 0.01, n)).astype(np.float32)
    y[np.abs(np.mod(t - synth.T0, 1.0) - 0.02) < 0.004] -= 0.02
    freqs = np.concatenate([[1.0, 2.0, 0.5], np.linspace(0.98, 1.02, 150), np.linspace(0.1, 3, 150)])
    out.append(("crowded_exact_nb100", [bls.CurveInput(t, y, None, freqs=freqs, nb=100, qmin=0.01,
                                                       qmax=0.3)], 100, 0.01, 0.3))
    c = b.curves[0]
    out.append(("wrapped_tmem_nb240", [bls.CurveInput(c.t, c.y, c.dy, nf=300, fmin=0.2, df=0.01,
                                                      nb=240, qmin=0.005, qmax=0.1)], 240, 0.005, 0.1))
    out.append(("seeded_kmin3", [bls.CurveInput(c.t, c.y, c.dy, nf=300, fmin=0.2, df=0.01,
                                                nb=100, qmin=0.03, qmax=0.15)], 100, 0.03, 0.15))
    out.append(("shared_sweep_nb300", [bls.CurveInput(c.t, c.y, c.dy, nf=300, fmin=0.2, df=0.01,
                                                      nb=300, qmin=0.005, qmax=0.1)], 300, 0.005, 0.1))
    return out


def _search(cis, nb, qmin, qmax, T=0, sign="dips"):
    nf = sum(len(ci.freqs) if ci.freqs is not None else ci.nf for ci in cis)
    spec = np.zeros(nf, np.float32)
    # nb = 300 cannot take the TMEM copy: the plan asks for the warp-specialised kernel, whose
    # sweep group then sweeps from shared memory (the automatic choice would not take it)
    kern = "ws" if nb > 256 else "auto"
    with bls.Plan(nb=nb, qmin=qmin, qmax=qmax, topk=2, sign=sign, freqs_per_block=T,
                  fold_kernel=kern) as p:
        pk = p.search(cis, spectrum=spec)
    return spec, pk


def _oracle_check(cis, spec, nb, qmin, qmax, sign):
    kmin, kmax = oracle.kminmax(nb, qmin, qmax)
    o = 0
    for ci in cis:
        t, y = np.asarray(ci.t, np.float64), np.asarray(ci.y, np.float32)
        dy = None if ci.dy is None else np.asarray(ci.dy, np.float32)
        if ci.freqs is not None:
            P = oracle.bls(t, y, dy, nb, kmin, kmax, freqs=np.asarray(ci.freqs), sign=sign)[0]
        else:
            P = oracle.bls(t, y, dy, nb, kmin, kmax, fmin=ci.fmin, df=ci.df, nf=ci.nf, sign=sign)[0]
        scal = prep_of(ci)[3]
        sro = np.sqrt(P)
        srg = spec[o:o + len(P)].astype(np.float64)   # the spectrum holds SR = sqrt(P)
        bad = np.abs(srg - sro) > sr_tol(sro, scal[3])
        assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(srg - sro) - sr_tol(sro, scal[3]))))
        o += len(P)


@pytest.mark.parametrize("case", range(5))
@pytest.mark.parametrize("sign", ["dips", "both"])
def test_spectrum_matches_oracle_every_tile_width(case, sign):
    name, cis, nb, qmin, qmax = _cases()[case]
    ref = None
    for T in (128, 96, 64, 32, 48, 80, 112, 104, 120, 72, 24):   # 104 .. 24: packed strides
        try:
            spec, pk = _search(cis, nb, qmin, qmax, T=T, sign=sign)
        except bls.BLSError as e:   # T columns of nb bins exceed shared memory
            assert "shared memory" in str(e) and T > 64
            continue
        if ref is None:
            _oracle_check(cis, spec, nb, qmin, qmax, bls.SIGN[sign])
            ref = (spec, pk)
        else:   # warp-specialised at every width: identical to the first width run
            assert np.array_equal(spec, ref[0]), (name, T)
            for f in ("j", "i1", "k", "power"):
                assert np.array_equal(pk[f], ref[1][f]), (name, T, f)


_CHILD = r"""
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
from tests import test_gpu_ws as W
name, cis, nb, qmin, qmax = W._cases()[int(sys.argv[2])]
spec, pk = W._search(cis, nb, qmin, qmax, sign=sys.argv[3])
np.save(sys.argv[4], spec)
np.save(sys.argv[5], pk)
"""


@pytest.mark.parametrize("case", [0, 1])
def test_one_group_kernel_agrees(case, tmp_path):
    name, cis, nb, qmin, qmax = _cases()[case]
    spec, pk = _search(cis, nb, qmin, qmax)
    env = dict(os.environ, BLS_FOLD_WS="0")
    f1, f2 = str(tmp_path / "spec.npy"), str(tmp_path / "pk.npy")
    subprocess.run([sys.executable, "-c", _CHILD, ROOT, str(case), "dips", f1, f2], env=env,
                   check=True, timeout=600, cwd=ROOT)
    spec1, pk1 = np.load(f1), np.load(f2)
    np.testing.assert_allclose(spec, spec1, rtol=1e-6, atol=0)
    for f in ("j", "i1", "k", "power"):   # the best peak of each curve
        assert np.array_equal(pk[:, 0][f], pk1[:, 0][f]), (name, f)


def test_bounded_handover_wait_runs_out_and_plan_recovers(monkeypatch):
    """With the hand-over limit set to 1 microsecond (BLS_HANDOFF_LIMIT_US, a test setting
    read at every launch), a long curve's tile takes longer to bin than the sweep group
    waits: the wait runs out, the kernel records the timeout and both warp groups stop
    (nothing faults, no arrival is withheld), and the call fails with ERR_INTERNAL.  The
    next search on the same plan, with the limit back at its default, is correct: equal to
    a fresh plan's bit for bit."""
    rng = np.random.default_rng(12)
    n = 20000
    t = synth.T0 + np.sort(rng.uniform(0, 60, n))
    y = (1 + rng.normal(0, 0.01, n)).astype(np.float32)
    dy = np.full(n, 0.01, np.float32)
    ci = bls.CurveInput(t, y, dy, nf=1024, fmin=0.2, df=0.002, nb=200, qmin=0.005, qmax=0.15)
    spec = np.zeros(1024, np.float32)
    with bls.Plan(nb=200, qmin=0.005, qmax=0.15, topk=2) as p:
        monkeypatch.setenv("BLS_HANDOFF_LIMIT_US", "1")
        with pytest.raises(bls.BLSError) as ei:
            p.search([ci], spectrum=spec)
        assert ei.value.status == bls.ERR_INTERNAL and "bounded wait" in str(ei.value)
        monkeypatch.delenv("BLS_HANDOFF_LIMIT_US")
        pk = p.search([ci], spectrum=spec)
    spec2 = np.zeros(1024, np.float32)
    with bls.Plan(nb=200, qmin=0.005, qmax=0.15, topk=2) as p2:
        pk2 = p2.search([ci], spectrum=spec2)
    assert np.array_equal(spec, spec2)
    assert np.array_equal(pk, pk2)


@pytest.mark.parametrize("nb", [200, 256])
def test_kahan_sums_in_both_kernels(nb):
    """Kahan-compensated histograms (16-byte entries) in the warp-specialised kernel (the
    default for such plans) and in the one-group kernel: both within the parity tolerance
    of the oracle, and within FP32 rounding of each other (the warp-specialised kernel
    adds the pre-merged weights of points sharing a bin in one compensated addition)."""
    b = synth.config2(ncurves=3, nf=900, seed=44)
    cis = [bls.CurveInput(ci.t, ci.y, ci.dy, nf=ci.nf, fmin=ci.fmin, df=ci.df, nb=nb,
                          qmin=ci.qmin, qmax=ci.qmax) for ci in bls.curves_from_batch(b)]
    out = {}
    for kern in ("auto", "one_group"):
        spec = np.zeros(3 * 900, np.float32)
        with bls.Plan(nb=nb, qmin=b.qmin, qmax=b.qmax, topk=2, sum="kahan",
                      fold_kernel=kern) as p:
            pk = p.search(cis, spectrum=spec)
        _oracle_check(cis, spec, nb, b.qmin, b.qmax, 0)
        out[kern] = (spec, pk)
    np.testing.assert_allclose(out["auto"][0], out["one_group"][0], rtol=1e-6, atol=0)
    assert np.array_equal(out["auto"][1]["j"][:, 0], out["one_group"][1]["j"][:, 0])


@pytest.mark.parametrize("nb", [200, 256])
@pytest.mark.parametrize("sums", ["fixed", "f32"])
def test_fixed_and_f32_sums_in_both_kernels(sums, nb):
    """Fixed-point sums (the default: exact integer bin sums, converted to FP32 for the
    sweep) and plain FP32 sums, in the warp-specialised and the one-group kernel: both
    within the parity tolerance of the oracle.  With fixed-point sums the two kernels bin
    into identical integers, so their spectra differ only by the sweeps' approximations."""
    b = synth.config2(ncurves=3, nf=900, seed=45)
    cis = [bls.CurveInput(ci.t, ci.y, ci.dy, nf=ci.nf, fmin=ci.fmin, df=ci.df, nb=nb,
                          qmin=ci.qmin, qmax=ci.qmax) for ci in bls.curves_from_batch(b)]
    out = {}
    for kern in ("auto", "one_group"):
        spec = np.zeros(3 * 900, np.float32)
        with bls.Plan(nb=nb, qmin=b.qmin, qmax=b.qmax, topk=2, sum=sums,
                      fold_kernel=kern) as p:
            pk = p.search(cis, spectrum=spec)
            assert p.tile_shape()["fold_kernel"] == ("ws" if kern == "auto" else "one_group")
        _oracle_check(cis, spec, nb, b.qmin, b.qmax, 0)
        out[kern] = (spec, pk)
    np.testing.assert_allclose(out["auto"][0], out["one_group"][0], rtol=1e-6, atol=0)
    assert np.array_equal(out["auto"][1]["j"][:, 0], out["one_group"][1]["j"][:, 0])
