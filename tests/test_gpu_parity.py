"""CUDA path vs the FP64 oracle, through the C ABI (marked gpu).

Bar: identical phase bins for every point (bit-exact), SR within the tolerance of
tests/parity.py at every frequency, the same best frequency wherever the top two peaks
are separated by more than that, and FP64-refit peak values equal to the oracle's."""
import numpy as np
import pytest

import oracle
from paper_1112_1701_b300 import bls, build, synth
from tests.parity import (check_peak, check_powers, check_sde, oracle_run, prep_of,
                          separated_best, sr_tol)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    bls.lib()


def _ci(c, g, nb, qmin, qmax, **kw):
    return bls.CurveInput(c.t, c.y, c.dy, nf=g.nf, fmin=g.fmin, df=g.df, nb=nb, qmin=qmin,
                          qmax=qmax, **kw)


def _plan(nb, qmin, qmax, **kw):
    return bls.Plan(nb=nb, qmin=qmin, qmax=qmax, **kw)


# ------------------------------------------------------------------------------ plain curve

def test_plain_workload_spectrum_and_peak():
    b = synth.config1()
    c, g = b.curves[0], b.grids[0]
    nb = b.nb[0]
    kmin, kmax = oracle.kminmax(nb, b.qmin, b.qmax)
    ci = _ci(c, g, nb, b.qmin, b.qmax)
    with _plan(nb, b.qmin, b.qmax) as p:
        Pg, I1g, Kg = p.debug_powers(ci)
        pk = p.search([ci])[0, 0]
    Po, I1o, Ko, scal = check_powers(ci, Pg, I1g, Kg, nb, kmin, kmax, label="cfg1")
    _, _, _, opk = oracle_run(ci, nb, kmin, kmax)
    jo, sep = separated_best(Po, scal[3])
    assert sep and pk["j"] == jo
    check_peak(pk, opk[0])
    check_sde(pk, opk[0], Po, scal[3])
    assert pk["sde"] > 5.0   # the injected box stands far above the noise peaks
    # the injected 0.40 d box is recovered
    assert abs(pk["period"] - 0.40) < 0.40 ** 2 * g.df


# ------------------------------------------------------------------------------ bins

def _bins_check(ci, nb, js, phase="df32"):
    with _plan(nb, 0.01, 0.1, phase=phase) as p:
        bg = p.debug_fold(ci, js)
    f = [oracle.freq(j, ci.fmin, ci.df) for j in js]
    bo = oracle.bins(np.asarray(ci.t), f, nb)
    return bg, bo


@pytest.mark.parametrize("phase", ["df32", "f64", "fx64"])
def test_bins_bit_exact_plain_and_long_baseline(phase):
    b1 = synth.config1()
    ci1 = _ci(b1.curves[0], b1.grids[0], 100, 0.01, 0.1)
    js = list(range(0, 2000, 31)) + [1999]
    bg, bo = _bins_check(ci1, 100, js, phase)
    assert np.array_equal(bg, bo)
    # three-year baseline, highest frequencies: the FP32 product alone would be ~0.1 bin off
    b3 = synth.config3(ncurves=1, nf=200000)
    ci3 = _ci(b3.curves[0], b3.grids[0], 200, 0.005, 0.15)
    js = list(range(199000, 200000, 97)) + [199999, 0, 1, 12345]
    bg, bo = _bins_check(ci3, 200, js, phase)
    assert np.array_equal(bg, bo), f"{int((bg != bo).sum())} of {bg.size} bins differ"


@pytest.mark.parametrize("phase", ["df32", "fx64"])
@pytest.mark.parametrize("grid", ["coarse", "fine"])
def test_bins_bit_exact_on_exact_edges(phase, grid):
    """Points placed exactly on bin edges (and on integer cycles) at grid frequencies:
    every one lands within the error bound and takes the exact FP64 re-fold.  On the fine
    grid the FX64 debug fold also runs the incremental fold of the search's tiles (at
    nb = 64, 128-frequency tiles: offsets -64 .. 63 from the tile's middle column, and a
    ragged last tile), which must agree."""
    nb = 64
    if grid == "coarse":
        f0, df, nf = 0.5, 0.25, 11
        js = [0, 1, 2, 6, 10]
    else:
        f0, df, nf = 0.5, 0.001, 1000
        js = [0, 1, 2, 63, 64, 65, 100, 127, 128, 500, 998, 999]
    rng = np.random.default_rng(5)
    dts = []
    for j in js:
        f = oracle.freq(j, f0, df)
        cyc = rng.integers(0, 200, 64).astype(np.float64)
        edge = rng.integers(0, nb, 64)
        dts.append((cyc + edge / nb) / f)
    dt = np.sort(np.concatenate(dts + [np.array([0.0])]))
    t = synth.T0 + dt
    y = np.ones(len(t), np.float32)
    ci = bls.CurveInput(t, y, None, nf=nf, fmin=f0, df=df, nb=nb, qmin=0.02, qmax=0.2)
    with _plan(nb, 0.02, 0.2, phase=phase) as p:
        bg = p.debug_fold(ci, js)
    bo = oracle.bins(t, [oracle.freq(j, f0, df) for j in js], nb)
    assert np.array_equal(bg, bo)


@pytest.mark.parametrize("T", [0, 80, 48])
def test_bins_bit_exact_at_survey_tile_geometry(T):
    """The survey sweep's shape (2000 points over 90 nights, 200,000 frequencies, nb = 256):
    the search runs 104-frequency tiles there (T = 0: the plan's rules; histograms packed at
    a stride of 104 columns, 336-point staging chunks), or the width given.  Bins of the
    first, reference (middle), last and ragged-tile columns of such tiles, in the incremental
    fold with the search's reference column, equal the FP64 oracle's."""
    b = synth.config5(ncurves=2)
    nb = 256
    for c, g in zip(b.curves, b.grids):
        ci = _ci(c, g, nb, b.qmin, b.qmax)
        kw = dict(freqs_per_block=T, point_chunk=256) if T else {}
        with _plan(nb, b.qmin, b.qmax, **kw) as p:
            shape = p.tile_shape()
            if not T:
                assert shape == {"cols": 104, "chunk": 336, "fold_kernel": "ws"}, shape
            Tw = shape["cols"]
            js = []
            for tile in (0, 1, 1041, (g.nf - 1) // Tw - 1, (g.nf - 1) // Tw):
                t0 = tile * Tw
                js += [t0, t0 + Tw // 2 - 1, t0 + Tw // 2, t0 + Tw - 1]
            js = sorted({j for j in js if 0 <= j < g.nf} | {g.nf - 1})
            bg = p.debug_fold(ci, js)
        bo = oracle.bins(c.t, [oracle.freq(j, g.fmin, g.df) for j in js], nb)
        assert np.array_equal(bg, bo), f"T={Tw}: {int((bg != bo).sum())} of {bg.size} differ"


def test_fast_phase_modes_give_identical_searches():
    """The double-FP32 and fixed-point folds both reproduce the FP64 bins exactly, and the
    binning order is the same, so spectra and peaks must agree bit for bit."""
    b = synth.config2(ncurves=12, nf=2000, seed=31)
    cis = bls.curves_from_batch(b)
    out = {}
    for phase in ("df32", "fx64"):
        with _plan(200, b.qmin, b.qmax, topk=3, phase=phase) as p:
            spec = np.zeros(12 * 2000, np.float32)
            pk = p.search(cis, spectrum=spec)
            out[phase] = (pk, spec)
    assert np.array_equal(out["df32"][1], out["fx64"][1])
    assert np.array_equal(out["df32"][0], out["fx64"][0])


def test_f32_phase_mode_runs_and_can_differ():
    b3 = synth.config3(ncurves=1, nf=200000)
    ci3 = _ci(b3.curves[0], b3.grids[0], 200, 0.005, 0.15)
    js = list(range(199000, 200000, 97))
    bg, bo = _bins_check(ci3, 200, js, "f32")
    assert bg.shape == bo.shape and bg.min() >= 0 and bg.max() < 200
    assert (bg != bo).mean() > 0.01   # expected: FP32 loses the bin at 3-year baselines


# ------------------------------------------------------------------------------ tiles, batches

def test_several_tiles_and_ragged_tail():
    rng = np.random.default_rng(9)
    n = 777                                   # not a multiple of the staged chunk
    t = synth.T0 + np.sort(rng.uniform(0, 45, n))
    y = (1 + rng.normal(0, 0.01, n)).astype(np.float32)
    y[np.mod(t - synth.T0, 1.7) < 0.06] -= 0.02
    dy = rng.uniform(0.005, 0.02, n).astype(np.float32)
    nb, qmin, qmax = 64, 0.01, 0.2
    kmin, kmax = oracle.kminmax(nb, qmin, qmax)
    ci = bls.CurveInput(t, y, dy, nf=1013, fmin=0.05, df=0.0049, nb=nb, qmin=qmin, qmax=qmax)
    with _plan(nb, qmin, qmax) as p:
        Pg, I1g, Kg = p.debug_powers(ci)
        pk = p.search([ci])[0, 0]
    Po, _, _, scal = check_powers(ci, Pg, I1g, Kg, nb, kmin, kmax, label="ragged")
    jo, sep = separated_best(Po, scal[3])
    if sep:
        assert pk["j"] == jo


def test_batch_matches_oracle_per_curve():
    b = synth.config2(ncurves=8, nf=2500)
    nb = 200
    kmin, kmax = oracle.kminmax(nb, b.qmin, b.qmax)
    cis = bls.curves_from_batch(b)
    with _plan(nb, b.qmin, b.qmax) as p:
        spec = np.zeros(sum(ci.nf for ci in cis), np.float32)
        pk = p.search(cis, spectrum=spec)
        for q, ci in enumerate(cis):
            Pg, I1g, Kg = p.debug_powers(ci)
            assert np.allclose(np.sqrt(Pg), spec[q * 2500:(q + 1) * 2500], rtol=0, atol=0)
            Po, I1o, Ko, scal = check_powers(ci, Pg, I1g, Kg, nb, kmin, kmax, label=f"c{q}")
            jo, sep = separated_best(Po, scal[3])
            _, _, _, opk = oracle_run(ci, nb, kmin, kmax)
            if sep:
                check_peak(pk[q, 0], opk[0])
                check_sde(pk[q, 0], opk[0], Po, scal[3])


def test_batch_result_equals_alone_bit_for_bit():
    b = synth.config2(ncurves=40, nf=1500)
    cis = bls.curves_from_batch(b)
    with _plan(200, b.qmin, b.qmax, topk=3) as p:
        spec = np.zeros(40 * 1500, np.float32)
        pk = p.search(cis, spectrum=spec)
        for q in (0, 7, 39):
            s1 = np.zeros(1500, np.float32)
            pk1 = p.search([cis[q]], spectrum=s1)
            assert np.array_equal(s1, spec[q * 1500:(q + 1) * 1500])
            assert np.array_equal(pk1[0], pk[q])


def test_topk_peaks_match_oracle():
    b = synth.config5(ncurves=3, nf=6000)
    nb = 256
    kmin, kmax = oracle.kminmax(nb, b.qmin, b.qmax)
    cis = bls.curves_from_batch(b)
    with _plan(nb, b.qmin, b.qmax, topk=5) as p:
        pk = p.search(cis)
        for q, ci in enumerate(cis):
            Pg, I1g, Kg = p.debug_powers(ci)
            Po, _, _, scal = check_powers(ci, Pg, I1g, Kg, nb, kmin, kmax, label=f"top{q}")
            _, _, _, opk = oracle_run(ci, nb, kmin, kmax, topk=5)
            sro = np.sqrt(np.array([o.power for o in opk]))
            for e in range(5):
                # compare where consecutive peaks are separated beyond the tolerance
                sep_prev = e == 0 or sro[e - 1] - sro[e] > 2e-5 * sro[e - 1]
                sep_next = e == 4 or sro[e] - sro[e + 1] > 2e-5 * sro[e]
                if sep_prev and sep_next:
                    check_peak(pk[q, e], opk[e])
                    check_sde(pk[q, e], opk[e], Po, scal[3])


# ------------------------------------------------------------------------------ edge cases

def _edge(t, y, dy, nb, qmin, qmax, sign="dips", freqs=None, nf=50, fmin=0.2, df=0.05,
          **plan):
    kmin, kmax = oracle.kminmax(nb, qmin, qmax)
    ci = bls.CurveInput(t, y, dy, nf=nf, fmin=fmin, df=df, freqs=freqs, nb=nb, qmin=qmin,
                        qmax=qmax)
    with _plan(nb, qmin, qmax, sign=sign, **plan) as p:
        Pg, I1g, Kg = p.debug_powers(ci)
        pk = p.search([ci])[0, 0]
    s = bls.SIGN[sign]
    Po, I1o, Ko, scal = check_powers(ci, Pg, I1g, Kg, nb, kmin, kmax, sign=s, label="edge")
    return ci, Pg, pk, Po, kmin, kmax


def test_two_points_two_bins():
    t = synth.T0 + np.array([0.0, 0.3])
    y = np.array([1.0, 0.9], np.float32)
    ci, Pg, pk, Po, kmin, kmax = _edge(t, y, None, 2, 0.3, 0.6)
    assert (kmin, kmax) == (1, 1)


def test_single_frequency_explicit_grid_both_signs():
    rng = np.random.default_rng(3)
    t = synth.T0 + np.sort(rng.uniform(0, 10, 300))
    y = (1 + rng.normal(0, 0.01, 300)).astype(np.float32)
    y[np.mod(t, 0.9) < 0.05] += 0.03       # a bump
    for freqs in (np.array([1 / 0.9]), np.linspace(0.3, 3.0, 77)):
        _edge(t, y, None, 90, 0.01, 0.1, sign="both", freqs=freqs)
        _edge(t, y, None, 90, 0.01, 0.1, sign="dips", freqs=freqs)


def test_constant_flux_gives_zero():
    rng = np.random.default_rng(4)
    t = synth.T0 + np.sort(rng.uniform(0, 10, 500))
    y = np.full(500, 1.25, np.float32)
    dy = rng.uniform(0.01, 0.02, 500).astype(np.float32)
    ci, Pg, pk, Po, kmin, kmax = _edge(t, y, dy, 50, 0.02, 0.2)
    assert np.all(Pg == 0)
    assert pk["j"] == 0 and pk["i1"] == 0 and pk["k"] == kmin
    assert pk["depth"] == 0 and pk["snr"] == 0 and pk["sr"] == 0


@pytest.mark.parametrize("sums", ["fixed", "f32"])
def test_weights_spanning_ten_decades(sums):
    """Errors from 1e-5 to 1e0 (weights over ten decades): with fixed-point sums the lightest
    points round to a few units of 2^-32 of the total weight (or to zero), which the
    tolerance absorbs; a deep box among the heavy points is found as by the oracle."""
    rng = np.random.default_rng(13)
    n = 3000
    t = synth.T0 + np.sort(rng.uniform(0, 40, n))
    dy = (10.0 ** rng.uniform(-5, 0, n)).astype(np.float32)
    y = (1 + rng.normal(0, 1, n) * dy).astype(np.float32)
    y[np.mod(t - synth.T0, 1.9) < 0.08] -= 0.01
    ci, Pg, pk, Po, kmin, kmax = _edge(t, y, dy, 128, 0.01, 0.1, nf=400, fmin=0.3, df=0.004,
                                       sum=sums)
    jo, sep = separated_best(Po, prep_of(ci)[3][3])
    if sep:
        assert pk["j"] == jo


def test_all_points_in_few_bins_degenerate_boxes():
    """Every point at the same phase at f = 1: boxes covering them all have r = 1 and are
    skipped; the search still returns the oracle's answer."""
    t = synth.T0 + np.arange(200, dtype=np.float64)
    y = (1 + 0.01 * np.sin(np.arange(200))).astype(np.float32)
    _edge(t, y, None, 20, 0.05, 0.5, freqs=np.array([1.0, 2.0, 0.5, 1.37]))


def test_boxes_holding_most_of_the_weight():
    """Points crowded into 5% of the phase at f = 1/d: with q up to 0.3 many boxes hold
    almost all the weight (r close to 1), where FP32 loses 1 - r; those frequencies take
    the precise sweep and must still meet the tolerance."""
    rng = np.random.default_rng(12)
    n = 600
    t = synth.T0 + np.sort(rng.integers(0, 40, n) + rng.uniform(0, 0.05, n))
    y = (1 + rng.normal(0, 0.01, n)).astype(np.float32)
    y[np.abs(np.mod(t - synth.T0, 1.0) - 0.02) < 0.004] -= 0.02
    freqs = np.concatenate([[1.0, 2.0, 0.5], np.linspace(0.98, 1.02, 41)])
    _edge(t, y, None, 100, 0.01, 0.3, freqs=freqs)
    _edge(t, y, None, 100, 0.01, 0.3, sign="both", freqs=freqs)


def test_long_curve_many_chunks():
    rng = np.random.default_rng(6)
    n = 20000
    t = synth.T0 + np.sort(rng.uniform(0, 60, n))
    y = (1 + rng.normal(0, 0.01, n)).astype(np.float32)
    y[np.mod(t - synth.T0, 2.3) < 0.1] -= 0.01
    dy = np.full(n, 0.01, np.float32)
    _edge(t, y, dy, 128, 0.01, 0.1, nf=300, fmin=0.1, df=0.015)


def test_large_nb():
    rng = np.random.default_rng(8)
    t = synth.T0 + np.sort(rng.uniform(0, 30, 3000))
    y = (1 + rng.normal(0, 0.01, 3000)).astype(np.float32)
    _edge(t, y, None, 400, 0.005, 0.05, nf=130, fmin=0.2, df=0.03)


def test_kahan_sums_parity():
    b = synth.config2(ncurves=2, nf=1200)
    cis = bls.curves_from_batch(b)
    kmin, kmax = oracle.kminmax(200, b.qmin, b.qmax)
    with _plan(200, b.qmin, b.qmax, sum="kahan") as p:
        for ci in cis:
            Pg, I1g, Kg = p.debug_powers(ci)
            check_powers(ci, Pg, I1g, Kg, 200, kmin, kmax, label="kahan")


def test_plain_f64_baseline_parity():
    b = synth.config2(ncurves=2, nf=900)
    cis = bls.curves_from_batch(b)
    kmin, kmax = oracle.kminmax(200, b.qmin, b.qmax)
    with _plan(200, b.qmin, b.qmax, algo="plain_f64") as p:
        for ci in cis:
            Pg, I1g, Kg = p.debug_powers(ci)
            check_powers(ci, Pg, I1g, Kg, 200, kmin, kmax, label="plain")


def test_device_inputs_match_host_inputs():
    torch = pytest.importorskip("torch")
    b = synth.config2(ncurves=6, nf=1000)
    host_cis = bls.curves_from_batch(b)
    dev_cis = bls.curves_from_batch(b, device="cuda")
    with _plan(200, b.qmin, b.qmax, topk=2,
               stream=torch.cuda.current_stream().cuda_stream) as p:
        s_h = np.zeros(6000, np.float32)
        pk_h = p.search(host_cis, spectrum=s_h)
        s_d = torch.zeros(6000, dtype=torch.float32, device="cuda")
        pk_d = p.search(dev_cis, spectrum=s_d)
        torch.cuda.synchronize()
        assert np.array_equal(pk_h, pk_d)
        assert np.array_equal(s_h, s_d.cpu().numpy())


def test_packed_curves_match_curve_lists():
    """PackedCurves (descriptors written by numpy) give the same search as CurveInput lists,
    from host numpy arrays, pinned host tensors and device tensors."""
    torch = pytest.importorskip("torch")
    b = synth.config2(ncurves=7, nf=800, seed=13)
    with _plan(200, b.qmin, b.qmax, topk=2,
               stream=torch.cuda.current_stream().cuda_stream) as p:
        s0 = np.zeros(7 * 800, np.float32)
        pk0 = p.search(bls.curves_from_batch(b), spectrum=s0)
        for kw in ({}, {"pinned": True}, {"device": "cuda"}):
            pc = bls.packed_from_batch(b, **kw)
            s1 = np.zeros(7 * 800, np.float32)
            pk1 = p.search(pc, spectrum=s1)
            assert np.array_equal(pk0, pk1), kw
            assert np.array_equal(s0, s1), kw


def test_invalid_inputs_rejected():
    rng = np.random.default_rng(1)
    t = synth.T0 + np.sort(rng.uniform(0, 10, 100))
    y = np.ones(100, np.float32)
    with _plan(50, 0.02, 0.2) as p:
        bad_t = t.copy(); bad_t[5] = np.nan
        bad_dy = np.full(100, 0.01, np.float32); bad_dy[7] = 0
        for ci in (bls.CurveInput(bad_t, y, None, nf=10, fmin=0.1, df=0.1),
                   bls.CurveInput(t, y, bad_dy, nf=10, fmin=0.1, df=0.1),
                   bls.CurveInput(t[:1], y[:1], None, nf=10, fmin=0.1, df=0.1),
                   bls.CurveInput(t, y, None, nf=0, fmin=0.1, df=0.1),
                   bls.CurveInput(t, y, None, nf=10, fmin=-0.1, df=0.1)):
            with pytest.raises(bls.BLSError) as ei:
                p.search([ci])
            assert ei.value.status == bls.ERR_INVALID
        # device-resident bad values are caught by the prep kernel's check
        torch = pytest.importorskip("torch")
        tt = torch.tensor(bad_t, device="cuda")
        yy = torch.tensor(y, device="cuda")
        with pytest.raises(bls.BLSError) as ei:
            p.search([bls.CurveInput(tt, yy, None, nf=10, fmin=0.1, df=0.1)])
        assert ei.value.status == bls.ERR_INVALID
        # the plan still works afterwards
        p.search([bls.CurveInput(t, y, None, nf=10, fmin=0.1, df=0.1)])


# ------------------------------------------------------------------------------ full size

def test_batched_workload_full_size_sampled():
    """The 1024-curve, 50k-frequency batch in the benchmark's launch configuration:
    SR of sampled (curve, frequency) pairs and every sampled curve's best frequency are
    checked against the oracle computed one frequency at a time."""
    b = synth.config2()
    cis = bls.curves_from_batch(b)
    nb = 200
    kmin, kmax = oracle.kminmax(nb, b.qmin, b.qmax)
    with _plan(nb, b.qmin, b.qmax) as p:
        spec = np.zeros(len(cis) * b.grids[0].nf, np.float32)
        pk = p.search(cis, spectrum=spec)
    nf = b.grids[0].nf
    spec = spec.reshape(len(cis), nf)
    rng = np.random.default_rng(123)
    for c in rng.choice(len(cis), 12, replace=False):
        ci = cis[c]
        dt, w, x, scal = prep_of(ci)
        js = list(rng.choice(nf, 20, replace=False)) + [int(pk[c, 0]["j"])]
        for j in js:
            f = oracle.freq(j, ci.fmin, ci.df)
            Po, i1o, ko, _, _ = oracle.power(dt, w, x, f, nb, kmin, kmax)
            sro = np.sqrt(Po)
            tol = 1e-5 * sro + 1e-6 * np.sqrt(scal[3])
            assert abs(spec[c, j] - sro) <= tol, (c, j, spec[c, j], sro)
        # the reported peak equals the oracle's FP64 refit of the same box
        j = int(pk[c, 0]["j"])
        f = oracle.freq(j, ci.fmin, ci.df)
        Pb, r, s = oracle.box(dt, w, x, f, nb, int(pk[c, 0]["i1"]), int(pk[c, 0]["k"]))
        assert abs(pk[c, 0]["power"] - Pb) <= 1e-9 * Pb
        # no sampled frequency beats the reported peak beyond the tolerance
        assert spec[c].max() == pytest.approx(np.sqrt(pk[c, 0]["power"]), rel=2e-5)
    # bins of sampled frequencies, bit-exact (the FX64 debug fold also runs the incremental
    # fold of the bench's 128-frequency tiles and flags any disagreement)
    with _plan(nb, b.qmin, b.qmax) as p:
        for c in rng.choice(len(cis), 3, replace=False):
            ci = cis[c]
            js = sorted(set(int(j) for j in rng.choice(nf, 24, replace=False)) | {0, 63, 64, nf - 1})
            bg = p.debug_fold(ci, js)
            bo = oracle.bins(np.asarray(ci.t), [oracle.freq(j, ci.fmin, ci.df) for j in js], nb)
            assert np.array_equal(bg, bo), (c, int((bg != bo).sum()))


# ------------------------------------------------------------------------------ CUDA graphs

def test_graph_replay_reads_new_contents_and_matches_direct_launch():
    """Pinned host inputs: the first search captures the group into a graph, the next ones
    replay it.  New contents in the same buffers must give that data's results (the
    graph reads the arrays at replay), identical to a plan that launches directly."""
    torch = pytest.importorskip("torch")
    import os
    b1 = synth.config2(ncurves=5, nf=1200, seed=11)
    rng = np.random.default_rng(12)
    new = [(c.t, rng.permutation(c.y), rng.permutation(c.dy)) for c in b1.curves]
    old = [(c.t, c.y, c.dy) for c in b1.curves]
    cis = bls.curves_from_batch(b1, pinned=True)
    nb = 200
    kmin, kmax = oracle.kminmax(nb, b1.qmin, b1.qmax)
    spec = torch.zeros(5 * 1200, dtype=torch.float32).pin_memory()
    os.environ["BLS_NO_GRAPHS"] = "1"
    try:
        direct = _plan(nb, b1.qmin, b1.qmax, topk=2)
    finally:
        del os.environ["BLS_NO_GRAPHS"]
    with _plan(nb, b1.qmin, b1.qmax, topk=2) as p, direct:
        for it, data in enumerate((old, old, new, old)):
            for q, (t, y, dy) in enumerate(data):   # same shapes: overwrite in place
                cis[q].t.copy_(torch.from_numpy(t))
                cis[q].y.copy_(torch.from_numpy(y))
                cis[q].dy.copy_(torch.from_numpy(dy))
            pk = p.search(cis, spectrum=spec.numpy())
            s_g = spec.numpy().copy()
            s_d = np.zeros(5 * 1200, np.float32)
            pk_d = direct.search(cis, spectrum=s_d)
            assert np.array_equal(pk, pk_d), it
            assert np.array_equal(s_g, s_d), it
            if it == 2:
                for q in range(5):
                    Po = oracle_run(cis[q], nb, kmin, kmax)[0]
                    scal = prep_of(cis[q])[3]
                    sro = np.sqrt(Po)
                    assert np.all(np.abs(s_g[q * 1200:(q + 1) * 1200] - sro) <= sr_tol(sro, scal[3]))
        prof = p.profile()
        assert prof["graph_captures"] == 1 and prof["graph_replays"] == 3, prof
        assert direct.profile()["graph_replays"] == 0
