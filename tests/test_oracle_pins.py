"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

The paper (Sec. 2.2.2) uses the BLS of Kovacs et al. 2002 and prints no formula, no
worked example and no periodogram values, so the oracle is pinned by:
  * hand-derived cases (tests/golden/hand_cases.txt, working shown there);
  * brute force: every cyclic bin run fitted on the points by weighted least squares
    (numpy lstsq), chi2 computed directly, on tiny random inputs;
  * closed forms: constant flux gives zero power, a noise-free box on bin edges gives
    SR = depth*sqrt(r(1-r)) and the injected depth;
  * invariants: flux offset, error scale, P <= sum w x^2, cyclic wrap;
  * fold special cases: exact integer cycles land in bin 0, exact edges in the bin
    they open;
  * recovery of the injected 0.40 d box of the plain single-curve workload.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1112_1701_b300 import synth

T0 = synth.T0


# ----------------------------------------------------------------------------- helpers

def _run_case(c):
    t = T0 + np.array(c["t_offsets"])
    y = np.array(c["y"], dtype=np.float32)
    dy = np.array(c["dy"], dtype=np.float32)
    P, i1, k, pk = oracle.bls(t, y, dy, int(c["nb"]), int(c["kmin"]), int(c["kmax"]),
                              freqs=[c["f"]], sign=int(c["sign"]), topk=1)
    return t, y, dy, P, i1, k, pk[0]


def brute_force(t, y, dy, f, nb, kmin, kmax, sign):
    """Best box by explicit least squares on the points (no histogram, no box sums).

    For each cyclic run of k bins the two-level model (L inside, H outside) is fitted
    to the points with numpy.linalg.lstsq under weights dy^-2; the improvement over a
    constant model, sum w x^2 - chi2, is the BLS power of that box.  Dips only when
    sign == 0 (L < H)."""
    wraw = 1.0 / np.asarray(dy, np.float64) ** 2
    w = wraw / wraw.sum()
    yy = np.asarray(y, np.float64)
    ybar = (w * yy).sum()
    sw2 = (w * (yy - ybar) ** 2).sum()
    b = oracle.bins(t, [f], nb)[0]
    sq = np.sqrt(w)
    best, arg = 0.0, (0, kmin)
    table = []
    for i1 in range(nb):
        for k in range(kmin, kmax + 1):
            run = [(i1 + m) % nb for m in range(k)]
            inb = np.isin(b, run)
            r = w[inb].sum()
            if not (0.0 < r < 1.0) or inb.all() or not inb.any():
                continue
            A = np.stack([inb, ~inb], axis=1).astype(np.float64)
            coef, *_ = np.linalg.lstsq(A * sq[:, None], yy * sq, rcond=None)
            L, H = coef
            if sign == 0 and not (L < H):
                continue
            chi2 = (w * (yy - A @ coef) ** 2).sum()
            D = sw2 - chi2
            table.append(D)
            if D > best + 1e-14:
                best, arg = D, (i1, k)
    table.sort(reverse=True)
    gap = table[0] - table[1] if len(table) > 1 else np.inf
    return best, arg, sw2, gap


# ----------------------------------------------------------------------------- golden

@pytest.mark.parametrize("name", ["A", "B", "C", "C-dips", "D"])
def test_hand_cases(golden_cases, name):
    c = golden_cases[name]
    t, y, dy, P, i1, k, pk = _run_case(c)
    assert i1[0] == int(c["expect_i1"]) and k[0] == int(c["expect_k"])
    assert P[0] == pytest.approx(c["expect_P"], rel=1e-13, abs=1e-15)
    assert pk.j == 0
    assert pk.depth == pytest.approx(c["expect_depth"], rel=1e-12)
    assert pk.sr == pytest.approx(c["expect_sr"], rel=1e-12)
    assert pk.snr == pytest.approx(c["expect_snr"], rel=1e-12)
    assert pk.epoch - T0 == pytest.approx(c["expect_epoch_offset"], abs=1e-9)
    assert pk.duration == pytest.approx(c["expect_duration"], rel=1e-12)
    dt, w, x, scal = oracle.prep(t, y, dy)
    assert scal[3] == pytest.approx(c["expect_sumwx2"], rel=1e-12)
    if "expect_bins" in c:
        assert list(oracle.bins(t, [c["f"]], int(c["nb"]))[0]) == [int(v) for v in c["expect_bins"]]


# ----------------------------------------------------------------------------- brute force

@pytest.mark.parametrize("seed", range(40))
def test_bruteforce_chi2(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(3, 13))
    nb = int(rng.integers(2, 9))
    kmin = int(rng.integers(1, nb))
    kmax = int(rng.integers(kmin, nb))
    sign = int(seed % 2)
    t = T0 + np.sort(rng.uniform(0, 3.0, n))
    y = (1.0 + rng.normal(0, 0.1, n)).astype(np.float32)
    dy = rng.uniform(0.5, 2.0, n).astype(np.float32)
    freqs = rng.uniform(0.2, 4.0, 3)
    P, I1, K, _ = oracle.bls(t, y, dy, nb, kmin, kmax, freqs=freqs, sign=sign)
    for q, f in enumerate(freqs):
        best, arg, sw2, gap = brute_force(t, y, dy, f, nb, kmin, kmax, sign)
        assert P[q] == pytest.approx(best, abs=1e-12 * max(sw2, 1e-300))
        # chi2_min = sum w x^2 - P, non-negative
        assert sw2 - P[q] >= -1e-12 * sw2
        if gap > 1e-9 * sw2 and best > 0:
            assert (I1[q], K[q]) == arg


def test_box_power_matches_bruteforce_for_every_box():
    rng = np.random.default_rng(77)
    n, nb = 10, 6
    t = T0 + np.sort(rng.uniform(0, 3.0, n))
    y = (1.0 + rng.normal(0, 0.1, n)).astype(np.float32)
    dy = rng.uniform(0.5, 2.0, n).astype(np.float32)
    dt, w, x, scal = oracle.prep(t, y, dy)
    f = 1.37
    b = oracle.bins(t, [f], nb)[0]
    yy = y.astype(np.float64)
    for i1 in range(nb):
        for k in range(1, nb):
            P, r, s = oracle.box(dt, w, x, f, nb, i1, k, sign=1)
            inb = np.isin(b, [(i1 + m) % nb for m in range(k)])
            assert r == pytest.approx(w[inb].sum(), abs=1e-15)
            if 0 < r < 1:
                A = np.stack([inb, ~inb], axis=1).astype(np.float64)
                sq = np.sqrt(w)
                coef, *_ = np.linalg.lstsq(A * sq[:, None], yy * sq, rcond=None)
                chi2 = (w * (yy - A @ coef) ** 2).sum()
                assert P == pytest.approx(scal[3] - chi2, abs=1e-12)
    # the sweep's best box has the sweep's power
    Pbest, i1b, kb, _, _ = oracle.power(dt, w, x, f, nb, 1, nb - 1, sign=1)
    assert oracle.box(dt, w, x, f, nb, i1b, kb, sign=1)[0] == Pbest


# ----------------------------------------------------------------------------- closed forms

def test_constant_flux_zero_power():
    rng = np.random.default_rng(7)
    t = T0 + np.sort(rng.uniform(0, 20, 300))
    y = np.full(300, 1.2345, dtype=np.float32)
    dy = rng.uniform(0.01, 0.05, 300).astype(np.float32)
    kmin, kmax = oracle.kminmax(50, 0.01, 0.2)
    P, I1, K, pk = oracle.bls(t, y, dy, 50, kmin, kmax, fmin=0.1, df=0.01, nf=200, sign=1,
                              topk=3)
    assert np.all(P == 0.0)
    assert pk[0].j == 0 and pk[0].i1 == 0 and pk[0].k == kmin
    assert pk[0].depth == 0.0 and pk[0].snr == 0.0 and pk[0].sr == 0.0
    dt, w, x, scal = oracle.prep(t, y, dy)
    assert np.all(x == 0.0) and scal[3] == 0.0


@pytest.mark.parametrize("nb,i1,k", [(100, 10, 4), (64, 60, 8), (200, 0, 12)])
def test_noise_free_box_on_bin_edges(nb, i1, k):
    """Points strictly inside bins at f* = 2.5; a box exactly on bins [i1, i1+k) gives
    s = -depth r (1-r), hence SR = depth*sqrt(r(1-r)) and depth recovered exactly."""
    rng = np.random.default_rng(nb + i1)
    fstar, depth0 = 2.5, 0.03
    n = 400
    cycles = rng.integers(0, 40, n).astype(np.float64)
    b = rng.integers(0, nb, n)
    frac = rng.uniform(0.2, 0.8, n)           # stay away from bin edges
    dt = (cycles + (b + frac) / nb) / fstar
    order = np.argsort(dt)
    dt, b = dt[order], b[order]
    dt[0] = 0.0
    b[0] = 0
    t = T0 + dt
    inbox = np.isin(b, [(i1 + m) % nb for m in range(k)])
    y = np.where(inbox, 1.0 - depth0, 1.0).astype(np.float32)
    dy = np.full(n, 0.01, np.float32)
    P, I1, K, pk = oracle.bls(t, y, dy, nb, 1, min(nb - 1, k + 5), freqs=[fstar], sign=0)
    r = inbox.sum() / n
    yy = y.astype(np.float64)
    d_eff = yy[~inbox].mean() - yy[inbox].mean()   # depth after FP32 rounding of y
    assert (I1[0], K[0]) == (i1, k)
    assert math.sqrt(P[0]) == pytest.approx(d_eff * math.sqrt(r * (1 - r)), rel=1e-12)
    assert pk[0].depth == pytest.approx(d_eff, rel=1e-12)
    dt_, w, x, scal = oracle.prep(t, y, dy)
    assert P[0] == pytest.approx(scal[3], rel=1e-12)   # perfect fit: chi2 = 0


def test_boxes_holding_every_point_or_none_do_not_count():
    """Integer-day sampling: at f = 1 every point has phase 0, so no box has points on
    both sides and the power is 0.  At f = 1/2 the points split into bins 0 and 5 (nb = 10);
    with the odd days 0.02 low, equal weights give r = 1/2, s = -1/2 * 0.01, P = 1e-4.  For
    dips, of the boxes holding only bin 5 the smallest (i1, k) with k <= 4 is (2, 4); with
    both signs the bump box (0, 1) over bin 0 has the same power and comes first."""
    t = T0 + np.arange(50.0)
    y = np.where(np.arange(50) % 2 == 1, 0.98, 1.0).astype(np.float32)
    for sign in (0, 1):
        P, I1, K, _ = oracle.bls(t, y, None, 10, 1, 4, freqs=[1.0, 0.5], sign=sign)
        assert P[0] == 0.0
        yy = y.astype(np.float64)
        d = yy[0] - yy[1]                    # 0.02 after FP32 rounding
        assert P[1] == pytest.approx((0.5 * d / 2) ** 2 / 0.25, rel=1e-12)
        assert (I1[1], K[1]) == ((2, 4) if sign == 0 else (0, 1))


def test_box_across_phase_zero_wraps():
    nb, fstar = 50, 1.25
    rng = np.random.default_rng(3)
    n = 300
    cyc = rng.integers(0, 30, n)
    b = rng.integers(0, nb, n)
    dt = np.sort((cyc + (b + rng.uniform(0.3, 0.7, n)) / nb) / fstar)
    dt -= dt[0]
    b = oracle.bins(T0 + dt, [fstar], nb)[0]
    inbox = np.isin(b, [47, 48, 49, 0, 1])
    y = np.where(inbox, 0.95, 1.0).astype(np.float32)
    P, I1, K, pk = oracle.bls(T0 + dt, y, np.full(n, 0.01, np.float32), nb, 1, 8,
                              freqs=[fstar], sign=0)
    assert (I1[0], K[0]) == (47, 5)
    assert pk[0].depth == pytest.approx(0.05, rel=1e-6)


# ----------------------------------------------------------------------------- invariants

def _grid_case(seed=11, n=400):
    rng = np.random.default_rng(seed)
    t = T0 + np.sort(rng.uniform(0, 30, n))
    # flux on a 2^-12 lattice so that the offset below is exact in FP32
    y = np.round((1.0 + rng.normal(0, 0.01, n)) * 4096) / 4096
    y[(np.mod(t - T0, 0.7) < 0.05)] -= 0.03
    dy = rng.uniform(0.005, 0.02, n)
    return t, y.astype(np.float32), dy.astype(np.float32)


def test_flux_offset_invariance():
    t, y, dy = _grid_case()
    kmin, kmax = oracle.kminmax(80, 0.01, 0.12)
    P0, I0, K0, pk0 = oracle.bls(t, y, dy, 80, kmin, kmax, fmin=0.2, df=0.003, nf=600)
    y1 = (y.astype(np.float64) + 1.0).astype(np.float32)
    assert np.all(y1.astype(np.float64) - y.astype(np.float64) == 1.0)
    P1, I1, K1, pk1 = oracle.bls(t, y1, dy, 80, kmin, kmax, fmin=0.2, df=0.003, nf=600)
    scale = P0.max()
    assert np.max(np.abs(P1 - P0)) <= 1e-12 * scale
    assert pk1[0].j == pk0[0].j and (pk1[0].i1, pk1[0].k) == (pk0[0].i1, pk0[0].k)
    assert pk1[0].depth == pytest.approx(pk0[0].depth, rel=1e-10)


def test_error_scale_invariance():
    t, y, dy = _grid_case(12)
    kmin, kmax = oracle.kminmax(80, 0.01, 0.12)
    P0, _, _, pk0 = oracle.bls(t, y, dy, 80, kmin, kmax, fmin=0.2, df=0.003, nf=600)
    # a power of two scales every inverse variance exactly: identical weights
    P2, _, _, pk2 = oracle.bls(t, y, dy * 2, 80, kmin, kmax, fmin=0.2, df=0.003, nf=600)
    assert np.array_equal(P0, P2)
    assert pk2[0].snr == pytest.approx(pk0[0].snr / 2, rel=1e-15)
    # any other scale: equal up to rounding, SNR divided by the scale
    P3, _, _, pk3 = oracle.bls(t, y, (dy.astype(np.float64) * 3).astype(np.float32), 80,
                               kmin, kmax, fmin=0.2, df=0.003, nf=600)
    assert np.max(np.abs(P3 - P0)) <= 1e-6 * P0.max()  # dy*3 rounds in FP32
    assert pk3[0].j == pk0[0].j
    assert pk3[0].snr == pytest.approx(pk0[0].snr / 3, rel=1e-5)


def test_power_bounded_by_total_variance_and_dips_subset():
    t, y, dy = _grid_case(13)
    kmin, kmax = oracle.kminmax(60, 0.01, 0.2)
    Pd, _, _, _ = oracle.bls(t, y, dy, 60, kmin, kmax, fmin=0.1, df=0.01, nf=300, sign=0)
    Pb, _, _, _ = oracle.bls(t, y, dy, 60, kmin, kmax, fmin=0.1, df=0.01, nf=300, sign=1)
    dt, w, x, scal = oracle.prep(t, y, dy)
    assert np.all(Pd <= scal[3] * (1 + 1e-12))
    assert np.all(Pd <= Pb)        # dips only is a subset of the boxes


def test_unit_weights_when_dy_missing():
    t, y, dy = _grid_case(14)
    kmin, kmax = oracle.kminmax(60, 0.01, 0.2)
    Pn, _, _, _ = oracle.bls(t, y, None, 60, kmin, kmax, fmin=0.1, df=0.01, nf=100)
    P1, _, _, _ = oracle.bls(t, y, np.ones_like(dy), 60, kmin, kmax, fmin=0.1, df=0.01, nf=100)
    assert np.array_equal(Pn, P1)


# ----------------------------------------------------------------------------- fold

def test_fold_integer_cycles_land_in_bin_zero():
    P = 0.25
    for m in range(0, 4000, 37):
        assert oracle.fold(m * P, 1.0 / P, 100) == 0


def test_fold_exact_edges_and_top_bin():
    # dt*f = m + b/nb exactly (powers of two): the point opens bin b
    for nb in (8, 16, 64):
        for b in range(nb):
            dt = 3.0 + b / nb
            assert oracle.fold(dt, 1.0, nb) == b
    # the largest phase below 1 stays in the last bin
    assert oracle.fold(1.0 - 2.0 ** -53, 1.0, 100) == 99
    assert oracle.fold(np.nextafter(5.0, 0.0), 1.0, 7) == 6


def test_freq_grid_rounding():
    fmin, df = 0.1, 4.9 / 49999
    for j in (0, 1, 12345, 49999):
        assert oracle.freq(j, fmin, df) == fmin + float(np.float64(j) * df)


def test_kminmax_readings():
    assert oracle.kminmax(100, 0.01, 0.10) == (1, 10)
    assert oracle.kminmax(200, 0.005, 0.15) == (1, 30)
    assert oracle.kminmax(256, 0.005, 0.15) == (1, 39)
    assert oracle.kminmax(10, 0.5, 0.95) == (5, 9)


# ----------------------------------------------------------------------------- recovery

def test_injected_box_recovery_plain_workload():
    b = synth.config1()
    c, g, nb = b.curves[0], b.grids[0], b.nb[0]
    kmin, kmax = oracle.kminmax(nb, b.qmin, b.qmax)
    P, I1, K, pk = oracle.bls(c.t, c.y, c.dy, nb, kmin, kmax, fmin=g.fmin, df=g.df,
                              nf=g.nf, topk=1)
    p = pk[0]
    tr = c.truth
    ftrue = 1.0 / tr["period"]
    assert abs(p.freq - ftrue) <= g.df                       # within one grid step
    # within one bin: the true duration spans duration*f*nb bins at the found frequency,
    # which is off by up to half a grid step (1% slack for that)
    assert abs(p.k - tr["duration"] * p.freq * nb) <= 1.01
    mid_true = tr["epoch"] + tr["duration"] / 2
    dphi = ((p.epoch - mid_true) / p.period) % 1.0
    assert min(dphi, 1 - dphi) * nb <= 1.0                   # epoch within one bin
    sigma_depth = p.depth / p.snr
    assert abs(p.depth - tr["depth"]) <= 3 * sigma_depth


def test_topk_peaks_are_ranked_local_maxima():
    b = synth.config2(ncurves=1, nf=3000)
    c, g = b.curves[0], b.grids[0]
    kmin, kmax = oracle.kminmax(200, b.qmin, b.qmax)
    P, I1, K, pk = oracle.bls(c.t, c.y, c.dy, 200, kmin, kmax, fmin=g.fmin, df=g.df,
                              nf=g.nf, topk=5)
    js = [p.j for p in pk]
    assert js[0] == int(np.argmax(P))
    vals = [P[j] for j in js]
    assert all(vals[i] >= vals[i + 1] for i in range(4))
    for j in js:
        assert j == 0 or P[j] > P[j - 1]
        assert j == len(P) - 1 or P[j] >= P[j + 1]
    # nothing outside the list is a larger local maximum
    lm = [j for j in range(len(P)) if (j == 0 or P[j] > P[j - 1]) and
          (j == len(P) - 1 or P[j] >= P[j + 1])]
    assert sorted(lm, key=lambda j: (-P[j], j))[:5] == js


def test_many_matches_single_and_threads():
    b = synth.config2(ncurves=3, nf=700)
    kmin, kmax = oracle.kminmax(200, b.qmin, b.qmax)
    cur = [dict(t=c.t, y=c.y, dy=c.dy, nb=200, kmin=kmin, kmax=kmax, fmin=g.fmin,
                df=g.df, nf=g.nf) for c, g in zip(b.curves, b.grids)]
    pk1, P1 = oracle.bls_many(cur, nthreads=1, topk=2, want_power=True)
    pk4, P4 = oracle.bls_many(cur, nthreads=4, topk=2, want_power=True)
    assert np.array_equal(P1, P4)
    for q, (c, g) in enumerate(zip(b.curves, b.grids)):
        P, _, _, pk = oracle.bls(c.t, c.y, c.dy, 200, kmin, kmax, fmin=g.fmin, df=g.df,
                                 nf=g.nf, topk=2)
        assert np.array_equal(P, P1[q * 700:(q + 1) * 700])
        assert [p.j for p in pk] == [p.j for p in pk1[q]]
        # the threaded driver reports the same records, SDE included
        for a, b_ in zip(pk, pk1[q]):
            assert a == b_
            assert a.sde != 0.0


# ------------------------------------------------------------------------------ SDE

def _sde_case(scale=1.0, offset=0.0, err_scale=1.0):
    b = synth.config1()
    c, g = b.curves[0], b.grids[0]
    y = (1.0 + offset + scale * (c.y.astype(np.float64) - 1.0)).astype(np.float32)
    dy = (c.dy * err_scale).astype(np.float32)
    kmin, kmax = oracle.kminmax(100, b.qmin, b.qmax)
    P, _, _, pk = oracle.bls(c.t, y, dy, 100, kmin, kmax, fmin=g.fmin, df=g.df, nf=g.nf, topk=3)
    return P, pk


def test_sde_is_the_spectrum_statistic():
    """SDE = (SR_peak - mean SR) / population sd of SR over the whole spectrum."""
    P, pk = _sde_case()
    sr = np.sqrt(P)
    for p in pk:
        assert p.sde == pytest.approx((p.sr - sr.mean()) / sr.std(), rel=1e-12)
    assert pk[0].sde > pk[1].sde > pk[2].sde


def test_sde_invariances():
    """SDE does not change when the flux deviations and errors scale together (SR scales,
    the spectrum's mean and spread scale with it), when the flux is offset, or when the
    errors alone scale (normalised weights).  A factor 2 on the deviations and on the
    errors is exact in FP32, so those spectra agree to FP64 rounding; the offset flux is
    re-rounded to FP32 (about 1e-7 of a 1% noise level), hence the looser bound there."""
    _, base = _sde_case()
    for kw, rel in ((dict(scale=2.0, err_scale=2.0), 1e-9), (dict(err_scale=3.0), 1e-9),
                    (dict(offset=0.5), 1e-5)):
        _, pk = _sde_case(**kw)
        for a, b in zip(pk, base):
            assert a.j == b.j
            assert a.sde == pytest.approx(b.sde, rel=rel), kw


def test_sde_flat_spectrum_is_zero():
    t = synth.T0 + np.linspace(0, 10, 50)
    y = np.ones(50, np.float32)
    _, _, _, pk = oracle.bls(t, y, None, 20, 1, 4, fmin=0.3, df=0.1, nf=30)
    assert pk[0].sde == 0.0
