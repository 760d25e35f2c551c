"""Eclipse-window detection efficiency: CUDA kernel vs the FP64 oracle (marked gpu).

The efficiency and the per-(frequency, phase) eclipse counts are integers decided by FP64
arithmetic in the same operation order on both sides, so they must agree exactly."""
import numpy as np
import pytest

import oracle
from paper_1112_1701_b300 import bls, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    bls.lib()


def _both(t, nphi, **kw):
    eg, cg = bls.window_efficiency(t, nphi, want_counts=True, **kw)
    eo, co = oracle.window(t, nphi, want_counts=True, **kw)
    return eg, cg, eo, co


def test_survey_cadence_uniform_grid():
    """A 60-night field with weather losses: 500 frequencies in [0.1, 5] 1/d (periods
    0.2-10 d), eclipses 0.04 d long, 64 phases."""
    t = synth.survey_cadence(seed=6, nights=60)
    eg, cg, eo, co = _both(t, 64, fmin=0.1, df=4.9 / 499, nf=500, duration=0.04)
    assert np.array_equal(cg, co)
    assert np.array_equal(eg, eo)
    assert 0.0 < eg.min() and eg.max() == 1.0   # short periods nearly always seen


def test_multichunk_multipass_fraction_of_period():
    """More times than one staged chunk (5000 > 2048) and more phases than one block
    pass (300 > 256); duration given as a fraction of the period; 2 points per eclipse."""
    t = synth.survey_cadence(seed=8, nights=120, cadence_min=5.0, p_weather=0.2)
    assert len(t) > 5000
    rng = np.random.default_rng(2)
    freqs = np.sort(rng.uniform(0.05, 3.0, 37))
    eg, cg, eo, co = _both(t, 300, freqs=freqs, qfrac=0.03, min_points=2)
    assert np.array_equal(cg, co) and np.array_equal(eg, eo)


@pytest.mark.parametrize("min_eclipses", [0, 1, 3])
def test_min_eclipses(min_eclipses):
    t = synth.survey_cadence(seed=9, nights=30)
    eg, cg, eo, co = _both(t, 40, fmin=0.2, df=0.01, nf=80, duration=0.05,
                           min_eclipses=min_eclipses)
    assert np.array_equal(cg, co) and np.array_equal(eg, eo)


def test_integer_day_alias_and_tiny_cases():
    nights = 40
    t = synth.T0 + np.arange(nights, dtype=np.float64) + 0.2
    eg, cg, eo, co = _both(t, 100, freqs=np.array([1.0, 1 / 1.07, 0.5]), duration=0.105)
    assert np.array_equal(cg, co) and np.array_equal(eg, eo)
    assert eg[0] == 0.10
    one = np.array([synth.T0 + 3.0])
    eg, cg, eo, co = _both(one, 1, freqs=np.array([0.7]), qfrac=0.2, min_eclipses=1)
    assert np.array_equal(cg, co) and np.array_equal(eg, eo)


def test_device_buffers_match_host():
    torch = pytest.importorskip("torch")
    t = synth.survey_cadence(seed=10, nights=45)
    freqs = np.linspace(0.1, 5.0, 333)
    eh, ch = bls.window_efficiency(t, 48, freqs=freqs, duration=0.03, want_counts=True)
    td = torch.tensor(t, device="cuda")
    fd = torch.tensor(freqs, device="cuda")
    ed = torch.zeros(333, dtype=torch.float64, device="cuda")
    cd = torch.zeros((333, 48), dtype=torch.int32, device="cuda")
    bls.window_efficiency(td, 48, freqs=fd, duration=0.03, eff=ed, counts=cd,
                          stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.array_equal(ed.cpu().numpy(), eh) and np.array_equal(cd.cpu().numpy(), ch)


def test_invalid_inputs_rejected():
    t = synth.survey_cadence(seed=11, nights=10)
    bad = t.copy()
    bad[5], bad[6] = bad[6], bad[5]
    with pytest.raises(bls.BLSError) as ei:
        bls.window_efficiency(bad, 8, freqs=np.array([1.0]), duration=0.05)
    assert ei.value.status == bls.ERR_INVALID
    nan = t.copy()
    nan[3] = np.nan
    with pytest.raises(bls.BLSError):
        bls.window_efficiency(nan, 8, freqs=np.array([1.0]), duration=0.05)
    with pytest.raises(bls.BLSError):
        bls.window_efficiency(t, 8, freqs=np.array([1.0, -1.0]), duration=0.05)
    with pytest.raises(bls.BLSError):
        bls.window_efficiency(t, 8, freqs=np.array([1.0]))   # no duration
    # the context stays usable
    e, _ = bls.window_efficiency(t, 8, freqs=np.array([1.0]), duration=0.05)
    assert 0.0 <= e[0] <= 1.0


def test_injection_recovery_matches_oracle_search():
    """The recovery harness on the GPU search gives the oracle's best frequency wherever
    the oracle's top two peaks are separated, hence the same recovered flags there."""
    from paper_1112_1701_b300 import efficiency
    from tests.parity import separated_best
    t = synth.survey_cadence(seed=12, nights=30)
    b = synth.eclipse_injections(t, [0.45, 1.7, 3.3], 3, duration=0.04, depth=0.03,
                                 sigma=0.01, seed=13, nf=3000)
    f_best, ok = efficiency.injection_recovery(b)
    kmin, kmax = oracle.kminmax(200, b.qmin, b.qmax)
    g = b.grids[0]
    checked = 0
    for i, c in enumerate(b.curves):
        P, _, _, pk = oracle.bls(c.t, c.y, c.dy, 200, kmin, kmax, fmin=g.fmin, df=g.df, nf=g.nf)
        scal = oracle.prep(c.t, c.y, c.dy)[3]
        jo, sep = separated_best(P, scal[3])
        if sep:
            checked += 1
            assert f_best[i] == pk[0].freq
            assert ok[i] == efficiency.recovered([pk[0].freq], [1.0 / c.truth["period"]], g.df)[0]
    assert checked >= 5
    assert ok.mean() > 0.5      # 3% eclipses at 1% noise are mostly recovered


def test_detection_efficiency_curve():
    from paper_1112_1701_b300 import efficiency
    t = synth.survey_cadence(seed=14, nights=40)
    periods = np.array([0.3, 0.55, 1.0, 1.9, 4.2, 9.5])
    ec = efficiency.detection_efficiency(t, periods, 4, duration=0.04, depth=0.05,
                                         sigma=0.01, nf=4000, nphi=128)
    eo, _ = oracle.window(t, 128, freqs=1.0 / periods, duration=0.04)
    assert np.array_equal(ec.window, eo)
    assert ec.recovery.shape == (6,) and np.all((ec.recovery >= 0) & (ec.recovery <= 1))
    assert ec.window[0] == 1.0 and ec.recovery[0] >= 0.75
