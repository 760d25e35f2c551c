"""Host logic of the detection-efficiency harness: the recovery criterion and the
injection generator (no GPU)."""
import numpy as np

from paper_1112_1701_b300 import efficiency, synth


def test_recovery_criterion():
    df = 0.001
    ft = np.array([1.0, 1.0, 1.0, 1.0, 1.0, 0.3])
    fb = np.array([1.0015, 2.0019, 0.5, 1.0031, 1.5, 0.3])
    ok = efficiency.recovered(fb, ft, df, steps=2.0)
    assert ok.tolist() == [True, True, True, False, False, True]
    assert efficiency.recovered(fb, ft, df, steps=2.0, harmonics=(1.0,)).tolist() == \
        [True, False, False, False, False, True]


def test_injections_carry_their_eclipse():
    t = synth.survey_cadence(seed=3, nights=20)
    b = synth.eclipse_injections(t, [0.7, 2.5], 3, duration=0.05, depth=0.1, sigma=1e-6,
                                 seed=5, nf=100)
    assert len(b) == 6 and b.grids[0].nf == 100
    for c in b.curves:
        P, ep, D = c.truth["period"], c.truth["epoch"], c.truth["duration"]
        inside = np.mod(c.t - ep, P) < D
        assert np.array_equal(c.t, t)
        assert np.all(np.abs(c.y[inside] - 0.9) < 1e-4)
        assert np.all(np.abs(c.y[~inside] - 1.0) < 1e-4)


def test_cadence_shape():
    t = synth.survey_cadence(seed=4, nights=30, cadence_min=20.0, p_weather=0.0)
    assert np.all(np.diff(t) > 0)
    nights = np.unique(np.floor(t - synth.T0 + 0.5))
    assert len(nights) == 30
    per = len(t) / 30
    assert 14 <= per <= 15     # 4.8 h window every 20 min
