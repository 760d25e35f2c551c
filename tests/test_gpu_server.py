"""Serving (bls_submit / bls_poll): continuous batching on one GPU (marked gpu).

Requests that arrive while others run join at the next scheduler step; each result must
equal the same curve searched alone (the per-frequency arithmetic is the same, so equal
bit for bit); admission never exceeds the plan's device-memory budget; cancellation,
timeouts, invalid requests and simulated allocation failures are handled on the host
(no GPU fault is provoked)."""
import os
import time

import numpy as np
import pytest

from paper_1112_1701_b300 import bls, build, synth

# a stuck request must fail the test, not hold the GPU: bounded polls plus a watchdog
pytestmark = [pytest.mark.gpu, pytest.mark.timeout(240, method="thread")]
WAIT = 60_000   # ms


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    bls.lib()


def _requests(nreq, seed=4):
    b = synth.config4_requests(nreq, seed=seed, n_range=(200, 3000), nf_range=(2000, 9000),
                               nb_range=(100, 400))
    return [bls.CurveInput(c.t, c.y, c.dy, nf=g.nf, fmin=g.fmin, df=g.df, nb=nb,
                           qmin=b.qmin, qmax=b.qmax) for c, g, nb in zip(b.curves, b.grids, b.nb)]


def test_served_results_equal_results_alone():
    reqs = _requests(14)
    rng = np.random.default_rng(0)
    with bls.Plan(nb=200, topk=2, max_active_requests=8, step_point_freqs=200_000_000) as p:
        tickets = []
        for ci in reqs:
            tickets.append(p.submit(ci))
            time.sleep(float(rng.exponential(0.002)))   # arrivals while others run
        served = []
        for tk in tickets:
            st, pk = p.poll(tk, timeout_ms=WAIT)
            assert st == bls.OK
            served.append(pk)
        stats = p.stats()
        assert stats["completed"] == len(reqs) and stats["failed"] == 0
        assert stats["steps"] > 1
        for ci, pk in zip(reqs, served):
            alone = p.search([ci])[0]
            diff = [f for f in bls.PEAK_DTYPE.names if not np.array_equal(alone[f], pk[f])]
            assert not diff, (diff, alone[diff], pk[diff])


def test_plain_and_unbinned_plans_are_served_sequentially():
    """Plans of the plain FP64 baseline and of the unbinned search take requests through
    the same queue, one at a time, oldest first: each served result equals the same plan's
    bls_search of that curve bit for bit, and a request the algorithm refuses fails alone."""
    reqs = _requests(5, seed=11)
    for algo in ("plain_f64", "unbinned"):
        with bls.Plan(nb=200, topk=2, algo=algo) as p:
            tickets = [p.submit(ci) for ci in reqs]
            served = []
            for tk in tickets:
                st, pk = p.poll(tk, timeout_ms=WAIT)
                assert st == bls.OK
                served.append(pk)
            stats = p.stats()
            assert stats["completed"] == len(reqs) and stats["steps"] == len(reqs)
            for ci, pk in zip(reqs, served):
                alone = p.search([ci])[0]
                diff = [f for f in bls.PEAK_DTYPE.names if not np.array_equal(alone[f], pk[f])]
                assert not diff, (algo, diff)
    # the unbinned search refuses curves above its point limit: that request fails, the
    # next one is served
    rng = np.random.default_rng(2)
    t = synth.T0 + np.sort(rng.uniform(0, 30, 40000))
    big = bls.CurveInput(t, np.ones(len(t), np.float32), None, nf=100, fmin=0.2, df=0.01,
                         nb=200, qmin=0.005, qmax=0.15)
    with bls.Plan(nb=200, algo="unbinned") as p:
        tb = p.submit(big)
        tg = p.submit(reqs[1])
        with pytest.raises(bls.BLSError):
            p.poll(tb, timeout_ms=WAIT)
        st, _ = p.poll(tg, timeout_ms=WAIT)
        assert st == bls.OK


def test_admission_respects_memory_budget():
    reqs = _requests(10, seed=7)
    # room for a few requests at a time: each needs ~40 B per point + 4 B per frequency
    budget = 3 * max(40 * len(c.t) + 4 * c.nf + 8192 for c in reqs)
    with bls.Plan(nb=200, max_device_bytes=budget) as p:
        tks = [p.submit(ci) for ci in reqs]
        for tk in tks:
            st, _ = p.poll(tk, timeout_ms=WAIT)
            assert st == bls.OK
        s = p.stats()
        assert 0 < s["device_bytes_peak"] <= budget
        assert s["device_bytes_in_use"] == 0


def test_request_over_budget_is_refused():
    ci = _requests(1)[0]
    with bls.Plan(nb=200, max_device_bytes=4096) as p:
        with pytest.raises(bls.BLSError) as ei:
            p.submit(ci)
        assert ei.value.status == bls.ERR_NOMEM


def test_cancel_and_timeouts():
    big = bls.CurveInput(*(_make_big()), nf=90000, fmin=0.1, df=5e-5, nb=300, qmin=0.005,
                         qmax=0.15)
    small = _requests(2)
    with bls.Plan(nb=200, max_active_requests=1, step_point_freqs=20_000_000) as p:
        t_big = p.submit(big)
        t_small = p.submit(small[0])          # queued behind the big one
        st, _ = p.poll(t_big, timeout_ms=0)
        assert st == bls.PENDING
        st, _ = p.poll(t_big, timeout_ms=1)
        assert st in (bls.ERR_TIMEOUT, bls.OK)
        p.cancel(t_small)                     # still queued: cancelled at once
        with pytest.raises(bls.BLSError) as ei:
            p.poll(t_small, timeout_ms=WAIT)
        assert ei.value.status == bls.ERR_CANCELLED
        p.cancel(t_big)                       # active: cancelled at the next step
        with pytest.raises(bls.BLSError) as ei:
            p.poll(t_big, timeout_ms=WAIT)
        assert ei.value.status in (bls.ERR_CANCELLED,)
        # the server keeps working afterwards
        t2 = p.submit(small[1])
        st, pk = p.poll(t2, timeout_ms=WAIT)
        assert st == bls.OK
        with pytest.raises(bls.BLSError) as ei:
            p.poll(t2, timeout_ms=0)          # retired ticket
        assert ei.value.status == bls.ERR_INVALID
        with pytest.raises(bls.BLSError) as ei:
            p.poll(123456789, timeout_ms=0)
        assert ei.value.status == bls.ERR_INVALID


def _make_big():
    rng = np.random.default_rng(3)
    n = 20000
    t = synth.T0 + np.sort(rng.uniform(0, 60, n))
    y = (1 + rng.normal(0, 0.01, n)).astype(np.float32)
    return t, y, np.full(n, 0.01, np.float32)


def test_invalid_requests_rejected_at_submit():
    t = synth.T0 + np.linspace(0, 10, 50)
    y = np.ones(50, np.float32)
    y_bad = y.copy()
    y_bad[3] = np.inf
    with bls.Plan(nb=50, qmin=0.02, qmax=0.2) as p:
        for ci in (bls.CurveInput(t, y_bad, None, nf=10, fmin=0.1, df=0.1),
                   bls.CurveInput(t[:1], y[:1], None, nf=10, fmin=0.1, df=0.1),
                   bls.CurveInput(t, y, np.zeros(50, np.float32), nf=10, fmin=0.1, df=0.1)):
            with pytest.raises(bls.BLSError) as ei:
                p.submit(ci)
            assert ei.value.status == bls.ERR_INVALID
        torch = pytest.importorskip("torch")
        with pytest.raises(bls.BLSError) as ei:   # device input checked after the copy
            p.submit(bls.CurveInput(torch.tensor(t, device="cuda"),
                                    torch.tensor(y_bad, device="cuda"), None, nf=10, fmin=0.1,
                                    df=0.1))
        assert ei.value.status == bls.ERR_INVALID


def test_simulated_allocation_failures_leave_server_running(monkeypatch):
    monkeypatch.setenv("BLS_SERVER_FAIL_ALLOC_EVERY", "3")
    reqs = _requests(7, seed=9)
    with bls.Plan(nb=200) as p:
        tks = [p.submit(ci) for ci in reqs]
        ok = fail = 0
        for tk in tks:
            try:
                st, _ = p.poll(tk, timeout_ms=WAIT)
                ok += st == bls.OK
            except bls.BLSError as e:
                assert e.status == bls.ERR_NOMEM
                fail += 1
        assert fail == 2 and ok == 5
        assert p.stats()["failed"] == 2
