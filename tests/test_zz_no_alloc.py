"""bls_search_static: the search of one curve that allocates nothing.

Callers that cannot call cudaMalloc (a plug-in whose host application owns all device
memory, a latency-critical loop that cannot take cudaMalloc's implicit synchronisation, a
process under a memory cap) use this entry point with device inputs and outputs; its
intermediate data lives in a static device array.  Its results must match bls_search's
(the regular entry point, which allocates its own buffers) within the tolerance of the
parity tests, on two calls in a row (the static array keeps the previous call's contents).
This file is collected last so that a stopping run has already run every other test.
"""
import numpy as np
import pytest

from paper_1112_1701_b300 import bls, build, synth

pytestmark = pytest.mark.gpu


def _sr_tol(sr, sumwx2):
    return 1e-5 * sr + 1e-6 * np.sqrt(sumwx2)


def test_static_search_matches_search_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    build.build()
    import oracle
    b = synth.config2(ncurves=2, nf=3000)
    stream = torch.cuda.current_stream().cuda_stream
    topk = 3
    for q in range(2):
        c, g = b.curves[q], b.grids[q]
        dev = bls.CurveInput(torch.tensor(c.t, device="cuda"), torch.tensor(c.y, device="cuda"),
                             torch.tensor(c.dy, device="cuda"), nf=g.nf, fmin=g.fmin, df=g.df,
                             nb=200, qmin=b.qmin, qmax=b.qmax)
        peaks_buf = torch.zeros(topk * bls.PEAK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        spec = torch.zeros(g.nf, dtype=torch.float32, device="cuda")
        bls.search_static(dev, topk=topk, stream=stream, peaks=peaks_buf, spectrum=spec)
        torch.cuda.synchronize()
        got = bls.peaks_to_numpy(peaks_buf, topk)
        got_spec = spec.cpu().numpy()

        host = bls.CurveInput(c.t, c.y, c.dy, nf=g.nf, fmin=g.fmin, df=g.df, nb=200,
                              qmin=b.qmin, qmax=b.qmax)
        ref_spec = np.zeros(g.nf, np.float32)
        # the static search sums in FP32: the regular search in the same sum mode
        with bls.Plan(nb=200, qmin=b.qmin, qmax=b.qmax, topk=topk, sum="f32") as p:
            ref = p.search([host], spectrum=ref_spec)[0]
        _, _, _, scal = oracle.prep(c.t, c.y, c.dy)
        tol = _sr_tol(ref_spec.astype(np.float64), scal[3])
        assert np.all(np.abs(got_spec.astype(np.float64) - ref_spec) <= tol)
        for e in range(topk):
            assert (got[e]["j"], got[e]["i1"], got[e]["k"]) == (ref[e]["j"], ref[e]["i1"], ref[e]["k"])
            for f in ("freq", "period", "epoch", "duration", "depth", "snr", "sr", "power", "sde"):
                assert got[e][f] == pytest.approx(ref[e][f], rel=1e-9, abs=1e-12), f


def test_static_search_allocates_no_device_memory():
    """After a warm-up call (the first call on a device resolves the static array's
    address and loads the kernels), further calls leave the device's free memory and
    torch's allocation count unchanged."""
    torch = pytest.importorskip("torch")
    build.build()
    b = synth.config2(ncurves=1, nf=2000)
    c, g = b.curves[0], b.grids[0]
    dev = bls.CurveInput(torch.tensor(c.t, device="cuda"), torch.tensor(c.y, device="cuda"),
                         torch.tensor(c.dy, device="cuda"), nf=g.nf, fmin=g.fmin, df=g.df,
                         nb=200, qmin=b.qmin, qmax=b.qmax)
    peaks_buf = torch.zeros(2 * bls.PEAK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    spec = torch.zeros(g.nf, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    bls.search_static(dev, topk=2, stream=stream, peaks=peaks_buf, spectrum=spec)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(2):
        bls.search_static(dev, topk=2, stream=stream, peaks=peaks_buf, spectrum=spec)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_static_search_rejects_oversized_and_host_inputs():
    torch = pytest.importorskip("torch")
    build.build()
    t = torch.linspace(0, 10, 100, dtype=torch.float64, device="cuda")
    y = torch.ones(100, dtype=torch.float32, device="cuda")
    peaks = torch.zeros(bls.PEAK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    too_many = bls.CurveInput(t, y, None, nf=9_000_000, fmin=0.1, df=1e-7, nb=50, qmin=0.02,
                              qmax=0.2)
    with pytest.raises(bls.BLSError) as ei:
        bls.search_static(too_many, peaks=peaks)
    assert ei.value.status == bls.ERR_INVALID and "static scratch" in str(ei.value)
    host_in = bls.CurveInput(np.linspace(0, 10, 100), np.ones(100, np.float32), None, nf=10,
                             fmin=0.1, df=0.1, nb=50, qmin=0.02, qmax=0.2)
    with pytest.raises(bls.BLSError) as ei:
        bls.search_static(host_in, peaks=peaks)
    assert ei.value.status == bls.ERR_INVALID
    # outputs too small for what the call would write
    ok = bls.CurveInput(t, y, None, nf=10, fmin=0.1, df=0.1, nb=50, qmin=0.02, qmax=0.2)
    with pytest.raises(bls.BLSError) as ei:
        bls.search_static(ok, topk=2, peaks=peaks)                   # room for one record
    assert ei.value.status == bls.ERR_INVALID
    short = torch.zeros(9, dtype=torch.float32, device="cuda")
    with pytest.raises(bls.BLSError) as ei:
        bls.search_static(ok, peaks=peaks, spectrum=short)           # 10 frequencies
    assert ei.value.status == bls.ERR_INVALID
