"""Search cases run by tests/test_gpu_debug.py in a subprocess, once with the regular
library and once with the BLS_DEBUG build (the build is chosen when the binding first
loads the library, so each build runs in its own process).

    python -m tests.debug_cases OUT.npz

Every search result (spectra, peak records) goes into OUT.npz, with the path of the
library that produced it.  A device-side index check that fails makes a search raise
(ERR_INTERNAL), which ends the process with an error."""
import sys

import numpy as np


def main(out):
    import torch
    from paper_1112_1701_b300 import bls, synth

    res = {"lib": np.array(bls.LIB_PATH)}

    def search(tag, cis, nb, qmin, qmax, **kw):
        nf = sum(len(c.freqs) if c.freqs is not None else c.nf for c in cis)
        spec = np.zeros(nf, np.float32)
        with bls.Plan(nb=nb, qmin=qmin, qmax=qmax, **kw) as p:
            pk = p.search(cis, spectrum=spec)
        res[tag + "_spec"] = spec
        res[tag + "_peaks"] = pk.view(np.uint8)

    b1 = synth.config1()
    search("plain", bls.curves_from_batch(b1), 100, b1.qmin, b1.qmax, topk=3)
    b2 = synth.config2(ncurves=24, nf=3000, seed=71)
    cis2 = bls.curves_from_batch(b2)
    search("batched", cis2, 200, b2.qmin, b2.qmax, topk=2)
    search("batched_both", cis2, 200, b2.qmin, b2.qmax, sign="both")
    search("batched_kmin", cis2, 200, 0.03, 0.15)
    search("batched_kahan", cis2, 200, b2.qmin, b2.qmax, sum="kahan")
    search("batched_onegroup", cis2, 200, b2.qmin, b2.qmax, fold_kernel="one_group")
    search("batched_df32", cis2, 200, b2.qmin, b2.qmax, phase="df32")
    b5 = synth.config5(ncurves=6, nf=20000)
    search("survey", bls.curves_from_batch(b5), 256, b5.qmin, b5.qmax, topk=5)
    search("survey_T48", bls.curves_from_batch(b5), 256, b5.qmin, b5.qmax, freqs_per_block=48)
    bw = synth.config2(ncurves=4, nf=1500, seed=72)
    search("nb400", bls.curves_from_batch(bw), 400, bw.qmin, bw.qmax)
    search("unbinned", bls.curves_from_batch(synth.config2(ncurves=3, nf=300, seed=73)), 200,
           0.005, 0.15, algo="unbinned")
    # serving: a few requests of different nb through the queue
    b4 = synth.config4_requests(6, n_range=(200, 3000), nf_range=(2000, 6000))
    reqs = [bls.CurveInput(c.t, c.y, c.dy, nf=g.nf, fmin=g.fmin, df=g.df, nb=nb, qmin=b4.qmin,
                           qmax=b4.qmax) for c, g, nb in zip(b4.curves, b4.grids, b4.nb)]
    with bls.Plan(nb=200, topk=1) as p:
        tickets = [p.submit(r) for r in reqs]
        served = []
        for t in tickets:
            st, pk = p.poll(t, timeout_ms=120000)
            assert st == bls.OK
            served.append(pk.view(np.uint8))
    res["served"] = np.concatenate(served)
    # the allocation-free entry point
    c, g = b2.curves[0], b2.grids[0]
    dev = bls.CurveInput(torch.tensor(c.t, device="cuda"), torch.tensor(c.y, device="cuda"),
                         torch.tensor(c.dy, device="cuda"), nf=g.nf, fmin=g.fmin, df=g.df,
                         nb=200, qmin=b2.qmin, qmax=b2.qmax)
    buf = torch.zeros(2 * bls.PEAK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    spec = torch.zeros(g.nf, dtype=torch.float32, device="cuda")
    bls.search_static(dev, topk=2, stream=torch.cuda.current_stream().cuda_stream, peaks=buf,
                      spectrum=spec)
    torch.cuda.synchronize()
    res["static_peaks"] = buf.cpu().numpy()
    res["static_spec"] = spec.cpu().numpy()
    np.savez(out, **res)


if __name__ == "__main__":
    main(sys.argv[1])
