#!/usr/bin/env python
"""Benchmark of the BLS search on one B300 (or N independent replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Headline workload: the survey-scale sweep of 100,000 light curves, timed on a subset of
2048 curves per rank (2000 points over 90 nights, FP64 times, FP32 flux, 5% with injected
boxes), 200,000 trial frequencies uniform in [0.1, 5] 1/d, nb = 256 phase bins, q in
[0.005, 0.15], top-5 peaks per curve.  A step is one bls_search over the subset: prep,
fold-bin-sweep, peak reduction; the full survey's time is extrapolated linearly in curves.

Metric: point x frequency evaluations per second (sum over curves of N * nf per step,
divided by the step time).  `value` is timed with CUDA events on the plan's stream with
inputs resident in device memory; L2 is flushed (256 MiB write) before every step inside
the timed region.  `e2e` is the same metric through the C ABI with pinned host buffers:
host-to-device copies of t, y, dy and the device-to-host copy of the peaks are inside.
Also in the line: `batched` (1024 curves x 50,000 frequencies, nb = 200, measured the same
way), `serving` (p50/p99 latency at 50/70/90% of the measured saturation rate, with the
plain FP64 one-curve-per-launch kernel served through the same queue at the same offered
rates), `plain_f64_gpu` (that kernel's throughput on the headline curves) and
`cpu_baseline` (the FP64 oracle on the host cores, bounded sample).

Roofline of the dominant kernel (fold-bin-sweep), shared-memory / FP32-issue model with the
unit rates probed on B300 (profiles/probes_b300.md):
  loop A (fold + bin), per point x frequency: 2 shared-memory read-modify-writes of 8 B,
      16 B at 127 B/clk/SM;
  loop B (box sweep), per box evaluation: 7 FP32 ops (2 adds, r(1-r), s^2, compare) at
      126 per clk per SM.
Multi-GPU (torchrun, N > 1): each rank searches its own curves (weak scaling);
value = all ranks' units / max over ranks of the step time.  No data-path collective.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1112_1701_b300 import synth  # noqa: E402

METRIC = "BLS point x freq evals/s"
UNIT = "point*freq/s"
NB, QMIN, QMAX = 200, 0.005, 0.15

# DRAM traffic of one fold-bin-sweep launch of the headline workload (dram__bytes_read.sum +
# dram__bytes_write.sum, one ncu capture of the timed launch after an L2 flush,
# profiles/fold_sweep_survey_2048x200k_dram.md), valid for the kernel source with the given
# SHA-256; reported as null once the source changes.
NCU_TRAFFIC = {"workload": "survey", "ncurves": 2048,
               "kernel_sha256": "dcf2a2ab73413f1f73f9a446ef059607beb54f2bd2cde447510583f65b7eebd6",
               "bytes_per_launch": 163674368 + 1615719168}


def kernel_sha():
    p = os.path.join(ROOT, "paper_1112_1701_b300", "csrc", "bls_kernels.cu")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}",
                                          f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.f.read())) if len(r) >= 9]
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(sm), "power_w_max": max(power) if power else None,
                "reasons": sorted(reasons)}


def box_evals(batch):
    from paper_1112_1701_b300 import bls
    tot = 0
    for g, nb in zip(batch.grids, batch.nb):
        kmin, kmax = bls.kminmax(nb, batch.qmin, batch.qmax)
        tot += nb * (kmax - kmin + 1) * g.nf
    return tot


def cpu_baseline(batch, seconds_hint=15.0, single_freqs=20000):
    """The FP64 oracle as it stands, on all host cores, on a bounded sample of curves (full
    grid each, sized to about seconds_hint of wall time), plus one thread on the first
    curve's first single_freqs frequencies; returns the CPU-baseline object."""
    import oracle
    cores = os.cpu_count() or 1
    nb = batch.nb[0]
    topk = int(batch.extra.get("topk", 1))
    kmin, kmax = oracle.kminmax(nb, batch.qmin, batch.qmax)

    def run(idx, threads=cores, nf=None):
        cur = [dict(t=batch.curves[i].t, y=batch.curves[i].y, dy=batch.curves[i].dy, nb=nb,
                    kmin=kmin, kmax=kmax, fmin=batch.grids[i].fmin, df=batch.grids[i].df,
                    nf=nf or batch.grids[i].nf) for i in idx]
        t0 = time.perf_counter()
        oracle.bls_many(cur, nthreads=threads, topk=topk)
        return time.perf_counter() - t0, sum(len(batch.curves[i].t) * (nf or batch.grids[i].nf)
                                             for i in idx)

    # calibrate on one curve (the oracle's threads share its frequency chunks), then size
    # the sample to ~seconds_hint
    dt0, u0 = run([0])
    ncur = int(min(len(batch), max(1, seconds_hint * (u0 / dt0) / u0)))
    dt, u = run(list(range(ncur)))
    kf = min(single_freqs, batch.grids[0].nf)
    dt1, u1 = run([0], threads=1, nf=kf)
    full_s = batch.point_freqs() / (u / dt)
    return {"value": u / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{ncur} of {len(batch)} curves x full {batch.grids[0].nf}-frequency grid "
                      f"(nb={nb}, top-{topk}), FP64 C oracle on {cores} host threads, {dt:.1f} s; "
                      f"the whole batch would take {full_s:.0f} s at this rate",
            "single_thread": {"value": u1 / dt1,
                              "sample": f"curve 0 x first {kf} frequencies, one thread"},
            "cpu_model": cpu_model()}


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def headline_batch(args, rank=0, world=1):
    """The headline workload of one rank: its own args.survey_curves curves of the
    100,000-curve survey sweep (2000 points over 90 nights, 200,000 frequencies in
    [0.1, 5] 1/d, nb = 256, q 0.005-0.15, top-5)."""
    return synth.config5(ncurves=args.survey_curves, nf=args.survey_nf,
                         first=rank * args.survey_curves)


def headline_config(batch, args, world=1):
    nb = batch.nb[0]
    return {"workload": f"survey sweep subset: {len(batch)} of 100000 curves x 2000 points over "
                        f"90 nights, {batch.grids[0].nf} freqs uniform in [0.1, 5]/d, nb={nb}, "
                        f"q {batch.qmin}-{batch.qmax}, top-5 peaks per curve",
            "ncurves": len(batch), "nf": batch.grids[0].nf, "nb": nb, "topk": 5,
            "points": int(sum(len(c.t) for c in batch.curves)),
            "l2": "inputs (64 MB of points + 1.6 GB of per-frequency results per step) exceed "
                  "L2; flushed (256 MiB write) before every step, inside the timed region",
            "inputs": "device-resident for value; pinned host for e2e",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    """Reference arm: the FP64 oracle timed on the host cores, same metric and workload
    (the survey sweep subset); each step searches a bounded sample of its curves (full
    grid each)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    batch = headline_batch(args)
    nb = batch.nb[0]
    cores = os.cpu_count() or 1
    kmin, kmax = oracle.kminmax(nb, batch.qmin, batch.qmax)
    per_step = max(1, min(len(batch), args.ref_curves or max(1, cores // 8)))
    times, units = [], []
    for s in range(args.warmup + args.steps):
        idx = [(s * per_step + i) % len(batch) for i in range(per_step)]
        cur = [dict(t=batch.curves[i].t, y=batch.curves[i].y, dy=batch.curves[i].dy, nb=nb,
                    kmin=kmin, kmax=kmax, fmin=batch.grids[i].fmin, df=batch.grids[i].df,
                    nf=batch.grids[i].nf) for i in idx]
        t0 = time.perf_counter()
        oracle.bls_many(cur, nthreads=cores, topk=5)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            units.append(sum(len(batch.curves[i].t) * batch.grids[i].nf for i in idx))
    value = sum(units) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": headline_config(batch, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} of {len(batch)} curves x full grid per "
                                       f"step, FP64 C oracle on {cores} host threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def serving_measurement(nreq, nplain, loads, step_units=0, plain=True):
    """Serving on one GPU: a Poisson stream of single-curve requests, each with its own
    grid and bin count (N log-uniform 200-20000, 10k-100k frequencies, nb 100-400).  The
    saturation rate comes from submitting all nreq at once; then, at each fraction of it,
    the requests arrive as a Poisson stream and p50/p99 (submit -> result) are read from
    the server.  The plain FP64 one-curve-per-launch kernel is served through the same
    queue (sequential plan) at the same offered rates on the first nplain requests of the
    same stream."""
    import threading
    from paper_1112_1701_b300 import bls
    b = synth.config4_requests(nreq)
    reqs = [bls.CurveInput(c.t, c.y, c.dy, nf=g.nf, fmin=g.fmin, df=g.df, nb=nb, qmin=b.qmin,
                           qmax=b.qmax) for c, g, nb in zip(b.curves, b.grids, b.nb)]
    units = sum(len(c.t) * g.nf for c, g in zip(b.curves, b.grids))

    def serve(rs, arrivals, **plan_kw):
        with bls.Plan(nb=200, qmin=QMIN, qmax=QMAX, topk=1, **plan_kw) as p:
            for tk in [p.submit(r) for r in rs[:2]]:     # warm-up (kernels, buffers)
                p.poll(tk, timeout_ms=600000)
            base = p.stats()["completed"]
            tickets = [None] * len(rs)

            def submitter():
                t0 = time.perf_counter()
                for i, r in enumerate(rs):
                    if arrivals is not None:
                        delay = arrivals[i] - (time.perf_counter() - t0)
                        if delay > 0:
                            time.sleep(delay)
                    tickets[i] = p.submit(r)

            th = threading.Thread(target=submitter)
            t0 = time.perf_counter()
            th.start()
            th.join()
            for tk in tickets:
                st, _ = p.poll(tk, timeout_ms=600000)
                assert st == bls.OK
            wall = time.perf_counter() - t0
            stt = p.stats()
            assert stt["completed"] - base == len(rs)
            return wall, stt

    kw = dict(step_point_freqs=step_units) if step_units else {}
    wall_sat, _ = serve(reqs, None, **kw)
    sat_rate = nreq / wall_sat
    out_loads = []
    for frac in loads:
        rate = frac * sat_rate
        arr = synth.poisson_arrivals(nreq, rate)
        wall, st = serve(reqs, arr, **kw)
        row = {"offered_fraction": frac, "offered_req_per_s": rate,
               "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
               "throughput_req_per_s": nreq / wall, "point_freq_per_s": units / wall,
               "steps": st["steps"]}
        if plain and nplain > 0:
            pw, pst = serve(reqs[:nplain], arr[:nplain], algo="plain_f64")
            row["plain_f64_served"] = {"requests": nplain, "p50_ms": pst["p50_ms"],
                                       "p99_ms": pst["p99_ms"],
                                       "throughput_req_per_s": nplain / pw}
        out_loads.append(row)
    return {"workload": f"serving: {nreq} requests, N log-uniform 200-20000, nf 10k-100k, "
                        f"nb 100-400, q {QMIN}-{QMAX}, Poisson arrivals",
            "requests": nreq, "latency": "submit -> result (server clock), p50/p99 over the "
                                         "load's requests plus 2 warm-up requests",
            "saturation": {"req_per_s": sat_rate, "point_freq_per_s": units / wall_sat},
            "loads": out_loads,
            "plain_f64": "one-curve-per-launch FP64 kernel served through the same queue "
                         "(sequential plan) on the first requests of each load's stream, same "
                         "arrival times" if plain and nplain > 0 else None}


def run_serving(args):
    """Serving benchmark alone (--serving): serving_measurement at args.requests."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    obj = serving_measurement(args.requests, args.plain_requests, args.loads, args.step_units)
    line = {"metric": "BLS serving latency and throughput",
            "value": obj["saturation"]["point_freq_per_s"], "unit": UNIT, "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic",
            "config": {"workload": obj["workload"], "requests": args.requests},
            "serving": obj}
    print(json.dumps(line), flush=True)
    return 0


def plain_curve_measurement(reps=20):
    """The plain workload: one light curve (500 times in 20 of 30 nightly windows, a 2%
    box at P = 0.40 d), 2000 frequencies in [0.2, 5] 1/d, nb = 100, q 0.01-0.10: the median
    time of a search (device-resident inputs, and from host arrays), the plain FP64 GPU
    kernel, the FP64 oracle on one thread and on all host threads, and the recovered period."""
    import torch
    import oracle
    from paper_1112_1701_b300 import bls
    b = synth.config1()
    c, g = b.curves[0], b.grids[0]
    units = len(c.t) * g.nf
    dev = bls.curves_from_batch(b, device="cuda")
    host = bls.curves_from_batch(b)
    stream = torch.cuda.current_stream()

    def timed(plan, cis):
        plan.search(cis)
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pk = plan.search(cis)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts), pk

    with bls.Plan(nb=100, qmin=b.qmin, qmax=b.qmax, topk=1, stream=stream.cuda_stream) as p:
        t_dev, pk = timed(p, dev)
        t_host, _ = timed(p, host)
    with bls.Plan(nb=100, qmin=b.qmin, qmax=b.qmax, topk=1, algo="plain_f64",
                  stream=stream.cuda_stream) as p:
        t_plain, _ = timed(p, dev)
    kmin, kmax = oracle.kminmax(100, b.qmin, b.qmax)
    cur = [dict(t=c.t, y=c.y, dy=c.dy, nb=100, kmin=kmin, kmax=kmax, fmin=g.fmin, df=g.df,
                nf=g.nf)]
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.bls_many(cur, nthreads=1, topk=1)
    t_o1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.bls_many(cur, nthreads=cores, topk=1)
    t_on = time.perf_counter() - t0
    return {"workload": "plain: one curve, 500 points in 20 of 30 nights, 2000 freqs in "
                        "[0.2, 5]/d, nb=100, q 0.01-0.10, injected box P = 0.40 d",
            "value": units / t_dev, "unit": UNIT, "latency_ms": 1000 * t_dev,
            "from_host_arrays": {"value": units / t_host, "latency_ms": 1000 * t_host},
            "plain_f64_gpu": {"value": units / t_plain, "latency_ms": 1000 * t_plain},
            "oracle_one_thread": {"value": units / t_o1, "ms": 1000 * t_o1},
            "oracle_all_threads": {"value": units / t_on, "ms": 1000 * t_on, "cores": cores},
            "best_period_d": float(pk[0, 0]["period"]), "injected_period_d": 0.40,
            "timing": f"median of {reps} searches, wall clock with the stream synchronised"}


def plain_f64_sample(batch, ncurves, value):
    """The plain FP64 one-curve-per-launch GPU kernel (the paper's decomposition without
    redesign) on the first ncurves curves of a batch, full grid each."""
    import torch
    from paper_1112_1701_b300 import bls
    sub = batch.subset(range(min(ncurves, len(batch))))
    pdev = bls.curves_from_batch(sub, device="cuda")
    with bls.Plan(nb=sub.nb[0], qmin=sub.qmin, qmax=sub.qmax, algo="plain_f64",
                  stream=torch.cuda.current_stream().cuda_stream) as pp:
        pp.search(pdev[:1])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pp.search(pdev)
        torch.cuda.synchronize()
        dtp = time.perf_counter() - t0
    rate = sub.point_freqs() / dtp
    return {"value": rate, "unit": UNIT,
            "sample": f"{len(sub)} curves x full grid, one launch per curve",
            "speedup_of_value": value / rate}


def run_precision(args):
    """Precision study on the three-year workload (3000 points over 1095 days with seasonal
    gaps, up to 5475 cycles at the highest frequency): every phase mode {f64, df32, f32} x
    sum mode {f32, kahan} against the FP64 oracle on a subset of curves, full grid.
    Reports the phase-bin mismatch rate (sampled frequencies, all points), the SR relative
    error over the spectrum, the peak-depth error, and best-frequency disagreements."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    st = precision_study(args.prec_curves, args.nf_prec, args.prec_bin_curves,
                         args.prec_bin_freqs)
    line = {"metric": "BLS precision study", "data": "synthetic", "n_gpus": 1,
            "config": st.pop("config"), **st}
    print(json.dumps(line), flush=True)
    return 0


def precision_study(ncurves, nf_grid, bin_curves, bin_freqs):
    """The precision study's measurements (see run_precision) as one object."""
    import oracle
    from paper_1112_1701_b300 import bls
    b = synth.config3(ncurves=ncurves, nf=nf_grid)
    nb = b.nb[0]
    kmin, kmax = oracle.kminmax(nb, b.qmin, b.qmax)
    cis = bls.curves_from_batch(b)
    nf = b.grids[0].nf
    cores = os.cpu_count() or 1
    cur = [dict(t=c.t, y=c.y, dy=c.dy, nb=nb, kmin=kmin, kmax=kmax, fmin=g.fmin, df=g.df,
                nf=g.nf) for c, g in zip(b.curves, b.grids)]
    t0 = time.perf_counter()
    opk, oP = oracle.bls_many(cur, nthreads=cores, topk=1, want_power=True)
    t_oracle = time.perf_counter() - t0
    osr = np.sqrt(oP).reshape(len(b), nf)
    sumwx2 = np.array([oracle.prep(c.t, c.y, c.dy)[3][3] for c in b.curves])
    # frequencies for the bin comparison: spread over the grid, the top 1% dense
    js = sorted(set(np.linspace(0, nf - 1, bin_freqs // 2).astype(int).tolist()
                    + np.linspace(int(0.99 * nf), nf - 1, bin_freqs // 2).astype(int).tolist()))
    freqs = [oracle.freq(j, b.grids[0].fmin, b.grids[0].df) for j in js]
    obins = [oracle.bins(c.t, freqs, nb) for c in b.curves[:bin_curves]]
    rows = []
    for phase in ("f64", "df32", "fx64", "f32"):
        for sm in ("fixed", "f32", "kahan"):
            with bls.Plan(nb=nb, qmin=b.qmin, qmax=b.qmax, topk=1, phase=phase, sum=sm) as p:
                spec = np.zeros(len(b) * nf, np.float32)
                pk = p.search(cis, spectrum=spec)
                mism = 0
                tot = 0
                for q in range(len(obins)):
                    bg = p.debug_fold(cis[q], js)
                    mism += int((bg != obins[q]).sum())
                    tot += bg.size
            gsr = spec.reshape(len(b), nf).astype(np.float64)
            rel = np.abs(gsr - osr) / np.maximum(osr, 1e-300)
            tol = 1e-5 * osr + 1e-6 * np.sqrt(sumwx2)[:, None]
            sig = osr > 1e-3 * osr.max(axis=1, keepdims=True)
            dj, dj_sep, ddepth = 0, 0, []
            for q in range(len(b)):
                jo = opk[q][0].j
                jg = int(pk[q, 0]["j"])
                srt = np.sort(osr[q])
                separated = (srt[-1] - srt[-2]) > 1e-5 * srt[-1]
                if jg != jo:
                    dj += 1
                    dj_sep += int(separated)
                else:
                    ddepth.append(abs(float(pk[q, 0]["depth"]) - opk[q][0].depth))
            rows.append({"phase": phase, "sum": sm,
                         "bin_mismatch_rate": mism / max(tot, 1),
                         "sr_rel_err_median": float(np.median(rel[sig])),
                         "sr_rel_err_p99": float(np.percentile(rel[sig], 99)),
                         "sr_rel_err_max": float(rel[sig].max()),
                         "frac_outside_parity_tol": float((np.abs(gsr - osr) > tol).mean()),
                         "depth_abs_err_max_same_j": max(ddepth) if ddepth else None,
                         "best_j_disagree": dj, "best_j_disagree_separated": dj_sep})
    return {"config": {"workload": f"three-year baseline: {len(b)} curves x 3000 points over "
                                   f"1095 d, seasonal gaps, {nf} freqs uniform in [0.05, 5]/d, "
                                   f"nb={nb}, q {b.qmin}-{b.qmax}",
                       "bin_check": f"{len(obins)} curves x {len(js)} frequencies x all points",
                       "oracle_s": round(t_oracle, 1), "oracle_threads": cores},
            "sr_rel_err_over": "frequencies with oracle SR > 1e-3 of the curve's maximum",
            "modes": rows}


def run_efficiency(args):
    """Detection-efficiency workload: the eclipse-window efficiency of a 60-night survey
    field (20-minute cadence through ~5-hour nightly windows, 30% of nights lost) at 20,000
    frequencies in [0.1, 10] 1/d and 256 eclipse phases, eclipses 0.04 d long; plus the
    injection-recovery curve on the same cadence (16 injections per period, 3% eclipses
    at 1% noise, batched search on 20,000 frequencies in [0.1, 5] 1/d)."""
    import torch
    import oracle
    from paper_1112_1701_b300 import bls, efficiency
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    t = synth.survey_cadence(seed=6, nights=60)
    nf, nphi, D = args.eff_nf, 256, 0.04
    fmin, fmax = 0.1, 10.0
    df = (fmax - fmin) / (nf - 1)
    td = torch.tensor(t, device="cuda")
    eff = torch.zeros(nf, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        bls.window_efficiency(td, nphi, fmin=fmin, df=df, nf=nf, duration=D, eff=eff,
                              stream=stream.cuda_stream)
    ts = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        bls.window_efficiency(td, nphi, fmin=fmin, df=df, nf=nf, duration=D, eff=eff,
                              stream=stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    units = len(t) * nf * nphi
    value = units / (ms / 1000.0)
    # FP64-pipe roofline: 3 FP64 instructions per (time, phase, frequency): u = v - phi,
    # u + 1/2, r = u - c (the floor and |r| <= h are integer operations on the bits); peak =
    # the part's nominal 1.25 TFLOP/s FP64 (0.625 T FP64 instructions/s)
    peak = 0.625e12 / 3.0
    # the oracle (one thread) on a bounded sample: the first kf frequencies; its result
    # also checks the timed configuration's output there
    kf = max(1, min(nf, int(args.eff_cpu_freqs)))
    t0 = time.perf_counter()
    eo, _ = oracle.window(t, nphi, fmin=fmin, df=df, nf=kf, duration=D)
    dt_cpu = time.perf_counter() - t0
    parity = bool(np.array_equal(eff.cpu().numpy()[:kf], eo))
    # injection-recovery curve
    periods = np.exp(np.linspace(np.log(0.25), np.log(9.0), 12))
    tr0 = time.perf_counter()
    ec = efficiency.detection_efficiency(t, periods, 16, duration=D, depth=0.03, sigma=0.01,
                                         nf=20000, nphi=nphi)
    dt_rec = time.perf_counter() - tr0
    line = {"metric": "eclipse-window evals/s", "value": value,
            "unit": "time*phase*freq/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"eclipse-window efficiency: 60-night field, {len(t)} "
                                   f"exposures, {nf} freqs in [0.1, 10]/d, {nphi} phases, "
                                   f"eclipse 0.04 d", "l2": "inputs (4.6 KB) stay in L2"},
            "roofline": {"bound": "alu", "achieved": value, "peak": peak,
                         "unit": "time*phase*freq/s (FP64 pipe, 3 instructions each)",
                         "frac": value / peak, "traffic": None,
                         "peak_source": "nominal 1.25 TFLOP/s FP64 of the part"},
            "gpu_launches": args.steps * 2,
            "parity_sampled_freqs": {"checked": kf, "equal": parity},
            "cpu_baseline": {"value": len(t) * kf * nphi / dt_cpu, "unit": "time*phase*freq/s",
                             "cores": 1, "kind": "oracle",
                             "sample": f"{kf} of {nf} frequencies, FP64 C oracle, one thread, "
                                       f"{dt_cpu:.1f} s"},
            "recovery_curve": {"periods_d": [round(float(p), 4) for p in periods],
                               "window": [float(x) for x in ec.window],
                               "recovered": [float(x) for x in ec.recovery],
                               "injections_per_period": 16, "wall_s": round(dt_rec, 2)}}
    print(json.dumps(line), flush=True)
    return 0


def run_variability(args):
    """High-variability pre-filter on one survey field: 11 chips x 5000 stars x 500 epochs
    (magnitudes 14-20.5, 3 mmag floor plus photon noise, 1% eclipsing variables)."""
    import torch
    import oracle
    from paper_1112_1701_b300 import bls
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    c = synth.chip_catalog(nchips=11, stars_per_chip=args.var_stars, npts=500, seed=12)
    off = torch.tensor(c.off, device="cuda")
    m = torch.tensor(c.m, device="cuda")
    chip = torch.tensor(c.chip, device="cuda")
    out = torch.zeros(len(c.chip) * bls.VAR_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(3, args.warmup)):
        bls.variability(off, m, chip, c.nchips, out=out, stream=stream.cuda_stream)
    ts = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        bls.variability(off, m, chip, c.nchips, out=out, stream=stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    npts = int(c.off[-1])
    g = out.cpu().numpy().view(bls.VAR_DTYPE)
    # the oracle (one thread) on the first chip, which also checks that chip's output
    first = np.flatnonzero(c.chip == 0)
    k = len(first)
    t0 = time.perf_counter()
    o = oracle.variability(c.off[:k + 1], c.m[:c.off[k]], c.chip[:k], 1)
    dt_cpu = time.perf_counter() - t0
    # the GPU sums in a warp's order, the oracle sequentially: values within the FP64
    # summation bound, decisions equal away from their thresholds (tests check both)
    parity = {"flags_equal": int(np.sum(g["flag"][:k] == o["flag"])), "stars": k,
              "rms_max_rel_diff": float(np.max(np.abs(g["rms"][:k] - o["rms"]) /
                                               np.maximum(o["rms"], 1e-300)))}
    flags = g["flag"].astype(bool)
    line = {"metric": "variability pre-filter points/s", "value": npts / (ms / 1000.0),
            "unit": "points/s", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": ms, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"one survey field: 11 chips x {args.var_stars} stars x 500 "
                                   f"epochs ({npts} points, {4 * npts / 1e6:.0f} MB of FP32 "
                                   f"magnitudes)", "l2": "flushed (256 MiB write) before every step"},
            "roofline": {"bound": "hbm", "achieved": 4.0 * npts / (ms / 1000.0) / 1e9,
                         "unit": "GB/s", "traffic": None,
                         "note": "algorithmic bytes = the 4-byte magnitudes, read once"},
            "gpu_launches": 5 * args.steps,
            "flagged": int(flags.sum()), "variables_flagged": int(flags[c.variable].sum()),
            "variables": int(c.variable.sum()),
            "parity_first_chip": parity,
            "cpu_baseline": {"value": int(c.off[k]) / dt_cpu, "unit": "points/s", "cores": 1,
                             "kind": "oracle",
                             "sample": f"chip 0 ({k} stars), FP64 C oracle, one thread, "
                                       f"{dt_cpu:.2f} s"}}
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    line["roofline"]["peak"] = hbm
    line["roofline"]["frac"] = line["roofline"]["achieved"] / hbm
    line["roofline"]["peak_source"] = f"{src} HBM copy bandwidth"
    print(json.dumps(line), flush=True)
    return 0


def run_unbinned(args):
    """Unbinned (edge-to-edge) search on a subset of the batched workload's curves (64
    curves, N log-uniform 500-5000, 5000 frequencies in [0.1, 5] 1/d, q 0.005-0.15),
    against the binned search of the same curves and the oracle on one curve."""
    import torch
    import oracle
    from paper_1112_1701_b300 import bls
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    b = synth.config2(args.ub_curves, nf=args.ub_nf)
    dev = bls.curves_from_batch(b, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    units = b.point_freqs()

    def timed(plan):
        for _ in range(max(3, args.warmup)):
            plan.search(dev)
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            plan.search(dev)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    with bls.Plan(nb=NB, qmin=QMIN, qmax=QMAX, algo="unbinned", stream=stream.cuda_stream) as p:
        ms_u = timed(p)
    with bls.Plan(nb=NB, qmin=QMIN, qmax=QMAX, stream=stream.cuda_stream) as p:
        ms_b = timed(p)
    # box evaluations of the unbinned search: for each start, the points within QMAX of
    # phase -- about qmax * N per start (the exact count depends on the phases)
    evals = sum(len(c.t) * int(QMAX * len(c.t)) * g.nf for c, g in zip(b.curves, b.grids))
    c0, g0 = b.curves[0], b.grids[0]
    kf = max(1, min(g0.nf, args.ub_cpu_freqs))
    t0 = time.perf_counter()
    oracle.ubls(c0.t, c0.y, c0.dy, QMIN, QMAX, fmin=g0.fmin, df=g0.df, nf=kf)
    dt_cpu = time.perf_counter() - t0
    value = units / (ms_u / 1000.0)
    peak = 148 * 128 * 2032e6 / 7.0
    line = {"metric": "unbinned BLS point x freq evals/s", "value": value, "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_u,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"unbinned BLS: {len(b)} curves, N log-uniform 500-5000, "
                                   f"{b.grids[0].nf} freqs in [0.1, 5]/d, q {QMIN}-{QMAX}",
                       "l2": "flushed (256 MiB write) before every step"},
            "box_evals_per_s": evals / (ms_u / 1000.0),
            "roofline": {"bound": "alu", "achieved": evals / (ms_u / 1000.0), "peak": peak,
                         "unit": "box evaluations/s (7 FP32 lane-ops each, 148 SMs x 128 "
                                 "lanes x 2032 MHz)",
                         "frac": evals / (ms_u / 1000.0) / peak, "traffic": None},
            "binned_same_curves": {"ms_per_step": ms_b, "value": units / (ms_b / 1000.0)},
            "gpu_launches": 3 * args.steps,
            "cpu_baseline": {"value": len(c0.t) * kf / dt_cpu, "unit": UNIT, "cores": 1,
                             "kind": "oracle",
                             "sample": f"curve 0 ({len(c0.t)} points) x {kf} frequencies, "
                                       f"one thread, {dt_cpu:.1f} s"}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(batch, args):
    return {"workload": f"batched BLS: {len(batch)} curves, N log-uniform 500-5000 over 60 "
                        f"nights, {batch.grids[0].nf} freqs uniform in [0.1, 5]/d, nb={NB}, "
                        f"q {QMIN}-{QMAX}",
            "ncurves": len(batch), "nf": batch.grids[0].nf, "nb": NB,
            "points": int(sum(len(c.t) for c in batch.curves)),
            "l2": "flushed (256 MiB write) before every step, inside the timed region",
            "inputs": "device-resident for value; pinned host for e2e",
            "parallelism": f"replicas x{args.gpus}"}


# Unit rates measured on B300 by paper_1112_1701_b300/csrc/probes.cu (profiles/probes_b300.md):
# shared-memory bytes and FP32 FMAs per SM per clock.
PROBE_SMEM_B_PER_CLK = 127.0
PROBE_FP32_PER_CLK = 126.0


def roofline(units, evals, launches_per_step, fold_ms, sms, clk_mhz, run_mhz, kernel):
    """Roofline of the fold-bin-sweep kernel: loop A moves 16 B of shared memory per point x
    frequency (two 8-byte read-modify-writes) at the probed 127 B/clk/SM; loop B takes 7
    FP32 operations per box evaluation at the probed 126 per clk per SM.  The model time of
    one launch is the sum of the two; achieved and peak are counted in lane-op equivalents
    (16 per point x frequency, 7 per box), so frac = model time / measured time."""
    u = units / max(1.0, launches_per_step)
    e = evals / max(1.0, launches_per_step)
    ops = 16.0 * u + 7.0 * e

    def model_s(mhz):
        return (16.0 * u / PROBE_SMEM_B_PER_CLK + 7.0 * e / PROBE_FP32_PER_CLK) / (sms * mhz * 1e6)

    t = fold_ms / 1000.0
    out = {"bound": "alu", "achieved": ops / t / 1e12, "peak": ops / model_s(clk_mhz) / 1e12,
           "unit": "T lane-op equivalents/s (16 per point x freq of shared-memory traffic, 7 "
                   "FP32 ops per box evaluation)",
           "frac": model_s(clk_mhz) / t, "traffic": None, "kernel": kernel,
           "peak_source": f"probes (127 B/clk/SM shared memory, 126 FP32 FMA/clk/SM) x {sms} "
                          f"SMs x {clk_mhz:.0f} MHz (max SM clock of the measured peaks)",
           "model_ms_per_launch": 1000 * model_s(clk_mhz), "fold_ms_per_launch": fold_ms,
           "loop_a_units_per_launch": u, "loop_b_units_per_launch": e}
    if run_mhz:
        out["frac_at_run_clock"] = model_s(run_mhz) / t
    return out


def measure(batch, topk, args, ctx, tune=True, e2e=True, steps=None, warmup=None, sums="fixed"):
    """Device-timed and end-to-end search of one batch: warm-up, then `steps` searches of
    the device-resident packed batch between barriers (CUDA events on the plan's stream,
    L2 flushed before each), then the same through pinned host buffers (wall clock)."""
    import torch
    from paper_1112_1701_b300 import autotune, bls
    steps = steps or args.steps
    warmup = args.warmup if warmup is None else warmup
    nb = batch.nb[0]
    stream = ctx["stream"]
    units = batch.point_freqs()
    evals = box_evals(batch)
    dev = bls.curves_from_batch(batch, device="cuda")
    tuned, launch_kw = None, {}
    if tune and not args.no_autotune:
        t0 = time.perf_counter()
        res = autotune.tune(dev, nb, batch.qmin, batch.qmax, stream=stream.cuda_stream,
                            cache=autotune.TuneCache(None), sums=sums)
        tuned = dict(res.to_json(), tuning_s=time.perf_counter() - t0)
        launch_kw = res.best.plan_kwargs()
    plan = bls.Plan(nb=nb, qmin=batch.qmin, qmax=batch.qmax, topk=topk, sum=sums,
                    stream=stream.cuda_stream, **launch_kw)
    flush = ctx["flush"]
    devp = bls.packed_from_batch(batch, device="cuda")
    for _ in range(warmup):
        flush.zero_()
        plan.search(devp)
    plan.profile(reset=True)
    clocks = Clocks(ctx["local"])
    clocks.start()
    ctx["barrier"]()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        flush.zero_()
        plan.search(devp)
    e1.record(stream)
    ctx["barrier"]()
    clk = clocks.stop()
    ms = ctx["max_over_ranks"](e0.elapsed_time(e1))
    prof = plan.profile(reset=True)
    world = ctx["world"]
    ms_step = ms / steps
    out = {"value": units * world / (ms_step / 1000.0), "ms_per_step": ms_step, "clocks": clk,
           "gpu_launches": int(prof["kernel_launches"]),
           "box_evals_per_s": evals * world / (ms_step / 1000.0),
           "kernel_ms": {"prep": prof["prep_ms"] / steps, "fold_sweep": prof["fold_ms"] / steps,
                         "reduce": prof["reduce_ms"] / steps},
           "launch": dict(launch_kw, source="autotuner", tile_shape=plan.tile_shape(), sums=sums)
                     if tuned else {"source": "library rules", "tile_shape": plan.tile_shape(),
                                    "sums": sums},
           "plan": plan, "dev": dev, "units": units, "evals": evals}
    if tuned:
        out["autotune"] = tuned
    peaks, _ = measured_peaks()
    props = torch.cuda.get_device_properties(ctx["local"])
    fold_ms = prof["fold_ms"] / max(1, prof["fold_launches"])
    out["roofline"] = roofline(units, evals, prof["fold_launches"] / max(1, steps), fold_ms,
                               props.multi_processor_count, float(peaks.get("sm_max_mhz", 2032.0)),
                               clk.get("sm_mhz"),
                               "fold_sweep_ws_kernel" if out["launch"]["tile_shape"]["fold_kernel"] == "ws"
                               else "fold_sweep_kernel")
    if e2e and not args.no_e2e:
        hostc = bls.packed_from_batch(batch, pinned=True)
        for _ in range(max(1, min(warmup, 2))):
            plan.search(hostc)
        ctx["barrier"]()
        t0 = time.perf_counter()
        for _ in range(steps):
            plan.search(hostc)
        ctx["barrier"]()
        wall = ctx["max_over_ranks"](time.perf_counter() - t0)
        npts = int(hostc.keep[0].numel())
        out["e2e"] = {"value": units * world * steps / wall, "unit": UNIT,
                      "h2d_bytes_per_step": npts * (8 + 4 + 4),
                      "d2h_bytes_per_step": len(batch) * topk * bls.C.sizeof(bls.PeakStruct)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--survey-curves", type=int, default=2048,
                    help="curves of the survey sweep per rank (headline workload)")
    ap.add_argument("--survey-nf", type=int, default=200000)
    ap.add_argument("--ncurves", type=int, default=1024, help="batched workload: curves")
    ap.add_argument("--nf", type=int, default=50000, help="batched workload: frequencies")
    ap.add_argument("--ref-curves", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-shapes", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched workload object")
    ap.add_argument("--no-kahan", action="store_true", help="skip the Kahan-sums object")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the single-curve and precision objects")
    ap.add_argument("--kahan-steps", type=int, default=3)
    ap.add_argument("--no-serving", action="store_true", help="skip the serving object")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the library's launch rules instead of the autotuner's choice")
    ap.add_argument("--plain-curves", type=int, default=4,
                    help="curves of the plain FP64 baseline timing (0 = skip)")
    ap.add_argument("--serving", action="store_true", help="run the serving benchmark alone")
    ap.add_argument("--requests", type=int, default=600)
    ap.add_argument("--plain-requests", type=int, default=100)
    ap.add_argument("--loads", type=float, nargs="*", default=[0.5, 0.7, 0.9])
    ap.add_argument("--step-units", type=int, default=0,
                    help="serving: point x frequency units per scheduler step (0: default)")
    ap.add_argument("--precision", action="store_true", help="run the precision study")
    ap.add_argument("--prec-curves", type=int, default=16)
    ap.add_argument("--nf-prec", type=int, default=200000)
    ap.add_argument("--prec-bin-curves", type=int, default=4)
    ap.add_argument("--prec-bin-freqs", type=int, default=400)
    ap.add_argument("--efficiency", action="store_true",
                    help="run the detection-efficiency workload")
    ap.add_argument("--eff-nf", type=int, default=20000)
    ap.add_argument("--eff-cpu-freqs", type=int, default=6000)
    ap.add_argument("--variability", action="store_true",
                    help="run the high-variability pre-filter workload")
    ap.add_argument("--var-stars", type=int, default=5000)
    ap.add_argument("--unbinned", action="store_true", help="run the unbinned search workload")
    ap.add_argument("--ub-curves", type=int, default=64)
    ap.add_argument("--ub-nf", type=int, default=5000)
    ap.add_argument("--ub-cpu-freqs", type=int, default=200)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.serving:
        return run_serving(args)
    if args.precision:
        return run_precision(args)
    if args.efficiency:
        return run_efficiency(args)
    if args.variability:
        return run_variability(args)
    if args.unbinned:
        return run_unbinned(args)

    import torch
    from paper_1112_1701_b300 import shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if not dist:
            return x
        t = torch.tensor([x], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    ctx = {"stream": torch.cuda.current_stream(), "local": local, "world": world,
           "barrier": barrier, "max_over_ranks": max_over_ranks,
           "flush": torch.empty(256 << 20, dtype=torch.uint8, device="cuda")}

    # ---- headline: the survey sweep (weak scaling: every rank its own curves)
    batch = headline_batch(args, rank, world)
    topk = 5
    m = measure(batch, topk, args, ctx)
    line = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": headline_config(batch, args, world),
            "roofline": m["roofline"], "clocks": m["clocks"], "gpu_launches": m["gpu_launches"],
            "box_evals_per_s": m["box_evals_per_s"], "kernel_ms": m["kernel_ms"]}
    line["config"]["launch"] = m["launch"]
    if (NCU_TRAFFIC["kernel_sha256"] == kernel_sha() and len(batch) == NCU_TRAFFIC["ncurves"]
            and batch.grids[0].nf == 200000):
        line["roofline"]["traffic"] = NCU_TRAFFIC["bytes_per_launch"]
    line["config"]["full_100k_curves_s_extrapolated"] = m["ms_per_step"] / 1000.0 * 100000 / len(batch)
    if "e2e" in m:
        line["e2e"] = m["e2e"]
    if "autotune" in m:
        line["autotune"] = m["autotune"]
    plan = m["plan"]
    last = plan.search(m["dev"])
    if rank == 0:
        inj = [i for i, c in enumerate(batch.curves) if c.truth is not None]
        rec = 0
        for i in inj:
            P = batch.curves[i].truth["period"]
            got = [float(x["period"]) for x in last[i] if x["j"] >= 0]
            rec += any(abs(g - P) / P < 0.01 or abs(2 * g - P) / P < 0.01 or
                       abs(g - 2 * P) / P < 0.01 for g in got)
        line["injected"] = {"curves": len(inj), "recovered_in_top5": rec}
    # the per-curve records of all ranks, gathered on rank 0 (outside the timed region)
    gathered = shard.search_curve_shards(world * len(batch), lambda a, b: last)
    if rank == 0:
        line["gathered_peaks"] = int(gathered.shape[0])
    plan.close()
    if args.plain_curves > 0 and rank == 0:
        line["plain_f64_gpu"] = plain_f64_sample(batch, args.plain_curves, m["value"] / world)
    del m

    # ---- the same workload with Kahan-compensated FP32 histograms and box sums
    if not args.no_kahan:
        mk = measure(batch, topk, args, ctx, e2e=False, steps=args.kahan_steps, warmup=1,
                     sums="kahan")
        line["kahan_sums"] = {"value": mk["value"], "unit": UNIT, "ms_per_step": mk["ms_per_step"],
                              "steps": args.kahan_steps, "warmup": 1,
                              "roofline_frac": mk["roofline"]["frac"],
                              "kernel_ms": mk["kernel_ms"], "launch": mk["launch"],
                              "note": "same roofline model (16 B per point x frequency counted "
                                      "as for plain sums; the Kahan entries move 32 B)"}
        mk["plan"].close()
        del mk

    # ---- secondary: the batched workload (1024 curves x 50,000 frequencies, nb = 200)
    if not args.no_batched:
        b2 = synth.config2(args.ncurves, nf=args.nf, first=rank * args.ncurves)
        m2 = measure(b2, 1, args, ctx)
        sec = {"config": workload_config(b2, args), "value": m2["value"], "unit": UNIT,
               "ms_per_step": m2["ms_per_step"], "roofline": m2["roofline"],
               "kernel_ms": m2["kernel_ms"], "gpu_launches": m2["gpu_launches"],
               "clocks": m2["clocks"], "launch": m2["launch"]}
        if "e2e" in m2:
            sec["e2e"] = m2["e2e"]
        if rank == 0 and not args.no_shapes:
            p2, dev2, flush, stream = m2["plan"], m2["dev"], ctx["flush"], ctx["stream"]

            def timed(fn):
                best = None
                for _ in range(3):
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    fn()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    best = e0.elapsed_time(e1) if best is None else min(best, e0.elapsed_time(e1))
                return best
            t_plain = timed(lambda: p2.search(dev2))
            t_shape = timed(lambda: p2.search_shapes(dev2))
            sec["shape_refit"] = {"extra_ms_per_step": t_shape - t_plain,
                                  "grid": "17 centres x 13 widths x 6 ingress fractions",
                                  "peaks": len(b2)}
        if args.plain_curves > 0 and rank == 0:
            sec["plain_f64_gpu"] = plain_f64_sample(b2, 8, m2["value"] / world)
        m2["plan"].close()
        line["batched"] = sec
        del m2

    # ---- serving: p50/p99 at fractions of saturation, ours and the plain FP64 kernel
    if rank == 0 and world == 1 and not args.no_serving:
        line["serving"] = serving_measurement(args.requests, args.plain_requests, args.loads,
                                              args.step_units)

    # ---- the plain single-curve workload and a reduced precision study
    if rank == 0 and world == 1 and not args.no_extras:
        line["plain_curve"] = plain_curve_measurement()
        line["precision"] = precision_study(2, 200000, 2, 200)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(batch)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
