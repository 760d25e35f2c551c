"""Multi-rank sharding of the batched search, on CPU with the gloo backend (world size 2).

The ranks stand in for GPUs: each searches its shard with the FP64 oracle (the host logic
under test is the split, the gather and the merge, not the search).  The sharded results
must equal the single-process oracle run over the whole batch or grid, record for record."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1112_1701_b300 import bls, shard, synth

NB = 100


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _records(peaks):
    """OraclePeak list -> PEAK_DTYPE array."""
    out = np.zeros(len(peaks), dtype=bls.PEAK_DTYPE)
    for q, p in enumerate(peaks):
        for f in ("freq", "period", "epoch", "duration", "depth", "snr", "sr", "power", "sde"):
            out[q][f] = getattr(p, f)
        out[q]["j"], out[q]["i1"], out[q]["k"] = p.j, p.i1, p.k
    return out


def _batch():
    return synth.config2(ncurves=7, nf=300, seed=21)


def _curve_search(b, kmin, kmax, topk):
    def search(lo, hi):
        cur = [dict(t=b.curves[i].t, y=b.curves[i].y, dy=b.curves[i].dy, nb=NB, kmin=kmin,
                    kmax=kmax, fmin=b.grids[i].fmin, df=b.grids[i].df, nf=b.grids[i].nf)
               for i in range(lo, hi)]
        if not cur:
            return np.zeros((0, topk), dtype=bls.PEAK_DTYPE)
        pk, _ = oracle.bls_many(cur, nthreads=1, topk=topk)
        return np.stack([_records(p) for p in pk])
    return search


def _freq_search(c, kmin, kmax):
    def search(freqs, lo):
        P, _, _, pk = oracle.bls(c.t, c.y, c.dy, NB, kmin, kmax, freqs=freqs)
        return _records(pk)[0], np.sqrt(P)
    return search


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _batch()
        kmin, kmax = oracle.kminmax(NB, b.qmin, b.qmax)
        allp = shard.search_curve_shards(len(b), _curve_search(b, kmin, kmax, 2))
        g = b.grids[0]
        best = shard.search_freq_shards(g.nf, g.fmin, g.df, _freq_search(b.curves[3], kmin, kmax))
        dist.barrier()
        if rank == 0:
            q.put(("ok", allp.tobytes(), allp.shape, best.tobytes()))
    except Exception as e:  # report to the parent instead of hanging it
        q.put(("err", repr(e)))
        raise
    finally:
        dist.destroy_process_group()


def test_curve_and_frequency_shards_match_single_process():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, port = 2, _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        msg = q.get(timeout=240)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert msg[0] == "ok", msg
    allp = np.frombuffer(msg[1], dtype=bls.PEAK_DTYPE).reshape(msg[2])
    best = np.frombuffer(msg[3], dtype=bls.PEAK_DTYPE)
    b = _batch()
    kmin, kmax = oracle.kminmax(NB, b.qmin, b.qmax)
    ref = _curve_search(b, kmin, kmax, 2)(0, len(b))
    assert np.array_equal(allp, ref)
    c, g = b.curves[3], b.grids[3]
    _, _, _, pk = oracle.bls(c.t, c.y, c.dy, NB, kmin, kmax, fmin=g.fmin, df=g.df, nf=g.nf)
    ref1 = _records(pk[:1])
    others = [f for f in bls.PEAK_DTYPE.names if f != "sde"]
    assert all(np.array_equal(best[f], ref1[f]) for f in others)
    # SDE from merged per-rank moments (the library takes FP32 spectra, as the GPU writes
    # them) vs the oracle's FP64 two-pass sum: each SR value rounds by at most 2^-24 of
    # itself, which moves the mean and the sd by at most that fraction of max SR, so
    # |d SDE| <= 2^-24 max SR (1 + |SDE|) / sd, taken twice over
    sr = np.sqrt(oracle.bls(c.t, c.y, c.dy, NB, kmin, kmax, fmin=g.fmin, df=g.df, nf=g.nf)[0])
    tol = 2 * 2.0 ** -24 * sr.max() * (1 + abs(ref1["sde"][0])) / sr.std()
    assert abs(best["sde"][0] - ref1["sde"][0]) <= tol


def test_ranges_cover_exactly_once():
    for n in (0, 1, 2, 7, 1024, 1025):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = shard.curve_range(n, world, r)
                assert 0 <= lo <= hi <= n
                seen.extend(range(lo, hi))
            assert seen == list(range(n))
    with pytest.raises(ValueError):
        shard.curve_range(4, 2, 2)


def test_sub_grid_is_bit_identical_to_the_uniform_grid():
    fmin, df = 0.1, 4.9 / 49999
    full = np.array([oracle.freq(j, fmin, df) for j in range(0, 50000, 7)])
    sub = np.concatenate([shard.sub_grid(fmin, df, lo, lo + 1) for lo in range(0, 50000, 7)])
    assert np.array_equal(full, sub)


def test_moments_and_sde_against_numpy():
    """The library's moments are numpy's FP64 mean and n x variance of the FP32 values, and
    the SDE is (sr - mean) / population sd (0 for a flat spectrum)."""
    rng = np.random.default_rng(6)
    x = rng.gamma(2.0, 1.0, 777).astype(np.float32)
    n, m, m2 = shard.spectrum_moments(x)
    xd = x.astype(np.float64)
    assert n == 777 and abs(m - xd.mean()) <= 1e-14 * xd.mean()
    assert abs(m2 - xd.var() * 777) <= 1e-12 * xd.var() * 777
    assert abs(bls.sde(5.0, (n, m, m2)) - (5.0 - xd.mean()) / xd.std()) <= 1e-12
    assert bls.sde(3.0, shard.spectrum_moments(np.full(10, 2.0, np.float32))) == 0.0
    assert bls.sde(3.0, (0, 0.0, 0.0)) == 0.0


def test_moments_merge_equals_whole():
    rng = np.random.default_rng(5)
    x = rng.gamma(2.0, 1.0, 1001).astype(np.float32)
    whole = shard.spectrum_moments(x)
    parts = [shard.spectrum_moments(x[a:b]) for a, b in ((0, 300), (300, 300), (300, 1001))]
    n, m, m2 = shard.merge_moments(parts)
    assert n == whole[0] and abs(m - whole[1]) < 1e-12 * whole[1]
    assert abs(m2 - whole[2]) < 1e-10 * whole[2]


def test_merge_order_key():
    a = np.zeros(3, dtype=bls.PEAK_DTYPE)
    a["power"] = [1.0, 2.0, 2.0]
    a["j"] = [0, 9, 5]
    assert int(shard.merge_best(list(a))[0]["j"]) == 5
    a["j"] = [0, 5, 5]
    a["i1"] = [0, 3, 2]
    assert int(shard.merge_best(list(a))[0]["i1"]) == 2


def test_single_process_without_group():
    b = _batch()
    kmin, kmax = oracle.kminmax(NB, b.qmin, b.qmax)
    allp = shard.search_curve_shards(len(b), _curve_search(b, kmin, kmax, 1))
    assert allp.shape == (len(b), 1)
    assert shard.world_info() == (1, 0)
