"""Served form: requests submitted while others are on the GPU, chunk by
chunk, give exactly the result each gives alone (and the oracle's)."""
import math
import random
import threading
import time

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1907_03620_gb300 as R
from paper_1907_03620_gb300.serve import RasterServer

pytestmark = pytest.mark.gpu


def _same(res, ref):
    s = res.sorted()
    assert s.key.cpu().numpy().tolist() == ref.key.tolist()
    assert s.count.cpu().numpy().tolist() == ref.count.astype(np.int64).tolist()
    assert s.cid.cpu().numpy().tolist() == ref.cid.tolist()
    assert res.n_clusters == ref.n_clusters
    assert res.n_distinct == ref.n_tiles
    assert res.n_significant == ref.n_significant


def _requests(count, seed, hi=300_000):
    ws = gen.batch_instances(count=count, seed=seed, lo=10, hi=hi)
    rng = random.Random(seed)
    return [(i, w, gen.points(w), rng.randint(1, 8)) for i, w in enumerate(ws)]


def _drain(srv, expect, timeout_s=120.0):
    got = {}
    t0 = time.time()
    while len(got) < expect:
        r = srv.poll(wait_ms=50)
        if r is not None:
            rid, res, lat = r
            got[rid] = (res, lat)
            srv.release(rid)
        assert time.time() - t0 < timeout_s, "requests did not complete"
    return got


def test_results_same_alone_and_in_the_mix():
    reqs = _requests(48, seed=61)
    srv = RasterServer(table_slots=1 << 27, result_rows=1 << 24, max_active=64)
    dev = {i: torch.from_numpy(xy).cuda() for i, w, xy, c in reqs}
    # interleave: submit everything, then push chunks round-robin from another thread
    for i, w, xy, c in reqs:
        srv.submit(i, w.precision, w.tau, w.mu, w.n, c)

    def pusher():
        pending = {i: list(gen.chunk_bounds(w.n, c)) for i, w, xy, c in reqs}
        while pending:
            for i in list(pending):
                lo, hi = pending[i].pop(0)
                srv.push(i, dev[i][lo:hi])
                if not pending[i]:
                    del pending[i]
            time.sleep(0.001)

    th = threading.Thread(target=pusher)
    th.start()
    got = _drain(srv, len(reqs))
    th.join()
    assert srv.stats()["steps"] >= 2
    for i, w, xy, c in reqs:
        ref, _ = oracle.raster(xy, w.precision, w.tau, w.mu)
        _same(got[i][0], ref)
        # and alone, through a plain handle
        with R.Raster(w.precision, w.tau, w.mu) as h:
            h.contract(dev[i])
            alone = h.agglomerate()
        a, b = alone.sorted(), got[i][0].sorted()
        assert torch.equal(a.key, b.key) and torch.equal(a.count, b.count) and torch.equal(a.cid, b.cid)
    srv.close()


def test_admission_waits_for_memory_and_completes_all():
    reqs = _requests(24, seed=62, hi=120_000)
    biggest = max(w.n for i, w, xy, c in reqs)
    cap = 4096
    while cap * 0.75 < biggest:
        cap *= 2
    # room for about two of the largest requests at a time
    srv = RasterServer(table_slots=2 * cap, result_rows=2 * biggest, max_active=8)
    dev = {i: torch.from_numpy(xy).cuda() for i, w, xy, c in reqs}
    for i, w, xy, c in reqs:
        srv.submit(i, w.precision, w.tau, w.mu, w.n, c)
        for lo, hi in gen.chunk_bounds(w.n, c):
            srv.push(i, dev[i][lo:hi])
    peak_waiting = max(srv.stats()["waiting"], 0)
    got = _drain(srv, len(reqs))
    assert peak_waiting > 0  # some had to wait for memory
    for i, w, xy, c in reqs:
        ref, _ = oracle.raster(xy, w.precision, w.tau, w.mu)
        _same(got[i][0], ref)
    srv.close()


def test_faulty_request_leaves_others_unchanged():
    reqs = _requests(10, seed=63, hi=50_000)
    srv = RasterServer(table_slots=1 << 24, result_rows=1 << 22, max_active=32)
    dev = {i: torch.from_numpy(xy).cuda() for i, w, xy, c in reqs}
    bad = np.array([[0.5, 0.5], [math.nan, 1.0], [0.25, math.inf], [0.5, 0.51]] * 50)
    bad_d = torch.from_numpy(bad).cuda()
    srv.submit(999, 2, 2, 1, bad.shape[0], 2)
    srv.push(999, bad_d[:100])
    for i, w, xy, c in reqs:
        srv.submit(i, w.precision, w.tau, w.mu, w.n, c)
        for lo, hi in gen.chunk_bounds(w.n, c):
            srv.push(i, dev[i][lo:hi])
    srv.push(999, bad_d[100:])
    got = _drain(srv, len(reqs) + 1)
    assert got[999][0].status == R._native.E_RANGE
    ref_bad, _ = oracle.raster(bad, 2, 2, 1)
    _same(got[999][0], ref_bad)
    for i, w, xy, c in reqs:
        assert got[i][0].status == 0
        ref, _ = oracle.raster(xy, w.precision, w.tau, w.mu)
        _same(got[i][0], ref)
    # argument errors are refused on the host, and a request that could never
    # fit the arenas is refused at submit
    with pytest.raises(R.RasterError) as e:
        srv.submit(5000, 2, 5, 4, 10**9, 1)
    assert e.value.status == R._native.E_LIMIT
    srv.submit(5001, 2, 5, 4, 10, 1)
    with pytest.raises(R.RasterError):
        srv.push(5001, torch.zeros((11, 2), dtype=torch.float64, device="cuda"))  # more points than announced
    srv.push(5001, torch.zeros((10, 2), dtype=torch.float64, device="cuda"))
    got = _drain(srv, 1)
    assert got[5001][0].n_distinct == 1
    assert srv.stats()["status"] == 0
    srv.close()


def test_zero_point_request():
    srv = RasterServer(table_slots=1 << 16, result_rows=1 << 12, max_active=4)
    srv.submit(1, 2, 5, 4, 0, 1)
    srv.push(1, torch.empty((0, 2), dtype=torch.float64, device="cuda"))
    got = _drain(srv, 1)
    assert got[1][0].key.numel() == 0 and got[1][0].n_clusters == 0
    srv.close()


def test_served_mix_bit_exact_against_stored_oracle():
    """A mix spanning the served workload's range -- sizes 1e4..2e7, 1..8
    chunks, every (p, tau, mu) combination -- submitted at once with chunks
    pushed round-robin: every request's rows hash to the oracle's stored
    digest (tests/golden/digests.py); a differing request is re-run through
    the oracle to show the first wrong row."""
    import os
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    import digests
    g = digests.load("served_mix")
    mix = digests.served_mix(g["seed"])
    assert len(mix) == len(g["requests"]) == 36
    dev = {j: torch.from_numpy(gen.points(w)).cuda() for j, (w, c) in enumerate(mix)}
    srv = RasterServer(max_active=64)
    for j, (w, c) in enumerate(mix):
        srv.submit(j, w.precision, w.tau, w.mu, w.n, c)
    pending = {j: list(gen.chunk_bounds(w.n, c)) for j, (w, c) in enumerate(mix)}
    while pending:
        for j in list(pending):
            lo, hi = pending[j].pop(0)
            srv.push(j, dev[j][lo:hi])
            if not pending[j]:
                del pending[j]
    got = _drain(srv, len(mix), timeout_s=300.0)
    for j, (w, c) in enumerate(mix):
        res, want = got[j][0], g["requests"][j]
        assert (w.n, c, w.precision, w.tau, w.mu) == (want["n"], want["chunks"], want["precision"], want["tau"],
                                                      want["mu"])
        assert res.status == 0
        stats = (res.n_distinct, res.n_significant, res.n_clusters, res.key.numel())
        assert stats == (want["n_tiles"], want["n_significant"], want["n_clusters"], want["n_kept"]), j
        h = digests.rows_digest(res.key.cpu().numpy(), res.count.cpu().numpy(), res.cid.cpu().numpy())
        if h != want["rows"]:
            ref, _ = oracle.raster(dev[j].cpu().numpy(), w.precision, w.tau, w.mu)
            _same(res, ref)
            pytest.fail(f"request {j} differs from the stored oracle digest")
    st = srv.stats()
    assert st["gpu_us"] > 0 and st["steps"] > 0 and st["refused"] == 0
    srv.close()
