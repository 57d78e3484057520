"""Failure paths of the bounded device loops and of served admission.

The bounds are lowered on the host (raster_set_test_limits): no GPU is made
to fault, trap or hang.  Every loop still ends, and the exhausted bound must
surface as a status from the one handle, batch instance or served request it
hit, while everything else keeps the oracle's exact result.  Served requests
are admitted by free device memory: with a reserve that leaves room for a few
requests they queue and all complete exactly; a request that cannot fit even
alone is refused with RASTER_E_OOM."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1907_03620_gb300 as R
from paper_1907_03620_gb300 import _native
from paper_1907_03620_gb300.batch import RasterBatch
from paper_1907_03620_gb300.serve import RasterServer

pytestmark = pytest.mark.gpu


def _limits(probe: int, unions: int):
    assert R.lib().raster_set_test_limits(probe, unions) == _native.OK


@pytest.fixture(autouse=True)
def _restore_limits():
    yield
    _limits(-1, -1)


def _same(res, ref):
    s = res.sorted()
    assert s.key.cpu().numpy().tolist() == ref.key.tolist()
    assert s.count.cpu().numpy().tolist() == ref.count.astype(np.int64).tolist()
    assert s.cid.cpu().numpy().tolist() == ref.cid.tolist()
    assert res.n_clusters == ref.n_clusters


def _work(seed, n=200_000):
    w = gen.Workload(n=n, clusters=n // 500, cluster_points=n * 9 // 10, canvas=100.0 * np.sqrt(n / 1e6) + 1,
                     precision=2, tau=5, mu=4, seed=seed)
    return w, gen.points(w)


def _status_of(fn):
    try:
        fn()
    except R.RasterError as e:
        return e.status
    return _native.OK


def test_single_handle_bounds_surface_and_leave_other_handles_exact():
    w, xy = _work(71)
    d = torch.from_numpy(xy).cuda()
    _limits(0, -1)  # no insertion may probe a slot
    full = R.Raster(w.precision, w.tau, w.mu)
    _limits(-1, 0)  # no union-find join may take a step
    nojoin = R.Raster(w.precision, w.tau, w.mu)
    _limits(-1, -1)
    plain = R.Raster(w.precision, w.tau, w.mu)
    assert _status_of(lambda: (full.contract(d), full.agglomerate())) == _native.E_TABLE_FULL
    assert _status_of(lambda: (nojoin.contract(d), nojoin.agglomerate())) == _native.E_INTERNAL
    plain.contract(d)
    ref, _ = oracle.raster(xy, w.precision, w.tau, w.mu)
    _same(plain.agglomerate(), ref)
    for h in (full, nojoin, plain):
        h.close()


def test_batch_bounds_surface_per_instance():
    ws = [_work(72 + i, 50_000 + 10_000 * i) for i in range(4)]
    dev = [torch.from_numpy(xy).cuda() for _, xy in ws]
    inst = [(d, w.precision, w.tau, w.mu) for d, (w, _) in zip(dev, ws)]
    for probe, unions, want in ((0, -1, _native.E_TABLE_FULL), (-1, 0, _native.E_INTERNAL)):
        _limits(probe, unions)
        b = RasterBatch(inst)
        _limits(-1, -1)
        b.run()
        assert _status_of(b.wait) == want
        for i in range(len(inst)):
            assert b.result(i).status == want
        b.close()
    b = RasterBatch(inst)
    b.run()
    b.wait()
    for i, (w, xy) in enumerate(ws):
        ref, _ = oracle.raster(xy, w.precision, w.tau, w.mu)
        _same(b.result(i), ref)
    b.close()


def test_served_bounds_hit_one_request_only():
    reqs = [_work(80 + i, 30_000 + 7_000 * i) for i in range(6)]
    dev = {i: torch.from_numpy(xy).cuda() for i, (_, xy) in enumerate(reqs)}
    srv = RasterServer(max_active=16)
    for i, (w, _) in enumerate(reqs):
        _limits(0, -1) if i == 1 else _limits(-1, 0) if i == 3 else _limits(-1, -1)
        srv.submit(i, w.precision, w.tau, w.mu, w.n, 2)
    _limits(-1, -1)
    for i, (w, _) in enumerate(reqs):
        for lo, hi in gen.chunk_bounds(w.n, 2):
            srv.push(i, dev[i][lo:hi])
    got = {}
    for _ in range(2000):
        r = srv.poll(wait_ms=50)
        if r is not None:
            got[r[0]] = r[1]
            srv.release(r[0])
        if len(got) == len(reqs):
            break
    assert len(got) == len(reqs)
    assert got[1].status == _native.E_TABLE_FULL
    assert got[3].status == _native.E_INTERNAL
    for i, (w, xy) in enumerate(reqs):
        if i in (1, 3):
            continue
        assert got[i].status == _native.OK
        ref, _ = oracle.raster(xy, w.precision, w.tau, w.mu)
        _same(got[i], ref)
    assert srv.stats()["status"] == _native.OK
    srv.close()


def _drain(srv, expect, timeout_polls=4000):
    got, peak_waiting, peak_bytes = {}, 0, 0
    for _ in range(timeout_polls):
        st = srv.stats()
        peak_waiting = max(peak_waiting, st["waiting"])
        peak_bytes = max(peak_bytes, st["device_bytes"])
        r = srv.poll(wait_ms=20)
        if r is not None:
            got[r[0]] = r[1]
            srv.release(r[0])
        if len(got) == expect:
            break
    return got, peak_waiting, peak_bytes


def test_served_admission_by_free_device_memory():
    """The reserve leaves free memory for about three requests of 3M points:
    the rest wait, memory comes back as requests finish, all results are
    exact, and the engine's pages go back to the device once it is idle."""
    reqs = [_work(90 + i, 3_000_000) for i in range(10)]
    dev = {i: torch.from_numpy(xy).cuda() for i, (_, xy) in enumerate(reqs)}
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    room = 420 << 20
    srv = RasterServer(max_active=64, reserve_bytes=int(free - room))
    for i, (w, _) in enumerate(reqs):  # all announced first: a few are admitted, the rest wait
        srv.submit(i, w.precision, w.tau, w.mu, w.n, 3)
    import time
    time.sleep(0.2)
    st = srv.stats()
    assert 0 < st["active"] < len(reqs) and st["waiting"] == len(reqs) - st["active"]
    for i, (w, _) in enumerate(reqs):
        for lo, hi in gen.chunk_bounds(w.n, 3):
            srv.push(i, dev[i][lo:hi])
    got, peak_waiting, peak_bytes = _drain(srv, len(reqs))
    peak_waiting = max(peak_waiting, st["waiting"])
    peak_bytes = max(peak_bytes, st["device_bytes"])
    assert len(got) == len(reqs)
    assert peak_waiting > 0  # admission had to wait for memory
    assert 0 < peak_bytes <= room
    for i, (w, xy) in enumerate(reqs):
        assert got[i].status == _native.OK
        ref, _ = oracle.raster(xy, w.precision, w.tau, w.mu)
        _same(got[i], ref)
    for _ in range(100):  # idle: cached pages are given back
        if srv.stats()["device_bytes"] == 0:
            break
        time.sleep(0.05)
    assert srv.stats()["device_bytes"] == 0
    assert srv.stats()["refused"] == 0
    srv.close()


def test_served_request_that_never_fits_is_refused():
    w, xy = _work(99, 3_000_000)
    d = torch.from_numpy(xy).cuda()
    torch.cuda.synchronize()
    free, total = torch.cuda.mem_get_info()
    srv = RasterServer(max_active=8, reserve_bytes=int(free - (40 << 20)))
    srv.submit(1, w.precision, w.tau, w.mu, w.n, 1)
    srv.push(1, d)
    got, _, _ = _drain(srv, 1)
    assert got[1].status == _native.E_OOM and got[1].key.numel() == 0
    assert srv.stats()["refused"] == 1 and srv.stats()["status"] == _native.OK
    # beyond the device's memory less the reserve: refused at submit
    with pytest.raises(R.RasterError) as e:
        srv.submit(2, 2, 5, 4, 4_000_000_000, 1)
    assert e.value.status == _native.E_LIMIT
    srv.close()
