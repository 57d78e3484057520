"""Batched form: every instance of a batch equals the CPU oracle run on that
instance alone, whatever the tuning knobs; graph replays are consistent."""
import math
import random

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1907_03620_gb300 as R
from paper_1907_03620_gb300.batch import RasterBatch

pytestmark = pytest.mark.gpu


def _same(res, ref):
    s = res.sorted()
    assert s.key.cpu().numpy().tolist() == ref.key.tolist()
    assert s.count.cpu().numpy().tolist() == ref.count.astype(np.int64).tolist()
    assert s.cid.cpu().numpy().tolist() == ref.cid.tolist()
    assert res.n_clusters == ref.n_clusters
    assert res.n_distinct == ref.n_tiles
    assert res.n_significant == ref.n_significant


def _small_instances(count, seed, hi=60_000):
    ws = gen.batch_instances(count=count, seed=seed, lo=10, hi=hi)
    return ws, [gen.points(w) for w in ws]


def test_batch_matches_oracle_per_instance():
    ws, pts = _small_instances(96, seed=41)
    dev = [torch.from_numpy(p).cuda() for p in pts]
    b = RasterBatch([(d, w.precision, w.tau, w.mu) for d, w in zip(dev, ws)])
    b.run()
    b.wait()
    for i, (w, p) in enumerate(zip(ws, pts)):
        ref, _ = oracle.raster(p, w.precision, w.tau, w.mu)
        _same(b.result(i), ref)


def test_batch_knobs_do_not_change_results():
    ws, pts = _small_instances(40, seed=42, hi=30_000)
    dev = [torch.from_numpy(p).cuda() for p in pts]
    inst = [(d, w.precision, w.tau, w.mu) for d, w in zip(dev, ws)]
    base = None
    for load in (0.5, 0.75):
        for block in (128, 512):
            for width in (1, 2, 8):
                for preagg in (0, 1):
                    b = RasterBatch(inst, load=load, block=block, width=width, preagg=preagg)
                    b.run()
                    b.wait()
                    rows = [b.result(i).sorted() for i in range(len(inst))]
                    got = [(r.key.cpu().tolist(), r.count.cpu().tolist(), r.cid.cpu().tolist(), r.n_clusters)
                           for r in rows]
                    if base is None:
                        base = got
                    assert got == base, (load, block, width, preagg)
                    b.close()


def test_batch_edge_instances_and_errors():
    g = np.random.default_rng(7)
    cases = [
        (np.zeros((0, 2)), 2, 5, 4),                                   # empty
        (np.array([[0.5, 0.5]]), 2, 1, 1),                              # one point
        (np.tile([[0.123, -0.456]], (5000, 1)), 2, 5, 1),               # one tile
        (g.uniform(-1, 1, size=(20000, 2)), 2, 3, 4),                   # dense, negative
        (np.array([[0.5, 0.5], [math.nan, 0.1], [0.51, 0.52]] * 10), 2, 2, 1),  # range errors
        (g.uniform(-3, 3, size=(7777, 2)), 3.5, 1, 2),                  # fractional precision
    ]
    dev = [torch.from_numpy(np.ascontiguousarray(c[0], dtype=np.float64)).cuda() for c in cases]
    b = RasterBatch([(d, p, t, m) for d, (_, p, t, m) in zip(dev, cases)])
    b.run()
    st = b.wait(allow_range_error=True)
    assert st == R._native.E_RANGE
    for i, (xy, p, t, m) in enumerate(cases):
        ref, _ = oracle.raster(np.ascontiguousarray(xy, dtype=np.float64), p, t, m)
        res = b.result(i)
        assert (res.status == R._native.E_RANGE) == (ref.status == oracle.E_RANGE)
        _same(res, ref)


def test_batch_replay_with_new_data_in_place():
    ws, pts = _small_instances(16, seed=43)
    dev = [torch.from_numpy(p).cuda() for p in pts]
    b = RasterBatch([(d, w.precision, w.tau, w.mu) for d, w in zip(dev, ws)])
    for rep in range(2):
        b.run()
        b.wait()
    # new points written into the same buffers: the graph picks them up
    rng = np.random.default_rng(3)
    new = []
    for d in dev:
        arr = rng.uniform(0, 2, size=tuple(d.shape))
        d.copy_(torch.from_numpy(arr))
        new.append(arr)
    b.run()
    b.wait()
    for i, (w, p) in enumerate(zip(ws, new)):
        ref, _ = oracle.raster(p, w.precision, w.tau, w.mu)
        _same(b.result(i), ref)


def test_batched_workload_full_size_sampled():
    """The 4096-instance workload (sizes 1K..2M) in the bench's launch
    configuration; a sample of instances is checked against the oracle and
    properties are checked on all of them."""
    ws = gen.batch_instances()
    total = sum(w.n for w in ws)
    flat = torch.empty((total, 2), dtype=torch.float64, device="cuda")
    offs = np.cumsum([0] + [w.n for w in ws])
    for i, w in enumerate(ws):
        flat[offs[i]:offs[i + 1]].copy_(torch.from_numpy(gen.points(w)))
    inst = [(flat[offs[i]:offs[i + 1]], w.precision, w.tau, w.mu) for i, w in enumerate(ws)]
    b = RasterBatch(inst)
    b.run()
    b.wait()
    rng = random.Random(5)
    for i in rng.sample(range(len(ws)), 12) + [int(np.argmax([w.n for w in ws]))]:
        w = ws[i]
        ref, _ = oracle.raster(flat[offs[i]:offs[i + 1]].cpu().numpy(), w.precision, w.tau, w.mu)
        _same(b.result(i), ref)
    for i, w in enumerate(ws):
        c = b.counts(i)
        assert c.n_tiles <= c.n_significant <= c.n_distinct <= w.n
        assert c.n_significant * w.tau <= w.n
        assert c.n_clusters * w.mu <= c.n_tiles
