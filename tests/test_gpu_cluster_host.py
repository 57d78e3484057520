"""raster_cluster_host: the whole method on host points in one call (one copy
of the points), against the oracle and against the three separate calls."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1907_03620_gb300 as R

pytestmark = pytest.mark.gpu


def check(res, lab, ref, ref_lab):
    s = res.sorted()
    assert s.key.cpu().numpy().tolist() == ref.key.tolist()
    assert s.count.cpu().numpy().tolist() == ref.count.astype(np.int64).tolist()
    assert s.cid.cpu().numpy().tolist() == ref.cid.tolist()
    assert (res.n_clusters, res.n_significant, res.n_distinct) == (ref.n_clusters, ref.n_significant, ref.n_tiles)
    assert np.array_equal(lab.numpy(), ref_lab)


def test_workload_1m_and_repeat():
    w = gen.C1_1M
    xy = gen.points(w)
    ref, ref_lab, _ = oracle.raster(xy, w.precision, w.tau, w.mu, with_labels=True)
    pinned = torch.from_numpy(xy).pin_memory()
    r = R.Raster(w.precision, w.tau, w.mu)
    res, lab = r.cluster_host(pinned)
    check(res, lab, ref, ref_lab)
    r.reset()  # the resident buffer is reused
    res, lab = r.cluster_host(pinned)
    check(res, lab, ref, ref_lab)
    r.close()


def test_many_chunks_and_pageable_memory():
    """40M points: three chunks of the copy pipeline; plain (pageable) host memory."""
    w = gen.Workload(n=40_000_000, clusters=40_000, cluster_points=36_000_000, canvas=600.0, precision=2,
                     tau=5, mu=4, seed=17)
    xy = gen.points(w)
    r = R.Raster(w.precision, w.tau, w.mu)
    res, lab = r.cluster_host(torch.from_numpy(xy), out=torch.empty(w.n, dtype=torch.int64))
    r2 = R.Raster(w.precision, w.tau, w.mu)
    d = torch.from_numpy(xy).cuda()
    r2.contract(d)
    res2 = r2.agglomerate()
    a, b = res.sorted(), res2.sorted()
    assert torch.equal(a.key, b.key) and torch.equal(a.count, b.count) and torch.equal(a.cid, b.cid)
    assert torch.equal(lab, r2.point_labels(d).cpu())
    # sampled labels against the oracle's projection of the same points
    idx = np.random.default_rng(3).choice(w.n, 20000, replace=False)
    keys, ok = oracle.project(xy[idx], oracle.scale_of(w.precision))
    cid_of = dict(zip(a.key.cpu().numpy().tolist(), a.cid.cpu().numpy().tolist()))
    assert lab.numpy()[idx].tolist() == [cid_of.get(int(k), R.NOISE) for k in keys]
    r.close()
    r2.close()


def test_three_coordinates():
    xyz = np.ascontiguousarray(gen.cubes3(500, 300, 0.08, 8.0, 20_000, 14))
    ref, ref_lab, _ = oracle.raster(xyz, 2, 3, 2, with_labels=True)
    r = R.Raster(2, 3, 2, dims=3)
    res, lab = r.cluster_host(torch.from_numpy(xyz).pin_memory())
    check(res, lab, ref, ref_lab)
    r.close()
