"""Parity of the extended neighbourhoods and the 2 x 2 group rule with the CPU
oracle, through the C ABI: neighbors(u, delta) for a Chebyshev or Manhattan
distance delta (Sect. 3.2) and the post-processing of Sect. 3.6 (Fig. 4)."""
import ctypes
import os
import random

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1907_03620_gb300 as R

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def run_both(xy, p, tau, mu, metric=R.CHEBYSHEV, delta=1, groups=False, chunks=1):
    ref, ref_lab, _ = oracle.raster(xy, p, tau, mu, with_labels=True, metric=metric, delta=delta, groups=groups,
                                    chunks=chunks)
    d = torch.from_numpy(np.ascontiguousarray(xy)).cuda()
    r = R.Raster(p, tau, mu, metric=metric, delta=delta, groups=groups)
    n = d.shape[0]
    for c in range(chunks):
        r.contract(d[n * c // chunks: n * (c + 1) // chunks])
    res = r.agglomerate()
    lab = r.point_labels(d).cpu().numpy()
    s = res.sorted()
    assert s.key.cpu().numpy().tolist() == ref.key.tolist()
    assert s.count.cpu().numpy().tolist() == ref.count.astype(np.int64).tolist()
    assert s.cid.cpu().numpy().tolist() == ref.cid.tolist()
    assert res.n_clusters == ref.n_clusters
    assert res.n_significant == ref.n_significant
    assert res.n_distinct == ref.n_tiles
    assert np.array_equal(lab, ref_lab)
    r.close()
    return ref


def test_fig4_groups_on_gpu():
    rows = {}
    with open(os.path.join(GOLDEN, "grid_layout.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                rows.setdefault(k, []).append(v)
    split = np.array([[float(a), float(b)] for a, b in rows["split"]])
    ref = run_both(split, 2, 4, 1, groups=True)
    assert ref.n_significant == int(rows["split_groups_significant"][0][0])
    assert ref.n_clusters == int(rows["split_groups_clusters"][0][0])


CASES = [(R.CHEBYSHEV, 1, True), (R.CHEBYSHEV, 2, False), (R.CHEBYSHEV, 3, True), (R.CHEBYSHEV, 4, False),
         (R.MANHATTAN, 1, False), (R.MANHATTAN, 2, True), (R.MANHATTAN, 4, False)]


@pytest.mark.parametrize("metric,delta,groups", CASES)
@pytest.mark.parametrize("seed", range(3))
def test_small_random_cases(metric, delta, groups, seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(2_000, 40_000))
    w = gen.Workload(n=n, clusters=int(rng.integers(3, 80)), cluster_points=int(n * 0.7), canvas=5.0, precision=2,
                     tau=int(rng.integers(2, 7)), mu=int(rng.integers(1, 5)), seed=400 + seed)
    run_both(gen.points(w), w.precision, w.tau, w.mu, metric, delta, groups, chunks=1 + seed)


@pytest.mark.parametrize("metric,delta,groups", [(R.CHEBYSHEV, 1, True), (R.CHEBYSHEV, 2, False),
                                                 (R.MANHATTAN, 1, False), (R.MANHATTAN, 3, True)])
def test_workload_1m(metric, delta, groups):
    w = gen.C1_1M
    run_both(gen.points(w), w.precision, w.tau, w.mu, metric, delta, groups)


def test_groups_sparse_layouts():
    """Points spread so that many tiles hold fewer than tau points while their
    2 x 2 groups reach it: the rule decides most of the significant set."""
    rng = random.Random(9)
    xy = []
    for _ in range(3000):
        cx, cy = rng.randint(-200, 200), rng.randint(-200, 200)
        for _ in range(rng.randint(1, 4)):
            xy.append(((cx + rng.uniform(0.0, 2.0)) / 100.0, (cy + rng.uniform(0.0, 2.0)) / 100.0))
    xy = np.array(xy)
    ref = run_both(xy, 2, 3, 1, groups=True)
    plain, _ = oracle.raster(xy, 2, 3, 1)
    assert ref.n_significant > plain.n_significant


def test_create_ex_argument_errors():
    L = R.lib()
    h = ctypes.c_void_p()
    for metric, delta, groups in ((2, 1, 0), (0, 0, 0), (1, R._native.MAX_DELTA + 1, 0), (0, 1, 2)):
        p = R._native.Params(2.0, 5, 4, metric, delta, groups)
        assert L.raster_create_ex(ctypes.byref(p), ctypes.byref(h)) == R._native.E_ARG
    assert L.raster_create_ex(None, ctypes.byref(h)) == R._native.E_ARG
