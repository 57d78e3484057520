"""RASTER' grouped output (Sect. 3.4, Fig. 2d) through the C ABI, against the
oracle's grouping: for every kept tile the same set of point indices, and the
per-point labels unchanged after grouping."""
import ctypes

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1907_03620_gb300 as R

pytestmark = pytest.mark.gpu


def _oracle_groups(xy, p, tau, mu):
    ref, ref_lab, o = oracle.raster(xy, p, tau, mu, with_labels=True)
    rs, idx = o.point_groups(xy)
    groups = {int(k): idx[rs[i]:rs[i + 1]] for i, k in enumerate(ref.key)}
    return ref, ref_lab, groups


def _check(xy, p, tau, mu, chunks=1):
    ref, ref_lab, want = _oracle_groups(xy, p, tau, mu)
    d = torch.from_numpy(np.ascontiguousarray(xy)).cuda()
    r = R.Raster(p, tau, mu)
    n = d.shape[0]
    for c in range(chunks):
        r.contract(d[n * c // chunks: n * (c + 1) // chunks])
    res = r.agglomerate()
    row_start, idx = r.point_groups(d, res.key.numel())
    keys, counts = res.key.cpu().numpy(), res.count.cpu().numpy()
    rs, ix = row_start.cpu().numpy(), idx.cpu().numpy()
    assert rs[0] == 0 and np.array_equal(np.diff(rs), counts.astype(np.int64))
    assert len(ix) == sum(len(v) for v in want.values())
    assert set(keys.tolist()) == set(want)
    for row, k in enumerate(keys.tolist()):
        assert np.array_equal(np.sort(ix[rs[row]:rs[row + 1]]), want[k]), k
    # grouping restores the label codes: labels still agree with the oracle
    assert np.array_equal(r.point_labels(d).cpu().numpy(), ref_lab)
    r.close()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_groups_small_random(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5_000, 60_000))
    w = gen.Workload(n=n, clusters=int(rng.integers(5, 60)), cluster_points=int(n * 0.8), canvas=6.0,
                     precision=2, tau=int(rng.integers(1, 6)), mu=int(rng.integers(1, 5)), seed=100 + seed)
    _check(gen.points(w), w.precision, w.tau, w.mu, chunks=1 + seed)


def test_groups_workload_1m():
    w = gen.C1_1M
    _check(gen.points(w), w.precision, w.tau, w.mu)


def test_groups_large_rows_and_empty():
    # one tile with 300k points spans many scan tiles; plus a run with no kept tile
    rng = np.random.default_rng(3)
    xy = np.concatenate([rng.uniform(0.1201, 0.1299, (300_000, 2)), rng.uniform(-50, 50, (20_000, 2))])
    _check(xy, 2, 5, 1)
    _check(rng.uniform(-1000, 1000, (10_000, 2)), 2, 5, 4)


def test_groups_capacity_and_state_errors():
    w = gen.Workload(n=20_000, clusters=10, cluster_points=18_000, canvas=3.0, precision=2, tau=3, mu=2, seed=77)
    d = torch.from_numpy(gen.points(w)).cuda()
    r = R.Raster(w.precision, w.tau, w.mu)
    L = R._native.lib()
    rs = torch.empty(1 << 16, dtype=torch.int64, device="cuda")
    m = ctypes.c_int64(-1)
    r.contract(d)
    # before agglomerate: state error
    assert L.raster_point_groups(r.handle, ctypes.c_void_p(d.data_ptr()), d.shape[0], ctypes.c_void_p(rs.data_ptr()),
                                 None, 0, ctypes.byref(m), None) == R._native.E_STATE
    res = r.agglomerate()
    assert res.key.numel() > 0
    # capacity 0: reports the number of grouped points and writes nothing
    assert L.raster_point_groups(r.handle, ctypes.c_void_p(d.data_ptr()), d.shape[0], ctypes.c_void_p(rs.data_ptr()),
                                 None, 0, ctypes.byref(m), None) == R._native.E_ARG
    assert m.value == int(res.count.sum())
    # the handle stays usable
    _, idx = r.point_groups(d, res.key.numel())
    assert idx.numel() == m.value
    r.close()
