"""Three-coordinate points (the generalisation to higher dimensions of
Sect. 3.6) through the C ABI, bit for bit against the CPU oracle: tile keys
and counts, cluster ids, statistics, labels and the RASTER' groups."""
import ctypes

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1907_03620_gb300 as R

pytestmark = pytest.mark.gpu


def cubes(n_clusters, per, side, canvas, noise, seed):
    return np.ascontiguousarray(gen.cubes3(n_clusters, per, side, canvas, noise, seed))


def run_both(xyz, p, tau, mu, metric=R.CHEBYSHEV, delta=1, chunks=1, allow_range=False, host=False):
    ref, ref_lab, o = oracle.raster(xyz, p, tau, mu, with_labels=True, metric=metric, delta=delta, chunks=chunks)
    r = R.Raster(p, tau, mu, metric=metric, delta=delta, dims=3)
    n = xyz.shape[0]
    if host:
        r.contract_host(torch.from_numpy(xyz))
        res = r.agglomerate(allow_range_error=allow_range)
        lab = r.point_labels_host(torch.from_numpy(xyz)).numpy()
        d = None
    else:
        d = torch.from_numpy(xyz).cuda()
        for c in range(chunks):
            r.contract(d[n * c // chunks: n * (c + 1) // chunks])
        res = r.agglomerate(allow_range_error=allow_range)
        lab = r.point_labels(d).cpu().numpy()
    s = res.sorted()
    assert s.key.cpu().numpy().tolist() == ref.key.tolist()
    assert s.count.cpu().numpy().tolist() == ref.count.astype(np.int64).tolist()
    assert s.cid.cpu().numpy().tolist() == ref.cid.tolist()
    assert res.n_clusters == ref.n_clusters
    assert res.n_significant == ref.n_significant
    assert res.n_distinct == ref.n_tiles
    assert np.array_equal(lab, ref_lab)
    return r, res, ref, o, d


@pytest.mark.parametrize("metric,delta", [(R.CHEBYSHEV, 1), (R.MANHATTAN, 1), (R.MANHATTAN, 2), (R.MANHATTAN, 3)])
@pytest.mark.parametrize("seed", range(3))
def test_small_cases(metric, delta, seed):
    g = np.random.default_rng(700 + seed)
    xyz = cubes(int(g.integers(5, 60)), int(g.integers(20, 300)), 0.05, 2.0, int(g.integers(100, 5000)), 800 + seed)
    r, *_ = run_both(xyz, 2, int(g.integers(1, 4)), int(g.integers(1, 5)), metric, delta, chunks=1 + seed)
    r.close()


@pytest.mark.parametrize("precision", [1, 1.5])  # narrow and wide scale significands
def test_cubes_2m(precision):
    xyz = cubes(2000, 900, 0.1, 20.0, 200_000, 11)
    r, res, ref, o, d = run_both(xyz, precision, 5, 4)
    assert ref.n_clusters > 100
    # RASTER' groups over the same points
    row_start, idx = r.point_groups(d, res.key.numel())
    rs, ix = row_start.cpu().numpy(), idx.cpu().numpy()
    ors, oidx = o.point_groups(xyz)
    want = {int(k): oidx[ors[i]:ors[i + 1]] for i, k in enumerate(ref.key)}
    for row, k in enumerate(res.key.cpu().numpy().tolist()):
        assert np.array_equal(np.sort(ix[rs[row]:rs[row + 1]]), want[k])
    r.close()


def test_host_buffers_and_streaming():
    xyz = cubes(300, 400, 0.08, 6.0, 30_000, 12)
    r, *_ = run_both(xyz, 2, 3, 2, host=True)
    r.close()
    r, *_ = run_both(xyz, 2, 3, 2, chunks=5)
    r.close()


def test_range_errors_are_skipped():
    xyz = cubes(50, 200, 0.1, 3.0, 1000, 13)
    bad = np.array([[2 ** 21 / 100.0, 0.5, 0.5], [0.5, -2 ** 21 / 100.0, 0.5], [0.5, 0.5, np.nan]])
    xyz = np.concatenate([xyz, bad])
    r, res, ref, *_ = run_both(xyz, 2, 3, 2, allow_range=True)
    assert ref.status == 2 and r.status() == R._native.E_RANGE
    r.close()


def test_create_ex_three_coordinates_argument_errors():
    L = R.lib()
    h = ctypes.c_void_p()
    for metric, delta, groups, dims in ((0, 2, 0, 3), (1, 4, 0, 3), (0, 1, 1, 3), (0, 1, 0, 4), (0, 1, 0, 1)):
        p = R._native.Params(2.0, 5, 4, metric, delta, groups, dims)
        assert L.raster_create_ex(ctypes.byref(p), ctypes.byref(h)) == R._native.E_ARG
