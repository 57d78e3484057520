"""raster_count_tiles_static: tile counts for callers that cannot allocate
device memory (the hash table lives in a fixed array inside the library).

Checks, through the C ABI, that two calls in a row give exactly the tile
counts of the regular handle path (raster_create / raster_contract /
raster_export_tiles) and of the CPU oracle on different inputs -- so the
shared array is cleared between calls -- that non-finite and out-of-range
points are reported as RASTER_E_RANGE while every other tile keeps its exact
count, that an empty input gives no rows, and that an input over the fixed
capacity is refused."""
import ctypes

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1907_03620_gb300 as R
from paper_1907_03620_gb300 import _native

pytestmark = pytest.mark.gpu


def _sorted_rows(key: np.ndarray, count: np.ndarray):
    order = np.argsort(key, kind="stable")
    return key[order], count[order]


def _handle_path(xy: torch.Tensor, precision):
    r = R.Raster(precision, 1, 1)
    r.contract(xy)
    key, cnt = r.export_tiles()
    r.close()
    return _sorted_rows(key.cpu().numpy(), cnt.cpu().numpy())


def _oracle_tiles(xy: np.ndarray, precision):
    o = oracle.Oracle(precision, 1, 1)
    st = o.add(xy)
    key, cnt = o.tiles()
    return st, _sorted_rows(key, cnt.astype(np.int64))


def _static_path(xy: torch.Tensor, precision, expect=_native.OK):
    L = R.lib()
    n = xy.shape[0]
    key = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
    cnt = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    rows = ctypes.c_int64(-1)
    ptr = ctypes.c_void_p(xy.data_ptr()) if n else None
    rc = L.raster_count_tiles_static(ptr, n, float(precision), ctypes.c_void_p(key.data_ptr()),
                                     ctypes.c_void_p(cnt.data_ptr()), ctypes.byref(rows),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == expect, _native.NAMES.get(rc, rc)
    d = rows.value
    return _sorted_rows(key[:d].cpu().numpy(), cnt[:d].cpu().numpy().astype(np.int64) & 0xFFFFFFFF)


def test_static_tile_counts_match_handle_path_and_oracle_on_two_calls():
    cases = [
        gen.Workload(n=500_000, clusters=500, cluster_points=450_000, canvas=40.0, precision=2, tau=1, mu=1,
                     seed=501),
        gen.Workload(n=120_001, clusters=50, cluster_points=100_000, canvas=3.0, precision=3.5, tau=1, mu=1,
                     seed=502),
    ]
    for w in cases:  # two calls in a row on different inputs
        host = gen.points(w)
        xy = torch.from_numpy(host).cuda()
        ref_key, ref_cnt = _handle_path(xy, w.precision)
        st, (o_key, o_cnt) = _oracle_tiles(host, w.precision)
        assert st == oracle.OK
        key, cnt = _static_path(xy, w.precision)
        assert np.array_equal(key, ref_key) and np.array_equal(cnt, ref_cnt)
        assert np.array_equal(key, o_key) and np.array_equal(cnt, o_cnt)
        assert int(cnt.sum()) == w.n


def test_static_range_errors_keep_other_counts():
    """Points that are not finite, or whose tile index leaves the int32 range,
    are skipped and reported; the other points' tiles are still written with
    their exact counts."""
    w = gen.Workload(n=200_000, clusters=200, cluster_points=180_000, canvas=20.0, precision=2, tau=1, mu=1,
                     seed=503)
    host = gen.points(w)
    bad = [(np.nan, 1.0), (1.0, np.inf), (-np.inf, -np.inf), (3.0e7, 0.5), (0.5, -2.2e7)]
    idx = np.random.default_rng(9).choice(w.n, len(bad), replace=False)
    for i, (x, y) in zip(idx, bad):
        host[i] = (x, y)
    st, (o_key, o_cnt) = _oracle_tiles(host, w.precision)
    assert st == oracle.E_RANGE
    key, cnt = _static_path(torch.from_numpy(host).cuda(), w.precision, expect=_native.E_RANGE)
    assert np.array_equal(key, o_key) and np.array_equal(cnt, o_cnt)
    assert int(cnt.sum()) == w.n - len(bad)


def test_static_empty_input():
    key, cnt = _static_path(torch.empty((0, 2), dtype=torch.float64, device="cuda"), 2)
    assert len(key) == 0 and len(cnt) == 0


def test_static_rejects_inputs_over_capacity():
    L = R.lib()
    rows = ctypes.c_int64(-1)
    n = _native.STATIC_MAX_POINTS + 1
    rc = L.raster_count_tiles_static(None, n, 2.0, None, None, ctypes.byref(rows), None)
    assert rc == _native.E_LIMIT
    assert rows.value == -1
