"""raster_count_tiles_static: tile counts for callers that cannot allocate
device memory (the hash table lives in a fixed array inside the library).

Checks, through the C ABI, that two calls in a row give exactly the tile
counts of the regular handle path (raster_create / raster_contract /
raster_export_tiles) on different inputs -- so the shared array is cleared
between calls -- and that an input over the fixed capacity is refused."""
import ctypes

import numpy as np
import pytest
import torch

import gen
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


def _static_path(xy: torch.Tensor, precision):
    L = R.lib()
    n = xy.shape[0]
    key = torch.empty(max(n, 1), dtype=torch.int64, device=xy.device)
    cnt = torch.empty(max(n, 1), dtype=torch.int32, device=xy.device)
    rows = ctypes.c_int64(-1)
    rc = L.raster_count_tiles_static(ctypes.c_void_p(xy.data_ptr()), n, float(precision),
                                     ctypes.c_void_p(key.data_ptr()), ctypes.c_void_p(cnt.data_ptr()),
                                     ctypes.byref(rows), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _native.OK, _native.NAMES.get(rc, rc)
    d = rows.value
    return _sorted_rows(key[:d].cpu().numpy(), cnt[:d].cpu().numpy().astype(np.int64) & 0xFFFFFFFF)


def test_static_tile_counts_match_handle_path_on_two_calls():
    cases = [
        gen.Workload(n=500_000, clusters=500, cluster_points=450_000, canvas=40.0, precision=2, tau=1, mu=1,
                     seed=501),
        gen.Workload(n=120_001, clusters=50, cluster_points=100_000, canvas=3.0, precision=3.5, tau=1, mu=1,
                     seed=502),
    ]
    for w in cases:  # two calls in a row on different inputs
        xy = torch.from_numpy(gen.points(w)).cuda()
        ref_key, ref_cnt = _handle_path(xy, w.precision)
        key, cnt = _static_path(xy, w.precision)
        assert np.array_equal(key, ref_key)
        assert np.array_equal(cnt, ref_cnt)
        assert int(cnt.sum()) == w.n


def test_static_rejects_inputs_over_capacity():
    L = R.lib()
    rows = ctypes.c_int64(-1)
    n = _native.STATIC_MAX_POINTS + 1
    rc = L.raster_count_tiles_static(None, n, 2.0, None, None, ctypes.byref(rows), None)
    assert rc == _native.E_LIMIT
    assert rows.value == -1
