"""Labels from stored tile keys (raster_contract_keys + raster_key_labels,
RASTER* of Sect. 4.1 with the projection of Sect. 3.2 done once per point).

The keys written during contraction must equal the oracle's projection of
every point bit for bit (RASTER_INVALID_KEY where the oracle reports a range
error), and the labels read from them must equal the oracle's labels, and the
labels of raster_point_labels, for every point."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1907_03620_gb300 as R
from paper_1907_03620_gb300 import _native

pytestmark = pytest.mark.gpu


def _expected_keys(xy, precision):
    keys, ok = oracle.project(xy, oracle.scale_of(precision))
    keys = keys.copy()
    keys[~ok] = R.INVALID_KEY
    return keys


def _run(xy, precision, tau, mu, chunks, allow_range=False):
    d = torch.from_numpy(np.ascontiguousarray(xy)).cuda()
    n = d.shape[0]
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    r = R.Raster(precision, tau, mu, dims=xy.shape[1]) if xy.shape[1] == 3 else R.Raster(precision, tau, mu)
    bounds = [n * c // chunks for c in range(chunks + 1)]
    for a, b in zip(bounds, bounds[1:]):
        r.contract_keys(d[a:b], keys[a:b])
    res = r.agglomerate(allow_range_error=allow_range)
    lab_k = r.key_labels(keys).cpu().numpy()
    lab_p = r.point_labels(d).cpu().numpy()
    return r, res, keys.cpu().numpy(), lab_k, lab_p


def test_workload_1m_keys_and_labels_bit_exact():
    w = gen.C1_1M
    xy = gen.points(w)
    ref, ref_lab, _ = oracle.raster(xy, w.precision, w.tau, w.mu, with_labels=True)
    r, res, keys, lab_k, lab_p = _run(xy, w.precision, w.tau, w.mu, chunks=3)
    assert np.array_equal(keys, _expected_keys(xy, w.precision))
    assert np.array_equal(lab_k, ref_lab)
    assert np.array_equal(lab_p, ref_lab)
    s = res.sorted()
    assert s.key.cpu().numpy().tolist() == ref.key.tolist()
    assert s.cid.cpu().numpy().tolist() == ref.cid.tolist()
    r.close()


@pytest.mark.parametrize("seed", range(3))
def test_ragged_chunks_range_errors_and_label_index(seed, monkeypatch):
    """Chunks that end inside a tile of pass 1, points that do not project
    (non-finite, or beyond the int32 tile range), and the label index both
    forced on and off."""
    g = np.random.default_rng(100 + seed)
    xy = gen.points(gen.Workload(n=700_001 + seed * 12_347, clusters=600, cluster_points=600_000, canvas=40.0,
                                 precision=2, tau=5, mu=4, seed=200 + seed))
    bad = g.choice(xy.shape[0], 37, replace=False)
    xy[bad[:10], 0] = np.nan
    xy[bad[10:20], 1] = np.inf
    xy[bad[20:30], 0] = 3.0e7  # tile index 3e9: beyond int32
    xy[bad[30:], 1] = -2.2e7
    ref, ref_lab, _ = oracle.raster(xy, 2, 5, 4, with_labels=True)
    for force in ("1", "0"):
        monkeypatch.setenv("RASTER_LABEL_INDEX", force)
        r, res, keys, lab_k, lab_p = _run(xy, 2, 5, 4, chunks=5 + seed, allow_range=True)
        exp = _expected_keys(xy, 2)
        assert np.array_equal(keys, exp)
        assert np.count_nonzero(keys == R.INVALID_KEY) == 37
        assert np.array_equal(lab_k, ref_lab)
        assert np.array_equal(lab_p, ref_lab)
        assert np.all(lab_k[bad] == R.NOISE)
        r.close()


def test_three_coordinates():
    g = np.random.default_rng(5)
    centres = g.uniform(0, 20, size=(300, 3))
    xy = np.concatenate([np.repeat(centres, 400, axis=0) + g.normal(0, 0.05, size=(120_000, 3)),
                         g.uniform(0, 20, size=(30_000, 3))])
    g.shuffle(xy)
    xy = np.ascontiguousarray(xy)
    ref, ref_lab, _ = oracle.raster(xy, 1.5, 5, 4, with_labels=True)
    r, res, keys, lab_k, lab_p = _run(xy, 1.5, 5, 4, chunks=2)
    assert np.array_equal(keys, _expected_keys(xy, 1.5))
    assert np.array_equal(lab_k, ref_lab)
    assert np.array_equal(lab_p, ref_lab)
    r.close()


def test_empty_state_and_argument_errors():
    r = R.Raster(2, 5, 4)
    d = torch.zeros((0, 2), dtype=torch.float64, device="cuda")
    keys = r.contract_keys(d)
    assert keys.numel() == 0
    L = R.lib()
    k = torch.zeros(4, dtype=torch.int64, device="cuda")
    lab = torch.empty(4, dtype=torch.int64, device="cuda")
    # labels before any agglomeration
    assert L.raster_key_labels(r._h, k.data_ptr(), 4, lab.data_ptr(), None) == _native.E_STATE
    r.agglomerate()
    assert r.key_labels(k[:0]).numel() == 0
    # misaligned keys
    assert L.raster_key_labels(r._h, k.data_ptr() + 4, 2, lab.data_ptr(), None) == _native.E_ARG
    xy = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    assert L.raster_contract_keys(r._h, xy.data_ptr(), 4, None, None) == _native.E_ARG
    # every label of an arbitrary key that holds no kept tile is noise
    lab = r.key_labels(torch.tensor([0, 5, R.INVALID_KEY, -1], dtype=torch.int64, device="cuda"))
    assert lab.cpu().tolist() == [R.NOISE] * 4
    r.close()
