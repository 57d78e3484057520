"""The labels' block index of kept tiles against the oracle.

The index (one entry per 8 x 8-tile block holding a kept tile) answers most
label lookups; the tile table answers the rest. Each case compares the labels
with the index forced on (RASTER_LABEL_INDEX=1), forced off (=0) and chosen
by size (unset) with the oracle, bit for bit. The cases are built to reach
every branch of the lookup:
- negative tile indices, where blocks are floor divisions;
- blocks with kept tiles of two or three clusters ("mixed", answered by the
  table);
- clusters whose id tile is more than 127 tiles from the block, alone or
  sharing a block with another cluster (same);
- blocks beyond the index's 24-bit range, and one cluster straddling the edge
  of that range;
- noise.
"""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1907_03620_gb300 as R
from paper_1907_03620_gb300 import _native

pytestmark = pytest.mark.gpu

# block index range at precision 2: blocks -(2^23 - 1) .. 2^23 - 2 of 8 tiles
EDGE_HI = ((1 << 23) - 2) * 8 + 7   # last tile inside
EDGE_LO = -((1 << 23) - 1) * 8      # first tile inside


def _blobs(rng, centres, per, sigma):
    pts = [c + rng.normal(0.0, sigma, size=(per, 2)) for c in centres]
    return np.concatenate(pts)


def index_case(seed):
    rng = np.random.default_rng(seed)
    parts = []
    # small clusters around the origin, both signs
    parts.append(_blobs(rng, rng.uniform(-3.0, 3.0, size=(300, 2)), 120, 0.012))
    # pairs of clusters three tiles apart: often in one block, never joined
    c = rng.uniform(-2.0, 2.0, size=(200, 2))
    parts.append(_blobs(rng, c, 40, 0.0015))
    parts.append(_blobs(rng, c + np.array([0.03, 0.0]), 40, 0.0015))
    # long clusters: a band 4 units (400 tiles) long, id tile far from most blocks
    for y in (-4.5, 4.5):
        t = rng.uniform(0.0, 4.0, size=20000)
        parts.append(np.stack([t - 2.0, y + rng.normal(0.0, 0.004, size=t.size)], axis=1))
    # clusters beyond the 24-bit block range, and straddling both of its edges
    for cx in (EDGE_HI / 100.0 + 0.5, (EDGE_HI + 1) / 100.0, EDGE_LO / 100.0, EDGE_LO / 100.0 - 3.0,
               2.5e7, -2.5e7):
        parts.append(_blobs(rng, np.array([[cx, 1.25], [cx, -7.5]]), 300, 0.02))
    # three clusters of two tiles in one 8 x 8 block (x tiles 8m, 8m+3, 8m+6)
    for m in range(40):
        X, Y = 8 * (m - 20), 600
        for dx in (0, 3, 6):
            for dy in (0, 1):
                parts.append(np.full((4, 2), ((X + dx + 0.5) / 100.0, (Y + dy + 0.5) / 100.0)))
    # a small cluster three tiles above the upper band, in the band's blocks
    for k in range(20):
        X = -150 + 16 * k
        for y in (454, 455):
            parts.append(np.full((4, 2), ((X + 0.5) / 100.0, (y + 0.5) / 100.0)))
    # noise
    parts.append(rng.uniform(-5.0, 5.0, size=(20000, 2)))
    xy = np.concatenate(parts)
    return xy[rng.permutation(xy.shape[0])]


def labels_with(monkeypatch, mode, xy, precision, tau, mu, chunks=1):
    if mode is None:
        monkeypatch.delenv("RASTER_LABEL_INDEX", raising=False)
    else:
        monkeypatch.setenv("RASTER_LABEL_INDEX", mode)
    d = torch.from_numpy(np.ascontiguousarray(xy)).cuda()
    r = R.Raster(precision, tau, mu)
    r.contract(d)
    res = r.agglomerate(allow_range_error=True)
    L = _native.lib()
    before = L.raster_kernel_launches()
    n = d.shape[0]
    lab = torch.cat([r.point_labels(d[n * c // chunks: n * (c + 1) // chunks]) for c in range(chunks)])
    torch.cuda.synchronize()
    launches = L.raster_kernel_launches() - before
    r.close()
    return res, lab.cpu().numpy(), launches


@pytest.mark.parametrize("seed", [0, 1])
def test_index_cases_bit_exact(monkeypatch, seed):
    xy = index_case(seed)
    ref, ref_lab, _ = oracle.raster(xy, 2, 3, 2, with_labels=True)
    assert ref.n_clusters > 500
    on_res, on, on_launches = labels_with(monkeypatch, "1", xy, 2, 3, 2, chunks=3)
    off_res, off, off_launches = labels_with(monkeypatch, "0", xy, 2, 3, 2, chunks=3)
    assert np.array_equal(off, ref_lab)
    assert np.array_equal(on, ref_lab)
    # the index was built once (count, zeros, build) and reused by later chunks
    assert on_launches == off_launches + 3
    assert on_res.n_clusters == ref.n_clusters
    # the cases do reach the table: mixed blocks, far ids and out-of-range blocks
    keys = ref.key
    x = keys >> 32
    assert (x > EDGE_HI).any() and (x < EDGE_LO).any()
    assert ((x >= EDGE_LO) & (x <= EDGE_HI)).any()
    cx = ref.cid >> 32
    assert (np.abs(x - cx) > 127).any()
    y = (keys << 32) >> 32
    ids = {}
    for b, c in zip(((x >> 3) * (1 << 32) + (y >> 3)).tolist(), ref.cid.tolist()):
        ids.setdefault(b, set()).add(c)
    per_block = [len(v) for v in ids.values()]
    assert per_block.count(2) > 50 and per_block.count(3) >= 40


def test_index_rebuilt_after_each_agglomeration(monkeypatch):
    monkeypatch.setenv("RASTER_LABEL_INDEX", "1")
    xy = index_case(7)
    half = xy.shape[0] // 2
    d = torch.from_numpy(np.ascontiguousarray(xy)).cuda()
    r = R.Raster(2, 3, 2)
    r.contract(d[:half])
    r.agglomerate(allow_range_error=True)
    lab1 = r.point_labels(d[:half]).cpu().numpy()
    r.contract(d[half:])
    r.agglomerate(allow_range_error=True)
    lab2 = r.point_labels(d).cpu().numpy()
    r.reset()
    r.contract(d[half:])
    r.agglomerate(allow_range_error=True)
    lab3 = r.point_labels(d[half:]).cpu().numpy()
    r.close()
    _, ref1, _ = oracle.raster(xy[:half], 2, 3, 2, with_labels=True)
    _, ref2, _ = oracle.raster(xy, 2, 3, 2, with_labels=True)
    _, ref3, _ = oracle.raster(xy[half:], 2, 3, 2, with_labels=True)
    assert np.array_equal(lab1, ref1)
    assert np.array_equal(lab2, ref2)
    assert np.array_equal(lab3, ref3)


def test_index_by_size_on_a_5m_workload(monkeypatch):
    """Unset, the index is used once the tile table outgrows 64 MiB: 5M points
    at the density of the 500M-point workload."""
    w = gen.Workload(n=5_000_000, clusters=10_000, cluster_points=4_750_000, canvas=300.0, precision=2,
                     tau=5, mu=4, seed=11)
    xy = gen.points(w)
    ref, ref_lab, _ = oracle.raster(xy, w.precision, w.tau, w.mu, with_labels=True)
    res, auto, auto_launches = labels_with(monkeypatch, None, xy, w.precision, w.tau, w.mu)
    _, off, off_launches = labels_with(monkeypatch, "0", xy, w.precision, w.tau, w.mu)
    assert auto_launches == off_launches + 3
    assert np.array_equal(auto, ref_lab)
    assert np.array_equal(off, ref_lab)
    assert res.n_clusters == ref.n_clusters


def test_small_problem_skips_the_index(monkeypatch):
    """Unset, a tile table that fits in L2 answers the labels by itself."""
    xy = index_case(3)[:20000]
    _, on, on_launches = labels_with(monkeypatch, "1", xy, 2, 3, 2)
    _, auto, auto_launches = labels_with(monkeypatch, None, xy, 2, 3, 2)
    assert auto_launches == on_launches - 3
    assert np.array_equal(on, auto)


@pytest.mark.parametrize("mode", ["0", "1"])
def test_reserve_after_agglomerate_keeps_labels_and_groups(monkeypatch, mode):
    """Growing the table under live results (raster_reserve after the
    agglomeration) moves every slot: the result rows find theirs again and get
    their label codes back, and the label index is rebuilt for the new
    regions. Labels before and after, and the RASTER' groups after, match the
    oracle."""
    monkeypatch.setenv("RASTER_LABEL_INDEX", mode)
    xy = index_case(5)
    ref, ref_lab, o = oracle.raster(xy, 2, 3, 2, with_labels=True)
    rs_ref, idx_ref = o.point_groups(xy)
    want = {int(k): idx_ref[rs_ref[i]:rs_ref[i + 1]] for i, k in enumerate(ref.key)}
    d = torch.from_numpy(np.ascontiguousarray(xy)).cuda()
    r = R.Raster(2, 3, 2)
    r.contract(d)
    res = r.agglomerate(allow_range_error=True)
    assert np.array_equal(r.point_labels(d).cpu().numpy(), ref_lab)
    cap = r.capacity
    r.reserve(8 * cap)  # several regions where there was one
    assert r.capacity > 4 * cap
    assert np.array_equal(r.point_labels(d).cpu().numpy(), ref_lab)
    row_start, idx = r.point_groups(d, res.key.numel())
    keys = res.key.cpu().numpy().tolist()
    rs, ix = row_start.cpu().numpy(), idx.cpu().numpy()
    assert set(keys) == set(want)
    for row, k in enumerate(keys):
        assert np.array_equal(np.sort(ix[rs[row]:rs[row + 1]]), want[k]), k
    assert np.array_equal(r.point_labels(d).cpu().numpy(), ref_lab)
    r.close()
