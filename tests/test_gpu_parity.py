"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results must agree bit for bit: the sorted set of (tile key, count,
cluster id), the statistics D, S and the number of clusters, and the label of
every point."""
import math
import random
import struct

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1907_03620_gb300 as R

pytestmark = pytest.mark.gpu


def gpu_run(xy: np.ndarray, precision, tau, mu, chunks=1, labels=True, allow_range=False):
    d = torch.from_numpy(np.ascontiguousarray(xy)).cuda()
    r = R.Raster(precision, tau, mu)
    n = d.shape[0]
    for c in range(chunks):
        r.contract(d[n * c // chunks: n * (c + 1) // chunks])
    res = r.agglomerate(allow_range_error=allow_range)
    lab = r.point_labels(d).cpu().numpy() if labels else None
    return r, res, lab


def assert_same(res, lab, ref, ref_lab=None):
    s = res.sorted()
    assert s.key.cpu().numpy().tolist() == ref.key.tolist()
    assert s.count.cpu().numpy().tolist() == ref.count.astype(np.int64).tolist()
    assert s.cid.cpu().numpy().tolist() == ref.cid.tolist()
    assert res.n_clusters == ref.n_clusters
    assert res.n_distinct == ref.n_tiles
    assert res.n_significant == ref.n_significant
    assert res.n_points == ref.points or ref.status != 0
    if ref_lab is not None:
        assert np.array_equal(lab, ref_lab)


def test_scale_matches_oracle_convention():
    for p in (0, 1, 2, 3, 3.5, 0.9, 0.73, -1, 5):
        r = R.Raster(p, 1, 1)
        assert r.scale == oracle.scale_of(p)
        r.close()


def _edge_points(seed, n_random=20000):
    rng = random.Random(seed)
    vals = [0.0, -0.0, 1.005, 0.29, 4.35, -0.001, -0.01, -1e-300, 5e-324, -5e-324, 1e-310,
            2.2250738585072014e-308, 1.7976931348623157e308, math.inf, -math.inf, math.nan,
            21474836.46, 21474836.47, -21474836.47, -21474836.48, 2147483646.0, 2147483646.5,
            2147483647.0, -2147483647.0, -2147483647.5, 1e15, 3.0000000000000004, 0.5, -0.5]
    for _ in range(n_random):
        k = rng.random()
        if k < 0.2:
            vals.append(struct.unpack("<d", struct.pack("<Q", rng.getrandbits(64)))[0])
        elif k < 0.5:
            vals.append(rng.uniform(-5000, 5000))
        else:
            n = rng.randint(-10**8, 10**8)
            base = n / 10 ** rng.randint(0, 5)
            vals.append(math.nextafter(base, math.inf if rng.random() < 0.5 else -math.inf))
    xs = np.array(vals)
    ys = np.roll(xs, 7)
    return np.stack([xs, ys], axis=1)


@pytest.mark.parametrize("precision", [2, 1, 3, 0, 3.5, 0.9, 0.73, -1, 4, 5])
def test_projection_bit_exact_on_edge_values(precision):
    """Every tile key and count equals the oracle's, including values just
    below/above tile borders, subnormals, zeros, huge and non-finite values
    (those are range errors on both sides)."""
    xy = _edge_points(int(precision * 100) + 7)
    scale = oracle.scale_of(precision)
    o = oracle.Oracle(precision, 1, 1)
    o_st = o.add(xy)
    ref_keys, ref_counts = o.tiles()
    d = torch.from_numpy(xy).cuda()
    r = R.Raster(precision, 1, 1)
    r.contract(d)
    st = r.status()
    key, cnt = r.export_tiles()
    order = oracle.tile_order(key.cpu().numpy())
    assert key.cpu().numpy()[order].tolist() == ref_keys.tolist()
    assert cnt.cpu().numpy()[order].tolist() == ref_counts.astype(np.int64).tolist()
    assert (st == R._native.E_RANGE) == (o_st == oracle.E_RANGE)
    assert r.scale == scale


def test_workload_1m_bit_exact():
    w = gen.C1_1M
    xy = gen.points(w)
    ref, ref_lab, _ = oracle.raster(xy, w.precision, w.tau, w.mu, with_labels=True)
    r, res, lab = gpu_run(xy, w.precision, w.tau, w.mu)
    assert_same(res, lab, ref, ref_lab)
    assert ref.n_clusters > 900
    # a second cycle on the same handle: the one round after the reset selects
    # the significant tiles as it writes the table, and the agglomeration uses
    # that selection instead of scanning the table
    d = torch.from_numpy(xy).cuda()
    for _ in range(2):
        r.reset()
        r.contract(d)
        assert_same(r.agglomerate(), r.point_labels(d).cpu().numpy(), ref, ref_lab)
    # agglomerating twice: the second one scans the table (the first rewrote aux)
    assert_same(r.agglomerate(), r.point_labels(d).cpu().numpy(), ref, ref_lab)


@pytest.mark.parametrize("seed", range(8))
def test_small_random_cases(seed):
    rng = random.Random(seed)
    n = rng.choice([1, 2, 31, 32, 33, 127, 129, 1000, 4097, 50_001])
    k = max(1, n // rng.choice([3, 50, 400]))
    w = gen.Workload(n=n, clusters=k, cluster_points=int(n * rng.choice([0.0, 0.5, 0.9, 1.0])),
                     canvas=rng.choice([0.05, 1.0, 30.0]), precision=rng.choice([1, 2, 3, 3.5]),
                     tau=rng.choice([1, 2, 3, 5]), mu=rng.choice([1, 2, 4]), seed=1000 + seed)
    xy = gen.points(w)
    xy[: n // 3] -= w.canvas / 2  # negative coordinates too
    ref, ref_lab, _ = oracle.raster(xy, w.precision, w.tau, w.mu, with_labels=True)
    r, res, lab = gpu_run(xy, w.precision, w.tau, w.mu)
    assert_same(res, lab, ref, ref_lab)


def test_empty_input():
    r = R.Raster(2, 5, 4)
    r.contract(torch.empty((0, 2), dtype=torch.float64, device="cuda"))
    res = r.agglomerate()
    assert res.key.numel() == 0 and res.n_clusters == 0 and res.n_distinct == 0
    lab = r.point_labels(torch.empty((0, 2), dtype=torch.float64, device="cuda"))
    assert lab.numel() == 0


def test_all_points_in_one_tile_and_dense_clusters():
    xy = np.tile(np.array([[0.123, -0.456]]), (100_000, 1))
    ref, ref_lab, _ = oracle.raster(xy, 2, 5, 1, with_labels=True)
    r, res, lab = gpu_run(xy, 2, 5, 1)
    assert_same(res, lab, ref, ref_lab)
    assert int(res.count[0]) == 100_000
    # one big square of fully significant tiles (one large component)
    g = np.random.default_rng(3)
    xy = g.uniform(-1.0, 1.0, size=(400_000, 2))
    ref, ref_lab, _ = oracle.raster(xy, 2, 3, 4, with_labels=True)
    r, res, lab = gpu_run(xy, 2, 3, 4)
    assert_same(res, lab, ref, ref_lab)


def test_large_percolating_components():
    """Dense uniform data (about 4 points per tile) forms huge, irregular
    components: many threads walk and rewrite the same union-find paths."""
    g = np.random.default_rng(11)
    xy = g.uniform(-10.0, 10.0, size=(16_000_000, 2))
    ref, ref_lab, _ = oracle.raster(xy, 2, 3, 4, with_labels=True)
    r, res, lab = gpu_run(xy, 2, 3, 4)
    assert_same(res, lab, ref, ref_lab)


def test_chunking_order_and_streaming():
    """Chunked contraction (any split, any order) equals one pass; agglomerating
    between chunks and then continuing gives the same final answer."""
    w = gen.Workload(n=300_000, clusters=300, cluster_points=270_000, canvas=30.0, precision=2, tau=5, mu=4,
                     seed=77)
    xy = gen.points(w)
    ref, ref_lab, _ = oracle.raster(xy, 2, 5, 4, with_labels=True)
    for chunks in (1, 7, 64):
        r, res, lab = gpu_run(xy[::-1].copy(), 2, 5, 4, chunks=chunks, labels=False)
        assert_same(res, None, ref)
    d = torch.from_numpy(xy).cuda()
    r = R.Raster(2, 5, 4)
    r.contract(d[:100_000])
    mid = r.agglomerate()
    ref_mid, _ = oracle.raster(xy[:100_000], 2, 5, 4)
    assert_same(mid, None, ref_mid)
    r.contract(d[100_000:])
    res = r.agglomerate()
    assert_same(res, r.point_labels(d).cpu().numpy(), ref, ref_lab)


def test_table_growth_reserve_and_reset():
    """Start from the minimum table; growing by rehash keeps every count."""
    g = np.random.default_rng(5)
    xy = g.uniform(0, 100, size=(2_000_000, 2))  # ~1.9M distinct tiles at p = 2
    ref, _ = oracle.raster(xy, 2, 1, 1)
    d = torch.from_numpy(xy).cuda()
    r = R.Raster(2, 1, 1)
    cap0 = r.capacity
    for c in range(20):
        r.contract(d[c * 100_000:(c + 1) * 100_000])
    res = r.agglomerate()
    assert r.capacity > cap0
    assert_same(res, None, ref)
    r.reset()
    r.contract(d)
    assert_same(r.agglomerate(), None, ref)
    r2 = R.Raster(2, 1, 1)
    r2.reserve(4_000_000)
    cap = r2.capacity
    r2.contract(d)
    assert r2.capacity == cap
    assert_same(r2.agglomerate(), None, ref)


def test_skewed_regions_spill_to_overflow_list():
    """A table of many regions and points that all fall into one spatial block:
    that region's staging segment overflows and the keys take the overflow
    list; counts must still be exact."""
    g = np.random.default_rng(9)
    xy = np.concatenate([g.uniform(0.0, 0.16, size=(3_000_000, 2)),   # one 16 x 16 tile block
                         g.uniform(0.0, 300.0, size=(200_000, 2))])
    g.shuffle(xy)
    ref, ref_lab, _ = oracle.raster(xy, 2, 5, 2, with_labels=True)
    d = torch.from_numpy(xy).cuda()
    r = R.Raster(2, 5, 2)
    r.reserve(20_000_000)  # many regions
    cap = r.capacity
    for c in range(3):
        r.contract(d[c * 1_066_667:(c + 1) * 1_066_667])
    res = r.agglomerate()
    assert r.capacity == cap  # spilling alone does not grow the table
    assert_same(res, r.point_labels(d).cpu().numpy(), ref, ref_lab)
    # one round after a reset, with spilled keys re-inserted after the buckets
    # were written: the selection made while writing them must not be used
    r.reset()
    r.contract(d)
    assert r.capacity == cap
    assert_same(r.agglomerate(), r.point_labels(d).cpu().numpy(), ref, ref_lab)


def test_host_buffer_variants():
    w = gen.Workload(n=40_000_000, clusters=40_000, cluster_points=36_000_000, canvas=600.0, precision=2,
                     tau=5, mu=4, seed=88)
    xy = gen.points(w)
    pinned = torch.from_numpy(xy).pin_memory()
    r = R.Raster(2, 5, 4)
    r.contract_host(pinned)
    res = r.agglomerate()
    lab_h = r.point_labels_host(pinned)
    r2 = R.Raster(2, 5, 4)
    d = pinned.cuda()
    r2.contract(d)
    res2 = r2.agglomerate()
    a, b = res.sorted(), res2.sorted()
    assert torch.equal(a.key, b.key) and torch.equal(a.count, b.count) and torch.equal(a.cid, b.cid)
    assert torch.equal(lab_h, r2.point_labels(d).cpu())
    # a numpy (pageable) source works too
    r3 = R.Raster(2, 5, 4)
    r3.contract_host(xy[:1_000_000])
    ref, _ = oracle.raster(xy[:1_000_000], 2, 5, 4)
    assert_same(r3.agglomerate(), None, ref)


def test_error_paths():
    r = R.Raster(2, 5, 4)
    d = torch.zeros((10, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(R.RasterError) as e:
        r.point_labels(d)  # before agglomerate
    assert e.value.status == R._native.E_STATE
    L = R.lib()
    import ctypes
    raw = torch.zeros(64, dtype=torch.uint8, device="cuda")
    assert L.raster_contract(r.handle, ctypes.c_void_p(raw.data_ptr() + 8), 2, None) == R._native.E_ARG
    # non-finite and out-of-range coordinates: reported, skipped, the rest counted
    xy = np.array([[0.5, 0.5], [math.nan, 0.5], [0.5, math.inf], [3e7, 0.5], [0.51, 0.52]] * 3)
    ref, ref_lab, _ = oracle.raster(xy, 2, 1, 1, with_labels=True)
    assert ref.status == oracle.E_RANGE
    r, res, lab = gpu_run(xy, 2, 1, 1, allow_range=True)
    assert res.status == R._native.E_RANGE
    assert_same(res, lab, ref, ref_lab)
    r.reset()
    assert r.status() == 0


def test_workload_50m_bit_exact():
    w = gen.C2_50M
    xy = gen.points(w)
    ref, ref_lab, _ = oracle.raster(xy, w.precision, w.tau, w.mu, with_labels=True)
    r, res, lab = gpu_run(xy, w.precision, w.tau, w.mu, chunks=3)
    assert_same(res, lab, ref, ref_lab)


def test_table_stats():
    """Diagnostics agree with the result: occupied slots = distinct tiles, and
    probe lengths lie within a bucket."""
    w = gen.C1_1M
    d = torch.from_numpy(gen.points(w)).cuda()
    r = R.Raster(w.precision, w.tau, w.mu)
    r.contract(d)
    res = r.agglomerate()
    st = r.table_stats()
    assert st["capacity"] == r.capacity and st["occupied"] == res.n_distinct
    assert 1.0 <= st["mean_probe"] <= st["max_probe"] <= 4096
    assert 0.0 < st["load"] <= 0.8
    r.reset()  # a void table reads as empty
    assert r.table_stats()["occupied"] == 0
    r.close()
