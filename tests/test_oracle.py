"""Pins for the CPU oracle: what the paper and mathematics fix, checked against
sources other than the oracle itself (CPU only)."""
import math
import os
import random
import struct

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_fixture(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows.append((parts[0], parts[1:]))
    return rows


# ---------------------------------------------------------------------------
# Projection (Alg. 1 project(); Sect. 3.2)

def test_worked_example_sect_3_2():
    rows = _read_fixture("worked_example.txt")
    p = float(dict(rows)["precision"][0])
    pts = np.array([[float(a), float(b)] for k, (a, b) in [(k, v) for k, v in rows if k == "point"]])
    tx, ty, tc = [int(v) for v in dict(rows)["tile"]]
    max_tau = int(dict(rows)["significant_max_tau"][0])
    for tau in range(1, 6):
        r, o = oracle.raster(pts, p, tau=tau, mu=1)
        keys, counts = o.tiles()
        assert list(keys) == [oracle.pack(tx, ty)]
        assert list(counts) == [tc]
        assert r.n_significant == (1 if tau <= max_tau else 0)


def _edge_doubles(rng):
    vals = [0.0, -0.0, 1.005, 0.29, 4.35, -0.001, -0.01, -1e-300, 5e-324, -5e-324, 1e-310,
            2.2250738585072014e-308, 1.7976931348623157e308, -1.7976931348623157e308,
            math.inf, -math.inf, math.nan, 0.5, -0.5, 21474836.46, 21474836.47, -21474836.47,
            -21474836.48, 2147483646.0, 2147483646.5, 2147483647.0, -2147483647.0, -2147483647.5,
            -2147483648.0, 1e15, 3.0000000000000004]
    for _ in range(3000):
        kind = rng.random()
        if kind < 0.3:  # random bit patterns: all exponents, signs, specials
            vals.append(struct.unpack("<d", struct.pack("<Q", rng.getrandbits(64)))[0])
        elif kind < 0.6:  # typical coordinates
            vals.append(rng.uniform(-3000, 3000))
        else:  # just below / above an integer after scaling by a power of ten
            n = rng.randint(-10**7, 10**7)
            base = n / 10 ** rng.randint(0, 4)
            vals.append(math.nextafter(base, math.inf if rng.random() < 0.5 else -math.inf))
    return vals


SCALES = [1.0, 10.0, 100.0, 1000.0, 10.0 ** 3.5, 10.0 ** 0.9, 10.0 ** 0.73, 10.0 ** 5, 0.1, 7.0, 2.0 ** 20]


@pytest.mark.parametrize("scale", SCALES)
def test_projection_matches_exact_rounding(scale):
    """ix = floor(RN(x * s)): the oracle's one-multiply-then-floor equals exact
    rational arithmetic rounded once to the nearest binary64 value."""
    rng = random.Random(hash(scale) & 0xFFFF)
    xs = _edge_doubles(rng)
    ys = list(reversed(xs))
    xy = np.array([xs, ys], dtype=np.float64).T.copy()
    keys, ok = oracle.project(xy, scale)
    for i, (x, y) in enumerate(zip(xs, ys)):
        ex, ey = oracle.project_exact(x, scale), oracle.project_exact(y, scale)
        if ex is None or ey is None:
            assert not ok[i], (x, y)
        else:
            assert ok[i], (x, y)
            assert keys[i] == oracle.pack(ex, ey), (x, y, scale)


def test_projection_floor_across_zero():
    """Tiles are uniform across the origin: floor, not truncation."""
    xy = np.array([[-0.005, 0.005], [-0.0, 0.0], [-0.01, 0.0099999], [-1e-9, -1e-9]])
    keys, ok = oracle.project(xy, 100.0)
    assert ok.all()
    ix, iy = oracle.unpack(keys)
    assert list(ix) == [-1, 0, -1, -1]
    assert list(iy) == [0, 0, 0, -1]


def test_counts_match_numpy_unique():
    """Counts per tile equal numpy's floor/unique over the same points, and sum to n."""
    w = gen.Workload(n=200_000, clusters=100, cluster_points=150_000, canvas=20.0, precision=2,
                     tau=5, mu=4, seed=11)
    xy = gen.points(w)
    r, o = oracle.raster(xy, 2, 5, 4)
    keys, counts = o.tiles()
    f = np.floor(xy * 100.0).astype(np.int64)
    uk, uc = np.unique(oracle.pack(f[:, 0], f[:, 1]), return_counts=True)
    order = oracle.tile_order(uk)
    assert np.array_equal(keys, uk[order])
    assert np.array_equal(counts, uc[order].astype(np.uint64))
    assert int(counts.sum()) == w.n
    assert r.points == w.n


# ---------------------------------------------------------------------------
# Threshold (Alg. 1 second loop; Sect. 3.6 grid layouts)

def test_grid_layout_fig4():
    rows = _read_fixture("grid_layout.txt")
    d = {}
    for k, v in rows:
        d.setdefault(k, []).append(v)
    p, tau, mu = float(d["precision"][0][0]), int(d["tau"][0][0]), int(d["mu"][0][0])
    split = np.array([[float(a), float(b)] for a, b in d["split"]])
    together = np.array([[float(a), float(b)] for a, b in d["together"]])
    r, _ = oracle.raster(split, p, tau, mu)
    assert r.n_significant == int(d["split_significant"][0][0]) and r.n_clusters == 0
    r, _ = oracle.raster(together, p, tau, mu)
    assert r.n_significant == int(d["together_significant"][0][0]) and r.n_clusters == 1
    tx, ty = [int(v) for v in d["together_tile"][0]]
    assert list(r.key) == [oracle.pack(tx, ty)] and list(r.cid) == [oracle.pack(tx, ty)]


def test_tau_one_makes_every_tile_significant():
    w = gen.Workload(n=20_000, clusters=10, cluster_points=15_000, canvas=5.0, precision=2,
                     tau=1, mu=1, seed=5)
    r, o = oracle.raster(gen.points(w), 2, 1, 1)
    assert r.n_significant == r.n_tiles
    assert len(r.key) == r.n_tiles  # mu = 1 keeps every component


def test_homogeneous_noise_has_no_clusters():
    """Uniform data at the workloads' noise density gives no cluster (App. A)."""
    w = gen.Workload(n=300_000, clusters=1, cluster_points=0, canvas=100.0, precision=2,
                     tau=5, mu=4, seed=9)
    r, _ = oracle.raster(gen.points(w), 2, 5, 4)
    assert r.n_significant == 0 and r.n_clusters == 0


# ---------------------------------------------------------------------------
# Agglomeration (Alg. 1 while loop): against all-pairs union-find, against a
# library connected-component labelling, and against invariants.

def _random_tiles(rng, t, span):
    """Random tile layouts with blobs, lines, diagonals and isolated tiles."""
    pts = []
    for _ in range(t):
        kind = rng.random()
        x0, y0 = rng.randint(-span, span), rng.randint(-span, span)
        if kind < 0.5:
            for _ in range(rng.randint(1, 12)):
                pts.append((x0 + rng.randint(-2, 2), y0 + rng.randint(-2, 2)))
        elif kind < 0.75:
            dx, dy = rng.choice([(1, 1), (1, -1), (1, 0), (0, 1)])
            for s in range(rng.randint(2, 8)):
                pts.append((x0 + s * dx, y0 + s * dy))
        else:
            pts.append((x0, y0))
    return pts


def _points_for_tiles(tiles, scale, rng, max_count=8):
    """Points inside given tiles (tile (a, b) covers [a/s, (a+1)/s) x [b/s, (b+1)/s))."""
    xy = []
    for (a, b) in tiles:
        for _ in range(rng.randint(1, max_count)):
            xy.append(((a + rng.uniform(0.05, 0.95)) / scale, (b + rng.uniform(0.05, 0.95)) / scale))
    rng.shuffle(xy)
    return np.array(xy, dtype=np.float64)


@pytest.mark.parametrize("seed", range(12))
def test_agglomeration_matches_brute_force(seed):
    rng = random.Random(seed)
    tiles = _random_tiles(rng, rng.randint(5, 120), span=rng.choice([6, 15, 40]))
    xy = _points_for_tiles(tiles, 100.0, rng)
    tau, mu = rng.choice([1, 2, 3, 5]), rng.choice([1, 2, 3, 4])
    r, o = oracle.raster(xy, 2, tau, mu)
    keys, counts = o.tiles()
    bk, bc, bcid, bn = oracle.brute_force(keys, counts, tau, mu)
    assert np.array_equal(r.key, bk)
    assert np.array_equal(r.count, bc)
    assert np.array_equal(r.cid, bcid)
    assert r.n_clusters == bn


def test_agglomeration_matches_scipy_label():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = random.Random(77)
    tiles = _random_tiles(rng, 400, span=60)
    xy = _points_for_tiles(tiles, 100.0, rng)
    tau, mu = 3, 3
    r, o = oracle.raster(xy, 2, tau, mu)
    keys, counts = o.tiles()
    ix, iy = oracle.unpack(keys)
    x0, y0 = ix.min(), iy.min()
    grid = np.zeros((ix.max() - x0 + 1, iy.max() - y0 + 1), dtype=bool)
    sig = counts >= tau
    grid[ix[sig] - x0, iy[sig] - y0] = True
    lab, nlab = ndimage.label(grid, structure=np.ones((3, 3), dtype=int))
    sizes = np.bincount(lab.ravel())
    kept_labels = {l for l in range(1, nlab + 1) if sizes[l] >= mu}
    assert r.n_clusters == len(kept_labels)
    rx, ry = oracle.unpack(r.key)
    cx, cy = oracle.unpack(r.cid)
    rl = lab[rx - x0, ry - y0]
    assert set(rl.tolist()) == kept_labels
    assert len(r.key) == sum(sizes[l] for l in kept_labels)
    for l in kept_labels:  # one id per component, and it is the (ix, iy)-smallest member
        sel = rl == l
        members = np.argwhere(lab == l)
        best = members[np.lexsort((members[:, 1], members[:, 0]))[0]]
        assert set(zip(cx[sel].tolist(), cy[sel].tolist())) == {(best[0] + x0, best[1] + y0)}


def check_invariants(r, keys, counts, tau, mu, n_points):
    """Properties any correct RASTER result has (usable at any size)."""
    assert int(np.asarray(counts, dtype=np.uint64).sum()) == n_points
    assert len(np.unique(r.key)) == len(r.key)  # clusters are disjoint
    assert (r.count >= tau).all()
    cnt_of = dict(zip(keys.tolist(), counts.tolist()))
    assert all(cnt_of[k] == c for k, c in zip(r.key.tolist(), r.count.tolist()))
    sig = set(k for k, c in cnt_of.items() if c >= tau)
    cid_of = dict(zip(r.key.tolist(), r.cid.tolist()))
    members = {}
    for k, c in cid_of.items():
        members.setdefault(c, []).append(k)
    assert len(members) == r.n_clusters
    for c, ms in members.items():
        assert len(ms) >= mu
        assert c in ms and min(ms, key=lambda k: (k >> 32, np.int32(np.uint32(k & 0xFFFFFFFF)))) == c
    # a significant neighbour of a kept tile is kept, in the same cluster;
    # each cluster is 8-connected (flood fill within it reaches all members)
    def nbrs(k):
        x, y = k >> 32, int(np.int32(np.uint32(k & 0xFFFFFFFF)))
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                if dx or dy:
                    yield int(oracle.pack(x + dx, y + dy))
    for k in cid_of:
        for nb in nbrs(k):
            if nb in sig:
                assert cid_of.get(nb) == cid_of[k]
    for c, ms in members.items():
        seen, stack, mset = {ms[0]}, [ms[0]], set(ms)
        while stack:
            u = stack.pop()
            for nb in nbrs(u):
                if nb in mset and nb not in seen:
                    seen.add(nb)
                    stack.append(nb)
        assert seen == mset


def test_invariants_on_clustered_workload():
    w = gen.Workload(n=100_000, clusters=100, cluster_points=90_000, canvas=10.0, precision=2,
                     tau=5, mu=4, seed=21)
    xy = gen.points(w)
    r, o = oracle.raster(xy, 2, 5, 4)
    keys, counts = o.tiles()
    check_invariants(r, keys, counts, 5, 4, w.n)
    assert r.n_clusters > 10


def test_chunking_and_order_do_not_change_result():
    """Sect. 3.6: input may be partitioned and processed in any order."""
    w = gen.Workload(n=50_000, clusters=40, cluster_points=45_000, canvas=5.0, precision=2,
                     tau=4, mu=3, seed=31)
    xy = gen.points(w)
    base, _ = oracle.raster(xy, 2, 4, 3)
    perm = np.random.default_rng(0).permutation(w.n)
    for chunks in (1, 3, 17):
        r, _ = oracle.raster(xy[perm], 2, 4, 3, chunks=chunks)
        assert np.array_equal(r.key, base.key) and np.array_equal(r.cid, base.cid)
        assert np.array_equal(r.count, base.count) and r.n_clusters == base.n_clusters


def test_labels_follow_kept_tiles():
    w = gen.Workload(n=30_000, clusters=30, cluster_points=27_000, canvas=4.0, precision=2,
                     tau=5, mu=4, seed=41)
    xy = gen.points(w)
    r, lab, o = oracle.raster(xy, 2, 5, 4, with_labels=True)
    cid_of = dict(zip(r.key.tolist(), r.cid.tolist()))
    f = np.floor(xy * 100.0).astype(np.int64)
    k = oracle.pack(f[:, 0], f[:, 1])
    expect = np.array([cid_of.get(int(v), oracle.NOISE) for v in k], dtype=np.int64)
    assert np.array_equal(lab, expect)
    assert (lab != oracle.NOISE).sum() > 0


def test_point_groups_raster_prime():
    """RASTER' (Sect. 3.4) returns clusters as points: every grouped point lies
    in its row's tile (numpy's floor decides), each row holds exactly that
    tile's count, and the grouped points are exactly the labelled ones."""
    w = gen.Workload(n=40_000, clusters=40, cluster_points=36_000, canvas=4.0, precision=2, tau=5, mu=4, seed=51)
    xy = gen.points(w)
    r, lab, o = oracle.raster(xy, 2, 5, 4, with_labels=True)
    row_start, idx = o.point_groups(xy)
    assert row_start[0] == 0 and len(row_start) == len(r.key) + 1
    assert np.array_equal(np.diff(row_start), r.count.astype(np.int64))
    f = np.floor(xy * 100.0).astype(np.int64)
    pk = oracle.pack(f[:, 0], f[:, 1])
    for row in range(len(r.key)):
        members = idx[row_start[row]:row_start[row + 1]]
        assert np.all(pk[members] == r.key[row])
        assert np.all(np.diff(members) > 0)
    assert np.array_equal(np.sort(idx), np.flatnonzero(lab != oracle.NOISE))


def test_range_errors_are_reported_and_skipped():
    xy = np.array([[0.5, 0.5], [math.nan, 0.5], [0.5, math.inf], [3e7, 0.5], [0.51, 0.52]])
    o = oracle.Oracle(2, 1, 1)
    st = o.add(xy)
    assert st == oracle.E_RANGE
    keys, counts = o.tiles()
    assert list(keys) == [oracle.pack(50, 50), oracle.pack(51, 52)]
    assert int(counts.sum()) == 2
    st, lab = o.labels(xy)
    assert st == oracle.E_RANGE and lab[1] == oracle.NOISE and lab[3] == oracle.NOISE


# ---------------------------------------------------------------------------
# P-RASTER (Sect. 3.5, Alg. 2-3; App. C Theorem 3): slicing the tile space
# into vertical slices, clustering each slice, and joining clusters across
# borders gives the same clusters as Alg. 1 -- for any slicing.

def _p_raster_agglomerate(sig_tiles, mu, borders):
    """A direct restatement of P-RASTER's agglomeration: per-slice clusters,
    clusters touching a border become join candidates, borders are joined one
    at a time from right to left, carrying clusters that touch the next border."""
    cols = sorted(set(borders))
    slice_of = lambda x: sum(1 for b in cols if x >= b)  # slice index by column
    nslices = len(cols) + 1
    by_slice = [set() for _ in range(nslices)]
    for t in sig_tiles:
        by_slice[slice_of(t[0])].add(t)

    def nb(t):
        return [(t[0] + dx, t[1] + dy) for dx in (-1, 0, 1) for dy in (-1, 0, 1) if dx or dy]

    def touches(c, i):  # cluster c touches border i (between slice i-1 and i)
        return any(slice_of(n[0]) != slice_of(t[0]) and
                   {slice_of(n[0]), slice_of(t[0])} == {i - 1, i} for t in c for n in nb(t))

    result, cand = [], []
    for s in range(nslices):
        rest = set(by_slice[s])
        while rest:
            t = rest.pop()
            c, stack = {t}, [t]
            while stack:
                u = stack.pop()
                for v in nb(u):
                    if v in rest:
                        rest.discard(v)
                        c.add(v)
                        stack.append(v)
            if any(touches(c, i) for i in (s, s + 1) if 1 <= i < nslices):
                cand.append(c)
            elif len(c) >= mu:
                result.append(c)
    for i in range(nslices - 1, 0, -1):
        clr = [c for c in cand if touches(c, i)]
        cand = [c for c in cand if not touches(c, i)]
        joined_all = []
        while clr:
            cj = set(clr.pop())
            grew = True
            while grew:
                grew = False
                for c in list(clr):
                    if any(v in c for u in cj for v in nb(u)):
                        cj |= c
                        clr.remove(c)
                        grew = True
            joined_all.append(cj)
        for cj in joined_all:
            if i - 1 >= 1 and touches(cj, i - 1):
                cand.append(cj)
            elif len(cj) >= mu:
                result.append(cj)
    for c in cand:  # candidates left touching no unjoined border
        if len(c) >= mu:
            result.append(c)
    return sorted(sorted(c) for c in result)


@pytest.mark.parametrize("seed", range(6))
def test_arbitrary_slicing_invariant(seed):
    rng = random.Random(100 + seed)
    tiles = _random_tiles(rng, 60, span=20)
    xy = _points_for_tiles(tiles, 100.0, rng)
    tau, mu = 2, 3
    r, o = oracle.raster(xy, 2, tau, mu)
    keys, counts = o.tiles()
    ix, iy = oracle.unpack(keys[counts >= tau])
    sig = list(zip(ix.tolist(), iy.tolist()))
    rx, ry = oracle.unpack(r.key)
    clusters = {}
    for x, y, c in zip(rx.tolist(), ry.tolist(), r.cid.tolist()):
        clusters.setdefault(c, []).append((x, y))
    expect = sorted(sorted(c) for c in clusters.values())
    for _ in range(4):
        borders = sorted(rng.sample(range(-22, 23), rng.randint(1, 6)))
        assert _p_raster_agglomerate(sig, mu, borders) == expect


# ---------------------------------------------------------------------------
# Extensions: the 2 x 2 group rule of Sect. 3.6 and neighbors(u, delta) for a
# Chebyshev or Manhattan distance delta (Sect. 3.2).

def test_grid_layout_fig4_with_groups():
    rows = _read_fixture("grid_layout.txt")
    d = {}
    for k, v in rows:
        d.setdefault(k, []).append(v)
    p, tau, mu = float(d["precision"][0][0]), int(d["tau"][0][0]), int(d["mu"][0][0])
    split = np.array([[float(a), float(b)] for a, b in d["split"]])
    r, _ = oracle.raster(split, p, tau, mu, groups=True)
    assert r.n_significant == int(d["split_groups_significant"][0][0])
    assert r.n_clusters == int(d["split_groups_clusters"][0][0])
    # without the rule the same points give nothing (Fig. 4)
    r, _ = oracle.raster(split, p, tau, mu)
    assert r.n_significant == 0


def _window_significant(keys, counts, tau):
    """Tiles kept by the 2 x 2 group rule, from window sums over a dense grid
    (numpy slicing; independent of the oracle's hash-map walk)."""
    ix, iy = oracle.unpack(keys)
    x0, y0 = int(ix.min()) - 1, int(iy.min()) - 1
    grid = np.zeros((int(ix.max()) - x0 + 2, int(iy.max()) - y0 + 2), dtype=np.int64)
    grid[ix - x0, iy - y0] = counts
    win = grid[:-1, :-1] + grid[1:, :-1] + grid[:-1, 1:] + grid[1:, 1:]  # anchored at (x, y): x..x+1, y..y+1
    ok = win >= tau
    gx, gy = ix - x0, iy - y0
    # a tile belongs to the windows anchored at (x-1|x, y-1|y)
    return ok[gx - 1, gy - 1] | ok[gx - 1, gy] | ok[gx, gy - 1] | ok[gx, gy] | (counts >= tau)


@pytest.mark.parametrize("seed", range(8))
def test_groups_match_window_sums_and_brute_force(seed):
    rng = random.Random(100 + seed)
    tiles = _random_tiles(rng, rng.randint(10, 120), span=rng.choice([8, 20]))
    xy = _points_for_tiles(tiles, 100.0, rng, max_count=4)
    tau, mu = rng.choice([3, 4, 6]), rng.choice([1, 2, 3])
    r, o = oracle.raster(xy, 2, tau, mu, groups=True)
    keys, counts = o.tiles()
    sig = _window_significant(keys, counts.astype(np.int64), tau)
    assert r.n_significant == int(sig.sum())
    bk, bc, bcid, bn = oracle.brute_force(keys, counts, tau, mu, significant=sig)
    assert np.array_equal(r.key, bk) and np.array_equal(r.cid, bcid) and np.array_equal(r.count, bc)
    assert r.n_clusters == bn
    # the rule only adds tiles: every plain significant tile is still significant
    rp, _ = oracle.raster(xy, 2, tau, 1)
    assert set(rp.key.tolist()) <= set(_kept_all(xy, tau).tolist())


def _kept_all(xy, tau):
    r, _ = oracle.raster(xy, 2, tau, 1, groups=True)
    return r.key


@pytest.mark.parametrize("metric,delta", [(oracle.CHEBYSHEV, 2), (oracle.CHEBYSHEV, 3), (oracle.MANHATTAN, 1),
                                          (oracle.MANHATTAN, 2), (oracle.MANHATTAN, 3)])
@pytest.mark.parametrize("seed", range(4))
def test_delta_metrics_match_brute_force(metric, delta, seed):
    rng = random.Random(200 + seed)
    tiles = _random_tiles(rng, rng.randint(10, 100), span=rng.choice([10, 25]))
    xy = _points_for_tiles(tiles, 100.0, rng)
    tau, mu = rng.choice([1, 2, 3]), rng.choice([1, 2, 4])
    r, o = oracle.raster(xy, 2, tau, mu, metric=metric, delta=delta)
    keys, counts = o.tiles()
    bk, bc, bcid, bn = oracle.brute_force(keys, counts, tau, mu, metric=metric, delta=delta)
    assert np.array_equal(r.key, bk) and np.array_equal(r.cid, bcid) and np.array_equal(r.count, bc)
    assert r.n_clusters == bn


def test_manhattan_one_matches_scipy_cross_labelling():
    """Manhattan distance 1 is 4-connectivity: scipy's labelling with the cross
    structure gives the same components."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = random.Random(7)
    tiles = _random_tiles(rng, 150, span=20)
    xy = _points_for_tiles(tiles, 100.0, rng)
    r, o = oracle.raster(xy, 2, 2, 1, metric=oracle.MANHATTAN, delta=1)
    keys, counts = o.tiles()
    sig = keys[counts >= 2]
    ix, iy = oracle.unpack(sig)
    x0, y0 = int(ix.min()), int(iy.min())
    grid = np.zeros((int(ix.max()) - x0 + 1, int(iy.max()) - y0 + 1), dtype=bool)
    grid[ix - x0, iy - y0] = True
    lab, n = ndimage.label(grid, structure=ndimage.generate_binary_structure(2, 1))
    assert r.n_clusters == n
    comp = lab[ix - x0, iy - y0]
    by_key = dict(zip(r.key.tolist(), r.cid.tolist()))
    for c in range(1, n + 1):
        members = sig[comp == c]
        assert len({by_key[int(k)] for k in members}) == 1


def test_delta_hand_cases():
    """Two tiles two steps apart join under Chebyshev 2, not under Chebyshev 1;
    a knight's move (2, 1) joins under Chebyshev 2 but not under Manhattan 2."""
    def clusters(tiles, metric, delta):
        xy = np.array([[(a + 0.5) / 100.0, (b + 0.5) / 100.0] for a, b in tiles])
        r, _ = oracle.raster(xy, 2, 1, 1, metric=metric, delta=delta)
        return r.n_clusters
    assert clusters([(0, 0), (2, 0)], oracle.CHEBYSHEV, 1) == 2
    assert clusters([(0, 0), (2, 0)], oracle.CHEBYSHEV, 2) == 1
    assert clusters([(0, 0), (1, 1)], oracle.MANHATTAN, 1) == 2
    assert clusters([(0, 0), (1, 1)], oracle.MANHATTAN, 2) == 1
    assert clusters([(0, 0), (2, 1)], oracle.CHEBYSHEV, 2) == 1
    assert clusters([(0, 0), (2, 1)], oracle.MANHATTAN, 2) == 2
    assert clusters([(0, 0), (2, 1)], oracle.MANHATTAN, 3) == 1


# ---------------------------------------------------------------------------
# Three coordinates (Sect. 3.6, "Generalizing to Higher Dimensions").

def _points3_for_tiles(tiles, scale, rng, max_count=6):
    xyz = []
    for t in tiles:
        for _ in range(rng.randint(1, max_count)):
            xyz.append(tuple((c + rng.uniform(0.05, 0.95)) / scale for c in t))
    rng.shuffle(xyz)
    return np.array(xyz, dtype=np.float64)


def _random_tiles3(rng, t, span):
    out = []
    for _ in range(t):
        x0, y0, z0 = (rng.randint(-span, span) for _ in range(3))
        if rng.random() < 0.6:
            for _ in range(rng.randint(1, 10)):
                out.append((x0 + rng.randint(-1, 1), y0 + rng.randint(-1, 1), z0 + rng.randint(-1, 1)))
        else:
            out.append((x0, y0, z0))
    return out


def test_3d_counts_match_numpy_unique():
    g = np.random.default_rng(31)
    xyz = np.concatenate([g.uniform(-5, 5, (50_000, 3)), g.normal(1.0, 0.02, (30_000, 3))])
    r, o = oracle.raster(xyz, 2, 3, 2)
    keys, counts = o.tiles()
    f = np.floor(xyz * 100.0).astype(np.int64)
    uk, uc = np.unique(oracle.pack3(f[:, 0], f[:, 1], f[:, 2]), return_counts=True)
    assert np.array_equal(keys, uk) and np.array_equal(counts, uc.astype(np.uint64))  # integer order is (x, y, z) order
    assert r.points == xyz.shape[0] and r.n_tiles == len(uk)


def test_3d_projection_range():
    """Each index must lie in [-(2^20 - 1), 2^20 - 2]."""
    lo, hi = -(2 ** 20 - 1), 2 ** 20 - 2
    xyz = np.array([[lo + 0.5, 0.5, 0.5], [hi + 0.5, 0.5, 0.5], [lo - 0.5, 0.5, 0.5], [hi + 1.5, 0.5, 0.5],
                    [0.5, np.nan, 0.5], [0.5, 0.5, -np.inf]])
    keys, ok = oracle.project(xyz, 1.0)
    assert ok.tolist() == [True, True, False, False, False, False]
    x, y, z = oracle.unpack3(keys[:2])
    assert x.tolist() == [lo, hi] and y.tolist() == [0, 0] and z.tolist() == [0, 0]


@pytest.mark.parametrize("metric,full", [(oracle.CHEBYSHEV, 3), (oracle.MANHATTAN, 1)])
@pytest.mark.parametrize("seed", range(3))
def test_3d_components_match_scipy_labelling(metric, full, seed):
    """Chebyshev distance 1 in 3-D is 26-connectivity and Manhattan 1 is
    6-connectivity: scipy's labelling with the matching structure gives the
    same components."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = random.Random(500 + seed)
    xyz = _points3_for_tiles(_random_tiles3(rng, 120, 8), 100.0, rng)
    tau = 2
    r, o = oracle.raster(xyz, 2, tau, 1, metric=metric)
    keys, counts = o.tiles()
    sig = keys[counts >= tau]
    c = np.stack(oracle.unpack3(sig), axis=1)
    c0 = c.min(axis=0)
    grid = np.zeros(tuple(c.max(axis=0) - c0 + 1), dtype=bool)
    grid[tuple((c - c0).T)] = True
    lab, n = ndimage.label(grid, structure=ndimage.generate_binary_structure(3, full))
    assert r.n_clusters == n
    comp = lab[tuple((c - c0).T)]
    by_key = dict(zip(r.key.tolist(), r.cid.tolist()))
    for k in range(1, n + 1):
        members = sig[comp == k]
        cids = {by_key[int(m)] for m in members}
        assert cids == {int(members.min())}  # id = lexicographically smallest tile = smallest key


@pytest.mark.parametrize("metric,delta", [(oracle.MANHATTAN, 2), (oracle.MANHATTAN, 3), (oracle.CHEBYSHEV, 1)])
@pytest.mark.parametrize("seed", range(3))
def test_3d_match_brute_force(metric, delta, seed):
    rng = random.Random(600 + seed)
    xyz = _points3_for_tiles(_random_tiles3(rng, 60, 10), 100.0, rng)
    tau, mu = rng.choice([1, 2, 3]), rng.choice([1, 2, 3])
    r, o = oracle.raster(xyz, 2, tau, mu, metric=metric, delta=delta)
    keys, counts = o.tiles()
    bk, bc, bcid, bn = oracle.brute_force(keys, counts, tau, mu, metric=metric, delta=delta, dims=3)
    assert np.array_equal(r.key, bk) and np.array_equal(r.cid, bcid) and np.array_equal(r.count, bc)
    assert r.n_clusters == bn


def test_3d_labels_and_groups():
    rng = random.Random(77)
    xyz = _points3_for_tiles(_random_tiles3(rng, 80, 6), 100.0, rng)
    r, lab, o = oracle.raster(xyz, 2, 2, 2, with_labels=True)
    keys, ok = oracle.project(xyz, 100.0)
    cid_of = dict(zip(r.key.tolist(), r.cid.tolist()))
    assert lab.tolist() == [cid_of.get(int(k), int(oracle.NOISE)) for k in keys]
    rs, idx = o.point_groups(xyz)
    for i, k in enumerate(r.key.tolist()):
        assert set(idx[rs[i]:rs[i + 1]].tolist()) == set(np.flatnonzero(keys == k).tolist())


def _count_keys_reference(xy, scale, keys):
    """Counts of the given tiles by numpy: floor of the scaled coordinates,
    rows with a non-finite or out-of-range index dropped, then a membership
    count per queried key."""
    with np.errstate(invalid="ignore", over="ignore"):
        f = np.floor(xy * scale)
    dims = xy.shape[1]
    lo, hi = (-(2**31 - 1), 2**31 - 2) if dims == 2 else (-(2**20 - 1), 2**20 - 2)
    ok = np.all(np.isfinite(f) & (f >= lo) & (f <= hi), axis=1)
    g = f[ok].astype(np.int64)
    pk = oracle.pack(g[:, 0], g[:, 1]) if dims == 2 else oracle.pack3(g[:, 0], g[:, 1], g[:, 2])
    uk, uc = np.unique(pk, return_counts=True)
    i = np.minimum(np.searchsorted(uk, keys), len(uk) - 1)
    return np.where(uk[i] == keys, uc[i], 0).astype(np.uint64)


@pytest.mark.parametrize("dims", [2, 3])
def test_count_keys_matches_numpy(dims):
    """oracle.count_keys recounts chosen tiles over a point set (the checker of
    the sampled large-workload tests): equal to numpy's floor + unique, with
    range-error points mixed in, absent and duplicated query keys, and the
    query order kept."""
    g = np.random.default_rng(40 + dims)
    xy = np.concatenate([g.uniform(0, 0.3, (20000, dims)), g.uniform(-2, 2, (5000, dims))])
    bad = np.array([[np.nan] * dims, [np.inf] * dims, [-np.inf] * dims, [3.0e7] * dims, [-2.2e7] * dims])
    xy = np.concatenate([xy, bad])[g.permutation(len(xy) + len(bad))]
    scale = 100.0
    keys_all, ok = oracle.project(xy, scale)
    present = np.unique(keys_all[ok])
    f = g.integers(-300, 300, (50, dims))
    absent = oracle.pack(f[:, 0], f[:, 1]) if dims == 2 else oracle.pack3(f[:, 0], f[:, 1], f[:, 2])
    q = np.concatenate([g.choice(present, 400, replace=False), absent, present[:3], present[:3]])
    q = q[g.permutation(len(q))]
    got = oracle.count_keys(xy, scale, q)
    want = _count_keys_reference(xy, scale, q)
    assert np.array_equal(got, want)
    assert int(got[np.isin(q, present)].min()) >= 1
    # the whole tile set recounted equals the oracle's own table
    o = oracle.Oracle(2, 1, 1, dims=dims)
    o.add(xy)
    tk, tc = o.tiles()
    assert np.array_equal(oracle.count_keys(xy, scale, tk), tc)
