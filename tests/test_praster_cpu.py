"""The multi-threaded P-RASTER baseline (Sect. 3.5, Alg. 2-3) against the
single-threaded oracle: by the arbitrary-slicing invariant (App. C, Theorem 3)
the slices and border joins must give exactly Alg. 1's clusters, whatever the
number of threads (which is also the number of slices).  The shapes cross
slice borders once, many times (a snake), along a border, and through
several slices; the counts, rows, ids and labels must all be equal.  CPU."""
import numpy as np
import pytest

import gen
import oracle


def _points_on_tiles(tiles, per, rng, scale=100.0):
    """`per` points uniformly inside each tile (ix, iy) at scale 100."""
    tiles = np.asarray(tiles, dtype=np.float64)
    out = np.repeat(tiles, per, axis=0) + rng.uniform(0.05, 0.95, (len(tiles) * per, 2))
    return out / scale


def _shapes(rng):
    tiles = []
    # a horizontal band across the whole canvas: crosses every border
    tiles += [(x, 0) for x in range(0, 400)]
    # a snake that crosses the same borders back and forth
    for k in range(12):
        x0 = 30 * k
        tiles += [(x0 + d, 10 + (k % 2) * 6) for d in range(31)]
        tiles += [(x0 + 30, 10 + j) for j in range(7)]
    # a vertical line and a diagonal
    tiles += [(200, y) for y in range(30, 90)]
    tiles += [(100 + d, 40 + d) for d in range(120)]
    # scattered small blobs (some below mu)
    for _ in range(300):
        x, y = rng.integers(0, 400), rng.integers(100, 300)
        tiles += [(x + dx, y + dy) for dx in range(rng.integers(1, 3)) for dy in range(rng.integers(1, 3))]
    return sorted(set(tiles))


@pytest.mark.parametrize("threads", [1, 2, 3, 5, 8, 13])
def test_praster_equals_oracle_on_border_crossing_shapes(threads):
    rng = np.random.default_rng(threads)
    xy = _points_on_tiles(_shapes(rng), 6, rng)
    noise = rng.uniform(0, 4.0, (20000, 2))
    xy = np.concatenate([xy, noise])[rng.permutation(len(xy) + len(noise))]
    ref, lab, _ = oracle.raster(xy, 2, 5, 4, with_labels=True)
    got, glab, _ = oracle.praster(xy, 2, 5, 4, threads, with_labels=True)
    assert (got.n_tiles, got.n_significant, got.n_clusters) == (ref.n_tiles, ref.n_significant, ref.n_clusters)
    assert np.array_equal(got.key, ref.key) and np.array_equal(got.count, ref.count)
    assert np.array_equal(got.cid, ref.cid)
    assert np.array_equal(glab, lab)


@pytest.mark.parametrize("threads", [4, 16])
def test_praster_equals_oracle_on_generated_workload(threads):
    w = gen.Workload(n=400_000, clusters=800, cluster_points=360_000, canvas=60.0, precision=2, tau=5, mu=4,
                     seed=77)
    xy = gen.points(w)
    xy[123] = (np.nan, 1.0)  # a range error is reported and the point skipped
    ref, lab, _ = oracle.raster(xy, w.precision, w.tau, w.mu, with_labels=True)
    got, glab, secs = oracle.praster(xy, w.precision, w.tau, w.mu, threads, with_labels=True)
    assert ref.status == got.status == oracle.E_RANGE
    assert got.n_clusters == ref.n_clusters and got.n_tiles == ref.n_tiles
    assert np.array_equal(got.key, ref.key) and np.array_equal(got.cid, ref.cid)
    assert np.array_equal(got.count, ref.count) and np.array_equal(glab, lab)
    assert min(secs.values()) >= 0.0
