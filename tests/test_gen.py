"""The seeded input generator: deterministic, sliceable, and of the stated shape."""
import numpy as np

import gen


def test_slices_equal_whole_and_deterministic():
    w = gen.Workload(n=100_003, clusters=37, cluster_points=90_000, canvas=7.0, precision=2,
                     tau=5, mu=4, seed=123)
    a = gen.points(w, nthreads=3)
    b = gen.points(w, nthreads=1)
    assert np.array_equal(a, b)
    assert np.array_equal(a[5000:70001], gen.points(w, 5000, 70001))


def test_permutation_is_a_bijection():
    for n in (1, 2, 3, 17, 1000, 4097):
        assert sorted(gen.perm_apply(n, 9, i) for i in range(n)) == list(range(n))


def test_shape_of_workload():
    w = gen.Workload(n=200_000, clusters=100, cluster_points=180_000, canvas=50.0, precision=2,
                     tau=5, mu=4, seed=5, shuffle=False)
    xy = gen.points(w)
    cl, noise = xy[:180_000], xy[180_000:]
    assert noise.min() >= 0.0 and noise.max() < 50.0
    # points of cluster c are at positions c, c+K, c+2K, ... and lie in a 0.1-wide square
    for c in (0, 7, 99):
        pts = cl[c::100]
        assert len(pts) == 1800
        span = pts.max(0) - pts.min(0)
        assert (span <= 0.1).all() and (span > 0.09).all()


def test_batched_instances_follow_recipe():
    inst = gen.batch_instances(count=256)
    sizes = np.array([w.n for w in inst])
    assert sizes.min() >= 1000 and sizes.max() < 2_000_000
    for w in inst:
        assert w.precision in (1, 2, 3) and w.tau in (3, 5, 8) and w.mu in (2, 4)
        assert w.cluster_points == w.n - int(w.n * 0.10)
        assert w.clusters == max(1, w.n // 500)


def test_cubes3_deterministic_and_in_range():
    a = gen.cubes3(50, 40, 0.1, 5.0, 300, 9)
    b = gen.cubes3(50, 40, 0.1, 5.0, 300, 9)
    assert a.shape == (50 * 40 + 300, 3) and np.array_equal(a, b)
    assert a.min() >= -0.05 and a.max() <= 5.05
