"""Planted mistakes: each test compiles a copy of the oracle with one
deliberate error (a dropped term, a wrong comparison, a transposed operand...)
and checks that the oracle's pins reject it.  CPU only."""
import os
import random

import numpy as np
import pytest

import gen
import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "raster_oracle.cpp")

MUTANTS = {
    "four_connected": ("if (dx == 0 && dy == 0 && dz == 0) continue;",
                       "if (dx == 0 && dy == 0 && dz == 0) continue;\n if (dx != 0 && dy != 0) continue;"),
    "strict_tau": ("kv.second >= s->tau", "kv.second > s->tau"),
    "truncate_not_floor": ("std::floor(scaled)", "std::trunc(scaled)"),
    "strict_mu": ("cluster.size() >= s->mu", "cluster.size() > s->mu"),
    "max_id": ("if (before(s, k, cid)) cid = k;", "if (before(s, cid, k)) cid = k;"),
    "transposed_key": ("*key = pack(ix, iy);", "*key = pack(iy, ix);"),
    "single_precision_scale": ("v * scale", "v * (double)(float)scale"),
    "lost_increment": ("        else\n            it->second += 1;",
                       "        else\n            it->second += (it->second > 3) ? 0 : 1;"),
    "range_off_by_one": ("f <= 2147483646.0", "f <= 2147483647.0"),
    "group_window_2x1": ("for (int gy = 0; gy <= 1; ++gy)", "for (int gy = 0; gy <= 0; ++gy)"),
    "group_strict_tau": ("if (total >= s->tau) keep = true;", "if (total > s->tau) keep = true;"),
    "manhattan_strict": ("std::abs(dx) + std::abs(dy) + std::abs(dz) > s->delta",
                         "std::abs(dx) + std::abs(dy) + std::abs(dz) >= s->delta"),
    "delta_ignored": ("for (int dx = -s->delta; dx <= s->delta; ++dx)", "for (int dx = -1; dx <= 1; ++dx)"),
    "third_axis_ignored": ("const int dz_max = s->dims == 3 ? s->delta : 0;", "const int dz_max = 0;"),
    "third_field_shift": ("((iy + BIAS3) << 21)", "((iy + BIAS3) << 20)"),
    "count_keys_lost_count": ("if (it != tally.end()) it->second += 1;",
                              "if (it != tally.end()) it->second = 1;"),
    "count_keys_counts_range_errors": ("if (!project_point(xy, i, dims, scale, &key)) continue;",
                                       "if (!project_point(xy, i, dims, scale, &key)) key = 0;"),
    "count_keys_two_dims": ("if (!project_point(xy, i, dims, scale, &key)) continue;",
                            "if (!project_point(xy, i, 2, scale, &key)) continue;"),
    "count_keys_one_slot_per_key": ("for (int64_t j = 0; j < k; ++j) counts[j] = tally.at(keys[j]);",
                                    "for (int64_t j = 0; j < k; ++j) counts[j] = tally.at(keys[j]);\n"
                                    " for (int64_t j = 1; j < k; ++j) if (keys[j] == keys[j - 1]) counts[j] = 0;"),
}


def _pins_pass(lib) -> bool:
    """A compact run of the oracle pins; False as soon as one disagrees."""
    # Sect. 3.2 worked example
    pts = np.array([[1.005, 1.000], [1.009, 1.002], [1.008, 1.006]])
    r, o = oracle.raster(pts, 2, 3, 1, lib=lib)
    k, c = o.tiles()
    if list(k) != [oracle.pack(100, 100)] or list(c) != [3] or r.n_significant != 1:
        return False
    # exact rounding of the product, incl. negatives and range limits
    rng = random.Random(5)
    xs = [rng.uniform(-30, 30) for _ in range(300)] + [-0.005, 0.29, 21474836.46, 21474836.47,
                                                       -21474836.47, 1.0 + 2 ** -40]
    xy = np.array([xs, xs[::-1]]).T.copy()
    for p in (2, 3.5, 0.73):
        s = oracle.scale_of(p)
        o = oracle.Oracle(p, 1, 1, lib=lib)
        o.add(xy)
        keys, _ = o.tiles()
        expect = set()
        for x, y in xy:
            ex, ey = oracle.project_exact(x, s), oracle.project_exact(y, s)
            if ex is not None and ey is not None:
                expect.add(int(oracle.pack(ex, ey)))
        if set(keys.tolist()) != expect:
            return False
    # counts vs numpy, and all-pairs agglomeration
    for seed in range(6):
        rng = random.Random(seed)
        tiles = []
        for _ in range(40):
            x0, y0 = rng.randint(-15, 15), rng.randint(-15, 15)
            for _ in range(rng.randint(1, 6)):
                tiles.append((x0 + rng.randint(-1, 1), y0 + rng.randint(-1, 1)))
        xy = []
        for (a, b) in tiles:
            for _ in range(rng.randint(1, 9)):
                xy.append(((a + rng.uniform(0.05, 0.95)) / 100.0, (b + rng.uniform(0.05, 0.95)) / 100.0))
        xy = np.array(xy)
        tau, mu = rng.choice([2, 3, 5]), rng.choice([2, 3, 4])
        r, o = oracle.raster(xy, 2, tau, mu, lib=lib)
        keys, counts = o.tiles()
        f = np.floor(xy * 100.0).astype(np.int64)
        uk, uc = np.unique(oracle.pack(f[:, 0], f[:, 1]), return_counts=True)
        if sorted(zip(keys.tolist(), counts.tolist())) != sorted(zip(uk.tolist(), uc.tolist())):
            return False
        bk, bc, bcid, bn = oracle.brute_force(uk, uc, tau, mu)
        if not (np.array_equal(r.key, bk) and np.array_equal(r.cid, bcid) and r.n_clusters == bn
                and np.array_equal(r.count, bc)):
            return False
        # neighbors(u, delta) for the other metrics and radii (Sect. 3.2)
        for metric, delta in ((oracle.CHEBYSHEV, 2), (oracle.MANHATTAN, 1), (oracle.MANHATTAN, 2)):
            r, _ = oracle.raster(xy, 2, tau, mu, lib=lib, metric=metric, delta=delta)
            bk, bc, bcid, bn = oracle.brute_force(uk, uc, tau, mu, metric=metric, delta=delta)
            if not (np.array_equal(r.key, bk) and np.array_equal(r.cid, bcid) and r.n_clusters == bn):
                return False
        # the 2 x 2 group rule (Sect. 3.6) against window sums over a dense grid
        r, _ = oracle.raster(xy, 2, tau, mu, lib=lib, groups=True)
        sig = _window_significant(uk, uc.astype(np.int64), tau)
        bk, bc, bcid, bn = oracle.brute_force(uk, uc, tau, mu, significant=sig)
        if not (np.array_equal(r.key, bk) and np.array_equal(r.cid, bcid) and r.n_clusters == bn
                and r.n_significant == int(sig.sum())):
            return False
    # recounts of chosen tiles (the checker of sampled large runs) against numpy;
    # query keys duplicated, absent, and the key 0 that a skipped point must not reach
    if not _count_keys_pass(lib):
        return False
    # three coordinates: counts against numpy, components against scipy (26-connectivity)
    g = np.random.default_rng(3)
    xyz = np.concatenate([g.uniform(0, 0.2, (4000, 3)), g.uniform(-1, 1, (3000, 3))])
    r, o = oracle.raster(xyz, 2, 2, 1, lib=lib)
    keys, counts = o.tiles()
    f = np.floor(xyz * 100.0).astype(np.int64)
    uk, uc = np.unique(oracle.pack3(f[:, 0], f[:, 1], f[:, 2]), return_counts=True)
    if not (np.array_equal(keys, uk) and np.array_equal(counts, uc.astype(np.uint64))):
        return False
    ndimage = pytest.importorskip("scipy.ndimage")
    sig = uk[uc >= 2]
    c = np.stack(oracle.unpack3(sig), axis=1)
    c0 = c.min(axis=0)
    grid = np.zeros(tuple(c.max(axis=0) - c0 + 1), dtype=bool)
    grid[tuple((c - c0).T)] = True
    _, n = ndimage.label(grid, structure=ndimage.generate_binary_structure(3, 3))
    if r.n_clusters != n:
        return False
    return True


def _count_keys_pass(lib) -> bool:
    g = np.random.default_rng(11)
    for dims in (2, 3):
        xy = np.concatenate([g.uniform(-0.05, 0.2, (3000, dims)),
                             np.array([[np.nan] * dims, [np.inf] * dims, [4.0e7] * dims])])
        with np.errstate(invalid="ignore", over="ignore"):
            f = np.floor(xy * 100.0)
        lim = 2**31 - 2 if dims == 2 else 2**20 - 2
        ok = np.all(np.isfinite(f) & (np.abs(f) <= lim), axis=1)
        f = f[ok].astype(np.int64)
        pk = oracle.pack(f[:, 0], f[:, 1]) if dims == 2 else oracle.pack3(f[:, 0], f[:, 1], f[:, 2])
        uk, uc = np.unique(pk, return_counts=True)
        q = np.concatenate([uk[:40], uk[39:45], np.array([0, int(oracle.pack(900, 900))], dtype=np.int64)])
        want = np.concatenate([uc[:40], uc[39:45], [int(uc[uk == 0][0]) if (uk == 0).any() else 0, 0]])
        got = oracle.count_keys(xy, 100.0, q, lib=lib)
        if not np.array_equal(got, want.astype(np.uint64)):
            return False
    return True


def _window_significant(keys, counts, tau):
    ix, iy = oracle.unpack(keys)
    x0, y0 = int(ix.min()) - 1, int(iy.min()) - 1
    grid = np.zeros((int(ix.max()) - x0 + 2, int(iy.max()) - y0 + 2), dtype=np.int64)
    grid[ix - x0, iy - y0] = counts
    ok = (grid[:-1, :-1] + grid[1:, :-1] + grid[:-1, 1:] + grid[1:, 1:]) >= tau
    gx, gy = ix - x0, iy - y0
    return ok[gx - 1, gy - 1] | ok[gx - 1, gy] | ok[gx, gy - 1] | ok[gx, gy] | (counts >= tau)


def test_real_oracle_passes_compact_pins():
    assert _pins_pass(None)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mutated = tmp_path / f"oracle_{name}.cpp"
    mutated.write_text(src.replace(old, new))
    lib = oracle.load_library(oracle.compile_source(str(mutated), str(tmp_path / f"lib_{name}.so")))
    assert not _pins_pass(lib), f"mutant {name} slipped through the pins"
