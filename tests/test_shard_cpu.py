"""Sharded RASTER (P-RASTER's partitioning across GPUs, Sect. 3.5, Alg. 2-3)
on world-size 2 and 4 gloo ranks on the CPU.  The exchange steps are the
product's (slices from the global x range, all-to-all of (key, count) to the
owners, edge-column exchange and border union, mu after the join); the
per-rank device work is stubbed with the oracle: a rank's tile counts come
from the oracle's projection, and an owner's slice components from the
oracle run on points placed at its tile centres with mu = 1.  Whatever the
partition of the points, the rows gathered from all ranks must equal the
single-process oracle bit for bit (Theorem 3: slicing does not change the
clusters)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _points(case: int) -> np.ndarray:
    sys.path.insert(0, ROOT)
    import gen
    rng = np.random.default_rng(case)
    if case == 0:  # long shapes across every slice border, a snake, scattered blobs
        tiles = [(x, 0) for x in range(-50, 350)]
        for k in range(12):
            tiles += [(30 * k + d, 10 + (k % 2) * 6) for d in range(31)] + [(30 * k + 30, 10 + j) for j in range(7)]
        for _ in range(300):
            x, y = rng.integers(-40, 360), rng.integers(-100, 100)
            tiles += [(x + dx, y + dy) for dx in range(rng.integers(1, 3)) for dy in range(rng.integers(1, 3))]
        t = np.array(sorted(set(tiles)), dtype=np.float64)
        xy = (np.repeat(t, 6, axis=0) + rng.uniform(0.05, 0.95, (len(t) * 6, 2))) / 100.0
        return np.concatenate([xy, rng.uniform(-0.5, 3.5, (20000, 2))])
    w = gen.Workload(n=300_000, clusters=600, cluster_points=270_000, canvas=40.0, precision=2, tau=5, mu=4,
                     seed=90 + case)
    return gen.points(w)


def _rank(rank, world, port, case, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import oracle
    from paper_1907_03620_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    xy = _points(case)
    part = np.random.default_rng(1000 + case).integers(0, world, len(xy))  # arbitrary partition
    mine = xy[part == rank]
    # stub of the device contraction: this rank's tile counts
    keys, ok = oracle.project(mine, oracle.scale_of(2))
    k, c = np.unique(keys[ok], return_counts=True)
    slices, okey, ocnt = shard.route_to_owners(k.astype(np.int64), c.astype(np.int64))
    # stub of the owner's device agglomeration: components of the slice (mu = 1)
    uk, inv = np.unique(okey, return_inverse=True)
    uc = np.bincount(inv, weights=ocnt).astype(np.int64)
    assert all(slices.owner(uk) == rank)
    centres = (np.stack([shard.tile_x(uk), shard.tile_y(uk)], 1).astype(np.float64) + 0.5) / 100.0
    res, _ = oracle.raster(np.repeat(centres, uc, axis=0), 2, 5, 1)
    rows = shard.finish_slice(slices, rank, res.key, res.count.astype(np.int64), res.cid, 4)
    gathered = shard.allgather_obj(rows)
    if rank == 0:
        key = np.concatenate([g[0] for g in gathered])
        cnt = np.concatenate([g[1] for g in gathered])
        cid = np.concatenate([g[2] for g in gathered])
        out.put((key.tolist(), cnt.tolist(), cid.tolist(), sum(g[3] for g in gathered)))
    dist.destroy_process_group()


@pytest.mark.parametrize("world,case", [(2, 0), (4, 0), (2, 1), (4, 2)])
def test_sharded_rows_equal_single_process_oracle(world, case):
    sys.path.insert(0, ROOT)
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    key, cnt, cid, n_clusters = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref, _ = oracle.raster(_points(case), 2, 5, 4)
    key, cnt, cid = (np.array(v, dtype=np.int64) for v in (key, cnt, cid))
    o = oracle.tile_order(key)
    assert np.array_equal(key[o], ref.key)
    assert np.array_equal(cnt[o], ref.count.astype(np.int64))
    assert np.array_equal(cid[o], ref.cid)
    assert n_clusters == ref.n_clusters
