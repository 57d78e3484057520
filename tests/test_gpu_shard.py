"""Sharded RASTER's device steps on the GPU.

raster_contract_tiles (adding counted tiles, the join of partial count maps,
Sect. 3.5) must give the same table and clusters as contracting the points,
with repeated keys and with keys outside the index range reported.  Then the
whole sharded run: two ranks (gloo processes that share this one GPU; their
kernels never wait on each other, only the host exchanges), each contracting
an arbitrary share of the points, routing tiles to slice owners, clustering
its slice on the device and joining borders; the gathered rows must equal
the oracle bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import gen
import oracle
import paper_1907_03620_gb300 as R

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
W = gen.Workload(n=1_000_000, clusters=2_000, cluster_points=900_000, canvas=60.0, precision=2, tau=5, mu=4, seed=55)


def test_contract_tiles_equals_contracting_the_points():
    xy = gen.points(W)
    keys, ok = oracle.project(xy, oracle.scale_of(2))
    k, c = np.unique(keys[ok], return_counts=True)
    # split every count in two entries, in shuffled order: keys repeat
    rng = np.random.default_rng(3)
    part = rng.integers(0, c + 1)
    kk = np.concatenate([k, k])
    cc = np.concatenate([part, c - part]).astype(np.int32)
    perm = rng.permutation(len(kk))
    kk, cc = kk[perm], cc[perm]
    h = R.Raster(2, 5, 4)
    h.contract_tiles(torch.from_numpy(kk).cuda(), torch.from_numpy(cc).cuda())
    got = h.agglomerate().sorted()
    tk, tc = (t.cpu().numpy() for t in h.export_tiles())
    ref, _ = oracle.raster(xy, 2, 5, 4)
    o = np.argsort(tk)
    assert np.array_equal(tk[o], k) and np.array_equal(tc[o], c)
    assert got.key.cpu().numpy().tolist() == ref.key.tolist()
    assert got.count.cpu().numpy().tolist() == ref.count.astype(np.int64).tolist()
    assert got.cid.cpu().numpy().tolist() == ref.cid.tolist()
    assert got.n_points == W.n
    # after more points arrive the usual way, the counts still add up
    h.contract(torch.from_numpy(xy[:1000]).cuda())
    assert int(h.export_tiles()[1].sum()) == W.n + 1000
    h.close()
    # keys outside the index range are skipped and reported
    bad = np.array([oracle.pack(5, 5), oracle.pack(-2**31, 5), oracle.pack(7, 7)], dtype=np.int64)
    h = R.Raster(2, 1, 1)
    h.contract_tiles(torch.from_numpy(bad).cuda(), torch.from_numpy(np.array([3, 4, 0], np.int32)).cuda())
    with pytest.raises(R.RasterError) as e:
        h.agglomerate()
    assert e.value.status == R._native.E_RANGE
    res = h.agglomerate(allow_range_error=True)
    assert res.key.cpu().tolist() == [int(oracle.pack(5, 5))] and res.count.cpu().tolist() == [3]
    h.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    from paper_1907_03620_gb300.shard import ShardedRaster, allgather_obj
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    xy = gen.points(W)
    part = np.random.default_rng(7).integers(0, world, len(xy))
    s = ShardedRaster(2, 5, 4)
    mine = torch.from_numpy(np.ascontiguousarray(xy[part == rank])).cuda()
    half = mine.shape[0] // 2
    s.contract(mine[:half])  # in two chunks
    s.contract(mine[half:])
    res = s.agglomerate()
    rows = (res.key.cpu().numpy(), res.count.cpu().numpy(), res.cid.cpu().numpy(), res.n_clusters)
    s.close()
    gathered = allgather_obj(rows)
    if rank == 0:
        out.put(tuple(np.concatenate([g[i] for g in gathered]).tolist() for i in range(3))
                + (sum(g[3] for g in gathered),))
    dist.destroy_process_group()


def test_two_ranks_equal_the_oracle():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    key, cnt, cid, n_clusters = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref, _ = oracle.raster(gen.points(W), 2, 5, 4)
    key, cnt, cid = (np.array(v, dtype=np.int64) for v in (key, cnt, cid))
    o = oracle.tile_order(key)
    assert np.array_equal(key[o], ref.key) and np.array_equal(cnt[o], ref.count.astype(np.int64))
    assert np.array_equal(cid[o], ref.cid) and n_clusters == ref.n_clusters


def test_contract_tiles_three_coordinates():
    """Counted 3-D tiles (21-bit fields) give the clusters of the points."""
    g = np.random.default_rng(8)
    xyz = np.concatenate([g.uniform(0, 0.3, (60000, 3)), g.uniform(-1, 1, (20000, 3))])
    keys, ok = oracle.project(xyz, oracle.scale_of(2))
    k, c = np.unique(keys[ok], return_counts=True)
    h = R.Raster(2, 3, 2, dims=3)
    h.contract_tiles(torch.from_numpy(k).cuda(), torch.from_numpy(c.astype(np.int32)).cuda())
    got = h.agglomerate().sorted()
    ref, _ = oracle.raster(xyz, 2, 3, 2)
    assert got.key.cpu().numpy().tolist() == ref.key.tolist()
    assert got.cid.cpu().numpy().tolist() == ref.cid.tolist()
    assert got.n_clusters == ref.n_clusters
    h.close()
