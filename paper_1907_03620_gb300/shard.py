"""RASTER sharded over several GPUs, one process per GPU (P-RASTER's
partitioning, Sect. 3.5; Alg. 2 and Alg. 3; App. C, Theorem 3).

Each rank holds an arbitrary share of the points (the input may be cut
anywhere: the counts depend only on the multiset of points, Sect. 3.6).

    s = ShardedRaster(precision, tau, mu)   # inside an initialised process group
    s.contract(xy)                          # this rank's points, any number of calls
    rows = s.agglomerate()                  # this rank's vertical slice, global ids

1. contraction: every rank counts its own points per tile on its GPU;
2. owners: the tile space is cut into one vertical slice per rank, evenly
   spaced between the smallest and largest x index of all ranks' tiles;
3. exchange: one all-to-all of (key, count) sends every tile to its owner,
   which adds the counts into its own table (raster_contract_tiles);
4. slices: each owner applies tau and finds the components of its slice on
   its GPU (mu = 1 there, so no component is dropped before the join);
5. borders (Alg. 3): each owner sends the tiles of its two edge columns to
   its neighbours; components joined by a pair of adjacent tiles across a
   border are merged by a union-find over component ids, and the merged size
   decides mu.  The cluster id of a merged cluster is the (ix, iy)-smallest of
   its components' ids, i.e. its smallest tile, as for one GPU.

The per-tile work runs in the CUDA library; the host moves tile arrays
between ranks and joins the components that touch a border.  Collectives go
through torch.distributed with point-to-point messages (gloo has no
all-to-all), so the same code runs on NCCL.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

from . import Raster, Result


def _dev_of(group=None) -> torch.device:
    if dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def alltoallv(send: list[np.ndarray], group=None) -> list[np.ndarray]:
    """send[r] goes to rank r; returns the arrays received from every rank
    (int64 only).  Sizes are exchanged first, then one message per pair."""
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    dev = _dev_of(group)
    sizes = torch.tensor([len(a) for a in send], dtype=torch.int64, device=dev)
    table = [torch.empty_like(sizes) for _ in range(world)]
    dist.all_gather(table, sizes, group=group)
    recv_n = [int(table[r][rank]) for r in range(world)]
    out = [torch.empty(recv_n[r], dtype=torch.int64, device=dev) for r in range(world)]
    ops = []
    for r in range(world):
        if r == rank:
            out[r] = torch.from_numpy(np.ascontiguousarray(send[r], dtype=np.int64)).to(dev)
            continue
        if len(send[r]):
            ops.append(dist.P2POp(dist.isend, torch.from_numpy(np.ascontiguousarray(send[r], dtype=np.int64)).to(dev),
                                  r, group))
        if recv_n[r]:
            ops.append(dist.P2POp(dist.irecv, out[r], r, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    return [o.cpu().numpy() for o in out]


def allgather_obj(obj, group=None) -> list:
    out = [None] * dist.get_world_size(group)
    dist.all_gather_object(out, obj, group=group)
    return out


def tile_x(key: np.ndarray) -> np.ndarray:
    return (np.asarray(key, dtype=np.int64) >> 32).astype(np.int64)


def tile_y(key: np.ndarray) -> np.ndarray:
    return (np.asarray(key, dtype=np.int64) & 0xFFFFFFFF).astype(np.uint32).astype(np.int32).astype(np.int64)


def pack(ix, iy) -> np.ndarray:
    return ((np.asarray(ix, dtype=np.int64) << 32) | (np.asarray(iy, dtype=np.int64) & 0xFFFFFFFF)).astype(np.int64)


def lex_order(key: np.ndarray) -> np.ndarray:
    """(ix, iy) lexicographic order as one signed int64: ix stays signed in the
    high half, and iy's sign bit is flipped so that the low half sorts as
    unsigned."""
    return np.asarray(key, dtype=np.int64) ^ np.int64(0x80000000)


class Slices:
    """One vertical slice of tile x indices per rank, evenly spaced (Sect. 3.5)."""

    def __init__(self, xmin: int, xmax: int, world: int):
        self.xmin, self.xmax, self.world = int(xmin), int(xmax), int(world)
        self.width = max(1, (self.xmax - self.xmin) // world + 1)

    def owner(self, key: np.ndarray) -> np.ndarray:
        return np.minimum(self.world - 1, (tile_x(key) - self.xmin) // self.width).astype(np.int64)

    def lo(self, r: int) -> int:
        return self.xmin + r * self.width

    def hi(self, r: int) -> int:
        return self.xmax if r == self.world - 1 else self.xmin + (r + 1) * self.width - 1


class _UnionFind:
    def __init__(self):
        self.parent: dict[int, int] = {}

    def find(self, a: int) -> int:
        p = self.parent.setdefault(a, a)
        while p != self.parent[p]:
            self.parent[p] = self.parent[self.parent[p]]
            p = self.parent[p]
        self.parent[a] = p
        return p

    def union(self, a: int, b: int):
        ra, rb = self.find(a), self.find(b)
        if ra == rb:
            return
        # the root is the (ix, iy)-smallest id
        if (int(lex_order(np.int64(rb))) < int(lex_order(np.int64(ra)))):
            ra, rb = rb, ra
        self.parent[rb] = ra


def join_borders(slices: Slices, rank: int, key: np.ndarray, cid: np.ndarray, group=None):
    """Alg. 3 for one rank's slice: exchange the edge columns with the
    neighbouring slices, pair components across each border, and merge them
    everywhere.  key/cid: the slice's significant tiles and their local
    component ids (the smallest tile of each component).  Returns (cid, size)
    per tile after the join."""
    world = slices.world
    x = tile_x(key)
    left = key[x == slices.lo(rank)] if rank > 0 else key[:0]
    right = key[x == slices.hi(rank)] if rank < world - 1 else key[:0]
    cid_of = dict(zip(key.tolist(), cid.tolist()))
    send = [np.empty(0, np.int64) for _ in range(world)]
    if rank > 0:
        send[rank - 1] = np.stack([left, np.array([cid_of[k] for k in left.tolist()], np.int64)], 1).ravel()
    if rank < world - 1:
        send[rank + 1] = np.stack([right, np.array([cid_of[k] for k in right.tolist()], np.int64)], 1).ravel()
    got = alltoallv(send, group)
    pairs = []
    for r, arr in enumerate(got):
        if r == rank or not len(arr):
            continue
        nk, nc = arr.reshape(-1, 2).T
        mine = right if r == rank + 1 else left
        dx = 1 if r == rank + 1 else -1
        pos = set(mine.tolist())
        for k, c in zip(nk.tolist(), nc.tolist()):  # a neighbour's edge tile and its component
            kx, ky = int(tile_x(np.int64(k))), int(tile_y(np.int64(k)))
            for dy in (-1, 0, 1):
                if not -(2**31 - 1) <= ky + dy <= 2**31 - 2:
                    continue
                m = int(pack(kx - dx, ky + dy))
                if m in pos:
                    pairs.append((cid_of[m], c))
    # component sizes of every component that touches a border
    uniq, sizes = np.unique(cid, return_counts=True)
    size_of = dict(zip(uniq.tolist(), sizes.tolist()))
    edge_ids = set(cid_of[k] for k in np.concatenate([left, right]).tolist())
    everything = allgather_obj((pairs, {c: size_of[c] for c in edge_ids}), group)
    uf = _UnionFind()
    total: dict[int, int] = {}
    for prs, sz in everything:
        for c, n in sz.items():
            uf.find(c)
            total[c] = total.get(c, 0) + n
        for a, b in prs:
            uf.union(a, b)
    merged: dict[int, int] = {}
    for c, n in total.items():
        root = uf.find(c)
        merged[root] = merged.get(root, 0) + n
    out_cid = np.array([uf.find(c) if c in total else c for c in cid.tolist()], dtype=np.int64)
    out_size = np.array([merged[uf.find(c)] if c in total else size_of[c] for c in cid.tolist()], dtype=np.int64)
    return out_cid, out_size


def route_to_owners(key: np.ndarray, cnt: np.ndarray, group=None):
    """Steps 2-3: the slices from all ranks' x range, then every (key, count)
    to the rank that owns its slice.  Returns (slices, keys, counts) received
    by this rank; a key may arrive from several ranks."""
    world = dist.get_world_size(group)
    lo_hi = allgather_obj((int(tile_x(key).min()), int(tile_x(key).max())) if len(key) else None, group)
    rng = [v for v in lo_hi if v is not None]
    slices = Slices(min(v[0] for v in rng), max(v[1] for v in rng), world) if rng else Slices(0, 0, world)
    own = slices.owner(key) if len(key) else np.empty(0, np.int64)
    send = [np.stack([key[own == r], cnt[own == r]], 1).ravel() for r in range(world)]
    got = np.concatenate(alltoallv(send, group)).reshape(-1, 2)
    return slices, np.ascontiguousarray(got[:, 0]), np.ascontiguousarray(got[:, 1])


def finish_slice(slices: Slices, rank: int, key, count, cid, mu: int, group=None):
    """Step 5: border joins, then the mu test on the joined sizes.  Returns
    (key, count, cluster id, clusters whose id tile lies in this slice)."""
    gcid, size = join_borders(slices, rank, key, cid, group)
    keep = size >= mu
    key, count, gcid = key[keep], count[keep], gcid[keep]
    return key, count, gcid, int(np.count_nonzero(key == gcid))


class ShardedRaster:
    """RASTER over all ranks of a process group, one GPU per rank."""

    def __init__(self, precision: float, tau: int, mu: int, group=None):
        self.precision, self.tau, self.mu, self.group = precision, int(tau), int(mu), group
        self.local = Raster(precision, 1, 1)

    def contract(self, xy: torch.Tensor):
        self.local.contract(xy)

    def agglomerate(self) -> Result:
        group = self.group
        rank = dist.get_rank(group)
        dev = torch.device("cuda", torch.cuda.current_device())
        key, cnt = (t.cpu().numpy() for t in self.local.export_tiles())
        cnt = cnt.astype(np.int64)
        slices, okey, ocnt = route_to_owners(key, cnt, group)
        owner = Raster(self.precision, self.tau, 1)
        if len(okey):
            owner.contract_tiles(torch.from_numpy(okey).to(dev), torch.from_numpy(ocnt.astype(np.int32)).to(dev))
        res = owner.agglomerate()  # 4. components of the slice, nothing dropped yet
        k, c, cid = res.key.cpu().numpy(), res.count.cpu().numpy(), res.cid.cpu().numpy()
        n_distinct, n_sig = res.n_distinct, res.n_significant
        owner.close()
        k, c, gcid, n_clusters = finish_slice(slices, rank, k, c, cid, self.mu, group)
        return Result(torch.from_numpy(k).to(dev), torch.from_numpy(c).to(dev), torch.from_numpy(gcid).to(dev),
                      n_clusters, n_distinct, n_sig, int(cnt.sum()), 0)

    def close(self):
        self.local.close()
