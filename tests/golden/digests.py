"""Oracle digests of the full-size workloads, for bit-exact parity tests.

The CPU oracle (Alg. 1 written out) is too slow to run inside a GPU test on
the three largest workloads, so this script runs it once and stores SHA-256
digests of its complete outputs under ``tests/golden/``:

  * the 500M-point workload (Sect. 4.2-style shuffled squares plus 5% noise,
    p = 2, tau = 5, mu = 4): every tile's (key, count), every kept tile's
    (key, count, cluster id), and all 500M point labels (RASTER*, Sect. 4.1),
    each as 64 block digests so that a mismatch names the block;
  * the 4,096-instance batched workload: (D, S, clusters, rows) and the kept
    rows of every instance, in 64 groups of 64 instances;
  * the served mix (36 requests spanning sizes 1e4..2e7, 1..8 chunks and all
    18 combinations of p, tau, mu): one digest per request.

Every stored value comes from ``oracle`` alone, on inputs from ``gen`` alone.
The canonical byte form is defined here and used by the tests to hash the
GPU's outputs the same way: rows sorted by key as signed 64-bit integers,
then the little-endian int64 keys, uint64 counts and int64 cluster ids.

    python tests/golden/digests.py [500m] [batch] [served]
"""
from __future__ import annotations

import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

BLOCKS = 64
GROUP = 64
PATHS = {name: os.path.join(HERE, f"digests_{name}.json") for name in ("500m", "batch4096", "served_mix")}


def _h(*arrays) -> str:
    m = hashlib.sha256()
    for a in arrays:
        m.update(np.ascontiguousarray(a).tobytes())
    return m.hexdigest()


def canonical_rows(key, count=None, cid=None):
    """Rows sorted by signed key; int64 keys, uint64 counts, int64 ids (little endian)."""
    key = np.asarray(key).astype("<i8")
    o = np.argsort(key, kind="stable")
    out = [key[o]]
    if count is not None:
        out.append(np.asarray(count).astype("<u8")[o])
    if cid is not None:
        out.append(np.asarray(cid).astype("<i8")[o])
    return out


def block_digests(arrays, blocks: int = BLOCKS) -> list[str]:
    """Digest of each of `blocks` contiguous, nearly equal index ranges of the
    (already canonical) arrays, which all have the same length."""
    n = len(arrays[0])
    out = []
    for b in range(blocks):
        lo, hi = n * b // blocks, n * (b + 1) // blocks
        out.append(_h(*[a[lo:hi] for a in arrays]))
    return out


def rows_digest(key, count, cid) -> str:
    return _h(*canonical_rows(key, count, cid))


def first_mismatch(got: list[str], want: list[str]) -> int:
    """Index of the first differing block digest, or -1."""
    for i, (a, b) in enumerate(zip(got, want)):
        if a != b:
            return i
    return -1 if len(got) == len(want) else min(len(got), len(want))


# ---------------------------------------------------------------------------
# The served mix: every (p, tau, mu) combination twice, sizes log-uniform in
# [1e4, 2e7) with both ends present, chunk counts 1..8.
def served_mix(seed: int = 6):
    import gen
    combos = [(p, t, m) for p in gen.PRECISIONS for t in gen.TAUS for m in gen.MUS]
    out = []
    for j in range(2 * len(combos)):
        p, t, m = combos[j % len(combos)]
        if j == 0:
            size = 19_999_999
        elif j == 1:
            size = 10_000
        else:
            u = gen.u01(seed, 11, j)
            size = int(np.floor(np.exp(np.log(1e4) + u * (np.log(2e7) - np.log(1e4)))))
        base = gen._instance(seed, j, size, 0.10)
        w = gen.Workload(n=base.n, clusters=base.clusters, cluster_points=base.cluster_points, canvas=base.canvas,
                         precision=p, tau=t, mu=m, seed=base.seed)
        out.append((w, 1 + j % 8))
    return out


# ---------------------------------------------------------------------------
def _oracle_rows(xy, w, chunks: int = 1):
    import oracle
    r, o = oracle.raster(xy, w.precision, w.tau, w.mu, chunks=chunks)
    return r, o


def make_500m() -> dict:
    import gen
    import oracle
    w = gen.C3_500M
    t0 = time.time()
    xy = gen.points(w)
    o = oracle.Oracle(w.precision, w.tau, w.mu)
    st = o.add(xy)
    r = o.finish()
    tk, tc = o.tiles()
    tiles = block_digests(canonical_rows(tk, tc))
    del tk, tc
    kept = block_digests(canonical_rows(r.key, r.count, r.cid))
    lst, lab = o.labels(xy)
    labels = block_digests([lab.astype("<i8")])
    return {"workload": w.asdict(), "status": int(st), "labels_status": int(lst), "n_tiles": int(r.n_tiles),
            "n_significant": int(r.n_significant), "n_clusters": int(r.n_clusters), "n_kept": int(len(r.key)),
            "n_noise_points": int((lab == oracle.NOISE).sum()), "tiles_blocks": tiles, "kept_blocks": kept,
            "labels_blocks": labels, "seconds": round(time.time() - t0, 1)}


def _one_instance(w) -> tuple:
    import gen
    xy = gen.points(w, nthreads=1)
    r, _ = _oracle_rows(xy, w)
    return (int(r.n_tiles), int(r.n_significant), int(r.n_clusters), int(len(r.key)),
            rows_digest(r.key, r.count, r.cid))


def instance_group_digest(stats: list[tuple]) -> str:
    m = hashlib.sha256()
    for s in stats:
        m.update(json.dumps(list(s)).encode())
    return m.hexdigest()


def make_batch() -> dict:
    import gen
    ws = gen.batch_instances()
    t0 = time.time()
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        stats = pool.map(_one_instance, ws, chunksize=4)
    groups = [instance_group_digest(stats[g:g + GROUP]) for g in range(0, len(ws), GROUP)]
    return {"count": len(ws), "group": GROUP, "total_points": int(sum(w.n for w in ws)),
            "n_clusters": int(sum(s[2] for s in stats)), "groups": groups, "seconds": round(time.time() - t0, 1)}


def _one_request(arg) -> dict:
    import gen
    w, chunks = arg
    xy = gen.points(w, nthreads=1)
    r, _ = _oracle_rows(xy, w, chunks=chunks)
    return {"n": w.n, "chunks": chunks, "precision": w.precision, "tau": w.tau, "mu": w.mu,
            "n_tiles": int(r.n_tiles), "n_significant": int(r.n_significant), "n_clusters": int(r.n_clusters),
            "n_kept": int(len(r.key)), "rows": rows_digest(r.key, r.count, r.cid)}


def make_served() -> dict:
    mix = served_mix()
    t0 = time.time()
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        reqs = pool.map(_one_request, mix, chunksize=1)
    return {"seed": 6, "requests": reqs, "seconds": round(time.time() - t0, 1)}


def load(name: str) -> dict:
    with open(PATHS[name]) as f:
        return json.load(f)


def main(argv):
    which = argv or ["served", "batch", "500m"]
    makers = {"500m": ("500m", make_500m), "batch": ("batch4096", make_batch), "served": ("served_mix", make_served)}
    for arg in which:
        name, fn = makers[arg]
        d = fn()
        with open(PATHS[name], "w") as f:
            json.dump(d, f, indent=1)
            f.write("\n")
        print(name, "written in", d.get("seconds"), "s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
