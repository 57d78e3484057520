"""The 500M-point workload in the bench's launch configuration (one handle,
the whole array in one contract call), bit for bit against the oracle: every
tile's (key, count), every kept tile's (key, count, cluster id) and all 500M
labels are hashed the same way as the oracle's stored outputs
(tests/golden/digests.py); a mismatch names the block of rows and recounts
its first tiles with the oracle.  Sampled tile counts are also recomputed one
by one over all points, sampled clusters are re-grown from the exported
counts, sampled labels are checked, and the totals must hold."""
import os
import sys

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1907_03620_gb300 as R

pytestmark = pytest.mark.gpu

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import digests  # noqa: E402


def _sorted_lookup(sorted_keys, values, q):
    i = np.searchsorted(sorted_keys, q)
    i = np.minimum(i, len(sorted_keys) - 1)
    found = sorted_keys[i] == q
    return found, np.where(found, values[i], 0)


def _check_digests(xy, w, res, tk, tc, lab):
    g = digests.load("500m")
    assert g["workload"] == w.asdict()
    assert (len(tk), res.n_significant, res.n_clusters, len(res.key)) == \
        (g["n_tiles"], g["n_significant"], g["n_clusters"], g["n_kept"])
    rows = digests.canonical_rows(tk, tc)
    b = digests.first_mismatch(digests.block_digests(rows), g["tiles_blocks"])
    if b >= 0:
        lo = len(rows[0]) * b // digests.BLOCKS
        keys = rows[0][lo:lo + 10_000]
        want = oracle.count_keys(xy, oracle.scale_of(w.precision), keys)
        bad = np.flatnonzero(want != rows[1][lo:lo + 10_000])
        detail = f"first differing row {lo + bad[0]}: key {keys[bad[0]]}" if len(bad) else "not in its first rows"
        pytest.fail(f"tile block {b} differs from the oracle's; {detail}")
    b = digests.first_mismatch(digests.block_digests(digests.canonical_rows(
        res.key.cpu().numpy(), res.count.cpu().numpy(), res.cid.cpu().numpy())), g["kept_blocks"])
    assert b < 0, f"kept-tile block {b} of {digests.BLOCKS} differs from the oracle's"
    lab_h = lab.cpu().numpy()
    assert int((lab_h == oracle.NOISE).sum()) == g["n_noise_points"]
    b = digests.first_mismatch(digests.block_digests([lab_h.astype("<i8")]), g["labels_blocks"])
    assert b < 0, f"labels of points [{w.n * b // 64}, {w.n * (b + 1) // 64}) differ from the oracle's"


def test_workload_500m_bit_exact():
    w = gen.C3_500M
    xy = gen.points(w)
    d = torch.from_numpy(xy).cuda()
    r = R.Raster(w.precision, w.tau, w.mu)
    r.contract(d)
    res = r.agglomerate()
    tk, tc = r.export_tiles()
    lab = r.point_labels(d)
    tk, tc = tk.cpu().numpy(), tc.cpu().numpy()
    assert len(tk) == res.n_distinct and int(tc.sum()) == w.n
    _check_digests(xy, w, res, tk, tc, lab)
    assert res.n_significant == int((tc >= w.tau).sum())
    order = np.argsort(tk)
    sk, sc = tk[order], tc[order]
    rng = np.random.default_rng(17)
    # 1. counts of sampled tiles (half of them significant) recomputed by the oracle over all points
    sig = np.flatnonzero(tc >= w.tau)
    sample = np.concatenate([tk[rng.choice(len(tk), 1000, replace=False)],
                             tk[sig[rng.choice(len(sig), 1000, replace=False)]]])
    want = oracle.count_keys(xy, oracle.scale_of(w.precision), sample)
    _, got = _sorted_lookup(sk, sc, sample)
    assert np.array_equal(got.astype(np.uint64), want)
    # 2. sampled clusters re-grown over the exported counts (8-neighbour flood fill)
    kk, kc = res.key.cpu().numpy(), res.cid.cpu().numpy()
    korder = np.argsort(kk)
    kks, kcs = kk[korder], kc[korder]
    for cid in rng.choice(np.unique(kc), 60, replace=False):
        members = set(kk[kc == cid].tolist())
        start = int(cid)
        seen, stack = {start}, [start]
        while stack:
            u = stack.pop()
            x, y = int(np.int64(u) >> 32), int(np.int32(np.uint32(u & 0xFFFFFFFF)))
            nb = np.array([int(oracle.pack(x + dx, y + dy)) for dx in (-1, 0, 1) for dy in (-1, 0, 1)
                           if dx or dy], dtype=np.int64)
            found, cnt = _sorted_lookup(sk, sc, nb)
            for k, f, c in zip(nb.tolist(), found, cnt):
                if f and c >= w.tau and k not in seen:
                    seen.add(k)
                    stack.append(k)
        assert seen == members
        assert len(members) >= w.mu
        mx = min(members, key=lambda k: (np.int64(k) >> 32, np.int32(np.uint32(k & 0xFFFFFFFF))))
        assert mx == cid
    # 3. sampled labels: the point's tile (projected by the oracle) decides its label
    idx = rng.choice(w.n, 20000, replace=False)
    pk, ok = oracle.project(xy[idx], oracle.scale_of(w.precision))
    assert ok.all()
    found, cid = _sorted_lookup(kks, kcs, pk)
    expect = np.where(found, cid, oracle.NOISE)
    assert np.array_equal(lab[torch.from_numpy(idx).cuda()].cpu().numpy(), expect)
    # 4. the same points streamed as 10 chunks of 50M into one table (Sect. 3.6) give the same table
    r.close()
    r2 = R.Raster(w.precision, w.tau, w.mu)
    for c in range(10):
        r2.contract(d[c * 50_000_000:(c + 1) * 50_000_000])
    res2 = r2.agglomerate()
    k2, c2 = r2.export_tiles()
    k2, c2 = k2.cpu().numpy(), c2.cpu().numpy()
    o2 = np.argsort(k2)
    assert np.array_equal(k2[o2], sk) and np.array_equal(c2[o2], sc)
    a, b = res.sorted(), res2.sorted()
    assert torch.equal(a.key, b.key) and torch.equal(a.count, b.count) and torch.equal(a.cid, b.cid)
    r2.close()
    # 5. the key path of the bench step: one contract call that stores every point's key, then the
    #    labels read from the keys -- the same table, kept rows and all 500M labels (checked above
    #    against the oracle's digests), and sampled keys equal to the oracle's projection
    r3 = R.Raster(w.precision, w.tau, w.mu)
    keys = r3.contract_keys(d)
    res3 = r3.agglomerate()
    k3, c3 = r3.export_tiles()
    k3, c3 = k3.cpu().numpy(), c3.cpu().numpy()
    o3 = np.argsort(k3)
    assert np.array_equal(k3[o3], sk) and np.array_equal(c3[o3], sc)
    e = res3.sorted()
    assert torch.equal(a.key, e.key) and torch.equal(a.count, e.count) and torch.equal(a.cid, e.cid)
    assert torch.equal(r3.key_labels(keys), lab)
    assert np.array_equal(keys[torch.from_numpy(idx).cuda()].cpu().numpy(), pk)
    # 6. the bench's steady step: reset, one round that also selects the significant tiles as it
    #    writes the table, agglomeration from that selection, labels from the keys
    for _ in range(2):
        r3.reset()
        r3.contract_keys(d, keys)
        f = r3.agglomerate().sorted()
        assert torch.equal(a.key, f.key) and torch.equal(a.count, f.count) and torch.equal(a.cid, f.cid)
        assert torch.equal(r3.key_labels(keys), lab)
    r3.close()
