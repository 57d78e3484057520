"""More than 2^30 points in one contract call run as several contraction
rounds: the table must be the same as for the same points given in chunks,
the counts must sum to n, and sampled tile counts (half of them significant
tiles) must equal the oracle's recount over all points."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1907_03620_gb300 as R

pytestmark = pytest.mark.gpu


def test_call_above_one_round():
    w = gen.Workload(n=(1 << 30) + 50_000_000, clusters=2_000_000, cluster_points=(1 << 30), canvas=4500.0,
                     precision=2, tau=5, mu=4, seed=41)
    host = torch.empty((w.n, 2), dtype=torch.float64)
    gen.points_into(host.numpy(), w)
    d = host.cuda()
    r = R.Raster(w.precision, w.tau, w.mu)
    r.contract(d)  # two rounds
    a = r.agglomerate().sorted()
    k1, c1 = (t.cpu().numpy() for t in r.export_tiles())
    r.close()
    r2 = R.Raster(w.precision, w.tau, w.mu)
    cuts = [0, 300_000_000, 700_000_000, w.n]
    for lo, hi in zip(cuts, cuts[1:]):
        r2.contract(d[lo:hi])
    b = r2.agglomerate().sorted()
    k2, c2 = (t.cpu().numpy() for t in r2.export_tiles())
    r2.close()
    o1, o2 = np.argsort(k1), np.argsort(k2)
    assert np.array_equal(k1[o1], k2[o2]) and np.array_equal(c1[o1], c2[o2])
    assert int(c1.sum()) == w.n
    rng = np.random.default_rng(43)
    sig = np.flatnonzero(c1 >= w.tau)
    sample = np.concatenate([k1[rng.choice(len(k1), 1000, replace=False)],
                             k1[sig[rng.choice(len(sig), 1000, replace=False)]]])
    want = oracle.count_keys(host.numpy(), oracle.scale_of(w.precision), sample)
    got = c1[o1][np.searchsorted(k1[o1], sample)]
    assert np.array_equal(got.astype(np.uint64), want)
    assert torch.equal(a.key, b.key) and torch.equal(a.count, b.count) and torch.equal(a.cid, b.cid)
    assert a.n_points == w.n and a.n_clusters == b.n_clusters
