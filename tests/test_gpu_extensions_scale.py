"""The extensions at scale: the 50M-point workload with the 2 x 2 group rule
and with Chebyshev distance 2, bit for bit against the oracle; and the
100M-point three-coordinate bench workload, checked where the oracle can
follow it (sampled tile counts over all points, sampled clusters re-grown
from the exported counts, sampled labels)."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1907_03620_gb300 as R

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kw", [dict(groups=True), dict(delta=2)])
def test_workload_50m(kw):
    w = gen.C2_50M
    xy = gen.points(w)
    ref, ref_lab, _ = oracle.raster(xy, w.precision, w.tau, w.mu, with_labels=True, **kw)
    d = torch.from_numpy(xy).cuda()
    r = R.Raster(w.precision, w.tau, w.mu, **kw)
    r.contract(d)
    res = r.agglomerate().sorted()
    assert res.key.cpu().numpy().tolist() == ref.key.tolist()
    assert res.count.cpu().numpy().tolist() == ref.count.astype(np.int64).tolist()
    assert res.cid.cpu().numpy().tolist() == ref.cid.tolist()
    assert (res.n_clusters, res.n_significant, res.n_distinct) == (ref.n_clusters, ref.n_significant, ref.n_tiles)
    assert np.array_equal(r.point_labels(d).cpu().numpy(), ref_lab)
    r.close()


def test_three_coordinates_100m_sampled():
    c3 = gen.CUBES_100M
    xyz = gen.cubes3(**c3)
    p, tau, mu = 1.5, 5, 4
    d = torch.from_numpy(xyz).cuda()
    r = R.Raster(p, tau, mu, dims=3)
    r.contract(d)
    res = r.agglomerate()
    tk, tc = (t.cpu().numpy() for t in r.export_tiles())
    lab = r.point_labels(d)
    assert len(tk) == res.n_distinct and int(tc.sum()) == xyz.shape[0]
    assert res.n_significant == int((tc >= tau).sum())
    order = np.argsort(tk)
    sk, sc = tk[order], tc[order]
    rng = np.random.default_rng(23)
    scale = oracle.scale_of(p)
    # sampled counts, recomputed by the oracle over all points
    sig = np.flatnonzero(tc >= tau)
    sample = np.concatenate([tk[rng.choice(len(tk), 500, replace=False)], tk[sig[rng.choice(len(sig), 500, replace=False)]]])
    want = oracle.count_keys(xyz, scale, sample)
    i = np.searchsorted(sk, sample)
    assert np.array_equal(sc[i].astype(np.uint64), want)
    # sampled clusters re-grown over the exported counts (26 neighbours)
    kk, kc = res.key.cpu().numpy(), res.cid.cpu().numpy()

    def count_of(keys):
        j = np.minimum(np.searchsorted(sk, keys), len(sk) - 1)
        return np.where(sk[j] == keys, sc[j], 0)

    offs = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1) if a or b or c])
    for cid in rng.choice(np.unique(kc), 40, replace=False):
        members = set(kk[kc == cid].tolist())
        seen, stack = {int(cid)}, [int(cid)]
        while stack:
            u = stack.pop()
            x, y, z = (int(v[0]) for v in oracle.unpack3(np.array([u])))
            nb = oracle.pack3(x + offs[:, 0], y + offs[:, 1], z + offs[:, 2])
            for k, c in zip(nb.tolist(), count_of(nb).tolist()):
                if c >= tau and k not in seen:
                    seen.add(k)
                    stack.append(k)
        assert seen == members and len(members) >= mu and min(members) == cid
    # sampled labels: the point's tile (projected by the oracle) decides its label
    idx = rng.choice(xyz.shape[0], 20000, replace=False)
    pk, ok = oracle.project(xyz[idx], scale)
    assert ok.all()
    cid_of = dict(zip(kk.tolist(), kc.tolist()))
    assert lab[torch.from_numpy(idx).cuda()].cpu().numpy().tolist() == [cid_of.get(int(k), R.NOISE) for k in pk]
    r.close()
