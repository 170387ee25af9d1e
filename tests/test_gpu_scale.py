"""Full-size parity cases: the 10,000-particle uneven-mesh batch (icospheres of
80/320/1280 triangles and convex hulls, radii 0.5-4, clustered), the
100,000-particle local-time-stepping layout (dense FCC blobs and free
particles, per-particle steps log-uniform in [1e-5, 1e-2]) and the
1,000,000-particle settling column over a static floor of 199,712 triangles.

The GPU runs the whole step on all pairs; the oracle checks the candidate
set (in full, or the partners of sampled particles where O(N^2) is too slow)
and a seeded sample of pairs one by one.
"""
import numpy as np
import pytest

import oracle
from floor_oracle import floor_pair_oracle
from paper_2309_15417_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(dem, w, prec=0, max_pairs=1 << 20):
    c = dem.Context(K=w.K, tol=w.tol, precision=prec, max_particles=w.n, max_pairs=max_pairs,
                    max_contacts=1 << 22, max_triangles=w.n_tris)
    sc = dem.Scene.from_workload(w)
    c.step_fused(sc)
    c.check()
    m = int(c.n_pairs.item())
    nc = int(c.n_contacts.item())
    out = dict(pairs=c.pairs[:m].cpu().numpy(), dmin=c.dmin[:m].cpu().numpy(), pa=c.pa[:m].cpu().numpy(),
               pb=c.pb[:m].cpu().numpy(), tri_ab=c.tri_ab[:m].cpu().numpy(), flag=c.flag[:m].cpu().numpy(),
               t_coll=c.t_coll[:m].cpu().numpy(), status=c.status[:m].cpu().numpy(),
               ct_ab=c.ct_ab[:m].cpu().numpy(), contacts=c.contacts[:nc].cpu().numpy(),
               ids=c.cluster_id[:w.n].cpu().numpy(), n_clusters=int(c.n_clusters.item()))
    c.close()
    return out


def _check_sampled_pairs(w, g, idx):
    sel = g["pairs"][idx]
    on = oracle.narrow_phase(w, sel)
    oc = oracle.collision_times(w, sel)
    for key in ("flag", "tri_ab", "dmin", "pa", "pb"):
        assert np.array_equal(g[key][idx], on[key]), key
    assert np.array_equal(g["status"][idx], oc["status"])
    assert np.array_equal(g["t_coll"][idx], oc["t_coll"])
    assert np.array_equal(g["ct_ab"][idx], oc["tri_ab"])
    # contact keys of the sampled pairs
    gk = g["contacts"]
    rows = np.isin(gk[:, 0], idx)
    remap = {int(k): q for q, k in enumerate(idx)}
    sub = gk[rows].copy()
    sub[:, 0] = [remap[int(k)] for k in sub[:, 0]]
    assert np.array_equal(sub, on["contacts"])
    return oc


def test_uneven_10k_full_size(dem):
    w = W.uneven_meshes(0)
    g = _run(dem, w)
    o = oracle.broad_phase(w)
    assert len(o) > 100
    assert np.array_equal(g["pairs"], o)
    ids, nc = oracle.clusters(w.n, o, w.is_static)
    assert np.array_equal(g["ids"], ids) and g["n_clusters"] == nc
    # sample: the costliest pairs (largest T_i * T_j) plus random ones
    cnt = w.tri_counts()
    cost = cnt[o[:, 0]] * cnt[o[:, 1]]
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([np.argsort(-cost)[:4], rng.choice(len(o), 16, replace=False)]))
    _check_sampled_pairs(w, g, idx)


def test_lts_100k_full_size(dem):
    w = W.lts_mixed_steps(0)
    g = _run(dem, w)
    pairs = g["pairs"]
    assert len(pairs) > 1000
    assert np.all(pairs[:, 0] < pairs[:, 1])
    assert np.all(np.diff(pairs[:, 0].astype(np.int64) * w.n + pairs[:, 1]) > 0)
    # candidate partners of sampled particles (blob and free)
    rng = np.random.default_rng(1)
    blob = int(w.meta["n_blob"])
    parts = np.concatenate([rng.choice(blob, 150, replace=False), blob + rng.choice(w.n - blob, 150, replace=False)])
    for p in parts:
        op = oracle.broad_partners(w, int(p))
        gp = pairs[(pairs[:, 0] == p) | (pairs[:, 1] == p)]
        assert np.array_equal(op, gp), p
    # clusters of the candidate graph
    ids, nc = oracle.clusters(w.n, pairs, w.is_static)
    assert np.array_equal(g["ids"], ids) and g["n_clusters"] == nc
    # sampled pairs, including every pair whose search bisected (status 2)
    idx = np.unique(np.concatenate([np.where(g["status"] == 2)[0][:8], rng.choice(len(pairs), 16, replace=False)]))
    oc = _check_sampled_pairs(w, g, idx)
    assert set(np.unique(oc["status"])) >= {0, 1}


def test_settling_column_full_size(dem):
    """10^6 icospheres (80 / 320 triangles) on a jittered lattice over a static
    316 x 316-quad floor: the whole step on the GPU; the floor's partners and
    sampled particles' partners against brute force, clusters in full, and
    sampled pairs (with and without the floor) one by one."""
    w = W.settling_column(0)
    floor = w.n - 1
    g = _run(dem, w)
    pairs = g["pairs"]
    key = pairs[:, 0].astype(np.int64) * w.n + pairs[:, 1]
    assert np.all(np.diff(key) > 0)
    assert not np.any(pairs[:, 0] == floor)
    # the floor pairs with the whole bottom layer
    op = oracle.broad_partners(w, floor)
    assert np.array_equal(pairs[pairs[:, 1] == floor], op)
    assert len(op) == 100 * 100
    rng = np.random.default_rng(2)
    bottom = np.where(w.state[W.F_Z, :floor] < 1.5)[0]
    for p in np.concatenate([rng.choice(bottom, 40, replace=False), rng.choice(floor, 60, replace=False)]):
        gp = pairs[(pairs[:, 0] == p) | (pairs[:, 1] == p)]
        assert np.array_equal(oracle.broad_partners(w, int(p)), gp), p
    ids, nc = oracle.clusters(w.n, pairs, w.is_static)
    assert np.array_equal(g["ids"], ids) and g["n_clusters"] == nc
    # a few hundred pairs between particles, one by one against the oracle
    others = np.where(pairs[:, 1] != floor)[0]
    _check_sampled_pairs(w, g, np.sort(rng.choice(others, 240, replace=False)))
    # floor pairs: every one whose search bisected (status 2), and sampled
    # ones in contact at the start and apart, each on its reduced floor
    fl = np.where(pairs[:, 1] == floor)[0]
    touching = fl[g["flag"][fl] == 1]
    apart = fl[g["flag"][fl] == 0]
    bis = fl[g["status"][fl] == 2]
    assert len(touching) > 100 and len(apart) > 100
    gk = g["contacts"]
    for k in np.unique(np.concatenate([bis, rng.choice(touching, 40, replace=False),
                                       rng.choice(apart, 40, replace=False)])):
        on, oc, kept = floor_pair_oracle(w, int(pairs[k, 0]), floor)
        for key in ("flag", "tri_ab", "dmin", "pa", "pb"):
            assert np.array_equal(g[key][k:k + 1], on[key]), (k, key)
        assert g["status"][k] == oc["status"][0] and g["t_coll"][k] == oc["t_coll"][0], k
        assert np.array_equal(g["ct_ab"][k], oc["tri_ab"][0]), k
        sub = gk[gk[:, 0] == k][:, 1:]
        assert np.array_equal(sub, on["contacts"][:, 1:]), k
        assert 0 < kept < 2000


def test_every_launch_configuration_gives_identical_results(dem):
    """The autotuner's space (CTAs per SM, warp flush size, costliest-first or
    index hand-out) changes only the schedule: on the uneven-mesh batch every
    configuration gives the same outputs bit for bit, equal to the oracle on
    the costliest pairs; dem_autotune keeps one of them."""
    w = W.uneven_meshes(2, n=2000, box=80.0)
    sc = dem.Scene.from_workload(w)
    c = dem.Context(K=w.K, tol=w.tol, max_particles=w.n, max_pairs=1 << 16, max_contacts=1 << 20,
                    max_triangles=w.n_tris)
    c.build_candidates(sc)
    c.check()
    m = int(c.n_pairs.item())
    assert m > 20

    def outputs():
        nc = int(c.n_contacts.item())
        return [t.cpu().numpy().copy() for t in (c.dmin[:m], c.tri_ab[:m], c.flag[:m], c.t_coll[:m], c.status[:m],
                                                c.ct_ab[:m], c.contacts[:nc])]

    ref = None
    for order in (0, 1):
        for wf in (32, 64):
            for cps in (1, 4):
                c.set_tuning(dem.DEM_TUNE_DETECT, ctas_per_sm=cps, wflush=wf, cost_order=order)
                c.detect(sc)
                c.check()
                got = outputs()
                if ref is None:
                    ref = got
                assert all(np.array_equal(a, b) for a, b in zip(ref, got)), (order, wf, cps)
    best = c.autotune(sc, dem.DEM_TUNE_DETECT)
    assert best["wflush"] in (32, 64) and best["cost_order"] in (0, 1) and 1 <= best["ctas_per_sm"] <= 4
    assert c.get_tuning(dem.DEM_TUNE_DETECT)["ctas_per_sm"] == best["ctas_per_sm"]
    got = outputs()
    assert all(np.array_equal(a, b) for a, b in zip(ref, got))
    c.check()
    pairs = c.pairs[:m].cpu().numpy()
    cnt = w.tri_counts()
    idx = np.sort(np.argsort(-(cnt[pairs[:, 0]] * cnt[pairs[:, 1]]))[:6])
    on, oc = oracle.narrow_phase(w, pairs[idx]), oracle.collision_times(w, pairs[idx])
    assert np.array_equal(ref[0][idx], on["dmin"]) and np.array_equal(ref[4][idx], oc["status"])
    assert np.array_equal(ref[3][idx], oc["t_coll"])
    c.close()
