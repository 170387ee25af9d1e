"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Bar (per output):
  candidate pairs, contact flags, contact (pair, a, b) sets and order, closest
  triangle pair (a, b), collision statuses and times, cluster ids: bit-exact;
  closest-pair distance and points: bit-exact (they come from the binary64
  recomputation in both precision modes);
  contact-list geometry: bit-exact in FP64 mode, within 1e-5 * R in FP32 mode
  (R = particle radius; a contact far from the halo boundary keeps its FP32
  distance and points).
"""
import numpy as np
import pytest

import oracle
from paper_2309_15417_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PRECS = [0, 1]


def _torch():
    import torch
    return torch


def _ctx(dem, w, prec, max_pairs=None, max_contacts=1 << 20):
    return dem.Context(K=w.K, tol=w.tol, precision=prec, max_particles=max(w.n, 16),
                       max_pairs=max_pairs or max(4096, 4 * w.n), max_contacts=max_contacts)


def _pairs_tensor(pairs):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)).cuda()


def gpu_candidates(dem, w, prec=0):
    c = _ctx(dem, w, prec)
    sc = dem.Scene.from_workload(w)
    c.build_candidates(sc)
    c.check()
    m = int(c.n_pairs.item())
    return c.pairs[:m].cpu().numpy()


def gpu_narrow(dem, w, pairs, prec, t_eval=None):
    torch = _torch()
    c = _ctx(dem, w, prec, max_pairs=max(len(pairs), 1))
    sc = dem.Scene.from_workload(w)
    pt = _pairs_tensor(pairs)
    te = None if t_eval is None else torch.from_numpy(np.ascontiguousarray(t_eval, np.float64)).cuda()
    c.narrow_phase(sc, pairs=pt, n_pairs=None, t_eval=te)
    c.check()
    m = len(pairs)
    nc = int(c.n_contacts.item())
    return dict(dmin=c.dmin[:m].cpu().numpy(), pa=c.pa[:m].cpu().numpy(), pb=c.pb[:m].cpu().numpy(),
                tri_ab=c.tri_ab[:m].cpu().numpy(), flag=c.flag[:m].cpu().numpy(),
                dmin32=c.dmin32[:m].cpu().numpy(), contacts=c.contacts[:nc].cpu().numpy(),
                geom=c.contact_geom[:nc].cpu().numpy(), stats=c.stats(reset=True))


def gpu_ctime(dem, w, pairs, prec):
    c = _ctx(dem, w, prec, max_pairs=max(len(pairs), 1))
    sc = dem.Scene.from_workload(w)
    pt = _pairs_tensor(pairs)
    c.collision_times(sc, pairs=pt)
    c.check()
    m = len(pairs)
    return dict(t_coll=c.t_coll[:m].cpu().numpy(), status=c.status[:m].cpu().numpy(),
                tri_ab=c.ct_ab[:m].cpu().numpy(), stats=c.stats(reset=True))


def _world_tri(w, p, t, a):
    R, X = oracle.pose(w.state, int(p), float(t))
    k = int(w.tri_off[p]) + int(a)
    return np.stack([R @ w.tris[s, k, :3].astype(np.float64) + X for s in range(3)])


def assert_contact_geometry(g_keys, g_geom, o_geom, w, pairs, t_eval, tol):
    """FP32 contact geometry: the distance within tol; the closest points are
    not unique for (near-)parallel triangles (paper Section 5, contact
    points), so each point must lie on its triangle and |pa - pb| = d, within
    tol."""
    assert np.max(np.abs(g_geom[:, 0] - o_geom[:, 0]), initial=0.0) <= tol
    for (k, a, b), gg in zip(g_keys, g_geom):
        i, j = pairs[k]
        t = t_eval[k] if t_eval is not None else min(w.state[W.F_TCUR, i], w.state[W.F_TCUR, j])
        TA, TB = _world_tri(w, i, t, a), _world_tri(w, j, t, b)
        da, _ = oracle.closest_pt_tri(gg[1:4], TA)
        db, _ = oracle.closest_pt_tri(gg[4:7], TB)
        assert np.sqrt(da) <= tol and np.sqrt(db) <= tol
        assert abs(np.linalg.norm(gg[1:4] - gg[4:7]) - gg[0]) <= tol


def assert_narrow_equal(g, o, w, pairs, prec, t_eval=None):
    R = float(np.max(w.state[W.F_RADIUS]))
    assert np.array_equal(g["flag"], o["flag"])
    assert np.array_equal(g["tri_ab"], o["tri_ab"])
    assert np.array_equal(g["dmin"], o["dmin"])
    assert np.array_equal(g["pa"], o["pa"]) and np.array_equal(g["pb"], o["pb"])
    assert np.array_equal(g["contacts"], o["contacts"])
    if prec == 1:
        assert np.array_equal(g["geom"], o["geom"])
    else:
        assert_contact_geometry(g["contacts"], g["geom"], o["geom"], w, pairs, t_eval, 1e-5 * R)
    # raw FP32 minimum is close to the FP64 one
    fin = np.isfinite(o["dmin"])
    assert np.max(np.abs(g["dmin32"][fin] - o["dmin"][fin]), initial=0.0) <= 1e-5 * R


# ----------------------------------------------------------------------------- broad phase

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_broad_phase_small(dem, seed):
    w = W.small_icospheres(seed)
    assert np.array_equal(gpu_candidates(dem, w), oracle.broad_phase(w))


def test_broad_phase_dense_full_size(dem):
    w = W.dense_packing(0)
    g = gpu_candidates(dem, w)
    o = oracle.broad_phase(w)
    assert len(o) > 1000
    assert np.array_equal(g, o)


def test_broad_phase_uneven_radii(dem):
    w = W.uneven_meshes(0, n=600, box=60.0)
    assert np.array_equal(gpu_candidates(dem, w), oracle.broad_phase(w))


def test_broad_phase_empty_and_static(dem):
    w = W.small_icospheres(0, n=8)
    w.state[W.F_X] += np.arange(8) * 100.0  # far apart: no pairs
    assert len(gpu_candidates(dem, w)) == 0
    w2 = W.small_icospheres(0)
    w2.is_static[:2] = 1  # injected overlapping pair (0,1) becomes static-static
    g = gpu_candidates(dem, w2)
    assert np.array_equal(g, oracle.broad_phase(w2))
    assert (0, 1) not in {tuple(p) for p in g}


# ----------------------------------------------------------------------------- narrow phase

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("seed", [0, 1])
def test_narrow_small_icospheres(dem, seed, prec):
    w = W.small_icospheres(seed)
    pairs = oracle.broad_phase(w)
    g = gpu_narrow(dem, w, pairs, prec)
    o = oracle.narrow_phase(w, pairs)
    assert_narrow_equal(g, o, w, pairs, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_narrow_dense_subset(dem, prec):
    w = W.dense_packing(3, nside=4)
    pairs = oracle.broad_phase(w)
    g = gpu_narrow(dem, w, pairs, prec)
    o = oracle.narrow_phase(w, pairs)
    assert (o["flag"] == 1).any() and (o["flag"] == 0).any() and (o["dmin"] == 0).any()
    assert_narrow_equal(g, o, w, pairs, prec)


_DENSE_ORACLE = {}


def _dense_oracle():
    """The oracle's narrow phase and collision times of every candidate pair of
    the dense packing (computed once per session: ~5e8 triangle-pair distances)."""
    if not _DENSE_ORACLE:
        w = W.dense_packing(0)
        pairs = oracle.broad_phase(w)
        _DENSE_ORACLE.update(w=w, pairs=pairs, on=oracle.narrow_phase(w, pairs), oc=oracle.collision_times(w, pairs))
    return _DENSE_ORACLE


@pytest.mark.parametrize("prec", PRECS)
def test_dense_full_size_exhaustive(dem, prec):
    """1000 icospheres (320 triangles), the benchmark's dense packing: every
    candidate pair, narrow phase at the pair start and collision times in one
    launch (dem_detect), against the oracle pair by pair."""
    d = _dense_oracle()
    w, pairs, on, oc = d["w"], d["pairs"], d["on"], d["oc"]
    c = _ctx(dem, w, prec, max_pairs=len(pairs))
    sc = dem.Scene.from_workload(w)
    c.build_candidates(sc)
    c.detect(sc)
    c.check()
    m = int(c.n_pairs.item())
    assert np.array_equal(c.pairs[:m].cpu().numpy(), pairs)
    nc = int(c.n_contacts.item())
    g = dict(dmin=c.dmin[:m].cpu().numpy(), pa=c.pa[:m].cpu().numpy(), pb=c.pb[:m].cpu().numpy(),
             tri_ab=c.tri_ab[:m].cpu().numpy(), flag=c.flag[:m].cpu().numpy(), dmin32=c.dmin32[:m].cpu().numpy(),
             contacts=c.contacts[:nc].cpu().numpy(), geom=c.contact_geom[:nc].cpu().numpy())
    assert_narrow_equal(g, on, w, pairs, prec)
    assert np.array_equal(c.status[:m].cpu().numpy(), oc["status"])
    assert np.array_equal(c.t_coll[:m].cpu().numpy(), oc["t_coll"])
    assert np.array_equal(c.ct_ab[:m].cpu().numpy(), oc["tri_ab"])
    c.close()


@pytest.mark.parametrize("prec", PRECS)
def test_narrow_uneven_meshes_multi_tile(dem, prec):
    """Ragged sizes: 80/320/1280-triangle icospheres and 20-200-point hulls
    (1280 > one shared-memory tile: several tiles per particle)."""
    w = W.uneven_meshes(1, n=300, box=30.0)
    pairs = oracle.broad_phase(w)
    cnt = w.tri_counts()
    big = pairs[(cnt[pairs[:, 0]] * cnt[pairs[:, 1]]) >= 1280 * 80]
    rest = pairs[(cnt[pairs[:, 0]] * cnt[pairs[:, 1]]) < 1280 * 80]
    sel = np.concatenate([big[:6], rest[:20]])
    sel = sel[np.lexsort((sel[:, 1], sel[:, 0]))]
    assert len(sel) >= 10
    g = gpu_narrow(dem, w, sel, prec)
    o = oracle.narrow_phase(w, sel)
    assert_narrow_equal(g, o, w, sel, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_narrow_time_eval_and_empty(dem, prec):
    w = W.small_icospheres(0)
    pairs = np.array([[0, 1], [2, 3], [4, 5], [2, 3]], np.int32)
    te = np.array([0.0, 4.5e-4, 1e-3, 9e-4])
    g = gpu_narrow(dem, w, pairs, prec, t_eval=te)
    o = oracle.narrow_phase(w, pairs, t_eval=te)
    assert_narrow_equal(g, o, w, pairs, prec, t_eval=te)
    # zero pairs
    g0 = gpu_narrow(dem, w, np.zeros((0, 2), np.int32), prec)
    assert len(g0["contacts"]) == 0


@pytest.mark.parametrize("prec", PRECS)
def test_narrow_adversarial_triangles(dem, prec):
    """One-triangle particles in near-degenerate configurations (near-parallel
    edges, slivers, near-touching, near-intersecting)."""
    rng = np.random.default_rng(11)
    for trial in range(40):
        A = rng.normal(0, 1, (3, 3))
        B = A.copy()
        kind = trial % 4
        if kind == 0:    # parallel copy at a small offset
            B += np.cross(A[1] - A[0], A[2] - A[0]) / np.linalg.norm(np.cross(A[1] - A[0], A[2] - A[0])) * rng.uniform(1e-4, 0.05)
            B += rng.normal(0, 0.3, 3) * np.array([1, 1, 0])
        elif kind == 1:  # sliver
            B = np.array([A[0], A[1], A[1] + rng.normal(0, 1e-3, 3)]) + rng.normal(0, 0.05, 3)
        elif kind == 2:  # near-parallel edges
            d = A[1] - A[0]
            B = np.array([A[0] + rng.normal(0, 1e-3, 3) + 0.02, A[1] + rng.normal(0, 1e-3, 3) + 0.02,
                          A[0] + rng.normal(0, 1, 3)])
        else:            # crossing / touching
            B = rng.normal(0, 1, (3, 3)) * 0.5 + A.mean(axis=0)
        eps = 0.01
        w = W.single_triangles(A, B, eps=eps / 2)
        pairs = np.array([[0, 1]], np.int32)
        g = gpu_narrow(dem, w, pairs, prec)
        o = oracle.narrow_phase(w, pairs)
        assert_narrow_equal(g, o, w, pairs, prec)


# ----------------------------------------------------------------------------- collision times

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ctime_small_icospheres(dem, seed, prec):
    w = W.small_icospheres(seed)
    pairs = oracle.broad_phase(w)
    g = gpu_ctime(dem, w, pairs, prec)
    o = oracle.collision_times(w, pairs)
    assert set(o["status"]) >= {0, 1, 2}
    for key in ("status", "t_coll", "tri_ab"):
        assert np.array_equal(g[key], o[key]), key
    assert g["stats"]["pair_evals"] == int(o["n_evals"].sum())


@pytest.mark.parametrize("prec", PRECS)
def test_ctime_dense_subset(dem, prec):
    w = W.dense_packing(4, nside=4)
    pairs = oracle.broad_phase(w)
    g = gpu_ctime(dem, w, pairs, prec)
    o = oracle.collision_times(w, pairs)
    for key in ("status", "t_coll", "tri_ab"):
        assert np.array_equal(g[key], o[key]), key


@pytest.mark.parametrize("prec", PRECS)
def test_ctime_dense_full_size_sampled(dem, prec):
    w = W.dense_packing(0)
    pairs = oracle.broad_phase(w)
    g = gpu_ctime(dem, w, pairs, prec)
    rng = np.random.default_rng(3)
    idx = np.sort(rng.choice(len(pairs), 16, replace=False))
    o = oracle.collision_times(w, pairs[idx])
    for key in ("status", "t_coll", "tri_ab"):
        assert np.array_equal(g[key][idx], o[key]), key


@pytest.mark.parametrize("prec", PRECS)
def test_ctime_search_heavy_packing(dem, prec):
    """The bench's search-heavy packing (14^3 icospheres of 320 triangles at
    volume fraction 0.35, v ~ N(0,10), w ~ N(0,2), dt = 1e-2): most pairs
    start apart and a fifth meet inside the step, so the samples and the
    bisection do the work.  The GPU computes every candidate pair; every pair
    that bisected (status 2) and a sample of the others equal the oracle."""
    w = W.dense_packing(0, nside=14, phi=0.35, vsig=10.0, wsig=2.0, dt=1e-2)
    pairs = oracle.broad_phase(w)
    g = gpu_ctime(dem, w, pairs, prec)
    rng = np.random.default_rng(3)
    bis = np.nonzero(g["status"] == 2)[0]
    assert len(bis) >= 100
    idx = np.unique(np.concatenate([bis, rng.choice(len(pairs), 120, replace=False)]))
    o = oracle.collision_times(w, pairs[idx])
    assert np.array_equal(g["status"][idx], o["status"])
    assert np.array_equal(g["t_coll"][idx], o["t_coll"])
    assert np.array_equal(g["tri_ab"][idx], o["tri_ab"])


@pytest.mark.parametrize("prec", PRECS)
def test_ctime_head_on_closed_form(dem, prec):
    for frac in (0.05, 0.5, 0.93):
        gap = 0.1 + frac * 1e-3
        w = W.injected_head_on(gap, 1.0, 0.05, 1e-3)
        pairs = np.array([[0, 1]], np.int32)
        g = gpu_ctime(dem, w, pairs, prec)
        o = oracle.collision_times(w, pairs)
        assert g["status"][0] == 2
        assert np.array_equal(g["t_coll"], o["t_coll"])
        tstar = (gap - 0.1) / 1.0
        assert tstar - 1e-15 <= g["t_coll"][0] <= tstar + 1e-6 + 1e-15


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("spill", [0, 1])
def test_ctime_after_interval_list_overflow(dem, prec, spill):
    """A fast head-on approach (320-triangle icospheres closing 0.8 over the
    step) puts more triangle pairs within eps + delta at the pair start than
    the shared-memory part of the pair-interval list holds: with the default
    global spill the samples and bisection steps decide on the spilled list,
    with a one-entry spill on full evaluations, in the separate and the fused
    call alike."""
    for frac in (0.3, 0.6, 0.93):
        gap = 0.1 + frac * 0.8
        w = W.injected_head_on(gap, 800.0, 0.05, 1e-3, subdiv=2)
        pairs = np.array([[0, 1]], np.int32)
        o = oracle.collision_times(w, pairs)
        assert o["status"][0] == 2
        c = dem.Context(K=w.K, tol=w.tol, precision=prec, max_particles=16, max_pairs=4096, max_contacts=1 << 20,
                        list_spill=spill)
        sc = dem.Scene.from_workload(w)
        c.collision_times(sc, pairs=_pairs_tensor(pairs))
        c.check()
        assert c.status[0].item() == o["status"][0] and c.t_coll[0].item() == o["t_coll"][0]
        assert np.array_equal(c.ct_ab[:1].cpu().numpy(), o["tri_ab"])
        c.close()
        c = dem.Context(K=w.K, tol=w.tol, precision=prec, max_particles=16, max_pairs=4096, max_contacts=1 << 20,
                        list_spill=spill)
        sc = dem.Scene.from_workload(w)
        c.step_fused(sc)
        c.check()
        assert int(c.n_pairs.item()) == 1
        assert c.status[0].item() == 2 and c.t_coll[0].item() == o["t_coll"][0]


# ----------------------------------------------------------------------------- clusters

def gpu_clusters(dem, n, edges, is_static):
    torch = _torch()
    c = dem.Context(max_particles=max(n, 16), max_pairs=max(len(edges), 16), max_contacts=16)
    et = _pairs_tensor(edges) if len(edges) else torch.zeros((1, 2), dtype=torch.int32, device="cuda")
    st = torch.from_numpy(np.ascontiguousarray(is_static, np.uint8)).cuda()
    ids = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    nc = torch.zeros(1, dtype=torch.int64, device="cuda")
    dem.dem_clusters(c.h, n, et, len(edges), None, st, ids, nc)
    c.check()
    return ids[:n].cpu().numpy(), int(nc.item())


def test_clusters_random_graphs(dem):
    rng = np.random.default_rng(0)
    for n, e in ((10, 0), (50, 30), (1000, 900), (20000, 25000)):
        edges = rng.integers(0, n, (e, 2)).astype(np.int32)
        edges = edges[edges[:, 0] != edges[:, 1]]
        st = (rng.random(n) < 0.03).astype(np.uint8)
        g, gn = gpu_clusters(dem, n, edges, st)
        o, on = oracle.clusters(n, edges, st)
        assert np.array_equal(g, o) and gn == on


def test_clusters_of_candidate_graph(dem):
    w = W.dense_packing(0)
    pairs = oracle.broad_phase(w)
    g, gn = gpu_clusters(dem, w.n, pairs, w.is_static)
    o, on = oracle.clusters(w.n, pairs, w.is_static)
    assert np.array_equal(g, o) and gn == on


def test_clusters_long_path(dem):
    n = 5000
    perm = np.random.default_rng(1).permutation(n)
    edges = np.stack([perm[:-1], perm[1:]], axis=1).astype(np.int32)
    g, gn = gpu_clusters(dem, n, edges, np.zeros(n, np.uint8))
    assert gn == 1 and np.all(g == 0)


# ----------------------------------------------------------------------------- whole step

@pytest.mark.parametrize("prec", PRECS)
def test_full_step_device_counts(dem, prec):
    """The four calls chained on device-side counts (no host round trip)."""
    w = W.small_icospheres(2)
    c = _ctx(dem, w, prec)
    sc = dem.Scene.from_workload(w)
    c.step(sc)
    c.check()
    m = int(c.n_pairs.item())
    pairs = c.pairs[:m].cpu().numpy()
    op = oracle.broad_phase(w)
    assert np.array_equal(pairs, op)
    on = oracle.narrow_phase(w, op)
    oc = oracle.collision_times(w, op)
    oi, onc = oracle.clusters(w.n, op, w.is_static)
    assert np.array_equal(c.flag[:m].cpu().numpy(), on["flag"])
    assert np.array_equal(c.status[:m].cpu().numpy(), oc["status"])
    assert np.array_equal(c.t_coll[:m].cpu().numpy(), oc["t_coll"])
    assert np.array_equal(c.cluster_id[:w.n].cpu().numpy(), oi)
    assert int(c.n_clusters.item()) == onc


def _adversarial_batch(n_pairs, seed):
    """Many one-triangle particle pairs in near-degenerate configurations,
    each pair far from the others, with random rigid poses."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(seed)
    meshes, pos, quat = [], [], []
    for k in range(n_pairs):
        scale = 10.0 ** rng.uniform(-2, 1.5)
        A = rng.normal(0, 1, (3, 3))
        kind = k % 6
        if kind == 0:    # parallel copy at a small offset
            n = np.cross(A[1] - A[0], A[2] - A[0])
            B = A + n / np.linalg.norm(n) * rng.uniform(1e-6, 0.05) + rng.normal(0, 0.3, 3) * [1, 1, 0]
        elif kind == 1:  # sliver
            B = np.array([A[0], A[1], A[1] + rng.normal(0, 1e-4, 3)]) + rng.normal(0, 0.05, 3)
        elif kind == 2:  # near-parallel edges
            B = np.array([A[0] + rng.normal(0, 1e-4, 3) + 0.02, A[1] + rng.normal(0, 1e-4, 3) + 0.02,
                          A[0] + rng.normal(0, 1, 3)])
        elif kind == 3:  # crossing or touching
            B = rng.normal(0, 1, (3, 3)) * 0.5 + A.mean(axis=0)
        elif kind == 4:  # vertex almost on the face
            c = A.mean(axis=0)
            n = np.cross(A[1] - A[0], A[2] - A[0])
            n /= np.linalg.norm(n)
            B = np.array([c + n * rng.uniform(-1e-5, 1e-5), c + n + rng.normal(0, 0.3, 3),
                          c + n + rng.normal(0, 0.3, 3)])
        else:            # generic, near
            B = rng.normal(0, 1, (3, 3)) + rng.normal(0, 0.5, 3)
        A, B = A * scale, B * scale
        q = Rotation.random(random_state=rng).as_quat()  # x y z w
        far = rng.normal(0, 50.0, 3)
        for T in (A, B):
            meshes.append(T.astype(np.float32).reshape(1, 3, 3))
            pos.append(far)
            quat.append([q[3], q[0], q[1], q[2]])
    n = len(meshes)
    w = W._assemble("adversarial", meshes, list(range(n)), pos, np.zeros((n, 3)), quat, np.zeros((n, 3)),
                    0.0, 1e-3, 0.0)
    # halo of each pair near its own distance scale: contact decisions land near the band
    pairs = np.array([(2 * k, 2 * k + 1) for k in range(n_pairs)], np.int32)
    return w, pairs


@pytest.mark.parametrize("seed", [0, 1])
def test_fp32_error_band_adversarial(dem, seed):
    """Near-degenerate one-triangle pairs (parallel offsets, slivers,
    near-parallel edges, crossings, a vertex on the face) with halos at half
    each pair's distance: every decision matches binary64."""
    w, pairs = _adversarial_batch(600, seed)
    o = oracle.narrow_phase(w, pairs)
    # halos at a fraction of each pair's distance, so the FP32 band is hit
    eps = np.zeros(w.n)
    eps[pairs[:, 0]] = eps[pairs[:, 1]] = 0.5 * o["dmin"] * (1 + np.random.default_rng(seed).normal(0, 1e-7, len(pairs)))
    w.state[W.F_EPS] = eps
    o = oracle.narrow_phase(w, pairs)
    g = gpu_narrow(dem, w, pairs, 0)
    assert_narrow_equal(g, o, w, pairs, 0)
    # the raw FP32 minimum is reported, not relied on (decisions rest on
    # certificates and binary64 values); on these well-scaled cases it stays
    # close to the binary64 one
    R = w.state[W.F_RADIUS]
    X = w.state[W.F_X:W.F_Z + 1]
    S = R[pairs[:, 0]] + R[pairs[:, 1]] + np.linalg.norm(X[:, pairs[:, 1]] - X[:, pairs[:, 0]], axis=0)
    rel = np.abs(g["dmin32"].astype(np.float64) - o["dmin"]) / S
    assert np.median(rel) <= 2.0 ** -21, np.median(rel)


def _worst_case_batch(n_pairs, seed):
    """Two-triangle particles at the worst cases of the FP32 filter's error
    analysis, each pair far from the others, random rigid poses:
      * near-parallel edges (angle 2^-10 .. 2^-14 rad, where the FP32 clamped
        segment-segment parameter is least accurate) whose closest points are
        interior, at distances 1e-7 .. 1e-4 of the edge length, plus a
        competing vertex over the other triangle's face just above or below
        that distance (the closest pair is decided by binary64);
      * a vertex on a Voronoi-region boundary of the other triangle (over an
        edge's line, over a vertex), a hair inside or outside;
      * a sliver triangle against a face.
    Returns (workload, pairs, the distance scale of each pair)."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(seed)
    meshes, pos, quat, scales = [], [], [], []
    for k in range(n_pairs):
        L = 10.0 ** rng.uniform(-1, 0.5)
        kind = k % 3
        if kind == 0:
            th = 2.0 ** -rng.uniform(10, 14)
            d0 = L * 10.0 ** rng.uniform(-7, -4)
            A1 = np.array([[0, 0, 0], [L, 0, 0], [L / 2, -L, 0]])
            c, sn = np.cos(th), np.sin(th)
            B1 = np.array([[L / 2 - L / 2 * c, -L / 2 * sn, d0], [L / 2 + L / 2 * c, L / 2 * sn, d0],
                           [L / 2, L, d0 + L]])
            h = d0 * (1.0 + rng.uniform(-0.3, 0.3)) + L * rng.uniform(0, 2e-6)
            p = A1.mean(axis=0)
            B2 = np.array([p + [0, 0, h], p + [0.3 * L, 0.1 * L, h + L], p + [-0.2 * L, 0.3 * L, h + L]])
            A2 = A1 + [10 * L, 0, 0]
            scale = d0
        elif kind == 1:
            A1 = np.array([[0, 0, 0], [L, 0, 0], [0.3 * L, 0.8 * L, 0]])
            h = L * 10.0 ** rng.uniform(-5, -1)
            if rng.uniform() < 0.5:  # over the line of edge 0-1 (edge / face / outside boundary)
                p = np.array([0.4 * L, rng.normal(0, 1e-7) * L, h])
            else:                    # over vertex 0 (vertex / edge boundaries)
                p = np.array([rng.normal(0, 1e-7) * L, rng.normal(0, 1e-7) * L, h])
            B1 = np.array([p, p + [0.2 * L, 0.1 * L, L], p + [-0.1 * L, 0.2 * L, L]])
            A2 = A1 + [10 * L, 0, 0]
            B2 = B1 + [10 * L, 0, 3 * L]
            scale = h
        else:
            A1 = np.array([[0, 0, 0], [L, 0, 0], [0.5 * L, 0.7 * L, 0]])
            h = L * 10.0 ** rng.uniform(-6, -2)
            base = np.array([0.3 * L, 0.2 * L, h])
            B1 = np.array([base, base + [0.5 * L, 0.1 * L, 1e-5 * L], base + [0.5 * L, 0.1 * L + 1e-6 * L, 2e-5 * L]])
            A2 = A1 + [10 * L, 0, 0]
            B2 = B1 + [0, 0, 2 * L]
            scale = h
        q = Rotation.random(random_state=rng).as_quat()  # x y z w
        far = rng.normal(0, 50.0, 3)
        for T in (np.stack([A1, A2]), np.stack([B1, B2])):
            meshes.append(T.astype(np.float32))
            pos.append(far)
            quat.append([q[3], q[0], q[1], q[2]])
        scales.append(scale)
    n = len(meshes)
    w = W._assemble("worst-cases", meshes, list(range(n)), pos, np.zeros((n, 3)), quat, np.zeros((n, 3)),
                    0.0, 1e-3, 0.0)
    pairs = np.array([(2 * k, 2 * k + 1) for k in range(n_pairs)], np.int32)
    return w, pairs, np.array(scales)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fp32_decisions_at_the_error_analysis_worst_cases(dem, prec, seed):
    """Closest pairs, contact flags, contact lists and collision statuses
    equal the oracle's on the worst cases of the FP32 error analysis, with
    halos that put every decision at the threshold (eps_pair at 0.5, 0.999,
    1.001 and 2 times each pair's binary64 distance)."""
    w, pairs, _ = _worst_case_batch(240, seed)
    o = oracle.narrow_phase(w, pairs)
    g = gpu_narrow(dem, w, pairs, prec)
    for key in ("flag", "tri_ab", "dmin", "pa", "pb"):
        assert np.array_equal(g[key], o[key]), key
    rng = np.random.default_rng(seed)
    for f in (0.5, 0.999, 1.001, 2.0):
        eps = np.zeros(w.n)
        eps[pairs[:, 0]] = eps[pairs[:, 1]] = 0.5 * f * o["dmin"] * (1 + rng.normal(0, 1e-9, len(pairs)))
        w.state[W.F_EPS] = eps
        o = oracle.narrow_phase(w, pairs)
        oc = oracle.collision_times(w, pairs)
        g = gpu_narrow(dem, w, pairs, prec)
        assert np.array_equal(g["flag"], o["flag"]), f
        assert np.array_equal(g["contacts"], o["contacts"]), f
        assert np.array_equal(g["tri_ab"], o["tri_ab"]) and np.array_equal(g["dmin"], o["dmin"]), f
        c = _ctx(dem, w, prec, max_pairs=len(pairs))
        sc = dem.Scene.from_workload(w)
        c.collision_times(sc, pairs=_pairs_tensor(pairs))
        c.check()
        m = len(pairs)
        assert np.array_equal(c.status[:m].cpu().numpy(), oc["status"]), f
        assert np.array_equal(c.t_coll[:m].cpu().numpy(), oc["t_coll"]), f
        assert np.array_equal(c.ct_ab[:m].cpu().numpy(), oc["tri_ab"]), f
        c.close()


@pytest.mark.parametrize("prec", PRECS)
def test_step_in_cuda_graph_matches_direct_calls(dem, prec):
    """The four calls captured in one CUDA graph (device-side counts keep the
    graph static) give the same outputs as direct calls."""
    import torch
    w = W.dense_packing(5, nside=5)
    sc = dem.Scene.from_workload(w)
    c1, c2 = _ctx(dem, w, prec), _ctx(dem, w, prec)
    c1.step(sc)
    c1.check()
    c2.step(sc)  # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        c2.step(sc)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    c2.check()
    m = int(c1.n_pairs.item())
    assert m == int(c2.n_pairs.item()) and m > 0
    for name in ("pairs", "dmin", "pa", "pb", "tri_ab", "flag", "t_coll", "status", "ct_ab"):
        assert torch.equal(getattr(c1, name)[:m], getattr(c2, name)[:m]), name
    nc = int(c1.n_contacts.item())
    assert nc == int(c2.n_contacts.item())
    assert torch.equal(c1.contacts[:nc], c2.contacts[:nc])
    assert torch.equal(c1.cluster_id[:w.n], c2.cluster_id[:w.n])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", ["small", "dense", "uneven"])
def test_detect_equals_separate_calls_and_oracle(dem, prec, kind):
    """dem_detect (narrow phase at the pair start + collision times in one
    launch) gives the outputs of the two separate calls."""
    import torch
    if kind == "small":
        w = W.small_icospheres(1)
    elif kind == "dense":
        w = W.dense_packing(6, nside=5)
    else:
        w = W.uneven_meshes(2, n=200, box=25.0)
    sc = dem.Scene.from_workload(w)
    c1, c2 = _ctx(dem, w, prec), _ctx(dem, w, prec)
    c1.build_candidates(sc)
    c1.narrow_phase(sc)
    c1.collision_times(sc)
    c1.check()
    c2.build_candidates(sc)
    c2.detect(sc)
    c2.check()
    m = int(c1.n_pairs.item())
    assert m > 0
    for name in ("dmin", "pa", "pb", "tri_ab", "flag", "t_coll", "status", "ct_ab"):
        assert torch.equal(getattr(c1, name)[:m], getattr(c2, name)[:m]), name
    nc = int(c1.n_contacts.item())
    assert nc == int(c2.n_contacts.item())
    assert torch.equal(c1.contacts[:nc], c2.contacts[:nc])
    if prec == 1:
        assert torch.equal(c1.contact_geom[:nc], c2.contact_geom[:nc])
    else:
        # FP32 contact geometry is defined to within the FP32 tolerance
        R = float(np.max(w.state[W.F_RADIUS]))
        assert float((c1.contact_geom[:nc] - c2.contact_geom[:nc]).abs().max()) <= 1e-5 * R
    if kind == "small":
        pairs = c2.pairs[:m].cpu().numpy()
        oc = oracle.collision_times(w, pairs)
        on = oracle.narrow_phase(w, pairs)
        assert np.array_equal(c2.status[:m].cpu().numpy(), oc["status"])
        assert np.array_equal(c2.t_coll[:m].cpu().numpy(), oc["t_coll"])
        assert np.array_equal(c2.ct_ab[:m].cpu().numpy(), oc["tri_ab"])
        assert np.array_equal(c2.dmin[:m].cpu().numpy(), on["dmin"])
