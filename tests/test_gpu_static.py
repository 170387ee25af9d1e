"""Static objects on the GPU (paper Section 3, static geometric objects):
candidate pairs against the widened boxes of static particles, the static
member second in its pair, narrow phase and collision times against meshes of
many 320-triangle tiles (tile culling), and clusters that ignore static
members.  Bar as in test_gpu_parity: integer outputs, decisions, closest pairs
and times bit-exact against the oracle; FP32 contact geometry within 1e-5 of
the largest particle radius.
"""
import numpy as np
import pytest

import oracle
from paper_2309_15417_gb300 import workloads as W
from test_gpu_parity import assert_narrow_equal, gpu_candidates

pytestmark = pytest.mark.gpu

PRECS = [0, 1]


def _step(dem, w, prec, max_pairs=1 << 16, max_contacts=1 << 21):
    c = dem.Context(K=w.K, tol=w.tol, precision=prec, max_particles=max(w.n, 16), max_pairs=max_pairs,
                    max_contacts=max_contacts, max_triangles=w.n_tris)
    sc = dem.Scene.from_workload(w)
    c.step_fused(sc)
    c.check()
    m = int(c.n_pairs.item())
    nc = int(c.n_contacts.item())
    g = dict(pairs=c.pairs[:m].cpu().numpy(), dmin=c.dmin[:m].cpu().numpy(), pa=c.pa[:m].cpu().numpy(),
             pb=c.pb[:m].cpu().numpy(), tri_ab=c.tri_ab[:m].cpu().numpy(), flag=c.flag[:m].cpu().numpy(),
             dmin32=c.dmin32[:m].cpu().numpy(), contacts=c.contacts[:nc].cpu().numpy(),
             geom=c.contact_geom[:nc].cpu().numpy(), t_coll=c.t_coll[:m].cpu().numpy(),
             status=c.status[:m].cpu().numpy(), ct_ab=c.ct_ab[:m].cpu().numpy(),
             ids=c.cluster_id[:w.n].cpu().numpy(), n_clusters=int(c.n_clusters.item()),
             stats=c.stats(reset=True))
    c.close()
    return g


def _subset(g, idx):
    """Narrow-phase outputs of the pairs idx, contacts renumbered to the subset."""
    out = {k: g[k][idx] for k in ("dmin", "pa", "pb", "tri_ab", "flag", "dmin32")}
    rows = np.isin(g["contacts"][:, 0], idx)
    remap = {int(k): q for q, k in enumerate(idx)}
    keys = g["contacts"][rows].copy()
    keys[:, 0] = [remap[int(k)] for k in keys[:, 0]]
    out["contacts"] = keys
    out["geom"] = g["geom"][rows]
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_broad_phase_static_boxes(dem, seed):
    w = W.floor_scene(seed)
    g = gpu_candidates(dem, w)
    o = oracle.broad_phase(w)
    assert np.array_equal(g, o)
    assert (o[:, 1] == 0).sum() > 5  # pairs with the floor (index 0), floor second


def test_broad_phase_static_anywhere(dem):
    """Static particles at the first, last and middle indices of a dense
    packing (moving icospheres marked static: their box is taken at t_cur)."""
    w = W.dense_packing(0, nside=6)
    w.is_static[[0, 5, 100, 215]] = 1
    g = gpu_candidates(dem, w)
    o = oracle.broad_phase(w)
    assert np.array_equal(g, o)
    assert np.isin(o[:, 1], [0, 5, 100, 215]).sum() > 4


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("seed", [0, 1])
def test_floor_scene_full_step(dem, seed, prec):
    """The floor (10 tiles of 320 triangles) and a static post against moving
    icospheres: every output of the fused step against the oracle."""
    w = W.floor_scene(seed)
    g = _step(dem, w, prec)
    o = oracle.broad_phase(w)
    assert np.array_equal(g["pairs"], o)
    on = oracle.narrow_phase(w, o)
    assert_narrow_equal(_subset(g, np.arange(len(o))), on, w, o, prec)
    oc = oracle.collision_times(w, o)
    assert np.array_equal(g["status"], oc["status"])
    assert np.array_equal(g["t_coll"], oc["t_coll"])
    assert np.array_equal(g["ct_ab"], oc["tri_ab"])
    assert {1, 2} <= set(oc["status"].tolist())
    ids, nc = oracle.clusters(w.n, o, w.is_static)
    assert np.array_equal(g["ids"], ids) and g["n_clusters"] == nc
    assert g["ids"][0] == -1


@pytest.mark.parametrize("prec", PRECS)
def test_settling_column_small(dem, prec):
    """A 10^3 settling column over a 64 x 64-quad floor (26 tiles): the
    candidate set and clusters in full, the pairs with the floor and a sample
    of the others one by one."""
    w = W.settling_column(0, nside=10, nq=64)
    g = _step(dem, w, prec)
    o = oracle.broad_phase(w)
    assert np.array_equal(g["pairs"], o)
    ids, nc = oracle.clusters(w.n, o, w.is_static)
    assert np.array_equal(g["ids"], ids) and g["n_clusters"] == nc
    floor = w.n - 1
    on_floor = np.where(o[:, 1] == floor)[0]
    assert len(on_floor) == 100  # the whole bottom layer
    rng = np.random.default_rng(0)
    others = np.where(o[:, 1] != floor)[0]
    idx = np.unique(np.concatenate([rng.choice(on_floor, 24, replace=False),
                                    rng.choice(others, min(12, len(others)), replace=False)]))
    sel = o[idx]
    on = oracle.narrow_phase(w, sel)
    assert_narrow_equal(_subset(g, idx), on, w, sel, prec)
    oc = oracle.collision_times(w, sel)
    assert np.array_equal(g["status"][idx], oc["status"])
    assert np.array_equal(g["t_coll"][idx], oc["t_coll"])
    assert np.array_equal(g["ct_ab"][idx], oc["tri_ab"])
    assert g["flag"][on_floor].sum() > 0


def test_floor_tiles_are_culled(dem):
    """The narrow phase of the pairs with the floor (26 tiles) scans only the
    floor tiles near each particle (both passes of the closest-pair search
    together stay far below one pass over every tile pair)."""
    import torch
    w = W.settling_column(0, nside=10, nq=64)
    floor = w.n - 1
    sel = oracle.broad_phase(w)
    sel = sel[sel[:, 1] == floor]
    n_tiles = int(np.ceil(w.tri_counts()[floor] / 320))
    for prec in PRECS:
        c = dem.Context(K=w.K, tol=w.tol, precision=prec, max_particles=w.n, max_pairs=len(sel),
                        max_contacts=1 << 20, max_triangles=w.n_tris)
        sc = dem.Scene.from_workload(w)
        c.narrow_phase(sc, pairs=torch.from_numpy(np.ascontiguousarray(sel)).cuda(), n_pairs=None)
        c.check()
        st = c.stats(reset=True)
        c.close()
        full = len(sel) * n_tiles  # every tile pair of one pass
        print(f"prec {prec}: {len(sel)} floor pairs, tile pairs scanned {st['tile_pairs']} of {full} per pass "
              f"({st['tile_pairs'] / full:.3f}), fp32 {st['dist_fp32']}, fp64 {st['dist_fp64']}")
        assert 0 < st["tile_pairs"] < 0.2 * full


def hovering_over_floor(seed, n=40, nq=48, size=34.0, eps=0.01):
    """Icospheres (320 triangles) hovering 1-4 halo widths above a static floor
    of nq x nq quads (Morton order, 15 tiles of 320 triangles), at rest: the
    closest floor triangle of every particle lies farther than the pass-0
    threshold, in a tile whose box bound also exceeds it."""
    rng = np.random.default_rng(seed)
    ico = W.icosphere(2)
    R = W.mesh_radius(ico)
    floor = W.floor_grid(nq, size)
    xy = rng.uniform(-size / 2 + 2.0, size / 2 - 2.0, size=(n, 2))
    gap = rng.uniform(1.05, 4.0, size=n) * 2 * eps
    pos = np.concatenate([np.column_stack([xy, R + gap]), [[0.0, 0.0, 0.0]]])
    quat = np.concatenate([W.random_quaternions(rng, n), [[1.0, 0.0, 0.0, 0.0]]])
    st = np.zeros(n + 1, np.uint8)
    st[n] = 1
    z = np.zeros((n + 1, 3))
    return W._assemble(f"hovering-{n}", [floor, ico], [1] * n + [0], pos, z, quat, z, 0.0, 1e-3, eps,
                       is_static=st)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("seed", [0, 1])
def test_closest_pair_in_a_tile_culled_by_the_first_pass(dem, prec, seed):
    """The closest pair's search beyond the first pass must scan the pairs of
    tiles that the first pass culled (regression: it skipped every triangle
    pair whose sphere bound was within the first threshold, as if the first
    pass had evaluated it)."""
    import torch
    w = hovering_over_floor(seed)
    pairs = np.array([[p, w.n - 1] for p in range(w.n - 1)], np.int32)
    on = oracle.narrow_phase(w, pairs)
    oc = oracle.collision_times(w, pairs)
    assert (on["dmin"] > 0.02).all()
    c = dem.Context(K=w.K, tol=w.tol, precision=prec, max_particles=w.n, max_pairs=1024, max_contacts=1 << 14,
                    max_triangles=w.n_tris)
    sc = dem.Scene.from_workload(w)
    gp = torch.from_numpy(pairs).cuda()
    c.narrow_phase(sc, pairs=gp)
    c.collision_times(sc, pairs=gp)
    c.check()
    m = len(pairs)
    assert np.array_equal(c.dmin[:m].cpu().numpy(), on["dmin"])
    assert np.array_equal(c.tri_ab[:m].cpu().numpy(), on["tri_ab"])
    assert np.array_equal(c.flag[:m].cpu().numpy(), on["flag"])
    assert np.array_equal(c.status[:m].cpu().numpy(), oc["status"])
    assert np.array_equal(c.ct_ab[:m].cpu().numpy(), oc["tri_ab"])
    c.close()
