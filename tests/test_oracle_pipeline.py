"""Pins of the oracle's broad phase, narrow phase, collision-time search and
clusters against closed forms, library routines, brute force and physical
invariants.

Paper sections: broad phase and clusters (Section 3), collision-time search
and narrowing (Section 5, case distinction and Eq. "max time span between two
particles"), contact points (Section 5, Definition of a contact point).
"""
import math

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components
from scipy.spatial import cKDTree

import oracle
from paper_2309_15417_gb300 import workloads as W


# ----------------------------------------------------------------------------- broad phase

def test_broad_phase_equal_spheres_matches_kdtree():
    """All particles share one swept radius: candidates are the pairs within
    2 rho of each other's swept centres (scipy k-d tree)."""
    rng = np.random.default_rng(0)
    n = 600
    w = W._assemble("equal", [W.icosphere(1)], [0] * n, rng.uniform(0, 20, (n, 3)),
                    np.zeros((n, 3)), W.random_quaternions(rng, n), np.zeros((n, 3)), 0.0, 1e-3, 0.05)
    pairs = oracle.broad_phase(w)
    rho = w.state[W.F_RADIUS, 0] + 0.05
    ref = np.array(sorted(cKDTree(w.state[0:3].T).query_pairs(2 * rho)), dtype=np.int32).reshape(-1, 2)
    assert len(pairs) > 50
    assert np.array_equal(pairs, ref)


def test_broad_phase_boundary_closed_form():
    """Two particles on the x axis, swept spheres touching exactly (dyadic
    values, so the touching case is exact in binary64)."""
    eps, dt = 0.0625, 2.0 ** -10
    for gap, expect in ((0.0, 1), (2.0 ** -30, 0), (-(2.0 ** -30), 1)):
        R = 1.0
        v = 0.5
        # rho = R + eps + |v| dt / 2 ; swept centres move by v dt / 2 towards each other
        rho = R + eps + v * dt / 2
        D = 2 * rho + v * dt + gap
        w = W._assemble("two", [W.icosphere(1)], [0, 0], [[0, 0, 0], [D, 0, 0]],
                        [[v, 0, 0], [-v, 0, 0]], [[1, 0, 0, 0]] * 2, np.zeros((2, 3)), 0.0, dt, eps)
        w.state[W.F_RADIUS] = R
        assert len(oracle.broad_phase(w)) == expect


def test_broad_phase_is_conservative():
    """Every pair whose meshes come within the halo sum at some time of the
    step is a candidate (the swept spheres cover the particles, Section 3)."""
    for seed in range(3):
        w = W.small_icospheres(seed, n=24)
        w.state[W.F_VX:W.F_VZ + 1] *= 200.0   # large motion over the step
        cand = {tuple(p) for p in oracle.broad_phase(w)}
        allp = np.array([(i, j) for i in range(w.n) for j in range(i + 1, w.n)], np.int32)
        for t in np.linspace(0.0, 1e-3, 5):
            r = oracle.narrow_phase(w, allp, t_eval=np.full(len(allp), t), n_threads=8)
            touching = {tuple(p) for p, f in zip(allp, r["flag"]) if f}
            assert touching <= cand


def test_broad_phase_skips_static_static():
    w = W.small_icospheres(0, n=16, inject=True)
    w.is_static[:] = 0
    w.is_static[0] = w.is_static[1] = 1
    pairs = oracle.broad_phase(w)
    assert (0, 1) not in {tuple(p) for p in pairs}


def _static_pair(static_tris, quat, shift, at, rho=1.5, eps=0.25):
    """A static mesh (particle 0) and a resting icosphere (particle 1) whose
    swept sphere has radius ``rho`` (radius field overridden)."""
    w = W._assemble("static-box", [np.asarray(static_tris, np.float32), W.icosphere(1)], [0, 1],
                    [shift, at], np.zeros((2, 3)), [quat, (1, 0, 0, 0)], np.zeros((2, 3)), 0.0, 1e-3,
                    eps, is_static=[1, 0])
    w.state[W.F_RADIUS, 1] = rho - eps
    return w


def test_broad_phase_static_box_closed_form():
    """A static object pairs with a moving particle exactly when the swept
    sphere reaches the box of its world vertices widened by eps_s (Section 3,
    static geometry and axis-aligned boxes).  Dyadic values make touching
    exact: the triangle (0,0,0), (4,0,0), (0,4,0) turned by 180 degrees about
    z and moved by (1,2,3) has the world box [-3,1] x [-2,2] x [3,3]; widened
    by 0.25 and met by a sphere of radius 1.5 on a face, beyond an edge and
    off a corner (gaps 1, 1, 0.5).  The static particle is written second."""
    tri = [[[0, 0, 0], [4, 0, 0], [0, 4, 0]]]
    turn, shift = (0.0, 0.0, 0.0, 1.0), (1.0, 2.0, 3.0)
    tiny = 2.0 ** -30
    cases = [((1.0 + 0.25 + 1.5, 0.0, 3.0), 1), ((1.0 + 0.25 + 1.5 + tiny, 0.0, 3.0), 0),
             ((-3.0 - 0.25 - 1.5, 0.0, 3.0), 1), ((-3.0 - 0.25 - 1.5 - tiny, 0.0, 3.0), 0),
             ((0.0, 0.0, 3.0 + 0.25 + 1.5), 1), ((0.0, 0.0, 3.0 - 0.25 - 1.5 - tiny), 0),
             ((1.25 + 1.0, 2.25 + 1.0, 3.25 + 0.5), 1), ((1.25 + 1.0 + tiny, 2.25 + 1.0, 3.25 + 0.5), 0)]
    for at, expect in cases:
        pairs = oracle.broad_phase(_static_pair(tri, turn, shift, at))
        assert pairs.tolist() == ([[1, 0]] if expect else []), at


def test_broad_phase_static_box_not_sphere():
    """Particles well above a floor, inside the floor's bounding sphere but
    outside its widened box, are not candidates; those that reach the box are,
    and every pair with a static member has it second."""
    w = W.floor_scene(0)
    pairs = oracle.broad_phase(w)
    st = w.is_static.astype(bool)
    assert not st[pairs[:, 0]].any()
    floor_partners = set(pairs[pairs[:, 1] == 0, 0].tolist())
    kinds = np.array(w.meta["kind"])
    movers = [p for p in range(w.n) if not st[p]]
    clear = [p for p, k in zip(movers, kinds) if k == 3]
    resting = [p for p, k in zip(movers, kinds) if k == 0]
    R0 = w.state[W.F_RADIUS, 0]
    assert clear and resting
    for p in clear:
        assert p not in floor_partners
        assert np.linalg.norm(w.state[0:3, p] - w.state[0:3, 0]) < R0  # the sphere test would pair it
    assert set(resting) <= floor_partners
    # output sorted by (first, second)
    key = pairs[:, 0].astype(np.int64) * w.n + pairs[:, 1]
    assert np.all(np.diff(key) > 0)


def test_broad_phase_static_is_conservative():
    """Every (moving, static) pair whose meshes come within the halo sum at
    some time of the step is a candidate."""
    for seed in range(3):
        w = W.floor_scene(seed)
        cand = {tuple(p) for p in oracle.broad_phase(w)}
        statics = np.where(w.is_static)[0]
        allp = np.array([(p, s) for p in range(w.n) if not w.is_static[p] for s in statics], np.int32)
        hit = set()
        for t in np.linspace(0.0, 1e-3, 6):
            r = oracle.narrow_phase(w, allp, t_eval=np.full(len(allp), t), n_threads=8)
            hit |= {tuple(p) for p, f in zip(allp, r["flag"]) if f}
        assert len(hit) > 5
        assert hit <= cand


def test_static_member_does_not_limit_the_pair_interval():
    """A static object has no time step of its own (Section 3): a triangle
    falling flat onto a static floor triangle collides at t* = (h - eps_pair) / v
    in the moving particle's interval, although the floor's own t_cur (-1)
    and step (1e-6) would give an interval that misses it.  Dyadic values."""
    h, v, eps, dt = 0.25, 128.0, 2.0 ** -6, 2.0 ** -9
    floor = np.array([[[-8, -8, 0], [8, -8, 0], [0, 8, 0]]], np.float32)
    tri = np.array([[[-0.5, -0.5, 0], [0.5, -0.5, 0], [0, 0.5, 0]]], np.float32)
    w = W._assemble("static-interval", [floor, tri], [0, 1], [(0, 0, 0), (0, 0, h)], [(0, 0, 0), (0, 0, -v)],
                    [(1, 0, 0, 0)] * 2, np.zeros((2, 3)), 0.0, dt, eps, is_static=[1, 0])
    w.state[W.F_TCUR, 0] = -1.0
    w.state[W.F_DT, 0] = 1e-6
    pairs = oracle.broad_phase(w)
    assert pairs.tolist() == [[1, 0]]
    r = oracle.narrow_phase(w, pairs)
    assert r["dmin"][0] == h and r["flag"][0] == 0
    c = oracle.collision_times(w, pairs)
    tstar = (h - 2 * eps) / v
    assert c["status"][0] == 2
    assert tstar <= c["t_coll"][0] <= tstar + w.tol * dt


# ----------------------------------------------------------------------------- narrow phase

def test_narrow_contacts_are_exactly_the_close_triangle_pairs():
    w = W.dense_packing(0, nside=3)
    pairs = oracle.broad_phase(w)[:6]
    r = oracle.narrow_phase(w, pairs, n_threads=8)
    eps = w.state[W.F_EPS, 0] * 2
    for k, (i, j) in enumerate(pairs):
        rows = r["contacts"][r["contacts"][:, 0] == k]
        geom = r["geom"][r["contacts"][:, 0] == k]
        assert np.all(geom[:, 0] <= eps)
        # lexicographic order
        keys = rows[:, 1].astype(np.int64) * 100000 + rows[:, 2]
        assert np.all(np.diff(keys) > 0)
        # dmin is the minimum and attained by tri_ab; flag iff dmin <= eps
        assert r["flag"][k] == (r["dmin"][k] <= eps)
        if len(rows):
            assert r["dmin"][k] == geom[:, 0].min()
            first = np.argmin(geom[:, 0])
            assert tuple(rows[first, 1:]) == tuple(r["tri_ab"][k])
        assert abs(np.linalg.norm(r["pa"][k] - r["pb"][k]) - r["dmin"][k]) < 1e-12


def test_narrow_pair_symmetry():
    w = W.dense_packing(1, nside=3)
    pairs = oracle.broad_phase(w)[:5]
    r1 = oracle.narrow_phase(w, pairs, n_threads=8)
    r2 = oracle.narrow_phase(w, pairs[:, ::-1].copy(), n_threads=8)
    assert np.allclose(r1["dmin"], r2["dmin"], atol=1e-13, rtol=0)
    assert np.array_equal(r1["flag"], r2["flag"])
    s1 = {(k, a, b) for k, a, b in r1["contacts"]}
    s2 = {(k, b, a) for k, a, b in r2["contacts"]}
    assert s1 == s2


def test_narrow_rigid_motion_invariance():
    """Moving the whole scene rigidly leaves distances unchanged."""
    w = W.dense_packing(2, nside=3)
    pairs = oracle.broad_phase(w)[:5]
    r1 = oracle.narrow_phase(w, pairs, n_threads=8)
    w2 = W.dense_packing(2, nside=3)
    w2.state[W.F_X:W.F_Z + 1] += np.array([[37.5], [-12.25], [3.0]])
    r2 = oracle.narrow_phase(w2, pairs, n_threads=8)
    assert np.allclose(r1["dmin"], r2["dmin"], atol=1e-12, rtol=0)


# ----------------------------------------------------------------------------- collision times

def test_collision_time_head_on_closed_form():
    """Two vertex tips closing at speed v: d(t) = gap - v t, the halos meet at
    t* = (gap - eps_pair) / v; the search returns the upper end of a
    bisection bracket of width <= tol T that contains t*."""
    for frac in (0.05, 0.37, 0.5, 0.93):
        eps, dt, v = 0.05, 1e-3, 1.0
        gap = 2 * eps + frac * v * dt
        w = W.injected_head_on(gap, v, eps, dt)
        r = oracle.collision_times(w, np.array([[0, 1]]))
        tstar = (gap - 2 * eps) / v
        assert r["status"][0] == 2
        t = r["t_coll"][0]
        assert tstar - 1e-15 <= t <= tstar + w.tol * dt + 1e-15, (frac, t, tstar)
        assert tuple(r["tri_ab"][0]) != (-1, -1)


def test_collision_time_translating_triangle_closed_form():
    """A triangle translating along the normal of a parallel triangle:
    d(t) = h0 - v t."""
    A = np.array([[-1, -1, 0], [2, -1, 0], [-1, 2, 0]], np.float32)
    B = np.array([[0, 0, 0], [0.5, 0, 0], [0, 0.5, 0]], np.float32)
    for h0, v in ((0.03, 10.0), (0.021, 1.5), (0.05, 37.0)):
        eps, dt = 0.01, 1e-3
        w = W.single_triangles(A, B, pos_b=(0, 0, h0), vel_b=(0, 0, -v), eps=eps, dt=dt)
        r = oracle.collision_times(w, np.array([[0, 1]]))
        tstar = (h0 - 2 * eps) / v
        if tstar <= dt:
            assert r["status"][0] == 2
            assert tstar - 1e-15 <= r["t_coll"][0] <= tstar + w.tol * dt + 1e-15
        else:
            assert r["status"][0] == 0 and r["t_coll"][0] == dt


def test_collision_time_pure_rotation_closed_form():
    """A vertex at distance L from the body origin rotating about y with rate
    w0 over a plane at depth h: d(t) = h - L sin(w0 t), t* = asin((h-eps)/L)/w0."""
    L, h, w0, eps, dt = 1.0, 0.3, 400.0, 0.01, 1e-3
    A = np.array([[-5, -5, 0], [15, -5, 0], [-5, 15, 0]], np.float32)   # covers |x|,|y| <= 2
    B = np.array([[L, 0, 0], [-0.1, 0.1, 0], [-0.1, -0.1, 0]], np.float32)
    w = W.single_triangles(A, B, pos_a=(0, 0, -h), pos_b=(0, 0, 0), omega_b=(0, w0, 0), eps=eps, dt=dt)
    w.state[W.F_EPS] = eps / 2  # eps_pair = eps
    r = oracle.collision_times(w, np.array([[0, 1]]))
    tstar = math.asin((h - eps) / L) / w0
    assert tstar < dt
    assert r["status"][0] == 2
    assert tstar - 1e-12 <= r["t_coll"][0] <= tstar + w.tol * dt + 1e-12


def test_collision_time_status_cases():
    w = W.small_icospheres(0)
    r = oracle.collision_times(w, np.array([[0, 1], [2, 3], [4, 5]]))
    assert list(r["status"]) == [1, 2, 0]
    assert r["t_coll"][0] == 1e-3 and r["t_coll"][2] == 1e-3
    assert tuple(r["tri_ab"][2]) == (-1, -1)
    # evaluations: 1 for status 1, 1 + K for status 0, 1 + k + bisection for status 2
    assert r["n_evals"][0] == 1 and r["n_evals"][2] == 1 + w.K
    assert 1 + 1 <= r["n_evals"][1] <= 1 + w.K + 8


def test_collision_time_is_monotone_in_the_definition():
    """f(t) <= eps at the returned time, f > eps at the lower bracket end."""
    w = W.injected_head_on(0.1 + 0.4e-3, 1.0, 0.05, 1e-3)
    r = oracle.collision_times(w, np.array([[0, 1]]))
    t = r["t_coll"][0]
    at = oracle.narrow_phase(w, np.array([[0, 1]]), t_eval=np.array([t]), n_threads=1)
    assert at["flag"][0] == 1
    before = oracle.narrow_phase(w, np.array([[0, 1]]), t_eval=np.array([t - w.tol * 1e-3]), n_threads=1)
    assert before["flag"][0] == 0


# ----------------------------------------------------------------------------- clusters

def _scipy_min_labels(n, edges, is_static):
    keep = [(u, v) for u, v in edges if not is_static[u] and not is_static[v]]
    if keep:
        e = np.array(keep)
        g = coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n))
    else:
        g = coo_matrix((n, n))
    nc, lab = connected_components(g, directed=False)
    out = np.full(n, -1, np.int32)
    for c in range(nc):
        members = np.where((lab == c) & (is_static == 0))[0]
        if len(members):
            out[members] = members.min()
    return out


def test_clusters_match_scipy_connected_components():
    rng = np.random.default_rng(0)
    for n, e in ((50, 30), (400, 350), (1000, 2000)):
        edges = rng.integers(0, n, (e, 2)).astype(np.int32)
        edges = edges[edges[:, 0] != edges[:, 1]]
        st = (rng.random(n) < 0.05).astype(np.uint8)
        ids, nc = oracle.clusters(n, edges, st)
        ref = _scipy_min_labels(n, edges, st)
        assert np.array_equal(ids, ref)
        assert nc == len({x for x in ref if x >= 0})


def test_clusters_closed_form_graphs():
    # path 0-1-...-9 given backwards: one cluster labelled 0
    n = 10
    path = np.array([(i + 1, i) for i in range(n - 1)][::-1], np.int32)
    ids, nc = oracle.clusters(n, path)
    assert nc == 1 and np.all(ids == 0)
    # star around 7 plus isolated nodes
    star = np.array([(7, k) for k in (3, 5, 9)], np.int32)
    ids, nc = oracle.clusters(n, star)
    assert list(ids) == [0, 1, 2, 3, 4, 3, 6, 3, 8, 3] and nc == 7
    # two cliques joined only through a static node stay apart
    cl = [(a, b) for a in range(3) for b in range(a + 1, 3)] + \
         [(a, b) for a in range(4, 7) for b in range(a + 1, 7)] + [(2, 3), (3, 4)]
    st = np.zeros(7, np.uint8)
    st[3] = 1
    ids, nc = oracle.clusters(7, np.array(cl, np.int32), st)
    assert list(ids) == [0, 0, 0, -1, 4, 4, 4] and nc == 2
    # no edges: every particle its own cluster
    ids, nc = oracle.clusters(5, np.zeros((0, 2), np.int32))
    assert list(ids) == [0, 1, 2, 3, 4] and nc == 5


def test_broad_partners_agree_with_full_brute_force():
    for w in (W.dense_packing(0, nside=4), W.floor_scene(1)):
        if not w.is_static.any():
            w.is_static[3] = w.is_static[7] = 1
        full = oracle.broad_phase(w)
        for p in range(w.n):
            part = oracle.broad_partners(w, p)
            mine = full[(full[:, 0] == p) | (full[:, 1] == p)]
            assert np.array_equal(part, mine), p
