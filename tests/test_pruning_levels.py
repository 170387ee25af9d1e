"""Pruning levels measured against each other (CPU, binary64): the pair
kernel's bounding-sphere levels (32-triangle groups, 8-triangle subgroups,
triangles) against the paper's surrogate meshes (Section 5: coarser triangle
meshes that are conservative -- every fine triangle lies within a thickness h
of its coarse parent -- and cheaper to test), on the candidate pairs of a dense
packing of 320-triangle icospheres.

The surrogates of a subdivision-2 icosphere are its own coarser levels: the
80 faces of subdivision 1 (parents of 4 consecutive fine triangles) and the 20
icosahedron faces (parents of 16); h of a coarse face is the largest distance
from a fine vertex below it to the face, so d(t1, t2) >= d(T1, T2) - h1 - h2
for fine triangles t below coarse T.  A coarse test is a triangle-pair
distance, as expensive as a fine one; a sphere test is a dozen flops.

The test counts, per path, the tests of each kind and the fine distances
left, checks that every path keeps every triangle pair within the threshold
(conservative), and that the sphere levels need fewer flops than the
surrogate meshes for any plausible cost of a triangle-pair distance."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2309_15417_gb300 import workloads as W  # noqa: E402

SPHERE_FLOPS = 13  # one sphere-pair test: centre difference, squared norm, compare


def _world(w, p, t):
    R, X = oracle.pose(w.state, p, t)
    T = w.tris[:, w.tri_off[p]:w.tri_off[p + 1], :3].astype(np.float64)  # (3, n, 3)
    return np.einsum("ab,snb->nsa", R, T) + X, R, X  # (n, 3 vertices, 3)


def _tri_spheres(V):
    c = V.mean(axis=1)
    r = np.linalg.norm(V - c[:, None, :], axis=2).max(axis=1)
    return c, r


def _level_spheres(c, r, size):
    """Box centre of the triangle spheres of each run of `size`, radius covering them."""
    n = len(c) // size
    cc, rr = c[:n * size].reshape(n, size, 3), r[:n * size].reshape(n, size)
    lo, hi = (cc - rr[..., None]).min(axis=1), (cc + rr[..., None]).max(axis=1)
    g = 0.5 * (lo + hi)
    gr = (np.linalg.norm(cc - g[:, None, :], axis=2) + rr).max(axis=1)
    return g, gr


def _thickness(fine, coarse, per):
    """h of each coarse face: the largest distance of a fine vertex below it."""
    h = np.zeros(len(coarse))
    for k, T in enumerate(coarse):
        for t in fine[k * per:(k + 1) * per]:
            for v in t:
                d2, _ = oracle.closest_pt_tri(v, T)
                h[k] = max(h[k], np.sqrt(d2))
    return h


def _sphere_path(cA, rA, cB, rB, thr):
    """Survivors of the group -> subgroup -> triangle sphere tests."""
    tests = 0
    gA, grA = _level_spheres(cA, rA, 32)
    gB, grB = _level_spheres(cB, rB, 32)
    hA, hrA = _level_spheres(cA, rA, 8)
    hB, hrB = _level_spheres(cB, rB, 8)
    dg = np.linalg.norm(gA[:, None] - gB[None], axis=2) - grA[:, None] - grB[None]
    tests += dg.size
    out = []
    for ga, gb in zip(*np.nonzero(dg <= thr)):
        ha, hb = np.arange(4 * ga, 4 * ga + 4), np.arange(4 * gb, 4 * gb + 4)
        dh = np.linalg.norm(hA[ha][:, None] - hB[hb][None], axis=2) - hrA[ha][:, None] - hrB[hb][None]
        tests += dh.size
        for x, y in zip(*np.nonzero(dh <= thr)):
            ta, tb = np.arange(8 * ha[x], 8 * ha[x] + 8), np.arange(8 * hb[y], 8 * hb[y] + 8)
            dt = np.linalg.norm(cA[ta][:, None] - cB[tb][None], axis=2) - rA[ta][:, None] - rB[tb][None]
            tests += dt.size
            for u, v in zip(*np.nonzero(dt <= thr)):
                out.append((ta[u], tb[v]))
    return tests, out


def _surrogate_path(LA, LB, hA, hB, thr):
    """Survivors of the coarse levels (lists of (faces, thickness, children per face)), each test a
    binary64 triangle-pair distance less the two thicknesses."""
    tests = 0
    live = [(a, b) for a in range(len(LA[0])) for b in range(len(LB[0]))]
    for lvl in range(len(LA)):
        FA, FB, per = LA[lvl], LB[lvl], 4  # every face has 4 children one level down
        nxt = []
        for a, b in live:
            d, _, _ = oracle.tri_dist(FA[a], FB[b])
            tests += 1
            if d - hA[lvl][a] - hB[lvl][b] <= thr:
                nxt.extend((per * a + x, per * b + y) for x in range(per) for y in range(per))
        live = nxt
    return tests, live


def _coarse_levels(w, p, t):
    """World-frame levels of particle p's icosphere: subdivision 0, 1 (surrogates) and 2 (fine)."""
    R, X = oracle.pose(w.state, p, t)
    return [np.einsum("ab,nsb->nsa", R, W.icosphere(s).astype(np.float64)) + X for s in (0, 1, 2)]


def test_sphere_levels_prune_cheaper_than_surrogate_meshes():
    oracle.build()
    w = W.dense_packing(0, nside=5)
    pairs = oracle.broad_phase(w)
    rng = np.random.default_rng(0)
    pairs = pairs[rng.choice(len(pairs), 24, replace=False)]
    # fine mesh and its surrogates in the body frame; thicknesses once
    body = [W.icosphere(s).astype(np.float64) for s in (0, 1, 2)]
    assert np.array_equal(body[2].astype(np.float32), w.tris[:, :320, :3].transpose(1, 0, 2))
    h0 = _thickness(body[2], body[0], 16)
    h1 = _thickness(body[2], body[1], 4)
    tot = dict(sph_tests=0, sph_dist=0, sur_tests=0, sur_dist=0, mix_sph=0, mix_sur=0, mix_dist=0, near=0)
    for i, j in pairs:
        t = min(w.state[W.F_TCUR, i], w.state[W.F_TCUR, j])
        eps = w.state[W.F_EPS, i] + w.state[W.F_EPS, j]
        T = min(w.state[W.F_DT, i], w.state[W.F_DT, j])
        vel = [np.linalg.norm(w.state[W.F_VX:W.F_VZ + 1, p]) for p in (i, j)]
        om = [np.linalg.norm(w.state[W.F_WX:W.F_WZ + 1, p]) for p in (i, j)]
        thr = eps + (vel[0] + vel[1] + om[0] * w.state[W.F_RADIUS, i] + om[1] * w.state[W.F_RADIUS, j]) * T
        VA, _, _ = _world(w, int(i), t)
        VB, _, _ = _world(w, int(j), t)
        cA, rA = _tri_spheres(VA)
        cB, rB = _tri_spheres(VB)
        # sphere levels
        nt, sph = _sphere_path(cA, rA, cB, rB, thr)
        tot["sph_tests"] += nt
        tot["sph_dist"] += len(sph)
        # surrogate meshes (subdivision 0, then 1, then the fine triangles)
        LA, LB = _coarse_levels(w, int(i), t), _coarse_levels(w, int(j), t)
        ns, sur = _surrogate_path(LA[:2], LB[:2], [h0, h1], [h0, h1], thr)
        tot["sur_tests"] += ns
        tot["sur_dist"] += len(sur)
        # spheres down to subgroups, then the subdivision-1 surrogates (2 per subgroup)
        gA, grA = _level_spheres(cA, rA, 8)
        gB, grB = _level_spheres(cB, rB, 8)
        dh = np.linalg.norm(gA[:, None] - gB[None], axis=2) - grA[:, None] - grB[None]
        tot["mix_sph"] += dh.size
        for x, y in zip(*np.nonzero(dh <= thr)):
            for a in (2 * x, 2 * x + 1):
                for b in (2 * y, 2 * y + 1):
                    d, _, _ = oracle.tri_dist(LA[1][a], LB[1][b])
                    tot["mix_sur"] += 1
                    if d - h1[a] - h1[b] <= thr:
                        tot["mix_dist"] += 16
        # every path keeps every triangle pair within the threshold
        # (a triangle lies in its sphere, so only pairs of spheres within thr can be)
        gap = np.linalg.norm(cA[:, None] - cB[None], axis=2) - rA[:, None] - rB[None]
        near = {(a, b) for a, b in zip(*np.nonzero(gap <= thr))
                if oracle.tri_dist(VA[a], VB[b])[0] <= thr}
        tot["near"] += len(near)
        assert near <= set(sph) and near <= set(sur)
    print("\npruning levels on", len(pairs), "dense-packing pairs:", tot)
    for F in (200, 600, 1300, 2000):  # FP32 flops of one triangle-pair distance
        sphere = SPHERE_FLOPS * tot["sph_tests"] + F * tot["sph_dist"]
        surrogate = F * (tot["sur_tests"] + tot["sur_dist"])
        mixed = SPHERE_FLOPS * tot["mix_sph"] + F * (tot["mix_sur"] + tot["mix_dist"])
        print(f"F={F}: sphere levels {sphere:.3e} flops, surrogate meshes {surrogate:.3e}, "
              f"subgroup spheres + surrogates {mixed:.3e}")
        assert sphere < surrogate and sphere < mixed
