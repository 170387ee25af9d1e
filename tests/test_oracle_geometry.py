"""Pins of the oracle's geometry against closed forms, library routines and
brute force (independent of the oracle's own formulas).

Section 5 of the paper ("Collision time detection") decomposes the
triangle-triangle distance into vertex-triangle and edge-edge distances; the
pose follows Section 2.1 (constant linear and angular velocity between
snapshots, spherical interpolation of the rotation).
"""
import math
import os

import numpy as np
import pytest
from scipy.optimize import minimize
from scipy.spatial.transform import Rotation, Slerp

import oracle
from paper_2309_15417_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _state_one(x=(0, 0, 0), v=(0, 0, 0), q=(1, 0, 0, 0), w=(0, 0, 0), t_cur=0.0):
    s = np.zeros((W.DEM_NFIELDS, 1))
    s[W.F_X:W.F_Z + 1, 0] = x
    s[W.F_VX:W.F_VZ + 1, 0] = v
    s[W.F_QW:W.F_QZ + 1, 0] = q
    s[W.F_WX:W.F_WZ + 1, 0] = w
    s[W.F_TCUR, 0] = t_cur
    return s


# ----------------------------------------------------------------------------- pose

def test_pose_rotation_about_z_closed_form():
    w0 = 0.7
    for h in (0.0, 1e-4, -3e-3, 0.1, 1.3, -2.5):
        s = _state_one(w=(0, 0, w0), t_cur=0.25)
        R, X = oracle.pose(s, 0, 0.25 + h)
        th = w0 * h
        Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
        assert np.max(np.abs(R - Rz)) < 4e-16
        assert np.all(X == 0)


def test_pose_matches_scipy_rotvec_composition():
    """World-frame angular velocity: R(t) = exp([w] h) R(q0) (scipy Rotation)."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        q0 = W.random_quaternions(rng, 1)[0]
        w = rng.normal(0, 2.0, 3)
        x, v = rng.normal(0, 5, 3), rng.normal(0, 1, 3)
        tc = rng.uniform(-1, 1)
        h = rng.uniform(-0.5, 0.5)
        if np.linalg.norm(w) * abs(h) / 2 > 1.5:
            continue
        s = _state_one(x, v, q0, w, tc)
        R, X = oracle.pose(s, 0, tc + h)
        ref = (Rotation.from_rotvec(w * h) * Rotation.from_quat([q0[1], q0[2], q0[3], q0[0]])).as_matrix()
        assert np.max(np.abs(R - ref)) < 2e-15
        # X = x + v h, checked against the same arithmetic on x, v
        assert np.max(np.abs(X - (x + v * h))) <= 4e-16 * (np.abs(x).max() + 1)


def test_pose_is_slerp_between_snapshots():
    """The paper interpolates rotations between snapshots with slerp; for a
    constant angular velocity the oracle's pose is that geodesic."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        q0 = W.random_quaternions(rng, 1)[0]
        w = rng.normal(0, 1.0, 3)
        T = 0.4
        s = _state_one(q=q0, w=w)
        R0, _ = oracle.pose(s, 0, 0.0)
        R1, _ = oracle.pose(s, 0, T)
        sl = Slerp([0.0, T], Rotation.from_matrix([R0, R1]))
        for t in np.linspace(0, T, 7):
            Rt, _ = oracle.pose(s, 0, t)
            assert np.max(np.abs(Rt - sl([t]).as_matrix()[0])) < 1e-13


def test_pose_series_truncation_at_domain_edge():
    # phi = |w| h / 2 = 1.5 is the documented edge of the 10-term series
    s = _state_one(w=(0, 3.0, 0))
    R, _ = oracle.pose(s, 0, 1.0)
    ref = Rotation.from_rotvec([0, 3.0, 0]).as_matrix()
    assert np.max(np.abs(R - ref)) < 1e-15


# ----------------------------------------------------------------------------- triangle distance

def _golden_cases():
    cases = []
    with open(os.path.join(GOLDEN, "tri_dist_closed_forms.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            vals = [float(x) for x in line.split()]
            assert len(vals) == 19
            cases.append((np.array(vals[0:9]).reshape(3, 3), np.array(vals[9:18]).reshape(3, 3), vals[18]))
    return cases


def test_tri_dist_golden_closed_forms():
    cases = _golden_cases()
    assert len(cases) >= 8
    for A, B, d in cases:
        got, pa, pb = oracle.tri_dist(A, B)
        assert abs(got - d) <= 1e-15 * max(1.0, d), (A, B, d, got)
        assert abs(np.linalg.norm(pa - pb) - got) <= 1e-14


def test_tri_dist_skew_edges_closed_form():
    """Edges crossing in projection with vertical offset: distance of the two
    lines |(p2-p1).(d1 x d2)| / |d1 x d2| when the closest points are interior."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        h = rng.uniform(0.01, 1.0)
        ang = rng.uniform(0.3, math.pi - 0.3)
        # edge 1 along x through the origin, edge 2 at height h at angle ang
        d1 = np.array([1.0, 0, 0])
        d2 = np.array([math.cos(ang), math.sin(ang), 0])
        A = np.array([-d1, d1, [0.0, 0.0, -3.0]])            # third vertex far below
        B = np.array([h * np.array([0, 0, 1]) - d2, h * np.array([0, 0, 1]) + d2, [0.0, 0.0, h + 3.0]])
        R = Rotation.random(random_state=rng).as_matrix()
        t = rng.normal(0, 3, 3)
        A2, B2 = A @ R.T + t, B @ R.T + t
        got, pa, pb = oracle.tri_dist(A2, B2)
        n = np.cross(d1, d2)
        ref = abs(np.dot(np.array([0, 0, h]), n)) / np.linalg.norm(n)
        assert abs(got - ref) < 1e-13


def _rand_tri(rng, scale=1.0):
    return rng.normal(0, scale, (3, 3))


def _qp_distance(A, B):
    """min |A^T l - B^T m| over the two probability simplices (scipy SLSQP),
    several starts."""
    best = np.inf
    cons = [{"type": "eq", "fun": lambda z: z[0] + z[1] + z[2] - 1.0},
            {"type": "eq", "fun": lambda z: z[3] + z[4] + z[5] - 1.0}]

    def f(z):
        r = z[:3] @ A - z[3:] @ B
        return r @ r

    def g(z):
        r = z[:3] @ A - z[3:] @ B
        return np.concatenate([2 * A @ r, -2 * B @ r])

    for z0 in (np.full(6, 1 / 3), np.array([1, 0, 0, 1, 0, 0.0]), np.array([0, 1, 0, 0, 0, 1.0]),
               np.array([0, 0, 1, 0, 1, 0.0])):
        res = minimize(f, z0, jac=g, bounds=[(0, 1)] * 6, constraints=cons, method="SLSQP",
                       options=dict(ftol=1e-16, maxiter=500))
        best = min(best, float(res.fun))
    return math.sqrt(max(best, 0.0))


def test_tri_dist_matches_convex_qp():
    rng = np.random.default_rng(4)
    n_int = 0
    for k in range(300):
        A = _rand_tri(rng)
        B = _rand_tri(rng) + rng.normal(0, 1.5, 3)
        d, pa, pb = oracle.tri_dist(A, B)
        ref = _qp_distance(A, B)
        n_int += d == 0.0
        assert abs(d - ref) < 2e-6, (k, d, ref)
    assert n_int > 5  # intersecting cases are exercised


def _bary_ok(P, T, tol=1e-9):
    # P in triangle T: solve barycentric least squares
    M = np.stack([T[1] - T[0], T[2] - T[0]], axis=1)
    uv, *_ = np.linalg.lstsq(M, P - T[0], rcond=None)
    res = np.linalg.norm(M @ uv - (P - T[0]))
    return res < tol and uv[0] >= -tol and uv[1] >= -tol and uv.sum() <= 1 + tol


def test_tri_dist_closest_points_are_valid():
    rng = np.random.default_rng(5)
    for _ in range(500):
        A = _rand_tri(rng)
        B = _rand_tri(rng) + rng.normal(0, 2.0, 3)
        d, pa, pb = oracle.tri_dist(A, B)
        assert _bary_ok(pa, A) and _bary_ok(pb, B)
        assert abs(np.linalg.norm(pa - pb) - d) < 1e-12


def test_tri_dist_symmetric_and_rigid_invariant():
    rng = np.random.default_rng(6)
    for _ in range(300):
        A = _rand_tri(rng)
        B = _rand_tri(rng) + rng.normal(0, 2.0, 3)
        d, pa, pb = oracle.tri_dist(A, B)
        d2, qa, qb = oracle.tri_dist(B, A)
        assert abs(d - d2) <= 1e-13
        R = Rotation.random(random_state=rng).as_matrix()
        t = rng.normal(0, 10.0, 3)
        d3, _, _ = oracle.tri_dist(A @ R.T + t, B @ R.T + t)
        assert abs(d - d3) <= 1e-12 * (1 + np.linalg.norm(t))


def test_tri_dist_brute_force_barycentric_sampling():
    """Sampled minimum over barycentric grids is >= d and converges from
    above as the grid is refined."""
    rng = np.random.default_rng(7)

    def samples(T, m):
        i, j = np.meshgrid(np.arange(m + 1), np.arange(m + 1), indexing="ij")
        keep = i + j <= m
        u, v = i[keep] / m, j[keep] / m
        return T[0] + np.outer(u, T[1] - T[0]) + np.outer(v, T[2] - T[0])

    for _ in range(20):
        A = _rand_tri(rng)
        B = _rand_tri(rng) + rng.normal(0, 2.5, 3)
        d, _, _ = oracle.tri_dist(A, B)
        prev = np.inf
        for m in (4, 16, 64):
            SA, SB = samples(A, m), samples(B, m)
            dd = np.sqrt(((SA[:, None, :] - SB[None, :, :]) ** 2).sum(-1)).min()
            assert dd >= d - 1e-12
            assert dd <= prev + 1e-12
            prev = dd
        # edge length / 64 resolution bound
        h = max(np.linalg.norm(A[1] - A[0]), np.linalg.norm(A[2] - A[0]), np.linalg.norm(B[1] - B[0]),
                np.linalg.norm(B[2] - B[0])) / 64
        assert prev - d <= 2 * h


def test_closest_point_on_triangle_regions():
    T = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.0, 1, 0]])
    cases = [((-1, -1, 2), (0, 0, 0)), ((2, -1, 0), (1, 0, 0)), ((-1, 3, -1), (0, 1, 0)),
             ((0.5, -2, 1), (0.5, 0, 0)), ((-2, 0.25, 0), (0, 0.25, 0)),
             ((1, 1, 3), (0.5, 0.5, 0)), ((0.2, 0.3, -4), (0.2, 0.3, 0))]
    for p, q in cases:
        d2, got = oracle.closest_pt_tri(np.array(p, float), T)
        assert np.allclose(got, q, atol=1e-15)
        assert abs(d2 - np.sum((np.array(p) - np.array(q)) ** 2)) < 1e-14


def test_seg_seg_closed_forms():
    # parallel overlapping segments at distance 2
    d2, c1, c2 = oracle.seg_seg([0, 0, 0], [2, 0, 0], [1, 2, 0], [3, 2, 0])
    assert abs(d2 - 4.0) < 1e-15
    # perpendicular crossing at offset 0.5
    d2, c1, c2 = oracle.seg_seg([-1, 0, 0], [1, 0, 0], [0, -1, 0.5], [0, 1, 0.5])
    assert abs(d2 - 0.25) < 1e-15 and np.allclose(c1, [0, 0, 0]) and np.allclose(c2, [0, 0, 0.5])
    # endpoint-endpoint
    d2, c1, c2 = oracle.seg_seg([0, 0, 0], [1, 0, 0], [2, 1, 0], [3, 5, 0])
    assert abs(d2 - 2.0) < 1e-15 and np.allclose(c1, [1, 0, 0]) and np.allclose(c2, [2, 1, 0])


# ----------------------------------------------------------------------------- meshes

def _inradius(soup):
    n = np.cross(soup[:, 1] - soup[:, 0], soup[:, 2] - soup[:, 0]).astype(np.float64)
    return float(np.min(np.abs(np.einsum("ij,ij->i", n, soup[:, 0])) / np.linalg.norm(n, axis=1)))


@pytest.mark.parametrize("subdiv", [1, 2])
def test_icosphere_pair_distance_bounds(subdiv):
    """Two icospheres at centre distance D: D - 2R <= d <= D - 2 r_in."""
    rng = np.random.default_rng(10 + subdiv)
    mesh = W.icosphere(subdiv)
    R = W.mesh_radius(mesh)
    rin = _inradius(mesh.astype(np.float64))
    for D in (2.05, 2.2, 3.0):
        pos = np.array([[0.0, 0, 0], D * W.random_quaternions(rng, 1)[0, 1:] /
                        np.linalg.norm(W.random_quaternions(rng, 1)[0, 1:])])
        pos[1] = D * pos[1] / np.linalg.norm(pos[1])
        w = W._assemble("pair", [mesh], [0, 0], pos, np.zeros((2, 3)), W.random_quaternions(rng, 2),
                        np.zeros((2, 3)), 0.0, 1e-3, 0.01)
        r = oracle.narrow_phase(w, np.array([[0, 1]]), n_threads=4)
        d = r["dmin"][0]
        assert D - 2 * R - 1e-12 <= d <= D - 2 * rin + 1e-12, (D, d, R, rin)
