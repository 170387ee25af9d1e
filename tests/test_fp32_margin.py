"""The FP32 certificate margin E = 2^-17 M checked against the binary64 oracle
(CPU).  The pair kernel's FP32 arithmetic for one triangle pair is emulated
operation by operation in numpy float32: the relative pose formed in FP32
from the rounded binary64 rotations and positions (separate roundings, and
the fused form the compiler may choose), B's vertices moved by fmaf chains,
the dot products of the separation certificate as fmaf chains, and the
normalisation gap * rsqrtf(n.n) with rsqrtf pushed to the far end of its
2-ulp bound.  An fmaf is emulated as the exact float64 product plus the
addend, rounded to float32 (the float64 sum may round once more; the
analysis has room for that).

On near-parallel edges, vertices over faces, slivers and random pairs, at
scales from 1e-3 to 1e2, body origins up to 20 triangle sizes away and world
positions up to 1e3 away from the origin, the certificate less E never
exceeds the oracle's binary64 distance plus m64 = 2^-40 (S + |X_A| + |X_B|),
and its error against the exact separation stays below the derived 45u M
(u = 2^-24): the analysis's terms, not only the margin, are checked."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

U = 2.0 ** -24
ERR_REL32 = 2.0 ** -17
ERR_REL64 = 2.0 ** -40
f32 = np.float32


def fma32(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def relative_pose32(RA, XA, RB, XB, fused):
    """Rr = R_A^T R_B and t = R_A^T (X_B - X_A), each entry from the rounded
    binary64 values in FP32 (lane 3r+c: sum over k of RA[k][r] RB[k][c])."""
    Rr = np.zeros((3, 3), np.float32)
    t = np.zeros(3, np.float32)
    d = [f32(XB[k] - XA[k]) for k in range(3)]
    for r in range(3):
        ra = [f32(RA[k][r]) for k in range(3)]
        for c in range(3):
            rb = [f32(RB[k][c]) for k in range(3)]
            if fused:
                Rr[r, c] = fma32(ra[2], rb[2], fma32(ra[1], rb[1], f32(ra[0] * rb[0])))
            else:
                Rr[r, c] = f32(f32(f32(ra[0] * rb[0]) + f32(ra[1] * rb[1])) + f32(ra[2] * rb[2]))
        if fused:
            t[r] = fma32(ra[2], d[2], fma32(ra[1], d[1], f32(ra[0] * d[0])))
        else:
            t[r] = f32(f32(f32(ra[0] * d[0]) + f32(ra[1] * d[1])) + f32(ra[2] * d[2]))
    return Rr, t


def move32(Rr, t, b):
    """Rr b + t as the kernel's fmaf chains."""
    return np.array([fma32(Rr[r, 0], b[0], fma32(Rr[r, 1], b[1], fma32(Rr[r, 2], b[2], t[r]))) for r in range(3)],
                    np.float32)


def dot32(n, v):
    return fma32(n[2], v[2], fma32(n[1], v[1], f32(n[0] * v[0])))


def certificate32(X, Y, n):
    """Separation of the float32 point sets X (A) and Y (B) along n, as the
    kernel computes it, with rsqrtf at the end of its 2-ulp bound that makes
    the certificate larger."""
    mx = max(dot32(n, x) for x in X)
    mn = min(dot32(n, y) for y in Y)
    gap = f32(mn - mx)
    nn = dot32(n, n)
    if not nn > 1e-30:
        return -np.inf
    rs = f32(1.0 / np.sqrt(np.float64(nn)))
    rs = f32(np.float64(rs) * (1.0 + 4 * U if gap > 0 else 1.0 - 4 * U))
    return float(f32(gap * rs))


def _pair(rng, kind, L):
    """Two triangles in their body frames (float32) and their poses."""
    if kind == 0:  # near-parallel edges, interior closest points
        th = 2.0 ** -rng.uniform(8, 14)
        d0 = L * 10.0 ** rng.uniform(-7, -2)
        A = np.array([[0, 0, 0], [L, 0, 0], [L / 2, -L, 0]])
        c, s = np.cos(th), np.sin(th)
        B = np.array([[L / 2 - L / 2 * c, -L / 2 * s, d0], [L / 2 + L / 2 * c, L / 2 * s, d0], [L / 2, L, d0 + L]])
    elif kind == 1:  # a vertex over the face, near a Voronoi boundary
        h = L * 10.0 ** rng.uniform(-6, -1)
        A = np.array([[0, 0, 0], [L, 0, 0], [0.3 * L, 0.8 * L, 0]])
        p = np.array([0.4 * L, rng.normal(0, 1e-6) * L, h])
        B = np.array([p, p + [0.2 * L, 0.1 * L, L], p + [-0.1 * L, 0.2 * L, L]])
    elif kind == 2:  # a sliver against a face
        h = L * 10.0 ** rng.uniform(-6, -2)
        A = np.array([[0, 0, 0], [L, 0, 0], [0.5 * L, 0.7 * L, 0]])
        base = np.array([0.3 * L, 0.2 * L, h])
        B = np.array([base, base + [0.5 * L, 0.1 * L, 1e-5 * L], base + [0.5 * L, 0.1 * L + 1e-6 * L, 2e-5 * L]])
    else:  # random triangles near each other
        A = rng.normal(0, L, (3, 3))
        B = rng.normal(0, L, (3, 3)) + rng.normal(0, 2 * L, 3)
    # body frames: each particle's triangle about its own centre, float32; the
    # centres up to 20 L away, so that coordinates (and M) dwarf the distance
    off = L * 10.0 ** rng.uniform(-0.3, 1.3)
    ca, cb = A.mean(axis=0) + rng.normal(0, off, 3), B.mean(axis=0) + rng.normal(0, off, 3)
    RA, RB = rot(rng.normal(size=4)), rot(rng.normal(size=4))
    far = rng.normal(0, 10.0 ** rng.uniform(0, 3), 3)
    XA = far + RA @ ca
    XB = far + RA @ cb
    RBw = RA @ RB  # B's body frame turned by RB relative to A's
    a32 = (A - ca).astype(np.float32)
    b32 = (RB.T @ (B - cb).T).T.astype(np.float32)
    return a32, b32, RA, XA, RBw, XB


def test_certificate_margin_holds_with_the_derived_terms():
    oracle.build()
    rng = np.random.default_rng(7)
    worst = 0.0
    n_cases = 0
    for k in range(2400):
        kind = k % 4
        L = 10.0 ** rng.uniform(-3, 2)
        a32, b32, RA, XA, RB, XB = _pair(rng, kind, L)
        # binary64 world vertices (the oracle's) and its distance
        WA = (RA @ a32.astype(np.float64).T).T + XA
        WB = (RB @ b32.astype(np.float64).T).T + XB
        d64, pa, pb = oracle.tri_dist(WA, WB)
        # exact A-frame geometry of the same float32 vertices, and its scale
        Yx = (RA.T @ ((RB @ b32.astype(np.float64).T).T + XB - XA).T).T
        for fused in (False, True):
            Rr, t = relative_pose32(RA, XA, RB, XB, fused)
            Y = np.array([move32(Rr, t, b) for b in b32])
            X = a32
            RAd = float(np.max(np.linalg.norm(a32.astype(np.float64), axis=1)))
            RBd = float(np.max(np.linalg.norm(b32.astype(np.float64), axis=1)))
            S = RAd + RBd + float(np.sqrt(f32(np.sum(t.astype(np.float32) ** 2))))
            E = ERR_REL32 * S
            m64 = ERR_REL64 * (S + np.linalg.norm(XA) + np.linalg.norm(XB))
            # directions: the exact closest points (A frame), rounded, and perturbed ones
            qa = RA.T @ (pa - XA)
            qb = RA.T @ (pb - XA)
            dirs = [(qb - qa).astype(np.float32)]
            for _ in range(2):
                dirs.append((qb - qa + rng.normal(0, 1e-3 * L + np.linalg.norm(qb - qa) * 0.1, 3)).astype(np.float32))
            for n in dirs:
                if not np.all(np.isfinite(n)) or float(np.dot(n, n)) < 1e-30:
                    continue
                c = certificate32(X, Y, n)
                assert c - E <= d64 + m64, (kind, fused, c, E, d64, m64)
                # the exact separation along n of the exact A-frame sets
                nd = n.astype(np.float64)
                sep = (min(Yx @ nd) - max(a32.astype(np.float64) @ nd)) / np.linalg.norm(nd)
                worst = max(worst, (c - sep) / (U * S))
                n_cases += 1
    print(f"\n{n_cases} certificates; worst error against the exact separation: {worst:.2f} u S (derived: 45)")
    assert n_cases > 8000
    assert worst <= 45.0
