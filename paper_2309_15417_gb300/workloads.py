"""Seeded synthetic inputs for the contact-detection path.

This module only builds input data: triangle meshes in the body frame, particle
poses and velocities, and packings.  It contains none of the method's
arithmetic (no poses at a time, no distances, no predicates), so that both the
CPU oracle and the CUDA library can be fed from it without sharing code.

Data layout (the layout the C-ABI expects, see include/dem.h):

* ``state``: float64, shape ``(DEM_NFIELDS, n)``, field-major structure of
  arrays.  Field order: x y z | vx vy vz | qw qx qy qz | wx wy wz | t_cur | dt |
  eps | radius.  ``(x, y, z)`` is the centre of mass at ``t_cur``; ``q`` is the
  unit quaternion rotating body-frame vectors into the world frame at ``t_cur``;
  ``w`` is the angular velocity in the world frame; ``dt`` is the particle's
  own step size; ``eps`` its halo width; ``radius`` bounds the distance of every
  body-frame vertex from the body origin.
* ``tris``: float32, shape ``(3, T, 4)``: vertex slot (v0, v1, v2) x triangle
  x (x, y, z, 0).  The triangles of particle ``p`` are ``tri_off[p] ..
  tri_off[p+1]-1``.  Body-frame coordinates are float32 values, so the FP64
  paths promote them exactly.
* ``is_static``: uint8 per particle.

The particle model follows the paper's rigid particle with halo (Section 2.1)
and its triangulated geometry (Section 5, "Geometric model"); the packings are
stand-ins for the paper's scenes (Section 8), which are not available.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DEM_NFIELDS = 17
(F_X, F_Y, F_Z, F_VX, F_VY, F_VZ, F_QW, F_QX, F_QY, F_QZ,
 F_WX, F_WY, F_WZ, F_TCUR, F_DT, F_EPS, F_RADIUS) = range(DEM_NFIELDS)


@dataclass
class Workload:
    name: str
    state: np.ndarray          # (DEM_NFIELDS, n) float64
    is_static: np.ndarray      # (n,) uint8
    tri_off: np.ndarray        # (n+1,) int64
    tris: np.ndarray           # (3, T, 4) float32
    K: int = 8
    tol: float = 1e-3
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.state.shape[1])

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[1])

    def tri_counts(self) -> np.ndarray:
        return np.diff(self.tri_off)

    def subset(self, idx) -> "Workload":
        """Particles ``idx`` only (meshes re-packed), same parameters."""
        idx = np.asarray(idx, dtype=np.int64)
        counts = self.tri_counts()[idx]
        off = np.zeros(len(idx) + 1, np.int64)
        off[1:] = np.cumsum(counts)
        tris = np.zeros((3, int(off[-1]), 4), np.float32)
        for k, p in enumerate(idx):
            tris[:, off[k]:off[k + 1]] = self.tris[:, self.tri_off[p]:self.tri_off[p + 1]]
        return Workload(self.name + "-subset", np.ascontiguousarray(self.state[:, idx]),
                        np.ascontiguousarray(self.is_static[idx]), off, tris,
                        self.K, self.tol, dict(self.meta))


# --------------------------------------------------------------------------
# meshes (body frame)
# --------------------------------------------------------------------------

_GOLD = (1.0 + math.sqrt(5.0)) / 2.0
_ICO_V = np.array([
    (-1, _GOLD, 0), (1, _GOLD, 0), (-1, -_GOLD, 0), (1, -_GOLD, 0),
    (0, -1, _GOLD), (0, 1, _GOLD), (0, -1, -_GOLD), (0, 1, -_GOLD),
    (_GOLD, 0, -1), (_GOLD, 0, 1), (-_GOLD, 0, -1), (-_GOLD, 0, 1)], dtype=np.float64)
_ICO_F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
          (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
          (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
          (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]


def icosphere(subdiv: int, radius: float = 1.0) -> np.ndarray:
    """Triangle soup (T, 3, 3) float32 of an icosphere with 20*4**subdiv faces.

    Midpoint subdivision of the regular icosahedron, vertices pushed onto the
    sphere.  Children of a face are emitted consecutively (depth first), so
    neighbouring indices are neighbouring in space.  Vertices are rounded to
    float32 once; shared vertices are bit-identical.
    """
    verts = [v / np.linalg.norm(v) for v in _ICO_V]
    cache: dict = {}

    def mid(i, j):
        key = (min(i, j), max(i, j))
        if key not in cache:
            m = verts[i] + verts[j]
            verts.append(m / np.linalg.norm(m))
            cache[key] = len(verts) - 1
        return cache[key]

    out = []

    def rec(f, depth):
        a, b, c = f
        if depth == 0:
            out.append(f)
            return
        ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
        for g in ((a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)):
            rec(g, depth - 1)

    for f in _ICO_F:
        rec(f, subdiv)
    V = (np.array(verts) * radius).astype(np.float32)
    return V[np.array(out)]


def convex_hull_mesh(rng: np.random.Generator, n_points: int, radius: float = 1.0) -> np.ndarray:
    """Convex hull of ``n_points`` Gaussian points, scaled to max vertex radius
    ``radius``, as a float32 triangle soup with outward orientation."""
    from scipy.spatial import ConvexHull
    while True:
        P = rng.normal(size=(n_points, 3))
        P -= P.mean(axis=0)
        P *= radius / np.max(np.linalg.norm(P, axis=1))
        hull = ConvexHull(P)
        if len(hull.vertices) >= 4:
            break
    V = P.astype(np.float32)
    F = []
    for simplex, eq in zip(hull.simplices, hull.equations):
        a, b, c = simplex
        n = np.cross(P[b] - P[a], P[c] - P[a])
        if np.dot(n, eq[:3]) < 0:
            b, c = c, b
        F.append((a, b, c))
    # order faces by direction of their centroid (spatial coherence)
    F = np.array(F)
    cen = P[F].mean(axis=1)
    key = np.lexsort((np.arctan2(cen[:, 1], cen[:, 0]), np.round(cen[:, 2] * 4)))
    return V[F[key]]


def _morton2(ix: np.ndarray, iy: np.ndarray) -> np.ndarray:
    """Interleave the bits of two non-negative integers below 2^16 (Z-order)."""
    def spread(v):
        v = v.astype(np.uint64) & np.uint64(0xFFFF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x00FF00FF)
        v = (v | (v << np.uint64(4))) & np.uint64(0x0F0F0F0F)
        v = (v | (v << np.uint64(2))) & np.uint64(0x33333333)
        v = (v | (v << np.uint64(1))) & np.uint64(0x55555555)
        return v
    return spread(ix) | (spread(iy) << np.uint64(1))


def floor_grid(nq: int, size: float, z: float = 0.0) -> np.ndarray:
    """Static floor: an ``nq`` x ``nq`` grid of quads (2 triangles each),
    centred at the origin of its body frame, spanning ``size``.  Quads are in
    Z-order (Morton order) of their grid cell and the two triangles of a quad
    are adjacent, so every run of consecutive triangles covers a compact patch
    of the floor."""
    xs = np.linspace(-size / 2, size / 2, nq + 1)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    P = np.stack([X, Y, np.full_like(X, z)], axis=-1).astype(np.float32)
    ix, iy = np.meshgrid(np.arange(nq), np.arange(nq), indexing="ij")
    ix, iy = ix.ravel(), iy.ravel()
    order = np.argsort(_morton2(ix, iy), kind="stable")
    ix, iy = ix[order], iy[order]
    a, b, c, d = P[ix, iy], P[ix + 1, iy], P[ix + 1, iy + 1], P[ix, iy + 1]
    t1 = np.stack([a, b, c], axis=1)
    t2 = np.stack([a, c, d], axis=1)
    return np.stack([t1, t2], axis=1).reshape(-1, 3, 3)


def mesh_radius(soup: np.ndarray) -> float:
    """An upper bound on the distance of any vertex from the body origin."""
    r = float(np.max(np.linalg.norm(soup.reshape(-1, 3).astype(np.float64), axis=1)))
    return float(np.nextafter(np.nextafter(r, np.inf), np.inf))


# --------------------------------------------------------------------------
# poses
# --------------------------------------------------------------------------

def random_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random unit quaternions (Shoemake's method), columns (w,x,y,z)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.stack([b * np.cos(2 * np.pi * u3), a * np.sin(2 * np.pi * u2),
                  a * np.cos(2 * np.pi * u2), b * np.sin(2 * np.pi * u3)], axis=1)
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _assemble(name, meshes, mesh_of, pos, vel, quat, omega, t_cur, dt, eps, is_static=None,
              K=8, tol=1e-3, meta=None) -> Workload:
    n = len(mesh_of)
    mesh_of = np.asarray(mesh_of, np.int64).reshape(n)
    mesh_len = np.array([len(m) for m in meshes], np.int64)
    radii = np.array([mesh_radius(m) for m in meshes], np.float64)
    counts = mesh_len[mesh_of]
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum(counts)
    tris = np.zeros((3, int(off[-1]), 4), np.float32)
    M = np.concatenate([np.asarray(m, np.float32).reshape(-1, 3, 3) for m in meshes]) if meshes else \
        np.zeros((0, 3, 3), np.float32)
    mo = np.zeros(len(meshes) + 1, np.int64)
    mo[1:] = np.cumsum(mesh_len)
    chunk = 1 << 16  # particles per block of the copy (bounds temporaries)
    for p0 in range(0, n, chunk):
        p1 = min(n, p0 + chunk)
        c = counts[p0:p1]
        local = np.arange(int(off[p1] - off[p0]), dtype=np.int64) - np.repeat(off[p0:p1] - off[p0], c)
        g = np.repeat(mo[mesh_of[p0:p1]], c) + local
        for s in range(3):
            tris[s, off[p0]:off[p1], :3] = M[g, s, :]
    st = np.zeros((DEM_NFIELDS, n), np.float64)
    st[F_X:F_Z + 1] = np.asarray(pos, np.float64).T
    st[F_VX:F_VZ + 1] = np.asarray(vel, np.float64).T
    st[F_QW:F_QZ + 1] = np.asarray(quat, np.float64).T
    st[F_WX:F_WZ + 1] = np.asarray(omega, np.float64).T
    st[F_TCUR] = t_cur
    st[F_DT] = dt
    st[F_EPS] = eps
    st[F_RADIUS] = radii[mesh_of] if n else 0.0
    if is_static is None:
        is_static = np.zeros(n, np.uint8)
    return Workload(name, st, np.asarray(is_static, np.uint8), off, tris, K, tol, meta or {})


def _rsa(rng, n, lo, hi, min_dist, existing=None, max_tries=200000):
    """Random sequential addition of ``n`` centres in the box [lo, hi]^3."""
    pts = [] if existing is None else list(existing)
    tries = 0
    while len(pts) < n + (0 if existing is None else len(existing)):
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random sequential addition did not converge")
        c = rng.uniform(lo, hi, size=3)
        if pts:
            d = np.linalg.norm(np.asarray(pts) - c, axis=1)
            if np.min(d) < min_dist:
                continue
        pts.append(c)
    return np.asarray(pts[0 if existing is None else len(existing):])


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------

def small_icospheres(seed: int = 0, n: int = 64, inject: bool = True) -> Workload:
    """64 icospheres (subdivision 1, 80 triangles, radius 1) in a 12^3 box,
    non-overlapping, uniform random rotations, v ~ N(0,1), w ~ N(0,0.5),
    dt = 1e-3, halo eps = 0.05, all FP64.

    With ``inject`` the first six particles form three pairs placed along the
    direction of an icosahedron vertex, identity rotation and no spin, so that
    the nearest features are two vertex tips: pair (0,1) already overlaps
    (collision-time status 1), pair (2,3) approaches head on and closes its gap
    to the halo sum half way through the step (status 2), pair (4,5) starts
    just outside the halo sum and slides sideways (status 0).
    """
    rng = np.random.default_rng(seed)
    r, eps, dt = 1.0, 0.05, 1e-3
    mesh = icosphere(1, r)
    R = mesh_radius(mesh)
    pos = np.zeros((n, 3))
    vel = rng.normal(0.0, 1.0, size=(n, 3))
    omega = rng.normal(0.0, 0.5, size=(n, 3))
    quat = random_quaternions(rng, n)
    k0 = 0
    if inject:
        u = mesh[0, 0].astype(np.float64)
        u /= np.linalg.norm(u)
        vrel = 1.0
        side = np.cross(u, [0.0, 0.0, 1.0])
        side /= np.linalg.norm(side)
        gaps = [2 * eps - 0.03, 2 * eps + 0.5 * vrel * dt, 2 * eps + 0.3 * vrel * dt]
        dirs = [u, u, side]
        anchors = [np.array([1.5, 1.5, 1.5]), np.array([1.5, 1.5, 10.0]), np.array([10.0, 1.5, 1.5])]
        for k, (g, a, dv) in enumerate(zip(gaps, anchors, dirs)):
            i, j = 2 * k, 2 * k + 1
            D = 2 * R + g
            pos[i] = a - 0.5 * D * u
            pos[j] = a + 0.5 * D * u
            vel[i] = +0.5 * vrel * dv
            vel[j] = -0.5 * vrel * dv
            quat[i] = quat[j] = (1.0, 0.0, 0.0, 0.0)
            omega[i] = omega[j] = 0.0
        k0 = 6
    pos[k0:] = _rsa(rng, n - k0, 0.0, 12.0, 2 * r + 2 * eps, existing=pos[:k0] if k0 else None)
    return _assemble("icospheres-64-s1", [mesh], [0] * n, pos, vel, quat, omega, 0.0, dt, eps,
                     meta=dict(seed=seed, inject=inject, box=12.0))


def dense_packing(seed: int = 0, nside: int = 10, phi: float = 0.5, jitter: float = 0.1,
                  subdiv: int = 2, eps: float = 0.02, dt: float = 1e-4,
                  vsig: float = 0.2, wsig: float = 0.2) -> Workload:
    """Dense packing: nside^3 icospheres (subdivision 2, 320 triangles, radius 1)
    on a jittered simple-cubic lattice at volume fraction ``phi`` (spacing
    (4 pi r^3 / 3 / phi)^(1/3)), jitter uniform in +-``jitter`` per axis,
    uniform random rotations, v ~ N(0, vsig), w ~ N(0, wsig), dt = 1e-4,
    eps = 0.02.  Some neighbours overlap (intersecting meshes)."""
    rng = np.random.default_rng(seed)
    r = 1.0
    mesh = icosphere(subdiv, r)
    a = (4.0 * math.pi * r ** 3 / 3.0 / phi) ** (1.0 / 3.0)
    g = np.arange(nside) * a
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    n = len(P)
    P = P + rng.uniform(-jitter, jitter, size=P.shape)
    vel = rng.normal(0.0, vsig, size=(n, 3))
    omega = rng.normal(0.0, wsig, size=(n, 3))
    quat = random_quaternions(rng, n)
    return _assemble(f"dense-packing-{n}-s{subdiv}", [mesh], [0] * n, P, vel, quat, omega,
                     0.0, dt, eps, meta=dict(seed=seed, spacing=a, phi=phi))


def injected_head_on(gap: float, vrel: float, eps: float = 0.05, dt: float = 1e-3,
                     subdiv: int = 1) -> Workload:
    """Two icospheres, identity rotation, no spin, approaching head on along an
    icosahedron-vertex direction; the nearest features are the two vertex tips
    at distance ``gap`` at t=0, closing at speed ``vrel``."""
    mesh = icosphere(subdiv, 1.0)
    R = mesh_radius(mesh)
    u = mesh[0, 0].astype(np.float64)
    u /= np.linalg.norm(u)
    D = 2 * R + gap
    pos = np.stack([-0.5 * D * u, 0.5 * D * u])
    vel = np.stack([0.5 * vrel * u, -0.5 * vrel * u])
    quat = np.array([[1.0, 0, 0, 0], [1.0, 0, 0, 0]])
    return _assemble("head-on", [mesh], [0, 0], pos, vel, quat, np.zeros((2, 3)), 0.0, dt, eps,
                     meta=dict(gap=gap, vrel=vrel, u=u.tolist()))


def single_triangles(tri_a: np.ndarray, tri_b: np.ndarray, pos_a=(0, 0, 0), pos_b=(0, 0, 0),
                     vel_a=(0, 0, 0), vel_b=(0, 0, 0), quat_a=(1, 0, 0, 0), quat_b=(1, 0, 0, 0),
                     omega_a=(0, 0, 0), omega_b=(0, 0, 0), eps=0.01, dt=1e-3) -> Workload:
    """Two one-triangle "particles" (body-frame triangles given as (3,3))."""
    ma = np.asarray(tri_a, np.float32).reshape(1, 3, 3)
    mb = np.asarray(tri_b, np.float32).reshape(1, 3, 3)
    return _assemble("two-triangles", [ma, mb], [0, 1], [pos_a, pos_b], [vel_a, vel_b],
                     [quat_a, quat_b], [omega_a, omega_b], 0.0, dt, eps)


def uneven_meshes(seed: int = 0, n: int = 10000, box: float = 200.0, n_clusters: int = 10,
                  frac_clustered: float = 0.6, sigma: float = 15.0, dt: float = 1e-3) -> Workload:
    """Batched uneven meshes: one third each icospheres with 80 / 320 / 1280
    triangles and convex hulls of 20-200 Gaussian points; radii log-uniform in
    [0.5, 4]; 60% of the particles in Gaussian clusters, the rest free in a
    box^3; v ~ N(0,1), w ~ N(0,0.5); eps = 0.02 * radius."""
    rng = np.random.default_rng(seed)
    kind = rng.integers(0, 4, size=n)
    radius = np.exp(rng.uniform(np.log(0.5), np.log(4.0), size=n))
    meshes, mesh_of = [], []
    unit = [icosphere(1), icosphere(2), icosphere(3)]
    for p in range(n):
        if kind[p] < 3:
            meshes.append((unit[kind[p]] * np.float32(radius[p])).astype(np.float32))
        else:
            meshes.append(convex_hull_mesh(rng, int(rng.integers(20, 201)), radius[p]))
        mesh_of.append(p)
    centres = rng.uniform(0, box, size=(n_clusters, 3))
    order = rng.permutation(n)
    pos = np.zeros((n, 3))
    n_cl = int(frac_clustered * n)
    # overlap test against the placed spheres through a grid hash (cell =
    # largest diameter, so every sphere that can overlap is in the 27 cells)
    h = 2.0 * float(radius.max())
    grid: dict = {}
    for rank, p in enumerate(order):
        for _ in range(1000):
            if rank < n_cl:
                c = centres[rank % n_clusters] + rng.normal(0, sigma, size=3)
            else:
                c = rng.uniform(0, box, size=3)
            k = np.floor(c / h).astype(int)
            clash = False
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        for q in grid.get((k[0] + dx, k[1] + dy, k[2] + dz), ()):
                            if np.linalg.norm(pos[q] - c) - radius[q] < radius[p]:
                                clash = True
                                break
                        if clash:
                            break
                    if clash:
                        break
                if clash:
                    break
            if clash:
                continue
            break
        pos[p] = c
        k = np.floor(c / h).astype(int)
        grid.setdefault((k[0], k[1], k[2]), []).append(p)
    vel = rng.normal(0, 1.0, size=(n, 3))
    omega = rng.normal(0, 0.5, size=(n, 3))
    quat = random_quaternions(rng, n)
    return _assemble(f"uneven-{n}", meshes, mesh_of, pos, vel, quat, omega, 0.0, dt,
                     0.02 * radius, meta=dict(seed=seed))


def lts_mixed_steps(seed: int = 0, n: int = 100_000, blob_frac: float = 0.2, n_blobs: int = 10,
                    phi_blob: float = 0.55, phi_free: float = 0.02, jitter: float = 0.1,
                    dt_range=(1e-5, 1e-2), eps: float = 0.02) -> Workload:
    """Local time stepping with mixed step sizes: icospheres (320 triangles,
    radius 1); ``blob_frac`` of them in dense blobs on an FCC lattice at volume
    fraction ``phi_blob`` (nearest-neighbour spacing 2 r (0.7405/phi)^(1/3),
    jitter +-``jitter``), the rest free on a jittered simple-cubic lattice at
    volume fraction ``phi_free`` (non-overlapping by construction); each
    particle's step log-uniform in ``dt_range``; v ~ N(0,1), w ~ N(0,0.5)."""
    rng = np.random.default_rng(seed)
    r = 1.0
    mesh = icosphere(2, r)
    n_blob = int(round(blob_frac * n))
    n_free = n - n_blob
    # free particles: simple-cubic lattice with large jitter
    s_free = (4.0 * math.pi * r ** 3 / 3.0 / phi_free) ** (1.0 / 3.0)
    side = int(math.ceil(n_free ** (1.0 / 3.0)))
    g = np.arange(side) * s_free
    F = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)[:n_free]
    amp = max(0.0, 0.5 * (s_free - 2 * r) - 0.05)
    F = F + rng.uniform(-amp, amp, size=F.shape)
    # blobs: FCC, placed along a line outside the free lattice
    d_nn = 2 * r * (0.7405 / phi_blob) ** (1.0 / 3.0)
    a = d_nn * math.sqrt(2.0)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) * a
    per = int(math.ceil(n_blob / n_blobs))
    cells = int(math.ceil((per / 4.0) ** (1.0 / 3.0)))
    c = np.arange(cells) * a
    C3 = np.stack(np.meshgrid(c, c, c, indexing="ij"), axis=-1).reshape(-1, 3)
    one = (C3[:, None, :] + basis[None, :, :]).reshape(-1, 3)[:per]
    blobs = []
    for b in range(n_blobs):
        off = np.array([-(cells * a + 20.0) * (b + 1), 0.0, 0.0])
        blobs.append(one + off)
    B = np.concatenate(blobs)[:n_blob]
    B = B + rng.uniform(-jitter, jitter, size=B.shape)
    pos = np.concatenate([B, F])
    vel = rng.normal(0.0, 1.0, size=(n, 3))
    omega = rng.normal(0.0, 0.5, size=(n, 3))
    quat = random_quaternions(rng, n)
    dt = np.exp(rng.uniform(np.log(dt_range[0]), np.log(dt_range[1]), size=n))
    return _assemble(f"lts-{n}", [mesh], [0] * n, pos, vel, quat, omega, 0.0, dt, eps,
                     meta=dict(seed=seed, n_blob=n_blob, spacing_free=s_free, d_nn=d_nn))


def floor_scene(seed: int = 0, n_side: int = 6, nq: int = 40, size: float = 24.0, eps: float = 0.02,
                dt: float = 1e-3) -> Workload:
    """Static geometry: particle 0 is a static floor (``nq`` x ``nq`` quads,
    Morton order, z = 0, more than one 320-triangle tile), the particle in the
    middle of the index range is a static icosphere post standing on it, and
    the others are moving icospheres (80 or 320 triangles, radius 1) over an
    ``n_side`` x ``n_side`` grid of the floor, one of four kinds at random:
    resting within the halo sum of the floor, falling onto it during the step,
    sliding just above it, or clear of it (well above the floor's box but inside
    its bounding sphere).  Random rotations, w ~ N(0, 0.5)."""
    rng = np.random.default_rng(seed)
    floor = floor_grid(nq, size)
    small, big = icosphere(1), icosphere(2)
    R = max(mesh_radius(small), mesh_radius(big))
    spacing = size / (n_side + 1)
    g = (np.arange(n_side) - (n_side - 1) / 2) * spacing
    XY = np.stack(np.meshgrid(g, g, indexing="ij"), axis=-1).reshape(-1, 2)
    m = len(XY)
    kind = rng.integers(0, 4, size=m)
    z = np.empty(m)
    vel = rng.normal(0.0, 0.2, size=(m, 3))
    eps_pair = 2 * eps
    for q in range(m):
        if kind[q] == 0:    # resting: lowest point within the halo sum
            z[q] = R + rng.uniform(0.1, 0.9) * eps_pair
        elif kind[q] == 1:  # falling: reaches the floor part way through the step
            gap = rng.uniform(0.05, 0.3)
            z[q] = R + eps_pair + gap
            vel[q, 2] = -gap / (dt * rng.uniform(0.2, 0.9))
        elif kind[q] == 2:  # sliding just above the halo sum
            z[q] = R + eps_pair + rng.uniform(0.002, 0.02)
            vel[q, :2] = rng.normal(0.0, 20.0, size=2)
            vel[q, 2] = 0.0
        else:               # clear: far above the box, inside the bounding sphere
            z[q] = R + rng.uniform(3.0, 8.0)
    pos = np.concatenate([XY, z[:, None]], axis=1)
    post_at = (m + 2) // 2
    # particle list: floor, first half of the spheres, post, second half
    n = m + 2
    mesh_of = np.empty(n, np.int64)
    mesh_of[0] = 0
    kinds_mesh = rng.integers(1, 3, size=m)
    others = [p for p in range(n) if p not in (0, post_at)]
    mesh_of[others] = kinds_mesh
    mesh_of[post_at] = 2
    P = np.zeros((n, 3))
    V = np.zeros((n, 3))
    W = np.zeros((n, 3))
    Q = np.zeros((n, 4))
    Q[:, 0] = 1.0
    P[others] = pos
    V[others] = vel
    W[others] = rng.normal(0.0, 0.5, size=(m, 3))
    Q[others] = random_quaternions(rng, m)
    # the post sits on the floor between two grid points, touching its neighbours' halos
    P[post_at] = (0.5 * spacing, 0.5 * spacing, R)
    st = np.zeros(n, np.uint8)
    st[0] = st[post_at] = 1
    return _assemble(f"floor-scene-{n}", [floor, small, big], mesh_of, P, V, Q, W, 0.0, dt, eps,
                     is_static=st, meta=dict(seed=seed, kind=kind.tolist(), post=post_at))


def settling_column(seed: int = 0, nside: int = 100, spacing: float = 2.2, jitter: float = 0.1,
                    nq: int = None, eps: float = 0.01, dt: float = 1e-3, vsig: float = 0.1,
                    wsig: float = 0.1, lift: float = 0.005) -> Workload:
    """Throughput scale: a settling column of nside^3 icospheres of radius 1,
    half with 80 and half with 320 triangles (types shuffled), on a simple-cubic
    lattice of spacing ``spacing``, jitter uniform in +-``jitter`` per axis
    (horizontal only in the bottom layer, whose lowest points stay ``lift``
    above the floor), over a static floor of ``nq`` x ``nq`` quads (Morton
    order) spanning the column's footprint; by default nq keeps the quads of
    the full column's 316 x 316 floor (nq = 316 for nside = 100, smaller
    columns get a proportionally smaller floor).  The floor is the last
    particle.
    v ~ N(0, vsig), w ~ N(0, wsig), dt = 1e-3, eps = 0.01.  ``meta['gravity']``
    is the acceleration a stepping loop applies between steps (free flight
    within a step is at constant velocity)."""
    rng = np.random.default_rng(seed)
    small, big = icosphere(1), icosphere(2)
    R = max(mesh_radius(small), mesh_radius(big))
    n = nside ** 3
    g = np.arange(nside) * spacing
    IX, IY, IZ = np.meshgrid(g, g, g, indexing="ij")
    P = np.stack([IX, IY, IZ], axis=-1).reshape(-1, 3)
    J = rng.uniform(-jitter, jitter, size=P.shape)
    bottom = P[:, 2] == 0.0
    J[bottom, 2] = 0.0
    P = P + J
    P[:, 2] += R + lift
    foot = (nside - 1) * spacing
    size = foot + 2 * (R + 2 * jitter + 1.0)
    if nq is None:
        nq = max(8, int(round(316 * size / (99 * spacing + 2 * (R + 2 * jitter + 1.0)))))
    floor = floor_grid(nq, size)
    types = rng.permutation(np.arange(n) % 2) + 1
    mesh_of = np.concatenate([types, [0]])
    pos = np.concatenate([P, [[foot / 2, foot / 2, 0.0]]])
    vel = np.concatenate([rng.normal(0.0, vsig, size=(n, 3)), np.zeros((1, 3))])
    omega = np.concatenate([rng.normal(0.0, wsig, size=(n, 3)), np.zeros((1, 3))])
    quat = np.concatenate([random_quaternions(rng, n), [[1.0, 0.0, 0.0, 0.0]]])
    st = np.zeros(n + 1, np.uint8)
    st[n] = 1
    return _assemble(f"settling-column-{n}", [floor, small, big], mesh_of, pos, vel, quat, omega, 0.0, dt,
                     eps, is_static=st, meta=dict(seed=seed, gravity=(0.0, 0.0, -9.81), floor=n))
