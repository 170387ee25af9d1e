"""The oracle's result for a particle against a large static floor, computed
on the floor triangles that can change it (shared by the full-size parity
test of the settling column and its CPU check)."""
import numpy as np

import oracle
from paper_2309_15417_gb300 import workloads as W


def _rot(q):
    w_, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w_ * z), 2 * (x * z + w_ * y)],
                     [2 * (x * y + w_ * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w_ * x)],
                     [2 * (x * z - w_ * y), 2 * (y * z + w_ * x), 1 - 2 * (x * x + y * y)]])


def floor_pair_oracle(w, p, floor):
    """The oracle's narrow phase and collision times of the pair (p, floor) on
    a reduced floor that holds every floor triangle able to change them:
    with U an upper bound on the pair minimum at the start (the oracle's
    minimum over the 64 floor triangles nearest to p), a floor triangle whose
    bounding sphere stays farther than R_p + max(U, eps_pair + delta) from
    p's centre (delta = the largest vertex motion over the pair interval) can
    be neither the closest triangle nor within eps_pair at any time of the
    interval.  The floor keeps its pose; kept triangles keep their order, and
    the outputs are mapped back to the full floor's triangle indices."""
    off = w.tri_off
    ft = w.tris[:, off[floor]:off[floor + 1], :3].astype(np.float64)  # (3, T, 3) body frame
    Rf = _rot(w.state[W.F_QW:W.F_QZ + 1, floor])
    Xf = w.state[W.F_X:W.F_Z + 1, floor]
    world = np.einsum("ab,stb->sta", Rf, ft) + Xf
    cen = world.mean(axis=0)
    rad = np.linalg.norm(world - cen[None], axis=2).max(axis=0)
    xp = w.state[W.F_X:W.F_Z + 1, p]
    Rp = w.state[W.F_RADIUS, p]
    dist = np.linalg.norm(cen - xp, axis=1) - rad

    def reduced(keep):
        keep = np.sort(keep)
        sub = w.subset([p, floor])
        sub.tris = np.ascontiguousarray(w.tris[:, off[floor] + keep])
        sub.tris = np.concatenate([w.tris[:, off[p]:off[p + 1]], sub.tris], axis=1)
        sub.tri_off = np.array([0, off[p + 1] - off[p], off[p + 1] - off[p] + len(keep)], np.int64)
        return sub, keep

    sub, near = reduced(np.argsort(dist)[:64])
    U = float(oracle.narrow_phase(sub, np.array([[0, 1]], np.int32))["dmin"][0])
    v = np.linalg.norm(w.state[W.F_VX:W.F_VZ + 1, p])
    om = np.linalg.norm(w.state[W.F_WX:W.F_WZ + 1, p])
    delta = (v + om * Rp) * w.state[W.F_DT, p] * (1.0 + 1e-9)
    eps = w.state[W.F_EPS, p] + w.state[W.F_EPS, floor]
    sub, keep = reduced(np.nonzero(dist <= Rp + max(U, eps + delta) + 1e-9)[0])
    pr = np.array([[0, 1]], np.int32)
    on, oc = oracle.narrow_phase(sub, pr), oracle.collision_times(sub, pr)
    for d, key in ((on, "tri_ab"), (oc, "tri_ab")):
        if d[key][0, 1] >= 0:
            d[key][0, 1] = keep[d[key][0, 1]]
    if len(on["contacts"]):
        on["contacts"][:, 2] = keep[on["contacts"][:, 2]]
    return on, oc, len(keep)
