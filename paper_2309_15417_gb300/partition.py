"""Spatial partition of one detection step over several ranks (one GPU each).

The paper runs on one shared-memory node and names distributed memory as
future work (Section 1 and the conclusion); this module is the build's own
decomposition of the contact-detection step, host logic around the per-rank
compute:

* Space is cut into slabs along x at quantiles of the particles' swept-sphere
  centres m = x + v dt / 2 (equal particle counts per slab).  Rank r owns the
  moving particles whose m_x falls in its slab.
* Ghosts: every moving particle whose m_x lies within 2 rho_max of the slab
  (rho = R + eps + |v| dt / 2 the swept radius, rho_max over all moving
  particles) -- the candidate predicate |m_i - m_j| <= rho_i + rho_j can only
  hold for partners that close.  Static particles (floors, walls) are held by
  every rank.
* Each rank runs the broad phase on its local set (owned + ghosts + statics)
  and keeps the pairs it owns: a pair belongs to the owner of its first
  (moving) member.  The pairs of all ranks are then exactly the global
  candidate set, each once.  Narrow phase and collision times run on the
  owned pairs only (no exchange: every pair's particles are local).
* Clusters (connected components of the candidate graph): every rank keeps a
  label per global particle, starting at the particle's own index; each round
  takes, per local component of the rank's owned pairs, the smallest label of
  its members, then an all-reduce (minimum) over ranks; rounds repeat until no
  label changes.  The fixed point labels every particle with the smallest
  index of its global component (statics -1), the single-domain definition.

The per-rank compute is injected (an object with ``broad_phase``,
``narrow_phase`` and ``collision_times`` methods taking a workload and local
pairs); with one GPU per rank it is :class:`GpuCompute` over the CUDA
library.  The only collective is the label all-reduce (``allreduce_min``, a
callable: torch.distributed over NCCL between GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import workloads as W


@dataclass
class Slab:
    rank: int
    world: int
    lo: float             # slab bounds on m_x (lo inclusive, hi exclusive; outer slabs unbounded)
    hi: float
    owned: np.ndarray     # global indices of the moving particles this rank owns
    local: np.ndarray     # global indices of its local set (owned, ghosts, statics), sorted
    reach: float          # ghost reach 2 rho_max


def swept_spheres(state: np.ndarray):
    """Centre x (m_x) and radius of every particle's swept sphere over its own
    step (the broad phase's predicate, binary64)."""
    hdt = state[W.F_DT] * 0.5
    mx = state[W.F_X] + state[W.F_VX] * hdt
    v = np.sqrt(state[W.F_VX] ** 2 + state[W.F_VY] ** 2 + state[W.F_VZ] ** 2)
    rho = (state[W.F_RADIUS] + state[W.F_EPS]) + v * hdt
    return mx, rho


def make_slab(w: W.Workload, rank: int, world: int) -> Slab:
    mx, rho = swept_spheres(w.state)
    moving = np.nonzero(w.is_static == 0)[0]
    static = np.nonzero(w.is_static != 0)[0]
    reach = 2.0 * float(rho[moving].max()) if len(moving) else 0.0
    # slab boundaries: quantiles of m_x over moving particles
    qs = np.sort(mx[moving])
    cut = [-np.inf] + [float(qs[min(len(qs) - 1, (len(qs) * k) // world)]) for k in range(1, world)] + [np.inf]
    lo, hi = cut[rank], cut[rank + 1]
    own = moving[(mx[moving] >= lo) & (mx[moving] < hi)]
    ghost = moving[(mx[moving] >= lo - reach) & (mx[moving] < hi + reach)]
    local = np.unique(np.concatenate([own, ghost, static]))
    return Slab(rank, world, lo, hi, own, local, reach)


def owned_pairs(slab: Slab, local_pairs: np.ndarray) -> np.ndarray:
    """Global pairs of the local broad phase that this rank owns (first member
    owned), in (first, second) order."""
    g = slab.local[local_pairs.astype(np.int64)] if len(local_pairs) else np.zeros((0, 2), np.int64)
    if not len(g):
        return g.astype(np.int32).reshape(0, 2)
    keep = np.isin(g[:, 0], slab.owned)
    g = g[keep]
    order = np.lexsort((g[:, 1], g[:, 0]))
    return g[order].astype(np.int32)


def local_components(n: int, is_static: np.ndarray, pairs: np.ndarray) -> np.ndarray:
    """Connected components of this rank's owned pairs (global indices):
    comp[i] = smallest index in i's local component (i itself if it has no
    local edge).  Edges with a static endpoint are ignored.  Edge relaxation
    to a fixed point (host arithmetic; any exact components routine will do,
    e.g. dem_clusters on the rank's GPU)."""
    comp = np.arange(n, dtype=np.int64)
    st = is_static.astype(bool)
    if not len(pairs):
        return comp
    edges = pairs[~(st[pairs[:, 0]] | st[pairs[:, 1]])].astype(np.int64)
    a, b = edges[:, 0], edges[:, 1]
    while len(a):
        m = np.minimum(comp[a], comp[b])
        before = comp.copy()
        np.minimum.at(comp, a, m)
        np.minimum.at(comp, b, m)
        comp = comp[comp]  # pointer jumping: labels are indices of smaller members
        if np.array_equal(before, comp):
            break
    return comp


def merge_clusters(n: int, is_static: np.ndarray, pairs: np.ndarray, allreduce_min, comp=None,
                   max_rounds: int = 1 << 20):
    """Connected components over ranks.  Each round takes, for every local
    component of this rank's owned pairs, the smallest label of its members,
    then the all-reduce (minimum) over ranks; rounds repeat until no label
    changes.  Returns (ids, rounds): ids[i] = smallest particle index of i's
    global component, -1 for static particles."""
    if comp is None:
        comp = local_components(n, is_static, pairs)
    lab = np.arange(n, dtype=np.int64)
    rounds = 0
    while rounds < max_rounds:
        rounds += 1
        cmin = np.full(n, np.iinfo(np.int64).max, dtype=np.int64)
        np.minimum.at(cmin, comp, lab)
        new = allreduce_min(cmin[comp])
        if np.array_equal(new, lab):
            break
        lab = new
    ids = lab.copy()
    ids[is_static.astype(bool)] = -1
    return ids.astype(np.int32), rounds


def detect_step(w: W.Workload, rank: int, world: int, compute, allreduce_min):
    """One detection step on this rank: its slab's candidate pairs (global
    indices, the pairs it owns), their narrow phase and collision times, and
    the global cluster ids.  Returns a dict."""
    slab = make_slab(w, rank, world)
    lw = w.subset(slab.local)
    lp = compute.broad_phase(lw)
    pairs = owned_pairs(slab, lp)
    # the owned pairs in the local numbering, for the pair computations
    pos = {int(g): k for k, g in enumerate(slab.local)}
    loc = np.array([[pos[int(i)], pos[int(j)]] for i, j in pairs], np.int32).reshape(-1, 2)
    nar = compute.narrow_phase(lw, loc)
    ct = compute.collision_times(lw, loc)
    ids, rounds = merge_clusters(w.n, w.is_static, pairs, allreduce_min)
    return dict(slab=slab, pairs=pairs, narrow=nar, ctime=ct, ids=ids, rounds=rounds)


class GpuCompute:
    """Per-rank compute over the CUDA library (one device per rank)."""

    def __init__(self, device, precision=0, max_pairs=1 << 20, max_contacts=1 << 20):
        from . import dem
        self.dem = dem
        self.device = device
        self.precision = precision
        self.max_pairs = max_pairs
        self.max_contacts = max_contacts

    def _ctx(self, w):
        return self.dem.Context(K=w.K, tol=w.tol, precision=self.precision, max_particles=max(w.n, 16),
                                max_pairs=self.max_pairs, max_contacts=self.max_contacts,
                                max_triangles=max(w.n_tris, 1), device=self.device)

    def broad_phase(self, w):
        c = self._ctx(w)
        sc = self.dem.Scene.from_workload(w, device=self.device)
        c.build_candidates(sc)
        c.check()
        m = int(c.n_pairs.item())
        out = c.pairs[:m].cpu().numpy().copy()
        c.close()
        return out

    def narrow_phase(self, w, pairs):
        import torch
        c = self._ctx(w)
        sc = self.dem.Scene.from_workload(w, device=self.device)
        gp = torch.from_numpy(np.ascontiguousarray(pairs)).to(self.device)
        c.narrow_phase(sc, pairs=gp)
        c.check()
        m = len(pairs)
        nc = int(c.n_contacts.item())
        out = dict(dmin=c.dmin[:m].cpu().numpy(), flag=c.flag[:m].cpu().numpy(), tri_ab=c.tri_ab[:m].cpu().numpy(),
                   contacts=c.contacts[:nc].cpu().numpy())
        c.close()
        return out

    def collision_times(self, w, pairs):
        import torch
        c = self._ctx(w)
        sc = self.dem.Scene.from_workload(w, device=self.device)
        gp = torch.from_numpy(np.ascontiguousarray(pairs)).to(self.device)
        c.collision_times(sc, pairs=gp)
        c.check()
        m = len(pairs)
        out = dict(status=c.status[:m].cpu().numpy(), t_coll=c.t_coll[:m].cpu().numpy(),
                   tri_ab=c.ct_ab[:m].cpu().numpy())
        c.close()
        return out
