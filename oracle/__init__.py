"""Python binding of the FP64 CPU oracle (``dem_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, obviously correct
definition of the contact-detection path (Noble & Weinzierl, Sections 2-5)
that the CUDA library is checked against.  Only ``tests/``, the smoke check
and the benchmark's CPU-baseline leg import this module; the product path
never does, and the two share no code.

Functions whose parity is not pinned by an independent check: none (every
function is pinned in tests/test_oracle_*.py).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libdem_oracle.so")
_SRC = [os.path.join(_HERE, "dem_oracle.c")]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC + [os.path.join(_HERE, "dem_oracle.h")])
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-o", tmp] + _SRC + ["-lm", "-lpthread"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp, fp, i64p, i32p, u8p = (C.POINTER(C.c_double), C.POINTER(C.c_float),
                                       C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_uint8))
            L.demo_pose.argtypes = [dp, C.c_int64, C.c_int64, C.c_double, dp, dp]
            L.demo_pose.restype = None
            L.demo_tri_dist.argtypes = [dp, dp, dp, dp]
            L.demo_tri_dist.restype = C.c_double
            L.demo_closest_pt_tri.argtypes = [dp, dp, dp]
            L.demo_closest_pt_tri.restype = C.c_double
            L.demo_seg_seg.argtypes = [dp, dp, dp, dp, dp, dp]
            L.demo_seg_seg.restype = C.c_double
            L.demo_broad_phase.argtypes = [dp, u8p, C.c_int64, i64p, fp, C.c_int64, i32p, C.c_int64]
            L.demo_broad_phase.restype = C.c_int64
            L.demo_broad_partners.argtypes = [dp, u8p, C.c_int64, i64p, fp, C.c_int64, C.c_int64, i32p,
                                              C.c_int64]
            L.demo_broad_partners.restype = C.c_int64
            L.demo_narrow_phase.argtypes = [dp, u8p, C.c_int64, i64p, fp, C.c_int64, i32p, C.c_int64,
                                            dp, dp, dp, dp, i32p, u8p, i32p, dp, C.c_int64, C.c_int]
            L.demo_narrow_phase.restype = C.c_int64
            L.demo_collision_times.argtypes = [dp, u8p, C.c_int64, i64p, fp, C.c_int64, i32p, C.c_int64,
                                               C.c_int, C.c_double, dp, u8p, i32p, i32p, C.c_int]
            L.demo_collision_times.restype = None
            L.demo_collision_times_narrowing.argtypes = [dp, u8p, C.c_int64, i64p, fp, C.c_int64, i32p,
                                                         C.c_int64, C.c_double, dp, u8p, i32p, i32p, C.c_int]
            L.demo_collision_times_narrowing.restype = None
            L.demo_clusters.argtypes = [C.c_int64, i32p, C.c_int64, u8p, i32p]
            L.demo_clusters.restype = C.c_int64
            L.demo_lts_sweep.argtypes = [dp, dp, u8p, C.c_int64, i64p, fp, C.c_int64, C.c_int, C.c_double,
                                         C.c_double, C.c_double, dp, C.c_int, C.c_int, i32p, C.c_int64, u8p, dp,
                                         i32p, u8p, dp, i64p, i64p, C.c_int, dp]
            L.demo_hose_meet.argtypes = [dp, dp, C.c_int64, C.c_int64, C.c_int64]
            L.demo_hose_meet.restype = C.c_int
            L.demo_lts_sweep.restype = C.c_int64
            _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())


# ---------------------------------------------------------------------------

def pose(state, p: int, t: float):
    state = _c(state, np.float64)
    R = np.zeros(9)
    X = np.zeros(3)
    lib().demo_pose(_p(state, C.c_double), state.shape[1], p, t, _p(R, C.c_double), _p(X, C.c_double))
    return R.reshape(3, 3), X


def tri_dist(A, B):
    A = _c(A, np.float64).reshape(9)
    B = _c(B, np.float64).reshape(9)
    pa, pb = np.zeros(3), np.zeros(3)
    d = lib().demo_tri_dist(_p(A, C.c_double), _p(B, C.c_double), _p(pa, C.c_double), _p(pb, C.c_double))
    return d, pa, pb


def closest_pt_tri(p, T):
    p = _c(p, np.float64).reshape(3)
    T = _c(T, np.float64).reshape(9)
    q = np.zeros(3)
    d2 = lib().demo_closest_pt_tri(_p(p, C.c_double), _p(T, C.c_double), _p(q, C.c_double))
    return d2, q


def seg_seg(p1, q1, p2, q2):
    a = [_c(x, np.float64).reshape(3) for x in (p1, q1, p2, q2)]
    c1, c2 = np.zeros(3), np.zeros(3)
    d2 = lib().demo_seg_seg(*[_p(x, C.c_double) for x in a], _p(c1, C.c_double), _p(c2, C.c_double))
    return d2, c1, c2


def _geometry(w):
    return (_c(w.state, np.float64), _c(w.is_static, np.uint8), _c(w.tri_off, np.int64),
            _c(w.tris, np.float32))


def broad_phase(w):
    """All candidate pairs (first, second), sorted; a static member is second."""
    state, st, off, tris = _geometry(w)
    n = state.shape[1]
    cap = 1024
    while True:
        pairs = np.zeros((cap, 2), np.int32)
        cnt = lib().demo_broad_phase(_p(state, C.c_double), _p(st, C.c_uint8), n, _p(off, C.c_int64),
                                     _p(tris, C.c_float), tris.shape[1], _p(pairs, C.c_int32), cap)
        if cnt <= cap:
            return pairs[:cnt].copy()
        cap = int(cnt)


def broad_partners(w, p):
    """The candidate pairs that contain particle p, by brute force over the others."""
    state, st, off, tris = _geometry(w)
    n = state.shape[1]
    cap = 256
    while True:
        pairs = np.zeros((cap, 2), np.int32)
        cnt = lib().demo_broad_partners(_p(state, C.c_double), _p(st, C.c_uint8), n, _p(off, C.c_int64),
                                        _p(tris, C.c_float), tris.shape[1], int(p), _p(pairs, C.c_int32), cap)
        if cnt <= cap:
            return pairs[:cnt].copy()
        cap = int(cnt)


def narrow_phase(w, pairs, t_eval=None, n_threads=None, cap=None):
    """Returns dict(dmin, pa, pb, tri_ab, flag, contacts (c,3) int32, geom (c,7))."""
    state, sta, off, tris = _geometry(w)
    pairs = _c(pairs, np.int32).reshape(-1, 2)
    m = len(pairs)
    te = None if t_eval is None else _c(t_eval, np.float64)
    dmin, pa, pb = np.zeros(m), np.zeros((m, 3)), np.zeros((m, 3))
    tri_ab = np.zeros((m, 2), np.int32)
    flag = np.zeros(m, np.uint8)
    cap = cap if cap is not None else max(1024, 64 * m)
    nt = n_threads or default_threads()
    while True:
        contacts = np.zeros((cap, 3), np.int32)
        geom = np.zeros((cap, 7))
        nc = lib().demo_narrow_phase(
            _p(state, C.c_double), _p(sta, C.c_uint8), state.shape[1], _p(off, C.c_int64), _p(tris, C.c_float),
            tris.shape[1],
            _p(pairs, C.c_int32), m, None if te is None else _p(te, C.c_double),
            _p(dmin, C.c_double), _p(pa, C.c_double), _p(pb, C.c_double), _p(tri_ab, C.c_int32),
            _p(flag, C.c_uint8), _p(contacts, C.c_int32), _p(geom, C.c_double), cap, nt)
        if nc <= cap:
            return dict(dmin=dmin, pa=pa, pb=pb, tri_ab=tri_ab, flag=flag,
                        contacts=contacts[:nc].copy(), geom=geom[:nc].copy())
        cap = int(nc)


def collision_times(w, pairs, K=None, tol=None, n_threads=None):
    """Returns dict(t_coll, status, tri_ab, n_evals)."""
    state, sta, off, tris = _geometry(w)
    pairs = _c(pairs, np.int32).reshape(-1, 2)
    m = len(pairs)
    K = w.K if K is None else K
    tol = w.tol if tol is None else tol
    t = np.zeros(m)
    status = np.zeros(m, np.uint8)
    tri_ab = np.zeros((m, 2), np.int32)
    ne = np.zeros(m, np.int32)
    lib().demo_collision_times(
        _p(state, C.c_double), _p(sta, C.c_uint8), state.shape[1], _p(off, C.c_int64), _p(tris, C.c_float),
        tris.shape[1],
        _p(pairs, C.c_int32), m, int(K), float(tol), _p(t, C.c_double), _p(status, C.c_uint8),
        _p(tri_ab, C.c_int32), _p(ne, C.c_int32), n_threads or default_threads())
    return dict(t_coll=t, status=status, tri_ab=tri_ab, n_evals=ne)


def collision_times_narrowing(w, pairs, tol=None, n_threads=None):
    """The paper's narrowing procedure; returns dict(t_coll, status, tri_ab, n_iter)."""
    state, sta, off, tris = _geometry(w)
    pairs = _c(pairs, np.int32).reshape(-1, 2)
    m = len(pairs)
    tol = w.tol if tol is None else tol
    t = np.zeros(m)
    status = np.zeros(m, np.uint8)
    tri_ab = np.zeros((m, 2), np.int32)
    it = np.zeros(m, np.int32)
    lib().demo_collision_times_narrowing(
        _p(state, C.c_double), _p(sta, C.c_uint8), state.shape[1], _p(off, C.c_int64), _p(tris, C.c_float),
        tris.shape[1], _p(pairs, C.c_int32), m, float(tol), _p(t, C.c_double), _p(status, C.c_uint8),
        _p(tri_ab, C.c_int32), _p(it, C.c_int32), n_threads or default_threads())
    return dict(t_coll=t, status=status, tri_ab=tri_ab, n_iter=it)


def clusters(n, edges, is_static=None):
    """Returns (id int32[n], n_clusters)."""
    edges = _c(edges, np.int32).reshape(-1, 2)
    st = _c(np.zeros(n, np.uint8) if is_static is None else is_static, np.uint8)
    ids = np.zeros(n, np.int32)
    c = lib().demo_clusters(n, _p(edges, C.c_int32), len(edges), _p(st, C.c_uint8), _p(ids, C.c_int32))
    return ids, int(c)


def hose_meet(cur, old, i, j):
    """Space-time hose test of moving particles i, j (cur, old: [17][n] float64)."""
    cur = _c(cur, np.float64)
    old = _c(old, np.float64)
    return bool(lib().demo_hose_meet(_p(cur, C.c_double), _p(old, C.c_double), cur.shape[1], int(i), int(j)))


def lts_sweep(w, old, dt_max, alpha=2.0, gravity=(0.0, 0.0, 0.0), zero_on_contact=True, hose=False,
              n_threads=None):
    """One local-time-stepping sweep; updates w.state (current snapshot) and
    ``old`` (old snapshot, same layout) in place.  Returns dict(pairs, status,
    t_coll, ids, active, t_global, rollbacks, rollbacks_before_old,
    consolidated), consolidated = the current snapshot after the
    consolidation (the state the collision times are evaluated on)."""
    assert w.state.flags["C_CONTIGUOUS"] and w.state.dtype == np.float64
    assert old.flags["C_CONTIGUOUS"] and old.dtype == np.float64 and old.shape == w.state.shape
    _, sta, off, tris = _geometry(w)
    n = w.n
    g = np.asarray(gravity, np.float64)
    ids = np.zeros(n, np.int32)
    active = np.zeros(n, np.uint8)
    tg = np.zeros(1)
    rb = np.zeros(1, np.int64)
    rbb = np.zeros(1, np.int64)
    cap = 1024
    while True:
        cur0, old0 = w.state.copy(), old.copy()
        pairs = np.zeros((cap, 2), np.int32)
        status = np.zeros(cap, np.uint8)
        tcol = np.zeros(cap)
        cons = np.zeros_like(w.state)
        m = lib().demo_lts_sweep(
            _p(w.state, C.c_double), _p(old, C.c_double), _p(sta, C.c_uint8), n, _p(off, C.c_int64),
            _p(tris, C.c_float), tris.shape[1], int(w.K), float(w.tol), float(dt_max), float(alpha),
            _p(g, C.c_double), int(bool(zero_on_contact)), int(bool(hose)), _p(pairs, C.c_int32), cap,
            _p(status, C.c_uint8),
            _p(tcol, C.c_double), _p(ids, C.c_int32), _p(active, C.c_uint8), _p(tg, C.c_double),
            _p(rb, C.c_int64), _p(rbb, C.c_int64), n_threads or default_threads(), _p(cons, C.c_double))
        if m <= cap:
            return dict(pairs=pairs[:m].copy(), status=status[:m].copy(), t_coll=tcol[:m].copy(), ids=ids,
                        active=active, t_global=float(tg[0]), rollbacks=int(rb[0]),
                        rollbacks_before_old=int(rbb[0]), consolidated=cons)
        # too many pairs for the outputs: undo and run again with room for all
        w.state[...] = cur0
        old[...] = old0
        cap = int(m)
