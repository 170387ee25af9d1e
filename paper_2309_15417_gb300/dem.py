"""Thin Python binding of the C-ABI in include/dem.h (ctypes).

Argument marshalling only: every step of the contact-detection path runs in
the CUDA library ``libdem.so``.  Arrays are torch tensors on the CUDA device
(torch provides device memory and streams); their data pointers are passed
through unchanged.  There is no CPU fallback: if the library cannot be built
or loaded, :func:`load` raises.

Function names follow the C-ABI: :func:`dem_create`, :func:`dem_build_candidates`,
:func:`dem_narrow_phase`, :func:`dem_collision_times`, :func:`dem_clusters`,
:func:`dem_check`, :func:`dem_get_stats`.  :class:`Context` and
:class:`Scene` wrap them for convenience (capacities, output allocation).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

DEM_NFIELDS = 17
DEM_PREC_FP32_FIXUP = 0
DEM_PREC_FP64 = 1

DEM_OK, DEM_ERR_ARG, DEM_ERR_CAPACITY, DEM_ERR_CUDA, DEM_ERR_NONFINITE, DEM_ERR_TIMEOUT, DEM_ERR_INDEX = \
    0, -1, -2, -3, -4, -5, -6
STATUS = {0: "DEM_OK", -1: "DEM_ERR_ARG", -2: "DEM_ERR_CAPACITY", -3: "DEM_ERR_CUDA", -4: "DEM_ERR_NONFINITE",
          -5: "DEM_ERR_TIMEOUT", -6: "DEM_ERR_INDEX"}

# every symbol include/dem.h declares
EXPORTS = ["dem_create", "dem_destroy", "dem_last_error", "dem_build_candidates", "dem_narrow_phase",
           "dem_collision_times", "dem_detect", "dem_clusters", "dem_lts_sweep", "dem_check", "dem_get_stats",
           "dem_build_candidates_noalloc", "dem_noalloc_check", "dem_set_wait_polls", "dem_trace",
           "dem_trace_read", "dem_autotune", "dem_get_tuning", "dem_set_tuning",
           # include/dem_probe.h (measurement support)
           "dem_probe_fma_peak", "dem_count_dist_flops"]
DEM_NOALLOC_MAX_PARTICLES = 16384
DEM_WAIT_POLLS_DEFAULT = 4194304
# launch groups of the trace (dem_trace)
TRACE_SITES = {0: "broad phase", 1: "tile spheres", 2: "pair kernel", 3: "contact sort", 4: "clusters",
               5: "LTS bookkeeping"}
DEM_CTIME_SAMPLES, DEM_CTIME_NARROWING = 0, 1


class DemError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class dem_config(C.Structure):
    _fields_ = [("K", C.c_int32), ("bisect_tol", C.c_double), ("precision", C.c_int32),
                ("ctime_method", C.c_int32), ("max_particles", C.c_int64), ("max_pairs", C.c_int64),
                ("max_contacts", C.c_int64), ("max_triangles", C.c_int64), ("list_spill", C.c_int64)]


class dem_particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("state", C.c_void_p), ("is_static", C.c_void_p), ("tri_off", C.c_void_p),
                ("tris", C.c_void_p), ("n_tris", C.c_int64)]


class dem_narrow_out(C.Structure):
    _fields_ = [("dmin", C.c_void_p), ("pa", C.c_void_p), ("pb", C.c_void_p), ("tri_ab", C.c_void_p),
                ("flag", C.c_void_p), ("dmin32", C.c_void_p), ("contacts", C.c_void_p),
                ("contact_geom", C.c_void_p), ("contact_cap", C.c_int64), ("n_contacts", C.c_void_p)]


class dem_lts_params(C.Structure):
    _fields_ = [("dt_max", C.c_double), ("alpha", C.c_double), ("gravity", C.c_double * 3),
                ("zero_on_contact", C.c_int32), ("hose", C.c_int32)]


class dem_lts_out(C.Structure):
    _fields_ = [("pairs", C.c_void_p), ("max_pairs", C.c_int64), ("n_pairs", C.c_void_p), ("t_coll", C.c_void_p),
                ("status", C.c_void_p), ("tri_ab", C.c_void_p), ("cluster_id", C.c_void_p),
                ("n_clusters", C.c_void_p), ("active", C.c_void_p), ("t_global", C.c_void_p),
                ("narrow", C.c_void_p)]


class dem_tuning(C.Structure):
    _fields_ = [("ctas_per_sm", C.c_int32), ("wflush", C.c_int32), ("cost_order", C.c_int32), ("ms", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


DEM_TUNE_NARROW, DEM_TUNE_CTIME, DEM_TUNE_DETECT, DEM_TUNE_NARROWING = 0, 1, 2, 3


class dem_stats(C.Structure):
    _fields_ = [("sphere_tests", C.c_int64), ("group_tests", C.c_int64), ("dist_fp32", C.c_int64),
                ("dist_fp64", C.c_int64), ("pair_evals", C.c_int64), ("method_checks", C.c_int64),
                ("bisect_steps", C.c_int64), ("contacts", C.c_int64), ("pairs_done", C.c_int64),
                ("kernel_launches", C.c_int64), ("tile_pairs", C.c_int64), ("rollbacks", C.c_int64),
                ("rollbacks_before_old", C.c_int64), ("advances", C.c_int64), ("cta_busy_ns", C.c_int64),
                ("cta_busy_ns_max", C.c_int64), ("ctas", C.c_int64), ("reserved", C.c_int64 * 1)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "reserved"}


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libdem.so (building it in-tree first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_needed else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library missing: {path}")
        L = C.CDLL(path)
        vp, i64 = C.c_void_p, C.c_int64
        L.dem_create.argtypes = [C.POINTER(dem_config), C.POINTER(vp)]
        L.dem_create.restype = C.c_int
        L.dem_destroy.argtypes = [vp]
        L.dem_destroy.restype = None
        L.dem_last_error.argtypes = [vp]
        L.dem_last_error.restype = C.c_char_p
        L.dem_build_candidates.argtypes = [vp, C.POINTER(dem_particles), vp, i64, vp, vp]
        L.dem_build_candidates.restype = C.c_int
        L.dem_narrow_phase.argtypes = [vp, C.POINTER(dem_particles), vp, i64, vp, vp, C.POINTER(dem_narrow_out), vp]
        L.dem_narrow_phase.restype = C.c_int
        L.dem_collision_times.argtypes = [vp, C.POINTER(dem_particles), vp, i64, vp, vp, vp, vp, vp]
        L.dem_collision_times.restype = C.c_int
        L.dem_detect.argtypes = [vp, C.POINTER(dem_particles), vp, i64, vp, C.POINTER(dem_narrow_out), vp, vp,
                                 vp, vp]
        L.dem_detect.restype = C.c_int
        L.dem_clusters.argtypes = [vp, i64, vp, i64, vp, vp, vp, vp, vp]
        L.dem_clusters.restype = C.c_int
        L.dem_check.argtypes = [vp, vp]
        L.dem_check.restype = C.c_int
        L.dem_get_stats.argtypes = [vp, C.POINTER(dem_stats), C.c_int]
        L.dem_get_stats.restype = C.c_int
        L.dem_build_candidates_noalloc.argtypes = [C.POINTER(dem_particles), vp, i64, vp, vp]
        L.dem_build_candidates_noalloc.restype = C.c_int
        L.dem_lts_sweep.argtypes = [vp, C.POINTER(dem_particles), vp, vp, C.POINTER(dem_lts_params),
                                    C.POINTER(dem_lts_out), vp]
        L.dem_lts_sweep.restype = C.c_int
        L.dem_noalloc_check.argtypes = [vp]
        L.dem_noalloc_check.restype = C.c_int
        L.dem_set_wait_polls.argtypes = [vp, i64]
        L.dem_set_wait_polls.restype = C.c_int
        L.dem_trace.argtypes = [vp, C.c_int32]
        L.dem_trace.restype = C.c_int
        L.dem_trace_read.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_float), C.c_int32,
                                     C.POINTER(C.c_int32)]
        L.dem_trace_read.restype = C.c_int
        L.dem_autotune.argtypes = [vp, C.c_int32, C.POINTER(dem_particles), vp, i64, vp, C.POINTER(dem_narrow_out),
                                   vp, vp, vp, C.c_int32, C.POINTER(dem_tuning), vp]
        L.dem_autotune.restype = C.c_int
        L.dem_get_tuning.argtypes = [vp, C.c_int32, C.POINTER(dem_tuning)]
        L.dem_get_tuning.restype = C.c_int
        L.dem_set_tuning.argtypes = [vp, C.c_int32, C.POINTER(dem_tuning)]
        L.dem_set_tuning.restype = C.c_int
        L.dem_probe_fma_peak.argtypes = [C.c_int32, C.c_int32, vp, C.POINTER(C.c_double)]
        L.dem_probe_fma_peak.restype = C.c_int
        L.dem_count_dist_flops.argtypes = [vp, i64, vp, vp]
        L.dem_count_dist_flops.restype = C.c_int
        _lib = L
        return L


# ------------------------------------------------------------------ helpers

def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _cuda(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name}: expected a contiguous CUDA tensor of {dtype}")
    return t


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _check(ctx, rc):
    if rc != 0:
        L = load()
        raise DemError(rc, L.dem_last_error(ctx).decode() if ctx else "")


# ------------------------------------------------------------------ C-ABI mirrors

def dem_create(K=8, tol=1e-3, precision=DEM_PREC_FP32_FIXUP, max_particles=65536, max_pairs=1 << 20,
               max_contacts=1 << 20, max_triangles=0, ctime_method=0, list_spill=0):
    L = load()
    cfg = dem_config(K=K, bisect_tol=tol, precision=precision, ctime_method=ctime_method,
                     max_particles=max_particles, max_pairs=max_pairs, max_contacts=max_contacts,
                     max_triangles=max_triangles, list_spill=list_spill)
    h = C.c_void_p()
    rc = L.dem_create(C.byref(cfg), C.byref(h))
    if rc != 0:
        raise DemError(rc, "dem_create")
    return h


def dem_destroy(ctx):
    load().dem_destroy(ctx)


def dem_build_candidates(ctx, P: dem_particles, pairs, cap: int, n_pairs, stream=None):
    _check(ctx, load().dem_build_candidates(ctx, C.byref(P), _ptr(pairs), int(cap), _ptr(n_pairs), _stream(stream)))


def dem_narrow_phase(ctx, P: dem_particles, pairs, max_pairs: int, n_pairs, t_eval, out: dem_narrow_out,
                     stream=None):
    _check(ctx, load().dem_narrow_phase(ctx, C.byref(P), _ptr(pairs), int(max_pairs), _ptr(n_pairs),
                                        _ptr(t_eval), C.byref(out), _stream(stream)))


def dem_collision_times(ctx, P: dem_particles, pairs, max_pairs: int, n_pairs, t_coll, status, tri_ab,
                        stream=None):
    _check(ctx, load().dem_collision_times(ctx, C.byref(P), _ptr(pairs), int(max_pairs), _ptr(n_pairs),
                                           _ptr(t_coll), _ptr(status), _ptr(tri_ab), _stream(stream)))


def dem_detect(ctx, P: dem_particles, pairs, max_pairs: int, n_pairs, out: dem_narrow_out, t_coll, status, tri_ab,
               stream=None):
    _check(ctx, load().dem_detect(ctx, C.byref(P), _ptr(pairs), int(max_pairs), _ptr(n_pairs), C.byref(out),
                                  _ptr(t_coll), _ptr(status), _ptr(tri_ab), _stream(stream)))


def dem_clusters(ctx, n: int, edges, max_edges: int, n_edges, is_static, cluster_id, n_clusters, stream=None):
    _check(ctx, load().dem_clusters(ctx, int(n), _ptr(edges), int(max_edges), _ptr(n_edges), _ptr(is_static),
                                    _ptr(cluster_id), _ptr(n_clusters), _stream(stream)))


def dem_lts_sweep(ctx, P: dem_particles, cur, old, prm: dem_lts_params, out: dem_lts_out, stream=None):
    _check(ctx, load().dem_lts_sweep(ctx, C.byref(P), _ptr(cur), _ptr(old), C.byref(prm), C.byref(out),
                                     _stream(stream)))


def dem_build_candidates_noalloc(P: dem_particles, pairs, cap: int, n_pairs, stream=None) -> int:
    """Candidate pairs with the library's fixed scratch (no device allocation;
    for callers that cannot allocate).  Returns the C status code."""
    return int(load().dem_build_candidates_noalloc(C.byref(P), _ptr(pairs), int(cap), _ptr(n_pairs),
                                                   _stream(stream)))


def dem_noalloc_check(stream=None) -> int:
    """Error word of the allocation-free candidate search (synchronises the
    stream, clears the word).  Returns the C status code."""
    return int(load().dem_noalloc_check(_stream(stream)))


def dem_probe_fma_peak(precision: int, iters: int = 1 << 16, stream=None) -> float:
    """Measured FP32 (0) or FP64 (1) FMA-chain peak of the current GPU, FLOP/s."""
    r = C.c_double()
    _check(None, load().dem_probe_fma_peak(int(precision), int(iters), _stream(stream), C.byref(r)))
    return float(r.value)


def dem_count_dist_flops(tri, stream=None):
    """FP32 operations of the pair kernel's triangle-pair distance for each
    row of tri (CUDA float32 [n, 18]); returns an int64 CUDA tensor [n]."""
    import torch
    tri = _cuda(tri, torch.float32, "tri")
    ops = torch.zeros(tri.shape[0], dtype=torch.int64, device=tri.device)
    _check(None, load().dem_count_dist_flops(_ptr(tri), int(tri.shape[0]), _ptr(ops), _stream(stream)))
    return ops


def dem_check(ctx, stream=None):
    _check(ctx, load().dem_check(ctx, _stream(stream)))


def dem_set_wait_polls(ctx, polls: int):
    _check(ctx, load().dem_set_wait_polls(ctx, int(polls)))


def dem_autotune(ctx, kind, P: dem_particles, pairs, max_pairs: int, n_pairs, out, t_coll, status, tri_ab,
                 reps: int = 1, stream=None) -> dict:
    best = dem_tuning()
    _check(ctx, load().dem_autotune(ctx, int(kind), C.byref(P), _ptr(pairs), int(max_pairs), _ptr(n_pairs),
                                    C.byref(out) if out is not None else None, _ptr(t_coll), _ptr(status),
                                    _ptr(tri_ab), int(reps), C.byref(best), _stream(stream)))
    return best.as_dict()


def dem_get_tuning(ctx, kind) -> dict:
    t = dem_tuning()
    _check(ctx, load().dem_get_tuning(ctx, int(kind), C.byref(t)))
    return t.as_dict()


def dem_set_tuning(ctx, kind, ctas_per_sm=0, wflush=64, cost_order=1):
    t = dem_tuning(ctas_per_sm=ctas_per_sm, wflush=wflush, cost_order=cost_order)
    _check(ctx, load().dem_set_tuning(ctx, int(kind), C.byref(t)))


def dem_trace(ctx, cap: int):
    _check(ctx, load().dem_trace(ctx, int(cap)))


def dem_trace_read(ctx, cap: int = 4096):
    """[(site, ms)] of the records taken since dem_trace started."""
    site = (C.c_int32 * max(cap, 1))()
    ms = (C.c_float * max(cap, 1))()
    n = C.c_int32()
    _check(ctx, load().dem_trace_read(ctx, site, ms, int(cap), C.byref(n)))
    return [(int(site[k]), float(ms[k])) for k in range(min(n.value, cap))]


def dem_get_stats(ctx, reset=False) -> dict:
    st = dem_stats()
    _check(ctx, load().dem_get_stats(ctx, C.byref(st), 1 if reset else 0))
    return st.as_dict()


# ------------------------------------------------------------------ convenience

class Scene:
    """Particle arrays resident on the device (the dem_particles of the C-ABI)."""

    def __init__(self, state, is_static, tri_off, tris):
        import torch
        self.state = _cuda(state, torch.float64, "state")
        self.is_static = _cuda(is_static, torch.uint8, "is_static")
        self.tri_off = _cuda(tri_off, torch.int64, "tri_off")
        self.tris = _cuda(tris, torch.float32, "tris")
        self.n = int(self.state.shape[1])
        self.n_tris = int(self.tris.shape[1])
        self.P = dem_particles(n=self.n, state=self.state.data_ptr(), is_static=self.is_static.data_ptr(),
                               tri_off=self.tri_off.data_ptr(), tris=self.tris.data_ptr(), n_tris=self.n_tris)

    @classmethod
    def from_workload(cls, w, device="cuda"):
        import torch
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        return cls(t(w.state), t(w.is_static), t(w.tri_off), t(w.tris))


class Context:
    """Owns a dem_ctx and output buffers sized for its capacities."""

    def __init__(self, K=8, tol=1e-3, precision=DEM_PREC_FP32_FIXUP, max_particles=65536, max_pairs=1 << 20,
                 max_contacts=1 << 20, max_triangles=0, ctime_method=0, device="cuda", list_spill=0):
        import torch
        self.device = torch.device(device)
        self.max_pairs = int(max_pairs)
        self.max_contacts = int(max_contacts)
        self.h = dem_create(K, tol, precision, max_particles, max_pairs, max_contacts, max_triangles, ctime_method,
                            list_spill)
        z = lambda *s, dt: torch.zeros(*s, dtype=dt, device=self.device)
        self.pairs = z(self.max_pairs, 2, dt=torch.int32)
        self.n_pairs = z(1, dt=torch.int64)
        self.dmin = z(self.max_pairs, dt=torch.float64)
        self.pa = z(self.max_pairs, 3, dt=torch.float64)
        self.pb = z(self.max_pairs, 3, dt=torch.float64)
        self.tri_ab = z(self.max_pairs, 2, dt=torch.int32)
        self.flag = z(self.max_pairs, dt=torch.uint8)
        self.dmin32 = z(self.max_pairs, dt=torch.float32)
        self.contacts = z(self.max_contacts, 3, dt=torch.int32)
        self.contact_geom = z(self.max_contacts, 7, dt=torch.float64)
        self.n_contacts = z(1, dt=torch.int64)
        self.t_coll = z(self.max_pairs, dt=torch.float64)
        self.status = z(self.max_pairs, dt=torch.uint8)
        self.ct_ab = z(self.max_pairs, 2, dt=torch.int32)
        self.n_clusters = z(1, dt=torch.int64)
        self.cluster_id = None
        self.out = dem_narrow_out(dmin=self.dmin.data_ptr(), pa=self.pa.data_ptr(), pb=self.pb.data_ptr(),
                                  tri_ab=self.tri_ab.data_ptr(), flag=self.flag.data_ptr(),
                                  dmin32=self.dmin32.data_ptr(), contacts=self.contacts.data_ptr(),
                                  contact_geom=self.contact_geom.data_ptr(), contact_cap=self.max_contacts,
                                  n_contacts=self.n_contacts.data_ptr())

    def close(self):
        if self.h:
            dem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # one call each ------------------------------------------------------
    def build_candidates(self, scene: Scene, stream=None):
        dem_build_candidates(self.h, scene.P, self.pairs, self.max_pairs, self.n_pairs, stream)

    def narrow_phase(self, scene: Scene, pairs=None, n_pairs=None, t_eval=None, stream=None):
        """Default: the candidate pairs held by this context (device count)."""
        if pairs is None:
            pairs, m, cnt = self.pairs, self.max_pairs, self.n_pairs
        else:
            m, cnt = int(pairs.shape[0]), n_pairs
        dem_narrow_phase(self.h, scene.P, pairs, m, cnt, t_eval, self.out, stream)

    def collision_times(self, scene: Scene, pairs=None, n_pairs=None, stream=None):
        if pairs is None:
            pairs, m, cnt = self.pairs, self.max_pairs, self.n_pairs
        else:
            m, cnt = int(pairs.shape[0]), n_pairs
        dem_collision_times(self.h, scene.P, pairs, m, cnt, self.t_coll, self.status, self.ct_ab, stream)

    def detect(self, scene: Scene, pairs=None, n_pairs=None, stream=None):
        """Narrow phase at the pair start and collision times in one launch."""
        if pairs is None:
            pairs, m, cnt = self.pairs, self.max_pairs, self.n_pairs
        else:
            m, cnt = int(pairs.shape[0]), n_pairs
        dem_detect(self.h, scene.P, pairs, m, cnt, self.out, self.t_coll, self.status, self.ct_ab, stream)

    def clusters(self, scene: Scene, edges=None, n_edges=None, stream=None):
        import torch
        if self.cluster_id is None or self.cluster_id.numel() < scene.n:
            self.cluster_id = torch.zeros(max(scene.n, 1), dtype=torch.int32, device=self.device)
        if edges is None:
            edges, m, cnt = self.pairs, self.max_pairs, self.n_pairs
        else:
            m, cnt = int(edges.shape[0]), n_edges
        dem_clusters(self.h, scene.n, edges, m, cnt, scene.is_static, self.cluster_id, self.n_clusters, stream)

    def step(self, scene: Scene, stream=None):
        """One pass of the whole path: candidates, narrow phase at the pair
        start, collision times, clusters of the candidate graph."""
        self.build_candidates(scene, stream)
        self.narrow_phase(scene, stream=stream)
        self.collision_times(scene, stream=stream)
        self.clusters(scene, stream=stream)

    def step_fused(self, scene: Scene, stream=None):
        """The same step with the narrow phase and the collision times fused
        (dem_detect): candidates, detect, clusters."""
        self.build_candidates(scene, stream)
        self.detect(scene, stream=stream)
        self.clusters(scene, stream=stream)

    def lts_sweep(self, scene: Scene, old, dt_max, alpha=2.0, gravity=(0.0, 0.0, 0.0), zero_on_contact=True,
                  hose=False, narrow=False, stream=None):
        """One local-time-stepping sweep: scene.state is the current snapshot
        and ``old`` (same shape) the old one; both are updated in place.
        Outputs in this context's buffers (pairs, n_pairs, t_coll, status,
        ct_ab, cluster_id, n_clusters, active, t_global); with narrow=True
        also the narrow phase of the sweep's pairs at their start time (dmin,
        pa, pb, tri_ab, flag, dmin32, contacts, contact_geom, n_contacts)."""
        import torch
        if self.cluster_id is None or self.cluster_id.numel() < scene.n:
            self.cluster_id = torch.zeros(max(scene.n, 1), dtype=torch.int32, device=self.device)
        if getattr(self, "active", None) is None or self.active.numel() < scene.n:
            self.active = torch.zeros(max(scene.n, 1), dtype=torch.uint8, device=self.device)
            self.t_global = torch.zeros(1, dtype=torch.float64, device=self.device)
        if old.dtype != torch.float64 or not old.is_contiguous() or old.shape != scene.state.shape:
            raise ValueError("old must be a contiguous float64 tensor shaped like the state")
        prm = dem_lts_params(dt_max=float(dt_max), alpha=float(alpha), gravity=(C.c_double * 3)(*gravity),
                             zero_on_contact=int(bool(zero_on_contact)), hose=int(bool(hose)))
        out = dem_lts_out(pairs=self.pairs.data_ptr(), max_pairs=self.max_pairs, n_pairs=self.n_pairs.data_ptr(),
                          t_coll=self.t_coll.data_ptr(), status=self.status.data_ptr(), tri_ab=self.ct_ab.data_ptr(),
                          cluster_id=self.cluster_id.data_ptr(), n_clusters=self.n_clusters.data_ptr(),
                          active=self.active.data_ptr(), t_global=self.t_global.data_ptr(),
                          narrow=C.addressof(self.out) if narrow else None)
        dem_lts_sweep(self.h, scene.P, scene.state, old, prm, out, stream)

    def check(self, stream=None):
        dem_check(self.h, stream)

    def autotune(self, scene: Scene, kind=DEM_TUNE_DETECT, pairs=None, n_pairs=None, reps=1, stream=None):
        """Tune the pair kernel's launch configuration for `kind` on these pairs
        (default: the context's candidate pairs); returns the chosen one."""
        if pairs is None:
            pairs, m, cnt = self.pairs, self.max_pairs, self.n_pairs
        else:
            m, cnt = int(pairs.shape[0]), n_pairs
        return dem_autotune(self.h, kind, scene.P, pairs, m, cnt, self.out, self.t_coll, self.status, self.ct_ab,
                            reps, stream)

    def get_tuning(self, kind=DEM_TUNE_DETECT):
        return dem_get_tuning(self.h, kind)

    def set_tuning(self, kind=DEM_TUNE_DETECT, **kw):
        dem_set_tuning(self.h, kind, **kw)

    def set_wait_polls(self, polls: int):
        dem_set_wait_polls(self.h, polls)

    def trace(self, cap: int):
        dem_trace(self.h, cap)

    def trace_read(self, cap: int = 4096):
        return dem_trace_read(self.h, cap)

    def stats(self, reset=False):
        return dem_get_stats(self.h, reset)
