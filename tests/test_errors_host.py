"""Argument errors that the C-ABI detects on the host before touching the
device: every call given a null context, a null or malformed configuration,
or out-of-range settings returns DEM_ERR_ARG (no GPU needed)."""
import ctypes as C

import pytest

from paper_2309_15417_gb300 import dem as D


@pytest.fixture(scope="module")
def L():
    return D.load()


def test_null_context_is_an_argument_error(L):
    P = D.dem_particles()
    out = D.dem_narrow_out()
    prm = D.dem_lts_params(dt_max=1e-3, alpha=2.0)
    lo = D.dem_lts_out()
    st = D.dem_stats()
    n = C.c_int32()
    site = (C.c_int32 * 4)()
    ms = (C.c_float * 4)()
    calls = [
        L.dem_build_candidates(None, C.byref(P), None, 0, None, None),
        L.dem_narrow_phase(None, C.byref(P), None, 0, None, None, C.byref(out), None),
        L.dem_collision_times(None, C.byref(P), None, 0, None, None, None, None, None),
        L.dem_detect(None, C.byref(P), None, 0, None, C.byref(out), None, None, None, None),
        L.dem_clusters(None, 0, None, 0, None, None, None, None, None),
        L.dem_lts_sweep(None, C.byref(P), None, None, C.byref(prm), C.byref(lo), None),
        L.dem_check(None, None),
        L.dem_get_stats(None, C.byref(st), 0),
        L.dem_set_wait_polls(None, 10),
        L.dem_trace(None, 4),
        L.dem_trace_read(None, site, ms, 4, C.byref(n)),
        L.dem_autotune(None, 2, C.byref(P), None, 0, None, C.byref(out), None, None, None, 1, None, None),
        L.dem_get_tuning(None, 2, C.byref(D.dem_tuning())),
        L.dem_set_tuning(None, 2, C.byref(D.dem_tuning(wflush=64, cost_order=1))),
    ]
    assert calls == [D.DEM_ERR_ARG] * len(calls)
    assert L.dem_last_error(None) == b"null context"
    L.dem_destroy(None)  # a no-op


def test_noalloc_rejects_null_arguments_before_any_launch(L):
    P = D.dem_particles(n=4)
    n = C.c_int64()
    assert L.dem_build_candidates_noalloc(None, None, 0, C.byref(n), None) == D.DEM_ERR_ARG
    # n > 0 with null state and tri_off
    assert L.dem_build_candidates_noalloc(C.byref(P), None, 0, C.byref(n), None) == D.DEM_ERR_ARG
    # null count, negative capacity, capacity without an output array
    P0 = D.dem_particles(n=0)
    assert L.dem_build_candidates_noalloc(C.byref(P0), None, 0, None, None) == D.DEM_ERR_ARG
    assert L.dem_build_candidates_noalloc(C.byref(P0), None, -1, C.byref(n), None) == D.DEM_ERR_ARG
    assert L.dem_build_candidates_noalloc(C.byref(P0), None, 8, C.byref(n), None) == D.DEM_ERR_ARG


@pytest.mark.parametrize("field,value", [("K", -1), ("bisect_tol", -1e-3), ("precision", 7), ("ctime_method", 5),
                                         ("max_particles", -1), ("max_pairs", -5), ("max_contacts", -1),
                                         ("max_triangles", -1), ("max_pairs", 1 << 40), ("list_spill", -1),
                                         ("list_spill", (1 << 24) + 1)])
def test_bad_configuration_is_rejected_before_any_allocation(L, field, value):
    cfg = D.dem_config()
    setattr(cfg, field, value)
    h = C.c_void_p()
    assert L.dem_create(C.byref(cfg), C.byref(h)) == D.DEM_ERR_ARG
    assert not h.value


def test_create_needs_an_output_handle(L):
    assert L.dem_create(None, None) == D.DEM_ERR_ARG
