"""Failure paths of the C-ABI on the GPU, each provoked on the host (no
fault, trap or hang of the device): output capacities smaller than needed,
a tri_off range beyond the triangles, non-finite state and vertices, a
first tile-copy wait limited to zero polls, null pointers and sizes beyond
the context's capacities.  After each, the context stays usable and a
correct call equals the oracle."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2309_15417_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _ctx(dem, w, **kw):
    args = dict(K=w.K, tol=w.tol, max_particles=max(w.n, 16), max_pairs=4096, max_contacts=1 << 16)
    args.update(kw)
    return dem.Context(**args)


def _status(dem, ctx):
    try:
        ctx.check()
        return dem.DEM_OK
    except dem.DemError as e:
        return e.status


def test_candidate_capacity_exceeded_then_recovered(dem):
    w = W.dense_packing(0)
    ref = oracle.broad_phase(w)
    sc = dem.Scene.from_workload(w)
    small = _ctx(dem, w, max_pairs=64)
    small.build_candidates(sc)
    assert _status(dem, small) == dem.DEM_ERR_CAPACITY
    assert int(small.n_pairs.item()) == len(ref)  # the required count is reported
    assert _status(dem, small) == dem.DEM_OK  # dem_check cleared the word
    small.close()
    big = _ctx(dem, w, max_pairs=len(ref))
    big.build_candidates(sc)
    assert _status(dem, big) == dem.DEM_OK
    assert np.array_equal(big.pairs[:len(ref)].cpu().numpy(), ref)
    big.close()


def test_contact_capacity_exceeded_then_recovered(dem):
    w = W.small_icospheres(0)
    pairs = oracle.broad_phase(w)
    on = oracle.narrow_phase(w, pairs)
    nc = len(on["contacts"])
    assert nc > 8
    sc = dem.Scene.from_workload(w)
    small = _ctx(dem, w, max_contacts=8)
    small.build_candidates(sc)
    small.narrow_phase(sc)
    assert _status(dem, small) == dem.DEM_ERR_CAPACITY
    need = int(small.n_contacts.item())  # a sufficient capacity (FP32: staged candidates)
    assert need >= nc
    small.close()
    big = _ctx(dem, w, max_contacts=need)
    big.build_candidates(sc)
    big.narrow_phase(sc)
    assert _status(dem, big) == dem.DEM_OK
    assert np.array_equal(big.contacts[:nc].cpu().numpy(), on["contacts"])
    assert np.array_equal(big.flag[:len(pairs)].cpu().numpy(), on["flag"])
    big.close()


def test_tri_off_beyond_the_triangles_is_an_index_error(dem):
    import torch
    w = W.small_icospheres(0)
    pairs = oracle.broad_phase(w)
    bad = int(pairs[0, 0])  # a particle that has candidates
    off = w.tri_off.copy()
    off[bad + 1] = w.n_tris + 4096  # its range runs past the end; the next one's is negative
    sc = dem.Scene.from_workload(w)
    sc.tri_off.copy_(torch.from_numpy(off).cuda())
    ctx = _ctx(dem, w)
    gp = torch.from_numpy(pairs).cuda()
    ctx.narrow_phase(sc, pairs=gp)
    ctx.collision_times(sc, pairs=gp)
    assert _status(dem, ctx) == dem.DEM_ERR_INDEX
    # pairs that do not touch the two broken ranges are still the oracle's
    keep = ~np.isin(pairs, [bad, bad + 1]).any(axis=1)
    on = oracle.narrow_phase(w, pairs)
    oc = oracle.collision_times(w, pairs)
    m = len(pairs)
    assert np.array_equal(ctx.flag[:m].cpu().numpy()[keep], on["flag"][keep])
    assert np.array_equal(ctx.tri_ab[:m].cpu().numpy()[keep], on["tri_ab"][keep])
    assert np.array_equal(ctx.status[:m].cpu().numpy()[keep], oc["status"][keep])
    assert np.array_equal(ctx.t_coll[:m].cpu().numpy()[keep], oc["t_coll"][keep])
    # the broken pairs report "no triangles"
    assert (ctx.tri_ab[:m].cpu().numpy()[~keep] == -1).all()
    ctx.close()


@pytest.mark.parametrize("field", [0, 7, 13])  # x, a quaternion component, t_cur
def test_nonfinite_state_is_reported_and_its_particle_skipped(dem, field):
    import torch
    w = W.small_icospheres(0)
    ref = oracle.broad_phase(w)
    bad = int(ref[0, 0])
    st = w.state.copy()
    st[field, bad] = np.nan if field != 13 else np.inf
    sc = dem.Scene.from_workload(w)
    sc.state.copy_(torch.from_numpy(st).cuda())
    ctx = _ctx(dem, w)
    ctx.build_candidates(sc)
    assert _status(dem, ctx) == dem.DEM_ERR_NONFINITE
    m = int(ctx.n_pairs.item())
    keep = ref[~np.isin(ref, [bad]).any(axis=1)]
    assert np.array_equal(ctx.pairs[:m].cpu().numpy(), keep)
    # the narrow phase given the full list skips the pairs of that particle
    gp = torch.from_numpy(ref).cuda()
    ctx.narrow_phase(sc, pairs=gp)
    assert _status(dem, ctx) == dem.DEM_ERR_NONFINITE
    on = oracle.narrow_phase(w, ref)
    ok = ~np.isin(ref, [bad]).any(axis=1)
    assert np.array_equal(ctx.flag[:len(ref)].cpu().numpy()[ok], on["flag"][ok])
    assert (ctx.tri_ab[:len(ref)].cpu().numpy()[~ok] == -1).all()
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_nonfinite_vertex_is_reported(dem, prec):
    import torch
    w = W.small_icospheres(0)
    pairs = oracle.broad_phase(w)
    bad = int(pairs[0, 1])
    tris = w.tris.copy()
    tris[1, w.tri_off[bad] + 3, 2] = np.nan  # z of vertex 1 of the particle's 4th triangle
    sc = dem.Scene.from_workload(w)
    sc.tris.copy_(torch.from_numpy(tris).cuda())
    ctx = _ctx(dem, w, precision=prec)
    ctx.narrow_phase(sc, pairs=torch.from_numpy(pairs).cuda())
    assert _status(dem, ctx) == dem.DEM_ERR_NONFINITE
    ctx.close()


def test_first_wait_with_zero_polls_times_out_and_the_context_recovers(dem):
    w = W.small_icospheres(0)
    pairs = oracle.broad_phase(w)
    sc = dem.Scene.from_workload(w)
    ctx = _ctx(dem, w)
    ctx.build_candidates(sc)
    ctx.set_wait_polls(0)
    ctx.narrow_phase(sc)
    with pytest.raises(dem.DemError) as ei:
        ctx.check()
    assert ei.value.status == dem.DEM_ERR_TIMEOUT
    assert "copy in flight landed" in str(ei.value)
    ctx.set_wait_polls(dem.DEM_WAIT_POLLS_DEFAULT)
    ctx.narrow_phase(sc)
    ctx.collision_times(sc)
    assert _status(dem, ctx) == dem.DEM_OK
    on, oc = oracle.narrow_phase(w, pairs), oracle.collision_times(w, pairs)
    m = len(pairs)
    assert np.array_equal(ctx.dmin[:m].cpu().numpy(), on["dmin"])
    assert np.array_equal(ctx.status[:m].cpu().numpy(), oc["status"])
    with pytest.raises(dem.DemError):
        ctx.set_wait_polls(-1)
    ctx.close()


def test_null_pointers_and_oversize_arguments_are_rejected_on_the_host(dem):
    import torch
    L = dem.load()
    w = W.small_icospheres(0)
    sc = dem.Scene.from_workload(w)
    ctx = _ctx(dem, w, max_particles=w.n, max_pairs=256, max_contacts=1024)
    h = ctx.h
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = sc.P
    pp, npp = C.c_void_p(ctx.pairs.data_ptr()), C.c_void_p(ctx.n_pairs.data_ptr())
    ARG, CAP = dem.DEM_ERR_ARG, dem.DEM_ERR_CAPACITY
    assert L.dem_build_candidates(h, None, pp, 256, npp, s) == ARG
    assert L.dem_build_candidates(h, C.byref(P), None, 256, npp, s) == ARG
    assert L.dem_build_candidates(h, C.byref(P), pp, 256, None, s) == ARG
    assert L.dem_build_candidates(h, C.byref(P), pp, -1, npp, s) == ARG
    big = dem.dem_particles(n=w.n + 1, state=P.state, is_static=P.is_static, tri_off=P.tri_off, tris=P.tris,
                            n_tris=P.n_tris)
    assert L.dem_build_candidates(h, C.byref(big), pp, 256, npp, s) == CAP
    mis = dem.dem_particles(n=P.n, state=P.state, is_static=P.is_static, tri_off=P.tri_off, tris=P.tris + 4,
                            n_tris=P.n_tris)
    assert L.dem_build_candidates(h, C.byref(mis), pp, 256, npp, s) == ARG
    nostate = dem.dem_particles(n=P.n, state=None, is_static=P.is_static, tri_off=P.tri_off, tris=P.tris,
                                n_tris=P.n_tris)
    assert L.dem_build_candidates(h, C.byref(nostate), pp, 256, npp, s) == ARG
    out = ctx.out
    tc, stt, ab = (C.c_void_p(t.data_ptr()) for t in (ctx.t_coll, ctx.status, ctx.ct_ab))
    assert L.dem_narrow_phase(h, C.byref(P), pp, 256, npp, None, None, s) == ARG
    assert L.dem_narrow_phase(h, C.byref(P), None, 256, npp, None, C.byref(out), s) == ARG
    assert L.dem_narrow_phase(h, C.byref(P), pp, 257, npp, None, C.byref(out), s) == CAP
    assert L.dem_collision_times(h, C.byref(P), pp, 256, npp, None, stt, ab, s) == ARG
    assert L.dem_collision_times(h, C.byref(P), pp, 257, npp, tc, stt, ab, s) == CAP
    assert L.dem_detect(h, C.byref(P), pp, 257, npp, C.byref(out), tc, stt, ab, s) == CAP
    assert L.dem_detect(h, C.byref(P), pp, 256, npp, C.byref(out), None, stt, ab, s) == ARG
    cid = C.c_void_p(torch.zeros(w.n, dtype=torch.int32, device="cuda").data_ptr())
    assert L.dem_clusters(h, w.n, pp, 256, npp, None, cid, None, s) == ARG
    assert L.dem_clusters(h, w.n, None, 256, npp, None, cid, C.c_void_p(ctx.n_clusters.data_ptr()), s) == ARG
    assert L.dem_clusters(h, -1, pp, 256, npp, None, cid, C.c_void_p(ctx.n_clusters.data_ptr()), s) == ARG
    # nothing was launched by the rejected calls: the context is clean and works
    assert _status(dem, ctx) == dem.DEM_OK
    ctx.build_candidates(sc)
    ctx.check()
    ref = oracle.broad_phase(w)
    assert np.array_equal(ctx.pairs[:len(ref)].cpu().numpy(), ref)
    ctx.close()


def test_trace_times_each_launch_group(dem):
    """The trace records the call's launch groups in order, with positive
    durations, directly and inside a CUDA graph replay."""
    import torch
    w = W.small_icospheres(0)
    sc = dem.Scene.from_workload(w)
    ctx = _ctx(dem, w)
    ctx.trace(64)
    ctx.build_candidates(sc)
    ctx.detect(sc)
    ctx.clusters(sc)
    torch.cuda.synchronize()
    rec = ctx.trace_read()
    sites = [r[0] for r in rec]
    assert sites == [0, 1, 2, 3, 4]  # broad, tiles, pair kernel, contacts, clusters
    assert all(ms > 0 for _, ms in rec)
    ctx.trace(64)  # restart: the graph's records are 0..4
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        ctx.build_candidates(sc)  # warm-up outside the capture
    torch.cuda.synchronize()
    ctx.trace(64)
    with torch.cuda.graph(g):
        ctx.build_candidates(sc)
        ctx.detect(sc)
        ctx.clusters(sc)
    g.replay()
    torch.cuda.synchronize()
    rec = ctx.trace_read()
    assert [r[0] for r in rec] == [0, 1, 2, 3, 4]
    assert all(ms > 0 for _, ms in rec)
    ctx.check()
    del g
    ctx.close()
