"""The paper's narrowing (DEM_CTIME_NARROWING) on the GPU against the oracle's
narrowing procedure: status, collision time and triangle pair bit for bit, in
both precision modes (the procedure itself is binary64 throughout; the FP32
mode only changes how the pair-interval list is culled); and dem_detect with
the narrowing equals the two separate calls.
"""
import numpy as np
import pytest

import oracle
from paper_2309_15417_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PRECS = [0, 1]


def _gpu_narrowing(dem, w, pairs, prec, list_spill=0):
    import torch
    c = dem.Context(K=w.K, tol=w.tol, precision=prec, max_particles=max(w.n, 16), max_pairs=max(len(pairs), 1),
                    max_contacts=1 << 18, max_triangles=w.n_tris, ctime_method=dem.DEM_CTIME_NARROWING,
                    list_spill=list_spill)
    sc = dem.Scene.from_workload(w)
    pt = torch.from_numpy(np.ascontiguousarray(pairs, np.int32).reshape(-1, 2)).cuda()
    c.collision_times(sc, pairs=pt)
    c.check()
    m = len(pairs)
    out = dict(t_coll=c.t_coll[:m].cpu().numpy(), status=c.status[:m].cpu().numpy(),
               tri_ab=c.ct_ab[:m].cpu().numpy(), stats=c.stats(reset=True))
    c.close()
    return out


def _check(dem, w, pairs, prec, list_spill=0):
    o = oracle.collision_times_narrowing(w, pairs)
    g = _gpu_narrowing(dem, w, pairs, prec, list_spill)
    assert np.array_equal(g["status"], o["status"])
    assert np.array_equal(g["t_coll"], o["t_coll"])
    assert np.array_equal(g["tri_ab"], o["tri_ab"])
    return o


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_narrowing_small_icospheres(dem, seed, prec):
    w = W.small_icospheres(seed)
    o = _check(dem, w, oracle.broad_phase(w), prec)
    assert {1, 2} <= set(o["status"].tolist())


@pytest.mark.parametrize("prec", PRECS)
def test_narrowing_translation_only(dem, prec):
    w = W.dense_packing(3, nside=5, vsig=150.0, wsig=0.0)
    w.state[W.F_WX:W.F_WZ + 1] = 0.0
    o = _check(dem, w, oracle.broad_phase(w), prec)
    assert (o["status"] == 2).sum() > 3


@pytest.mark.parametrize("prec", PRECS)
def test_narrowing_rotating_packing(dem, prec):
    w = W.dense_packing(1, nside=4, vsig=60.0, wsig=60.0)
    _check(dem, w, oracle.broad_phase(w), prec)


@pytest.mark.parametrize("prec", PRECS)
def test_narrowing_static_floor(dem, prec):
    """Multi-tile static floor, static post, static pair intervals."""
    w = W.floor_scene(0)
    o = _check(dem, w, oracle.broad_phase(w), prec)
    assert 2 in set(o["status"].tolist())


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("spill", [0, 1])
def test_narrowing_list_overflow(dem, prec, spill):
    """Fast head-on 320-triangle icospheres: the pair-interval list outgrows
    its 512 shared-memory entries; with the default global spill the list
    holds them, with a one-entry spill it overflows and every narrowing
    iteration runs over all triangle pairs."""
    for frac in (0.3, 0.9):
        w = W.injected_head_on(0.1 + frac * 0.8, 800.0, 0.05, 1e-3, subdiv=2)
        o = _check(dem, w, np.array([[0, 1]], np.int32), prec, list_spill=spill)
        assert o["status"][0] == 2


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("spill", [0, 1])
def test_narrowing_fast_rotating_packing(dem, seed, prec, spill):
    """v, w ~ N(0, 150): the narrowing's motion bound (~0.3) lets far more
    triangle pairs into the pair-interval list than its shared-memory part
    holds (the global spill takes them; with a one-entry spill the iterations
    visit every triangle pair, pruned by bounding spheres and, in the FP32
    mode, certified FP32 lower bounds at ts)."""
    w = W.dense_packing(seed, nside=4, vsig=150.0, wsig=150.0)
    o = _check(dem, w, oracle.broad_phase(w), prec, list_spill=spill)
    assert (o["status"] == 2).sum() >= 3


def test_detect_with_narrowing_equals_separate_calls(dem):
    w = W.small_icospheres(1)
    c1 = dem.Context(K=w.K, tol=w.tol, max_particles=w.n, max_pairs=4096, ctime_method=dem.DEM_CTIME_NARROWING)
    c2 = dem.Context(K=w.K, tol=w.tol, max_particles=w.n, max_pairs=4096, ctime_method=dem.DEM_CTIME_NARROWING)
    sc = dem.Scene.from_workload(w)
    c1.step(sc)
    c2.step_fused(sc)
    c1.check()
    c2.check()
    m = int(c1.n_pairs.item())
    for name in ("flag", "tri_ab", "dmin", "t_coll", "status", "ct_ab"):
        assert np.array_equal(getattr(c1, name)[:m].cpu().numpy(), getattr(c2, name)[:m].cpu().numpy()), name
    o = oracle.collision_times_narrowing(w, c1.pairs[:m].cpu().numpy())
    assert np.array_equal(c2.t_coll[:m].cpu().numpy(), o["t_coll"])
