"""Local-time-stepping sweeps on the GPU (dem_lts_sweep) against the oracle's
sweeps, several sweeps in a row: the current and old snapshots (every field),
the candidate pairs with their statuses and collision times, the clusters,
the active set and the masking bound, all bit for bit, in both precision
modes; and the sweeps captured in one CUDA graph equal the direct calls.
"""
import numpy as np
import pytest

import oracle
from paper_2309_15417_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PRECS = [0, 1]


def _mixed_time_stamps(w, dt_max, seed):
    """Particles at different time stamps with different histories."""
    rng = np.random.default_rng(seed)
    mv = w.is_static == 0
    w.state[W.F_TCUR, mv] = np.round(rng.uniform(0.0, 0.5 * dt_max, mv.sum()) * 2 ** 30) / 2 ** 30
    old = w.state.copy()
    old[W.F_TCUR, mv] = w.state[W.F_TCUR, mv] - np.round(rng.uniform(0.0, dt_max, mv.sum()) * 2 ** 30) / 2 ** 30
    return old


def _compare_narrow(c, w, r, m):
    """The sweep's narrow phase (pairs at their start time after the
    consolidation) against the oracle's narrow phase on the oracle's
    consolidated snapshot."""
    wc = W.Workload(w.name, r["consolidated"], w.is_static, w.tri_off, w.tris, w.K, w.tol)
    on = oracle.narrow_phase(wc, r["pairs"])
    assert np.array_equal(c.flag[:m].cpu().numpy(), on["flag"])
    assert np.array_equal(c.tri_ab[:m].cpu().numpy(), on["tri_ab"])
    assert np.array_equal(c.dmin[:m].cpu().numpy(), on["dmin"])
    nc = int(c.n_contacts.item())
    assert np.array_equal(c.contacts[:nc].cpu().numpy(), on["contacts"])
    return nc


def _compare_sweeps(dem, w, old, prec, sweeps, dt_max, gravity, max_pairs=1 << 16, hose=False, narrow=False):
    import torch
    c = dem.Context(K=w.K, tol=w.tol, precision=prec, max_particles=max(w.n, 16), max_pairs=max_pairs,
                    max_contacts=1 << 16, max_triangles=w.n_tris)
    sc = dem.Scene.from_workload(w)
    g_old = torch.from_numpy(old.copy()).cuda()
    o_w = W.Workload(w.name, w.state.copy(), w.is_static, w.tri_off, w.tris, w.K, w.tol)
    o_old = old.copy()
    seen = set()
    contacts = 0
    for s in range(sweeps):
        c.lts_sweep(sc, g_old, dt_max, gravity=gravity, hose=hose, narrow=narrow)
        c.check()
        r = oracle.lts_sweep(o_w, o_old, dt_max, gravity=gravity, hose=hose)
        m = int(c.n_pairs.item())
        if narrow:
            contacts += _compare_narrow(c, w, r, m)
        assert np.array_equal(c.pairs[:m].cpu().numpy(), r["pairs"]), s
        assert np.array_equal(c.status[:m].cpu().numpy(), r["status"]), s
        assert np.array_equal(c.t_coll[:m].cpu().numpy(), r["t_coll"]), s
        assert np.array_equal(c.cluster_id[:w.n].cpu().numpy(), r["ids"]), s
        assert np.array_equal(c.active[:w.n].cpu().numpy(), r["active"]), s
        assert c.t_global.item() == r["t_global"], s
        assert np.array_equal(sc.state.cpu().numpy(), o_w.state), s
        assert np.array_equal(g_old.cpu().numpy(), o_old), s
        st = c.stats(reset=True)
        assert st["rollbacks"] == r["rollbacks"] and st["rollbacks_before_old"] == r["rollbacks_before_old"]
        assert st["advances"] == int(r["active"].sum())
        seen |= set(r["status"].tolist())
    c.close()
    if narrow:
        assert contacts > 0
    return seen


@pytest.mark.parametrize("prec", PRECS)
def test_lts_sweeps_small_icospheres(dem, prec):
    w = W.small_icospheres(0)
    seen = _compare_sweeps(dem, w, w.state.copy(), prec, 6, 1e-3, (0.0, 0.0, -9.81))
    assert {1, 2} <= seen


@pytest.mark.parametrize("prec", PRECS)
def test_lts_sweeps_mixed_time_stamps(dem, prec):
    """Dense FCC blobs and free particles at scattered time stamps: the
    consolidation rolls particles back and masking holds clusters back."""
    w = W.lts_mixed_steps(0, n=1500)
    old = _mixed_time_stamps(w, 4e-3, 1)
    _compare_sweeps(dem, w, old, prec, 4, 4e-3, (0.0, 0.0, 0.0))


@pytest.mark.parametrize("prec", PRECS)
def test_lts_sweeps_floor_scene(dem, prec):
    w = W.floor_scene(1)
    seen = _compare_sweeps(dem, w, w.state.copy(), prec, 6, 1e-3, (0.0, 0.0, -9.81))
    assert 1 in seen


@pytest.mark.parametrize("prec", PRECS)
def test_lts_sweeps_with_hoses(dem, prec):
    """The space-time hose check in the broad phase: mixed time stamps (old
    segments matter) and fast free particles."""
    w = W.lts_mixed_steps(1, n=1500)
    w.state[W.F_VX:W.F_VZ + 1] *= 20.0
    old = _mixed_time_stamps(w, 4e-3, 2)
    _compare_sweeps(dem, w, old, prec, 4, 4e-3, (0.0, 0.0, 0.0), hose=True)
    w = W.small_icospheres(2)
    w.state[W.F_VX:W.F_VZ + 1] *= 150.0
    _compare_sweeps(dem, w, w.state.copy(), prec, 4, 1e-3, (0.0, 0.0, -9.81), hose=True)


def test_lts_sweeps_settling_column(dem):
    w = W.settling_column(0, nside=6, nq=32)
    _compare_sweeps(dem, w, w.state.copy(), 0, 8, 1e-3, (0.0, 0.0, -9.81))


@pytest.mark.parametrize("prec", PRECS)
def test_lts_sweeps_with_narrow_phase(dem, prec):
    """Sweeps that also emit the narrow phase of their pairs (one launch with
    the collision times): snapshots as without it, contacts as the oracle's
    narrow phase on the consolidated snapshot."""
    w = W.settling_column(0, nside=6, nq=32)
    _compare_sweeps(dem, w, w.state.copy(), prec, 6, 1e-3, (0.0, 0.0, -9.81), narrow=True)
    w = W.floor_scene(1)
    _compare_sweeps(dem, w, w.state.copy(), prec, 4, 1e-3, (0.0, 0.0, -9.81), narrow=True)
    w = W.lts_mixed_steps(0, n=1500)
    old = _mixed_time_stamps(w, 4e-3, 1)
    _compare_sweeps(dem, w, old, prec, 3, 4e-3, (0.0, 0.0, 0.0), narrow=True)


def test_lts_sweeps_in_a_cuda_graph(dem):
    """Several sweeps captured in one CUDA graph and replayed give the same
    snapshots as the same sweeps called directly."""
    import torch
    w = W.floor_scene(0)
    dt_max, sweeps = 1e-3, 4

    def fresh():
        c = dem.Context(K=w.K, tol=w.tol, precision=0, max_particles=w.n, max_pairs=4096, max_contacts=1 << 14,
                        max_triangles=w.n_tris)
        return c, dem.Scene.from_workload(w), torch.from_numpy(w.state.copy()).cuda()

    c, sc, old = fresh()
    for _ in range(sweeps):
        c.lts_sweep(sc, old, dt_max, gravity=(0.0, 0.0, -9.81))
    c.check()
    direct = (sc.state.cpu().numpy(), old.cpu().numpy())
    c.close()

    c, sc, old = fresh()
    cur0, old0 = sc.state.clone(), old.clone()
    c.lts_sweep(sc, old, dt_max, gravity=(0.0, 0.0, -9.81))  # first call outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(sweeps):
            c.lts_sweep(sc, old, dt_max, gravity=(0.0, 0.0, -9.81))
    sc.state.copy_(cur0)
    old.copy_(old0)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    c.check()
    assert np.array_equal(sc.state.cpu().numpy(), direct[0])
    assert np.array_equal(old.cpu().numpy(), direct[1])
    c.close()
