"""Pins of the oracle's second collision-time procedure, the paper's
narrowing (Section 5, "Collision time detection": vertex-triangle on the
straight relative path with rotation neglected, edge-edge samples at the
middle and the end of the span, narrowing to the earliest contact, widening).

Closed forms: a flat triangle falling onto a larger one crosses the plane at
t = h / v, so the procedure returns h / v plus the widening tol * T; a spin
about the fall direction leaves the heights linear in time and the answer
unchanged.  Brackets: for head-on vertex tips closing at speed v every
candidate is a time when some feature is within the halo, so the result lies
between the first halo contact (gap - eps) / v and the tips' meeting time
gap / v plus the widening.  Status 1 is the sampling procedure's.
"""
import numpy as np

import oracle
from paper_2309_15417_gb300 import workloads as W


def _falling(h, v, eps, dt, spin=0.0):
    floor = [[-4.0, -4.0, 0.0], [4.0, -4.0, 0.0], [0.0, 4.0, 0.0]]
    tri = [[-0.5, -0.5, 0.0], [0.5, -0.5, 0.0], [0.0, 0.5, 0.0]]
    return W.single_triangles(floor, tri, pos_b=(0.0, 0.0, h), vel_b=(0.0, 0.0, -v), omega_b=(0.0, 0.0, spin),
                              eps=eps, dt=dt)


def test_flat_fall_closed_form():
    h, v, eps, dt = 0.1875, 128.0, 2.0 ** -6, 2.0 ** -9
    for spin in (0.0, 300.0):
        w = _falling(h, v, eps, dt, spin)
        pairs = np.array([[0, 1]], np.int32)
        r = oracle.collision_times_narrowing(w, pairs)
        assert r["status"][0] == 2 and r["tri_ab"][0].tolist() == [0, 0]
        expect = h / v + w.tol * dt
        assert abs(r["t_coll"][0] - expect) <= 1e-12 * dt, (spin, r["t_coll"][0], expect)
        assert 2 <= r["n_iter"][0] <= 4
        # the sampling procedure finds the first halo contact instead
        s = oracle.collision_times(w, pairs)
        assert s["status"][0] == 2
        assert (h - 2 * eps) / v <= s["t_coll"][0] <= (h - 2 * eps) / v + w.tol * dt


def test_head_on_bracket():
    eps, dt = 0.05, 1e-3
    for frac in (0.2, 0.5, 0.8):
        for vrel in (1.0, 40.0):
            gap = 2 * eps + frac * vrel * dt
            w = W.injected_head_on(gap, vrel, eps, dt, subdiv=2)
            pairs = np.array([[0, 1]], np.int32)
            r = oracle.collision_times_narrowing(w, pairs)
            t_first, t_meet = (gap - 2 * eps) / vrel, gap / vrel
            if t_first >= dt:
                continue
            assert r["status"][0] == 2
            assert t_first - 1e-15 <= r["t_coll"][0] <= min(t_meet, dt) + w.tol * dt + 1e-15


def test_status_one_and_zero_agree_with_sampling():
    """Pairs in contact at the start give status 1 in both procedures; a pair
    that slides past without contact gives status 0 in both."""
    w = W.small_icospheres(0)
    pairs = oracle.broad_phase(w)
    r = oracle.collision_times_narrowing(w, pairs)
    s = oracle.collision_times(w, pairs)
    one = s["status"] == 1
    assert one.any()
    assert np.array_equal(r["status"] == 1, one)
    assert np.array_equal(r["t_coll"][one], s["t_coll"][one])
    assert np.array_equal(r["tri_ab"][one], s["tri_ab"][one])
    # injected pair (4, 5) slides sideways just outside the halo sum
    k = int(np.where((pairs[:, 0] == 4) & (pairs[:, 1] == 5))[0][0])
    assert s["status"][k] == 0 and r["status"][k] == 0
    assert r["t_coll"][k] == s["t_coll"][k]


def test_translation_only_contacts_are_real():
    """Without rotation the relative path is exactly straight, so every
    contact the procedure reports is a time at which the exact pair distance
    is within the halo sum (checked with the narrow phase at that time, less
    the widening)."""
    w = W.dense_packing(3, nside=5, vsig=150.0, wsig=0.0)
    w.state[W.F_WX:W.F_WZ + 1] = 0.0
    pairs = oracle.broad_phase(w)
    r = oracle.collision_times_narrowing(w, pairs)
    two = np.where(r["status"] == 2)[0]
    assert len(two) > 3
    T = w.state[W.F_DT, 0]
    t_hit = r["t_coll"][two] - w.tol * T
    inside = t_hit <= T
    n = oracle.narrow_phase(w, pairs[two][inside], t_eval=t_hit[inside])
    # within the halo at the contact time (up to the rounding of the crossing time)
    eps_pair = 2 * w.state[W.F_EPS, 0]
    assert np.all(n["dmin"] <= eps_pair + 1e-9)
    # the statuses agree with the sampling procedure on this layout
    assert np.array_equal(r["status"], oracle.collision_times(w, pairs)["status"])
