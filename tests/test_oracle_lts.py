"""Pins of the oracle's local-time-stepping sweep (paper Section 2.2 substeps;
Section 3, Eq. "damped particle time step size"; Section 4, consolidation and
Eq. "cluster time step"; cluster masking and snapshot roll-over; the theorems
on valid snapshots and termination as invariants).

Closed forms use dyadic times and velocities, so every expected value is exact
in binary64; rotations are checked against scipy's Slerp.
"""
import numpy as np
from scipy.spatial.transform import Rotation, Slerp

import oracle
from paper_2309_15417_gb300 import workloads as W

XQT = [W.F_X, W.F_Y, W.F_Z, W.F_TCUR]


def _far_apart(n, spacing=50.0, v=(1.0, 0.0, 0.0)):
    """n single icospheres far apart from each other, moving with velocity v."""
    pos = np.stack([np.arange(n) * spacing, np.zeros(n), np.zeros(n)], axis=1)
    return W._assemble("far", [W.icosphere(1)], [0] * n, pos, np.tile(v, (n, 1)), [(1, 0, 0, 0)] * n,
                       np.zeros((n, 3)), 0.0, 1e-3, 0.01)


def _rot(state, p):
    q = state[W.F_QW:W.F_QZ + 1, p]
    return Rotation.from_quat([q[1], q[2], q[3], q[0]])


def test_damped_steps_masking_and_advance():
    """Three isolated particles: the step of each is min(2 (t_cur - t_old),
    dt_max) (dt_max without history); the earliest new time stamp masks the
    particle whose time stamp lies beyond it; the others advance to
    t_cur + step in free flight and roll their snapshots over."""
    dt_max = 2.0 ** -10
    w = _far_apart(3)
    w.state[W.F_TCUR] = [0.0, 2.0 ** -12, 2.0 ** -9]
    old = w.state.copy()
    old[W.F_TCUR] = [0.0, 2.0 ** -13, 2.0 ** -9 - 2.0 ** -14]
    cur0 = w.state.copy()
    r = oracle.lts_sweep(w, old, dt_max)
    steps = [dt_max, 2.0 ** -12, 2.0 ** -13]
    assert w.state[W.F_DT].tolist() == steps
    assert len(r["pairs"]) == 0 and r["ids"].tolist() == [0, 1, 2]
    assert r["t_global"] == 2.0 ** -11
    assert r["active"].tolist() == [1, 1, 0]
    for p in (0, 1):
        assert w.state[W.F_TCUR, p] == cur0[W.F_TCUR, p] + steps[p]
        assert w.state[W.F_X, p] == cur0[W.F_X, p] + 1.0 * steps[p]
        assert np.array_equal(old[XQT, p], cur0[XQT, p])  # rolled over
    assert np.array_equal(w.state[XQT, 2], cur0[XQT, 2])  # masked: unchanged
    assert r["rollbacks"] == 0


def test_gravity_and_stop_on_contact():
    """The stand-in update: a free particle gains g * step; a particle in
    contact stops (zero v and w)."""
    dt_max = 2.0 ** -10
    w = _far_apart(2)
    old = w.state.copy()
    oracle.lts_sweep(w, old, dt_max, gravity=(0.0, 0.0, -8.0))
    assert w.state[W.F_VZ].tolist() == [-8.0 * dt_max] * 2
    # two touching particles (centre distance 2 R - 0.001: meshes intersect)
    g = W.injected_head_on(-0.05, 0.5, 0.05, 1e-3)
    old = g.state.copy()
    r = oracle.lts_sweep(g, old, 1e-3, gravity=(0.0, 0.0, -8.0))
    assert r["status"].tolist() == [1]
    assert np.all(g.state[W.F_VX:W.F_VZ + 1] == 0.0) and np.all(g.state[W.F_WX:W.F_WZ + 1] == 0.0)


def test_consolidation_rolls_back_along_the_slerp():
    """Two particles of one cluster at different time stamps: the later one
    goes back to the earlier time stamp on the straight line and on the slerp
    geodesic between its snapshots (scipy Slerp), and both take the smaller
    step (Eq. "cluster time step")."""
    rng = np.random.default_rng(3)
    w = W._assemble("pair", [W.icosphere(1)], [0, 0], [(0, 0, 0), (2.0, 0, 0)],
                    [(0, 1.0, 0), (0, 1.0, 0)], [(1, 0, 0, 0)] * 2, np.zeros((2, 3)), 0.0, 1e-3, 0.01)
    old = w.state.copy()
    # particle 1 moved from t = 0 to t = h with velocity (0,1,0) and spin w1
    h = 2.0 ** -9
    old[W.F_WX:W.F_WZ + 1, 1] = rng.normal(0, 20.0, 3)
    old[W.F_QW:W.F_QZ + 1, 1] = W.random_quaternions(rng, 1)[0]
    old[W.F_TCUR, 1] = 0.0
    R1, X1 = oracle.pose(old, 1, h)
    q1 = Rotation.from_matrix(R1)
    w.state[W.F_X:W.F_Z + 1, 1] = X1
    w.state[W.F_QX:W.F_QZ + 1, 1] = q1.as_quat()[:3]
    w.state[W.F_QW, 1] = q1.as_quat()[3]
    w.state[W.F_WX:W.F_WZ + 1, 1] = old[W.F_WX:W.F_WZ + 1, 1]
    w.state[W.F_TCUR, 1] = h
    # particle 0 is at t = 2^-10 (step 2 (2^-10 - 2^-11) = 2^-10)
    w.state[W.F_TCUR, 0] = 2.0 ** -10
    old[W.F_TCUR, 0] = 2.0 ** -11
    old0 = old.copy()
    r = oracle.lts_sweep(w, old, 1e-3, zero_on_contact=False)
    t = 2.0 ** -10
    assert r["ids"].tolist() == [0, 0]
    assert r["rollbacks"] == 1 and r["rollbacks_before_old"] == 0
    assert w.state[W.F_DT].tolist() == [t, t]
    # the only cluster is the earliest: it advanced, and its old snapshot is
    # now the consolidated state at t
    assert r["active"].tolist() == [1, 1]
    assert old[W.F_TCUR].tolist() == [t, t]
    assert old[W.F_Y, 1] == 1.0 * t and old[W.F_X, 1] == 2.0
    ref = Slerp([0.0, h], Rotation.concatenate([_rot(old0, 1), q1]))([t])[0]
    assert np.max(np.abs(_rot(old, 1).as_matrix() - ref.as_matrix())) < 1e-13


def test_head_on_pair_advances_to_its_collision_time():
    """A head-on pair (vertex tips closing at speed vrel) and a far particle:
    the pair's cluster gets the collision time t* = (gap - eps_pair) / vrel
    (to the bisection tolerance) as its new time stamp, which masks nothing
    earlier; the far particle advances by its full step."""
    gap, vrel, eps, dt = 0.1 + 0.4e-3, 1.0, 0.05, 1e-3
    pair = W.injected_head_on(gap, vrel, eps, dt)
    far = _far_apart(1)
    w = W._assemble("pair+far", [W.icosphere(1)], [0, 0, 0],
                    np.concatenate([pair.state[0:3].T, [[100.0, 0, 0]]]),
                    np.concatenate([pair.state[3:6].T, [[1.0, 0, 0]]]),
                    np.concatenate([pair.state[6:10].T, [[1.0, 0, 0, 0]]]), np.zeros((3, 3)), 0.0, dt, eps)
    del far
    old = w.state.copy()
    r = oracle.lts_sweep(w, old, dt)
    tstar = (gap - 2 * eps) / vrel
    assert r["status"].tolist() == [2]
    tc = r["t_coll"][0]
    assert tstar <= tc <= tstar + w.tol * dt
    assert r["t_global"] == tc
    assert r["active"].tolist() == [1, 1, 1]
    assert w.state[W.F_TCUR].tolist() == [tc, tc, dt]
    # the colliding pair stops; the free particle keeps its velocity
    assert np.all(w.state[W.F_VX:W.F_VZ + 1, :2] == 0.0) and w.state[W.F_VX, 2] == 1.0


def _min_tcur(w):
    mv = w.is_static == 0
    return float(np.min(w.state[W.F_TCUR, mv]))


def test_invariants_over_sweeps():
    """Over several sweeps with gravity (small icospheres, a floor scene):
    no roll-back ever reaches before a particle's old snapshot (Theorem "valid
    snapshots"); the earliest time stamp grows every sweep (Theorem
    "termination"); t_old <= t_cur everywhere; static particles never change;
    exactly the clusters at or before the global minimum advance."""
    for w, dt_max in ((W.small_icospheres(1), 1e-3), (W.floor_scene(2), 1e-3)):
        old = w.state.copy()
        st0 = w.state[:, w.is_static == 1].copy()
        last = _min_tcur(w)
        for sweep in range(5):
            before = w.state.copy()
            r = oracle.lts_sweep(w, old, dt_max, gravity=(0.0, 0.0, -9.81))
            assert r["rollbacks_before_old"] == 0
            now = _min_tcur(w)
            assert now > last, sweep
            last = now
            mv = w.is_static == 0
            assert np.all(old[W.F_TCUR, mv] <= w.state[W.F_TCUR, mv])
            assert np.array_equal(w.state[:, w.is_static == 1], st0)
            adv = w.state[W.F_TCUR] != before[W.F_TCUR]
            assert np.array_equal(adv[mv], r["active"][mv].astype(bool))


# ----------------------------------------------------------------------------- space-time hoses

def _two_movers(p1, v1, p2, v2, R=0.5, eps=0.25, dt=2.0 ** -9):
    w = W._assemble("two", [W.icosphere(1)], [0, 0], [p1, p2], [v1, v2], [(1, 0, 0, 0)] * 2, np.zeros((2, 3)),
                    0.0, dt, eps)
    w.state[W.F_RADIUS] = R
    return w


def test_hose_parallel_and_following_movers():
    """The paper's motivating cases for Check 2: two fast particles moving in
    parallel, and one following the other, have overlapping swept spheres but
    hoses that never meet (constant separation above the radius sum)."""
    v = (1024.0, 0.0, 0.0)  # moves 2 over the step
    for w in (_two_movers((0, 0, 0), v, (0, 1.75, 0), v), _two_movers((0, 0, 0), v, (-1.75, 0, 0), v)):
        assert oracle.broad_phase(w).tolist() == [[0, 1]]
        assert not oracle.hose_meet(w.state, w.state, 0, 1)
    # approaching head on they meet
    w = _two_movers((0, 0, 0), v, (3.0, 0, 0), (-1024.0, 0.0, 0.0))
    assert oracle.hose_meet(w.state, w.state, 0, 1)


def test_hose_crossing_paths_closed_form():
    """Paths crossing at right angles at heights h apart: the closest approach
    is h at t = 1/k, so the hoses meet exactly when h <= r_i + r_j = 1.5."""
    k = 1024.0
    for h, expect in ((1.5, True), (1.5 + 2.0 ** -30, False), (1.0, True)):
        w = _two_movers((-1.0, 0, 0), (k, 0, 0), (0, -1.0, h), (0, k, 0))
        assert oracle.hose_meet(w.state, w.state, 0, 1) == expect, h


def test_hose_follows_the_old_segment():
    """Before its current time stamp a particle is on the straight segment
    from its old snapshot (not on a backward extrapolation of its current
    velocity): a particle that moved along +y during its previous step and now
    moves along +x passes through a resting particle at t = T/4."""
    T = 2.0 ** -9
    c = 2.0 ** 11
    w = _two_movers((0, 0, 0), (c, 0, 0), (0, -c * T / 4, 5.0), (0, 0, 0), R=0.125, eps=0.0625, dt=T)
    cur = w.state.copy()
    cur[W.F_TCUR, 0] = T / 2
    cur[W.F_Z, 1] = 0.0
    cur[W.F_Y, 1] = c * T / 4 - c * T / 2  # particle 0's position at T/4 on its old path
    old = cur.copy()
    old[W.F_TCUR, 0] = 0.0
    old[W.F_X, 0], old[W.F_Y, 0] = 0.0, -c * T / 2
    old[W.F_VX, 0], old[W.F_VY, 0] = 0.0, c
    assert oracle.hose_meet(cur, old, 0, 1)
    # the same current snapshot with a straight history (old = current) misses
    assert not oracle.hose_meet(cur, cur, 0, 1)


def test_hose_is_conservative():
    """At a common time stamp every moving pair that touches at some sampled
    time of its interval passes the hose test (the spheres cover the
    particles and their halos)."""
    for seed in range(2):
        w = W.small_icospheres(seed)
        w.state[W.F_VX:W.F_VZ + 1] *= 150.0
        pairs = oracle.broad_phase(w)
        hit = set()
        for t in np.linspace(0.0, 1e-3, 6):
            r = oracle.narrow_phase(w, pairs, t_eval=np.full(len(pairs), t))
            hit |= {tuple(p) for p, f in zip(pairs, r["flag"]) if f}
        kept = {tuple(p) for p in pairs if oracle.hose_meet(w.state, w.state, p[0], p[1])}
        assert len(hit) > 2 and hit <= kept
        assert len(kept) < len(pairs)  # the check removes some candidates


def test_lts_sweep_with_hoses_keeps_invariants():
    w = W.lts_mixed_steps(0, n=600)
    old = w.state.copy()
    last = None
    for sweep in range(3):
        r = oracle.lts_sweep(w, old, 4e-3, hose=True)
        assert r["rollbacks_before_old"] == 0
        now = float(np.min(w.state[W.F_TCUR]))
        assert last is None or now > last
        last = now
