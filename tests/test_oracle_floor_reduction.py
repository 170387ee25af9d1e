"""The reduced-floor oracle used by the full-size settling-column parity test
gives exactly the full-floor oracle's narrow phase, collision times and
contacts (small column, every floor pair; no GPU)."""
import numpy as np

import oracle
from floor_oracle import floor_pair_oracle
from paper_2309_15417_gb300 import workloads as W


def test_reduced_floor_equals_full_floor():
    w = W.settling_column(0, nside=6)
    w.state[W.F_VX:W.F_VZ + 1] *= 20.0  # larger motion bounds: more floor triangles kept
    floor = w.n - 1
    pairs = oracle.broad_phase(w)
    fl = pairs[pairs[:, 1] == floor]
    assert len(fl) >= 30
    on, oc = oracle.narrow_phase(w, fl), oracle.collision_times(w, fl)
    assert set(np.unique(oc["status"])) >= {0, 1}
    for q in range(len(fl)):
        r_on, r_oc, kept = floor_pair_oracle(w, int(fl[q, 0]), floor)
        assert kept < w.tri_counts()[floor]
        for key in ("flag", "tri_ab", "dmin", "pa", "pb"):
            assert np.array_equal(on[key][q:q + 1], r_on[key]), (q, key)
        assert oc["status"][q] == r_oc["status"][0] and oc["t_coll"][q] == r_oc["t_coll"][0]
        assert np.array_equal(oc["tri_ab"][q], r_oc["tri_ab"][0])
        assert np.array_equal(on["contacts"][on["contacts"][:, 0] == q][:, 1:], r_on["contacts"][:, 1:])
