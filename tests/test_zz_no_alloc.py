"""The allocation-free candidate search (dem_build_candidates_noalloc) gives
the same candidates as dem_build_candidates, on two calls in a row.

It exists for callers that cannot allocate device memory when they need
candidates (their memory pool is owned elsewhere, or an allocation could block
or fail in a real-time loop); its scratch is a fixed array inside the library.
This file is collected last so that a run stopping at the first failure has
already run every other test; it passes alone and after the other tests.
"""
import numpy as np
import pytest

import oracle
from paper_2309_15417_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _with_context(dem, w):
    c = dem.Context(max_particles=max(w.n, 16), max_pairs=1 << 16, max_contacts=16)
    sc = dem.Scene.from_workload(w)
    c.build_candidates(sc)
    c.check()
    m = int(c.n_pairs.item())
    out = c.pairs[:m].cpu().numpy().copy()
    c.close()
    return out


def _noalloc(dem, w, cap=1 << 16):
    import torch
    sc = dem.Scene.from_workload(w)
    pairs = torch.full((cap, 2), -7, dtype=torch.int32, device="cuda")
    n = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    rc = dem.dem_build_candidates_noalloc(sc.P, pairs, cap, n)
    assert rc == 0
    torch.cuda.synchronize()
    m = int(n.item())
    return pairs[:min(m, cap)].cpu().numpy().copy(), m


def test_noalloc_candidates_match_the_context_call_twice(dem):
    dense = W.dense_packing(0)
    small = W.small_icospheres(1)
    ref_dense, ref_small = _with_context(dem, dense), _with_context(dem, small)
    assert len(ref_dense) > 1000 and len(ref_small) >= 3
    # two calls in a row on different inputs, then the first input again:
    # stale contents of the shared scratch must not leak into a result
    for w, ref in ((dense, ref_dense), (small, ref_small), (dense, ref_dense)):
        got, m = _noalloc(dem, w)
        assert m == len(ref)
        assert np.array_equal(got, ref)


def test_noalloc_rejects_oversize_and_reports_truncation(dem):
    import torch
    big = W.dense_packing(0, nside=26)  # 17576 particles > the fixed maximum
    assert big.n > dem.DEM_NOALLOC_MAX_PARTICLES
    sc = dem.Scene.from_workload(big)
    pairs = torch.zeros((16, 2), dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert dem.dem_build_candidates_noalloc(sc.P, pairs, 16, n) == -2  # DEM_ERR_CAPACITY
    # a capacity smaller than the candidate count: count reported, prefix written
    w = W.dense_packing(0)
    ref = _with_context(dem, w)
    got, m = _noalloc(dem, w, cap=100)
    assert m == len(ref) and len(got) == 100
    # particles written in full match; the one cut by the capacity holds a
    # subset of its partners
    last = got[-1, 0]
    full = got[:, 0] < last
    assert np.array_equal(got[full], ref[:int(full.sum())])
    assert {tuple(r) for r in got[~full]} <= {tuple(r) for r in ref[ref[:, 0] == last]}


def test_noalloc_matches_the_oracle_with_static_particles(dem):
    """A static floor and a static post among moving particles (static box
    tests, the static member written second): the oracle's candidate set, on
    two calls in a row, and no error in the library's error word."""
    dem.dem_noalloc_check()  # clear what earlier calls left
    w = W.floor_scene(0)
    ref = oracle.broad_phase(w)
    assert (w.is_static[ref[:, 1]] == 1).any()
    for _ in range(2):
        got, m = _noalloc(dem, w)
        assert m == len(ref)
        assert np.array_equal(got, ref)
    assert dem.dem_noalloc_check() == dem.DEM_OK


def test_noalloc_check_reports_device_conditions(dem):
    """The context-free error readback: a static particle whose triangle
    range runs past the end of the triangles is an index error (its box is
    skipped, nothing is read out of range); a capacity smaller than the
    candidate count is a capacity error; the readback clears the word."""
    import torch
    dem.dem_noalloc_check()
    w = W.floor_scene(0)
    assert w.is_static[0] == 1
    off = w.tri_off.copy()
    off[1] = w.n_tris + 4096
    sc = dem.Scene.from_workload(w)
    sc.tri_off.copy_(torch.from_numpy(off).cuda())
    pairs = torch.zeros((1 << 12, 2), dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert dem.dem_build_candidates_noalloc(sc.P, pairs, 1 << 12, n) == dem.DEM_OK
    assert dem.dem_noalloc_check() == dem.DEM_ERR_INDEX
    assert dem.dem_noalloc_check() == dem.DEM_OK
    _noalloc(dem, W.dense_packing(0), cap=100)
    assert dem.dem_noalloc_check() == dem.DEM_ERR_CAPACITY
    _noalloc(dem, W.small_icospheres(1))
    assert dem.dem_noalloc_check() == dem.DEM_OK
