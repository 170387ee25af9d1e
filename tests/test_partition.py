"""Spatial partition of a detection step over ranks (gloo, world sizes 2 and
3, on CPU): slabs along x with ghosts within the swept-sphere reach, pairs
owned by the rank of their first member, and the label-min cluster merge.
The per-rank compute is the oracle here (on GPUs it is the CUDA library); the
union of the ranks' results must equal the single-domain oracle bit for bit:
candidate pairs (each owned once), narrow phase, collision times, clusters."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _workload(name):
    from paper_2309_15417_gb300 import workloads as W
    if name == "column":
        return W.settling_column(0, nside=5)  # a static floor held by every rank
    if name == "dense":
        return W.dense_packing(1, nside=7, subdiv=1, vsig=2.0, wsig=2.0, dt=1e-2)
    return W.small_icospheres(0)


class OracleCompute:
    def broad_phase(self, w):
        import oracle
        return oracle.broad_phase(w)

    def narrow_phase(self, w, pairs):
        import oracle
        return oracle.narrow_phase(w, pairs, n_threads=1)

    def collision_times(self, w, pairs):
        import oracle
        return oracle.collision_times(w, pairs, n_threads=1)


def _worker(rank, world, port, name, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2309_15417_gb300 import partition as Pn
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def allreduce_min(a):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.int64))
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        return t.numpy().copy()

    try:
        w = _workload(name)
        r = Pn.detect_step(w, rank, world, OracleCompute(), allreduce_min)
        q.put((rank, r["pairs"], {k: r["narrow"][k] for k in ("dmin", "flag", "tri_ab", "contacts")},
               {k: r["ctime"][k] for k in ("status", "t_coll", "tri_ab")}, r["ids"], r["rounds"],
               len(r["slab"].owned), len(r["slab"].local)))
    except Exception as e:  # report instead of hanging the other ranks' collectives
        q.put((rank, repr(e)))
        raise
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("world,name", [(2, "column"), (3, "dense"), (2, "small")])
def test_partitioned_step_equals_single_domain_oracle(world, name):
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, name, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=600) for _ in ps]
    for p in ps:
        p.join(timeout=120)
    for r in res:
        assert len(r) > 2, f"rank {r[0]} failed: {r[1]}"
    assert all(p.exitcode == 0 for p in ps)
    res.sort(key=lambda r: r[0])
    w = _workload(name)
    ref = oracle.broad_phase(w)
    on = oracle.narrow_phase(w, ref)
    oc = oracle.collision_times(w, ref)
    oid, _ = oracle.clusters(w.n, ref, w.is_static)
    # every global pair owned by exactly one rank
    allp = np.concatenate([r[1] for r in res])
    order = np.lexsort((allp[:, 1], allp[:, 0]))
    assert np.array_equal(allp[order], ref)
    row = {(int(i), int(j)): k for k, (i, j) in enumerate(ref)}
    contacts = []
    for rank, pairs, nar, ct, ids, rounds, n_own, n_loc in res:
        g = np.array([row[(int(i), int(j))] for i, j in pairs], np.int64)
        if len(g):
            assert np.array_equal(nar["dmin"], on["dmin"][g])
            assert np.array_equal(nar["flag"], on["flag"][g])
            assert np.array_equal(nar["tri_ab"], on["tri_ab"][g])
            assert np.array_equal(ct["status"], oc["status"][g])
            assert np.array_equal(ct["t_coll"], oc["t_coll"][g])
            assert np.array_equal(ct["tri_ab"], oc["tri_ab"][g])
            c = nar["contacts"].copy()
            c[:, 0] = g[c[:, 0]]
            contacts.append(c)
        # every rank ends with the same, global cluster ids
        assert np.array_equal(ids, oid)
        assert n_own < w.n and n_loc <= w.n
    c = np.concatenate(contacts) if contacts else np.zeros((0, 3), np.int32)
    c = c[np.lexsort((c[:, 2], c[:, 1], c[:, 0]))]
    assert np.array_equal(c, on["contacts"])
    assert sum(r[6] for r in res) == int((w.is_static == 0).sum())  # the slabs split the moving particles


def test_cluster_merge_needs_several_rounds_across_slabs():
    """A path graph whose edges alternate between two ranks: the label-min
    rounds converge to the path's smallest index on both."""
    sys.path.insert(0, ROOT)
    from paper_2309_15417_gb300 import partition as Pn
    n = 12
    st = np.zeros(n, np.uint8)
    edges = np.array([[k, k + 1] for k in range(n - 1)], np.int32)
    parts = [edges[0::2], edges[1::2]]
    comps = [Pn.local_components(n, st, e) for e in parts]
    labs = [np.arange(n, dtype=np.int64) for _ in parts]
    rounds = 0
    while True:  # the two ranks' rounds in lockstep, all-reduce = element-wise minimum
        rounds += 1
        cand = []
        for comp, lab in zip(comps, labs):
            cmin = np.full(n, np.iinfo(np.int64).max)
            np.minimum.at(cmin, comp, lab)
            cand.append(cmin[comp])
        new = np.minimum(*cand)
        if all(np.array_equal(new, lab) for lab in labs):
            break
        labs = [new.copy() for _ in parts]
    assert (labs[0] == 0).all() and rounds > 3
