#!/usr/bin/env python
"""Benchmark of the space-time contact-detection step on GB300.

One step = one pass of the whole path over the dense packing of 1,000
icospheres (320 triangles, radius 1; jittered simple-cubic lattice at volume
fraction 0.5, jitter +-0.1; dt = 1e-4, eps = 0.02; K = 8 samples, bisection to
1e-3 of the step): candidate pairs -> narrow phase at the pair start ->
collision times -> clusters of the candidate graph, all four through the C-ABI
library, FP32 distances with binary64 recomputation.

Metric: triangle-pair distance checks per second as the method defines them
(per candidate pair T_i * T_j for the narrow phase plus T_i * T_j for every
pair-distance evaluation of the collision-time search), plus particle-steps
per second, and the same step with every distance in FP64 for comparison.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (launched with torch.distributed.run): every rank runs an independent
replica (its own seeded packing) -- weak scaling, no collective on the data
path; value = checks of all ranks / max time over ranks.
--impl reference: the FP64 CPU oracle on this machine's cores, same workload,
each step on a bounded sample of the candidate pairs.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "triangle-pair distance checks/sec and particle-steps/sec at 1 GB300, FP32+fixup vs all-FP64"
UNIT = "triangle-pair checks/s"
WORKLOAD = ("dense packing: 1000 icospheres (subdivision 2, 320 triangles, r=1), jittered simple-cubic "
            "lattice at volume fraction 0.5 (jitter +-0.1), v~N(0,0.2), w~N(0,0.2), dt=1e-4, eps=0.02; "
            "K=8 samples then bisection to 1e-3 of the step; FP32 distances with FP64 recomputation")
L2_BYTES = 129 * 1024 * 1024
FLUSH_BYTES = 512 * 1024 * 1024

# FP32 operations per unit of work of the collision-time kernel (FMA = 2), counted
# from the formulas in csrc/geom.cuh and csrc/pairs.cu on their common path:
#   triangle-sphere test: 3 sub, |d|^2 (mul + 2 fma), 2 add, 1 mul, 1 compare  -> 12
#   group-sphere test: as above plus sqrt                                     -> 13
#   triangle-pair distance: 6 segment-triangle crossing tests (31 each, no crossing),
#   6 vertex-triangle closest points (~90 each, face region), 9 segment-segment
#   closest points (~65 each)                                                -> 1311
F_SPHERE = 12
F_GROUP = 13
F_DIST32 = 1311
# FP32 peak: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2070 MHz maximum SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "detect_kernel_dense1000.md")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-fp64", action="store_true", help="skip the all-FP64 comparison")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    p.add_argument("--cpu-sample", type=int, default=96, help="candidate pairs per oracle sample")
    p.add_argument("--no-lts", action="store_true", help="skip the local-time-stepping measurements")
    p.add_argument("--no-narrowing", action="store_true", help="skip the narrowing-vs-sampling comparison")
    p.add_argument("--column-sweeps", type=int, default=50, help="sweeps of the settling column per replay")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples during the timed region (clock, max clock, reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ GPU arm

def _profile_traffic():
    """DRAM bytes per launch of the fused pair kernel from the committed
    ncu summary, if it was taken on the current kernel source."""
    try:
        txt = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", txt)
    if not m or not h:
        return None
    src = open(os.path.join(ROOT, "paper_2309_15417_gb300", "csrc", "pair_kernel.cuh"), "rb").read()
    geo = open(os.path.join(ROOT, "paper_2309_15417_gb300", "csrc", "geom.cuh"), "rb").read()
    if hashlib.sha256(src + geo).hexdigest() != h.group(1):
        return None
    return float(m.group(1))


def run_step(ctx, sc, ev=None, fused=True):
    """One detection step: candidates, narrow phase at the pair start and
    collision times (fused: one dem_detect launch; else the two calls),
    clusters.  Optional events: before the narrow phase, between the two calls
    (not fused), after the collision times."""
    ctx.build_candidates(sc)
    if ev:
        ev[0].record()
    if fused:
        ctx.detect(sc)
        if ev:
            ev[1].record()
    else:
        ctx.narrow_phase(sc)
        if ev:
            ev[1].record()
        ctx.collision_times(sc)
    if ev:
        ev[2].record()
    ctx.clusters(sc)


def gpu_arm(args, rank, world, local):
    import torch
    from paper_2309_15417_gb300 import dem
    from paper_2309_15417_gb300 import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = W.dense_packing(args.seed + rank)
    sc = dem.Scene.from_workload(w, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    mk = lambda prec: dem.Context(K=w.K, tol=w.tol, precision=prec, max_particles=w.n, max_pairs=1 << 16,
                                  max_contacts=1 << 20, device=dev)

    def measure(prec, steps, warmup, detail, fused=True):
        """Stage split from direct calls (CUDA events between the calls), then
        the timed steps as replays of the step captured in a CUDA graph."""
        ctx = mk(prec)
        for _ in range(warmup):
            run_step(ctx, sc, fused=fused)
        ctx.check()
        ctx.stats(reset=True)
        # stage split: direct calls
        nsplit = max(3, min(steps, 10))
        E = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(nsplit)]
        for k in range(nsplit):
            flush.fill_(float(k))
            e = E[k]
            e[0].record()
            run_step(ctx, sc, ev=(e[1], e[2], e[3]), fused=fused)
            e[4].record()
        torch.cuda.synchronize()
        ct_ms = [e[2].elapsed_time(e[3]) for e in E]
        nw_ms = [e[1].elapsed_time(e[2]) for e in E]
        det_ms = [e[1].elapsed_time(e[3]) for e in E]
        direct_ms = [e[0].elapsed_time(e[4]) for e in E]
        # the whole step as one CUDA graph
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            run_step(ctx, sc, fused=fused)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        l0 = ctx.stats()["kernel_launches"]
        with torch.cuda.graph(g):
            run_step(ctx, sc, fused=fused)
        launches_step = ctx.stats()["kernel_launches"] - l0
        g.replay()
        torch.cuda.synchronize()
        ctx.check()
        ctx.stats(reset=True)
        G = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clk = ClockSampler(local) if detail else None
        if clk:
            clk.start()
        t0 = time.perf_counter()
        for k in range(steps):
            flush.fill_(float(k))  # L2 flush between steps, outside the timed events
            G[k][0].record()
            g.replay()
            G[k][1].record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if world > 1:
            torch.distributed.barrier()
        clocks = clk.stop() if clk else None
        ctx.check()
        st = ctx.stats(reset=True)
        st["kernel_launches"] = launches_step * steps
        step_ms = [e[0].elapsed_time(e[1]) for e in G]
        return ctx, dict(step_ms=step_ms, ct_ms=ct_ms, nw_ms=nw_ms, det_ms=det_ms, stats=st, wall=wall,
                         clocks=clocks, direct_ms=direct_ms, graph=g)

    ctx32, r32 = measure(dem.DEM_PREC_FP32_FIXUP, args.steps, args.warmup, True)
    K = args.steps
    checks_step = r32["stats"]["method_checks"] / K
    t_total = sum(r32["step_ms"]) / 1e3
    n_pairs = int(ctx32.n_pairs.item())

    # dominant kernel (the fused pair kernel of dem_detect): counters of one
    # call alone, duration from the events around dem_detect
    ctx32.stats(reset=True)
    run_step(ctx32, sc)
    torch.cuda.synchronize()
    ctx32.stats(reset=True)
    ctx32.detect(sc)
    st_ct = ctx32.stats(reset=True)
    ct_flops = F_SPHERE * st_ct["sphere_tests"] + F_GROUP * st_ct["group_tests"] + F_DIST32 * st_ct["dist_fp32"]
    ct_ms = float(np.mean(r32["det_ms"]))
    achieved = ct_flops / (ct_ms / 1e3) / 1e12
    # the same step through the four separate calls (narrow phase and
    # collision times as two launches)
    ctx4, r4 = measure(dem.DEM_PREC_FP32_FIXUP, max(3, min(K, 10)), 2, False, fused=False)
    four_call = {"ms_per_step": float(np.mean(r4["step_ms"])), "narrow_ms": float(np.mean(r4["nw_ms"])),
                 "collision_times_ms": float(np.mean(r4["ct_ms"]))}
    ctx4.close()

    # FP32 error against FP64 (pair minima), R = 1
    fin = torch.isfinite(ctx32.dmin[:n_pairs])
    d64 = ctx32.dmin[:n_pairs][fin]
    d32 = ctx32.dmin32[:n_pairs][fin].double()
    err = (d32 - d64).abs().cpu().numpy()
    fp32_err = {"max_abs_over_R": float(err.max()) if err.size else 0.0,
                "p99_abs_over_R": float(np.percentile(err, 99)) if err.size else 0.0,
                "output": "pair minimum distance"}

    fp64 = None
    if not args.no_fp64:
        k64 = max(3, min(K, 5))
        ctx64, r64 = measure(dem.DEM_PREC_FP64, k64, 2, False)
        t64 = sum(r64["step_ms"]) / 1e3
        c64 = r64["stats"]["method_checks"] / k64
        # same contact set and collision times in both precisions
        m = int(ctx64.n_pairs.item())
        same = (m == n_pairs and torch.equal(ctx64.flag[:m], ctx32.flag[:m])
                and torch.equal(ctx64.status[:m], ctx32.status[:m])
                and torch.equal(ctx64.t_coll[:m], ctx32.t_coll[:m])
                and int(ctx64.n_contacts.item()) == int(ctx32.n_contacts.item())
                and torch.equal(ctx64.contacts[:int(ctx64.n_contacts.item())],
                                ctx32.contacts[:int(ctx32.n_contacts.item())]))
        fp64 = {"value": c64 * k64 / t64, "unit": UNIT, "ms_per_step": t64 * 1e3 / k64,
                "speedup_fp32_fixup_over_fp64": (checks_step * K / t_total) / (c64 * k64 / t64),
                "results_identical": bool(same), "steps": k64}
        if same:
            # FP32 error of the contact list: the FP32+fixup run keeps the FP32
            # distance and points of contacts outside the band; the FP64 run
            # has the same contact keys with binary64 geometry (R = 1).  The
            # points of (near-)parallel triangles are not unique, so a point
            # difference can also be a different valid point.
            nc = int(ctx32.n_contacts.item())
            g32, g64 = ctx32.contact_geom[:nc], ctx64.contact_geom[:nc]
            ed = (g32[:, 0] - g64[:, 0]).abs().cpu().numpy()
            ep = torch.maximum((g32[:, 1:4] - g64[:, 1:4]).norm(dim=1),
                               (g32[:, 4:7] - g64[:, 4:7]).norm(dim=1)).cpu().numpy()
            if nc:
                fp32_err["contact_distance"] = {"max_abs_over_R": float(ed.max()),
                                                "p99_abs_over_R": float(np.percentile(ed, 99))}
                fp32_err["contact_points"] = {"max_abs_over_R": float(ep.max()),
                                              "p99_abs_over_R": float(np.percentile(ep, 99)),
                                              "note": "largest of |pa32 - pa64|, |pb32 - pb64| per contact"}
        ctx64.close()

    # end to end through the public API from pinned host buffers
    e2e = e2e_arm(dem, w, ctx32, sc, max(3, min(K, 10)), r32["graph"])

    res = dict(value_local=checks_step * K, time_local=t_total, particles=w.n, K=K, n_pairs=n_pairs,
               ms=float(np.mean(r32["step_ms"])), ct_ms=ct_ms, four_call=four_call,
               direct_ms=float(np.mean(r32["direct_ms"])),
               achieved=achieved, ct_flops=ct_flops, st_ct=st_ct, clocks=r32["clocks"], wall=r32["wall"],
               launches=r32["stats"]["kernel_launches"], fp32_err=fp32_err, fp64=fp64, e2e=e2e,
               checks_step=checks_step, stats_step={k: v / K for k, v in r32["stats"].items()})
    ctx32.close()
    del sc, flush
    torch.cuda.empty_cache()
    # the further legs (not part of the timed step) run on a single GPU only,
    # so that a multi-GPU run does not hold its GPUs for them
    if world == 1 and not args.no_lts:
        res["lts"] = lts_legs(args, dem, W, dev)
    if world == 1 and not args.no_narrowing:
        res["narrowing"] = narrowing_leg(args, dem, W, dev)
    return res


def lts_measure(dem, w, old_np, prec, sweeps, reps, dt_max, gravity, dev, max_pairs, hose=False):
    """Sweeps of the local-time-stepping cycle captured in one CUDA graph and
    replayed `reps` times from the same starting snapshots (restored between
    replays, outside the timed events).  Returns times, counters and the final
    snapshots."""
    import torch
    sc = dem.Scene.from_workload(w, device=dev)
    old = torch.from_numpy(old_np).to(dev)
    cur0, old0 = sc.state.clone(), old.clone()
    ctx = dem.Context(K=w.K, tol=w.tol, precision=prec, max_particles=w.n, max_pairs=max_pairs,
                      max_contacts=1 << 16, max_triangles=w.n_tris, device=dev)
    ctx.lts_sweep(sc, old, dt_max, gravity=gravity, hose=hose)  # first call outside the capture
    torch.cuda.synchronize()
    ctx.check()
    l0 = ctx.stats()["kernel_launches"]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(sweeps):
            ctx.lts_sweep(sc, old, dt_max, gravity=gravity, hose=hose)
    launches = ctx.stats()["kernel_launches"] - l0
    ms, st = [], {}
    for r in range(reps + 1):  # the first replay warms up
        sc.state.copy_(cur0)
        old.copy_(old0)
        torch.cuda.synchronize()
        ctx.stats(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        if r:
            ms.append(e0.elapsed_time(e1))
            for k, v in ctx.stats(reset=True).items():  # counters of every timed replay
                st[k] = st.get(k, 0) + v
    ctx.check()
    st = {k: v / reps for k, v in st.items()}  # per replay
    out = dict(ms=float(np.mean(ms)), stats=st, launches=launches, pairs=int(ctx.n_pairs.item()),
               clusters=int(ctx.n_clusters.item()), cur=sc.state.cpu().numpy(), old=old.cpu().numpy(),
               t_min=float(sc.state[13][torch.from_numpy(w.is_static == 0).to(dev)].min().item()))
    ctx.close()
    del sc, old, cur0, old0, g
    torch.cuda.empty_cache()
    return out


def narrowing_leg(args, dem, W, dev, reps=10):
    """Collision times by the paper's narrowing against K samples + bisection
    on the same candidate pairs: time per call (CUDA events, L2 flushed
    between calls), method checks/s, and how the two procedures' answers
    compare (statuses; for pairs with status 2 in both, the narrowing time
    minus the sampling time, in units of the pair's step)."""
    import torch
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    out = {}
    cases = (("dense-packing-1000 (the benchmark workload)", W.dense_packing(args.seed)),
             ("fast dense packing: 5^3 icospheres (320 triangles), v ~ N(0,150), w ~ N(0,150), dt = 1e-4",
              W.dense_packing(args.seed + 3, nside=5, vsig=150.0, wsig=150.0)))
    for name, w in cases:
        sc = dem.Scene.from_workload(w, device=dev)
        res = {}
        for method, key in ((dem.DEM_CTIME_SAMPLES, "samples_bisection"), (dem.DEM_CTIME_NARROWING, "narrowing")):
            ctx = dem.Context(K=w.K, tol=w.tol, precision=dem.DEM_PREC_FP32_FIXUP, max_particles=w.n,
                              max_pairs=1 << 16, max_contacts=1 << 20, ctime_method=method, device=dev)
            ctx.build_candidates(sc)
            ctx.collision_times(sc)
            torch.cuda.synchronize()
            ctx.stats(reset=True)
            ms = []
            for k in range(reps):
                flush.fill_(float(k))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                ctx.collision_times(sc)
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            ctx.check()
            st = ctx.stats(reset=True)
            m = int(ctx.n_pairs.item())
            res[key] = dict(ms=float(np.mean(ms)), checks_per_s=st["method_checks"] / (sum(ms) / 1e3),
                            status=ctx.status[:m].cpu().numpy(), t=ctx.t_coll[:m].cpu().numpy(), pairs=m)
            ctx.close()
        a, b = res["samples_bisection"], res["narrowing"]
        both2 = (a["status"] == 2) & (b["status"] == 2)
        T = float(w.state[W.F_DT, 0])
        d = (b["t"][both2] - a["t"][both2]) / T
        out[name] = {
            "candidate_pairs": a["pairs"],
            "samples_bisection": {"ms": a["ms"], "checks_per_s": a["checks_per_s"],
                                  "status_counts": np.bincount(a["status"], minlength=3).tolist()},
            "narrowing": {"ms": b["ms"], "checks_per_s": b["checks_per_s"],
                          "status_counts": np.bincount(b["status"], minlength=3).tolist()},
            "same_status": int((a["status"] == b["status"]).sum()),
            "status2_in_both": int(both2.sum()),
            "t_narrowing_minus_t_sampling_over_T": {"mean": float(d.mean()) if d.size else None,
                                                    "min": float(d.min()) if d.size else None,
                                                    "max": float(d.max()) if d.size else None}}
        del sc
    del flush
    torch.cuda.empty_cache()
    return out


def lts_legs(args, dem, W, dev):
    """The local-time-stepping measurements: one cycle on the 100,000-particle
    mixed-step layout, and 50 sweeps of the 1,000,000-particle settling column
    in FP32 + fixup and in all-FP64 (final snapshots compared bit for bit)."""
    res = {}
    # one cycle, 100k particles; the log-uniform steps are the particles'
    # histories: t_old = t_cur - dt_p / alpha, so the damped step is dt_p
    w = W.lts_mixed_steps(args.seed)
    old = w.state.copy()
    old[W.F_TCUR] = w.state[W.F_TCUR] - w.state[W.F_DT] / 2.0
    r = lts_measure(dem, w, old, dem.DEM_PREC_FP32_FIXUP, 1, 5, 1e-2, (0.0, 0.0, 0.0), dev, 1 << 20)
    st = r["stats"]
    res["lts_cycle_100k"] = {
        "workload": "lts-100k: 100,000 icospheres (320 triangles), 20% FCC blobs at volume fraction 0.55, 80% "
                    "free at 0.02; particle steps log-uniform in [1e-5, 1e-2] as step histories "
                    "(t_old = t_cur - dt/2, alpha = 2, dt_max = 1e-2)",
        "ms_per_cycle": r["ms"], "cuda_graph": "one sweep (step sizes, candidates, clusters, consolidation, "
                                               "collision times, masking, advance) captured as one graph",
        "particle_steps_per_s": st["advances"] / (r["ms"] / 1e3),
        "checks_per_s": st["method_checks"] / (r["ms"] / 1e3),
        "advances_per_cycle": st["advances"], "candidate_pairs": r["pairs"], "clusters": r["clusters"],
        "kernels_per_cycle": r["launches"]}
    # the same cycle with the space-time hose check (Check 2) in the broad phase
    rh = lts_measure(dem, w, old, dem.DEM_PREC_FP32_FIXUP, 1, 5, 1e-2, (0.0, 0.0, 0.0), dev, 1 << 20, hose=True)
    res["lts_cycle_100k"]["with_hose_check"] = {
        "ms_per_cycle": rh["ms"], "candidate_pairs": rh["pairs"], "clusters": rh["clusters"],
        "advances_per_cycle": rh["stats"]["advances"],
        "final_snapshots_identical_to_without": bool(np.array_equal(rh["cur"], r["cur"]) and
                                                     np.array_equal(rh["old"], r["old"]))}
    del w, old, r, rh
    # the settling column: sweeps in a graph, both precisions
    S = args.column_sweeps
    w = W.settling_column(args.seed)
    col = {}
    for prec, name in ((dem.DEM_PREC_FP32_FIXUP, "fp32_fixup"), (dem.DEM_PREC_FP64, "fp64")):
        r = lts_measure(dem, w, w.state.copy(), prec, S, 1, 1e-3, (0.0, 0.0, -9.81), dev, 1 << 21)
        st = r["stats"]
        col[name] = dict(ms_per_sweep=r["ms"] / S, particle_steps_per_s=st["advances"] / (r["ms"] / 1e3),
                         checks_per_s=st["method_checks"] / (r["ms"] / 1e3), advances=st["advances"],
                         last_sweep_pairs=r["pairs"], earliest_t_after=r["t_min"], kernels=r["launches"],
                         final=(r["cur"], r["old"]))
    same = bool(np.array_equal(col["fp32_fixup"]["final"][0], col["fp64"]["final"][0]) and
                np.array_equal(col["fp32_fixup"]["final"][1], col["fp64"]["final"][1]))
    for v in col.values():
        del v["final"]
    res["settling_column_1m"] = {
        "workload": "settling column: 100^3 icospheres (half 80, half 320 triangles), lattice spacing 2.2, "
                    "jitter +-0.1, over a static 316x316-quad floor (199,712 triangles); eps = 0.01, "
                    "dt_max = 1e-3, gravity (0,0,-9.81), particles in contact stop (stand-in update)",
        "sweeps": S, "cuda_graph": f"{S} sweeps captured in one graph", **col,
        "speedup_fp32_fixup_over_fp64": col["fp64"]["ms_per_sweep"] / col["fp32_fixup"]["ms_per_sweep"],
        "final_snapshots_identical": same}
    return res


def e2e_arm(dem, w, ctx, sc, steps, graph):
    """Through the public API from pinned host buffers: host-to-device copies
    of the particle data into the scene the step graph was captured on, the
    step, device-to-host copies of every output."""
    import torch
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_state, h_static, h_off, h_tris = pin(w.state), pin(w.is_static), pin(w.tri_off), pin(w.tris)
    h_out = {}
    bi = sum(t.numel() * t.element_size() for t in (h_state, h_static, h_off, h_tris))
    times, bo = [], 0
    for k in range(steps + 2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sc.state.copy_(h_state, non_blocking=True)
        sc.is_static.copy_(h_static, non_blocking=True)
        sc.tri_off.copy_(h_off, non_blocking=True)
        sc.tris.copy_(h_tris, non_blocking=True)
        graph.replay()
        m = int(ctx.n_pairs.item())
        nc = min(int(ctx.n_contacts.item()), ctx.max_contacts)
        outs = [ctx.pairs[:m], ctx.flag[:m], ctx.dmin[:m], ctx.tri_ab[:m], ctx.t_coll[:m], ctx.status[:m],
                ctx.ct_ab[:m], ctx.cluster_id[:w.n], ctx.n_clusters, ctx.contacts[:nc], ctx.contact_geom[:nc]]
        host = [t.to("cpu", non_blocking=True) for t in outs]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if k >= 2:
            times.append(dt)
            bo = 2 * 8 + sum(t.numel() * t.element_size() for t in host)
        h_out = host
    ctx.check()
    st = ctx.stats(reset=True)
    checks = st["method_checks"] / (steps + 2)
    h_out.clear()
    return {"value": checks / float(np.mean(times)), "unit": UNIT, "h2d_bytes_per_step": int(bi),
            "d2h_bytes_per_step": int(bo), "ms_per_step": 1e3 * float(np.mean(times))}


# ------------------------------------------------------------------ CPU oracle

def cpu_sample(w, pairs, n_sample, seed):
    import oracle
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(len(pairs), min(n_sample, len(pairs)), replace=False))
    sp = pairs[idx]
    cnt = np.diff(w.tri_off)
    nt = oracle.default_threads()
    t0 = time.perf_counter()
    bp = oracle.broad_phase(w)
    r = oracle.narrow_phase(w, sp, n_threads=nt)
    c = oracle.collision_times(w, sp, n_threads=nt)
    ids, ncl = oracle.clusters(w.n, bp, w.is_static)
    dt = time.perf_counter() - t0
    tt = (cnt[sp[:, 0]] * cnt[sp[:, 1]]).astype(np.float64)
    checks = float(np.sum(tt * (1 + c["n_evals"])))
    return checks, dt, nt, len(sp), len(pairs)


def cpu_baseline(args, w=None):
    import oracle
    from paper_2309_15417_gb300 import workloads as W
    w = w or W.dense_packing(args.seed)
    pairs = oracle.broad_phase(w)
    checks, dt, nt, ns, npairs = cpu_sample(w, pairs, args.cpu_sample, args.seed)
    return {"value": checks / dt, "unit": UNIT, "cores": nt, "kind": "oracle",
            "sample": f"{ns} of {npairs} candidate pairs (narrow phase + collision times, every triangle pair "
                      f"in FP64); broad phase and clusters over all {w.n} particles",
            "seconds": dt}


def reference_arm(args, rank, world):
    """The FP64 CPU oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    from paper_2309_15417_gb300 import workloads as W
    oracle.build()
    w = W.dense_packing(args.seed)
    pairs = oracle.broad_phase(w)
    for k in range(args.warmup):
        cpu_sample(w, pairs, max(4, args.cpu_sample // 8), args.seed + 100 + k)
    tot_c, tot_t, nt, ns = 0.0, 0.0, 1, 0
    for k in range(args.steps):
        c, t, nt, ns, _ = cpu_sample(w, pairs, max(4, args.cpu_sample // 4), args.seed + k)
        tot_c += c
        tot_t += t
    v = tot_c / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "impl": "FP64 CPU oracle"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": nt, "kind": "oracle",
                             "sample": f"per step {ns} of {len(pairs)} candidate pairs (narrow phase + collision "
                                       f"times); broad phase and clusters over all {w.n} particles"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the contact-detection path has no CPU fallback)")
    from paper_2309_15417_gb300 import dem
    dem.load()
    r = gpu_arm(args, rank, world, local)
    vals = aggregate(r["value_local"], r["time_local"], world)
    if rank == 0:
        cpu = None
        if not args.no_cpu:
            cpu = cpu_baseline(args)
        total_checks, tmax = vals
        value = total_checks / tmax
        K = args.steps
        ms = 1e3 * tmax / K
        roof = {"bound": "alu", "kernel": "pair_kernel<FP32, narrow phase + collision times>", "achieved": r["achieved"],
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": r["achieved"] / FP32_PEAK_TFLOPS,
                "traffic": _profile_traffic(), "peak_source": "recipe unit counts: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                "flops_per_launch": r["ct_flops"], "ms_per_launch": r["ct_ms"]}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "particles": r["particles"], "candidate_pairs": r["n_pairs"],
                           "precision": "FP32 + FP64 recomputation in the FP32 error band",
                           "l2": "flushed (512 MB write) between timed steps", "parallelism": f"replicas x{world}"},
                "particle_steps_per_s": world * r["particles"] * K / tmax,
                "checks_per_step": r["checks_step"],
                "stage_ms": {"detect (narrow phase + collision times)": r["ct_ms"],
                             "step_without_graph": r["direct_ms"]},
                "four_call_step": r["four_call"],
                "cuda_graph": "timed steps are replays of the step (candidates, detect, clusters) captured in "
                              "one CUDA graph",
                "roofline": roof, "cpu_baseline": cpu, "e2e": r["e2e"], "clocks": r["clocks"],
                "gpu_launches": int(r["launches"]), "fp64_form": r["fp64"], "fp32_error": r["fp32_err"],
                "counters_per_step": r["stats_step"], "local_time_stepping": r.get("lts"),
                "narrowing_vs_sampling": r.get("narrowing")}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def aggregate(checks_local, time_local, world):
    """Sum of checks over ranks and max of time over ranks."""
    if world == 1:
        return checks_local, time_local
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if torch.distributed.get_backend() == "nccl" else "cpu"
    t = torch.tensor([checks_local, time_local], dtype=torch.float64, device=dev)
    c = t[:1].clone()
    torch.distributed.all_reduce(c, op=torch.distributed.ReduceOp.SUM)
    m = t[1:].clone()
    torch.distributed.all_reduce(m, op=torch.distributed.ReduceOp.MAX)
    return float(c.item()), float(m.item())


if __name__ == "__main__":
    main()
