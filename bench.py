#!/usr/bin/env python
"""Benchmark of batched flow refinement (Sanders & Schulz, Section 4.1 / 4.1.1) on GB300.

One step = one sweep of fr_refine_batch over the 3D random geometric graph
(n = 4,194,304, mean degree ~12, omega in [1,10], c in [1,4], k = 64, eps = 0.01,
alpha = 4, most balanced cuts): boundary scan, quotient-graph rounds, and per
round one persistent launch doing corridor BFS, network build, max flow,
residual SCCs / sweeps and the commit.  The partition is restored before every
step, so each step refines the same input.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica (the pairs of a round never
exchange data, and no rank shares a graph with another); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "block-pair refinements/sec"
UNIT = "pairs/s"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ----------------------------------------------------------------- workloads --

def make_workload(name):
    from paper_1012_0006_gb300 import inputs as I
    if name == "rgg3d":
        w = I.config(4)
        desc = "rgg3d n=4194304 deg~12 omega[1,10] c[1,4] k=64 eps=0.01 alpha=4 MB R=1"
    elif name == "grid3d":
        w = I.config(3)
        desc = "grid3d 128^3 k=16 eps=0.03 alpha=2 MB R=1"
    elif name == "grid2d":
        w = I.config(1)
        desc = "grid2d 64x64 k=2 eps=0.03 alpha=1 (quick checks)"
    elif name == "rgg2d":
        w = dict(I.config(2), alpha=16.0)
        desc = "rgg2d n=65536 deg~8 k=2 eps=0.03 alpha=16 (one pair, the largest adaptive corridor)"
    else:
        raise SystemExit(f"unknown workload {name}")
    return w, desc


# ---------------------------------------------------------------- clocks ----

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = os.path.join(os.environ.get("FR_CLOCKS_DIR", tempfile.gettempdir()), f"clocks_rank{device}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ distributed ----

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def reduce_max(pg, x, device=None):
    """Max over ranks of a float (gloo or nccl)."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(pg, x, device=None):
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------ CPU baseline ----

def oracle_sample(w, budget_s=12.0):
    """The oracle as it stands, on the first pairs of one sweep in round order (bounded sample)."""
    import oracle as O
    t0 = time.perf_counter()
    st, _, done = O.refine_batch_sample(w, 4)
    t_small = time.perf_counter() - t0
    assert st == 0
    per = max(t_small / max(done, 1), 1e-4)
    pa, pb, pr, nr = O.rounds(w)
    P = int(min(len(pa), max(4, budget_s / per)))
    t0 = time.perf_counter()
    st, _, done = O.refine_batch_sample(w, P)
    el = time.perf_counter() - t0
    return dict(value=done / el, unit=UNIT, cores=1, kind="oracle",
                sample=f"first {done} of {len(pa)} pairs of one sweep in round order, one validation pass "
                       f"and rounds included, single thread, {el:.1f} s"), done, el


def oracle_pair_parallel(w, per_pair_s, budget_s=12.0):
    """The oracle's sweep with the pairs of each round on all host cores
    (fro_refine_batch_mt; the per-pair arithmetic is the single-threaded oracle's),
    over as many leading rounds as fit the budget at the single-thread rate."""
    import numpy as np
    import oracle as O
    cores = len(os.sched_getaffinity(0))
    if per_pair_s is None:   # single-thread rate from the first two pairs
        t0 = time.perf_counter()
        st, _, done = O.refine_batch_sample(w, 2)
        per_pair_s = (time.perf_counter() - t0) / max(done, 1)
    pa, pb, pr, nr = O.rounds(w)
    counts = np.bincount(pr, minlength=nr)
    R, est = 0, 0.0
    while R < nr and (R == 0 or est + per_pair_s * np.ceil(counts[R] / cores) <= budget_s):
        est += per_pair_s * np.ceil(counts[R] / cores)
        R += 1
    t0 = time.perf_counter()
    st, _, _, _, done = O.refine_batch_mt(w, cores, max_rounds=R)
    el = time.perf_counter() - t0
    assert st == 0
    return dict(value=round(done / el, 3), unit=UNIT, cores=cores, kind="oracle, pair-parallel",
                sample=f"first {R} of {nr} rounds ({done} of {len(pa)} pairs) of one sweep, the pairs of a round "
                       f"on {cores} threads, validation and rounds included, {el:.1f} s")


# ---------------------------------------------------------------- roofline ----

def measured_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Device code of the flow sweep: the queue kernel (every phase of every pair), the
# round-by-round step and cluster kernels, and the kernels that write what they read.  A
# recorded DRAM traffic of the sweep's dominant kernel holds only while these are unchanged.
SWEEP_KERNEL_SOURCES = ("cluster_flow.cu", "cluster_flow.cuh", "fr_internal.cuh", "prep_kernel.cu",
                        "round_kernel.cu", "round_kernel.cuh", "step_kernel.cuh", "queue_sweep.cu",
                        "queue_sweep.cuh")


def kernel_source_hash():
    """Hash of the sweep's kernel sources (a recorded DRAM traffic is used only while
    they are unchanged)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1012_0006_gb300", "csrc")
    for f in SWEEP_KERNEL_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """DRAM bytes per launch from a committed ncu summary, if it matches the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        e = rec.get(kernel)
        if e and e.get("source_hash") == kernel_source_hash():
            return e.get("dram_bytes_per_launch_full"), e
    except Exception:
        pass
    return None, None


def bytes_model(P):
    """Algorithmic HBM bytes per kernel type for one sweep (element bytes the method must touch).
    In a queue sweep every phase runs in the one queue kernel: its pairs' boundary scans
    read the per-block candidate lists, and local ids come from the visit list alone."""
    n, nnz = P["n"], P["nnz"]
    queue = bool(P.get("queue"))
    # boundary scan over the candidate list: entry and part[v] per listed vertex,
    # xadj per row of the round's blocks, adjncy and part[u] per arc of those rows
    scan = 8 * P["scan_listed"] + 8 * P["scan_rows"] + 8 * P["scan_arcs"]
    vis, arcs = P["bfs_visited"], P["bfs_arcs"]
    nc, m = P["corridor_n"], P["corridor_arcs"]
    bfs = 16 * vis + 12 * arcs                              # queue entries, dist, adjncy + part + dist per arc
    select = 4 * 8 * vis                                    # four radix passes over the overflow levels
    # marks, bitmap words (round by round), gid/sid/lid
    lid = 12 * vis + (0 if queue else (n // 8) * P["nrounds"]) + 12 * nc
    build = 12 * nc + 28 * m                                # rows, head, rev, res, cap, ranks
    cut = 24 * nc                                           # DAG of components, sweeps, eval, commit
    step = bfs + select + lid + build + cut
    # cluster kernel: network in (vertex 32 B: ids, offsets, excess, flow, border;
    # arc 24 B: head, reverse, residual, both capacities), results out (vertex 20 B,
    # arc residual 4 B)
    cluster = 52 * nc + 28 * m
    return dict(scan=scan, step=step, bfs=bfs, build=build, cluster=cluster, queue=scan + step + cluster)


# ------------------------------------------------------------------ ours ----

def run_ours(args, world, rank, local, pg):
    import numpy as np
    import torch
    from paper_1012_0006_gb300 import flowref as F

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t0 = time.time()
    w, desc = make_workload(args.workload)
    log(f"[rank {rank}] workload {w['name']} generated in {time.time() - t0:.1f}s")
    g = F.DeviceGraph.from_workload(w, device=dev)
    part0 = torch.as_tensor(np.array(w["part"], np.int32)).to(dev)
    part = part0.clone()
    ctx = F.Context(local)
    opts = F.default_options(mb=int(w["mb"]), sweep_sched=args.sweep_sched)
    k, eps, alpha = w["k"], w["eps"], w["alpha"]
    tuned = None
    if not args.no_autotune:
        t0 = time.time()
        best, ms = ctx.autotune(g, part0, k, eps, alpha, opts, trials=1)
        tuned = dict(block_threads=best.block_threads, grid_blocks=best.grid_blocks, gr_interval=best.gr_interval,
                     inner_ops=best.inner_ops, pulse_passes=best.pulse_passes, cluster_ctas=best.cluster_ctas,
                     flow_sched=best.flow_sched, pre_waves=best.pre_waves,
                     ms=round(ms, 3))
        log(f"[rank {rank}] autotune {tuned} in {time.time() - t0:.1f}s")

    def step():
        part.copy_(part0)
        st, _, summ = ctx.refine_batch(g, part, k, eps, alpha, opts, results=False)
        return summ

    for _ in range(args.warmup):
        summ = step()
    torch.cuda.synchronize()
    barrier(pg)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    barrier(pg)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev0.record()
    pairs = arcs = flow_ns = 0
    launches = 0
    for i in range(args.steps):
        summ = step()
        evs[i].record()
        pairs += summ["npairs"]
        arcs += summ["corridor_arcs"]
        flow_ns += summ["flow_ns"]
        launches += ctx.last_launches
    ev1.record()
    torch.cuda.synchronize()
    barrier(pg)
    clk = clocks.stop()
    t_ms = ev0.elapsed_time(ev1)
    per_step = [ev0.elapsed_time(evs[0])] + [evs[i - 1].elapsed_time(evs[i]) for i in range(1, args.steps)]
    t_max = reduce_max(pg, t_ms, dev)
    pairs_all = reduce_sum(pg, pairs, dev)
    value = pairs_all / (t_max / 1e3)

    # per-kernel timing with CUDA events around each launch (same workload, after the timed region)
    ctx.set_profiling(True)
    profs = []
    for _ in range(3):
        step()
        profs.append(ctx.profile())
    ctx.set_profiling(False)
    P = profs[-1]
    nr = P["nrounds"]
    scan_ms = statistics.median(p["scan_ms"] for p in profs)
    step_ms = statistics.median(p["step_ms"] for p in profs)
    clu_ms = statistics.median(p["cluster_ms"] for p in profs)
    bm = bytes_model(P)
    peak, peak_kind = measured_peak_gbs()
    if P["queue"]:
        # one queue kernel per sweep runs every phase of every pair; its setup launches
        # (pair fill, clears, the per-block lists) are the rest
        per = {"queue_kernel": (bm["queue"], clu_ms, 1), "queue_setup": (0, scan_ms, 5)}
    else:
        launches_per_round = 2 if clu_ms > 0 else 1          # step kernels per round
        per = {"scan_kernel": (bm["scan"], scan_ms, nr),
               "step_kernel": (bm["step"], step_ms, nr * launches_per_round)}
        if clu_ms > 0:
            per["cluster_flow_kernel"] = (bm["cluster"], clu_ms, nr)
    dominant = max(per, key=lambda kk: per[kk][1])
    kernels = {}
    for name, (byts, ms, nl) in per.items():
        gbs = byts / nl / (ms / nl * 1e-3) / 1e9 if ms > 0 else 0.0
        kernels[name] = {"launches_per_sweep": nl, "ms_per_launch": round(ms / nl, 4),
                         "bytes_per_launch": int(byts / nl), "gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
                         "share": round(ms / (scan_ms + step_ms + clu_ms), 4)}
    byts, ms, nl = per[dominant]
    achieved = byts / nl / (ms / nl * 1e-3) / 1e9
    traffic, _ = recorded_traffic(dominant)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": dominant,
                "peak_kind": peak_kind, "bytes_per_launch": int(byts / nl), "launch_ms": round(ms / nl, 4)}
    ph = P["phase_ms"]
    if P["queue"]:
        # the pairs' max flows overlap in the queue kernel's clusters: their summed
        # in-kernel time (network load, flow to t, return) over the clusters running them
        cp = P["cluster_phase_ms"]
        flow_ms = (cp["load"] + cp["flow"] + cp["return"]) / max(P["queue_clusters"], 1)
    else:
        # wall time of the max flows: the cluster kernels (flow, reach and SCCs of every
        # pair) plus the grid-wide flow phases of pairs left to them
        flow_ms = clu_ms + ph["flow"] + ph["relabel"] + ph["return"]
    arcs_rate = reduce_sum(pg, P["corridor_arcs"] / max(flow_ms * 1e-3, 1e-12), dev)
    kernels.update({
        "schedule": ({"queue": True, "cluster_ctas": P["queue_ctas"], "clusters": P["queue_clusters"],
                      "boundary_scan_ms_summed_over_pairs": round(P["queue_scan_ms"], 3)}
                     if P["queue"] else {"queue": False, "rounds": nr}),
        "phases_ms": {kk: round(v, 3) for kk, v in ph.items()},
        "bfs_gbs": round(bm["bfs"] / max(ph["bfs"] * 1e-3, 1e-12) / 1e9, 1),
        "cluster_phases_ms_summed_over_pairs": {kk: round(v, 3) for kk, v in P["cluster_phase_ms"].items()},
        "counters": {kk: P[kk] for kk in ("bfs_visited", "bfs_arcs", "corridor_n", "corridor_arcs", "pulses",
                                           "relabels", "gr_arcs", "pr_arcs", "pushes", "scc_rounds",
                                           "barriers", "cluster_syncs", "cluster_remote_arcs",
                                           "fallback_pairs", "scan_listed", "scan_rows", "scan_arcs")},
    })

    # end to end through the host-buffer entry point: H2D of graph and part, D2H of part
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.int32)).pin_memory()
        hx, ha, hw, hv = pin(w["xadj"]), pin(w["adjncy"]), pin(w["adjwgt"]), pin(w["vwgt"])
        hp0 = np.array(w["part"], np.int32)
        hp = pin(hp0)
        ctx.refine_batch_host(hx, ha, hw, hv, hp, k, eps, alpha, opts)   # warm (allocations)
        n, nnz = w["n"], w["nnz"]
        tot = 0.0
        ke = max(3, args.steps // 2)
        for _ in range(ke):
            hp.numpy()[:] = hp0
            t0 = time.perf_counter()
            ctx.refine_batch_host(hx, ha, hw, hv, hp, k, eps, alpha, opts)
            tot += time.perf_counter() - t0
        tot = reduce_max(pg, tot, dev)
        e2e = {"value": round(pairs_all / args.steps * ke / tot, 2), "unit": UNIT,
               "h2d_bytes_per_step": 4 * ((n + 1) + 2 * nnz + 2 * n), "d2h_bytes_per_step": 4 * n,
               "ms_per_step": round(tot / ke * 1e3, 3)}

    compare = batched_vs_per_pair(F, ctx, dev) if args.compare else None
    rates = phase_rates(F, dev, P, pairs // max(args.steps, 1)) if args.compare else None
    active = active_blocks(F, ctx, g, part0, w) if args.active else None
    fm = fm_sweeps(F, ctx, g, part0, w) if args.fm else None
    mtp = multitry_pass(F, ctx, g, part0, w, cpu=not args.no_cpu) if args.mt else None
    kwr = kway_rounds(F, ctx, g, part0, w, cpu=not args.no_cpu) if args.mt else None
    vc = multilevel(F, ctx, g, part0, w) if args.vcycle else None
    nxt = next_rows(F, dev, cpu=not args.no_cpu) if args.next_rows else None
    spc = single_pair_configs(F, dev, cpu=not args.no_cpu) if args.next_rows else None

    serving = None
    if args.serve:
        serving = run_serving(F, local, full=args.serve_full, requests=args.serve_requests,
                              log_prefix=f"[rank {rank}] ")

    cpu = cpu_mt = None
    if rank == 0 and not args.no_cpu:
        cpu, done, el = oracle_sample(w, budget_s=args.cpu_budget)
        cpu["value"] = round(cpu["value"], 3)
        cpu_mt = oracle_pair_parallel(w, el / max(done, 1), budget_s=args.cpu_budget)
        if compare is not None:
            compare["cpu_pair_parallel"] = oracle_pair_parallel(make_workload("grid3d")[0], None,
                                                                budget_s=args.cpu_budget)

    if rank == 0:
        out = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 3),
            "per_step_ms": {"median": round(statistics.median(per_step), 3), "min": round(min(per_step), 3),
                            "max": round(max(per_step), 3)},
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": desc, "n": w["n"], "nnz": w["nnz"], "k": k,
                       "pairs_per_step": int(pairs / args.steps), "rounds_per_step": nr,
                       "l2": "inputs larger than L2 (graph + part ~0.45 GB per replica)",
                       "parallelism": "replicas" if world > 1 else "single", "launch_shape": tuned},
            "corridor_arcs_per_sec_through_maxflow": round(arcs_rate, 1),
            "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline, "kernels": kernels,
            "cpu_baseline": cpu, "cpu_baseline_pair_parallel": cpu_mt, "clocks": clk, "serving": serving, "batched_vs_per_pair": compare, "phase_rates": rates,
            "active_blocks": active, "fm": fm, "multitry": mtp, "kway_rounds": kwr, "next_rows_vs_oracle": nxt, "single_pair_configs": spc, "vcycle": vc,
        }
        print(json.dumps(out), flush=True)
    ctx.close()


# ------------------------------------------------------- active block scheduling ----

def active_blocks(F, ctx, g, part0, w, max_outer=16):
    """The bench workload under active block scheduling (fr_refine_active): outer
    rounds until no block is active, every pair with adaptive flow iterations from
    alpha = 1 up to alpha' = 16 (Section 4.1).  One run, after the timed region."""
    import torch
    opts = F.default_options(mb=int(w["mb"]), adaptive=1, max_iters=10, alpha_max=16.0)
    part = part0.clone()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, res, summ, nouter = ctx.refine_active(g, part, w["k"], w["eps"], 1.0, opts, max_outer=max_outer, cap=0)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    return {"workload": "bench workload, alpha 1 -> 16 adaptive, until no block is active",
            "outer_rounds": nouter, "refinements": summ["npairs"], "matchings": summ["nrounds"],
            "accepted": summ["accepted"], "cut_before": summ["cut_before"], "cut_after": summ["cut_after"],
            "ms": round(el * 1e3, 2), "refinements_per_s": round(summ["npairs"] / el, 2)}


def multitry_pass(F, ctx, g, part0, w, alpha=10, reps=2, cpu=True):
    """One multi-try FM pass (Section 4.2; k-way searches stopped by the KaSPar rule with
    alpha = 10 as in the paper's setup) over the first matching of the bench workload:
    device time (CUDA events around fr_multitry, min of reps after one warm run; the pass
    runs its searches in order on one warp), what it gained on the cut, and the oracle's
    pass on the host (one run, one thread)."""
    import numpy as np
    import torch
    part_np = part0.cpu().numpy()
    pairs = [(int(a), int(b)) for a, b, r in zip(*ctx.rounds(g, part0, w["k"])[:3]) if r == 0]
    part = part0.clone()
    st, tot, _ = ctx.multitry(g, part, w["k"], w["eps"], pairs, alpha)
    best = None
    for _ in range(reps):
        part.copy_(part0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.multitry(g, part, w["k"], w["eps"], pairs, alpha)
        e1.record()
        torch.cuda.synchronize()
        best = e0.elapsed_time(e1) if best is None else min(best, e0.elapsed_time(e1))
    out = {"workload": f"bench workload, first matching ({len(pairs)} pairs), alpha {alpha}",
           "ms": round(best, 3), "gain": tot["gain"], "searches": tot["searches"], "moves_tried": tot["tried"],
           "moves_kept": tot["kept"], "searches_per_s": round(tot["searches"] / (best / 1e3), 1)}
    if cpu:
        import oracle as O
        wo = dict(w, part=part_np)
        t0 = time.perf_counter()
        st, pref, tref, _ = O.multitry(wo, pairs, alpha)
        out["oracle_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
        out["parity"] = bool(tref == {f: tot[f] for f in ("gain", "searches", "tried", "kept")} and
                             np.array_equal(pref, part.cpu().numpy()))
    return out


def single_pair_configs(F, dev, cpu=True, reps=3):
    """The two single-pair configurations as they are defined: the 64 x 64 grid bisection
    (one plain flow refinement, alpha 1) and the rgg2d n = 65,536 bisection with adaptive
    flow iterations (alpha 1, 2, 4, ... up to 16, at most ten iterations), one pair per
    launch through fr_refine_pair; then the rgg2d bisection at fixed alpha 1, 2, 4, 8, 16,
    plain and most balanced, with the corridor and the max flow's share of the time.
    Device: CUDA events around the call, min of reps after a warm run; oracle: one run,
    one thread; parity: identical partitions, flow, cuts and iterations."""
    import numpy as np
    import torch
    import oracle as O
    from paper_1012_0006_gb300 import inputs as I
    ctx = F.Context(dev.index if dev.index is not None else 0)
    out = {}
    for name, cfg in (("grid2d 64x64 k=2 alpha=1, one refinement", 1),
                      ("rgg2d n=65536 k=2, adaptive alpha 1 -> 16", 2)):
        w = I.config(cfg)
        ok = dict(mb=int(w["mb"]), adaptive=int(w["adaptive"]), max_iters=int(w["max_iters"]),
                  alpha_max=float(w["alpha_max"]))
        g = F.DeviceGraph.from_workload(w, device=dev)
        part0 = torch.as_tensor(np.array(w["part"], np.int32)).to(dev)
        part = part0.clone()
        ctx.refine_pair(g, part, w["k"], 0, 1, w["eps"], w["alpha"], F.default_options(**ok))   # warm
        best, res = None, None
        for _ in range(reps):
            part.copy_(part0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st, res = ctx.refine_pair(g, part, w["k"], 0, 1, w["eps"], w["alpha"], F.default_options(**ok))
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        e = {"ms": round(best, 3), "refinements_per_s": round(1e3 / best, 1), "flow": res.flow,
             "cut_before": res.cut_before, "cut_after": res.cut_after, "iters": res.iters,
             "alpha_final": res.alpha_final, "corridor_n": res.corridor_n}
        if cpu:
            t0 = time.perf_counter()
            ost, pref, rref = O.refine_pair(w, opts=O.options(**ok))
            e["oracle_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
            e["parity"] = bool(ost == 0 and np.array_equal(pref, part.cpu().numpy()) and
                               (rref.flow, rref.cut_before, rref.cut_after, rref.iters) ==
                               (res.flow, res.cut_before, res.cut_after, res.iters))
        out[name] = e
    # the rgg2d bisection at fixed alpha (one refinement each, plain and most balanced):
    # corridor size and the max flow's share, through fr_refine_batch's phase timers
    # (k = 2: one pair, one round)
    w = I.config(2)
    g = F.DeviceGraph.from_workload(w, device=dev)
    part0 = torch.as_tensor(np.array(w["part"], np.int32)).to(dev)
    sweep = []
    for mb in (0, 1):
        for alpha in (1.0, 2.0, 4.0, 8.0, 16.0):
            opts = F.default_options(mb=mb)
            part = part0.clone()
            ctx2 = F.Context(dev.index if dev.index is not None else 0)
            ctx2.refine_batch(g, part, 2, w["eps"], alpha, opts, results=False)   # warm
            best = None
            for _ in range(reps):
                part.copy_(part0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                _, res, summ = ctx2.refine_batch(g, part, 2, w["eps"], alpha, opts)
                e1.record()
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1)
                best = t if best is None else min(best, t)
            got = part.cpu().numpy()
            ctx2.set_profiling(True)
            part.copy_(part0)
            ctx2.refine_batch(g, part, 2, w["eps"], alpha, opts, results=False)
            P = ctx2.profile()
            ctx2.close()
            ph, cp = P["phase_ms"], P["cluster_phase_ms"]
            flow_ms = ph["flow"] + ph["relabel"] + ph["return"] + cp["load"] + cp["flow"] + cp["return"]
            r = res[0]
            e = {"mb": mb, "alpha": alpha, "ms": round(best, 3), "corridor_n": r["corridor_n"],
                 "corridor_arcs": r["corridor_arcs"], "flow": r["flow"], "cut_after": r["cut_after"],
                 "max_flow_ms": round(flow_ms, 3),
                 "corridor_arcs_per_s_through_max_flow": round(r["corridor_arcs"] / max(flow_ms * 1e-3, 1e-12), 1)}
            if cpu:
                t0 = time.perf_counter()
                ost, pref, rref = O.refine_pair(w, alpha=alpha, opts=O.options(mb=mb))
                e["oracle_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
                e["parity"] = bool(ost == 0 and np.array_equal(pref, got) and rref.flow == r["flow"] and
                                   rref.cut_after == r["cut_after"])
            sweep.append(e)
    out["rgg2d n=65536 k=2, fixed alpha, one refinement"] = sweep
    ctx.close()
    return out


def next_rows(F, dev, cpu=True):
    """The rows next to the path on the bench workload at 1/16 scale (rgg3d n = 262,144,
    k = 64), each against the oracle on the same input: one sweep with the FM step
    before every pair's flow (fm_permille 10), active block scheduling with adaptive
    flow iterations (alpha 1 -> 16) and with a multi-try pass after every matching
    (mt_alpha 10, four outer rounds), one V-cycle, and (at 1/64 scale) a W- and an
    F-cycle with level split parameter 2.  Device time: CUDA events around
    the call, one run after a warm one; oracle: one run, one thread; parity: identical
    partitions and totals."""
    import numpy as np
    import torch
    import oracle as O
    from paper_1012_0006_gb300 import inputs as I
    w = I.config(4, scale=1 / 16)
    k, eps = w["k"], w["eps"]
    g = F.DeviceGraph.from_workload(w, device=dev)
    part0 = torch.as_tensor(np.array(w["part"], np.int32)).to(dev)
    ctx = F.Context(dev.index if dev.index is not None else 0)
    out = {"workload": f"rgg3d n={w['n']} k={k} eps={eps} (the bench workload at 1/16 scale)"}

    def timed(fn):
        part = part0.clone()
        fn(part)
        part.copy_(part0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn(part)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r, part.cpu().numpy()

    def host(fn):
        t0 = time.perf_counter()
        r = fn()
        return (time.perf_counter() - t0) * 1e3, r

    # FM step then flow, one sweep
    fo = dict(mb=1, fm_permille=10)
    ms, (st, _, summ), got = timed(lambda p: ctx.refine_batch(g, p, k, eps, w["alpha"], F.default_options(**fo),
                                                              results=False))
    e = {"ms": round(ms, 2), "pairs": summ["npairs"], "cut_before": summ["cut_before"], "cut_after": summ["cut_after"]}
    if cpu:
        oms, (ost, pref, rref, nr) = host(lambda: O.refine_batch(w, opts=O.options(**fo)))
        e.update(oracle_ms=round(oms, 1), parity=bool(ost == 0 and np.array_equal(pref, got) and nr == summ["nrounds"]))
    out["fm_sweep"] = e
    # active block scheduling, adaptive iterations; and with multi-try passes
    for name, ao, mo in (("active_adaptive", dict(mb=1, adaptive=1, max_iters=10, alpha_max=16.0), 16),
                         ("active_multitry", dict(mb=1, mt_alpha=10), 4)):
        ms, (st, res, summ, nouter), got = timed(
            lambda p: ctx.refine_active(g, p, k, eps, 1.0, F.default_options(**ao), max_outer=mo))
        e = {"ms": round(ms, 2), "outer_rounds": nouter, "refinements": len(res), "cut_before": summ["cut_before"],
             "cut_after": summ["cut_after"]}
        if cpu:
            oms, (ost, pref, rref, onr) = host(lambda: O.refine_active(w, alpha=1.0, opts=O.options(**ao), max_outer=mo))
            e.update(oracle_ms=round(oms, 1),
                     parity=bool(ost == 0 and np.array_equal(pref, got) and onr == nouter and len(rref) == len(res)))
        out[name] = e
    # one V-cycle
    ms, (st, r), got = timed(lambda p: ctx.vcycle(g, p, k, eps, w["alpha"], F.default_options(mb=1)))
    e = {"ms": round(ms, 2), "levels": r["levels"], "cut_before": r["cut_before"], "cut_after": r["cut_after"]}
    if cpu:
        oms, (ost, pref, rr) = host(lambda: O.vcycle(w, opts=O.options(mb=1)))
        e.update(oracle_ms=round(oms, 1),
                 parity=bool(ost == 0 and np.array_equal(pref, got) and rr["level_n"] == r["level_n"]))
    out["vcycle"] = e
    # W- and F-cycles (level split parameter 2) on the bench workload at 1/64 scale
    w2 = I.config(4, scale=1 / 64)
    g2 = F.DeviceGraph.from_workload(w2, device=dev)
    p2 = torch.as_tensor(np.array(w2["part"], np.int32)).to(dev)
    for kind in ("F", "W"):
        part = p2.clone()
        ctx.cycle(g2, part, w2["k"], w2["eps"], w2["alpha"], kind=kind, d=2, opts=F.default_options(mb=1))   # warm
        part.copy_(p2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st, c = ctx.cycle(g2, part, w2["k"], w2["eps"], w2["alpha"], kind=kind, d=2, opts=F.default_options(mb=1))
        e1.record()
        torch.cuda.synchronize()
        e = {"workload": f"rgg3d n={w2['n']} k={w2['k']} (1/64 scale)", "ms": round(e0.elapsed_time(e1), 2),
             "coarsenings": c["coarsenings"], "refinements": c["refinements"], "cut_before": c["cut_before"],
             "cut_after": c["cut_after"]}
        if cpu:
            oms, (ost, pref, rc) = host(lambda: O.cycle(w2, kind=kind, d=2, opts=O.options(mb=1)))
            e.update(oracle_ms=round(oms, 1),
                     parity=bool(ost == 0 and np.array_equal(pref, part.cpu().numpy()) and
                                 rc["coarsenings"] == c["coarsenings"] and rc["refinements"] == c["refinements"]))
        out[kind + "_cycle"] = e
    ctx.close()
    return out


def kway_rounds(F, ctx, g, part0, w, cpu=True):
    """Global k-way refinement rounds as the paper's setup runs them (Section 6: from the
    complete partition boundary, alpha = 10, at most ten rounds, stopping after a round
    without improvement) on the bench workload: device time (CUDA events around
    fr_kway_global, one run after a warm one), the rounds' totals, and the oracle's rounds
    on the host (one run, one thread) with a parity flag."""
    import numpy as np
    import torch
    part = part0.clone()
    ctx.kway_global(g, part, w["k"], w["eps"], init_mode=0, alpha=10, max_rounds=10, seed=0)   # warm
    part.copy_(part0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    st, tot = ctx.kway_global(g, part, w["k"], w["eps"], init_mode=0, alpha=10, max_rounds=10, seed=0)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out = {"workload": "bench workload and partition, whole-boundary start sets, alpha 10, <= 10 rounds",
           "ms": round(ms, 2), "rounds": tot["searches"], "gain": tot["gain"], "moves_tried": tot["tried"],
           "moves_kept": tot["kept"], "moves_per_s": round(tot["tried"] / (ms / 1e3), 1)}
    if cpu:
        import oracle as O
        wo = dict(w, part=part0.cpu().numpy())
        t0 = time.perf_counter()
        st, pref, tref, rref = O.kway_global(wo, alpha=10, init_mode=0, max_rounds=10, seed=0)
        out["oracle_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
        out["parity"] = bool((tref["gain"], tref["tried"], tref["kept"], rref) ==
                             (tot["gain"], tot["tried"], tot["kept"], tot["searches"]) and
                             np.array_equal(pref, part.cpu().numpy()))
    return out


def multilevel(F, ctx, g, part0, w, reps=2):
    """One V-cycle with the bench workload's partition (fr_vcycle, Section 5): greedy
    expansion*2 matchings inside blocks, contraction down to max(60 k, n / (60 k))
    vertices, then a flow sweep on every level from the coarsest up; device time (CUDA
    events around the call, min of reps after one warm run) and the cut against one flat
    sweep of the input level."""
    import torch
    opts = F.default_options(mb=int(w["mb"]))
    part = part0.clone()
    st, flat = ctx.refine_batch(g, part, w["k"], w["eps"], w["alpha"], opts, results=False)[::2]
    best, r = None, None
    for _ in range(reps + 1):
        part.copy_(part0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st, r = ctx.vcycle(g, part, w["k"], w["eps"], w["alpha"], opts)
        e1.record()
        torch.cuda.synchronize()
        if _ > 0:
            best = e0.elapsed_time(e1) if best is None else min(best, e0.elapsed_time(e1))
    out = {"workload": "bench workload and partition, one V-cycle, one sweep per level",
           "ms": round(best, 2), "levels": r["levels"], "level_n": r["level_n"], "level_pairs": r["level_pairs"],
           "coarsen_ms": round(r["coarsen_ms"], 2), "refine_ms": round(r["refine_ms"], 2),
           "cut_before": r["cut_before"], "cut_after": r["cut_after"], "cut_after_flat_sweep": flat["cut_after"]}
    # the F- and W-cycles of Section 5 (level split parameter 2), one run each
    for kind in ("F", "W"):
        part.copy_(part0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st, c = ctx.cycle(g, part, w["k"], w["eps"], w["alpha"], kind=kind, d=2, opts=opts)
        e1.record()
        torch.cuda.synchronize()
        out[kind + "_cycle"] = {"ms": round(e0.elapsed_time(e1), 2), "coarsenings": c["coarsenings"],
                                "refinements": c["refinements"], "cut_after": c["cut_after"]}
    return out


def fm_sweeps(F, ctx, g, part0, w, reps=3):
    """The bench workload's sweep with the two-way FM step (TopGain, Section 2.2) before
    every pair's flow, stopped after 1 % and 5 % of the pair's vertices moved without an
    improvement, against the flow-only sweep: device time per sweep (CUDA events around
    the call, min of reps after one warm run) and what each step gained on the cut."""
    import torch
    out = {"workload": "bench workload, FM then flow per pair"}
    base = None
    for pm in (0, 10, 50):
        opts = F.default_options(mb=int(w["mb"]), fm_permille=pm)
        part = part0.clone()
        st, res, summ = ctx.refine_batch(g, part, w["k"], w["eps"], w["alpha"], opts)
        best = None
        for _ in range(reps):
            part.copy_(part0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.refine_batch(g, part, w["k"], w["eps"], w["alpha"], opts, results=False)
            e1.record()
            torch.cuda.synchronize()
            best = e0.elapsed_time(e1) if best is None else min(best, e0.elapsed_time(e1))
        ctx.set_profiling(True)
        part.copy_(part0)
        ctx.refine_batch(g, part, w["k"], w["eps"], w["alpha"], opts, results=False)
        fm_ms = ctx.profile()["fm_ms"]
        ctx.set_profiling(False)
        d = {"ms_per_sweep": round(best, 3), "pairs_per_s": round(summ["npairs"] / (best / 1e3), 1),
             "cut_before": summ["cut_before"], "cut_after": summ["cut_after"],
             "fm_gain": int(sum(r["cut_before"] - r["cut_fm"] for r in res)),
             "flow_gain": int(sum(r["cut_fm"] - r["cut_after"] for r in res)),
             "fm_moves_kept": int(sum(r["fm_moves"] for r in res))}
        if pm == 0:
            base = best
            out["flow_only"] = d
        else:
            d["fm_ms_per_sweep"] = round(best - base, 3)
            d["fm_phases_ms_summed_over_pairs"] = {kk: round(v, 3) for kk, v in fm_ms.items()}
            out[f"fm_permille_{pm}"] = d
    return out


# ------------------------------------------------- batched vs one pair per launch ----

def batched_vs_per_pair(F, ctx0, dev, reps=3):
    """128^3 grid, k = 16: one fr_refine_batch sweep against the same pairs refined by
    fr_refine_pair one launch at a time, in round order (same results, checked).  Both
    arms run on one context whose launch shape fr_autotune chose for this workload."""
    import numpy as np
    import torch
    from paper_1012_0006_gb300 import inputs as I
    w = I.config(3)
    g = F.DeviceGraph.from_workload(w, device=dev)
    part0 = torch.as_tensor(np.array(w["part"], np.int32)).to(dev)
    opts = F.default_options(mb=1)
    k, eps, alpha = w["k"], w["eps"], w["alpha"]
    ctx = F.Context(dev.index if dev.index is not None else 0)
    best, _ = ctx.autotune(g, part0, k, eps, alpha, opts, trials=1)
    part = part0.clone()
    st, res, summ = ctx.refine_batch(g, part, k, eps, alpha, opts)
    ref = part.clone()
    pairs = [(r["a"], r["b"]) for r in res]
    tb, tp = [], []
    for _ in range(reps):
        part.copy_(part0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.refine_batch(g, part, k, eps, alpha, opts, results=False)
        tb.append(time.perf_counter() - t0)
        part.copy_(part0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for a, b in pairs:
            ctx.refine_pair(g, part, k, a, b, eps, alpha, opts)
        tp.append(time.perf_counter() - t0)
        assert torch.equal(part, ref), "one-pair-per-launch result differs from the batch"
    b, p = min(tb), min(tp)
    ctx.close()
    return {"workload": "grid3d 128^3 k=16 eps=0.03 alpha=2 MB", "pairs": len(pairs),
            "rounds": summ["nrounds"], "batched_ms": round(b * 1e3, 3), "per_pair_ms": round(p * 1e3, 3),
            "speedup": round(p / b, 2),
            "launch_shape": dict(flow_sched=best.flow_sched, cluster_ctas=best.cluster_ctas,
                                 inner_ops=best.inner_ops, gr_interval=best.gr_interval,
                                 pulse_passes=best.pulse_passes)}


def phase_rates_of(P, peak, npairs):
    """Corridor BFS and exact-relabel rates of one profiled sweep.  BFS: algorithmic bytes
    (16 B per visited entry, 12 B per scanned arc) over the BFS phase time.  Relabel: arcs
    whose tail passed its label on (the gr_arcs counter) over the relabel time; in a
    cluster the network sits in distributed shared memory, so those arcs move no HBM
    bytes; the grid-wide relabel reads head, residual and label per arc (12 B) from HBM.
    In a queue sweep the phase times are summed over pairs (each pair's own cluster),
    so a rate is one cluster's; `clusters` of them run side by side."""
    ph, cp = P["phase_ms"], P["cluster_phase_ms"]
    bm = bytes_model(P)
    bfs_ms = ph["bfs"]
    out = {"schedule": "queue" if P["queue"] else "rounds", "pairs": npairs, "rounds": P["nrounds"],
           "clusters": P["queue_clusters"] if P["queue"] else None, "corridor_n": P["corridor_n"],
           "corridor_arcs": P["corridor_arcs"]}
    gbs = bm["bfs"] / max(bfs_ms * 1e-3, 1e-12) / 1e9
    out["bfs"] = {"visited": P["bfs_visited"], "arcs": P["bfs_arcs"], "bytes": int(bm["bfs"]),
                  "ms": round(bfs_ms, 3), "gbs": round(gbs, 1), "frac": round(gbs / peak, 4)}
    rel_ms = cp["relabel"] + ph["relabel"]
    grid = ph["relabel"] > cp["relabel"]
    rate = P["gr_arcs"] / max(rel_ms * 1e-3, 1e-12)
    out["relabel"] = {"relabels": P["relabels"], "arcs": P["gr_arcs"], "ms": round(rel_ms, 3),
                      "arcs_per_s": round(rate, 1),
                      "memory": "hbm" if grid else "distributed shared memory (no HBM bytes)"}
    if grid:
        out["relabel"].update(gbs=round(12 * rate / 1e9, 1), frac=round(12 * rate / 1e9 / peak, 4))
    return out


def phase_rates(F, dev, P4, pairs4, reps=3):
    """BFS and relabel rates on the single-pair bisection at alpha 16 (its largest
    adaptive corridor), on the 128^3 grid (k = 16), and on the bench workload (P4:
    the profile the main run took), each with the sweep schedule the library picks."""
    import numpy as np
    import torch
    from paper_1012_0006_gb300 import inputs as I
    peak, peak_kind = measured_peak_gbs()
    out = {"peak_gbs": peak, "peak_kind": peak_kind}
    for name, cfg, alpha in (("rgg2d n=65536 k=2 alpha=16 (one pair)", 2, 16.0),
                             ("grid3d 128^3 k=16 alpha=2", 3, None)):
        w = I.config(cfg)
        g = F.DeviceGraph.from_workload(w, device=dev)
        part0 = torch.as_tensor(np.array(w["part"], np.int32)).to(dev)
        ctx = F.Context(dev.index if dev.index is not None else 0)
        opts = F.default_options(mb=int(w["mb"]))
        a = alpha if alpha is not None else w["alpha"]
        part = part0.clone()
        ctx.refine_batch(g, part, w["k"], w["eps"], a, opts, results=False)   # warm (allocations)
        ctx.set_profiling(True)
        profs = []
        for _ in range(reps):
            part.copy_(part0)
            _, _, summ = ctx.refine_batch(g, part, w["k"], w["eps"], a, opts, results=False)
            profs.append(ctx.profile())
        ctx.set_profiling(False)
        P = min(profs, key=lambda q: q["phase_ms"]["bfs"])
        out[name] = phase_rates_of(P, peak, summ["npairs"])
        ctx.close()
    if P4 is not None:
        out["rgg3d n=4194304 k=64 alpha=4 (bench workload)"] = phase_rates_of(P4, peak, pairs4)
    return out


# ------------------------------------------------------------------ serving ----

def run_serving(F, device, full=True, requests=None, log_prefix="", parity_budget_s=120.0):
    """Continuous-batching serving of seeded refinement requests (Poisson arrivals).

    Pool: 2D grids and 2D/3D rggs (mean degree 8-12, unit or [1,10] weights), k in {2,4,8},
    eps in {0.01,0.03,0.05}, alpha 2, most balanced cuts, one sweep of rounds per request.
    full: 48 graphs up to 2^21 vertices and 10,000 requests (the serving configuration);
    otherwise a bounded sample (24 graphs up to 2^18 vertices, 1,500 requests).
    First the closed-loop saturated rate is measured (max_inflight requests always queued),
    then requests arrive as a Poisson process at 0.7 x that rate; latency is submit ->
    completion on the host clock.  A seeded 1 % sample of the open-loop requests keeps its
    served partition, and the oracle refines the same inputs on all host cores (one
    request per thread): parity = every checked partition and cut equal."""
    import concurrent.futures as cf
    import threading
    import numpy as np
    from paper_1012_0006_gb300 import inputs as I
    import oracle as O
    t0 = time.time()
    if full:
        pool = I.serving_pool(count=48, max_n=1 << 21)
        nreq = requests or 10000
    else:
        pool = I.serving_pool(count=24, max_n=1 << 18)
        nreq = requests or 1500
    rs = np.random.Generator(np.random.Philox(I.SEED_BASE + 5))
    parts = {}
    reqs = []
    for t in range(nreq):
        gi = int(rs.integers(0, len(pool)))
        k = int(rs.choice([2, 4, 8]))
        if (gi, k) not in parts:
            parts[(gi, k)] = I.serving_partition(pool[gi], k)
        reqs.append((gi, k, float(rs.choice([0.01, 0.03, 0.05]))))
    log(f"{log_prefix}serving pool {len(pool)} graphs, {len(parts)} partitions, {nreq} requests "
        f"prepared in {time.time() - t0:.1f}s")
    nmax = max(g["n"] for g in pool)
    opts = F.default_options(mb=1)
    srv = F.Server(device, max_inflight=32, opts=opts)
    ids = [srv.add_graph(g["xadj"], g["adjncy"], g["adjwgt"], g["vwgt"]) for g in pool]
    # the parity sample: a seeded 1 % of the open-loop requests (tags 10,000,000 + index)
    sample = sorted(set(rs.integers(0, len(reqs), max(1, len(reqs) // 100)).tolist()))
    want = {10_000_000 + i for i in sample}
    served = {}

    def drain(count, lat, stat):
        for _ in range(count):
            resp, out = srv.next(nmax, timeout_ms=600000)
            lat.append(resp["latency_ms"])
            stat.append(resp["status"])
            if resp["tag"] in want:
                gi = reqs[resp["tag"] - 10_000_000][0]
                served[resp["tag"] - 10_000_000] = (out[:pool[gi]["n"]].copy(), resp)

    # closed loop: everything queued at once (saturated)
    nsat = min(len(reqs), 400)
    lat, stat = [], []
    t1 = time.perf_counter()
    for t, (gi, k, eps) in enumerate(reqs[:nsat]):
        srv.submit(ids[gi], parts[(gi, k)], k, eps, 2.0, t)
    drain(nsat, lat, stat)
    sat = nsat / (time.perf_counter() - t1)
    # open loop: Poisson arrivals at 0.7 x saturated
    lam = 0.7 * sat
    gaps = rs.exponential(1.0 / lam, len(reqs))
    lat, stat = [], []
    th = threading.Thread(target=drain, args=(len(reqs), lat, stat))
    th.start()
    t1 = time.perf_counter()
    nxt = t1
    for t, (gi, k, eps) in enumerate(reqs):
        nxt += gaps[t]
        d = nxt - time.perf_counter()
        if d > 0:
            time.sleep(d)
        srv.submit(ids[gi], parts[(gi, k)], k, eps, 2.0, 10_000_000 + t)
    th.join()
    el = time.perf_counter() - t1
    st = srv.stats()
    srv.close()
    lat = np.array(lat)
    log(f"{log_prefix}serving: {len(reqs)} requests in {el:.1f}s, p50 {np.percentile(lat, 50):.2f} ms, "
        f"p99 {np.percentile(lat, 99):.2f} ms")

    # parity and per-request CPU time: the oracle on the sample, one request per host thread
    # (the oracle is plain C behind ctypes, which releases the GIL during the call)
    def oracle_one(i):
        gi, k, eps = reqs[i]
        g = pool[gi]
        w = dict(n=g["n"], xadj=g["xadj"], adjncy=g["adjncy"], adjwgt=g["adjwgt"], vwgt=g["vwgt"],
                 part=parts[(gi, k)], k=k, eps=eps, alpha=2.0)
        c0 = time.thread_time()
        stq, part_o, res_o, _ = O.refine_batch(w, opts=O.options(mb=1))
        cpu_s = time.thread_time() - c0
        got, resp = served[i]
        ok = (stq == 0 and resp["status"] == 0 and np.array_equal(got, part_o) and resp["npairs"] == len(res_o)
              and resp["accepted"] == sum(r["accepted"] for r in res_o))
        return ok, cpu_s, g["n"]

    threads = len(os.sched_getaffinity(0))
    t2 = time.perf_counter()
    checked = equal = 0
    cpu_tot = 0.0
    nmax_checked = 0
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        futs = [ex.submit(oracle_one, i) for i in sample if i in served]
        for f in futs:
            left = parity_budget_s - (time.perf_counter() - t2)
            try:
                ok, cpu_s, n = f.result(timeout=max(left, 0.0))
            except cf.TimeoutError:
                break
            checked += 1
            equal += bool(ok)
            cpu_tot += cpu_s
            nmax_checked = max(nmax_checked, n)
        for f in futs:
            f.cancel()
    parity_s = time.perf_counter() - t2
    return {"requests": len(reqs), "failed": int(sum(1 for x in stat if x != 0)),
            "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "requests_per_s": round(len(reqs) / el, 2), "saturated_requests_per_s": round(sat, 2),
            "arrival_rate": round(lam, 2), "steps": st["steps"], "max_concurrent": st["max_concurrent"],
            "pool": f"{len(pool)} graphs up to {nmax} vertices" + ("" if full else " (bounded sample of the mix)"),
            "parity": bool(checked > 0 and equal == checked), "parity_checked": checked,
            "parity_sample": len(sample), "parity_largest_n": nmax_checked,
            "cpu_oracle_ms_per_request": round(cpu_tot * 1e3 / max(checked, 1), 2),
            "cpu_oracle_threads": threads, "cpu_oracle_wall_s": round(parity_s, 1)}


# --------------------------------------------------------- reference arm ----

def run_reference(args, world, rank, pg):
    """The reference arm: the oracle as it stands on the machine's host cores.  A step is one
    sweep (or its first --ref-rounds rounds) with the pairs of each round refined side by
    side on all cores (fro_refine_batch_mt, identical results to the sequential sweep);
    --ref-threads 1 times the single-threaded sweep on its first --ref-pairs pairs."""
    if rank != 0:
        return
    import oracle as O
    w, desc = make_workload(args.workload)
    threads = args.ref_threads if args.ref_threads > 0 else len(os.sched_getaffinity(0))
    per_step = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        if threads > 1:
            st, _, _, _, done = O.refine_batch_mt(w, threads, max_rounds=args.ref_rounds if args.ref_rounds > 0 else -1)
        else:
            st, _, done = O.refine_batch_sample(w, args.ref_pairs)
        el = time.perf_counter() - t0
        assert st == 0
        if i >= args.warmup:
            per_step.append((done, el))
    pairs = sum(d for d, _ in per_step)
    tot = sum(e for _, e in per_step)
    value = pairs / tot
    if threads > 1:
        sample = ((f"first {args.ref_rounds} round(s)" if args.ref_rounds > 0 else "the whole sweep") +
                  f" per step ({per_step[0][0]} pairs), the pairs of a round on {threads} threads "
                  f"(validation and rounds included)")
    else:
        sample = (f"first {args.ref_pairs} pairs of one sweep in round order per step (validation and rounds "
                  f"included), single thread")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot / args.steps * 1e3, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
           "config": {"workload": desc, "n": w["n"], "nnz": w["nnz"], "k": w["k"]},
           "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": threads,
                            "kind": "oracle" if threads == 1 else "oracle, pair-parallel", "sample": sample},
           "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rgg3d", choices=["rgg3d", "grid3d", "grid2d", "rgg2d"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--sweep-sched", type=int, default=0, choices=[0, 1],
                    help="0: queue sweep (every pair in one launch of clusters), 1: round by round")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-pairs", type=int, default=6, help="reference arm, single thread: pairs per step")
    ap.add_argument("--ref-threads", type=int, default=0, help="reference arm: host threads (0: all cores)")
    ap.add_argument("--ref-rounds", type=int, default=0, help="reference arm, threaded: rounds per step (0: the whole sweep)")
    ap.add_argument("--serve", action=argparse.BooleanOptionalAction, default=True,
                    help="serving measurement (p50/p99, parity on a 1 %% sample) in the JSON line")
    ap.add_argument("--serve-full", action=argparse.BooleanOptionalAction, default=True,
                    help="the full serving mix (48 graphs up to 2^21 vertices, 10,000 requests); "
                         "--no-serve-full: a bounded sample (24 graphs up to 2^18, 1,500 requests)")
    ap.add_argument("--compare", action=argparse.BooleanOptionalAction, default=True,
                    help="128^3 grid: batched sweep vs one pair per launch")
    ap.add_argument("--serve-requests", type=int, default=None)
    ap.add_argument("--active", action=argparse.BooleanOptionalAction, default=True,
                    help="active block scheduling with adaptive flow iterations on the bench workload")
    ap.add_argument("--fm", action=argparse.BooleanOptionalAction, default=True,
                    help="sweeps with the two-way FM step before each flow (1 %% and 5 %% stopping rules)")
    ap.add_argument("--vcycle", action=argparse.BooleanOptionalAction, default=True,
                    help="one multilevel V-, F- and W-cycle with the workload's partition, a sweep per level")
    ap.add_argument("--next-rows", action=argparse.BooleanOptionalAction, default=True,
                    help="FM sweep, active scheduling and a V-cycle at 1/16 scale, and the two single-pair "
                         "configurations, each against the oracle")
    ap.add_argument("--mt", action=argparse.BooleanOptionalAction, default=True,
                    help="one multi-try FM pass over the first matching and the global k-way rounds, against the oracle's")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        log("warm-up raised to 3 (timing rule)")
        args.warmup = 3
    world, rank, local, pg = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank, pg)
    else:
        run_ours(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
