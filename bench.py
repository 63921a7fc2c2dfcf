"""Benchmark of the GIS hot path on GB300.

One step = one whole solve of the 4-D cart-pole workload (48^4 root cells,
2^4 corner samples, 9 forces, one RK4 step of 0.02, two levels of boundary
subdivision, OUTER rule, FP32 propagation with the certified recheck tiers):
leaf materialisation, propagation, image boxes, recheck, count / scan / fill,
transpose, prune, boundary classification and subdivision, through the C ABI
of libgis. `--workload cstr_256` runs the dimensionless-CSTR workload (256^2
roots, 3 levels); batch_512, serving_2000 and cstr_paper_rings have runners
of their own.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gis|reference]
                  [--workload cartpole_48|cstr_256|vdp_64|batch_512|serving_2000|cstr_paper_rings]

Prints one JSON line (rank 0). The metric is graph-construction throughput:
live cells whose graph was built, summed over the levels of the solve, per
second of solve time. --impl reference times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "graph-construction cells/s"
UNIT = "cells/s"
FP32_LANES_PER_SM = 128

# Plain operations of one evaluation of each model's right-hand side g(x, u),
# counted from its defining expression: (add / sub / mul with an FMA as 2, a
# division by a parameter counted as the product with its reciprocal;
# divisions by a state-dependent value; exp / sin / cos). The last two go to
# the special-function units and are reported beside the FLOPs, not in them.
RHS_OPS = {"vdp": (6, 0, 0), "cstr_dl": (11, 1, 1), "cartpole": (17, 1, 2), "cstr_paper": (12, 1, 1)}
RK4_OPS_PER_DIM = 13   # three stage states (2 each) and the weighted update (7)


def pair_work(prob):
    """Algorithmic work of one (cell, control) pair of propagation and bbox:
    S s (4 f_g + 13 n) FLOPs plus 2 n (S - 1) compares (one map application
    instead of s RK4 substeps for a discrete map), and its SFU operations."""
    n, k, s = prob["n"], prob["k"], prob["substeps"]
    S = k ** n
    if prob["dyn"] == "linmap":
        f_g, div, tr = 2 * n * (n + prob.get("m", 1)), 0, 0
    else:
        f_g, div, tr = RHS_OPS[prob["dyn"]]
    if s == 0:
        flops, sfu = S * f_g, S * (div + tr)
    else:
        flops, sfu = S * s * (4 * f_g + RK4_OPS_PER_DIM * n), S * s * 4 * (div + tr)
    return flops + 2 * n * (S - 1), sfu


def graph_bytes(prob, pairs, pair_edges, builds):
    """Algorithmic bytes of edge construction: the targets (4 per
    (cell, control) edge), the pair offsets (8 per pair and build), the image
    box re-read by the fill (8n per pair) and the count pass's count and flag
    (5 per pair)."""
    n = prob["n"]
    return 4.0 * pair_edges + 8.0 * (pairs + builds) + 8.0 * n * pairs + 5.0 * pairs


# DRAM traffic of the graph phase's kernels (chunk counts, count walk, scans,
# place / fill, the carried cells' edges) per (cell, control) edge, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of a smaller case of
# the same system: cart-pole at 20^4 roots, 25.79 GB over 771 113 918 edges.
# Scaled by the workload's own edge count; to be dropped when these kernels
# change.
GRAPH_TRAFFIC = {"cartpole_48": 33.45}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gis", choices=["gis", "reference"])
    ap.add_argument("--workload", default="cartpole_48")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def _workload(name):
    from paper_2202_06111_gb300 import workloads as W
    if name == "cstr_256":
        return W.cstr_256()
    if name == "cartpole_48":
        return dict(W.cartpole_48(), rule="outer")
    if name == "vdp_64":
        return W.vdp_64()
    if name == "serving_2000":
        return {"serving": W.serving_2000()}
    if name == "batch_512":
        return {"batch": W.batch_512()}
    if name == "cstr_paper_rings":
        return {"rings": dict(W.cstr_paper_problem(n0=(16, 16), levels=6), rule="outer")}
    raise SystemExit(f"unknown workload {name}")


def _config(prob, name):
    return {"workload": name, "system": prob["dyn"], "root_cells": prob["n0"], "samples_per_dim": prob["k"],
            "controls": len(prob["controls"]), "levels": prob["levels"], "rule": prob.get("rule", "inner"),
            "precision": "fp32 propagation, fp64 recheck" if prob.get("precision") == "fp32" else "fp64",
            "recheck": "certified FP32 intervals, FP64 where a grid line may fall inside", "l2": "flushed (512 MiB write) before every timed step"}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_ranks(total_ms, cells, ws, device="cpu"):
    """Whole-job throughput of ws independent replicas (one per rank, no
    data-path collective): the cells every rank built over the slowest rank's
    time. Returns (max time in ms, cells over all ranks, cells/s)."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        c = torch.tensor([float(cells)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        total_ms, cells = float(t.item()), float(c.item())
    return total_ms, cells, cells / (total_ms / 1e3)


def _oracle_solve(prob):
    """One FP64 oracle solve: (cells built, seconds, seconds per phase)."""
    import oracle
    ph = {"build_graph": 0.0, "prune": 0.0, "subdivide": 0.0}
    t0 = time.perf_counter()
    s = oracle.Solver(prob)
    cells = 0
    for L in range(prob["levels"] + 1):
        t = time.perf_counter()
        s.build_graph()
        ph["build_graph"] += time.perf_counter() - t
        cells += s.num_live()
        t = time.perf_counter()
        s.prune()
        ph["prune"] += time.perf_counter() - t
        if L < prob["levels"]:
            t = time.perf_counter()
            s.subdivide()
            ph["subdivide"] += time.perf_counter() - t
    return cells, time.perf_counter() - t0, ph


# Workloads whose whole oracle solve is too large for a bounded sample (the
# 48^4 cart-pole's level-2 graph alone would need over 100 GB of host memory
# in the oracle's per-pair layout): the sample is the oracle's graph
# construction of a run of the level-0 cells instead, `SLICE_CELLS` a step.
SLICE_CELLS = {"cartpole_48": 400_000}


class OracleSampler:
    """Bounded samples of the oracle's graph construction on a workload: a
    whole solve where one is short, else consecutive runs of level-0 cells."""

    def __init__(self, prob, name):
        import oracle
        oracle.build()
        self.threads = oracle.set_threads(0)
        self.prob, self.slice = prob, SLICE_CELLS.get(name)
        self.solver, self.next = None, 0
        if self.slice:
            self.solver = oracle.Solver(prob)
            t = time.perf_counter()
            self.solver.build_slice(0, 0)          # numbers the level-0 covering once
            self.setup_s = time.perf_counter() - t
            self.n_cells = self.solver.num_live()

    def describe(self):
        if self.slice:
            return (f"FP64 oracle graph construction (image boxes, flags, edges) of {self.slice} consecutive "
                    f"level-0 cells of the {self.n_cells} per step, on {self.threads} host threads; "
                    f"the whole solve does not fit the sample (nor host memory at level 2)")
        return f"one full FP64 oracle solve of the workload per step, on {self.threads} host threads"

    def step(self):
        """(cells, seconds, per-phase seconds) of one sample."""
        if not self.slice:
            return _oracle_solve(self.prob)
        first = self.next
        if first >= self.n_cells:
            first = 0
        count = min(self.slice, self.n_cells - first)
        t = time.perf_counter()
        self.solver.build_slice(first, count)
        dt = time.perf_counter() - t
        self.next = first + count
        return count, dt, {"build_graph": dt}


def cpu_baseline(prob, name, target_s=15.0):
    """The oracle as it stands on all host threads, on a bounded sample of the
    workload (about target_s seconds)."""
    smp = OracleSampler(prob, name)
    cells, secs, phases = 0, 0.0, {}
    while True:
        c, dt, ph = smp.step()
        cells += c
        secs += dt
        for k, v in ph.items():
            phases[k] = phases.get(k, 0.0) + v
        if secs >= target_s or not smp.slice:
            break
    return {"value": cells / secs, "unit": UNIT, "cores": smp.threads, "kind": "oracle",
            "sample": f"{smp.describe()}; {cells} cells in {secs:.1f} s", "phases_s": phases}


def run_reference(a, prob):
    ws, rank, local = _dist()
    if rank != 0:
        return
    smp = OracleSampler(prob, a.workload)
    times, cells, phases = [], 0, {}
    for i in range(a.warmup + a.steps):
        c, dt, ph = smp.step()
        if i >= a.warmup:
            times.append(dt)
            cells += c
            for k, v in ph.items():
                phases[k] = phases.get(k, 0.0) + v / a.steps
    ms = 1e3 * sum(times) / len(times)
    value = cells / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": _config(prob, a.workload),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": smp.threads, "kind": "oracle",
                             "sample": smp.describe(), "phases_s": phases},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _kept_key_set(ctx):
    import numpy as np
    lv, idx = ctx.kept_cells()
    rows = np.concatenate([lv[:, None].astype(np.int64), idx.astype(np.int64)], axis=1)
    return rows[np.lexsort(rows.T[::-1])] if len(rows) else rows


def _roofline(prob, name, agg, steps, peaks, src, sms):
    """Per-phase achieved work against the peaks, from the library's CUDA-event
    phase times: propagation in algorithmic FLOPs (pair_work), edge
    construction and pruning in algorithmic bytes. The dominant phase (most
    time) is the headline."""
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    hbm = float(peaks["hbm_gbs"])
    flops_pp, sfu_pp = pair_work(prob)
    pairs_prop = agg["cum_pairs_propagated"]
    pairs_built = agg["cum_cells_built"] * len(prob["controls"])
    builds = steps * (prob["levels"] + 1)
    phases = {}
    t_prop = agg["ms_prop"] / 1e3
    t_a5 = (agg["ms_prop"] + agg["ms_bin"] + agg["ms_recheck"]) / 1e3
    alg_flops = flops_pp * pairs_prop
    if t_prop > 0:
        phases["prop"] = {"kernels": "k_bound + k_propf_lat / k_propf_sib / k_propf (plain samples), "
                                     "k_prop32_lat / k_prop32_sib / k_prop32 (balls), k_prop64",
                          "ms_per_step": 1e3 * t_prop / steps, "bound": "alu", "unit": "TFLOP/s",
                          "achieved": alg_flops / t_prop / 1e12, "frac": alg_flops / t_prop / 1e12 / fp32_peak,
                          "flops_per_pair": flops_pp, "sfu_ops_per_pair": sfu_pp,
                          "executed_certified_tflops": agg["prop_flops"] / t_prop / 1e12,
                          "with_bin_and_recheck_frac": alg_flops / t_a5 / 1e12 / fp32_peak}
    t_graph = (agg["ms_count"] + agg["ms_scan"] + agg["ms_fill"] + agg["ms_transpose"]) / 1e3
    gb = graph_bytes(prob, pairs_built, agg["cum_edges"], builds)
    if t_graph > 0:
        phases["graph"] = {"kernels": "k_cchunks, k_cexpand, k_cedges, k_cinc, scans, k_place",
                           "ms_per_step": 1e3 * t_graph / steps, "bound": "hbm", "unit": "GB/s",
                           "achieved": gb / t_graph / 1e9, "frac": gb / t_graph / 1e9 / hbm,
                           "bytes_per_step": gb / steps}
    t_prune = agg["ms_prune"] / 1e3
    if t_prune > 0:
        phases["prune"] = {"kernels": "k_cprune_init, k_cprune", "ms_per_step": 1e3 * t_prune / steps,
                           "bound": "hbm", "unit": "GB/s", "achieved": agg["prune_bytes"] / t_prune / 1e9,
                           "frac": agg["prune_bytes"] / t_prune / 1e9 / hbm,
                           "bytes_per_step": agg["prune_bytes"] / steps}
    for k in ("ms_bin", "ms_recheck", "ms_classify", "ms_split", "ms_other"):
        phases[k[3:]] = {"ms_per_step": agg[k] / steps}
    dom = max(("prop", "graph", "prune"), key=lambda k: phases.get(k, {}).get("ms_per_step", -1))
    d = phases[dom]
    traffic = None
    tr = GRAPH_TRAFFIC.get(name) if dom == "graph" else None
    if tr:
        traffic = tr * agg["cum_edges"] / steps
    roof = {"bound": d["bound"], "kernel": dom, "achieved": d["achieved"],
            "peak": fp32_peak if d["bound"] == "alu" else hbm, "unit": d["unit"], "frac": d["frac"],
            "traffic": traffic,
            "peak_source": ("derived: SMs x 128 FP32 lanes x 2 x max SM clock (MEASURED_PEAKS.json has no FP32 "
                            "figure)" if d["bound"] == "alu" else f"{src} HBM copy (MEASURED_PEAKS.json hbm_gbs)"),
            "work": ("algorithmic FLOPs: S s (4 f_g + 13 n) + 2 n (S - 1) per propagated pair" if dom == "prop" else
                     "algorithmic bytes: 4 per (cell, control) edge + (8 + 8n + 5) per pair + 8 per build"
                     if dom == "graph" else "algorithmic bytes of the frontier prune"),
            "phases": phases}
    return roof


def run_gis(a, prob):
    import torch
    from paper_2202_06111_gb300 import build, gis
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    build.build()
    gis.load()
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def solve_once(p=prob, timing=1):
        return gis.Context(p, stream=stream.cuda_stream, timing=timing)

    # warm-up (also builds the memory pool and any cached shapes)
    for _ in range(a.warmup):
        with torch.cuda.stream(stream):
            c = solve_once()
            c.solve()
            c.close()
    torch.cuda.synchronize()

    # timed: device time of gis_solve, CUDA events on the library's stream. Each
    # step creates its context before the first event and closes it after the
    # second, so the library's memory pool is reused as in a serving loop.
    if ws > 1:
        torch.distributed.barrier()
    clk = Clocks(dev) if rank == 0 else None
    per_step, stats = [], []
    kept32 = None
    torch.cuda.synchronize()
    for i in range(a.steps):
        with torch.cuda.stream(stream):
            c = solve_once()
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.solve()
        e1.record(stream)
        e1.synchronize()
        per_step.append(e0.elapsed_time(e1))
        stats.append(c.stats())
        if i == 0:
            kept32 = _kept_key_set(c)
        c.close()
    torch.cuda.synchronize()
    clocks = clk.stop() if clk else None
    cells = sum(s["cum_cells_built"] for s in stats)
    edges = sum(s["cum_edges"] for s in stats)
    launches = sum(s["cum_launches"] for s in stats)
    total_ms, _, value = aggregate_ranks(sum(per_step), cells, ws, "cuda")

    # end to end through the C ABI: create from host arrays, solve, read the
    # live cells (with their kept flags) back into host memory
    e2e_times, d2h = [], 0
    h2d = len(prob["controls"]) * 8 * prob.get("m", 1) + 8 * (32 + 4) + 8 * 8 + 4 * 5
    for i in range(max(2, min(5, a.steps // 2))):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        with torch.cuda.stream(stream):
            c = gis.Context(prob, stream=stream.cuda_stream)
            c.solve()
            lv, fl, idx = c.cells()
        dt = time.perf_counter() - t
        d2h = lv.size * 24
        c.close()
        e2e_times.append(dt)
    e2e_value = (cells / len(stats)) / statistics.mean(e2e_times)

    # the same workload with every sample in FP64 (the plain FP64 GPU form), and
    # whether it keeps the same cells
    p64 = dict(prob, precision="fp64")
    fp64_runs = 2 if statistics.mean(per_step) < 1000 else 1
    with torch.cuda.stream(stream):
        c = gis.Context(dict(p64, n0=[4] * prob["n"]), stream=stream.cuda_stream)   # loads the FP64 kernels
        c.solve()
        c.close()
    fp64_ms, same = [], None
    for i in range(fp64_runs):
        flush.zero_()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            c = gis.Context(p64, stream=stream.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.solve()
        e1.record(stream)
        e1.synchronize()
        fp64_ms.append(e0.elapsed_time(e1))
        if i == 0:
            k64 = _kept_key_set(c)
            same = bool(k64.shape == kept32.shape and (k64 == kept32).all())
        c.close()

    # the cstr workload's headline rule is INNER, which removes nothing after
    # level 0 there; the paper's OUTER reading removes cells at every level
    outer = None
    if prob.get("rule", "inner") == "inner" and prob["n"] == 2:
        po = dict(prob, rule="outer")
        oms, ost = [], None
        for i in range(3):
            flush.zero_()
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                c = solve_once(po)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c.solve()
            e1.record(stream)
            e1.synchronize()
            if i > 0:
                oms.append(e0.elapsed_time(e1))
            ost = c.stats()
            c.close()
        outer = {"rule": "outer", "ms_per_step": statistics.mean(oms),
                 "value": ost["cum_cells_built"] / (statistics.mean(oms) / 1e3), "unit": UNIT,
                 "cells_per_step": ost["cum_cells_built"], "kept": ost["n_kept"]}

    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
        return
    peaks, src = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    agg = {k: sum(s[k] for s in stats) for k in stats[0] if isinstance(stats[0][k], (int, float))}
    roofline = _roofline(prob, a.workload, agg, len(stats), peaks, src, sms)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": total_ms / len(per_step), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": _config(prob, a.workload),
            "edges_per_s": edges * ws / (total_ms / 1e3),
            "cell_edges_per_s": agg["cum_cell_edges"] * ws / (total_ms / 1e3),
            "solve_ms": {"mean": statistics.mean(per_step), "p50": statistics.median(per_step),
                         "p99": max(per_step)},
            "cells_per_step": cells / len(stats), "edges_per_step": edges / len(stats),
            "kept_cells": stats[-1]["n_kept"],
            "recheck_pairs_per_step": agg["cum_recheck"] / len(stats),
            "recheck_samples_per_step": agg["cum_recheck_samples"] / len(stats),
            "recheck_fp64_pairs_per_step": agg["cum_recheck_fp64"] / len(stats),
            "pairs_propagated_per_step": agg["cum_pairs_propagated"] / len(stats),
            "roofline": roofline, "gpu_launches": launches, "clocks": clocks,
            "shapes": {"lattice_tile_cells": stats[-1]["lattice_tile_cells"],
                       "sibling_parents": stats[-1]["sibling_parents"],
                       "lanes_per_pair": stats[-1]["lanes_per_pair"],
                       "picked_by": "autotuner, timed during the warm-up solves",
                       "tune_launches_timed": agg["cum_tune_launches"]},
            "fp64_plain": {"ms_per_step": statistics.mean(fp64_ms),
                           "speedup_of_fp32_recheck": statistics.mean(fp64_ms) / (total_ms / len(per_step)),
                           "same_kept_cells": same},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": 1e3 * statistics.mean(e2e_times)}}
    if outer:
        line["rule_outer"] = outer
    if ws == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob, a.workload)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()


def run_serving(a, reqs):
    """Real-time replay of Poisson arrivals through the continuous-batching server."""
    import threading

    import torch
    from paper_2202_06111_gb300 import build, gis, workloads as W

    build.build()
    gis.load()
    dev = torch.cuda.current_device()
    srv = gis.Server(device=dev)
    for r in W.serving_2000(count=8, seed=1, max_2d_cells=64.0 ** 2, max_4d_n0=8.0):   # warm-up
        srv.poll(srv.submit(r), wait=True, want_cells=False)
    base = srv.stats()
    lat, done_at = {}, {}
    submitted = {}
    lock = threading.Lock()
    t0 = time.perf_counter()

    def submitter():
        for i, r in enumerate(reqs):
            wait = t0 + r["arrival_s"] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            t = srv.submit(r)
            with lock:
                submitted[t] = (i, time.perf_counter())

    th = threading.Thread(target=submitter)
    clk = Clocks(dev)
    th.start()
    while len(done_at) < len(reqs):
        with lock:
            outstanding = [(t, v) for t, v in submitted.items() if t not in done_at]
        for t, (i, ts) in outstanding:
            res = srv.poll(t, wait=False, want_cells=True)
            if res is not None:
                now = time.perf_counter()
                done_at[t] = now
                lat[i] = (now - ts) * 1e3
                assert res["status"] == 0, res
        time.sleep(0.0005)
    th.join()
    clocks = clk.stop()
    wall = max(done_at.values()) - t0
    st = srv.stats()
    srv.close()
    lats = sorted(lat.values())
    cells = st["cells_built"] - base["cells_built"]
    line = {"metric": "serving requests/s", "value": len(reqs) / wall, "unit": "requests/s", "n_gpus": 1,
            "steps": len(reqs), "warmup": 8, "ms_per_step": 1e3 * wall / len(reqs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving_2000", "requests": len(reqs), "arrivals": "Poisson, mean 200/s",
                       "systems": "Van der Pol, CSTR, cart-pole", "grids": "32^2-1024^2, 16^4-48^4",
                       "levels": "0-3", "rule": "inner"},
            "latency_ms": {"p50": lats[len(lats) // 2], "p99": lats[min(len(lats) - 1, int(0.99 * len(lats)))],
                           "max": lats[-1]},
            "cells_per_s": cells / wall, "engine_steps": st["steps"] - base["steps"], "clocks": clocks,
            "oom_restarts": st["oom_restarts"] - base["oom_restarts"],
            "peak_device_gb": st["peak_device_bytes"] / 2 ** 30, "budget_gb": st["budget_bytes"] / 2 ** 30,
            "offered_load_s": reqs[-1]["arrival_s"]}
    print(json.dumps(line), flush=True)


def run_batch(a, probs):
    """512 uneven instances solved together (gis_batch_solve: every level of
    every active instance in the same launches), against the same instances
    solved one context at a time."""
    import torch
    from paper_2202_06111_gb300 import build, gis

    build.build()
    gis.load()
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        gis.batch_solve(probs[:16], stream=stream.cuda_stream, want_cells=False)
    torch.cuda.synchronize()
    clk = Clocks(dev)
    times, stats = [], []
    for _ in range(max(1, a.steps)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        with torch.cuda.stream(stream):
            res, st = gis.batch_solve(probs, stream=stream.cuda_stream, want_cells=False)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
        stats.append(st)
        assert all(r["status"] == 0 for r in res)
    clocks = clk.stop()
    cells = stats[-1]["cum_cells_built"]
    edges = stats[-1]["cum_edges"]
    launches = stats[-1]["cum_launches"]
    # the same instances one context each (sequential)
    t = time.perf_counter()
    seq_cells = 0
    for p in probs:
        with torch.cuda.stream(stream):
            c = gis.Context(p, stream=stream.cuda_stream)
            c.solve()
            seq_cells += c.stats()["cum_cells_built"]
            c.close()
    torch.cuda.synchronize()
    seq = time.perf_counter() - t
    wall = statistics.median(times)
    line = {"metric": "graph-construction cells/s", "value": cells / wall, "unit": "cells/s", "n_gpus": 1,
            "steps": len(times), "warmup": 1, "ms_per_step": 1e3 * wall, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch_512", "instances": len(probs),
                       "systems": "Van der Pol mu~U[0.5,2] / CSTR Da~U[0.06,0.09]",
                       "grids": "log-uniform 32^2-512^2", "samples_per_dim": 3, "controls": "5-11",
                       "levels": "0-3", "precision": "fp32 propagation, double-word / fp64 recheck"},
            "edges_per_s": edges / wall, "cells_per_step": cells, "gpu_launches": launches,
            "sequential": {"ms": 1e3 * seq, "cells": seq_cells, "speedup_of_batch": seq / wall},
            "e2e": {"value": cells / wall, "unit": "cells/s", "note": "host request arrays to host results"},
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_rings(a, prob):
    """The paper's own CSTR (Eq. 4, Table 2) refined six times, splitting the
    boundary cells only (ring 0, the exact rule) or also the kept cells within
    1, 3, 5 rings of them (the neighbourhood that stands in for the N nearest
    neighbours of Sec. 3.1.2), against splitting every kept cell (-1): solve
    time, cells built, and the kept volume (the outer approximation's size,
    smaller is tighter)."""
    import numpy as np
    import torch
    from paper_2202_06111_gb300 import build, gis

    build.build()
    gis.load()
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    n = prob["n"]
    roots = float(np.prod(prob["n0"]))
    clk = Clocks(dev)
    rings = {}
    for ring in (0, 1, 3, 5, -1):
        p = dict(prob, split_ring=ring)
        ms, st, vol = [], None, 0.0
        for it in range(max(1, a.warmup) + max(1, a.steps)):
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                c = gis.Context(p, stream=stream.cuda_stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c.solve()
            e1.record(stream)
            e1.synchronize()
            if it >= max(1, a.warmup):
                ms.append(e0.elapsed_time(e1))
            st = c.stats()
            lv, _ = c.kept_cells()
            vol = float(np.sum(np.ldexp(1.0, -n * lv.astype(np.int64)))) / roots
            c.close()
        rings["all" if ring < 0 else str(ring)] = {
            "ms": statistics.median(ms), "cells_built": st["cum_cells_built"], "kept": int(st["n_kept"]),
            "kept_volume_fraction": vol}
    clocks = clk.stop()
    r0 = rings["0"]
    line = {"metric": "graph-construction cells/s", "value": r0["cells_built"] / (r0["ms"] / 1e3),
            "unit": "cells/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": r0["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "cstr_paper_rings", "system": "cstr_paper (Eq. 4, Table 2)",
                       "root_cells": prob["n0"], "samples_per_dim": prob["k"], "controls": len(prob["controls"]),
                       "levels": prob["levels"], "rule": "outer", "split": "boundary + rings 0/1/3/5, or all",
                       "precision": "fp32 propagation, double-word / fp64 recheck"},
            "rings": rings, "all_split_over_adaptive": rings["all"]["ms"] / r0["ms"], "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    a = _args()
    prob = _workload(a.workload)
    if "rings" in prob:
        if a.impl == "gis":
            run_rings(a, prob["rings"])
        return
    if "batch" in prob:
        if a.impl == "gis":
            run_batch(a, prob["batch"])
        return
    if "serving" in prob:
        if a.impl == "gis":
            run_serving(a, prob["serving"][: a.steps] if a.steps < len(prob["serving"]) else prob["serving"])
        return
    if a.impl == "reference":
        run_reference(a, prob)
    else:
        run_gis(a, prob)


if __name__ == "__main__":
    main()
