#!/usr/bin/env python3
"""IFP2 PageRank benchmark on one GB300 (replicas on N GPUs).

Workload: the single-graph configuration -- directed R-MAT (a,b,c,d) =
(0.57,0.19,0.19,0.05), scale 22 (4,194,304 vertices), edge factor 16
(67,108,864 sampled edges; self-loops and repeats removed), out-edges of a
seeded 20% of vertices and in-edges of an independent 10% deleted, vertex
ids randomly relabelled; c = 0.85, uniform p, IFP2 stopped at residual L1
<= 1e-9, mass carried as double-float pairs (48-bit significand on FP32
instructions; GB300's FP64 pipe is 1/64 of its FP32 rate), with the IEEE
FP64 and FP32 forms measured alongside.  One step = one pr_solve on the resident, preprocessed
graph (frontier activation, push/pull rounds, phase 2, normalisation).

Metric: GEdges pushed per second = (sum over rounds of the frontier's valid
out-edges + phase-2 in-edges of dangling vertices) / solve time.  Alongside:
the same-GPU Power method timed to the same L1 error, the FP32 form, the
preprocessing time, the roofline of the dominant kernel, the end-to-end rate
through host buffers, SM clocks, and the FP64 oracle timed on the host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IFP2 GEdges/s + %HBM peak vs GPU Power method; served p50/p99 ms at L1<=1e-6"
UNIT = "GEdges/s"
C = 0.85


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--scale", type=int, default=22, help="R-MAT scale (22 = the benchmark workload)")
    ap.add_argument("--eps", type=float, default=1e-9)
    ap.add_argument("--skip-extras", action="store_true", help="only the timed IFP2 steps")
    ap.add_argument("--host-rounds", action="store_true",
                    help="launch rounds from the host instead of the CUDA-graph while loop (same kernels; "
                         "lets a profiler see each launch)")
    ap.add_argument("--out", default=None, help="also write the JSON line to this file")
    return ap.parse_args()


def workload(scale):
    return dict(workload=f"rmat{scale}_ifp2_df64", graph="R-MAT (0.57,0.19,0.19,0.05)", scale=scale,
                vertices=1 << scale, edge_factor=16, sampled_edges=16 << scale, dangling_deleted=0.20,
                unref_deleted=0.10, relabel="seeded random permutation", seed=1, c=C, p="uniform",
                algo="IFP2", precision="df64", eps=1e-9)


def make_graph(scale):
    import graphgen as gg
    return gg.rmat(scale, 16, dangling=0.20, unref=0.10, seed=1)


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ roofline
def algorithmic_bytes_pull_round(info, s, scan_entries, rows, active_rows):
    """k_round_pull: per scanned in-list entry 4 B (source id) + s (gathered w);
    per row 4 B (offset) + 2s (r read and write) + the next activation's s (w write)
    + s (1/deg) + 4 B (valid out-degree); per active row 2s (x read and write)."""
    return scan_entries * (4 + s) + rows * (8 + 4 * s) + active_rows * 2 * s


def algorithmic_bytes_activate(n_nd, s):
    """k_activate: per non-dangling vertex s (r) + s (w write) + 4 (out offset) + 4 (valid degree) + s (1/deg)."""
    return n_nd * (3 * s + 8)


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def source_hash():
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_2302_03245_gb300", "csrc"))):
        h.update(open(os.path.join(ROOT, "paper_2302_03245_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload_name):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    e = rec.get(f"{kernel}@{workload_name}")
    if not e or e.get("source_hash") != source_hash():
        return None
    return e.get("dram_bytes_per_launch")


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    """The FP64 oracle's synchronous-round IFP2 on the same graph, on host cores:
    each step is a bounded sample (the first rounds of the solve)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import graphgen as gg
    import oracle

    g = make_graph(args.scale)
    p = gg.p_uniform(g.n)
    rounds = 3 if args.scale >= 20 else 50
    times, edges = [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        out = oracle.ifp_rounds(oracle.IFP2, g, C, args.eps, p, max_rounds=rounds)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            edges.append(int(out["E"].sum()))
    value = sum(edges) / sum(times) / 1e9
    sample = (f"first {rounds} synchronous IFP2 rounds (snapshot, (1-c) reserve) of the FP64 oracle on the full "
              f"graph (n={g.n}, m={g.m}), single thread, per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload(args.scale),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    emit(line, args)


def emit(line, args):
    s = json.dumps(line)
    print(s, flush=True)
    if args.out:
        with open(args.out, "w") as f:
            f.write(s + "\n")


# ------------------------------------------------------------------ GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    import graphgen as gg
    import paper_2302_03245_gb300 as pr

    stream = torch.cuda.current_stream()
    pr.use_torch_allocator(True)
    g = make_graph(args.scale)
    st_g = g.stats()
    off, dst = g.csr32()
    d_off = torch.from_numpy(off).cuda()
    d_dst = torch.from_numpy(dst).cuda()
    torch.cuda.synchronize()
    G = pr.Graph(g.n, g.m, d_off, d_dst, mem_is_device=True, stream=stream)
    info = G.info
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)

    def solve(algo=pr.PR_IFP2, prec=pr.PR_DF64, eps=args.eps, opts=None):
        opts = dict(opts or {})
        if args.host_rounds:
            opts.setdefault("use_graph", -1)
        _, st, status = G.solve(C, eps, algo, prec, out=out, opts=opts)
        assert status == pr.PR_OK, st
        return st

    for _ in range(args.warmup):
        solve()
    clocks = Clocks(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms, edges, launches, rounds = [], [], 0, []
    t_all0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = solve()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        edges.append(st["edges_pushed"])
        launches += st["launches"]
        rounds.append(st["rounds"])
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_all0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    t_step = sum(ms) / len(ms)
    my_edges, my_time = float(sum(edges)), sum(ms) / 1e3
    if dist:
        tt = torch.tensor([my_time], device="cuda", dtype=torch.float64)
        ee = torch.tensor([my_edges], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dist.all_reduce(ee, op=dist.ReduceOp.SUM)
        my_time, my_edges = float(tt.item()), float(ee.item())
    value = my_edges / my_time / 1e9

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "df64 (fp32 hi+lo pairs; fp64 final sums and output)",
            "data": "synthetic",
            "config": dict(workload(args.scale), l2="512 MB buffer written between timed steps",
                           parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
            "gpu_launches": int(launches), "clocks": clk,
            "graph": {k: info[k] for k in ("n", "m", "n_nd", "n_ref", "n_d", "m_d", "n_u", "max_outdeg",
                                             "max_indeg")},
            "rounds": rounds[0], "edges_pushed_per_step": edges[0], "wall_s_timed": wall}
    if rank != 0 or args.skip_extras:
        if rank == 0:
            emit(line, args)
        if dist:
            dist.destroy_process_group()
        return

    peaks = measured_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    peak_src = "measured" if peaks else "fallback"

    # ---- per-kernel CUDA-event timing (instrumented pass of the same solve)
    prof_runs = 2
    agg = {}
    tr_cap = 4096
    for _ in range(prof_runs):
        flush.zero_()
        st = solve(opts=dict(profile=1, trace_cap=tr_cap))
        for k, v in st["profile"].items():
            a = agg.setdefault(k, dict(launches=0, ms=0.0))
            a["launches"] += v["launches"]
            a["ms"] += v["ms"]
    trace = st["trace"]
    nr = st["rounds"]
    modes = trace["mode"][:nr]
    pull_rounds = np.nonzero(modes == 2)[0]
    total_k_ms = sum(v["ms"] for v in agg.values())
    dom = max(agg, key=lambda k: agg[k]["ms"])
    s = 8
    # in-list entries read by the pull rounds: everything the solve scanned minus the push
    # rounds' out-edges and the phase-2 in-edges of dangling vertices
    push_rounds = np.nonzero(modes == 1)[0]
    pull_scan_total = st["edges_scanned"] - int(trace["E"][push_rounds].sum()) - info["m_d"]
    scan_ref = pull_scan_total / max(len(pull_rounds), 1)
    kernels = {k: dict(launches=v["launches"] // prof_runs, avg_ms=v["ms"] / max(v["launches"], 1),
                       share=v["ms"] / total_k_ms) for k, v in agg.items()}
    if dom == "k_round_pull":
        F = trace["F"][pull_rounds].astype(np.float64)
        rows = info["n_nd"]
        bytes_per = [algorithmic_bytes_pull_round(info, s, scan_ref, rows, f) for f in F]
        alg_bytes = float(np.mean(bytes_per))
    elif dom == "k_activate":
        alg_bytes = float(algorithmic_bytes_activate(info["n_nd"], s))
    else:
        alg_bytes = float(np.mean(trace["E"][:nr])) * (4 + 2 * s)
    avg_ms = kernels[dom]["avg_ms"]
    achieved = alg_bytes / (avg_ms / 1e3) / 1e9
    line["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                        "frac": achieved / hbm_peak, "peak_source": f"{peak_src} (copy bandwidth)",
                        "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_ms,
                        "traffic": recorded_traffic(dom, workload(args.scale)["workload"]),
                        "timing": "CUDA events around every launch on the graph's stream, instrumented pass"}
    line["kernels"] = kernels

    # ---- accuracy and the Power method at equal L1
    truth = torch.empty_like(out)
    _, st_t, _ = G.solve(C, 1e-14, pr.PR_POWER, pr.PR_FP64, out=truth)
    ref_bound = st_t["err_bound"]
    solve()
    ifp2_l1 = float((out - truth).abs().sum())
    ifp2_ms = t_step
    legs = {"reference_solution": f"GPU Power IEEE FP64 to ||delta||_1 <= 1e-14 (certified L1 <= {ref_bound:.2e})",
            "ifp2_df64": dict(ms=ifp2_ms, l1=ifp2_l1, rounds=rounds[0], gedges_s=value)}
    for nm, algo, prec, eps in (("ifp2_fp64", pr.PR_IFP2, pr.PR_FP64, args.eps),
                                ("ifp1_df64", pr.PR_IFP1, pr.PR_DF64, args.eps),
                                ("ifp2_fp32", pr.PR_IFP2, pr.PR_FP32, 1e-6)):
        tms = []
        for _ in range(3):
            flush.zero_()
            st = solve(algo=algo, prec=prec, eps=eps)
            tms.append(st["ms"])
        legs[nm] = dict(ms=statistics.median(tms), l1=float((out - truth).abs().sum()), rounds=st["rounds"],
                        fp64_rounds=st["fp64_rounds"], eps=eps,
                        gedges_s=st["edges_pushed"] / (statistics.median(tms) / 1e3) / 1e9)
    for pname, pprec in (("df64", pr.PR_DF64), ("fp64", pr.PR_FP64)):
        power = []
        for tol in (1e-7, 3e-8, 1e-8, 3e-9, 1e-9, 3e-10, 1e-10, 3e-11, 1e-11):
            tms = []
            for _ in range(3):
                flush.zero_()
                st = solve(algo=pr.PR_POWER, prec=pprec, eps=tol)
                tms.append(st["ms"])
            err = float((out - truth).abs().sum())
            power.append(dict(tol=tol, ms=statistics.median(tms), l1=err, iters=st["rounds"]))
            if err <= ifp2_l1:
                break
        eq = next((q for q in power if q["l1"] <= ifp2_l1), None)
        legs[f"power_{pname}_ladder"] = power
        if eq:
            legs[f"power_{pname}_at_equal_l1"] = dict(eq, speedup_ifp2=eq["ms"] / ifp2_ms)
    line["vs_power"] = legs
    pre = []
    for _ in range(3):
        G2 = pr.Graph(g.n, g.m, d_off, d_dst, mem_is_device=True, stream=stream)
        pre.append(G2.info["ms_preprocess"])
        G2.close()
    line["preprocess_ms"] = statistics.median(pre)
    # %HBM of the whole solve on its algorithmic bytes
    alg_solve = 0.0
    for t in range(nr):
        if modes[t] == 2:
            alg_solve += algorithmic_bytes_pull_round(info, s, scan_ref, info["n_nd"], trace["F"][t])
        else:
            alg_solve += trace["E"][t] * (4 + 2 * s) + trace["F"][t] * (16 + 3 * s)
        alg_solve += algorithmic_bytes_activate(info["n_nd"], s)
    alg_solve += info["m_d"] * (4 + s) + info["n_d"] * (8 + 2 * s)
    line["solve_hbm_frac"] = alg_solve / (t_step / 1e3) / 1e9 / hbm_peak

    # ---- end to end through the C ABI with pinned host buffers
    h_off = torch.from_numpy(off).pin_memory()
    h_dst = torch.from_numpy(dst).pin_memory()
    h_out = torch.empty(g.n, dtype=torch.float64).pin_memory()
    e2e_ms, e2e_edges = [], []
    for k in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gh = pr.pr_graph_create(g.n, g.m, h_off, h_dst, mem_is_device=False, stream=stream)
        _, st, status = pr.pr_solve(gh, C, args.eps, pr.PR_IFP2, pr.PR_DF64, out=h_out)
        pr.pr_destroy(gh)
        torch.cuda.synchronize()
        if k > 0:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
            e2e_edges.append(st["edges_pushed"])
    line["e2e"] = {"value": sum(e2e_edges) / (sum(e2e_ms) / 1e3) / 1e9, "unit": UNIT,
                   "h2d_bytes_per_step": int(off.nbytes + dst.nbytes), "d2h_bytes_per_step": int(8 * g.n),
                   "ms_per_step": statistics.median(e2e_ms),
                   "includes": "pr_graph_create from pinned host CSR (copy, validation, preprocessing) + "
                               "pr_solve IFP2 df64 + copy of pi to pinned host memory"}

    # ---- the oracle on the host cores (bounded sample)
    import oracle
    p = gg.p_uniform(g.n)
    rounds_cpu = 3
    t0 = time.perf_counter()
    o = oracle.ifp_rounds(oracle.IFP2, g, C, args.eps, p, max_rounds=rounds_cpu)
    dt = time.perf_counter() - t0
    line["cpu_baseline"] = {"value": float(o["E"].sum()) / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"first {rounds_cpu} synchronous IFP2 rounds of the FP64 oracle on the full "
                                      f"graph, single thread ({dt:.1f} s)"}
    emit(line, args)
    G.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
