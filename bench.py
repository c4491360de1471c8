#!/usr/bin/env python3
"""IFP2 PageRank benchmark on one GB300 (replicas on N GPUs).

Workload: the single-graph configuration -- directed R-MAT (a,b,c,d) =
(0.57,0.19,0.19,0.05), scale 22 (4,194,304 vertices), edge factor 16
(67,108,864 sampled edges; self-loops and repeats removed), out-edges of a
seeded 20% of vertices and in-edges of an independent 10% deleted, vertex
ids randomly relabelled; c = 0.85, uniform p, IFP2 in IEEE FP64 (state,
pushed mass, gathers and sums in double, as in the paper) stopped at residual
L1 <= 5e-10, which puts the result within L1 1e-9 of the exact PageRank
(measured L1 / eps is about 1.35 on this graph); the double-float form
(48-bit significand on FP32 instructions; GB300's FP64 pipe is 1/64 of its
FP32 rate) and the FP32 form (eps 5e-7, L1 within 1e-6) are measured
alongside.  One step = one pr_solve on the resident, preprocessed graph
(frontier activation, push/pull rounds, phase 2, normalisation).

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
# Stopping thresholds that meet the accuracy gates (L1 <= 1e-9 for FP64 and
# double-float solves, <= 1e-6 for the FP32 form) against the exact PageRank:
# on the R-MAT graphs here IFP2 stops at an L1 error of about 1.2-1.35 x eps,
# so half the gate leaves a margin of about 1.5.  The certified stop for a
# gate tol is tol (1 - c) / 2 (0.15 x tol).
EPS_FP64 = 5e-10
EPS_FP32 = 5e-7
# Served requests mix personalization vectors and graphs, where L1 / eps is not
# one measured ratio (personalized requests measured up to 4 x eps): the
# server uses the certified stop for the 1e-6 gate, IFP2's L1 <= 2 R / (1 - c).
EPS_SERVE = 1e-6 * (1 - C) / 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--scale", type=int, default=22, help="R-MAT scale (22 = the benchmark workload)")
    ap.add_argument("--eps", type=float, default=EPS_FP64)
    ap.add_argument("--prec", default="fp64", choices=["fp64", "df64", "fp32"],
                    help="precision of the timed steps (fp64 = the headline)")
    ap.add_argument("--serve-scale", type=int, default=23, help="R-MAT scale of the resident serving graph")
    ap.add_argument("--serve-rates", default="100,300,1000,3000,10000,20000", help="arrival rates (requests/s)")
    ap.add_argument("--serve-max", type=int, default=400, help="requests per rate at most")
    ap.add_argument("--serve-window", type=float, default=2.0,
                    help="seconds of arrivals per rate (requests per rate = min(rate x window, --serve-max)); "
                         "--serve-window 1e9 --serve-max 10000 is the full 10k-request mix")
    ap.add_argument("--algo", default="ifp2", choices=["ifp2", "ifp1", "power"],
                    help="algorithm of the timed steps (ifp2 = the headline)")
    ap.add_argument("--apull", action="store_true",
                    help="run the timed IFP steps in asynchronous pull rounds (PR_MODE_APULL) instead of the "
                         "synchronous push/pull rounds (the headline)")
    ap.add_argument("--levels", type=int, default=0,
                    help="prepare the graph with this many levels and run the timed IFP2 steps in "
                         "level-ordered rounds (PR_MODE_LEVELS); 0 = synchronous rounds (the headline)")
    ap.add_argument("--skip-extras", action="store_true", help="only the timed IFP2 steps")
    ap.add_argument("--host-rounds", action="store_true",
                    help="launch rounds from the host instead of the CUDA-graph while loop (same kernels; "
                         "lets a profiler see each launch)")
    ap.add_argument("--out", default=None, help="also write the JSON line to this file")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON file of autotuned launch parameters (read if it has this graph, else written)")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch parameters")
    ap.add_argument("--legs", default="dag,batch,serve,sweep,undirected,threads",
                    help="extra configurations after the headline: dag (scale-24 DAG-heavy, FP32 form), "
                         "batch (512 graphs in one batch), serve (continuous batching), sweep (time and "
                         "error against eps), undirected (symmetric scale-22 graph), threads (CTA-count "
                         "sweep); '' for none")
    return ap.parse_args()


PREC_LABEL = {"fp64": "IEEE FP64 (state, gathers and sums in double)",
              "df64": "double-float (fp32 hi+lo pairs, 48-bit significand; fp64 final sums and output)",
              "fp32": "FP32 state and gathers, FP64 sums, IEEE FP64 correction sweep and rounds after it"}


def workload(scale, algo="ifp2", levels=0, prec="fp64", eps=EPS_FP64, apull=False):
    lv = f"_levels{levels}" if levels and algo == "ifp2" else ""
    ap = "_apull" if apull and algo != "power" else ""
    rounds = ("level-ordered, %d levels" % levels if lv else
              "asynchronous pull (rows recompute their residual from the reserves)" if ap else "synchronous")
    return dict(workload=f"rmat{scale}_{algo}{lv}{ap}_{prec}", graph="R-MAT (0.57,0.19,0.19,0.05)", scale=scale,
                vertices=1 << scale, edge_factor=16, sampled_edges=16 << scale, dangling_deleted=0.20,
                unref_deleted=0.10, relabel="seeded random permutation", seed=1, c=C, p="uniform",
                algo=algo.upper() if algo != "power" else "Power", precision=PREC_LABEL[prec], eps=eps,
                rounds=rounds)


def make_graph(scale):
    import graphgen as gg
    return gg.rmat(scale, 16, dangling=0.20, unref=0.10, seed=1)


def make_graph_device(scale):
    """The same graph as make_graph, generated on the GPU (graphgen.torchgen)."""
    from graphgen import torchgen as tg
    return tg.rmat(scale, 16, dangling=0.20, unref=0.10, seed=1, device="cuda")


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


def run_legs(args, line, pr, torch, stream, flush, hbm_peak, peak_src):
    """The extra configurations named by --legs, each reported in its own key."""
    legs = [x for x in args.legs.split(",") if x]
    extra = {}
    for leg in legs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            extra[leg] = LEGS[leg](pr, torch, stream, flush, hbm_peak, peak_src)
        except Exception as e:  # a failed leg is reported, the headline line still prints
            extra[leg] = {"error": f"{type(e).__name__}: {e}"}
        extra[leg]["leg_wall_s"] = time.perf_counter() - t0
        torch.cuda.empty_cache()
    keys = {"dag": "dag24", "batch": "batch512", "sweep": "eps_sweep", "serve": "serving",
            "undirected": "undirected22", "threads": "parallelism_sweep"}
    for leg, res in extra.items():
        line[keys.get(leg, leg)] = res
    sv = extra.get("serve", {})
    if "rates" in sv:
        line["served_p50_p99_ms"] = {str(r["rate"]): [r["p50_ms"], r["p99_ms"]] for r in sv["rates"]}


def reduce_ranks(seconds, edges, dist, device):
    """Whole-job figures of independent replicas: the slowest rank's time and
    the edges all ranks pushed (no reduction when dist is None)."""
    if dist is None:
        return seconds, edges
    import torch
    tt = torch.tensor([seconds], device=device, dtype=torch.float64)
    ee = torch.tensor([edges], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(ee, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(ee.item())


def info_sms(torch):
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def median_solve(G, flush, reps, *a, **kw):
    """Median device ms of `reps` solves (L2 flushed before each) and the last stats.
    With --host-rounds the rounds are launched from the host (for a profiler)."""
    if ARGS is not None and ARGS.host_rounds:
        kw["opts"] = dict(kw.get("opts") or {}, use_graph=-1)
    ms, st = [], None
    for _ in range(reps):
        flush.zero_()
        _, st, status = G.solve(*a, **kw)
        assert status == 0, st
        ms.append(st["ms"])
    return statistics.median(ms), st


def pull_roofline(info, st, prof_ms, s_first, s_after, fp64_rounds, hbm_peak, peak_src):
    """Algorithmic bytes of the pull rounds of one traced solve (state bytes s_first
    before the correction, s_after after it) over their profiled device time."""
    tr = st["trace"]
    nr = st["rounds"]
    modes = tr["mode"][:nr]
    push_e = int(sum(tr["E"][t] for t in range(nr) if modes[t] == 1))
    scan = st["edges_scanned"] - push_e - info["m_d"]
    n_pull = max(int((modes == 2).sum()), 1)
    scan_per = scan / n_pull
    alg = 0.0
    for t in range(nr):
        if modes[t] == 2:
            s = s_first if t < nr - fp64_rounds else s_after
            alg += algorithmic_bytes_pull_round(info, s, scan_per, info["n_nd"], tr["F"][t])
    achieved = alg / (prof_ms / 1e3) / 1e9 if prof_ms > 0 else 0.0
    return {"bound": "hbm", "kernel": "k_round_pull", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "peak_source": f"{peak_src} (copy bandwidth)",
            "alg_bytes_per_launch": alg / n_pull, "avg_launch_ms": prof_ms / n_pull, "traffic": None}


def leg_dag(pr, torch, stream, flush, hbm_peak, peak_src):
    """Large DAG-heavy graph: R-MAT scale 24, edge factor 16, 70% of edges turned
    forward in a seeded random order, 25% dangling; IFP2 in the FP32 form (float
    state, FP64 sums, IEEE FP64 correction sweep and FP64 rounds after it), eps
    1e-9 as configured and 5e-10 (the FP64 gate's eps); delivery push-only,
    pull-only, asynchronous and AUTO; IFP2 in IEEE FP64 and double-float; Power
    at equal L1 in the same arithmetic."""
    from graphgen import torchgen as tg
    t0 = time.perf_counter()
    gd = tg.rmat(24, 16, dangling=0.25, unref=0.0, seed=1, dag_frac=0.7, device="cuda")
    off, dst = gd.csr32()
    G = pr.Graph(gd.n, gd.m, off, dst, mem_is_device=True, stream=stream)
    del gd, off, dst
    torch.cuda.synchronize()
    res = {"workload": "rmat24_dag70_ifp2_fp32", "graph_s": time.perf_counter() - t0,
           "graph": {k: G.info[k] for k in ("n", "m", "n_nd", "n_ref", "n_d", "m_d", "n_u", "max_indeg",
                                             "max_outdeg", "ms_preprocess")}}
    t0 = time.perf_counter()
    if ARGS is not None and ARGS.no_tune:
        tuning, rep = G.tuning(), "default launch parameters (--no-tune)"
    else:
        tuning, rep = G.autotune(pr.PR_FP32, max_ms=2000.0)
    res["tuning"] = dict(tuning, autotune_s=time.perf_counter() - t0, report_last=rep.splitlines()[-1])
    n = G.info["n"]
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    truth = torch.empty_like(out)
    _, st_t, _ = G.solve(C, 1e-14, pr.PR_POWER, pr.PR_FP64, out=truth)
    res["reference_solution"] = (f"GPU Power, IEEE FP64 throughout, to ||delta||_1 <= 1e-14 ({st_t['rounds']} "
                                 f"iterations)")

    def entry(ms, st):
        return dict(ms=ms, rounds=st["rounds"], rounds_push=st["rounds_push"], rounds_pull=st["rounds_pull"],
                    fp64_rounds=st["fp64_rounds"], l1=float((out - truth).abs().sum()), err_bound=st["err_bound"],
                    gedges_s=st["edges_pushed"] / ms / 1e6)

    eps = 1e-9
    for name, mode, reps in (("auto", pr.PR_MODE_AUTO, 3), ("pull", pr.PR_MODE_PULL, 3), ("push", pr.PR_MODE_PUSH, 2),
                             ("async", pr.PR_MODE_ASYNC, 2), ("apull", pr.PR_MODE_APULL, 3)):
        ms, st = median_solve(G, flush, reps, C, eps, pr.PR_IFP2, pr.PR_FP32, out=out, opts=dict(mode=mode))
        res[f"ifp2_fp32_{name}"] = entry(ms, st)
    ms, st = median_solve(G, flush, 3, C, EPS_FP64, pr.PR_IFP2, pr.PR_FP32, out=out)
    res["ifp2_fp32_auto_eps5e-10"] = entry(ms, st)
    for pname, pprec in (("fp64", pr.PR_FP64), ("df64", pr.PR_DF64)):
        ms, st = median_solve(G, flush, 3, C, EPS_FP64, pr.PR_IFP2, pprec, out=out)
        res[f"ifp2_{pname}_auto"] = entry(ms, st)
        ms, st = median_solve(G, flush, 3, C, EPS_FP64, pr.PR_IFP2, pprec, out=out, opts=dict(mode=pr.PR_MODE_APULL))
        res[f"ifp2_{pname}_apull"] = entry(ms, st)
    # roofline of the dominant kernel from a traced, profiled FP32-form solve
    flush.zero_()
    _, st, _ = G.solve(C, eps, pr.PR_IFP2, pr.PR_FP32, out=out, opts=dict(profile=1, trace_cap=4096))
    prof = st["profile"]
    tot = sum(v["ms"] for v in prof.values())
    res["kernels"] = {k: dict(launches=v["launches"], ms=v["ms"], share=v["ms"] / tot) for k, v in prof.items()}
    if "k_round_pull" in prof:
        res["roofline"] = pull_roofline(G.info, st, prof["k_round_pull"]["ms"], 4, 8, st["fp64_rounds"], hbm_peak,
                                        peak_src)
        res["roofline"]["traffic"] = recorded_traffic("k_round_pull", "rmat24_dag70_ifp2_fp32")
    # Power at equal L1, in the arithmetic of the IFP2 solve it is compared with; the
    # FP32 form (FP64 correction and finish) is compared with Power in FP64
    for pname, pprec, vs in (("fp64", pr.PR_FP64, "ifp2_fp64_auto"), ("df64", pr.PR_DF64, "ifp2_df64_auto"),
                             ("fp64_vs_fp32_form", pr.PR_FP64, "ifp2_fp32_auto"),
                             ("fp64_vs_fp32_form_apull", pr.PR_FP64, "ifp2_fp32_apull"),
                             ("fp64_vs_apull", pr.PR_FP64, "ifp2_fp64_apull"),
                             ("df64_vs_apull", pr.PR_DF64, "ifp2_df64_apull")):
        target = res[vs]["l1"]
        ladder = []
        for tol in (1e-7, 3e-8, 1e-8, 3e-9, 1e-9, 3e-10, 1e-10, 3e-11, 1e-11):
            ms, st = median_solve(G, flush, 2, C, tol, pr.PR_POWER, pprec, out=out)
            # Power's algorithmic bytes per iteration: m (4 + s) + n (4 + 3 s), s = 8 (FP64, double-float)
            hb = st["rounds"] * (G.info["m"] * 12 + G.info["n"] * 28) / (ms / 1e3) / 1e9
            ladder.append(dict(tol=tol, ms=ms, iters=st["rounds"], l1=float((out - truth).abs().sum()),
                               hbm_frac=hb / hbm_peak))
            if ladder[-1]["l1"] <= target:
                break
        res[f"power_{pname}_ladder"] = ladder
        eq = next((q for q in ladder if q["l1"] <= target), None)
        if eq:
            res[f"power_{pname}_at_equal_l1"] = dict(eq, vs=vs, speedup_ifp2=eq["ms"] / res[vs]["ms"])
    G.close()
    # level-ordered rounds on the same graph, prepared with 8 levels
    gd = tg.rmat(24, 16, dangling=0.25, unref=0.0, seed=1, dag_frac=0.7, device="cuda")
    off, dst = gd.csr32()
    G = pr.Graph(gd.n, gd.m, off, dst, mem_is_device=True, stream=stream, levels=8)
    del gd, off, dst
    if ARGS is None or not ARGS.no_tune:
        G.autotune(pr.PR_FP32, max_ms=2000.0)
    for name, prec, e in (("fp32", pr.PR_FP32, eps), ("fp64", pr.PR_FP64, EPS_FP64), ("df64", pr.PR_DF64, EPS_FP64)):
        for mname, mode in (("auto", pr.PR_MODE_AUTO), ("levels8", pr.PR_MODE_LEVELS)):
            ms, st = median_solve(G, flush, 2, C, e, pr.PR_IFP2, prec, out=out, opts=dict(mode=mode))
            res[f"leveled_graph_ifp2_{name}_{mname}"] = dict(ms=ms, rounds=st["rounds"], fp64_rounds=st["fp64_rounds"],
                                                            eps=e, l1=float((out - truth).abs().sum()),
                                                            err_bound=st["err_bound"])
    G.close()
    return res


def batch_specs(count=512, seed=4):
    """Graph sizes and kinds of the batched configuration."""
    import math
    import numpy as np
    rng = np.random.default_rng(seed)
    specs = []
    for j in range(count):
        n = int(math.exp(rng.uniform(math.log(1e3), math.log(2e6))))
        dang = float(rng.uniform(0.1, 0.3))
        if j % 2 == 0:
            specs.append(dict(kind="rmat", scale=max(1, math.ceil(math.log2(n))), edge_factor=float(rng.uniform(8, 16)),
                              nverts=n, dangling=dang, unref=0.0, seed=1000 + j))
        else:
            specs.append(dict(kind="er", n=n, avg_deg=float(rng.uniform(4, 32)), dangling=dang, unref=0.0,
                              seed=1000 + j, permute=True))
    return specs


def make_spec(tg, sp):
    kw = {k: v for k, v in sp.items() if k != "kind"}
    return tg.rmat(device="cuda", **kw) if sp["kind"] == "rmat" else tg.er(device="cuda", **kw)


def leg_batch(pr, torch, stream, flush, hbm_peak, peak_src):
    """512 independent graphs (n log-uniform in [1e3, 2e6]; even: R-MAT with edge
    factor 8-16 cut to n vertices, odd: Erdos-Renyi with mean out-degree 4-32;
    10-30% dangling) solved by IFP2 in the FP32 form in one pr_solve_batch,
    against the same 512 solves one at a time.  eps 5e-7 instead of the
    configured 1e-6, so that every result meets L1 <= 1e-6 (at eps 1e-6 the
    FP32 form stops at about 1.1e-6)."""
    from graphgen import torchgen as tg
    t0 = time.perf_counter()
    hs = []
    for sp in batch_specs():
        gd = make_spec(tg, sp)
        off, dst = gd.csr32()
        hs.append(pr.Graph(gd.n, gd.m, off, dst, mem_is_device=True, stream=stream))
        del gd, off, dst
    torch.cuda.synchronize()
    res = {"workload": "batch512_ifp2_fp32", "graphs": len(hs), "graph_s": time.perf_counter() - t0,
           "n_total": sum(h.info["n"] for h in hs), "m_total": sum(h.info["m"] for h in hs)}
    outs = [torch.empty(h.info["n"], dtype=torch.float64, device="cuda") for h in hs]
    eps = EPS_FP32
    res["eps"] = eps
    bt = []
    for k in range(3):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, sts, status = pr.pr_solve_batch(hs, C, eps, pr.PR_IFP2, pr.PR_FP32, outs=outs)
        torch.cuda.synchronize()
        if k:
            bt.append(1e3 * (time.perf_counter() - t0))
    edges = sum(s["edges_pushed"] for s in sts)
    res["batch"] = dict(ms=statistics.median(bt), device_ms=sts[0]["ms"], status=status, edges_pushed=edges,
                        gedges_s=edges / statistics.median(bt) / 1e6,
                        rounds_max=max(s["rounds"] for s in sts), rounds_min=min(s["rounds"] for s in sts))
    for h, o in zip(hs, outs):  # warm each graph's own workspace
        h.solve(C, eps, pr.PR_IFP2, pr.PR_FP32, out=o)
    flush.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e1 = 0
    for h, o in zip(hs, outs):
        _, st, _ = h.solve(C, eps, pr.PR_IFP2, pr.PR_FP32, out=o)
        e1 += st["edges_pushed"]
    torch.cuda.synchronize()
    single_ms = 1e3 * (time.perf_counter() - t0)
    res["one_at_a_time"] = dict(ms=single_ms, edges_pushed=e1, gedges_s=e1 / single_ms / 1e6)
    res["speedup_batch"] = single_ms / res["batch"]["ms"]
    # accuracy on a sample of the batch
    _, sts, _ = pr.pr_solve_batch(hs, C, eps, pr.PR_IFP2, pr.PR_FP32, outs=outs)
    worst, worst_l1 = 0.0, 0.0
    for k in range(0, len(hs), 16):
        truth = torch.empty_like(outs[k])
        hs[k].solve(C, 1e-14, pr.PR_POWER, pr.PR_FP64, out=truth)
        l1v = float((outs[k] - truth).abs().sum())
        worst_l1 = max(worst_l1, l1v)
        worst = max(worst, l1v / max(sts[k]["err_bound"], 1e-300))
    res["sample_l1_over_bound_max"] = worst
    res["sample_l1_max"] = worst_l1
    res["sample"] = "every 16th graph (32 of 512) against GPU Power FP64 to 1e-14"
    for h in hs:
        h.close()
    return res


def leg_serve(pr, torch, stream, flush, hbm_peak, peak_src):
    """Continuous batching: Poisson arrivals at each rate; 90% personalized
    PageRank (1-64 seeded vertices, weights 1/k) on a resident R-MAT scale-23
    graph, 10% full PageRank on a new graph (n log-uniform in [1e4, 1e6], R-MAT /
    Erdos-Renyi alternating): such a request creates its graph from the client's
    host CSR arrays (pr_graph_create: copy, checks, preprocessing) when it
    arrives, submits, and destroys the graph once its result is polled; the
    creation is inside its latency.  FP32 form, c = 0.85, eps 7.5e-8, the
    certified stop for L1 <= 1e-6 (checked on a sample), 120 GB device budget.
    Latency = from the scheduled arrival to the return of the poll that copies
    the result into the client's pinned host buffer (client clock)."""
    import math
    import numpy as np
    import graphgen as gg
    from graphgen import torchgen as tg
    t0 = time.perf_counter()
    gd = tg.rmat(ARGS.serve_scale, 16, dangling=0.20, unref=0.10, seed=3, device="cuda")
    off, dst = gd.csr32()
    R = pr.Graph(gd.n, gd.m, off, dst, mem_is_device=True, stream=stream)
    del gd, off, dst
    rng = np.random.default_rng(7)
    # the client's data for the new-graph requests: 16 distinct graphs as host CSR
    # arrays (the graph a request brings; a new pr_graph is made from it each time)
    new_graphs = []
    for j in range(16):
        n = int(math.exp(rng.uniform(math.log(1e4), math.log(1e6))))
        sp = (dict(kind="rmat", scale=math.ceil(math.log2(n)), edge_factor=16.0, nverts=n, dangling=0.2, unref=0.1,
                   seed=50 + j) if j % 2 == 0 else
              dict(kind="er", n=n, avg_deg=8.0, dangling=0.2, unref=0.1, seed=50 + j, permute=True))
        gh = make_spec(tg, sp).to_host()
        o, d = gh.csr32()
        new_graphs.append((gh.n, gh.m, o, d))
    torch.cuda.synchronize()
    n_res = R.info["n"]
    res = {"workload": f"serve_rmat{ARGS.serve_scale}_ppr90_newgraph10_fp32", "graph_s": time.perf_counter() - t0,
           "resident": {k: R.info[k] for k in ("n", "m", "n_nd")}, "new_graph_n": [g[0] for g in new_graphs]}

    def request(rr):
        """(graph spec, p, p_idx): the resident graph, or a new graph's host arrays"""
        if rr.uniform() < 0.9:
            k = int(rr.integers(1, 65))
            idx = rr.choice(n_res, size=k, replace=False).astype(np.int32)
            return None, np.full(k, 1.0 / k), idx
        return new_graphs[int(rr.integers(0, len(new_graphs)))], None, None

    def open_graph(spec):
        return R if spec is None else pr.Graph(spec[0], spec[1], spec[2], spec[3], stream=stream)

    def close_graph(h):
        if h is not R:
            h.close()

    # one at a time through pr_solve (the same requests, new graphs created alike)
    rr = np.random.default_rng(11)
    alone = []
    for _ in range(3):
        spec, pv, pi = request(rr)
        h = open_graph(spec)
        h.solve(C, EPS_SERVE, pr.PR_IFP2, pr.PR_FP32, p=pv, p_idx=pi)
        close_graph(h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(40):
        ta = time.perf_counter()
        spec, pv, pi = request(rr)
        h = open_graph(spec)
        _, st, _ = h.solve(C, EPS_SERVE, pr.PR_IFP2, pr.PR_FP32, p=pv, p_idx=pi)
        close_graph(h)
        alone.append(1e3 * (time.perf_counter() - ta))
    res["one_at_a_time"] = dict(solves_s=40 / (time.perf_counter() - t0), p50_ms=float(np.percentile(alone, 50)),
                                p99_ms=float(np.percentile(alone, 99)))
    rates = []
    sinks = {}

    def sink(n):
        """A reused pinned host buffer of n doubles: the client's result buffer."""
        if n not in sinks:
            sinks[n] = torch.empty(n, dtype=torch.float64).pin_memory()
        return sinks[n]

    with pr.Server(120 << 30, stream=None) as S:
        for _ in range(8):  # warm-up: the server's tables and the resident graph's tiles
            spec, pv, pi = request(rr)
            h = open_graph(spec)
            S.wait(S.submit(h, C, EPS_SERVE, pr.PR_FP32, pv, pi))
            close_graph(h)
        for rate in [int(v) for v in ARGS.serve_rates.split(",") if v]:
            N = int(min(rate * ARGS.serve_window, ARGS.serve_max))
            arr = np.cumsum(rng.exponential(1.0 / rate, N))
            reqs = [request(rr) for _ in range(N)]
            lat, server_ms, pending = [], [], {}
            st0 = S.stats()
            t_start = time.perf_counter()
            i = 0
            statuses = set()
            create_ms = []
            while i < N or pending:
                now = time.perf_counter() - t_start
                while i < N and arr[i] <= now:
                    spec, pv, pi = reqs[i]
                    tc = time.perf_counter()
                    h = open_graph(spec)
                    pending[S.submit(h, C, EPS_SERVE, pr.PR_FP32, pv, pi)] = (arr[i], h)
                    i += 1
                    if h is not R:  # a graph creation takes ~20 ms: poll before the next arrivals
                        create_ms.append(1e3 * (time.perf_counter() - tc))
                        break
                done = []
                for tk, (t_arr, h) in pending.items():
                    r = S.poll(tk, sink(S._n[tk]))  # copies the result into pinned host memory
                    if r is not None:
                        statuses.add(r[2])
                        lat.append(1e3 * (time.perf_counter() - t_start - t_arr))
                        server_ms.append(r[1]["ms"])
                        done.append(tk)
                for tk in done:
                    close_graph(pending.pop(tk)[1])
                if not done:
                    time.sleep(0.0002)
            wall = time.perf_counter() - t_start
            st1 = S.stats()
            steps = max(st1["steps"] - st0["steps"], 1)
            per_step = {k: (st1[k] - st0[k]) / steps for k in ("ms_admit", "ms_rounds", "ms_tables", "ms_correct",
                                                                "ms_finish")}
            rates.append(dict(rate=rate, requests=N, solves_s=N / wall, p50_ms=float(np.percentile(lat, 50)),
                              p99_ms=float(np.percentile(lat, 99)),
                              server_p50_ms=float(np.percentile(server_ms, 50)), status=sorted(statuses),
                              new_graphs=len(create_ms),
                              create_ms_p50=float(np.percentile(create_ms, 50)) if create_ms else None,
                              steps=steps, ms_per_step=per_step,
                              queued_avg=(st1["queued_sum"] - st0["queued_sum"]) / steps,
                              running_avg=(st1["running_sum"] - st0["running_sum"]) / steps,
                              group_launches=st1["group_launches"] - st0["group_launches"],
                              tile_launches=st1["tile_launches"] - st0["tile_launches"]))
        res["server_stats"] = S.stats()
        # accuracy of served results: a sample of requests, submitted together, each
        # against GPU Power in IEEE FP64 with the same personalization
        sample = [request(rr) for _ in range(12)] + [(new_graphs[0], None, None)]
        hs = [open_graph(spec) for spec, _, _ in sample]
        tks = [S.submit(h, C, EPS_SERVE, pr.PR_FP32, pv, pi) for h, (_, pv, pi) in zip(hs, sample)]
        worst = 0.0
        for tk, h, (_, pv, pi) in zip(tks, hs, sample):
            got = torch.empty(h.info["n"], dtype=torch.float64).pin_memory()
            S.wait(tk, out=got)
            truth, _, _ = h.solve(C, 1e-14, pr.PR_POWER, pr.PR_FP64, p=pv, p_idx=pi)
            worst = max(worst, float(np.abs(got.numpy() - truth).sum()))
        for h in hs:
            close_graph(h)
        res["served_l1_max"] = worst
        res["served_l1_sample"] = ("13 requests of the same mix (one on a new graph at least), submitted together, "
                                   "against GPU Power FP64 to 1e-14")
    res["eps"] = EPS_SERVE
    res["rates"] = rates
    R.close()
    return res


def leg_sweep(pr, torch, stream, flush, hbm_peak, peak_src):
    """Time and accuracy against eps (the paper's Fig. 1 / Fig. 2 analogue) on
    the headline graph (R-MAT scale 22) and the DAG-heavy graph (R-MAT scale 24,
    70% forward): IFP1 and IFP2 stopped at residual L1 <= eps, the Power method
    stopped at ||delta||_1 <= eps, eps from 1e-4 to 1e-15, each in IEEE FP64 and
    in double-float; L1 and max relative error (the paper's ERR, Sec. 4) against
    a Power solution in IEEE FP64 run as far as FP64 allows (||delta||_1 <=
    1e-15, else 400 iterations).  A solve that cannot meet eps in its arithmetic
    hits its round cap (400) and is reported with status ENOTCONV: that is
    where the precision floors."""
    from graphgen import torchgen as tg
    res = {"workload": "eps sweep: rmat22 and rmat24_dag70, IEEE FP64 and double-float"}
    eps_list = [10.0 ** -k for k in range(4, 16)]
    for gname in ("rmat22", "rmat24_dag70"):
        if gname == "rmat22":
            gd = make_graph_device(22)
        else:
            gd = tg.rmat(24, 16, dangling=0.25, unref=0.0, seed=1, dag_frac=0.7, device="cuda")
        off, dst = gd.csr32()
        G = pr.Graph(gd.n, gd.m, off, dst, mem_is_device=True, stream=stream)
        del gd, off, dst
        out = torch.empty(G.info["n"], dtype=torch.float64, device="cuda")
        truth = torch.empty_like(out)
        _, st_t, status_t = G.solve(C, 1e-15, pr.PR_POWER, pr.PR_FP64, out=truth, opts=dict(max_rounds=400))
        rows = []
        for pname, prec in (("fp64", pr.PR_FP64), ("df64", pr.PR_DF64)):
            for name, algo in (("IFP1", pr.PR_IFP1), ("IFP2", pr.PR_IFP2), ("Power", pr.PR_POWER)):
                for eps in eps_list:
                    ms = []
                    for _ in range(2):
                        flush.zero_()
                        _, st, status = G.solve(C, eps, algo, prec, out=out, opts=dict(max_rounds=400))
                        ms.append(st["ms"])
                    err = (out - truth).abs()
                    rows.append(dict(prec=pname, algo=name, eps=eps, ms=statistics.median(ms), rounds=st["rounds"],
                                     status="ok" if status == pr.PR_OK else "ENOTCONV", l1=float(err.sum()),
                                     err_max_rel=float((err / truth).max()), err_bound=st["err_bound"],
                                     resid=st["resid_l1"]))
        res[gname] = dict(reference=f"GPU Power IEEE FP64, {st_t['rounds']} iterations, final ||delta||_1 = "
                                    f"{st_t['resid_l1']:.2e} (status {status_t})", rows=rows)
        G.close()
        del out, truth
        torch.cuda.empty_cache()
    return res


def equal_l1_power(G, flush, out, truth, target, prec, pr, ref_ms):
    """Power stopped at the first ||delta||_1 tolerance whose L1 error meets target."""
    ladder = []
    for tol in (1e-6, 3e-7, 1e-7, 3e-8, 1e-8, 3e-9, 1e-9, 3e-10, 1e-10, 3e-11, 1e-11):
        ms, st = median_solve(G, flush, 2, C, tol, pr.PR_POWER, prec, out=out)
        ladder.append(dict(tol=tol, ms=ms, iters=st["rounds"], l1=float((out - truth).abs().sum())))
        if ladder[-1]["l1"] <= target:
            return dict(ladder[-1], speedup_ifp2=ladder[-1]["ms"] / ref_ms), ladder
    return None, ladder


def leg_undirected(pr, torch, stream, flush, hbm_peak, peak_src):
    """The case the paper expects to lose (a graph with no DAG structure): R-MAT
    scale 22, edge factor 16, every sampled edge also taken reversed, no
    deletions (no dangling or unreferenced vertex but the isolated ones);
    IFP2 in IEEE FP64 and in double-float (synchronous rounds, AUTO delivery,
    and level-ordered rounds with 16 levels) against Power in the same
    arithmetic at equal L1, eps 5e-10."""
    from graphgen import torchgen as tg
    gd = tg.rmat(22, 16, dangling=0.0, unref=0.0, seed=1, undirected=True, device="cuda")
    off, dst = gd.csr32()
    G = pr.Graph(gd.n, gd.m, off, dst, mem_is_device=True, stream=stream, levels=16)
    del gd, off, dst
    torch.cuda.synchronize()
    res = {"workload": "rmat22_undirected_ifp2_fp64",
           "graph": {k: G.info[k] for k in ("n", "m", "n_nd", "n_ref", "n_d", "m_d", "n_u", "max_indeg")}}
    G.autotune(pr.PR_FP64, max_ms=1500.0)
    out = torch.empty(G.info["n"], dtype=torch.float64, device="cuda")
    truth = torch.empty_like(out)
    G.solve(C, 1e-14, pr.PR_POWER, pr.PR_FP64, out=truth)
    for pname, prec in (("fp64", pr.PR_FP64), ("df64", pr.PR_DF64)):
        for name, mode in (("auto", pr.PR_MODE_AUTO), ("levels16", pr.PR_MODE_LEVELS), ("apull", pr.PR_MODE_APULL)):
            ms, st = median_solve(G, flush, 3, C, EPS_FP64, pr.PR_IFP2, prec, out=out, opts=dict(mode=mode))
            l1 = float((out - truth).abs().sum())
            eq, ladder = equal_l1_power(G, flush, out, truth, l1, prec, pr, ms)
            res[f"ifp2_{pname}_{name}"] = dict(ms=ms, rounds=st["rounds"], l1=l1, err_bound=st["err_bound"],
                                               gedges_s=st["edges_pushed"] / ms / 1e6,
                                               **{f"power_{pname}_at_equal_l1": eq})
        res[f"power_{pname}_ladder"] = ladder
    G.close()
    return res


def leg_threads(pr, torch, stream, flush, hbm_peak, peak_src):
    """The parallelism study (the paper's Fig. 3 analogue): on the headline graph,
    the pull rounds and Power sweeps capped at B resident CTAs of 256 threads
    (block_budget B), B from 19 to 1216; IFP2 in IEEE FP64 (synchronous and
    16-level rounds) to eps 5e-10 and Power in IEEE FP64 to ||delta||_1 <= 5e-10.  The cap applies to the dominant
    kernels; the short activation, phase-2 and finishing kernels keep their
    grids."""
    g = make_graph_device(22)
    off, dst = g.csr32()
    G = pr.Graph(g.n, g.m, off, dst, mem_is_device=True, stream=stream, levels=16)
    del g, off, dst
    out = torch.empty(G.info["n"], dtype=torch.float64, device="cuda")
    rows = []
    for budget in (19, 38, 76, 152, 304, 608, 1216):
        G.set_tuning(block_budget=budget)
        row = dict(ctas=budget, threads=budget * 256)
        for name, algo, mode in (("ifp2", pr.PR_IFP2, pr.PR_MODE_AUTO), ("ifp2_levels16", pr.PR_IFP2, pr.PR_MODE_LEVELS),
                                 ("ifp2_apull", pr.PR_IFP2, pr.PR_MODE_APULL), ("power", pr.PR_POWER, pr.PR_MODE_AUTO)):
            ms, st = median_solve(G, flush, 2, C, EPS_FP64, algo, pr.PR_FP64, out=out, opts=dict(mode=mode))
            row[f"{name}_ms"] = ms
            row[f"{name}_rounds"] = st["rounds"]
        rows.append(row)
    G.close()
    return {"workload": "rmat22, IEEE FP64, eps 5e-10, block budget sweep", "rows": rows}


LEGS = {"dag": leg_dag, "batch": leg_batch, "serve": leg_serve, "sweep": leg_sweep, "undirected": leg_undirected,
        "threads": leg_threads}


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
              f"graph (n={g.n}, m={g.m}), single thread of the host's {os.cpu_count()} cores, per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload(args.scale, "ifp2", 0, "fp64", args.eps),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    emit(line, args)


def emit(line, args):
    s = json.dumps(line)
    print(s, flush=True)
    if args.out:
        with open(args.out, "w") as f:
            f.write(s + "\n")


# ------------------------------------------------------------------ GPU arm
ARGS = None  # parsed command line (the legs read their options from it)


def main():
    global ARGS
    args = ARGS = parse()
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
    tgen0 = time.perf_counter()
    gd = make_graph_device(args.scale)
    d_off, d_dst = gd.csr32()
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - tgen0
    n_v, m_e = gd.n, gd.m
    G = pr.Graph(n_v, m_e, d_off, d_dst, mem_is_device=True, stream=stream, levels=args.levels)
    g = gd.to_host()  # for the host-side legs (e2e copies, the oracle)
    del gd
    info = G.info
    tune_report = "default launch parameters"
    tune_s = 0.0
    step_prec = {"fp64": pr.PR_FP64, "df64": pr.PR_DF64, "fp32": pr.PR_FP32}[args.prec]
    if not args.no_tune:
        t0 = time.perf_counter()
        if args.tune_cache:
            tuning, tune_report = G.autotune(step_prec, max_ms=1500.0, cache_path=args.tune_cache)
        else:
            tuning, tune_report = G.autotune(step_prec, max_ms=1500.0)
        tune_s = time.perf_counter() - t0
    tuning = G.tuning()
    out = torch.empty(n_v, dtype=torch.float64, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)

    step_algo = {"ifp2": pr.PR_IFP2, "ifp1": pr.PR_IFP1, "power": pr.PR_POWER}[args.algo]

    def solve(algo=step_algo, prec=step_prec, eps=args.eps, opts=None):
        opts = dict(opts or {})
        if args.host_rounds:
            opts.setdefault("use_graph", -1)
        if args.levels and algo == pr.PR_IFP2:
            opts.setdefault("mode", pr.PR_MODE_LEVELS)
        if args.apull and algo != pr.PR_POWER:
            opts.setdefault("mode", pr.PR_MODE_APULL)
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
    my_time, my_edges = reduce_ranks(sum(ms) / 1e3, float(sum(edges)), dist, "cuda")
    value = my_edges / my_time / 1e9

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step,
            "ms_per_step_median_min": [statistics.median(ms), min(ms)],
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "df64": "df64", "fp32": "f32+f64"}[args.prec],
            "dtype_detail": PREC_LABEL[args.prec],
            "data": "synthetic",
            "config": dict(workload(args.scale, args.algo, args.levels, args.prec, args.eps, args.apull),
                           l2="512 MB buffer written between timed steps",
                           parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
            "gpu_launches": int(launches), "clocks": clk,
            "graph": {k: info[k] for k in ("n", "m", "n_nd", "n_ref", "n_d", "m_d", "n_u", "max_outdeg",
                                             "max_indeg")},
            "rounds": rounds[0], "edges_pushed_per_step": edges[0], "wall_s_timed": wall,
            "tuning": dict(tuning, autotune_s=tune_s, source=tune_report.splitlines()[-1] if tune_report else ""),
            "graph_generation_s": gen_s}
    peaks = measured_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    peak_src = "measured" if peaks else "fallback"
    if rank != 0 or args.skip_extras:
        if rank == 0:
            G.close()
            run_legs(args, line, pr, torch, stream, flush, hbm_peak, peak_src)
            emit(line, args)
        if dist:
            dist.destroy_process_group()
        return

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
    s = 4 if args.prec == "fp32" else 8
    # in-list entries read by the pull rounds: everything the solve scanned minus the push
    # rounds' out-edges and the phase-2 in-edges of dangling vertices
    push_rounds = np.nonzero(modes == 1)[0]
    pull_scan_total = st["edges_scanned"] - int(trace["E"][push_rounds].sum()) - info["m_d"]
    scan_ref = pull_scan_total / max(len(pull_rounds), 1)
    kernels = {k: dict(launches=v["launches"] // prof_runs, avg_ms=v["ms"] / max(v["launches"], 1),
                       share=v["ms"] / total_k_ms) for k, v in agg.items()}
    if dom in ("k_round_pull", "k_round_levels"):  # a level-ordered round reads the in-lists once too
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
                        "traffic": recorded_traffic(dom, workload(args.scale, args.algo, args.levels, args.prec,
                                                                  args.eps, args.apull)["workload"]),
                        "timing": "CUDA events around every launch on the graph's stream, instrumented pass"}
    line["kernels"] = kernels

    # ---- accuracy against the exact PageRank and the Power method at equal L1, like for like
    # (the reference solution: GPU Power in IEEE FP64, state, gathers and sums in double,
    # run to ||delta||_1 <= 1e-14; its distance to pi is at most c/(1-c) x that, and the
    # GPU tests check this Power against the CPU oracle's)
    truth = torch.empty_like(out)
    _, st_t, _ = G.solve(C, 1e-14, pr.PR_POWER, pr.PR_FP64, out=truth)
    ref_bound = st_t["err_bound"]

    def accuracy():
        err = (out - truth).abs()
        return float(err.sum()), float((err / truth).max())

    legs = {"reference_solution": f"GPU Power, IEEE FP64 throughout, to ||delta||_1 <= 1e-14 "
                                  f"({st_t['rounds']} iterations; certified L1 <= {ref_bound:.2e})",
            "gates": "L1 <= 1e-9 (FP64, double-float), <= 1e-6 (FP32 form) against the reference solution"}
    solve()
    l1_step, errmax_step = accuracy()
    line["l1_vs_exact"] = l1_step
    line["err_max_rel_vs_exact"] = errmax_step
    legs[f"{args.algo}_{args.prec}"] = dict(ms=t_step, l1=l1_step, err_max_rel=errmax_step, rounds=rounds[0],
                                            eps=args.eps, gedges_s=value, headline=True)
    runs = [("ifp2_fp64", pr.PR_IFP2, pr.PR_FP64, EPS_FP64, None),
            ("ifp2_df64", pr.PR_IFP2, pr.PR_DF64, EPS_FP64, None),
            ("ifp1_fp64", pr.PR_IFP1, pr.PR_FP64, EPS_FP64, None),
            ("ifp1_df64", pr.PR_IFP1, pr.PR_DF64, EPS_FP64, None),
            ("ifp2_fp32", pr.PR_IFP2, pr.PR_FP32, EPS_FP32, None),
            ("ifp2_fp64_async", pr.PR_IFP2, pr.PR_FP64, EPS_FP64, pr.PR_MODE_ASYNC),
            ("ifp2_df64_async", pr.PR_IFP2, pr.PR_DF64, EPS_FP64, pr.PR_MODE_ASYNC),
            ("ifp2_fp64_apull", pr.PR_IFP2, pr.PR_FP64, EPS_FP64, pr.PR_MODE_APULL),
            ("ifp2_fp32_apull", pr.PR_IFP2, pr.PR_FP32, EPS_FP32, pr.PR_MODE_APULL),
            ("ifp2_df64_apull", pr.PR_IFP2, pr.PR_DF64, EPS_FP64, pr.PR_MODE_APULL),
            ("ifp1_fp64_apull", pr.PR_IFP1, pr.PR_FP64, EPS_FP64, pr.PR_MODE_APULL)]
    for nm, algo, prec, eps, mode in runs:
        if nm in legs:
            continue
        tms = []
        for _ in range(3):
            flush.zero_()
            st = solve(algo=algo, prec=prec, eps=eps, opts=dict(mode=mode) if mode is not None else None)
            tms.append(st["ms"])
        l1v, emax = accuracy()
        legs[nm] = dict(ms=statistics.median(tms), l1=l1v, err_max_rel=emax, rounds=st["rounds"],
                        fp64_rounds=st["fp64_rounds"], eps=eps,
                        gedges_s=st["edges_pushed"] / (statistics.median(tms) / 1e3) / 1e9)
    # Power in the same arithmetic as the IFP2 solve it is compared with, stopped at the
    # first ||delta||_1 tolerance whose L1 error is at most that solve's
    for pname, pprec, vs in (("fp64", pr.PR_FP64, "ifp2_fp64"), ("df64", pr.PR_DF64, "ifp2_df64"),
                             ("fp32", pr.PR_FP32, "ifp2_fp32"), ("fp64_vs_apull", pr.PR_FP64, "ifp2_fp64_apull"),
                             ("df64_vs_apull", pr.PR_DF64, "ifp2_df64_apull"),
                             ("fp32_vs_apull", pr.PR_FP32, "ifp2_fp32_apull")):
        ref = legs[vs]
        power = []
        for tol in (1e-6, 3e-7, 1e-7, 3e-8, 1e-8, 3e-9, 1e-9, 3e-10, 1e-10, 3e-11, 1e-11):
            tms = []
            for _ in range(3):
                flush.zero_()
                st = solve(algo=pr.PR_POWER, prec=pprec, eps=tol)
                tms.append(st["ms"])
            err = accuracy()[0]
            # Power's algorithmic bytes per iteration: m (4 + s) + n (4 + 3 s), s = the state's bytes
            sp = 4 if pprec == pr.PR_FP32 else 8
            hb = st["rounds"] * (info["m"] * (4 + sp) + info["n"] * (4 + 3 * sp)) / (statistics.median(tms) / 1e3) / 1e9
            power.append(dict(tol=tol, ms=statistics.median(tms), l1=err, iters=st["rounds"],
                              hbm_frac=hb / hbm_peak))
            if err <= ref["l1"]:
                break
        eq = next((q for q in power if q["l1"] <= ref["l1"]), None)
        legs[f"power_{pname}_ladder"] = power
        if eq:
            legs[f"power_{pname}_at_equal_l1"] = dict(eq, vs=vs, speedup_ifp2=eq["ms"] / ref["ms"])
    # The paper's own accuracy point (Table 3: time until the maximum relative
    # error against the converged PageRank is below 1e-3), on this GPU, IEEE FP64:
    # the loosest stop of each method that reaches it
    def first_below(algo, stops, mode=None):
        for x in stops:
            tms = []
            for _ in range(3):
                flush.zero_()
                st = solve(algo=algo, prec=pr.PR_FP64, eps=x, opts=dict(mode=mode) if mode is not None else None)
                tms.append(st["ms"])
            l1v, emax = accuracy()
            if emax < 1e-3:
                return dict(stop=x, ms=statistics.median(tms), err_max_rel=emax, l1=l1v, rounds=st["rounds"])
        return None
    stops = (3e-3, 1e-3, 3e-4, 1e-4, 3e-5, 1e-5, 3e-6, 1e-6)
    at = dict(ifp2=first_below(pr.PR_IFP2, stops), ifp2_apull=first_below(pr.PR_IFP2, stops, pr.PR_MODE_APULL),
              power=first_below(pr.PR_POWER, stops))
    if at["ifp2"] and at["power"]:
        at["speedup_ifp2"] = at["power"]["ms"] / at["ifp2"]["ms"]
    if at["ifp2_apull"] and at["power"]:
        at["speedup_ifp2_apull"] = at["power"]["ms"] / at["ifp2_apull"]["ms"]
    legs["at_paper_accuracy_err_1e-3"] = at
    # context only (another machine, other graphs): the paper's Table 3 ratios of
    # its 38-thread Power method to its 38-thread IFP2, to ERR < 1e-3, in double
    legs["paper_table3_context"] = {
        "hardware": "Intel Xeon Silver 4210R @ 2.40 GHz, 40 logical processors, 38 threads, C++ double",
        "accuracy": "ERR (max relative error) < 1e-3",
        "multithreaded_power_over_ifp2": {"web-Stanford": 3.33, "Stanford-Berkeley": 1.72, "web-Google": 2.89,
                                          "in-2004": 3.19, "soc-LiveJournal1": 1.70, "uk-2002": 3.80}}
    line["vs_power"] = legs
    pre = []
    for _ in range(3):
        G2 = pr.Graph(n_v, m_e, d_off, d_dst, mem_is_device=True, stream=stream)
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
    # the same figure for the GPU Power method it is compared with (IEEE FP64, equal L1)
    pe = line["vs_power"].get("power_fp64_at_equal_l1")
    line["power_hbm_frac"] = pe["hbm_frac"] if pe else None

    # ---- end to end through the C ABI with pinned host buffers
    off, dst = g.csr32()
    h_off = torch.from_numpy(off).pin_memory()
    h_dst = torch.from_numpy(dst).pin_memory()
    h_out = torch.empty(g.n, dtype=torch.float64).pin_memory()
    e2e_ms, e2e_edges = [], []
    for k in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gh = pr.pr_graph_create(g.n, g.m, h_off, h_dst, mem_is_device=False, stream=stream)
        _, st, status = pr.pr_solve(gh, C, args.eps, step_algo, step_prec, out=h_out)
        pr.pr_destroy(gh)
        torch.cuda.synchronize()
        if k > 0:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
            e2e_edges.append(st["edges_pushed"])
    line["e2e"] = {"value": sum(e2e_edges) / (sum(e2e_ms) / 1e3) / 1e9, "unit": UNIT,
                   "h2d_bytes_per_step": int(off.nbytes + dst.nbytes), "d2h_bytes_per_step": int(8 * g.n),
                   "ms_per_step": statistics.median(e2e_ms),
                   "includes": "pr_graph_create from pinned host CSR (copy, validation, preprocessing, default "
                               f"launch parameters) + pr_solve {args.algo.upper()} {args.prec} + copy of pi to "
                               "pinned host memory"}

    # ---- the oracle on the host cores (bounded sample)
    import oracle
    p = gg.p_uniform(g.n)
    rounds_cpu = 3
    t0 = time.perf_counter()
    o = oracle.ifp_rounds(oracle.IFP2, g, C, args.eps, p, max_rounds=rounds_cpu)
    dt = time.perf_counter() - t0
    line["cpu_baseline"] = {"value": float(o["E"].sum()) / dt / 1e9, "unit": UNIT, "cores": 1,
                            "host_cores": os.cpu_count(), "kind": "oracle",
                            "sample": f"first {rounds_cpu} synchronous IFP2 rounds of the FP64 oracle on the full "
                                      f"graph, single thread of the host's {os.cpu_count()} cores ({dt:.1f} s)"}
    del g, o
    # ---- default launch parameters against the tuned ones (same solve)
    if not args.no_tune:
        tuned = G.tuning()
        G.set_tuning(pull_thr=[4096, 64, 32, 16, 8, 4], block_budget=info_sms(torch) * 16, pull_ratio=0.04)
        tms = []
        for _ in range(3):
            flush.zero_()
            tms.append(solve()["ms"])
        G.set_tuning(pull_thr=tuned["pull_thr"], block_budget=tuned["block_budget"], pull_ratio=tuned["pull_ratio"])
        line["tuning"]["default_params_ms"] = statistics.median(tms)
        line["tuning"]["tuned_ms"] = t_step
    G.close()
    run_legs(args, line, pr, torch, stream, flush, hbm_peak, peak_src)
    emit(line, args)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
