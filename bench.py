#!/usr/bin/env python
"""Benchmark of the front/fluid coupling hot path on GB300.

One step = the five steps (bin, volume fraction, PPIC curvature, CSF force,
vertex velocities) on each front of the workload, through the C ABI.  The
metric is interfacial cells per second (sum over fronts of the interfacial
cells M, per step, divided by the device time of the step).

Workload (default): the 128^3 precision-study pair of the paper-shaped inputs,
a rough icosphere (s=6, 81,920 triangles, R=0.2, radial noise 1e-3 h) and the
ellipsoid (0.3, 0.2, 0.15) made from the same icosphere; synthetic, seeded.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32c]
  python bench.py --impl reference ...      # the FP64 CPU oracle, same metric

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank runs its own
replica on its own GPU (the path does not shard); value = all cells / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "interfacial cells/s for alpha+kappa (full five-step hot path per step)"
FLOPS_PER_FIT_PAIR = 130.0   # per (cell, fragment-in-support) pair of the volume fit
FLOPS_PER_FIT_SOLVE = 260.0  # per cell: 6x6 LDL^T (144), two triangular solves (72), curvature and normal
FLOPS_PER_CAND = 60.0        # clip: per candidate pair, cell-unit coordinates and the plane stages
FLOPS_PER_KEPT = 150.0       # clip: per kept pair, the fragment moments
FP64_PEAK_TFLOPS = 1.25      # GB300 nominal float64 (profiling recipe table)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # 152 SMs x 128 FMA/clk x 2 flops x 2.07 GHz
HBM_FALLBACK_GBS = 6800.0    # profiling recipe fallback, used only without MEASURED_PEAKS.json


def hbm_peak():
    """Measured STREAM-style copy bandwidth of the GB300s (GB/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return HBM_FALLBACK_GBS, "of fallback (profiling recipe, 6.8 TB/s)"


# Algorithmic work of one launch of each kernel on one front, from the work
# counts of that front (T triangles, V vertices, N grid cells, C candidate
# pairs, P kept pairs, M interfacial cells, fit_pairs, ring cells of the CSF
# step): ("hbm", bytes) or ("fp32" | "fp64", flops).
def kernel_work(name, w, fp32):
    T, V, N, C, P, M = w["T"], w["V"], w["N"], w["C"], w["P"], w["M"]
    R, FP = w["ring"], w["fit_pairs"]
    table = {
        "k_tri_setup": ("hbm", (248 if fp32 else 152) * T + 8 * M,
                        "84 B of indices and coordinates read, box and count (36 B) and the normal (32 B) or the "
                        "FP32 clip's 128 B record written per triangle; the previous cells' index-map entries reset"),
        "k_scan_reduce": ("hbm", 4 * T, "the triangle counts read"),
        "k_scan_expand": ("hbm", 8 * T + 4 * C, "counts read, offsets written, the triangle id of every "
                          "candidate slot written"),
        "k_cnt_reduce": ("hbm", 4 * N, "the per-key pair counts read"),
        "k_cnt_down": ("hbm", 4 * N + 16 * M, "counts read; cell key, offset, index map and counter written "
                       "per interfacial cell"),
        "k_place": ("hbm", 4 * C + 16 * P, "every candidate's key read; per kept pair its rank and its cell's "
                    "offset read, key and slot written"),
        "k_cell_order": ("hbm", 12 * M + (120 if fp32 else 216) * P, "per cell its offsets and counter; per "
                         "pair its slot read and written, its record read and written in cell order, its float "
                         "centroid written"),
        "k_alpha_cells32": ("hbm", 24 * M + 8 * P, "per pair the two record values of the column moment; "
                            "per cell offsets read, L and P written"),
        "k_alpha_cells": ("hbm", 24 * M + 16 * P, "per pair the two record values of the column moment; "
                          "per cell offsets read, L and P written"),
        "k_alpha_fill": ("hbm", 12 * N + 16 * M, "per grid cell the index map read and alpha written; per "
                         "interfacial cell L and P read"),
        "force clear (memset)": ("hbm", 24 * N, "the three force components written in every grid cell"),
        "k_zero_force": ("hbm", 24 * N, "the three force components written in every grid cell of every front"),
        "k_alpha_pack": ("hbm", 8 * N + N // 8 + 20 * M, "alpha read and one bit per cell written; per "
                         "interfacial cell its key and value read and the value written"),
        "k_csf_ring_list": ("hbm", 28 * M + 4 * R, "per interfacial cell its key and six face neighbours' "
                            "index-map entries read; the ring list written"),
        "k_csf_force": ("hbm", 84 * M + 176 * R, "per interfacial cell its key, six alpha values and kappa read "
                        "and the force written; per ring cell 26 index-map entries and six alpha values read and "
                        "the force written"),
        "k_interp": ("hbm", 288 * V, "per vertex its position read, its velocity written and about 30 face "
                     "values gathered"),
        "k_clip32": ("fp32", FLOPS_PER_CAND * C + FLOPS_PER_KEPT * P,
                     f"{FLOPS_PER_CAND:.0f} flops per candidate pair (cell-unit coordinates, plane stages, "
                     f"crossings), {FLOPS_PER_KEPT:.0f} per kept pair (fragment moments)"),
        "k_clip_list": ("fp64", (FLOPS_PER_CAND + FLOPS_PER_KEPT) * w["clip_f64"],
                        f"{FLOPS_PER_CAND + FLOPS_PER_KEPT:.0f} flops per pair the FP32 clip left to the binary64 "
                        "clip (the candidate's plane stages and the fragment moments)"),
        "k_clip": ("fp64", FLOPS_PER_CAND * C + FLOPS_PER_KEPT * P,
                   f"{FLOPS_PER_CAND:.0f} flops per candidate pair, {FLOPS_PER_KEPT:.0f} per kept pair"),
        "k_ppic_acc<float>": ("fp32", FLOPS_PER_FIT_PAIR * FP, f"{FLOPS_PER_FIT_PAIR:.0f} flops per (cell, "
                              "fragment-in-support) pair"),
        "k_ppic_acc<double>": ("fp64", FLOPS_PER_FIT_PAIR * FP, f"{FLOPS_PER_FIT_PAIR:.0f} flops per (cell, "
                               "fragment-in-support) pair"),
        "k_ppic_solve": ("fp64", FLOPS_PER_FIT_SOLVE * M, f"{FLOPS_PER_FIT_SOLVE:.0f} flops per cell"),
    }
    return table.get(name)


def read_traffic(workload):
    """DRAM bytes per launch of each kernel from the committed ncu summary of
    this workload (profiles/dram_traffic_<workload>.md), keyed by kernel name,
    with the source hash the capture was taken on: a kernel whose source file
    changed since then gets null."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"dram_traffic_{workload}.md")
    out = {}
    if not os.path.exists(path):
        return out, None
    for line in open(path):
        c = [x.strip() for x in line.strip().strip("|").split("|")]
        if len(c) < 5 or not c[0].startswith("`"):
            continue
        name, src, sha = c[0].strip("`"), c[1].strip("`"), c[2].strip("`")
        try:
            per_launch = float(c[4].replace(",", ""))
        except ValueError:
            continue
        fp = os.path.join(ROOT, "paper_2505_06932_gb300", "csrc", src)
        ok = os.path.exists(fp) and hashlib.sha256(open(fp, "rb").read()).hexdigest()[:12] == sha
        out[name] = per_launch if ok else None
    return out, os.path.relpath(path, ROOT)


def roofline_list(trace, works, fp32, workload_tag):
    """Per-kernel roofline entries from a trace of eager steps: the kernel's
    algorithmic work per launch (mean over the fronts) divided by its mean
    CUDA-event duration, against its bound's peak."""
    hbm, hbm_src = hbm_peak()
    traffic, tsrc = read_traffic(workload_tag)
    items = [(k, v) for k, v in trace.items() if k is not None]
    total = sum(ms for _, (n, ms) in items)
    out = []
    for name, (n, ms) in items:
        if n == 0:
            continue
        per = [kernel_work(name, w, fp32) for w in works]
        t_launch = ms / n * 1e-3
        e = {"kernel": name, "launches": n, "us_per_launch": round(1e3 * ms / n, 2),
             "share": round(ms / total, 4) if total else None}
        if per[0] is None:
            e.update(bound=None, note=NO_MODEL.get(name, "no algorithmic work model"))
        else:
            kind, _, what = per[0]
            amount = sum(p[1] for p in per) / len(per)
            if kind == "hbm":
                ach = amount / t_launch / 1e9
                e.update(bound="hbm", achieved=round(ach, 1), peak=hbm, unit="GB/s", frac=round(ach / hbm, 4),
                         algorithmic_per_launch=int(amount), peak_source=hbm_src)
            else:
                peak = FP32_PEAK_TFLOPS if kind == "fp32" else FP64_PEAK_TFLOPS
                ach = amount / t_launch / 1e12
                e.update(bound="alu", achieved=round(ach, 4), peak=round(peak, 3), unit="TFLOP/s",
                         frac=round(ach / peak, 4), algorithmic_per_launch=int(amount),
                         peak_source=("FP32: 152 SM x 128 FMA/clk x 2 x 2.07 GHz (recipe unit counts and clock)"
                                      if kind == "fp32" else "FP64: nominal 1.25 TFLOP/s (recipe table)"))
            e["work_model"] = what
            tr = traffic.get(name)
            e["traffic"] = tr
            if tr is not None:
                e["traffic_source"] = f"ncu dram__bytes_read.sum + dram__bytes_write.sum per launch ({tsrc})"
        out.append(e)
    out.sort(key=lambda e: -(e["share"] or 0))
    return out
NO_MODEL = {"k_cell_order_big": "no algorithmic work model: the block sort of the few cells with more than 256 "
                                 "pairs (their pair count is not counted)"}
# the paper's own PPIC neighbourhood and frame (ft_params.fit_ring / frame), not part of the timed step:
# their ring and vertex counts are not among the work counts
for _k in ("k_count (incidence)", "k_edge_max", "k_closest", "k_ppic_ring"):
    NO_MODEL[_k] = ("no algorithmic work model: a kernel of the paper's own PPIC neighbourhood and frame (an "
                    "option outside the timed step), whose ring sizes are not counted")
PARAB_FP64_FLOPS_PER_CELL = 72252.0  # FP64 flops (add + mul + 2 fma) executed per cell by k_parab_ppic on this workload (ncu)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "fp32c"], default="fp32c")
    ap.add_argument("--alt-steps", type=int, default=30, help="steps timed for the other precision (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-graph", action="store_true",
                    help="time eager launches instead of one CUDA graph per step")
    ap.add_argument("--phase-steps", type=int, default=20,
                    help="eager steps timed per phase (and as many traced per kernel)")
    ap.add_argument("--config-steps", type=int, default=10,
                    help="timed steps of the 32^3 droplet and 256^3 droplet/bubble legs, both forms (0: skip)")
    ap.add_argument("--profile-batch", type=int, default=0,
                    help="only run this many eager steps of the 512-front batch (for a profiler's launch list)")
    ap.add_argument("--paraboloid-reps", type=int, default=5,
                    help="timed calls of front_volume_fraction_ppic (the paper's own alpha) on the step's fits")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-mode", choices=("concurrent", "staggered", "graph"), default="graph",
                    help="e2e leg: the fronts on concurrent compute streams, or one after the other so that "
                         "the first front's outputs go down while the second is computed (eager, or that step "
                         "captured in one CUDA graph)")
    ap.add_argument("--e2e-compute", choices=("per_front", "shared"), default="per_front",
                    help="staggered/graph e2e leg: each front's calls on its own compute stream (the fronts "
                         "computed concurrently, as in the graph step), or both fronts on one compute stream")
    ap.add_argument("--e2e-upload-streams", type=int, default=1,
                    help="staggered/graph e2e leg: copy streams the face-velocity uploads are spread over "
                         "(round robin over the face arrays; vertices and triangles go first on the first)")
    ap.add_argument("--e2e-faces", choices=("inplace", "copy"), default="copy",
                    help="face velocities of the e2e leg: read in place from pinned host memory by the "
                         "interpolation kernel, or copied to the device every step (the other is measured beside)")
    ap.add_argument("--e2e-outputs", choices=("compact", "dense"), default="compact",
                    help="e2e leg: download alpha and the force in the compact form (front_alpha_pack, "
                         "front_csf_force_compact: the same information) or as dense arrays")
    ap.add_argument("--batch-no-fork", dest="batch_fork", action="store_false",
                    help="batched leg: the step's calls in order on one stream instead of the DAG")
    ap.add_argument("--no-fork", dest="fork", action="store_false",
                    help="graph steps with each front's five calls in order on one stream, instead of the DAG "
                         "per front (volume fraction beside the PPIC fit, the interpolation beside everything)")
    ap.add_argument("--autotune", action="store_true",
                    help="install ft_autotune's launch shapes on each front's workspace before timing")
    ap.add_argument("--batch-steps", type=int, default=5,
                    help="timed steps of the batched form (512 fronts); 0: skip")
    ap.add_argument("--batch-fronts", type=int, default=512)
    ap.add_argument("--serve-requests", type=int, default=48, help="requests per served run; 0: skip")
    ap.add_argument("--serve-rates", type=str, default="10,30,100,300,1000,2000",
                    help="Poisson arrival rates (req/s)")
    ap.add_argument("--serve-policies", type=str, default="fifo,backfill",
                    help="admission policies timed at every rate (serve.Scheduler)")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0, help="device memory for resident requests")
    return ap.parse_args()


def workload():
    from paper_2505_06932_gb300 import inputs as I
    return [I.rough_sphere_128(2), I.ellipsoid_128(3)]


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as td
        td.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as td
        td.barrier()


def allmax(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as td
    t = torch.tensor([x], dtype=torch.float64)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def allsum(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as td
    t = torch.tensor([x], dtype=torch.float64)
    td.all_reduce(t, op=td.ReduceOp.SUM)
    return float(t.item())


class Clocks:
    """nvidia-smi samples (SM clock, reasons) while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.p = None
        self.out = os.path.join(tempfile.gettempdir(), f"ft_bench_clocks_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.out), exist_ok=True)
            self.f = open(self.out, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(device), "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.out):
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
            except ValueError:
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_pass(w, sel=None):
    """The oracle's five steps on front w (FP64 C on the host cores): binning,
    alpha, PPIC (every interfacial cell, or only the cells `sel`), the CSF force
    (needs every cell's fit, so only with sel None) and the interpolation at the
    vertices.  Returns the interfacial cell count and the time of each step."""
    import numpy as np
    import oracle
    g = w["grid"]
    t = [time.perf_counter()]
    keys, _, _ = oracle.bin_pairs(w["verts"], w["tris"], g)
    t.append(time.perf_counter())
    al, _ = oracle.alpha(w["verts"], w["tris"], g)
    t.append(time.perf_counter())
    cells = np.unique(keys)
    kappa, normal, _, _ = oracle.ppic(w["verts"], w["tris"], g, cells if sel is None else sel)
    t.append(time.perf_counter())
    if sel is None:
        oracle.csf(g, al, cells, kappa, normal, oracle.DEFAULT_PARAMS["sigma"])
    t.append(time.perf_counter())
    oracle.interp(g, w["faces"], w["verts"])
    t.append(time.perf_counter())
    return len(cells), dict(zip(PHASES, (t[k + 1] - t[k] for k in range(5))))


def cpu_baseline(fronts, budget_s=10.0, one_core_budget_s=10.0):
    """The oracle (FP64 C) on the whole workload: passes of the five steps over
    every front on all host cores until budget_s has elapsed (at least one);
    then on one core, passes over the first front until one_core_budget_s."""
    import oracle
    oracle.set_threads(os.cpu_count() or 1)
    cells = passes = 0
    t0 = time.perf_counter()
    while passes == 0 or time.perf_counter() - t0 < budget_s:
        for w in fronts:
            cells += oracle_pass(w)[0]
        passes += 1
    dt = time.perf_counter() - t0
    out = dict(value=cells / dt, unit="interfacial cells/s", cores=oracle.get_threads(), kind="oracle",
               sample=f"{passes} pass{'es' if passes != 1 else ''} of the five steps over the whole workload "
                      f"({cells // passes} interfacial "
                      f"cells per pass, every cell fitted), {dt:.1f} s; cells/s = cells / time")
    if one_core_budget_s > 0:
        oracle.set_threads(1)
        c1 = p1 = 0
        t0 = time.perf_counter()
        while p1 == 0 or time.perf_counter() - t0 < one_core_budget_s:
            c1 += oracle_pass(fronts[0])[0]
            p1 += 1
        d1 = time.perf_counter() - t0
        out["one_core"] = dict(value=round(c1 / d1, 1), unit="interfacial cells/s", cores=oracle.get_threads(),
                               kind="oracle",
                               sample=f"{p1} pass{'es' if p1 != 1 else ''} of the five steps over "
                                      f"{fronts[0]['name']} ({c1 // p1} interfacial cells, every cell fitted), "
                                      f"{d1:.1f} s, one thread")
        oracle.set_threads(os.cpu_count() or 1)
    return out


PHASES = ("bin", "alpha", "ppic", "csf", "interp")


def run_ours(a):
    import numpy as np
    import torch
    from paper_2505_06932_gb300 import _front as F

    ws, rank, local = dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fronts = workload()
    prec = F.FT_FP64 if a.precision == "fp64" else F.FT_FP32C
    dfr = []
    for w in fronts:
        v = torch.from_numpy(w["verts"]).to(dev)
        t = torch.from_numpy(w["tris"]).to(dev)
        fa = [torch.from_numpy(f).to(dev) for f in w["faces"]]
        dfr.append((v, t, fa))
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MB > L2

    def make(precision, fronts=fronts):
        prm = F.make_params(precision=precision)
        fcs = [F.FrontCoupling(w["grid"], w["tris"].shape[0], w["verts"].shape[0], params=prm, device=local)
               for w in fronts]
        return prm, fcs

    def step_one(prm, fc, v, t, fa, ev=None):
        calls = (lambda: F.front_bin(fc.ws, v, t, prm),
                 lambda: F.front_volume_fraction(fc.ws, fc.alpha),
                 lambda: F.front_curvature_ppic(fc.ws, prm, fc.cell_keys, fc.kappa, fc.normal, fc.coeffs,
                                                fc.fit_status),
                 lambda: F.front_csf_force(fc.ws, prm, fc.alpha, fc.kappa, fc.normal, fc.force),
                 lambda: F.front_interp_velocity(fc.grid, fa[0], fa[1], fa[2], v, fc.vel[:v.shape[0]]))
        for name, call in zip(PHASES, calls):
            if ev is not None:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(torch.cuda.current_stream())
                call()
                e1.record(torch.cuda.current_stream())
                ev[name].append((e0, e1))
            else:
                call()

    def step(prm, fcs, ev=None, dfr=dfr):
        for (v, t, fa), fc in zip(dfr, fcs):
            step_one(prm, fc, v, t, fa, ev)

    def step_forked(prm, fc, v, t, fa, sd, sa, si):
        """One front's step as a small DAG: the volume fraction and the PPIC fit
        both need only the binning (they may share a workspace on two streams),
        the CSF force needs both, the interpolation only the face velocities.
        The force's clear needs nothing: it runs beside the binning; its ring
        list needs only the binning: it runs beside the fit (front_force_clear,
        front_csf_prepare, then front_csf_force_cells after the fit)."""
        with torch.cuda.stream(si):
            F.front_interp_velocity(fc.grid, fa[0], fa[1], fa[2], v, fc.vel[:v.shape[0]])
        with torch.cuda.stream(sa):
            F.front_force_clear(fc.ws, fc.force)
        with torch.cuda.stream(sd):
            F.front_bin(fc.ws, v, t, prm)
        sa.wait_stream(sd)
        with torch.cuda.stream(sa):
            F.front_volume_fraction(fc.ws, fc.alpha)
            F.front_csf_prepare(fc.ws)
        with torch.cuda.stream(sd):
            F.front_curvature_ppic(fc.ws, prm, fc.cell_keys, fc.kappa, fc.normal, fc.coeffs, fc.fit_status)
            sd.wait_stream(sa)
            F.front_csf_force_cells(fc.ws, prm, fc.alpha, fc.kappa, fc.normal, fc.force)

    def capture(prm, fcs, dfr=dfr):
        """One CUDA graph for a whole step; the fronts are independent, so each
        runs on its own streams forked from (and joined back to) the capture
        stream: as the DAG of step_forked, or (--no-fork) in order on one stream."""
        g = torch.cuda.CUDAGraph()
        per = 3 if a.fork else 1
        sides = [[torch.cuda.Stream(device=dev) for _ in range(per)] for _ in fcs]
        with torch.cuda.graph(g):
            cs = torch.cuda.current_stream()
            for ss in sides:
                for x in ss:
                    x.wait_stream(cs)
            for (v, t, fa), fc, ss in zip(dfr, fcs, sides):
                if a.fork:
                    step_forked(prm, fc, v, t, fa, *ss)
                else:
                    with torch.cuda.stream(ss[0]):
                        step_one(prm, fc, v, t, fa)
            for ss in sides:
                for x in ss:
                    cs.wait_stream(x)
        return g

    def measure(precision, steps, warmup, clocks=False, fronts=fronts, dfr=dfr, phase_steps=None):
        phase_steps = a.phase_steps if phase_steps is None else phase_steps
        prm, fcs = make(precision, fronts)
        for _ in range(max(3, warmup)):
            step(prm, fcs, dfr=dfr)
        torch.cuda.synchronize()
        tunings = None
        if a.autotune:
            tunings = [F.ft_autotune(fc.ws, prm, reps=3, verts=v, tris=t) for (v, t, fa), fc in zip(dfr, fcs)]
            for _ in range(max(3, warmup)):
                step(prm, fcs, dfr=dfr)
            torch.cuda.synchronize()
        counts = [fc.ws.counts() for fc in fcs]
        works = []
        for fc, w in zip(fcs, fronts):
            wc = fc.ws.work_counts()
            wc.update(V=int(w["verts"].shape[0]), N=int(w["grid"].ncells))
            works.append(wc)
        status = [fc.ws.status() for fc in fcs]
        if any(status):
            raise RuntimeError(f"device status after warm-up: {[F.status_names(x) for x in status]}")
        # eager steps with an event pair around every call (the per-phase
        # breakdown), then eager steps with an event pair around every kernel
        # (the per-kernel roofline); L2 flushed before each step
        ph = {n: [] for n in PHASES}
        l0 = F.launch_count()
        for _ in range(phase_steps):
            flush.zero_()
            step(prm, fcs, ph, dfr=dfr)
        torch.cuda.synchronize()
        kernels_per_step = (F.launch_count() - l0) / max(1, phase_steps)
        phase_ms = {n: sum(e0.elapsed_time(e1) for e0, e1 in ph[n]) / max(1, phase_steps) for n in PHASES}
        ppic_ms_eager = [e0.elapsed_time(e1) for e0, e1 in ph["ppic"]]
        F.trace_start(64 * max(1, phase_steps) * len(fcs))
        for _ in range(phase_steps):
            flush.zero_()
            step(prm, fcs, dfr=dfr)
        torch.cuda.synchronize()
        trace = F.trace_stop()
        graph = None if a.no_graph else capture(prm, fcs, dfr=dfr)
        if graph is not None:
            graph.replay()
            torch.cuda.synchronize()
            if any(fc.ws.status() for fc in fcs):
                raise RuntimeError("device status after graph replay")
        clk = Clocks(local) if clocks else None
        barrier(ws)
        torch.cuda.synchronize()
        l0 = F.launch_count()
        evs = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if graph is not None:
                graph.replay()
            else:
                step(prm, fcs, dfr=dfr)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        barrier(ws)
        launches = (kernels_per_step * steps) if graph is not None else (F.launch_count() - l0)
        clk = clk.stop() if clk else None
        total_ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
        return dict(prm=prm, fcs=fcs, counts=counts, works=works, total_ms=total_ms, phase_ms=phase_ms,
                    ppic_ms=ppic_ms_eager, launches=launches, clocks=clk, graph=graph, tunings=tunings,
                    trace=trace, kernels_per_step=kernels_per_step)

    def measure_batch_of_fronts(precision, steps):
        """The same fronts as one batch (one launch sequence for both), one CUDA
        graph per step, launch shapes from ft_autotune."""
        prm = F.make_params(precision=precision)
        dl = [dict(grid=w["grid"], verts=v, tris=t, U=fa[0], V=fa[1], W=fa[2]) for w, (v, t, fa) in zip(fronts, dfr)]
        bc = F.BatchCoupling(dl, params=prm, device=local)
        tune = F.ft_autotune(bc.ws, prm, reps=3)
        for _ in range(3):
            bc.step()
        torch.cuda.synchronize()
        if bc.ws.status() or any(bc.ws.front_status()):
            raise RuntimeError("batch of the bench fronts: device status")
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            bc.step()
        g.replay()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        M = bc.ws.counts()["M"]
        del g
        bc.ws.close()
        return dict(value=round(M * steps / (tot * 1e-3), 1), ms_per_step=round(tot / steps, 4), steps=steps,
                    tuning={k: tune[k] for k in ("clip_blocks_per_sm", "ppic_blocks_per_sm", "csf_blocks_per_sm",
                                                 "fill_blocks_per_sm", "ppic_min_blocks", "ppic_dynamic",
                                                 "sort_blocks")},
                    launch="the two fronts as one batch (front_*_batch), one CUDA graph per step")

    r = measure(prec, a.steps, a.warmup, clocks=True)
    counts = r["counts"]
    cells_per_step = sum(c["M"] for c in counts)
    fit_pairs = [c["fit_pairs"] for c in counts]
    tmax = allmax(ws, r["total_ms"])
    value = allsum(ws, cells_per_step * a.steps) / (tmax * 1e-3)

    # per-kernel rooflines from the traced eager steps; the headline object is
    # the kernel with the largest share of the traced device time
    tag = "fp32c_two_fronts_128" if prec == F.FT_FP32C else "fp64_two_fronts_128"
    kernels = roofline_list(r["trace"], r["works"], prec == F.FT_FP32C, tag)
    dom = next(e for e in kernels if e.get("bound"))
    roof = {k: dom[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
    roof.update(kernel=dom["kernel"], share_of_traced_time=dom["share"], us_per_launch=dom["us_per_launch"],
                algorithmic_per_launch=dom["algorithmic_per_launch"], work_model=dom["work_model"],
                peak_source=dom["peak_source"],
                timing="CUDA events around every launch of the kernel (ft_trace_start/stop) in "
                       f"{a.phase_steps} eager steps, L2 flushed before each step; the launch's own stream")
    if dom.get("traffic_source"):
        roof["traffic_source"] = dom["traffic_source"]
    try:
        probe = F.probe_fma_rate(0 if prec == F.FT_FP64 else 1, local) / 1e12
        roof["probe_measured_fma_peak"] = round(probe, 4)
    except Exception:
        pass
    phases = {n: round(v, 4) for n, v in r["phase_ms"].items()}

    alt = None
    if a.alt_steps > 0:
        other = F.FT_FP64 if prec == F.FT_FP32C else F.FT_FP32C
        ra = measure(other, a.alt_steps, 3)
        ta = allmax(ws, ra["total_ms"])
        alt = {"precision": "fp64" if other == F.FT_FP64 else "fp32c", "steps": a.alt_steps,
               "value": round(allsum(ws, cells_per_step * a.alt_steps) / (ta * 1e-3), 1),
               "ms_per_step": round(ta / a.alt_steps, 4),
               "phases_ms": {n: round(v, 4) for n, v in ra["phase_ms"].items()},
               "roofline_kernels": roofline_list(ra["trace"], ra["works"], other == F.FT_FP32C,
                                                 "fp32c_two_fronts_128" if other == F.FT_FP32C
                                                 else "fp64_two_fronts_128")}
        for fc in ra["fcs"]:
            fc.ws.close()

    one_batch = measure_batch_of_fronts(prec, a.steps) if a.alt_steps > 0 else None

    def config_leg(title, ws_fronts, tag, steps):
        """Another workload of the paper's shapes, both forms: cells/s of the
        graph step and the per-kernel rooflines of traced eager steps."""
        d_in = []
        for w in ws_fronts:
            d_in.append((torch.from_numpy(w["verts"]).to(dev), torch.from_numpy(w["tris"]).to(dev),
                         [torch.from_numpy(f).to(dev) for f in w["faces"]]))
        out = {"workload": title, "fronts": [w["name"] for w in ws_fronts],
               "triangles": [int(w["tris"].shape[0]) for w in ws_fronts],
               "l2": "flushed (512 MB write) before every timed step", "launch": "as the main line"}
        for precision, ptag in ((F.FT_FP32C, "fp32c"), (F.FT_FP64, "fp64")):
            rr = measure(precision, steps, 3, fronts=ws_fronts, dfr=d_in, phase_steps=max(2, min(5, steps)))
            tt = allmax(ws, rr["total_ms"])
            M = sum(c["M"] for c in rr["counts"])
            out[ptag] = {"value": round(allsum(ws, M * steps) / (tt * 1e-3), 1), "unit": "interfacial cells/s",
                         "ms_per_step": round(tt / steps, 4), "steps": steps, "cells_per_step": M,
                         "fit_pairs_per_step": sum(c["fit_pairs"] for c in rr["counts"]),
                         "clip_pairs_decided_in_fp64": sum(w["clip_f64"] for w in rr["works"]),
                         "candidate_pairs": sum(w["C"] for w in rr["works"]),
                         "phases_ms": {n: round(v, 4) for n, v in rr["phase_ms"].items()},
                         "roofline_kernels": roofline_list(rr["trace"], rr["works"], precision == F.FT_FP32C,
                                                           f"{ptag}_{tag}")}
            for fc in rr["fcs"]:
                fc.ws.close()
            del rr
        torch.cuda.empty_cache()
        return out

    configs = None
    if a.config_steps > 0:
        from paper_2505_06932_gb300 import inputs as I
        configs = {
            "laplace_droplet_32": config_leg("icosphere s4 (5,120 triangles) R 0.25, 32^3 grid (the paper's "
                                             "Laplace-equilibrium droplet shape)", [I.laplace_droplet_32(1)],
                                             "droplet_32", max(a.config_steps, 20)),
            "sh_droplet_bubble_256": config_leg(
                "icosphere s7 (327,680 triangles) R 0.2 with real SH deformation l 2..8 (oscillating droplet) "
                "and the flattened, dimpled bubble, 256^3 grid, Taylor-Green faces",
                [I.sh_droplet_256(seed=4), I.sh_droplet_256(seed=4, bubble=True)], "sh_droplet_bubble_256",
                a.config_steps)}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    prm, fcs = r["prm"], r["fcs"]
    hin = []
    for w in fronts:
        hv = torch.from_numpy(w["verts"]).pin_memory()
        ht = torch.from_numpy(w["tris"]).pin_memory()
        hf = [torch.from_numpy(f).pin_memory() for f in w["faces"]]
        hin.append((hv, ht, hf))
    hout = []
    dcomp = []
    h2d = d2h = 0
    compact = a.e2e_outputs == "compact" and a.e2e_mode != "concurrent"  # (concurrent: dense only)
    for (hv, ht, hf), fc, c in zip(hin, fcs, counts):
        M = c["M"]
        outs = dict(kappa=torch.empty(M, dtype=torch.float64).pin_memory(),
                    normal=torch.empty((M, 3), dtype=torch.float64).pin_memory(),
                    vel=torch.empty((hv.shape[0], 3), dtype=torch.float64).pin_memory())
        if compact:
            # compact outputs (the same information): alpha as one bit per cell plus
            # the interfacial values, the force at its non-zero cells with their keys;
            # the slot count of the force is measured once and copied with margin
            N = fc.grid.ncells
            d = dict(bits=torch.empty((N + 31) // 32, dtype=torch.int32, device=dev),
                     acells=torch.empty(M, dtype=torch.float64, device=dev),
                     count=torch.zeros(1, dtype=torch.int64, device=dev))
            cap0 = 16 * M + 1024
            d["keys"] = torch.empty(cap0, dtype=torch.int32, device=dev)
            d["force"] = torch.empty((cap0, 3), dtype=torch.float64, device=dev)
            F.front_csf_force_compact(fc.ws, prm, fc.alpha, fc.kappa, fc.normal, d["keys"], d["force"], d["count"])
            torch.cuda.synchronize()
            if fc.ws.status():
                raise RuntimeError("compact force: device status")
            cap = int(d["count"].item()) + 64 + int(d["count"].item()) // 10
            d["cap"] = cap
            dcomp.append(d)
            outs.update(bits=torch.empty_like(d["bits"], device="cpu").pin_memory(),
                        acells=torch.empty(M, dtype=torch.float64).pin_memory(),
                        count=torch.empty(1, dtype=torch.int64).pin_memory(),
                        keys=torch.empty(cap, dtype=torch.int32).pin_memory(),
                        force=torch.empty((cap, 3), dtype=torch.float64).pin_memory())
        else:
            dcomp.append(None)
            outs.update(alpha=torch.empty(fc.alpha.shape, dtype=torch.float64).pin_memory(),
                        force=torch.empty(fc.force.shape, dtype=torch.float64).pin_memory())
        hout.append(outs)
        h2d += hv.numel() * 8 + ht.numel() * 4 + sum(f.numel() * 8 for f in hf)
        d2h += sum(o.numel() * o.element_size() for o in outs.values())
    torch.cuda.synchronize()
    # One step's transfers and calls, enqueued on streams forked from `cs` and
    # joined back to it.  "staggered": one upload stream (vertices and
    # triangles of every front first, then the face velocities in front order),
    # a download stream per front, and the compute either on a stream per front
    # (--e2e-compute per_front: the fronts concurrently, the face upload under
    # the binning and the fit) or on one stream (shared: the first front's
    # outputs go down while the second is computed).
    # "concurrent": each front on its own compute stream with a copy stream (face
    # velocities up and alpha down during the binning and the fit).
    stag = a.e2e_mode in ("staggered", "graph")
    if stag:
        sd0 = torch.cuda.Stream(device=dev)
        e2e_streams = dict(sds=[torch.cuda.Stream(device=dev) for _ in fcs] if a.e2e_compute == "per_front"
                           else [sd0 for _ in fcs],
                           ups=[torch.cuda.Stream(device=dev) for _ in range(max(1, a.e2e_upload_streams))],
                           dns=[torch.cuda.Stream(device=dev) for _ in fcs],
                           sas=[torch.cuda.Stream(device=dev) for _ in fcs],
                           sis=[torch.cuda.Stream(device=dev) for _ in fcs])
    else:
        e2e_streams = dict(sides=[torch.cuda.Stream(device=dev) for _ in fcs],
                           copies=[torch.cuda.Stream(device=dev) for _ in fcs])

    def e2e_enqueue(cs, inplace):
        # inplace: the face velocities stay in the pinned host buffers and the
        # interpolation reads the values it needs there (no face upload)
        if stag:
            sds, ups, dns = e2e_streams["sds"], e2e_streams["ups"], e2e_streams["dns"]
            sas, sis = e2e_streams["sas"], e2e_streams["sis"]
            for x in sds + ups + dns + sas + sis:
                x.wait_stream(cs)
            vt_in = [torch.cuda.Event() for _ in fcs]
            faces_in = [[] for _ in fcs]  # per front: an event on every upload stream that carried its faces
            with torch.cuda.stream(ups[0]):
                for (hv, ht, hf), (v, t, fa), ev in zip(hin, dfr, vt_in):
                    v.copy_(hv, non_blocking=True)
                    t.copy_(ht, non_blocking=True)
                    ev.record(ups[0])
            j = 0
            for f, ((hv, ht, hf), (v, t, fa)) in enumerate(zip(hin, dfr)):
                used = []
                for dst, src in ([] if inplace else zip(fa, hf)):
                    u = ups[j % len(ups)]
                    j += 1
                    with torch.cuda.stream(u):
                        dst.copy_(src, non_blocking=True)
                    if u not in used:
                        used.append(u)
                for u in used:
                    ev = torch.cuda.Event()
                    ev.record(u)
                    faces_in[f].append(ev)
            for f, ((v, t, fa), fc, o, c, dn, d) in enumerate(zip(dfr, fcs, hout, counts, dns, dcomp)):
                # each front as the DAG of the graph step: alpha beside the PPIC fit,
                # the interpolation beside both (once the faces are up)
                alpha_ready, force_ready, vel_ready = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()
                sd, sa, si = sds[f], sas[f], sis[f]
                if d is None:
                    with torch.cuda.stream(sa):
                        F.front_force_clear(fc.ws, fc.force)  # beside the binning
                with torch.cuda.stream(sd):
                    sd.wait_event(vt_in[f])
                    F.front_bin(fc.ws, v, t, prm)
                sa.wait_stream(sd)
                with torch.cuda.stream(sa):
                    F.front_volume_fraction(fc.ws, fc.alpha)
                    if d is not None:
                        F.front_alpha_pack(fc.ws, fc.alpha, d["bits"], d["acells"])
                    else:
                        F.front_csf_prepare(fc.ws)  # the ring list beside the fit
                    alpha_ready.record(sa)
                with torch.cuda.stream(si):
                    si.wait_event(vt_in[f])
                    for ev in faces_in[f]:
                        si.wait_event(ev)
                    fu = hin[f][2] if inplace else fa
                    F.front_interp_velocity(fc.grid, fu[0], fu[1], fu[2], v, fc.vel[:v.shape[0]])
                    vel_ready.record(si)
                with torch.cuda.stream(sd):
                    F.front_curvature_ppic(fc.ws, prm, fc.cell_keys, fc.kappa, fc.normal, fc.coeffs, fc.fit_status)
                    sd.wait_event(alpha_ready)
                    if d is not None:
                        F.front_csf_force_compact(fc.ws, prm, fc.alpha, fc.kappa, fc.normal, d["keys"], d["force"],
                                                  d["count"])
                    else:
                        F.front_csf_force_cells(fc.ws, prm, fc.alpha, fc.kappa, fc.normal, fc.force)
                    force_ready.record(sd)
                with torch.cuda.stream(dn):
                    M = c["M"]
                    dn.wait_event(alpha_ready)
                    if d is not None:
                        o["bits"].copy_(d["bits"], non_blocking=True)
                        o["acells"].copy_(d["acells"], non_blocking=True)
                    else:
                        o["alpha"].copy_(fc.alpha, non_blocking=True)
                    dn.wait_event(force_ready)
                    if d is not None:
                        o["count"].copy_(d["count"], non_blocking=True)
                        o["keys"].copy_(d["keys"][:d["cap"]], non_blocking=True)
                        o["force"].copy_(d["force"][:d["cap"]], non_blocking=True)
                    else:
                        o["force"].copy_(fc.force, non_blocking=True)
                    o["kappa"].copy_(fc.kappa[:M], non_blocking=True)
                    o["normal"].copy_(fc.normal[:M], non_blocking=True)
                    dn.wait_event(vel_ready)
                    o["vel"].copy_(fc.vel[:v.shape[0]], non_blocking=True)
            for x in sds + ups + dns + sas + sis:
                cs.wait_stream(x)
        else:
            sides, copies = e2e_streams["sides"], e2e_streams["copies"]
            for sd, cp in zip(sides, copies):
                sd.wait_stream(cs)
                cp.wait_stream(cs)
            for (hv, ht, hf), (v, t, fa), fc, o, c, sd, cp in zip(hin, dfr, fcs, hout, counts, sides, copies):
                faces_in, alpha_ready = torch.cuda.Event(), torch.cuda.Event()
                with torch.cuda.stream(cp):
                    for dst, src in ([] if inplace else zip(fa, hf)):
                        dst.copy_(src, non_blocking=True)
                    faces_in.record(cp)
                with torch.cuda.stream(sd):
                    v.copy_(hv, non_blocking=True)
                    t.copy_(ht, non_blocking=True)
                    F.front_bin(fc.ws, v, t, prm)
                    F.front_volume_fraction(fc.ws, fc.alpha)
                    alpha_ready.record(sd)
                    F.front_curvature_ppic(fc.ws, prm, fc.cell_keys, fc.kappa, fc.normal, fc.coeffs, fc.fit_status)
                    F.front_csf_force(fc.ws, prm, fc.alpha, fc.kappa, fc.normal, fc.force)
                    sd.wait_event(faces_in)
                    fu = hf if inplace else fa
                    F.front_interp_velocity(fc.grid, fu[0], fu[1], fu[2], v, fc.vel[:v.shape[0]])
                    M = c["M"]
                    o["force"].copy_(fc.force, non_blocking=True)
                    o["kappa"].copy_(fc.kappa[:M], non_blocking=True)
                    o["normal"].copy_(fc.normal[:M], non_blocking=True)
                    o["vel"].copy_(fc.vel[:v.shape[0]], non_blocking=True)
                with torch.cuda.stream(cp):
                    cp.wait_event(alpha_ready)
                    o["alpha"].copy_(fc.alpha, non_blocking=True)
            for sd, cp in zip(sides, copies):
                cs.wait_stream(sd)
                cs.wait_stream(cp)

    def time_e2e(inplace):
        e2e_graph = None
        if a.e2e_mode == "graph":
            # the step above captured once (copies from and to the same pinned host
            # buffers, which a caller refills between steps) and replayed every step
            e2e_graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(e2e_graph):
                e2e_enqueue(torch.cuda.current_stream(), inplace)
            torch.cuda.synchronize()
        e2e_ms = 0.0
        for _ in range(a.e2e_steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if e2e_graph is not None:
                e2e_graph.replay()
            else:
                e2e_enqueue(stream, inplace)
            e1.record(stream)
            e1.synchronize()
            e2e_ms += e0.elapsed_time(e1)
        return allsum(ws, cells_per_step * a.e2e_steps) / (allmax(ws, e2e_ms) * 1e-3)

    # the main e2e number reads the faces in place (a.e2e_faces); the other way
    # is measured beside it
    faces_inplace = a.e2e_faces == "inplace"
    e2e_value = time_e2e(faces_inplace)
    e2e_other = time_e2e(not faces_inplace)
    h2d_faces = sum(f.numel() * 8 for _, _, hf in hin for f in hf)
    nv_all = sum(hv.shape[0] for hv, _, _ in hin)

    # the paper's own indicator on the same fits: alpha_P, surface-averaged kappa and normal
    parab = measure_paraboloid(fcs, counts, a.paraboloid_reps, flush, stream) if a.paraboloid_reps > 0 else None

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "interfacial cells/s", "n_gpus": ws,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(tmax / a.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == F.FT_FP64 else "f32+f64",
        "data": "synthetic (seeded icosphere fronts, solid-body face velocities)",
        "config": {"workload": "rough icosphere s6 R0.2 + ellipsoid (0.3,0.2,0.15), 128^3 grid, 81,920 tris each",
                   "fronts": [w["name"] for w in fronts], "cells_per_step": cells_per_step,
                   "pairs_per_step": sum(c["P"] for c in counts), "fit_pairs_per_step": sum(fit_pairs),
                   "candidate_pairs_per_step": sum(w["C"] for w in r["works"]),
                   "clip_pairs_decided_in_fp64": sum(w["clip_f64"] for w in r["works"]),
                   "precision": a.precision,
                   "stated_error": "FP32 form: |d alpha| <= 1e-6, |d kappa| <= 1e-4 rel. vs the FP64 oracle; "
                                   "FP64 path: 1e-12 / 1e-9 (checked by tests/test_gpu_parity.py)",
                   "l2": "flushed (512 MB write) before every timed step",
                   "launch": "eager" if a.no_graph else (
                       "one CUDA graph per step, per front a DAG on three streams (the force clear beside the "
                       "binning, alpha and the CSF ring list beside the PPIC fit, the interpolation beside all)"
                       if a.fork else
                       "one CUDA graph per step, the two fronts on two streams"),
                   "parallelism": f"replicas x{ws}",
                   "launch_shapes": ([{k: t[k] for k in ("clip_blocks_per_sm", "ppic_blocks_per_sm",
                                                          "csf_blocks_per_sm", "fill_blocks_per_sm",
                                                          "ppic_min_blocks", "ppic_dynamic", "sort_blocks")}
                                      for t in r["tunings"]] if r["tunings"] else "library defaults")},
        "phases_ms": phases,
        "phases_note": "eager per-call CUDA-event times per step (sum over fronts), not the graph replay",
        "roofline": roof,
        "roofline_kernels": kernels,
        "alt_precision": alt,
        "same_workload_as_one_batch": one_batch,
        "other_configs": configs,
        "paraboloid": parab,
        "e2e": {"value": round(e2e_value, 1), "unit": "interfacial cells/s",
                "h2d_bytes_per_step": h2d - (h2d_faces if faces_inplace else 0),
                "d2h_bytes_per_step": d2h, "steps": a.e2e_steps,
                "faces": ("left in the pinned host buffers and read in place by the interpolation kernel (at most "
                          f"54 face values, 432 B, per vertex: {432 * nv_all} B per step at most; "
                          f"{h2d_faces} B of face arrays in host memory)" if faces_inplace else
                          f"copied to the device every step ({h2d_faces} B)"),
                ("faces_copied" if faces_inplace else "faces_in_place"): {
                    "value": round(e2e_other, 1),
                    "h2d_bytes_per_step": h2d - (0 if faces_inplace else h2d_faces)},
                "mode": a.e2e_mode, "outputs": a.e2e_outputs + (
                    ": alpha as one bit per cell plus the interfacial values, the CSF force at its non-zero cells "
                    "with their keys, kappa, normal, vertex velocities" if compact else
                    ": dense alpha and force, kappa, normal, vertex velocities"),
                "launch": (("one CUDA graph per step: " if a.e2e_mode == "graph" else "eager calls; ") +
                           (("each front on its own compute stream (the fronts computed concurrently) "
                             if a.e2e_compute == "per_front" else
                             "the fronts one after the other on one compute stream (the first front's outputs go "
                             "down while the second is computed), ") +
                            "each front's calls as the DAG of the graph step, one upload stream (vertices and "
                            "triangles of every front" + ("" if faces_inplace else " first, then the face velocities")
                            + "), a download stream per front"
                            if stag else
                            "per front a compute stream and a copy stream (faces up and alpha down overlap the "
                            "binning and the fit), the two fronts concurrently"))},
        "gpu_launches": int(r["launches"]),
        "clocks": r["clocks"],
    }
    for fc in fcs:
        fc.ws.close()
    if a.batch_steps > 0:
        t_leg = time.perf_counter()
        line["batched"] = run_batched(a, dev, local, flush)
        line["batched"]["leg_wall_s"] = round(time.perf_counter() - t_leg, 1)
        torch.cuda.empty_cache()
    if a.serve_requests > 0:
        t_leg = time.perf_counter()
        line["served"] = run_served(a, local)
        line["served"]["leg_wall_s"] = round(time.perf_counter() - t_leg, 1)
        torch.cuda.empty_cache()
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(fronts)
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_paraboloid(fcs, counts, reps, flush, stream):
    """front_volume_fraction_ppic on the fits of the last step of every front:
    per interfacial cell the cell-below-paraboloid volume, the surface area and
    the surface-averaged curvature and normal (one FP64 thread per cell)."""
    import torch
    from paper_2505_06932_gb300 import _front as F

    outs = []
    for fc in fcs:
        cap = fc.coeffs.shape[0]
        dev = fc.coeffs.device
        outs.append(dict(k=torch.empty(cap, dtype=torch.float64, device=dev),
                         n=torch.empty((cap, 3), dtype=torch.float64, device=dev),
                         a=torch.empty(cap, dtype=torch.float64, device=dev),
                         s=torch.empty(cap, dtype=torch.int8, device=dev)))

    def call():
        for fc, o in zip(fcs, outs):
            F.front_volume_fraction_ppic(fc.ws, fc.coeffs, fc.alpha, o["k"], o["n"], o["a"], o["s"])

    call()
    torch.cuda.synchronize()
    if any(fc.ws.status() for fc in fcs):
        raise RuntimeError("front_volume_fraction_ppic: device status")
    ms = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = sum(ms) / len(ms)
    cells = sum(c["M"] for c in counts)
    misses = sum(int((o["s"][:c["M"]] != 0).sum()) for o, c in zip(outs, counts))
    roof = None
    if PARAB_FP64_FLOPS_PER_CELL:
        ach = PARAB_FP64_FLOPS_PER_CELL * cells / (t * 1e-3) / 1e12
        roof = {"kernel": "k_parab_ppic", "bound": "alu", "achieved": round(ach, 4), "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": round(ach / FP64_PEAK_TFLOPS, 4), "traffic": None,
                "flops_source": "FP64 operations per cell counted by ncu on this workload "
                                "(profiles/k_parab_ppic_two_fronts_128.md)",
                "peak_source": "nominal FP64 1.25 TFLOP/s (recipe table)"}
    return {"call": "front_volume_fraction_ppic", "cells_per_call": cells, "ms_per_call": round(t, 4),
            "cells_per_s": round(cells / (t * 1e-3), 1), "surface_misses": misses, "reps": reps,
            "timing": "CUDA events around both fronts' calls, L2 flushed before each", "roofline": roof}


def profile_batch(a):
    """Eager steps of the 512-front batched workload with the autotuner's usual
    choice fixed (clip 16, PPIC 4, CSF 4, fill 16 blocks per SM, dynamic PPIC
    schedule): a short, deterministic launch sequence for a profiler."""
    import torch
    from paper_2505_06932_gb300 import _front as F, inputs as I

    dev = torch.device("cuda", 0)
    dl = []
    for f in I.batch_fronts(5, a.batch_fronts):
        U, V, W = device_faces(f, dev)
        dl.append(dict(grid=f["grid"], verts=torch.from_numpy(f["verts"]).to(dev),
                       tris=torch.from_numpy(f["tris"]).to(dev), U=U, V=V, W=W))
    bc = F.BatchCoupling(dl, params=F.make_params(precision=F.FT_FP32C), headroom=1.02)
    F.ft_set_tuning(bc.ws, clip=16, ppic=4, csf=4, fill=16, ppic_min_blocks=4, ppic_dynamic=1)
    for _ in range(a.profile_batch):
        bc.step()
    torch.cuda.synchronize()
    print(json.dumps({"profile_batch_steps": a.profile_batch, "status": bc.ws.status(), "counts": bc.ws.counts()}))


def device_faces(f, dev):
    """Noise-free solid-body rotation u = omega x (x - c) at the face centres of
    front f's grid, built on the device (the batched workload's face velocities)."""
    import torch
    g = f["grid"]
    c = [float(x) for x in f["centre"]]
    w = [float(x) for x in f["omega"]]
    out = []
    for ax in range(3):
        n = list(g.n)
        n[ax] += 1
        xs = [g.origin[d] + g.h * (torch.arange(n[d], device=dev, dtype=torch.float64) + (0.0 if d == ax else 0.5))
              - c[d] for d in range(3)]
        X, Y, Z = torch.meshgrid(*xs, indexing="ij")
        u = (w[1] * Z - w[2] * Y, w[2] * X - w[0] * Z, w[0] * Y - w[1] * X)[ax]
        out.append(u.contiguous())
    return out


def run_batched(a, dev, local, flush):
    """The batched form: the 512-front workload (icospheres s3-6 on 32^3-96^3
    grids) through the batched entry points, one CUDA graph per step, launch
    shapes from ft_autotune; FP32-compensated and FP64, and the same fronts
    through the one-front entry points in a loop for comparison."""
    import torch
    from paper_2505_06932_gb300 import _front as F
    from paper_2505_06932_gb300 import inputs as I
    fr = I.batch_fronts(5, a.batch_fronts)
    dl = []
    for f in fr:
        U, V, W = device_faces(f, dev)
        dl.append(dict(grid=f["grid"], verts=torch.from_numpy(f["verts"]).to(dev),
                       tris=torch.from_numpy(f["tris"]).to(dev), U=U, V=V, W=W))
    stream = torch.cuda.current_stream()
    out = {"workload": f"{len(fr)} fronts: icosphere s3-6, grids 32^3/48^3/64^3/96^3, radius log-uniform in "
                       f"[3h, 20h] (capped at (N/2-8)h), radial roughness 1e-3 h",
           "fronts": len(fr), "triangles": int(sum(f["tris"].shape[0] for f in fr)),
           "grid_cells": int(sum(f["grid"].ncells for f in fr)),
           "radius_capped": int(sum(f["capped"] for f in fr)),
           "launch": ("one CUDA graph per step, a DAG on three streams: front_force_clear_batch beside "
                      "front_bin_batch, then front_volume_fraction_batch and front_csf_prepare beside "
                      "front_curvature_ppic, then front_csf_force_cells_batch and ft_batch_cell_ranges; "
                      "front_interp_velocity_batch beside all of them" if a.batch_fork else
                      "one CUDA graph per step: front_bin_batch, front_volume_fraction_batch, "
                      "front_curvature_ppic, front_csf_force_batch, ft_batch_cell_ranges, "
                      "front_interp_velocity_batch"),
           "l2": "inputs larger than L2 (dense fields alone 1.4 GB) and a 512 MB flush before every timed step"}
    tuning = None
    for prec, tag in ((F.FT_FP32C, "fp32c"), (F.FT_FP64, "fp64")):
        prm = F.make_params(precision=prec)
        bc = F.BatchCoupling(dl, params=prm, headroom=1.02, device=local)
        if tuning is None:
            tuning = F.ft_autotune(bc.ws, prm, reps=2)
            out["tuning"] = {k: tuning[k] for k in ("clip_blocks_per_sm", "ppic_blocks_per_sm",
                                                    "csf_blocks_per_sm", "fill_blocks_per_sm", "ppic_min_blocks",
                                                    "ppic_dynamic", "sort_blocks")}
        else:
            F.ft_set_tuning(bc.ws, clip=tuning["clip_blocks_per_sm"], ppic=tuning["ppic_blocks_per_sm"],
                            csf=tuning["csf_blocks_per_sm"], fill=tuning["fill_blocks_per_sm"],
                            ppic_min_blocks=tuning["ppic_min_blocks"], ppic_dynamic=tuning["ppic_dynamic"],
                            sort_blocks=tuning["sort_blocks"])
        for _ in range(3):
            bc.step()
        torch.cuda.synchronize()
        st = bc.ws.status()
        fst = bc.ws.front_status()
        if st or any(fst):
            raise RuntimeError(f"batched form: device status {F.status_names(st)}")
        c = bc.ws.counts()
        g = torch.cuda.CUDAGraph()
        if a.batch_fork:
            # the step as a DAG (as each front's step in the main leg): the force
            # clear beside the binning, the volume fraction beside the PPIC fit
            # (both need only the binning), the CSF force after both, the
            # interpolation beside everything
            sa, si = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
            with torch.cuda.graph(g):
                cs = torch.cuda.current_stream()
                si.wait_stream(cs)
                sa.wait_stream(cs)
                with torch.cuda.stream(si):
                    F.front_interp_velocity_batch(bc.ws)
                with torch.cuda.stream(sa):
                    F.front_force_clear_batch(bc.ws)
                F.front_bin_batch(bc.ws, prm)
                sa.wait_stream(cs)
                with torch.cuda.stream(sa):
                    F.front_volume_fraction_batch(bc.ws)
                    F.front_csf_prepare(bc.ws)
                F.front_curvature_ppic(bc.ws, prm, bc.cell_keys, bc.kappa, bc.normal, bc.coeffs, bc.fit_status)
                cs.wait_stream(sa)
                F.front_csf_force_cells_batch(bc.ws, prm, bc.kappa, bc.normal)
                F.ft_batch_cell_ranges(bc.ws, bc.off)
                cs.wait_stream(si)
        else:
            with torch.cuda.graph(g):
                bc.step()
        g.replay()
        torch.cuda.synchronize()
        steps = a.batch_steps if prec == F.FT_FP32C else max(1, a.batch_steps // 2)
        l0 = F.launch_count()
        bc.step()
        torch.cuda.synchronize()
        per_step = F.launch_count() - l0
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        if bc.ws.status() or any(bc.ws.front_status()):
            raise RuntimeError("batched form: device status after the timed steps")
        out[tag] = {"value": round(c["M"] * steps / (tot * 1e-3), 1), "ms_per_step": round(tot / steps, 3),
                    "steps": steps, "cells_per_step": c["M"], "pairs_per_step": c["P"],
                    "fit_pairs_per_step": c["fit_pairs"], "kernels_per_step": per_step,
                    "workspace_bytes": bc.ws.bytes}
        del g
        bc.ws.close()
        del bc
        torch.cuda.empty_cache()
    # the same fronts through the one-front entry points, front after front (eager)
    prm = F.make_params(precision=F.FT_FP32C)
    fcs = {}
    for f, d in zip(fr, dl):
        N = f["grid"].n[0]
        if N not in fcs:
            mt = max(x["tris"].shape[0] for x in fr if x["grid"].n[0] == N)
            mv = max(x["verts"].shape[0] for x in fr if x["grid"].n[0] == N)
            fcs[N] = F.FrontCoupling(f["grid"], mt, mv, params=prm, device=local)
    for _ in range(2):
        for f, d in zip(fr, dl):
            fcs[f["grid"].n[0]].step(d["verts"], d["tris"], (d["U"], d["V"], d["W"]))
    torch.cuda.synchronize()
    loop_steps = max(1, a.batch_steps // 2)
    tot = 0.0
    for _ in range(loop_steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for f, d in zip(fr, dl):
            fcs[f["grid"].n[0]].step(d["verts"], d["tris"], (d["U"], d["V"], d["W"]))
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    M = out["fp32c"]["cells_per_step"]
    out["per_front_loop_fp32c"] = {"value": round(M * loop_steps / (tot * 1e-3), 1),
                                   "ms_per_step": round(tot / loop_steps, 3), "steps": loop_steps,
                                   "launch": "eager, one-front entry points, fronts in sequence"}
    for fc in fcs.values():
        fc.ws.close()
    return out


def run_served(a, local):
    """The served form: request streams (Poisson arrivals) of SH-deformed fronts
    on 32^3-512^3 grids, 1-50 steps each, served with continuous batching in the
    FP32 form; the same stream served by the plain FP64 path one request at a
    time.  Latency = arrival -> end of the request's last step (wall clock)."""
    import torch
    from paper_2505_06932_gb300 import _front as F
    from paper_2505_06932_gb300 import inputs as I
    from paper_2505_06932_gb300 import serve as S

    rates = [float(x) for x in a.serve_rates.split(",") if x]
    # one stream; other rates rescale its Poisson arrival times (the same draws)
    base = I.served_requests(11, a.serve_requests, rates[0], pool_per_s=1)

    def requests(rate):
        f = rates[0] / rate
        return [S.Request(r["rid"], r["grid"], r["verts"], r["tris"], r["steps"], r["arrival"] * f, r["dt"],
                          tuple(r["centre"]), tuple(r["omega"])) for r in base]

    budget = int(a.serve_budget_gb * 2 ** 30)
    probe = requests(rates[0])
    cap = S.Capacity(budget_bytes=budget, max_fronts=256,
                     max_grid_cells=min(2 ** 32 - 2, budget // 56),
                     max_nt=sum(r.tris.shape[0] for r in probe),
                     max_cand=sum(S.candidate_estimate(r) for r in probe))
    policies = [x for x in a.serve_policies.split(",") if x]
    small = {r["rid"] for r in base if max(r["grid"].n) <= 128}
    out = {"workload": f"{a.serve_requests} requests per rate: icosphere s4-8 with real SH deformation "
                       f"(l 2-8, c ~ N(0,(0.05R)^2)), grids 32^3-512^3, 1-50 steps of dt = 0.25h each "
                       f"(bin, alpha, PPIC, CSF, RK4 advection), solid-body rotation about the front centre",
           "budget_bytes": budget,
           "admission": "by device footprint and batch capacities; fifo: the queue head blocks the requests "
                        "behind it; backfill: requests that fit pass a blocked head until it has waited 1 s",
           "classes": f"small: grid <= 128^3 ({len(small)} requests), large: 256^3 and 512^3 "
                      f"({len(base) - len(small)} requests)",
           "precision": "fp32c", "rates": {}}

    def by_class(outs):
        res = {}
        for cls, sel in (("small", lambda rid: rid in small), ("large", lambda rid: rid not in small)):
            lat = [o.latency for o in outs.values() if sel(o.rid) and not o.rejected and o.latency == o.latency]
            if lat:
                res[cls] = {"n": len(lat), "p50_ms": round(1e3 * statistics.median(lat), 3),
                            "p99_ms": round(1e3 * sorted(lat)[min(len(lat) - 1, int(0.99 * len(lat)))], 3)}
        return res

    ex = S.BatchExecutor(cap, F.make_params(precision=F.FT_FP32C), device=local)
    S.serve(requests(rates[0])[:2], ex, cap, realtime=False)          # warm-up
    for rate in rates:
        for pol in policies:
            torch.cuda.synchronize()
            outs, st = S.serve(requests(rate), ex, cap, realtime=True, policy=pol)
            st["by_class"] = by_class(outs)
            out["rates"].setdefault(str(int(rate)), {})[pol] = st
    ex.close()
    seq = S.SequentialExecutor(F.make_params(precision=F.FT_FP64), device=local)
    _, st = S.serve_sequential(requests(rates[0]), seq, realtime=True)
    st["rate"] = rates[0]
    out["plain_fp64_one_at_a_time"] = st
    return out


def run_reference(a):
    """The oracle as the reference arm: K timed steps of the five steps over the
    workload.  A step is a full pass over every front when one fits the per-step
    share of a two-minute budget; otherwise PPIC on a random sample of cells
    plus the other four steps' time (measured once, whole fronts) pro-rated per
    cell."""
    import numpy as np
    ws, rank, _ = dist()
    if rank != 0:
        return
    import oracle
    fronts = workload()
    oracle.set_threads(os.cpu_count() or 1)
    # one untimed full pass: cell counts and the time of each step per front
    full = [oracle_pass(w) for w in fronts]
    M = sum(m for m, _ in full)
    t_full = sum(sum(t.values()) for _, t in full)
    t_rest = sum(t[k] for _, t in full for k in ("bin", "alpha", "csf", "interp"))
    budget = 120.0 / max(1, a.steps + a.warmup)
    gen = np.random.Generator(np.random.PCG64(7))
    whole = t_full <= budget
    if whole:
        def step():
            t0 = time.perf_counter()
            n = sum(oracle_pass(w)[0] for w in fronts)
            return n, time.perf_counter() - t0
        sample = f"per step: the five steps over the whole workload ({M} interfacial cells)"
    else:
        # PPIC on S cells of the first front (its cells are the larger share)
        w = fronts[0]
        cells0 = np.unique(oracle.bin_pairs(w["verts"], w["tris"], w["grid"])[0])
        per_cell_ppic = full[0][1]["ppic"] / full[0][0]
        S = int(max(50, min(len(cells0), 0.8 * budget / per_cell_ppic)))

        def step():
            sel = np.sort(gen.choice(cells0, S, replace=False))
            t0 = time.perf_counter()
            oracle.ppic(w["verts"], w["tris"], w["grid"], sel)
            return S, time.perf_counter() - t0 + t_rest * S / M
        sample = (f"per step: PPIC on {S} random cells of {w['name']} + binning, alpha, CSF and interpolation of "
                  f"the whole workload pro-rated per cell ({t_rest:.2f} s for {M} cells)")
    for _ in range(a.warmup):
        step()
    n_tot, tot = 0, 0.0
    for _ in range(a.steps):
        n, dt = step()
        n_tot += n
        tot += dt
    value = n_tot / tot
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "interfacial cells/s",
            "n_gpus": ws, "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(1e3 * tot / a.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "rough icosphere s6 R0.2 + ellipsoid (0.3,0.2,0.15), 128^3 grid, 81,920 tris each"},
            "cpu_baseline": {"value": round(value, 1), "unit": "interfacial cells/s", "cores": oracle.get_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 1), "unit": "interfacial cells/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.profile_batch > 0:
        profile_batch(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
