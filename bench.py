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
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "interfacial cells/s for alpha+kappa (full five-step hot path per step)"
FLOPS_PER_FIT_PAIR = 130.0   # per (cell, fragment-in-support) pair of the volume fit
FLOPS_PER_FIT_SOLVE = 150.0  # per cell: the 6x6 solve
FP64_PEAK_TFLOPS = 1.25      # GB300 nominal float64 (profiling recipe table)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # 152 SMs x 128 FMA/clk x 2 flops x 2.07 GHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "fp32c"], default="fp64")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
        self.out = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")
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


def cpu_baseline(fronts, budget_s=20.0):
    """The oracle (FP64 C, all host cores) on a bounded sample of the first front:
    binning and alpha of the whole front, PPIC on a sample of its cells; the
    per-cell time is scaled to cells/s."""
    import numpy as np
    import oracle
    w = fronts[0]
    g = w["grid"]
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    t0 = time.perf_counter()
    keys, _, _ = oracle.bin_pairs(w["verts"], w["tris"], g)
    t1 = time.perf_counter()
    oracle.alpha(w["verts"], w["tris"], g)
    t2 = time.perf_counter()
    cells = np.unique(keys)
    M = len(cells)
    S = min(M, 1000)
    sel = cells[np.linspace(0, M - 1, S).astype(np.int64)]
    t3 = time.perf_counter()
    oracle.ppic(w["verts"], w["tris"], g, sel)
    t4 = time.perf_counter()
    per_cell = (t1 - t0 + t2 - t1) / M + (t4 - t3) / S
    return dict(value=1.0 / per_cell, unit="interfacial cells/s", cores=oracle.get_threads(), kind="oracle",
                sample=f"{w['name']}: bin + alpha of the whole front ({M} cells, {t2 - t0:.2f} s) + PPIC on "
                       f"{S} of its cells ({t4 - t3:.2f} s); cells/s = 1 / per-cell time"), (t0, t1, t2, M, S)


def run_ours(a):
    import numpy as np
    import torch
    from paper_2505_06932_gb300 import _front as F

    ws, rank, local = dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fronts = workload()
    prec = F.FT_FP64 if a.precision == "fp64" else F.FT_FP32C
    prm = F.make_params(precision=prec)
    dfr, fcs = [], []
    for w in fronts:
        v = torch.from_numpy(w["verts"]).to(dev)
        t = torch.from_numpy(w["tris"]).to(dev)
        fa = [torch.from_numpy(f).to(dev) for f in w["faces"]]
        dfr.append((v, t, fa))
        fcs.append(F.FrontCoupling(w["grid"], t.shape[0], v.shape[0], params=prm, device=local))
    stream = torch.cuda.current_stream()

    def step(ppic_ev=None):
        for (v, t, fa), fc in zip(dfr, fcs):
            F.front_bin(fc.ws, v, t, prm)
            F.front_volume_fraction(fc.ws, fc.alpha)
            if ppic_ev is not None:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            F.front_curvature_ppic(fc.ws, prm, fc.cell_keys, fc.kappa, fc.normal, fc.coeffs, fc.fit_status)
            if ppic_ev is not None:
                e1.record(stream)
                ppic_ev.append((e0, e1))
            F.front_csf_force(fc.ws, prm, fc.alpha, fc.kappa, fc.normal, fc.force)
            F.front_interp_velocity(fc.grid, fa[0], fa[1], fa[2], v, fc.vel[:v.shape[0]])

    for _ in range(max(3, a.warmup)):
        step()
    torch.cuda.synchronize()
    counts = [fc.ws.counts() for fc in fcs]
    status = [fc.ws.status() for fc in fcs]
    if any(status):
        raise RuntimeError(f"device status after warm-up: {[F.status_names(s) for s in status]}")
    cells_per_step = sum(c["M"] for c in counts)
    fit_pairs = [c["fit_pairs"] for c in counts]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MB > L2

    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    launches0 = F.launch_count()
    evs, ppic_ev = [], []
    for _ in range(a.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(ppic_ev)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    barrier(ws)
    launches = F.launch_count() - launches0
    clk = clocks.stop()
    total_ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    ppic_ms = [e0.elapsed_time(e1) for e0, e1 in ppic_ev]
    tmax = allmax(ws, total_ms)
    all_cells = allsum(ws, cells_per_step * a.steps)
    value = all_cells / (tmax * 1e-3)

    # roofline of the dominant kernel (PPIC), ALU-bound
    nf = len(fcs)
    flops = [FLOPS_PER_FIT_PAIR * fit_pairs[i] + FLOPS_PER_FIT_SOLVE * counts[i]["M"] for i in range(nf)]
    ach = sum(flops[i % nf] for i in range(len(ppic_ms))) / (sum(ppic_ms) * 1e-3) / 1e12
    peak = FP64_PEAK_TFLOPS if prec == F.FT_FP64 else FP32_PEAK_TFLOPS
    probe = None
    try:
        probe = F.probe_fma_rate(0 if prec == F.FT_FP64 else 1, local) / 1e12
    except Exception:
        probe = None
    roof = {"kernel": "k_ppic", "bound": "alu", "achieved": round(ach, 4), "peak": peak, "unit": "TFLOP/s",
            "frac": round(ach / peak, 4), "traffic": None,
            "peak_source": "nominal FP64 1.25 TFLOP/s (recipe table)" if prec == F.FT_FP64
            else "152 SM x 128 FP32 FMA/clk x 2 x 2.07 GHz",
            "probe_measured_peak": round(probe, 4) if probe else None,
            "share_of_step": round(sum(ppic_ms) / total_ms, 4),
            "flops_model": f"{FLOPS_PER_FIT_PAIR:.0f} per fit pair + {FLOPS_PER_FIT_SOLVE:.0f} per cell"}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    hin = []
    for w in fronts:
        hv = torch.from_numpy(w["verts"]).pin_memory()
        ht = torch.from_numpy(w["tris"]).pin_memory()
        hf = [torch.from_numpy(f).pin_memory() for f in w["faces"]]
        hin.append((hv, ht, hf))
    hout = []
    h2d = d2h = 0
    for (hv, ht, hf), fc, c in zip(hin, fcs, counts):
        M = c["M"]
        outs = dict(alpha=torch.empty(fc.alpha.shape, dtype=torch.float64).pin_memory(),
                    force=torch.empty(fc.force.shape, dtype=torch.float64).pin_memory(),
                    kappa=torch.empty(M, dtype=torch.float64).pin_memory(),
                    normal=torch.empty((M, 3), dtype=torch.float64).pin_memory(),
                    vel=torch.empty((hv.shape[0], 3), dtype=torch.float64).pin_memory())
        hout.append(outs)
        h2d += hv.numel() * 8 + ht.numel() * 4 + sum(f.numel() * 8 for f in hf)
        d2h += sum(o.numel() * o.element_size() for o in outs.values())
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(a.e2e_steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for (hv, ht, hf), (v, t, fa), fc, o, c in zip(hin, dfr, fcs, hout, counts):
            v.copy_(hv, non_blocking=True)
            t.copy_(ht, non_blocking=True)
            for dst, src in zip(fa, hf):
                dst.copy_(src, non_blocking=True)
            F.front_bin(fc.ws, v, t, prm)
            F.front_volume_fraction(fc.ws, fc.alpha)
            F.front_curvature_ppic(fc.ws, prm, fc.cell_keys, fc.kappa, fc.normal, fc.coeffs, fc.fit_status)
            F.front_csf_force(fc.ws, prm, fc.alpha, fc.kappa, fc.normal, fc.force)
            F.front_interp_velocity(fc.grid, fa[0], fa[1], fa[2], v, fc.vel[:v.shape[0]])
            M = c["M"]
            o["alpha"].copy_(fc.alpha, non_blocking=True)
            o["force"].copy_(fc.force, non_blocking=True)
            o["kappa"].copy_(fc.kappa[:M], non_blocking=True)
            o["normal"].copy_(fc.normal[:M], non_blocking=True)
            o["vel"].copy_(fc.vel[:v.shape[0]], non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_max = allmax(ws, e2e_ms)
    e2e_value = allsum(ws, cells_per_step * a.e2e_steps) / (e2e_max * 1e-3)

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "interfacial cells/s", "n_gpus": ws,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(tmax / a.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == F.FT_FP64 else "f32+f64",
        "data": "synthetic (seeded icosphere fronts, solid-body face velocities)",
        "config": {"workload": "rough icosphere s6 R0.2 + ellipsoid (0.3,0.2,0.15), 128^3 grid, 81,920 tris each",
                   "fronts": [w["name"] for w in fronts], "cells_per_step": cells_per_step,
                   "pairs_per_step": sum(c["P"] for c in counts), "fit_pairs_per_step": sum(fit_pairs),
                   "precision": a.precision, "l2": "flushed (512 MB write) before every timed step",
                   "parallelism": f"replicas x{ws}"},
        "roofline": roof,
        "e2e": {"value": round(e2e_value, 1), "unit": "interfacial cells/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": a.e2e_steps},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        cb, _ = cpu_baseline(fronts)
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    for fc in fcs:
        fc.ws.close()


def run_reference(a):
    """The oracle as the reference arm: K timed steps, each the oracle's PPIC on
    a sample of cells plus the pro-rated binning and alpha of the whole front."""
    import numpy as np
    ws, rank, _ = dist()
    if rank != 0:
        return
    import oracle
    fronts = workload()
    w = fronts[0]
    g = w["grid"]
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    t0 = time.perf_counter()
    keys, _, _ = oracle.bin_pairs(w["verts"], w["tris"], g)
    oracle.alpha(w["verts"], w["tris"], g)
    t_ba = time.perf_counter() - t0
    cells = np.unique(keys)
    M = len(cells)
    budget = 120.0 / max(1, a.steps + a.warmup)
    S = int(max(50, min(M, 400 * budget)))
    gen = np.random.Generator(np.random.PCG64(7))
    for _ in range(a.warmup):
        oracle.ppic(w["verts"], w["tris"], g, np.sort(gen.choice(cells, S, replace=False)))
    tot = 0.0
    for _ in range(a.steps):
        sel = np.sort(gen.choice(cells, S, replace=False))
        t1 = time.perf_counter()
        oracle.ppic(w["verts"], w["tris"], g, sel)
        tot += time.perf_counter() - t1 + t_ba * S / M
    value = S * a.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "interfacial cells/s",
            "n_gpus": ws, "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(1e3 * tot / a.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "rough icosphere s6 R0.2 + ellipsoid (0.3,0.2,0.15), 128^3 grid, 81,920 tris each"},
            "cpu_baseline": {"value": round(value, 1), "unit": "interfacial cells/s", "cores": oracle.get_threads(),
                             "kind": "oracle",
                             "sample": f"per step: PPIC on {S} random cells of {w['name']} + binning and alpha of the "
                                       f"whole front pro-rated per cell ({t_ba:.2f} s for {M} cells)"},
            "e2e": {"value": round(value, 1), "unit": "interfacial cells/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
