#!/usr/bin/env python
"""Benchmark of the hyperbolic self-gravity hot path (arXiv 1602.05700) on GB300.

Workload (one "step" = the gravity work of one hydro step, Sec. 2): a 512^3 grid on the unit cube with the
time-dependent source of two Gaussian blobs (sigma 0.05, mass 1 each) orbiting at radius 0.15 with omega = 2 pi;
c_h = 10 x the blob speed; hydro step 0.5 h / v_max split into 20 wave sub-steps (rho frozen, Sec. 2); Robin outer
boundary.  Per step: hg_set_density (rho of that hydro time, resident in HBM), 20 sub-steps, -grad phi.

Metric: Gcell-updates/s = 512^3 x 20 x steps / time (whole job, all ranks), FP32 with compensated increments;
the FP64 reference mode is measured on the same workload and reported beside it.  `roofline` is the sub-step
kernel's algorithmic bytes per launch / its CUDA-event duration inside the timed region, against the measured
copy bandwidth.  `e2e` repeats the measurement through the public API (hg_io_step) with each step's density
coming from pinned host memory and the acceleration copied back to pinned host memory every step.
`--impl reference` times the CPU oracle instead.

Multi-GPU: the path has no exchange step in this build (one independent grid per rank), so N ranks run N
independent problems (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import collections
import csv
import io
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SUB = 20
BYTES_PER_CELL = {"f32k": 24, "f64": 32}  # algorithmic HBM bytes of one sub-step: f32k read hi 4, lo code 2, dlt 4, s 4
#                                          and write hi 4, lo 2, dlt 4; f64 read phi^n, phi^{n-1}, s, write phi^{n+1}
DP_OPS_PER_CELL = 15                      # FP64 operations of the f64 update as written (11 for L, 4 more); the
                                          # sweep runs between 3 and 15 of them on the FP64 pipe (cell.cuh)
RELAX_SUBSTEPS = 2000                     # untimed sub-steps before the FP64 leg's relaxed-field measurement
FP64_NOMINAL_TFLOPS = 1.25                # GB300 FP64 (FMA = 2 flops): 0.625 T instructions/s; used only if the
#                                          measured rate (hg_probe_rate) is unavailable
FALLBACK_HBM_GBS = 6800.0


def workload(n):
    h = 1.0 / n
    v_max = 0.15 * 2.0 * math.pi
    c = 10.0 * v_max
    dt_hyd = 0.5 * h / v_max
    return dict(n=n, h=h, v_max=v_max, c=c, dt_hyd=dt_hyd, dt=dt_hyd / N_SUB, origin=(-0.5, -0.5, -0.5), G=1.0)


def workload_name(n):
    return (f"{n}^3 unit cube, two orbiting Gaussian blobs (sigma 0.05, mass 1, r 0.15, omega 2pi), Robin boundary, "
            f"c_h = 10 v_max, {N_SUB} sub-steps per hydro step; per step set_density + {N_SUB} sub-steps + -grad phi")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def source_hash(files=None):
    """sha256 over CUDA sources (all of csrc/, or the given file names), to tell whether a committed ncu figure was
    taken on the current kernels."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1602_05700_gb300", "csrc")
    for f in sorted(files or os.listdir(csrc)):
        if f.endswith((".cu", ".cuh")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()


IO_SETS = 4  # host buffer sets of the end-to-end measurement (steps in flight + 1)


def kernel_instructions(kernel, cells):
    """Warp instructions per launch (scaled to `cells`) from profiles/traffic.json, if counted on the current
    sources of that kernel."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    e = json.load(open(p)).get("kernels", {}).get(kernel)
    if not e or "warp_inst_per_launch" not in e or e.get("sources_sha256") != source_hash(e.get("sources")):
        return None
    return e["warp_inst_per_launch"] * cells / e["cells"]


# instruction-issue limit of the GPU: 152 SMs x 4 schedulers x one warp instruction per cycle at 2.07 GHz
ISSUE_PEAK_GWIPS = 152 * 4 * 2.07


def stencil_traffic(kernel, n):
    """DRAM bytes per launch (scaled to n^3 cells) from profiles/traffic.json, if taken on the current sources of
    that kernel (the entry lists the files it is built from and their sha256)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    e = json.load(open(p)).get("kernels", {}).get(kernel)
    if not e or e.get("sources_sha256") != source_hash(e.get("sources")):
        return None
    return round(e["dram_bytes_per_launch"] * (n ** 3) / e["cells"])


class Clocks:
    """nvidia-smi samples during the timed region (SM clock, limits, throttle reasons)."""

    def __init__(self, index):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                try:
                    rows.append((float(f[1]), float(f[2]), float(f[3]), f[5:9]))
                except ValueError:
                    pass
        os.unlink(self.path)
        if not rows:
            return None
        load = [r for r in rows if r[2] > 200.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in load for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_1602_05700_gb300 as hg
    from paper_1602_05700_gb300 import inputs as I

    from paper_1602_05700_gb300 import multi

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    multi.init("nccl", dev)
    W = workload(args.n)
    n = W["n"]
    steps, warm = args.steps, args.warmup
    # densities of consecutive hydro steps, generated before timing and resident in HBM (f32, 0.5 GB each at 512^3)
    t_off = rank * 0.25  # each rank its own phase of the orbit: independent problems
    rhos = [I.blob_density_torch(n, I.orbit_blobs(t_off + s * W["dt_hyd"]), dev, torch.float32)
            for s in range(warm + steps)]
    hbm_peak, peak_kind = peaks()
    # the FP64 pipe's measured rate on this GPU (independent FP64 FMA chains, best of five event-timed launches)
    try:
        fp64_peak = hg.probe_rate("f64")["instr_per_s"] / 1e9
        fp64_kind = "measured FP64 FMA rate (hg_probe_rate: independent DFMA chains, best of 5 event-timed launches)"
    except Exception:  # pragma: no cover
        fp64_peak, fp64_kind = FP64_NOMINAL_TFLOPS * 1e3 / 2, "nominal FP64 rate (1.25 TFLOP/s, FMA = 2)"

    def barrier():
        multi.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return multi.max_over_ranks(x, dev)

    def measure(prec, depth, k_steps, profile_region=False, relax=0):
        g = hg.Grid(n, n, n, W["h"], W["origin"], W["c"], W["G"], W["dt"], prec, "robin")
        if depth > 1:
            g.set_temporal_depth(depth)
        out = [torch.empty((n, n, n), device=dev, dtype=torch.float32) for _ in range(3)]
        if relax:  # untimed sub-steps at the first density: phi relaxed from 0 to the field of the blobs
            g.set_density(rhos[0])
            g.step(relax)

        def one(s):
            g.set_density(rhos[s % len(rhos)])
            g.step(N_SUB)
            g.accel(out=out)

        for s in range(warm):
            one(s)
        barrier()
        g.profile(True)
        g.profile_read()
        launches0 = g.profile_read()[2]
        clocks = Clocks(local_rank) if rank == 0 else None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if profile_region:
            torch.cuda.cudart().cudaProfilerStart()  # lets an external profiler capture just this region
        e0.record()
        for s in range(warm, warm + k_steps):
            one(s)
        e1.record()
        barrier()
        if profile_region:
            torch.cuda.cudart().cudaProfilerStop()
        ck = clocks.stop() if clocks else None
        ms = max_over_ranks(e0.elapsed_time(e1))
        kern_ms, kern_n, launches1 = g.profile_read()
        g.profile(False)
        st = g.stats(check=False)
        g.free()
        return dict(ms=ms, kern_ms=kern_ms, kern_n=kern_n, launches=launches1 - launches0, clocks=ck, stats=st,
                    depth=depth, steps=k_steps, prec=prec)

    cells = n ** 3

    def rate(r):
        return cells * N_SUB * r["steps"] * world / (r["ms"] * 1e-3) / 1e9

    def f64_roofline(avg):
        # HBM line of the FP64 sweep (32 B per cell); its FP64-pipe work depends on the field (between 3 and 15 FP64
        # instructions per cell, integer instructions for the rest), so the FP64 rate is given beside it at 15 per
        # cell as the upper bound of the pipe's share
        hbm = BYTES_PER_CELL["f64"] * cells / (avg * 1e-3) / 1e9
        dp15 = DP_OPS_PER_CELL * cells / (avg * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": round(hbm, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(hbm / hbm_peak, 4), "peak_kind": peak_kind,
                "traffic": stencil_traffic("k_step_f64", n), "kernel": "k_step_f64", "avg_launch_ms": round(avg, 5),
                "fp64_ops_at_15_per_cell_g_per_s": round(dp15, 1), "fp64_peak_g_per_s": round(fp64_peak, 1),
                "fp64_peak_kind": fp64_kind}

    def roofline(r):
        avg = r["kern_ms"] / max(r["kern_n"], 1)
        if r["prec"] == "f64":
            return f64_roofline(avg)
        subs = N_SUB * r["steps"] / max(r["kern_n"], 1)  # sub-steps per launch (the temporal depth)
        alg = BYTES_PER_CELL["f32k"] * cells  # one read of the state and one write per launch
        ach = alg / (avg * 1e-3) / 1e9
        kname = {1: "k_step_f32k_tma", 2: "k_temporal2_tma"}.get(r["depth"], f"k_temporal_f32k<{r['depth']}>")
        line = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(ach / hbm_peak, 4), "peak_kind": f"{peak_kind} copy bandwidth",
                "traffic": stencil_traffic(kname, n), "kernel": kname, "alg_bytes_per_launch": alg,
                "substeps_per_launch": round(subs, 3), "avg_launch_ms": round(avg, 5),
                "effective_single_sweep_gbs": round(ach * subs, 1),
                "effective_frac": round(ach * subs / hbm_peak, 4)}
        winst = kernel_instructions(kname, cells) if r["depth"] > 1 else None
        if winst:
            # fused sub-steps move half the bytes per sub-step and are bound by instruction issue instead: the
            # warp instructions of one launch (ncu count of the current sources, scaled to this grid) per second
            # against the issue limit (152 SMs x 4 schedulers x one warp instruction per cycle at 2.07 GHz)
            gwips = winst / (avg * 1e-3) / 1e9
            line.update({"bound": "alu", "achieved": round(gwips, 1), "peak": round(ISSUE_PEAK_GWIPS, 1),
                         "unit": "G warp-instr/s", "frac": round(gwips / ISSUE_PEAK_GWIPS, 4),
                         "peak_kind": "instruction issue limit (152 SMs x 4 schedulers x 2.07 GHz, nominal)",
                         "warp_inst_per_launch": round(winst), "hbm_achieved_gbs": round(ach, 1),
                         "hbm_frac": round(ach / hbm_peak, 4)})
        return line

    # temporal depth: a short sweep picks the fastest depth for the headline measurement
    if args.depth > 0 or args.prec == "f64":
        best = args.depth
        sweep = None
    else:
        sweep = {}
        for d in range(1, 9):
            sweep[d] = round(rate(measure("f32k", d, 3)), 2)
        best = max(sweep, key=sweep.get)
    if args.prec == "f64":  # the FP64 mode as the profiled headline (e.g. to capture its kernel alone)
        best, sweep = 1, None
    res = measure(args.prec, best, steps, profile_region=True)
    value = rate(res)
    line = {
        "metric": "Gcell-updates/s per wave sub-step (512^3, FP32 compensated; FP64 beside it)",
        "value": round(value, 3), "unit": "Gcell-updates/s", "n_gpus": world, "steps": steps, "warmup": warm,
        "ms_per_step": round(res["ms"] / steps, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.prec == "f32k" else "f64", "data": "synthetic",
        "config": {"workload": workload_name(n), "grid": [n, n, n], "substeps_per_step": N_SUB,
                   "precision": "f32 compensated (Kahan)" if args.prec == "f32k" else "f64",
                   "temporal_depth": best, "depth_sweep_gcells": sweep,
                   "parallelism": f"{world} independent grids (one per GPU)",
                   "l2": (f"working set {20 * cells / 1e9:.1f} GB per grid (hi, lo codes, dlt, s)" if args.prec == "f32k"
                          else f"working set {24 * cells / 1e9:.1f} GB per grid (phi^n, phi^(n-1), s)")
                         + " >> 129 MB L2 (no flush needed)"},
        "roofline": roofline(res),
        "gpu_launches": res["launches"],
        "clocks": res["clocks"],
    }
    if best != 1:
        r1 = measure("f32k", 1, max(3, steps // 2))
        line["single_sweep"] = {"value": round(rate(r1), 3), "unit": "Gcell-updates/s", "steps": r1["steps"],
                                "roofline": roofline(r1)}
    # FP64 reference mode on the same workload
    if not args.skip_fp64 and args.prec == "f32k":
        k64 = max(2, steps // 4)
        r64 = measure("f64", 1, k64)
        v64 = cells * N_SUB * k64 * world / (r64["ms"] * 1e-3) / 1e9
        avg64 = r64["kern_ms"] / max(r64["kern_n"], 1)
        line["fp64"] = {"value": round(v64, 3), "unit": "Gcell-updates/s", "steps": k64,
                        "ms_per_step": round(r64["ms"] / k64, 4), "roofline": f64_roofline(avg64),
                        "gpu_launches": r64["launches"]}
        # the same after the field has relaxed (2000 untimed sub-steps first): smooth phi everywhere, where the
        # FP64 sweep's Laplacian runs in integers
        rr = measure("f64", 1, k64, relax=RELAX_SUBSTEPS)
        vr = cells * N_SUB * k64 * world / (rr["ms"] * 1e-3) / 1e9
        line["fp64"]["relaxed"] = {"value": round(vr, 3), "untimed_substeps_first": RELAX_SUBSTEPS,
                                   "ms_per_step": round(rr["ms"] / k64, 4),
                                   "roofline": f64_roofline(rr["kern_ms"] / max(rr["kern_n"], 1))}
    # end to end through the public API: each step's density from pinned host memory, -grad phi back to pinned
    # host memory, with the copies of one step overlapping the sub-steps of the next (hg_io_step / hg_io_wait)
    if not args.skip_e2e:
        ke, we = max(4, steps), IO_SETS  # the whole run of steps, as the device-resident measurement; the warm-up
        # uses every host buffer set once
        # a rotation of four page-locked host buffers for the density and four sets for -grad phi, as a driver with
        # three steps in flight keeps them (each buffer is rewritten only after hg_io_wait has released it): the
        # densities of this workload are analytic in time, so a step's input does not wait for the previous output
        host_rho = [rhos[s % len(rhos)].cpu().pin_memory() for s in range(IO_SETS)]
        host_acc = [[torch.empty((n, n, n), dtype=torch.float32).pin_memory() for _ in range(3)]
                    for _ in range(IO_SETS)]
        g = hg.Grid(n, n, n, W["h"], W["origin"], W["c"], W["G"], W["dt"], "f32k", "robin")
        if best > 1:
            g.set_temporal_depth(best)

        def e2e_steps(first, count):
            for s in range(first, first + count):
                g.io_step(host_rho[s % IO_SETS], N_SUB, host_acc[s % IO_SETS])
                g.io_wait(IO_SETS - 1)  # step s-3 is done: its outputs are on the host, its buffers free again
            g.io_wait(0)

        e2e_steps(0, we)
        barrier()
        t0 = time.perf_counter()
        e2e_steps(we, ke)
        barrier()
        sec = max_over_ranks(time.perf_counter() - t0)
        g.free()
        line["e2e"] = {"value": round(cells * N_SUB * ke * world / sec / 1e9, 3), "unit": "Gcell-updates/s",
                       "h2d_bytes_per_step": 4 * cells, "d2h_bytes_per_step": 12 * cells, "steps": ke,
                       "temporal_depth": best,
                       "note": "each step: its density from pinned host memory in, -grad phi (3 x f32) out to "
                               "pinned host memory; three steps in flight, so the copies overlap the neighbouring steps' "
                               "sub-steps"}
    if rank == 0 and not args.skip_cpu:
        line["cpu_baseline"] = cpu_baseline(args.n, args.cpu_substeps)
    multi.finalize()
    return line


def cpu_baseline(n, substeps):
    """The oracle as it stands on the host cores, on the same grid and source, a bounded number of sub-steps: the
    checked single-threaded build, and the OpenMP build of the same C file (the same bits) on every core."""
    import numpy as np  # noqa: F401

    import oracle as O
    from paper_1602_05700_gb300 import inputs as I

    W = workload(n)
    g = O.Grid(n, n, n, W["h"], W["origin"], W["c"], W["G"], W["dt"], O.BC_ROBIN)
    rho = I.blob_density(n, I.orbit_blobs(0.0))
    p, q = O.initial_state(g, rho)
    O.build()
    O.build(openmp=True)
    t0 = time.perf_counter()
    O.run(g, p, q, rho, substeps)
    sec1 = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    sub_all = max(substeps, substeps * cores // 2)
    O.run_all_cores(g, p, q, rho, 1, cores)  # warm-up (thread pool start)
    t0 = time.perf_counter()
    O.run_all_cores(g, p, q, rho, sub_all, cores)
    secn = time.perf_counter() - t0
    del p, q, rho
    v1 = n ** 3 * substeps / sec1 / 1e9
    vn = n ** 3 * sub_all / secn / 1e9
    return {"value": round(vn, 5), "unit": "Gcell-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{n}^3 grid, same Robin/orbiting-blob workload, {sub_all} sub-steps ({secn:.1f} s) on "
                      f"{cores} host cores (os.cpu_count()): the oracle's C file built with OpenMP over z planes, "
                      "bit-identical to the checked single-threaded build",
            "single_thread": {"value": round(v1, 5), "unit": "Gcell-updates/s", "cores": 1, "kind": "oracle",
                              "sample": f"{substeps} sub-steps ({sec1:.1f} s), the checked single-threaded C oracle "
                                        "(oracle/hg_oracle.c)"}}


def run_reference(args):
    """The CPU oracle timed as the reference arm, on every host core (the OpenMP build of the oracle's C file, which
    computes the same bits as the checked single-threaded build): each step a bounded sample (a few sub-steps of
    the workload)."""
    import numpy as np  # noqa: F401

    import oracle as O
    from paper_1602_05700_gb300 import inputs as I

    W = workload(args.n)
    n = W["n"]
    g = O.Grid(n, n, n, W["h"], W["origin"], W["c"], W["G"], W["dt"], O.BC_ROBIN)
    O.build()
    O.build(openmp=True)
    cores = os.cpu_count() or 1
    sub = args.ref_substeps
    rho = I.blob_density(n, I.orbit_blobs(0.0))
    p, q = O.initial_state(g, rho)
    for _ in range(args.warmup):
        O.run_all_cores(g, p, q, rho, 1, cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.run_all_cores(g, p, q, rho, sub, cores)
    sec = time.perf_counter() - t0
    v = n ** 3 * sub * args.steps / sec / 1e9
    sample = (f"{n}^3 grid, same Robin/orbiting-blob workload, {sub} sub-step(s) per step (a bounded sample of the "
              f"{N_SUB}-sub-step hydro step), the C oracle built with OpenMP over z planes on {cores} host cores")
    return {"impl": "reference", "metric": "Gcell-updates/s per wave sub-step (512^3, FP32 compensated; FP64 beside it)",
            "value": round(v, 5), "unit": "Gcell-updates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sec / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(n), "grid": [n, n, n], "substeps_per_step": N_SUB,
                       "precision": "f64 (the oracle)", "parallelism": f"1 process, {cores} host cores"},
            "cpu_baseline": {"value": round(v, 5), "unit": "Gcell-updates/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 5), "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---- the other workloads (the default run above is the headline) -----------------------------------------------------

def run_precision(args):
    """Config 2: 256^3 sphere + 8 blobs (seed 1), multipole boundary l <= 4, 2000 sub-steps in FP32-compensated and
    FP64 on the GPU against the FP64 CPU oracle (which takes minutes on one core at this size)."""
    import numpy as np
    import torch

    import oracle as O
    import paper_1602_05700_gb300 as hg
    from paper_1602_05700_gb300 import inputs as I

    n, T = args.n, args.substeps
    rho = I.sphere_density(n) + I.blob_density(n, I.draw_blobs(8, 1))
    out = {"workload": f"{n}^3 sphere + 8 blobs, multipole Dirichlet l <= 4, {T} sub-steps, CFL 0.5", "results": {}}
    phis = {}
    for prec in ("f32k", "f64"):
        g = hg.Grid.unit_cube(n, 1.0, 1.0, 0.5, prec, "multipole", lmax=4)
        g.set_density(torch.from_numpy(rho).cuda())
        g.step(3)
        g.set_phi(torch.zeros((n, n, n), dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.step(T)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        phis[prec] = g.phi(torch.float64, "cpu")
        out["results"][prec] = {"gcell_updates_per_s": round(n ** 3 * T / (ms * 1e-3) / 1e9, 2), "ms": round(ms, 1)}
        g.free()
    og = O.unit_cube(n, 1.0, 1.0, 0.5, O.BC_DIRICHLET)
    p, q = O.initial_state(og, rho, lmax=4)
    t0 = time.perf_counter()
    O.run(og, p, q, rho, T)
    out["oracle_seconds"] = round(time.perf_counter() - t0, 1)
    ref = p[1:-1, 1:-1, 1:-1]
    for prec, phi in phis.items():
        out["results"][prec]["rel_l2_vs_oracle"] = float(np.linalg.norm(phi - ref) / np.linalg.norm(ref))
        out["results"][prec]["rel_linf_vs_oracle"] = float(np.abs(phi - ref).max() / np.abs(ref).max())
    return out


def run_batch(args):
    """Config 4: 48 grids, sides uniform in {64, 96, 128, 160, 192} (seed 7), 1-6 blobs each, FP32-compensated for
    even and FP64 for odd indices, Robin boundary, 500 sub-steps: one graph launch of batched sub-steps against
    sequential per-grid launches (same work, same results)."""
    import torch

    import paper_1602_05700_gb300 as hg
    from paper_1602_05700_gb300 import inputs as I

    sides = I.batch_sides(48, 7)
    nblobs = I.batch_blob_counts(48, 7)
    T = args.substeps

    def grids():
        gs = []
        for i, (n, nb) in enumerate(zip(sides, nblobs)):
            n = int(n)
            g = hg.Grid.unit_cube(n, 1.0, 1.0, 0.5, "f32k" if i % 2 == 0 else "f64", "robin")
            g.set_density(I.blob_density_torch(n, I.draw_blobs(int(nb), 700 + i), "cuda", torch.float64))
            gs.append(g)
        return gs

    cells = int(sum(int(n) ** 3 for n in sides))
    res = {"workload": f"48 grids, sides {sorted(set(int(s) for s in sides))} (seed 7), mixed f32k/f64, Robin, "
                       f"{T} sub-steps", "cells": cells}
    gs = grids()
    b = hg.Batch(gs)
    b.step(8)  # autotune + graph for 8
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.step(T)
    e1.record()
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1)
    res["batched_graph"] = {"ms": round(ms_b, 2), "gcell_updates_per_s": round(cells * T / (ms_b * 1e-3) / 1e9, 2),
                            **b.info()}
    gs2 = grids()
    for g in gs2:
        g.step(2)
    torch.cuda.synchronize()
    e0.record()
    for g in gs2:
        g.step(T)
    e1.record()
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    res["sequential_per_grid"] = {"ms": round(ms_s, 2), "gcell_updates_per_s": round(cells * T / (ms_s * 1e-3) / 1e9, 2)}
    res["speedup"] = round(ms_s / ms_b, 3)
    # the same batch once the fields have relaxed (RELAX_SUBSTEPS untimed sub-steps first): smooth phi, where the
    # FP64 grids' Laplacian runs in integers
    b.step(RELAX_SUBSTEPS)
    torch.cuda.synchronize()
    e0.record()
    b.step(T)
    e1.record()
    torch.cuda.synchronize()
    ms_r = e0.elapsed_time(e1)
    res["batched_graph_relaxed"] = {"ms": round(ms_r, 2), "untimed_substeps_first": RELAX_SUBSTEPS,
                                    "gcell_updates_per_s": round(cells * T / (ms_r * 1e-3) / 1e9, 2)}
    f32 = [i for i in range(48) if i % 2 == 0]
    f32_cells = int(sum(int(sides[i]) ** 3 for i in f32))
    f64_cells = cells - f32_cells
    res["f32k_cells"] = f32_cells
    for g in gs + gs2:
        g.free()
    b.free()

    # each precision alone in a batch of its own grids, and the floor of the mixed batch: the FP64 grids at the FP64
    # rate of a large grid (512^3, 128-cell tile rows, the pipe-bound rate) and the float grids at theirs
    def batch_alone(idx):
        gsub = []
        for i, g in enumerate(grids()):
            if i in idx:
                gsub.append(g)
            else:
                g.free()
        bb = hg.Batch(gsub)
        bb.step(8)
        torch.cuda.synchronize()
        e0.record()
        bb.step(T)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        info = bb.info()
        bb.free()
        for g in gsub:
            g.free()
        return ms, info

    ms32, info32 = batch_alone(set(f32))
    ms64, info64 = batch_alone(set(range(48)) - set(f32))
    hbm_peak, _ = peaks()
    res["f32k_only_batch"] = {"ms": round(ms32, 2), "gcell_updates_per_s": round(f32_cells * T / (ms32 * 1e-3) / 1e9, 2),
                              "single_sweep_roofline_gcells": round(hbm_peak / BYTES_PER_CELL["f32k"], 1), **info32}
    res["f64_only_batch"] = {"ms": round(ms64, 2), "gcell_updates_per_s": round(f64_cells * T / (ms64 * 1e-3) / 1e9, 2),
                             **info64}
    res["mixed_floor_ms"] = {"f64_alone_plus_f32k_alone": round(ms64 + ms32, 2), "f64_alone": round(ms64, 2),
                             "note": "overlapping the HBM-bound float blocks with the FP64-bound ones can hide the "
                                     "float part; the FP64 part alone is the floor"}
    return res


def run_adjoint(args):
    """Config 5: 128^3, 4 blobs (seed 3), T = 400, 64 probes in |x| < 0.4 (seed 11), target from the seed-4 density,
    L = sum (phi^T(x_p) - target)^2; dL/drho by the adjoint (no checkpoints, and checkpointed every K), checked against
    central differences on 32 random cells; time and memory against storing the whole trajectory."""
    import numpy as np
    import torch

    import paper_1602_05700_gb300 as hg
    from paper_1602_05700_gb300 import autograd as HA
    from paper_1602_05700_gb300 import inputs as I

    n, T = args.n, args.substeps
    out = {"workload": f"{n}^3, 4 blobs seed 3, T = {T}, 64 probes", "results": {}}
    for prec in ("f64", "f32k"):
        grid = hg.Grid.unit_cube(n, 1.0, 1.0, 0.5, prec, "robin")
        rho = I.blob_density_torch(n, I.draw_blobs(4, 3), "cuda", torch.float64)
        rho_t = I.blob_density_torch(n, I.draw_blobs(4, 4), "cuda", torch.float64)
        idx, w = HA.trilinear_probe_weights(grid, torch.from_numpy(I.probes(64, 11)))
        with torch.no_grad():
            target = (HA.potential(rho_t, grid, T).reshape(-1)[idx] * w).sum(1)

        def step_loss(m, phi):
            return (((phi.reshape(-1)[idx] * w).sum(1) - target) ** 2).sum()

        def loss_plain(r):
            return step_loss(T, HA.potential(r, grid, T))

        r = {}
        for name, K in [("no_checkpoints", None), ("K10", 10), ("K20", 20), ("K50", 50)]:
            for rep in range(2):  # the first pass pays one-time costs (shadow state, autograd set-up); time the second
                rr = rho.clone().requires_grad_(True)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if K is None:
                    L = loss_plain(rr)
                else:
                    L = HA.trajectory_loss(rr, grid, T, [T], step_loss, checkpoint_every=K)
                L.backward()
                torch.cuda.synchronize()
                sec = time.perf_counter() - t0
            mem = (grid.state_bytes() * int(np.ceil(T / K))) if K else 0
            r[name] = {"forward_backward_s": round(sec, 4), "saved_state_bytes": mem}
            if K is None:
                grad = rr.grad.detach().cpu().numpy()
            else:
                g2 = rr.grad.detach().cpu().numpy()
                r[name]["max_rel_diff_vs_no_checkpoints"] = float(np.abs(g2 - grad).max() / np.abs(grad).max())
        rng = np.random.default_rng(17)
        cells = [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(32)]
        errs = []
        eps = 1e-2
        for c in cells:
            with torch.no_grad():
                rp = rho.clone()
                rp[c] += eps
                rm = rho.clone()
                rm[c] -= eps
                fd = (loss_plain(rp) - loss_plain(rm)).item() / (2 * eps)
            errs.append(abs(fd - grad[c]) / np.abs(grad).max())
        r["fd_32_cells_max_err_rel_to_max_grad"] = float(max(errs))
        r["full_trajectory_bytes"] = T * n ** 3 * 8
        out["results"][prec] = r
        grid.free()
    return out


def poisson_periodic(rho, h, G=1.0):
    """The discrete periodic Poisson solution of Lap_h phi = 4 pi G (rho - mean rho) for the 7-point Laplacian (its
    Fourier symbol), zero mean -- the fixed point the sub-steps relax to, used as the reference of --config lag."""
    import numpy as np

    nz, ny, nx = rho.shape
    lam = 0.0
    for ax, n in ((0, nz), (1, ny), (2, nx)):
        shape = [1, 1, 1]
        shape[ax] = n
        lam = lam + (2.0 / (h * h)) * (np.cos(2.0 * np.pi * np.fft.fftfreq(n)).reshape(shape) - 1.0)
    f = np.fft.fftn(4.0 * np.pi * G * (rho - rho.mean()))
    lam = np.broadcast_to(lam, f.shape).copy()
    lam[0, 0, 0] = 1.0
    f /= lam
    f[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(f))


def blob_potential(blobs, x, y, z, G=1.0):
    """Free-space potential of Gaussian blobs (rows of (cx, cy, cz, sigma, peak)): -G M erf(r / (sqrt(2) sigma)) / r
    with M = peak (2 pi)^(3/2) sigma^3 -- the continuum solution, used as the boundary data of --config domain."""
    import numpy as np
    from scipy.special import erf

    phi = 0.0
    for cx, cy, cz, sg, a in blobs:
        m = a * (2.0 * np.pi) ** 1.5 * sg ** 3
        r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2)
        phi = phi - G * m * erf(r / (np.sqrt(2.0) * sg)) / r
    return phi


def poisson_dirichlet(rho, ghosts, h, G=1.0):
    """The discrete Poisson solution Lap_h phi = 4 pi G rho on the interior with the given ghost values (an array of
    the ghosted shape; only the face ghosts are used), by the sine transform that diagonalises the 7-point Laplacian
    with Dirichlet data one cell outside the interior."""
    import numpy as np
    from scipy.fft import dstn, idstn

    nz, ny, nx = rho.shape
    f = 4.0 * np.pi * G * rho.astype(np.float64)
    f[:, :, 0] -= ghosts[1:-1, 1:-1, 0] / h ** 2
    f[:, :, -1] -= ghosts[1:-1, 1:-1, -1] / h ** 2
    f[:, 0, :] -= ghosts[1:-1, 0, 1:-1] / h ** 2
    f[:, -1, :] -= ghosts[1:-1, -1, 1:-1] / h ** 2
    f[0, :, :] -= ghosts[0, 1:-1, 1:-1] / h ** 2
    f[-1, :, :] -= ghosts[-1, 1:-1, 1:-1] / h ** 2
    lam = 0.0
    for ax, n in ((0, nz), (1, ny), (2, nx)):
        shape = [1, 1, 1]
        shape[ax] = n
        lam = lam + (2.0 / h ** 2) * (np.cos(np.pi * np.arange(1, n + 1) / (n + 1)).reshape(shape) - 1.0)
    return idstn(dstn(f, type=1) / lam, type=1)


def run_domain(args):
    """Next row f1: the boundary error against the domain size, Robin against multipole Dirichlet, k_g 5 and 20 --
    a synthetic analogue of the models aD05, aR05 .. cR20 of Sec. 4 (its Table of models).  The orbiting blobs in
    cubes of side 0.75, 1.5 and 3 at a fixed cell size h = 1/64 (48^3, 96^3, 192^3 cells); the grid starts on the
    Poisson solution; the density is re-evaluated each hydro step (0.5 h / v_max) and frozen over its 2 k_g
    sub-steps (Sec. 2).  The reference after each hydro step is the discrete Poisson solution of that density with
    the free-space potential of the blobs as its boundary data; the error is the paper's average relative error
    <dphi~> (Eq. error) over the domain."""
    import numpy as np
    import torch

    import paper_1602_05700_gb300 as hg
    from paper_1602_05700_gb300 import inputs as I

    M = args.substeps
    h, v_max = 1.0 / 64, 0.15 * 2.0 * math.pi
    dt_hyd = 0.5 * h / v_max
    out = {"workload": f"orbiting blobs, h = 1/64, domains 0.75 / 1.5 / 3 (48^3 / 96^3 / 192^3), {M} hydro steps of "
                       "0.5 h / v_max, 2 k_g sub-steps each, source frozen per hydro step",
           "metric": "<dphi~> of Eq. error against the discrete Poisson solution with free-space boundary data: "
                     "mean over the last half of the hydro steps / maximum", "results": {}}
    models = [("aD05", 0.75, "multipole", 5), ("aR05", 0.75, "robin", 5), ("bR05", 1.5, "robin", 5),
              ("cR05", 3.0, "robin", 5), ("aR20", 0.75, "robin", 20), ("bR20", 1.5, "robin", 20),
              ("cR20", 3.0, "robin", 20)]
    refs = {}
    for side in sorted({m[1] for m in models}):
        n = int(round(side / h))
        lo = -0.5 * side
        cg = lo + (np.arange(-1, n + 1) + 0.5) * h
        Z, Y, X = np.meshgrid(cg, cg, cg, indexing="ij")
        def ref(t, n=n, lo=lo, X=X, Y=Y, Z=Z):
            b = I.orbit_blobs(t)
            return poisson_dirichlet(I.blob_density(n, b, h=h, lo=lo), blob_potential(b, X, Y, Z), h)
        refs[side] = (n, lo, ref, [ref(m * dt_hyd) for m in range(M + 1)])
    for name, side, bc, kg in models:
        n, lo, ref, rs = refs[side]
        c, nsub = kg * v_max, 2 * kg
        dt = dt_hyd / nsub
        g = hg.Grid(n, n, n, h, (lo, lo, lo), c, 1.0, dt, "f32k", bc, 4 if bc == "multipole" else 0)
        g.set_density(I.blob_density_torch(n, I.orbit_blobs(0.0), "cuda", torch.float32, h=h, lo=lo))
        g.set_phi(torch.from_numpy(rs[0]).cuda(), torch.from_numpy(ref(-dt)).cuda())
        errs = []
        for m in range(M):
            g.set_density(I.blob_density_torch(n, I.orbit_blobs(m * dt_hyd), "cuda", torch.float32, h=h, lo=lo))
            g.step(nsub)
            errs.append(g.compare(torch.from_numpy(rs[m + 1]).cuda())[2])
        g.free()
        out["results"][name] = {"cells": n ** 3, "mean": float(np.mean(errs[M // 2:])), "max": float(np.max(errs))}
    return out


def run_lag(args):
    """Next row f2: the lag of the hyperbolic potential behind the instantaneous Poisson solution (Sec. 4, Eq. error
    and Eq. Erreq.: the error is driven by (1/c_h^2) d^2 phi_P / dt^2, so it should fall as (v/c_h)^2), for the
    orbiting-blob density in a periodic box.  For c_h = k_g v_max, k_g in 5..40, and 2 k_g sub-steps per hydro step
    (dt_hyd = 0.5 h / v_max), the grid starts on the Poisson solution with its time derivative; after each hydro step
    phi_H is compared with the Poisson solution of the density at that time (relative L2, both mean-free; the
    pointwise ratio of Eq. error is undefined where the periodic phi_P crosses zero).  Two source schedules: the
    density re-evaluated at every sub-step ("smooth", which isolates the c_h lag), and frozen over each hydro step
    as in Sec. 2 ("frozen", which adds the jump of the source at every hydro step; in a periodic box the waves
    these jumps launch never leave)."""
    import numpy as np
    import torch

    import paper_1602_05700_gb300 as hg
    from paper_1602_05700_gb300 import inputs as I

    n, M = args.n, args.substeps
    h, v_max = 1.0 / n, 0.15 * 2.0 * math.pi
    dt_hyd = 0.5 * h / v_max
    rho_host = lambda t: I.blob_density(n, I.orbit_blobs(t))  # noqa: E731
    rho_dev = lambda t: I.blob_density_torch(n, I.orbit_blobs(t), "cuda", torch.float64)  # noqa: E731
    out = {"workload": f"{n}^3 periodic, two orbiting blobs (sigma 0.05, r 0.15, omega 2pi), {M} hydro steps of "
                       f"0.5 h / v_max, 2 k_g sub-steps each (nu sqrt 3 = 0.43)",
           "metric": "mean over the last half of the hydro steps of ||phi_H - phi_P||_2 / ||phi_P||_2", "results": {}}
    refs = [poisson_periodic(rho_host(m * dt_hyd), h) for m in range(M + 1)]
    kgs = (5, 10, 20, 40)
    for kg in kgs:
        c, nsub = kg * v_max, 2 * kg
        dt = dt_hyd / nsub
        row = {}
        for sched in ("smooth", "frozen"):
            for prec in ("f32k", "f64"):
                g = hg.Grid(n, n, n, h, (-0.5, -0.5, -0.5), c, 1.0, dt, prec, "periodic")
                g.set_phi(torch.from_numpy(refs[0]).cuda(), torch.from_numpy(poisson_periodic(rho_host(-dt), h)).cuda())
                errs = []
                for m in range(M):
                    if sched == "frozen":
                        g.set_density(rho_dev(m * dt_hyd))
                        g.step(nsub)
                    else:
                        for k in range(nsub):
                            g.set_density(rho_dev(m * dt_hyd + k * dt))
                            g.step(1)
                    phi = g.phi(torch.float64, "cpu")
                    d = (phi - phi.mean()) - refs[m + 1]
                    errs.append(float(np.linalg.norm(d) / np.linalg.norm(refs[m + 1])))
                g.free()
                row[f"{sched} {prec}"] = float(np.mean(errs[M // 2:]))
        out["results"][f"k_g={kg}"] = row
    for key in out["results"][f"k_g={kgs[0]}"]:
        e = np.log([out["results"][f"k_g={k}"][key] for k in kgs])
        out[f"slope_log_err_vs_log_kg {key}"] = round(float(np.polyfit(np.log(kgs), e, 1)[0]), 3)
    return out


def run_virial(args):
    """The paper's 3D star (Sec. 2; Sec. 3, Eq. VC): an n = 3 polytrope (M = 1, R = 1/3, G = 1) at the centre of
    [-1/2, 1/2]^3 on N^3 cells (the paper's 140^3 octant of a domain 1.5 R wide, mirrored: N = 280), gamma = 5/3, a
    dilute atmosphere of 1e-6 rho_c, evolved by the coupled GPU step (FP32 hydro, compensated-FP32 gravity, Robin
    boundary) for `substeps` hydro steps with Courant number 0.3 for both parts (c_g = k_g max(c_s + |v|) fixed
    from the initial state; each hydro step the largest multiple of the gravity sub-step within its own Courant
    limit): k_g = 5 unperturbed and with 1% random density perturbations (the paper's H models), and k_g = 20
    unperturbed (closer to the instantaneous-Poisson limit k_g -> infinity).  Reports VC and rho_max / rho_max(0)
    against time, and the time of a coupled hydro step split into its gravity and hydro parts."""
    import numpy as np
    import torch

    import paper_1602_05700_gb300 as hg
    from paper_1602_05700_gb300 import inputs as I

    n, steps, cfl = args.n, args.substeps, 0.3
    f64 = args.prec == "f64"  # FP64 hydro and gravity (the oracle-exact mode) instead of FP32 / compensated FP32
    h = 1.0 / n
    t_dyn = (1.0 / 3.0) ** 1.5  # sqrt(R^3 / (G M))
    res = {"workload": f"{n}^3 n=3 polytrope (M 1, R 1/3), gamma 5/3, Robin gravity, Courant {cfl:g}, "
                       f"{steps} hydro steps, {'FP64' if f64 else 'FP32 hydro + compensated FP32 gravity'}",
           "t_dyn": t_dyn}
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    for label, pert, kg in (("unperturbed", 0.0, 5.0), ("perturbed_1pct", 0.01, 5.0), ("unperturbed_kg20", 0.0, 20.0)):
        rho, P, phi, info = I.polytrope(n, pert=pert, seed=21)
        W = np.zeros((5, n, n, n), np.float64 if f64 else np.float32)
        W[0], W[4] = rho, P
        H = hg.Hydro(n, n, n, h, 5.0 / 3.0, 0.5 * info["rho_atm"], 0.5 * info["p_atm"], dtype="f64" if f64 else "f32")
        H.set_primitive(torch.from_numpy(W).cuda())
        del W
        s0 = H.max_speed()
        c = kg * s0
        dtg = cfl * h / (c * np.sqrt(3.0))
        g = hg.Grid(n, n, n, h, (-0.5, -0.5, -0.5), c, 1.0, dtg, "f64" if f64 else "f32k", "robin")
        g.set_phi(torch.from_numpy(phi).cuda())
        v0 = H.virial(g)
        trace = [(0.0, v0["VC"], 1.0)]
        t, nsub, wall = 0.0, None, 0.0
        every = max(1, steps // 40)
        e0, e1 = ev(), ev()
        H.profile(True)  # events around every stage launch of the evolution
        for it in range(steps):
            if it % 10 == 0:
                nsub = max(1, int(np.floor(cfl * h / H.max_speed() / dtg)))
            e0.record()
            H.step(nsub * dtg, g, nsub)
            e1.record()
            t += nsub * dtg
            if (it + 1) % every == 0:
                torch.cuda.synchronize()
                wall += e0.elapsed_time(e1)
                v = H.virial(g)
                trace.append((round(t / t_dyn, 4), v["VC"], v["rho_max"] / v0["rho_max"]))
        stage_ms, stage_n = H.profile_read()
        H.profile(False)
        vc = np.array([r[1] for r in trace])
        res[label] = {"k_g": kg, "t_end_over_t_dyn": round(t / t_dyn, 3), "substeps_per_hydro_step": nsub,
                      "VC_initial": trace[0][1], "VC_final": trace[-1][1],
                      "VC_max_abs": float(np.abs(vc).max()), "VC_max_abs_after_1_t_dyn":
                      max((abs(r[1]) for r in trace if r[0] >= 1.0), default=None),
                      "rho_max_ratio_final": trace[-1][2], "trace_t_VC_rhomax": trace[::4] + [trace[-1]],
                      "stage_kernel_ms_avg": round(stage_ms / max(stage_n, 1), 5), "stage_launches": stage_n}
        if label == "unperturbed":
            # time split of one coupled step: the whole step, its gravity part, and the hydro stages alone
            torch.cuda.synchronize()
            reps = 20
            dt = nsub * dtg

            def timed(fn):
                a, b = ev(), ev()
                fn()
                torch.cuda.synchronize()
                a.record()
                for _ in range(reps):
                    fn()
                b.record()
                torch.cuda.synchronize()
                return a.elapsed_time(b) / reps

            torch.cuda.cudart().cudaProfilerStart()  # an external profiler captures just these coupled steps
            ms_step = timed(lambda: H.step(dt, g, nsub))
            torch.cuda.cudart().cudaProfilerStop()
            rho_d = H.state()[0].contiguous()
            ms_grav = timed(lambda: (g.set_density(rho_d), g.step(nsub), g.accel()))
            ms_hyd = timed(lambda: H.step(dt))
            pk, kind = peaks()
            t_stage = res[label]["stage_kernel_ms_avg"] * 1e-3  # event-timed stage launches of the evolution
            alg = (124 if f64 else 62) * n ** 3  # bytes per stage launch with gravity: avg of (8 read + 5 write)
            #                                      and (13 + 5) values
            winst = None if f64 else kernel_instructions("k_hydro_stage<float>", n ** 3)
            res["timing"] = {"ms_per_coupled_step": round(ms_step, 4), "ms_gravity_substeps_and_accel": round(ms_grav, 4),
                             "ms_hydro_two_stages_without_gravity": round(ms_hyd, 4),
                             "gcell_hydro_steps_per_s": round(n ** 3 / (ms_step * 1e-3) / 1e9, 3),
                             "hydro_stage_roofline": {
                                 "bound": "alu", "kernel": "k_hydro_stage<double>" if f64 else "k_hydro_stage<float>",
                                 "unit": "G warp-instr/s",
                                 "achieved": round(winst / t_stage / 1e9, 1) if winst else None,
                                 "peak": round(ISSUE_PEAK_GWIPS, 1),
                                 "frac": round(winst / t_stage / 1e9 / ISSUE_PEAK_GWIPS, 4) if winst else None,
                                 "peak_kind": "instruction issue limit, 152 SMs x 4 schedulers x 2.07 GHz",
                                 "warp_inst_per_launch": round(winst) if winst else None,
                                 "avg_launch_ms": round(t_stage * 1e3, 5),
                                 "hbm_achieved_gbs": round(alg / t_stage / 1e9, 1),
                                 "hbm_frac": round(alg / t_stage / 1e9 / pk, 4), "hbm_peak_kind": kind,
                                 "alg_bytes_per_launch": alg,
                                 "traffic": None if f64 else stencil_traffic("k_hydro_stage<float>", n)}}
        g.free()
        H.free()
    return res


# ---- summaries of Nsight Compute output for the notes under profiles/ ----

NCU_SCALE = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0, "s": 1e3, "second": 1e3}

NCU_REPORT_METRICS = [
    ("gpu__time_duration.sum", "duration"),
    ("dram__bytes_read.sum", "DRAM read"),
    ("dram__bytes_write.sum", "DRAM write"),
    ("gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "DRAM throughput % of peak"),
    ("lts__t_sector_hit_rate.pct", "L2 hit rate %"),
    ("sm__throughput.avg.pct_of_peak_sustained_elapsed", "SM throughput %"),
    ("smsp__issue_active.avg.pct_of_peak_sustained_active", "issue active %"),
    ("sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active", "FMA pipe %"),
    ("sm__pipe_alu_cycles_active.avg.pct_of_peak_sustained_active", "ALU pipe %"),
    ("sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active", "FP64 pipe %"),
    ("sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active", "tensor pipe %"),
    ("sm__warps_active.avg.pct_of_peak_sustained_active", "warps active %"),
    ("launch__registers_per_thread", "registers/thread"),
    ("launch__occupancy_limit_registers", "blocks/SM (register limit)"),
    ("launch__grid_size", "grid"),
    ("launch__block_size", "block"),
    ("sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active", "LSU issue %"),
    ("sm__inst_executed_pipe_xu.avg.pct_of_peak_sustained_active", "XU issue %"),
    ("sm__inst_executed_pipe_adu.avg.pct_of_peak_sustained_active", "ADU issue %"),
    ("smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio", "stall long scoreboard"),
    ("smsp__average_warps_issue_stalled_short_scoreboard_per_issue_active.ratio", "stall short scoreboard"),
    ("smsp__average_warps_issue_stalled_wait_per_issue_active.ratio", "stall wait"),
    ("smsp__average_warps_issue_stalled_lg_throttle_per_issue_active.ratio", "stall LG throttle"),
    ("smsp__average_warps_issue_stalled_mio_throttle_per_issue_active.ratio", "stall MIO throttle"),
    ("smsp__average_warps_issue_stalled_not_selected_per_issue_active.ratio", "stall not selected"),
    ("smsp__average_warps_issue_stalled_barrier_per_issue_active.ratio", "stall barrier"),
    ("smsp__average_warps_issue_stalled_math_pipe_throttle_per_issue_active.ratio", "stall math pipe"),
    ("smsp__inst_executed.sum", "warp instructions"),
]


def ncu_short(name: str) -> str:
    for ns in ("(anonymous namespace)::", "<unnamed>::", "unnamed>::", "hg::"):
        name = name.replace(ns, "")
    return name.split("(")[0].replace("void ", "").strip()


def ncu_launches(path):
    """Per-kernel launches, total time and share of an ncu launch list (--metrics gpu__time_duration.sum --csv)."""
    rows = list(csv.reader(open(path)))
    h = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[h]
    ki, vi, ui = hdr.index("Kernel Name"), hdr.index("Metric Value"), hdr.index("Metric Unit")
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[h + 1:]:
        if len(r) <= vi or not r[vi]:
            continue
        agg[ncu_short(r[ki])][0] += 1
        agg[ncu_short(r[ki])][1] += float(r[vi].replace(",", "")) * NCU_SCALE[r[ui]]
    tot = sum(a[1] for a in agg.values())
    print(f"| kernel | launches | total ms | share |\n|---|---|---|---|")
    for k, (n, t) in sorted(agg.items(), key=lambda x: -x[1][1]):
        print(f"| `{k}` | {n} | {t:.3f} | {100 * t / tot:.2f}% |")
    print(f"| total | {sum(a[0] for a in agg.values())} | {tot:.3f} | |")


def ncu_report(path):
    """The headline counters of each launch of an ncu report (read with `ncu -i ... --page raw --csv`)."""
    out = subprocess.run(["ncu", "-i", path, "--page", "raw", "--csv"], capture_output=True, text=True, check=True)
    rows = list(csv.reader(io.StringIO(out.stdout)))
    hdr, units = rows[0], rows[1]
    for launch in rows[2:]:
        name = ncu_short(launch[hdr.index("Kernel Name")]) if "Kernel Name" in hdr else "?"
        print(f"launch: `{name}`\n\n| counter | value |\n|---|---|")
        for metric, label in NCU_REPORT_METRICS:
            if metric in hdr:
                i = hdr.index(metric)
                print(f"| {label} (`{metric}`) | {launch[i]} {units[i]} |")
        print()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--depth", type=int, default=0,
                    help="sub-steps fused per pass (temporal blocking); 0 = pick the fastest of 1..4 by a short sweep")
    ap.add_argument("--prec", choices=["f32k", "f64"], default="f32k",
                    help="precision of the headline measurement (f64: the FP64 mode's line, no second leg)")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-substeps", type=int, default=6)
    ap.add_argument("--ref-substeps", type=int, default=1)
    ap.add_argument("--config", choices=["headline", "precision", "batch", "adjoint", "lag", "domain", "virial"],
                    default="headline",
                    help="headline: the metric's 512^3 line (default); the others print the other workloads")
    ap.add_argument("--substeps", type=int, default=None,
                    help="sub-steps for --config precision/batch/adjoint; hydro steps for --config lag/domain/virial")
    ap.add_argument("--ncu-launches", metavar="CSV", default=None,
                    help="summarise an ncu launch list (per kernel: launches, total time, share) and exit")
    ap.add_argument("--ncu-report", metavar="NCU_REP", default=None,
                    help="print the headline counters of each launch in an ncu report and exit")
    args = ap.parse_args()
    if args.ncu_launches or args.ncu_report:
        if args.ncu_launches:
            ncu_launches(args.ncu_launches)
        if args.ncu_report:
            ncu_report(args.ncu_report)
        return
    from paper_1602_05700_gb300.multi import env_ranks

    rank, world, local_rank = env_ranks()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    import paper_1602_05700_gb300 as hg
    hg.build()
    if args.config != "headline":
        defaults = {"precision": (256, 2000), "batch": (0, 500), "adjoint": (128, 400), "lag": (128, 40),
                    "domain": (0, 40), "virial": (280, 2600)}
        n0, t0 = defaults[args.config]
        if args.n == 512 and n0:
            args.n = n0
        args.substeps = args.substeps or t0
        fn = {"precision": run_precision, "batch": run_batch, "adjoint": run_adjoint, "lag": run_lag,
              "domain": run_domain, "virial": run_virial}[args.config]
        if rank == 0:
            print(json.dumps({"config": args.config, **fn(args)}), flush=True)
        return
    line = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
