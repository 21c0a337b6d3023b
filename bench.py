#!/usr/bin/env python
"""Benchmark of the GMG-preconditioned FGMRES slab solve on one GB300 (or N replicas).

Step = one flexible-GMRES solve (V(2,2) additive-Vanka V-cycle per iteration) of the dG(k)
Q2/P1disc slab Newton system to 1e-8 relative residual, from x = 0, with the hierarchy assembled
and factored once beforehand (assembly and factorisation times are reported under "setup").
The headline `value` is seconds per solve of the fastest mixed-precision run: FP32 or BF16 cell
inverses, optionally with FP32 defects inside the V-cycle ("bf16+f32d"); the FGMRES products and
stopping test are FP64 in every run, and the plain FP64 path is timed in the same run ("fp64_s").

Prints ONE JSON line (rank 0). `--impl reference` times the CPU oracle (the plain FP64 reference
implementation written from the paper) on the same workload instead.
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

DEFAULT_WORKLOAD = "c2_2d_k2"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--precisions", default="f64,f32,bf16,bf16+f32d",
                    help="cell-inverse storage per run; INV+f32d also takes the V-cycle defects in FP32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--multi-restart", type=int, default=20)
    ap.add_argument("--robustness", action="store_true",
                    help="viscosity / damping study: Newton and FGMRES counts for nu x omega_d (V(4,4), tau 0.005)")
    ap.add_argument("--march", type=int, default=0,
                    help="time-march this many slabs (damped Newton per slab) and report the wake functional")
    ap.add_argument("--mesh-study", action="store_true",
                    help="FGMRES iterations of V(1,1) and V(4,4) as one coarse grid is refined (2D and 3D dG(1))")
    ap.add_argument("--newton", action="store_true",
                    help="time the damped Newton solve of the nonlinear slab problem instead of one linear solve")
    ap.add_argument("--oracle-child", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


def workload(name):
    import synth

    return synth.WORKLOADS[name]


def describe(wl, sizes):
    fine = sizes[-1]
    return {"workload": f"{wl.name}: {wl.dim}D channel {'x'.join(map(str, wl.fine_cells))} fine cells "
                        f"({'obstacle' if wl.obstacle_lo != wl.obstacle_hi else 'no obstacle'}), "
                        f"{wl.n_levels} levels, Q2/P1disc x dG({wl.k})",
            "dofs": fine["n_dofs"], "cells": fine["n_cells"], "n_local": fine["n_local"],
            "levels": wl.n_levels, "rtol": None, "smoother": f"additive Vanka V({wl.nu1},{wl.nu2}) omega={wl.omega}",
            "krylov": f"FGMRES({wl.restart})", "nu": wl.nu, "tau": wl.tau}


# ---------------------------------------------------------------------------------------------
# CPU oracle leg (run in a spawned child process so that it never shares the CUDA context)
# ---------------------------------------------------------------------------------------------
def oracle_child(spec_path):
    spec = json.load(open(spec_path))
    import numpy as np

    import synth
    from oracle import solvers

    wl = synth.WORKLOADS[spec["workload"]]
    t0 = time.perf_counter()
    H = solvers.Hierarchy(wl, synth.linearisation_point(wl))
    setup = time.perf_counter() - t0
    b = H.fine.dofs_from_lattice(synth.random_rhs(wl))
    times, iters = [], []
    for _ in range(spec["solves"]):
        t0 = time.perf_counter()
        x, info = H.solve(b, rtol=spec["rtol"], maxit=spec["maxit"])
        times.append(time.perf_counter() - t0)
        iters.append(info["iters"])
    sizes = {"n_dofs": int(H.fine.N), "n_cells": int(H.fine.C), "n_local": int(H.fine.n)}
    json.dump({"setup_s": setup, "solve_s": times, "iters": iters, "converged": bool(info["converged"]),
               "sizes": sizes}, open(spec["out"], "w"))


def run_oracle(wl_name, rtol, solves, maxit=1000, threads=1):
    with tempfile.TemporaryDirectory() as td:
        spec = {"workload": wl_name, "rtol": rtol, "solves": solves, "maxit": maxit, "out": os.path.join(td, "o.json")}
        sp = os.path.join(td, "spec.json")
        json.dump(spec, open(sp, "w"))
        env = dict(os.environ)
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[v] = str(threads)
        env["CUDA_VISIBLE_DEVICES"] = ""
        p = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child", sp], env=env,
                           capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("oracle child failed:\n" + p.stderr[-3000:])
        return json.load(open(spec["out"]))


# ---------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.path = tempfile.mktemp(suffix=".csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), hw=parts[5], hwt=parts[6], swt=parts[7],
                                 pcap=parts[8]))
            except ValueError:
                continue
        os.remove(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("pcap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def recorded_traffic(workload_name, kernel, prec=None):
    """DRAM bytes per launch of a finest-level kernel from a committed ncu capture, valid only
    while the kernel's source file is unchanged since the capture (sha256 of the file)."""
    import hashlib

    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "roofline_traffic.json")))
    except (OSError, ValueError):
        return None
    for e in rec.get("captures", []):
        if e.get("workload") != workload_name or e.get("kernel") != kernel:
            continue
        if prec is not None and e.get("precision") != prec:
            continue
        try:
            sha = hashlib.sha256(open(os.path.join(ROOT, e["source"]), "rb").read()).hexdigest()
        except (OSError, KeyError):
            continue
        if sha == e.get("source_sha256"):
            return {"per_launch_bytes": e["dram_bytes_read"] + e["dram_bytes_write"], "source": e["profile"]}
    return None


def spmv_roofline(r, wl, sizes, fp64_peak, workload_name):
    """Dominant kernel of the solve: the node-block FP64 product with the finest J (FP64-pipe bound).

    achieved = 2 * nnz FLOP per launch (one FMA per stored value) / average event time per launch;
    peak = FP64 FMA throughput measured in the same run (stm_measure_fp64_peak)."""
    f = r["finest"]["jacobian_spmv"]
    if f["ms"] <= 0 or f["launches"] == 0:
        return None
    nnz = sizes[-1]["nnz"]
    us = 1e3 * f["ms"] / f["launches"]
    achieved = 2.0 * nnz / (us * 1e-6) / 1e12
    traffic = recorded_traffic(workload_name, "k_spmv_nodeblock")
    return {"kernel": "k_spmv_nodeblock (J_g x, finest level, FP64)", "bound": "alu", "achieved": achieved,
            "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak if fp64_peak else None,
            "traffic": traffic["per_launch_bytes"] if traffic else None,
            "traffic_source": traffic["source"] if traffic else "no capture of the current kernel source",
            "peak_source": "FP64 FMA rate measured in this run (stm_measure_fp64_peak)",
            "flops_per_launch": 2.0 * nnz, "avg_launch_us": us,
            "algorithmic_bytes_per_launch": f["bytes"] / f["launches"],
            "hbm_gbs_algorithmic": f["bytes"] / (f["ms"] * 1e-3) / 1e9}


def defect_roofline(r, sizes, hbm, peak_source, workload_name):
    """The V-cycle's defect r - J_g d over the FP32 copies of J_g, finest level (HBM bound).

    achieved = (4 nnz + 20 N) algorithmic bytes per launch (FP32 values and d, FP64 r and t) / average
    event time per launch of the product kernel; peak = the measured copy bandwidth. The rounding of
    d to FP32 before it (12 N bytes, a launch of its own) is timed as class round_f32."""
    f = r["finest"]["defect_f32"]
    if f["ms"] <= 0 or f["launches"] == 0:
        return None
    us = 1e3 * f["ms"] / f["launches"]
    by = f["bytes"] / f["launches"]
    achieved = by / (us * 1e-6) / 1e9
    traffic = recorded_traffic(workload_name, "k_spmv_nodeblock_f32")
    return {"kernel": "k_spmv_nodeblock<float> (r - J_g d over FP32 values, finest level)", "bound": "hbm",
            "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic["per_launch_bytes"] if traffic else None,
            "traffic_source": traffic["source"] if traffic else "no capture of the current kernel source",
            "peak_source": peak_source, "bytes_per_launch": by, "avg_launch_us": us}


def max_over_ranks(value, dist, device):
    """Replicas (one independent slab solve per GPU): the job's time per step is the slowest rank's."""
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def split_precision(tok):
    """'bf16+f32d' -> ('bf16', 'f32'): cell-inverse storage and V-cycle defect precision."""
    inv, sep, d = tok.partition("+")
    if inv not in ("f64", "f32", "bf16") or (sep and d != "f32d"):
        raise ValueError(f"precision {tok!r}: expected f64|f32|bf16, optionally +f32d")
    return inv, ("f32" if d else "f64")


def hier_params(wl, tok, smoother="additive"):
    from paper_2107_10561_gb300 import make_params

    inv, dp = split_precision(tok)
    return make_params(wl.dim, wl.k, wl.n_levels, wl.coarse_cells, wl.length, wl.obstacle_lo, wl.obstacle_hi,
                       wl.tau, wl.nu, wl.gamma1, wl.gamma2, inv, smoother, wl.omega, wl.nu1, wl.nu2,
                       defect_precision=dp)


def dtype_label(tok):
    inv, dp = split_precision(tok)
    if inv == "f64" and dp == "f64":
        return "f64"
    parts = [f"{inv} cell inverses (f32 accumulate)"] if inv != "f64" else []
    if dp == "f32":
        parts.append("f32 V-cycle defects")
    return "f64 Krylov/Arnoldi SpMV/coarse + " + " + ".join(parts)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return None


# ---------------------------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------------------------
def gpu_leg(args, rank, world, local_rank):
    import numpy as np
    import torch

    import synth
    from paper_2107_10561_gb300 import Hierarchy, make_params
    from paper_2107_10561_gb300 import build as _build

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    _build.build()
    wl = workload(args.workload)
    state = synth.linearisation_point(wl)
    rhs_lat = synth.random_rhs(wl, seed_offset=rank)
    results = {}
    hs = {}
    for prec in args.precisions.split(","):
        p = hier_params(wl, prec, "additive")
        h = Hierarchy(p)
        idx = h.dof_lattice_index()
        X = torch.from_numpy(np.ascontiguousarray(state.reshape(-1)[idx])).cuda()
        b = torch.from_numpy(np.ascontiguousarray(rhs_lat.reshape(-1)[idx])).cuda()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        e0.record()
        h.assemble_jacobian(X)
        e1.record()
        h.factor_cells()
        e2.record()
        torch.cuda.synchronize()
        setup = {"assemble_ms": e0.elapsed_time(e1), "factor_ms": e1.elapsed_time(e2)}
        x = torch.zeros_like(b)
        for _ in range(args.warmup):
            x.zero_()
            info = h.gmres_solve(b, x, rtol=args.rtol, restart=wl.restart)
        hs[prec] = (h, b, x)
        results[prec] = {"setup": setup, "iters": info["iters"], "rel_res_true": info["rel_res_true"]}
    sizes = [hs[next(iter(hs))][0].sizes(g) for g in range(wl.n_levels)]
    # cumulative library launches before the timed region (lets an ncu launch list skip the set-up)
    print(f"library_launches_before_timed_region={Hierarchy.kernel_launches()}", file=sys.stderr)

    # timed region, every precision, K solves each
    sampler = ClockSampler(local_rank)
    sampler.start()
    time.sleep(0.3)
    stream = torch.cuda.current_stream()
    for prec, (h, b, x) in hs.items():
        # clean timed pass (CUDA graphs for the V-cycles, no per-kernel events): the reported time
        launches0 = Hierarchy.kernel_launches()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(f"timed_solves_{prec.replace('+', '_')}")  # lets a profiler select exactly these launches
        ev0.record(stream)
        for _ in range(args.steps):
            x.zero_()
            info = h.gmres_solve(b, x, rtol=args.rtol, restart=wl.restart)
        ev1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.steps
        if dist:
            ms = max_over_ranks(ms, dist, "cuda")
        r = results[prec]
        r["ms_per_solve"] = ms
        r["launches_per_step"] = (Hierarchy.kernel_launches() - launches0) / args.steps
        r["iters_timed"] = info["iters"]
        r["rel_res_true_timed"] = info["rel_res_true"]
        # profiled pass over the same steps: CUDA events around every launch of the library, recorded
        # on the launching stream (direct launches, no graphs), for the per-kernel split and roofline
        h.profile_enable(True)
        torch.cuda.synchronize()
        pv0, pv1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pv0.record(stream)
        for _ in range(args.steps):
            x.zero_()
            h.gmres_solve(b, x, rtol=args.rtol, restart=wl.restart)
        pv1.record(stream)
        torch.cuda.synchronize()
        r["ms_per_solve_profiled"] = pv0.elapsed_time(pv1) / args.steps
        r["kernels"] = {k: h.profile_read(k) for k in ("vanka_local", "jacobian_spmv", "defect_f32", "round_f32",
                                                       "vanka_combine", "transfer",
                                                       "coarse", "krylov")}
        r["finest"] = {k: h.profile_read(k, wl.n_levels - 1) for k in ("vanka_local", "jacobian_spmv", "defect_f32")}
        r["per_level"] = {k: [h.profile_read(k, g) for g in range(wl.n_levels)]
                          for k in ("vanka_local", "jacobian_spmv", "defect_f32", "vanka_combine", "transfer")}
        h.profile_enable(False)
    clocks = sampler.stop()
    fp64_peak = Hierarchy.measure_fp64_peak()

    # end-to-end through the host-buffer entry point (H2D of b, D2H of x inside the timed region)
    mixed = [p for p in results if p != "f64"]
    head = min(mixed, key=lambda p: results[p]["ms_per_solve"]) if mixed else "f64"
    h, b, x = hs[head]
    bh = b.cpu().pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    h.gmres_solve_host(bh, xh, rtol=args.rtol, restart=wl.restart)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        h.gmres_solve_host(bh, xh, rtol=args.rtol, restart=wl.restart)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    rows = other_rows(args, wl, hs, head, state, rhs_lat) if rank == 0 else {}
    return wl, sizes, results, head, clocks, e2e_s, dist, fp64_peak, rows


def other_rows(args, wl, hs, head, state, rhs_lat):
    """Timings of the rows that the headline solve does not isolate, on the same workload and the
    head precision: one V-cycle (Algorithm 1, direct launches), the adjoint solve J^T lambda = b
    (transposed Vanka, P/P^T, coarse inverse^T), and the solve with the coloured multiplicative and
    the literal overwrite smoother (Sec. 4.2)."""
    import numpy as np
    import torch

    from paper_2107_10561_gb300 import Hierarchy, make_params

    out = {}
    h, b, x = hs[head]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d = torch.zeros_like(b)
    h.vcycle(b, d)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(10):
        h.vcycle(b, d)
    ev1.record()
    torch.cuda.synchronize()
    out["vcycle_ms"] = ev0.elapsed_time(ev1) / 10
    x.zero_()
    h.gmres_solve(b, x, rtol=args.rtol, restart=wl.restart, transpose=True)  # warm-up (J^T values)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(args.steps):
        x.zero_()
        info = h.gmres_solve(b, x, rtol=args.rtol, restart=wl.restart, transpose=True)
    ev1.record()
    torch.cuda.synchronize()
    out["adjoint_solve"] = {"ms": ev0.elapsed_time(ev1) / args.steps, "iters": info["iters"],
                            "rel_res_true": info["rel_res_true"]}
    for smoother in ("coloured", "overwrite"):
        p = hier_params(wl, head, smoother)
        hv = Hierarchy(p)
        idx = hv.dof_lattice_index()
        X = torch.from_numpy(np.ascontiguousarray(state.reshape(-1)[idx])).cuda()
        bv = torch.from_numpy(np.ascontiguousarray(rhs_lat.reshape(-1)[idx])).cuda()
        hv.assemble_jacobian(X)
        hv.factor_cells()
        xv = torch.zeros_like(bv)
        hv.gmres_solve(bv, xv, rtol=args.rtol, restart=wl.restart, raise_on_fail=False)
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(args.steps):
            xv.zero_()
            info = hv.gmres_solve(bv, xv, rtol=args.rtol, restart=wl.restart, raise_on_fail=False)
        ev1.record()
        torch.cuda.synchronize()
        out[f"{smoother}_solve"] = {"ms": ev0.elapsed_time(ev1) / args.steps, "iters": info["iters"],
                                    "converged": info["status"] == "STM_OK"}
        hv.close()
    return out


def gpu_leg_multi(args, local_rank):
    """Multi-RHS workload: 32 right-hand sides b(U_j, nu) + c(w, w) sharing one hierarchy."""
    import numpy as np
    import torch

    import synth
    from paper_2107_10561_gb300 import Hierarchy, make_params
    from paper_2107_10561_gb300 import build as _build

    torch.cuda.set_device(local_rank)
    _build.build()
    wl = workload(args.workload)
    nrhs = wl.extra["nrhs"]
    prec = args.precisions.split(",")[-1]
    p = hier_params(wl, prec, "additive")
    t0 = time.perf_counter()
    h = Hierarchy(p)
    build_s = time.perf_counter() - t0
    idx = h.dof_lattice_index()
    X = torch.from_numpy(np.ascontiguousarray(synth.linearisation_point(wl).reshape(-1)[idx])).cuda()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    torch.cuda.synchronize()
    e0.record()
    h.assemble_jacobian(X)
    e1.record()
    h.factor_cells()
    e2.record()
    torch.cuda.synchronize()
    n = h.n_dofs()
    B = torch.empty((nrhs, n), dtype=torch.float64, device="cuda")
    for c, U in enumerate(synth.inflow_sweep(nrhs)):
        h.assemble_rhs(float(U), wl.nu, B[c], which=0)
    Xs = torch.zeros_like(B)
    for _ in range(args.warmup):
        Xs.zero_()
        infos = h.gmres_solve_multi(B, Xs, rtol=args.rtol, restart=args.multi_restart)
    sampler = ClockSampler(local_rank)
    sampler.start()
    h.profile_enable(True)
    launches0 = Hierarchy.kernel_launches()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        Xs.zero_()
        infos = h.gmres_solve_multi(B, Xs, rtol=args.rtol, restart=args.multi_restart)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    clocks = sampler.stop()
    kern = {k: h.profile_read(k) for k in ("vanka_local", "jacobian_spmv", "vanka_combine", "transfer", "coarse",
                                           "krylov")}
    fin = h.profile_read("vanka_local", wl.n_levels - 1)
    sizes = [h.sizes(g) for g in range(wl.n_levels)]
    pk = peaks()
    hbm = pk["hbm_gbs"] if pk else 6800.0
    ach = fin["bytes"] / (fin["ms"] * 1e-3) / 1e9 if fin["ms"] > 0 else None
    cfg = describe(wl, sizes)
    cfg.update({"rtol": args.rtol, "nrhs": nrhs, "rhs": "b(U_j, nu) + c(w, w), U_j = linspace(0.2, 0.45, 32)",
                "restart": args.multi_restart, "parallelism": "single GPU",
                "l2": "inputs larger than L2 (finest J %.1f GB)" % (sizes[-1]["nnz"] * 12 / 1e9)})
    line = {"metric": "GMG-GMRES s to 1e-8 rel. res (mixed vs FP64, one GB300); Vanka sweep GB/s",
            "value": ms / 1e3, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": f"f64 Krylov/SpMM/coarse + {split_precision(prec)[0]} cell inverses ({'tensor cores, ' if split_precision(prec)[0] == 'bf16' else ''}f32 accumulate); FP64 defects",
            "data": "synthetic", "config": cfg, "per_rhs_s": ms / 1e3 / nrhs,
            "iters": [i["iters"] for i in infos], "max_rel_res_true": max(i["rel_res_true"] for i in infos),
            "setup": {"build_hierarchy_s": build_s, "assemble_ms": e0.elapsed_time(e1), "factor_ms": e1.elapsed_time(e2)},
            "kernel_ms_per_solve": {k: v["ms"] / args.steps for k, v in kern.items()},
            "gpu_launches": int(Hierarchy.kernel_launches() - launches0),
            "roofline": {"kernel": f"k_vanka_mrhs ({prec}), finest level, 32 columns", "bound": "hbm",
                         "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm if ach else None,
                         "traffic": None, "avg_launch_us": 1e3 * fin["ms"] / max(fin["launches"], 1)},
            "clocks": clocks, "cpu_baseline": None,
            "cpu_baseline_note": "the FP64 oracle of this workload needs ~70 GB of host memory and hours; not timed"}
    print(json.dumps(line))


def gpu_leg_newton(args, local_rank):
    """Damped Newton for the slab problem F(X) = A X + c(X, X) - b(U, nu) = 0 from the seeded state,
    U = 0.3; stop at 1e-10 or a reduction by 1e4 (Sec. 5.1). Each step re-assembles J on every level,
    factors every cell inverse and the coarse inverse, and solves with GMG-FGMRES to args.rtol."""
    import numpy as np
    import torch

    import synth
    from paper_2107_10561_gb300 import Hierarchy, make_params
    from paper_2107_10561_gb300 import build as _build

    torch.cuda.set_device(local_rank)
    _build.build()
    wl = workload(args.workload)
    out = {}
    for prec in args.precisions.split(","):
        p = hier_params(wl, prec, "additive")
        h = Hierarchy(p)
        idx = h.dof_lattice_index()
        X0 = torch.from_numpy(np.ascontiguousarray(synth.linearisation_point(wl).reshape(-1)[idx])).cuda()
        X = torch.empty_like(X0)
        for _ in range(args.warmup):
            X.copy_(X0)
            info = h.newton_solve(X, wl.inflow_u, rtol=args.rtol, restart=wl.restart)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        launches0 = Hierarchy.kernel_launches()
        ev0.record()
        for _ in range(args.steps):
            X.copy_(X0)
            info = h.newton_solve(X, wl.inflow_u, rtol=args.rtol, restart=wl.restart)
        ev1.record()
        torch.cuda.synchronize()
        out[prec] = {"ms": ev0.elapsed_time(ev1) / args.steps, "info": info,
                     "launches": (Hierarchy.kernel_launches() - launches0) / args.steps}
        h.close()
    head = args.precisions.split(",")[-1]
    r = out[head]
    cfg = {"workload": f"{wl.name}: damped Newton for one slab, U = {wl.inflow_u}, from the seeded state",
           "stop": "||F|| <= max(1e-10, ||F_0|| / 1e4)", "linear_rtol": args.rtol, "parallelism": "single GPU"}
    line = {"metric": "damped-Newton slab solve s (GMG-FGMRES inner solves)", "value": r["ms"] / 1e3, "unit": "s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_label(head), "data": "synthetic", "config": cfg,
            "by_precision": {p: {"s": v["ms"] / 1e3, "newton_iters": v["info"]["newton_iters"],
                                 "gmres_iters": v["info"]["gmres_iters"], "res": v["info"]["res"],
                                 "lam": v["info"]["lam"]} for p, v in out.items()},
            "gpu_launches": int(r["launches"] * args.steps)}
    print(json.dumps(line))


def gpu_leg_march(args, local_rank):
    """Time marching (Problem 3.1): args.march slabs from the seeded state, slab n started from slab
    n-1 with its last time node as initial value, each solved by damped Newton (stop at 1e-10 or a
    reduction by 1e4) with GMG-FGMRES inner solves; the wake functional int_{I_n} int_wake v_1 per slab."""
    import numpy as np
    import torch

    import synth
    from paper_2107_10561_gb300 import Hierarchy, make_params
    from paper_2107_10561_gb300 import build as _build

    torch.cuda.set_device(local_rank)
    _build.build()
    wl = workload(args.workload)
    prec = args.precisions.split(",")[-1]
    p = hier_params(wl, prec, "additive")
    h = Hierarchy(p)
    idx = h.dof_lattice_index()
    X0 = torch.from_numpy(np.ascontiguousarray(synth.linearisation_point(wl).reshape(-1)[idx])).cuda()
    # wake: the two level-1 cell columns behind the obstacle at the obstacle's height (a full-height
    # box would measure the flux, which the inflow fixes)
    lo = (wl.obstacle_hi[0], wl.obstacle_lo[1]) + ((0,) if wl.dim == 3 else ())
    hi = (min(wl.obstacle_hi[0] + 2, wl.coarse_cells[0]), wl.obstacle_hi[1]) + \
        ((wl.coarse_cells[2],) if wl.dim == 3 else ())
    j = torch.empty(h.n_dofs(), dtype=torch.float64, device="cuda")
    h.functional_weights(lo, hi, j)
    h.time_march(X0, wl.inflow_u, 1, j=j, rtol=args.rtol, restart=wl.restart)  # warm-up slab
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    states, infos, values = h.time_march(X0, wl.inflow_u, args.march, j=j, rtol=args.rtol, restart=wl.restart)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    h.close()
    line = {"metric": "time-marching s per slab (damped Newton, GMG-FGMRES inner solves)",
            "value": ms / 1e3 / args.march, "unit": "s", "n_gpus": 1, "steps": args.march, "warmup": 1,
            "ms_per_step": ms / args.march, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_label(prec), "data": "synthetic",
            "config": {"workload": f"{wl.name}: {args.march} slabs of tau = {wl.tau} from the seeded state, "
                                   f"U = {wl.inflow_u}", "wake": {"lo": lo, "hi": hi}, "linear_rtol": args.rtol,
                       "parallelism": "single GPU"},
            "slabs": [{"newton_iters": i["newton_iters"], "gmres_step": i["gmres_step"], "res": i["res"],
                       "wake_functional": v} for i, v in zip(infos, values)]}
    print(json.dumps(line))


def gpu_leg_robustness(args, local_rank):
    """Sec. 5.3 / Table 5.4 on the synthetic channel: for nu in {1e-3, 5e-4, 3e-4, 2e-4, 1e-4} and
    omega_d in {1, 0.7}, one damped-Newton slab solve from the seeded state with V(4,4) cycles and
    tau = 0.005; reports Newton steps and FGMRES iterations per step (None: FGMRES did not reach the
    tolerance within 1000 iterations, the table's infinity)."""
    import dataclasses

    import numpy as np
    import torch

    import synth
    from paper_2107_10561_gb300 import Hierarchy, make_params
    from paper_2107_10561_gb300 import build as _build

    torch.cuda.set_device(local_rank)
    _build.build()
    base = workload(args.workload)
    prec = args.precisions.split(",")[-1]
    table = []
    t_all = time.perf_counter()
    for nu in (1e-3, 5e-4, 3e-4, 2e-4, 1e-4):
        for omega in (1.0, 0.7):
            wl = dataclasses.replace(base, nu=nu, omega=omega, nu1=4, nu2=4, tau=0.005)
            p = hier_params(wl, prec, "additive")
            h = Hierarchy(p)
            idx = h.dof_lattice_index()
            X = torch.from_numpy(np.ascontiguousarray(synth.linearisation_point(wl).reshape(-1)[idx])).cuda()
            t0 = time.perf_counter()
            info = h.newton_solve(X, wl.inflow_u, rtol=args.rtol, restart=wl.restart, max_iter=1000,
                                  raise_on_fail=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            ok = info["status"] == "STM_OK"
            table.append({"nu": nu, "omega_d": omega, "converged": ok, "newton_steps": info["newton_iters"],
                          "gmres_per_step": info["gmres_step"],
                          "gmres_avg": (float(np.mean(info["gmres_step"])) if ok and info["gmres_step"] else None),
                          "status": info["status"], "s": dt})
            h.close()
    line = {"metric": "Newton steps and FGMRES iterations per Newton step vs nu and omega_d (Table 5.4 setting)",
            "value": time.perf_counter() - t_all, "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": dtype_label(prec),
            "data": "synthetic",
            "config": {"workload": f"{base.name}, tau 0.005, V(4,4), additive Vanka, inner rtol {args.rtol}, "
                                   "FGMRES(30) capped at 1000 iterations", "parallelism": "single GPU"},
            "table": table}
    print(json.dumps(line))


def gpu_leg_mesh(args, local_rank):
    """Tables 5.1 and 5.5 setting on the synthetic channel: one linear FGMRES solve (seeded right-hand
    side, seeded linearisation point, rtol as given) with V(1,1) and with V(4,4) cycles while the same
    coarse grid is refined: 2D dG(1) on 3..6 levels, 3D dG(1) on 2..4 levels. The paper reports the
    average per Newton step over whole simulations; here each entry is one solve."""
    import dataclasses

    import numpy as np
    import torch

    import synth
    from paper_2107_10561_gb300 import Hierarchy
    from paper_2107_10561_gb300 import build as _build

    torch.cuda.set_device(local_rank)
    _build.build()
    prec = args.precisions.split(",")[-1]
    table = []
    t_all = time.perf_counter()
    for base_name, levels in (("c4_2d_k1", (3, 4, 5, 6)), ("c3_3d_k1", (2, 3, 4))):
        base = workload(base_name)
        for n_levels in levels:
            for sweeps in (1, 4):
                wl = dataclasses.replace(base, n_levels=n_levels, nu1=sweeps, nu2=sweeps)
                h = Hierarchy(hier_params(wl, prec, "additive"))
                idx = h.dof_lattice_index()
                X = torch.from_numpy(np.ascontiguousarray(synth.linearisation_point(wl).reshape(-1)[idx])).cuda()
                b = torch.from_numpy(np.ascontiguousarray(synth.random_rhs(wl).reshape(-1)[idx])).cuda()
                h.assemble_jacobian(X)
                h.factor_cells()
                x = torch.zeros_like(b)
                h.gmres_solve(b, x, rtol=args.rtol, restart=wl.restart, raise_on_fail=False)
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                x.zero_()
                torch.cuda.synchronize()
                ev0.record()
                info = h.gmres_solve(b, x, rtol=args.rtol, restart=wl.restart, raise_on_fail=False)
                ev1.record()
                torch.cuda.synchronize()
                table.append({"mesh": f"{wl.dim}D {'x'.join(map(str, wl.fine_cells))}", "levels": n_levels,
                              "dofs": h.n_dofs(), "cycle": f"V({sweeps},{sweeps})", "iters": info["iters"],
                              "converged": info["status"] == "STM_OK", "ms": ev0.elapsed_time(ev1)})
                h.close()
    line = {"metric": "FGMRES iterations per solve for V(1,1) / V(4,4) under refinement (Tables 5.1, 5.5 setting)",
            "value": time.perf_counter() - t_all, "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": dtype_label(prec),
            "data": "synthetic",
            "config": {"workload": "2D channel 16x4 coarse cells (obstacle), dG(1), 3..6 levels; 3D channel "
                                   "16x4x4 coarse cells (obstacle), dG(1), 2..4 levels; additive Vanka, omega 0.7",
                       "rtol": args.rtol, "parallelism": "single GPU"},
            "table": table}
    print(json.dumps(line))


def main():
    args = parse()
    if args.oracle_child:
        oracle_child(args.oracle_child)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        wl = workload(args.workload)
        samples = max(1, args.steps)
        o = run_oracle(args.workload, args.rtol, samples)
        t = statistics.mean(o["solve_s"])
        line = {"impl": "reference", "metric": "GMG-GMRES s to 1e-8 rel. res (mixed vs FP64, one GB300); Vanka sweep GB/s",
                "value": t, "unit": "s", "n_gpus": args.gpus, "steps": samples, "warmup": 0,
                "ms_per_step": 1e3 * t, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": dict(describe(wl, [o["sizes"]]), rtol=args.rtol,
                               parallelism="CPU oracle, one thread (rank 0 of the job)"),
                "cpu_baseline": {"value": t, "unit": "s", "cores": 1, "kind": "oracle",
                                 "sample": f"{samples} full FP64 oracle FGMRES solve(s) of the same workload ({o['iters'][-1]} "
                                           f"iterations each, single-threaded numpy/scipy) after "
                                           f"an untimed {o['setup_s']:.1f} s oracle setup"},
                "e2e": {"value": t, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.mesh_study:
        if rank == 0:
            gpu_leg_mesh(args, local_rank)
        return
    if args.newton:
        if rank == 0:
            gpu_leg_newton(args, local_rank)
        return
    if args.robustness:
        if rank == 0:
            gpu_leg_robustness(args, local_rank)
        return
    if args.march:
        if rank == 0:
            gpu_leg_march(args, local_rank)
        return
    if workload(args.workload).extra.get("nrhs"):
        if rank == 0:
            gpu_leg_multi(args, local_rank)
        return
    wl, sizes, results, head, clocks, e2e_s, dist, fp64_peak, rows = gpu_leg(args, rank, world, local_rank)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    pk = peaks()
    hbm = pk["hbm_gbs"] if pk else 6800.0
    r = results[head]
    vl = r["finest"]["vanka_local"]
    achieved = vl["bytes"] / (vl["ms"] * 1e-3) / 1e9 if vl["ms"] > 0 else None
    vk = "k_vanka_warp" if sizes[-1]["n_local"] <= 64 else "k_vanka_local"
    traffic = recorded_traffic(args.workload, vk, split_precision(head)[0])
    cfg = describe(wl, sizes)
    cfg["rtol"] = args.rtol
    inv_bytes = {"f64": 8, "f32": 4, "bf16": 2}
    l2_note = (f"inputs larger than L2: finest J {sizes[-1]['nnz'] * 12 / 1e6:.0f} MB, finest inverses "
               f"{sizes[-1]['n_cells'] * sizes[-1]['n_local'] ** 2 * inv_bytes[split_precision(head)[0]] / 1e6:.0f} MB ({head})")
    cfg["l2"] = l2_note
    cfg["parallelism"] = f"replicas x{world}" if world > 1 else "single GPU"
    line = {
        "metric": "GMG-GMRES s to 1e-8 rel. res (mixed vs FP64, one GB300); Vanka sweep GB/s",
        "value": r["ms_per_solve"] / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["ms_per_solve"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": dtype_label(head),
        "data": "synthetic", "config": cfg,
        "fp64_s": results["f64"]["ms_per_solve"] / 1e3 if "f64" in results else None,
        "speedup_vs_fp64": (results["f64"]["ms_per_solve"] / r["ms_per_solve"]) if "f64" in results else None,
        "by_precision": {p: {"s_per_solve": v["ms_per_solve"] / 1e3, "iters": v["iters_timed"],
                             "rel_res_true": v["rel_res_true_timed"], "setup_ms": v["setup"],
                             "vanka_sweep_gbs": (v["kernels"]["vanka_local"]["bytes"] / (v["kernels"]["vanka_local"]["ms"] * 1e-3) / 1e9)
                             if v["kernels"]["vanka_local"]["ms"] > 0 else None,
                             "spmv_gbs": (v["kernels"]["jacobian_spmv"]["bytes"] / (v["kernels"]["jacobian_spmv"]["ms"] * 1e-3) / 1e9)
                             if v["kernels"]["jacobian_spmv"]["ms"] > 0 else None,
                             "finest_vanka_gbs": (v["finest"]["vanka_local"]["bytes"] / (v["finest"]["vanka_local"]["ms"] * 1e-3) / 1e9)
                             if v["finest"]["vanka_local"]["ms"] > 0 else None,
                             "finest_spmv_gbs": (v["finest"]["jacobian_spmv"]["bytes"] / (v["finest"]["jacobian_spmv"]["ms"] * 1e-3) / 1e9)
                             if v["finest"]["jacobian_spmv"]["ms"] > 0 else None,
                             "finest_vanka_us": 1e3 * v["finest"]["vanka_local"]["ms"] / max(v["finest"]["vanka_local"]["launches"], 1),
                             "finest_spmv_us": 1e3 * v["finest"]["jacobian_spmv"]["ms"] / max(v["finest"]["jacobian_spmv"]["launches"], 1),
                             "finest_defect_f32_us": (1e3 * v["finest"]["defect_f32"]["ms"] / v["finest"]["defect_f32"]["launches"])
                             if v["finest"]["defect_f32"]["launches"] else None,
                             "finest_defect_f32_gbs": (v["finest"]["defect_f32"]["bytes"] / (v["finest"]["defect_f32"]["ms"] * 1e-3) / 1e9)
                             if v["finest"]["defect_f32"]["ms"] > 0 else None,
                             "kernel_ms_per_solve": {k: kv["ms"] / args.steps for k, kv in v["kernels"].items()},
                             "us_per_launch_by_level": {k: [round(1e3 * e["ms"] / e["launches"], 2) if e["launches"] else None
                                                            for e in lv] for k, lv in v["per_level"].items()},
                             "s_per_solve_profiled_pass": v["ms_per_solve_profiled"] / 1e3}
                         for p, v in results.items()},
        "gpu_launches": int(r["launches_per_step"] * args.steps),
        "other_rows": rows,
        "roofline": None,
        "roofline_spmv_f64": spmv_roofline(r, wl, sizes, fp64_peak, args.workload),
        "roofline_defect_f32": defect_roofline(r, sizes, hbm, "MEASURED_PEAKS.json hbm_gbs (of measured)" if pk
                                               else "fallback 6800 GB/s", args.workload),
        "roofline_vanka_sweep": {"kernel": f"{vk} (y_T = J_T^{{-1}} t_T), finest level, {head} inverses",
                                 "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                                 "frac": (achieved / hbm) if achieved else None,
                                 "traffic": traffic["per_launch_bytes"] if traffic else None,
                                 "traffic_source": traffic["source"] if traffic else "no capture of the current kernel source",
                                 "all_levels_gbs": (r["kernels"]["vanka_local"]["bytes"] / (r["kernels"]["vanka_local"]["ms"] * 1e-3) / 1e9)
                                 if r["kernels"]["vanka_local"]["ms"] > 0 else None,
                                 "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if pk else "fallback 6800 GB/s",
                                 "bytes_per_launch": vl["bytes"] / max(vl["launches"], 1),
                                 "avg_launch_us": 1e3 * vl["ms"] / max(vl["launches"], 1)},
        "vanka_sweep_gbs": achieved,
        "clocks": clocks,
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": sizes[-1]["n_dofs"] * 8,
                "d2h_bytes_per_step": sizes[-1]["n_dofs"] * 8,
                "path": f"stm_gmres_solve_host ({head}), pinned host b and x"},
    }
    # the dominant kernel: the finest-level class with the most event time per solve
    shares = {"roofline_vanka_sweep": r["finest"]["vanka_local"]["ms"],
              "roofline_spmv_f64": r["finest"]["jacobian_spmv"]["ms"],
              "roofline_defect_f32": r["finest"]["defect_f32"]["ms"]}
    dom = max((k for k in shares if line[k]), key=lambda k: shares[k])
    line["roofline"] = dict(line[dom], dominant_of={k: round(v / args.steps, 3) for k, v in shares.items()},
                            dominant_of_unit="ms per solve, finest level, profiled pass")
    if not args.no_cpu_baseline and world == 1:
        try:
            o = run_oracle(args.workload, args.rtol, 1)
            line["cpu_baseline"] = {"value": o["solve_s"][0], "unit": "s", "cores": 1, "kind": "oracle",
                                    "sample": f"one full FP64 oracle FGMRES solve of the same workload "
                                              f"({o['iters'][0]} iterations, single-threaded numpy/scipy) after an "
                                              f"untimed {o['setup_s']:.1f} s oracle setup"}
        except Exception as e:  # reported, never silently replaced
            line["cpu_baseline"] = {"value": None, "error": str(e)[-300:]}
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
