#!/usr/bin/env python
"""Benchmark of the GB300 screened-Poisson eikonal solve.

Workload (default): 2D 2048 x 2048 grid on [0,1]^2 (h = 1/2047), smooth
forcing f in [0.5, 1.5] from 8 seeded Fourier modes, 16 seeded random source
nodes, hbar = 0.005 (seeded synthetic input; the paper's maze / image
workloads are not available).  One step = one full solve through the C ABI:
eik_set_f (setup of the scaled operator) + eik_solve (Jacobi-PCG to the
componentwise tolerance, restarts, log epilogue).

Metric: stencil-PCG GLUPS = sum over steps of (unknowns x CG iterations) /
device seconds / 1e9, plus time-to-solution per step.  Both precision modes
are timed; the headline line reports the mode given by --precision.  The
mixed solve with the multigrid-preconditioned inner solve (componentwise tol
--mg-tol) is timed beside them and compared by time to solution
(--no-mg skips it; --modes mg times only it).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "stencil-PCG GLUPS and solve time, mixed vs FP64 plain at S err<=1e-6; %HBM peak"
UNIT = "GLUPS"

# Algorithmic bytes per grid node for one launch of each CG kernel: every
# array the kernel must read or write, counted once per node.
ALGO_BYTES_PER_NODE = {
    "cg_pass1_64": 32,   # read r, p, sig; write q            (4 x 8 B)
    "cg_pass2_64": 56,   # read x, r, p, q; write x, r, p     (7 x 8 B)
    # one single-reduction FP32 inner iteration: read r, p, sig, d; write r,
    # p (other buffer set) and d (7 x 4 B); the checking passes (every 4th
    # in later refinement steps) also read the FP32 iterate, not counted
    "mixed_cg": 28,
    "mixed_cg_init": 8,  # first pass of an inner solve: read r, sig
    # FP64 residual of a refinement step: read sig, x (f64); write r, p, d,
    # xref (f32)
    "mixed_residual64": 32,
    "mixed_update": 20,  # read d (f32), read and write x (f64)
    # one multigrid-preconditioned inner iteration (all its kernels), level 0:
    # V-cycle down (read r, sig, w; write the level-1 residual, 1/4 per
    # node) 13 B, V-cycle up (read r, sig, w, the level-1 correction; write
    # z) 17 B, direction (read z, p, sig; write p, q) 20 B, step (read p, q,
    # d, r; write d, r) 24 B; the coarse levels (read g, a, 4 coefficients,
    # k; write the next residual / read them again plus the parent
    # correction, write y: ~62 B per coarse node, n/3 coarse nodes) ~21 B;
    # in 3D (six coefficients, n/7 coarse nodes of ~85 B, level-0 transfers
    # of 1/8 per node) 73 + 12 = 85 B, see algo_bytes
    "mixed_mg": 95,
}


def algo_bytes(kernel, inst):
    """Algorithmic bytes per node of one launch of ``kernel`` on ``inst``."""
    if kernel == "mixed_mg" and len(inst.dims) == 3:
        return 85
    return ALGO_BYTES_PER_NODE[kernel]

# The FP64 passes are bound by the FP64 pipe, not by HBM: their roofline is
# algorithmic FP64 operations (an FMA counts 2) per node against the GB300's
# FP64 rate, 152 SMs x 2.07 GHz x 4 FP64 FLOP/clock = 1.26 TFLOP/s (nominal
# 1.25).  Pass 1: ptil = r + beta p (FMA), u = sig ptil, the 4 (6) neighbour
# additions, q = ptil - sig sum (FMA), <ptil, q> (FMA): 10 FLOP in 2D, 12 in
# 3D.  Pass 2: ptil, x, r updates and <r, r> (4 FMA): 8 FLOP.
FP64_PEAK_TFLOPS = 1.25
ALGO_FLOPS_PER_NODE = {("cg_pass1_64", 2): 10, ("cg_pass1_64", 3): 12,
                       ("cg_pass2_64", 2): 8, ("cg_pass2_64", 3): 8}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5", "fft", "paths"])
    ap.add_argument("--c4-count", type=int, default=256,
                    help="instances in the batched workload (c4)")
    ap.add_argument("--tol", type=float, default=None,
                    help="componentwise tolerance; default 1e-6, and 1e-7 for the batched "
                         "workload (c4), whose hbar = 8h instances need it for S err <= 1e-6")
    ap.add_argument("--per-launch", action="store_true",
                    help="launch every inner iteration on its own instead of in CUDA graphs "
                         "(no launches past convergence; for profiler captures, not for timing)")
    ap.add_argument("--workers", type=int, default=0,
                    help="batched workload: host worker threads driving the instances "
                         "(eik_batch_set_concurrency); 0 library choice")
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="mixed mode first inner-solve reduction (eik_options.inner_tol); "
                         "0 library choice")
    ap.add_argument("--band-bits", type=int, default=0,
                    help="mixed mode level-set band width (eik_options.band_bits): "
                         "0 library choice, negative never sweep")
    ap.add_argument("--tile-override", type=int, default=0,
                    help="inner-CG kernel variant (eik_options.tile_override): 0 library "
                         "choice, 1..4 the variants listed in include/eik.h")
    ap.add_argument("--mg-tol", type=float, default=1e-7,
                    help="componentwise tolerance of the multigrid-preconditioned "
                         "mode (2D single grids; at 1e-6 its S error can exceed 1e-6)")
    ap.add_argument("--no-mg", action="store_true",
                    help="skip the multigrid-preconditioned mode on 2D workloads")
    ap.add_argument("--modes", default="both", choices=["both", "one", "mg"],
                    help="single-grid workloads: time both precision modes (default) or only "
                         "--precision (shorter profiler captures); mg: only the "
                         "multigrid-preconditioned mixed mode (2D)")
    ap.add_argument("--batch-pack", type=int, default=0, choices=[-1, 0, 1],
                    help="batched workload: 0/1 packed (one launch per pass over all "
                         "instances), -1 each instance on its own stream")
    ap.add_argument("--batch-tile-rows", type=int, default=0,
                    help="packed batches: rows per tile (0 = autotuned)")
    ap.add_argument("--no-c3-block", action="store_true",
                    help="default 2D workload: skip timing the 3D 256^3 workload beside it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-iters", type=int, default=0,
                    help="oracle CG iterations in the CPU sample (0: sized to ~15 s)")
    return ap.parse_args()


def workload(name):
    from paper_1403_1937_gb300 import workloads as wl
    if name == "c2":
        inst = wl.config2()
        desc = {"workload": "2D 2048x2048 screened-Poisson eikonal, Fourier f in [0.5,1.5], "
                            "16 sources, hbar=0.005", "grid": [2048, 2048], "sources": 16,
                "hbar": 0.005}
    else:
        inst = wl.config3()
        desc = {"workload": "3D 256^3 screened-Poisson eikonal, box f in [0.5,2], "
                            "4 sources, hbar=0.02", "grid": [256, 256, 256], "sources": 4,
                "hbar": 0.02}
    return inst, desc


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_totals(seconds, units, ws, device):
    """Whole-job figures over ranks: the time is the maximum over ranks, the
    lattice updates are summed (each rank counts its own).  ws == 1: as is."""
    if ws == 1:
        return float(seconds), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def shard_instances(sizes, ws):
    """Deterministic split of independent instances over ws ranks, balanced
    by node count (largest first onto the least loaded rank).  Returns one
    sorted index list per rank."""
    load = [0] * ws
    parts = [[] for _ in range(ws)]
    for i in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        r = min(range(ws), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += sizes[i]
    return [sorted(p) for p in parts]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash(files):
    """Hash of the kernel sources with comments and whitespace removed, so a
    comment edit does not void the recorded ncu counters but any code change
    does."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1403_1937_gb300", "csrc")
    for name in files:
        with open(os.path.join(csrc, name), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic_field(kernel, workload_name, field):
    """One field of a committed ncu summary entry, or None when absent or
    taken on a different kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(f"{kernel}@{workload_name}")
    if not e or e.get("source_sha") != kernel_source_hash(e.get("source_files", [])):
        return None
    return e.get(field)


def ncu_traffic(kernel, workload_name):
    """DRAM bytes per launch of ``kernel`` from the committed ncu summary, or
    None when absent or taken on a different kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(f"{kernel}@{workload_name}")
    if not e or e.get("source_sha") != kernel_source_hash(e.get("source_files", [])):
        return None
    return e.get("dram_bytes_per_launch")


class Clocks:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.samples = []
        if self.proc is None:
            return
        time.sleep(0.2)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def summary(self):
        if not getattr(self, "samples", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, v in zip(names, s[5:9]):
                if v.lower() == "active":
                    reasons.add(k)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def flush_l2(buf):
    buf.add_(1.0)   # 256 MiB write, larger than the 129 MB L2


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1403_1937_gb300 import build as _build
    if not _build.up_to_date():
        _build.build()

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    inst, desc, n_unk, results = measure(args, args.workload, ws, local)
    if ws > 1:
        dist.barrier()
    return inst, desc, n_unk, results, ws, rank


def measure(args, wname, ws, local, modes=None):
    """Times one single-grid workload in the requested precision modes:
    device-resident steps (set_f + solve, L2 flushed between steps), the same
    through host buffers (e2e), and one step with per-launch CUDA events."""
    import torch
    import torch.distributed as dist
    from paper_1403_1937_gb300 import eik

    inst, desc = workload(wname)
    n_unk = inst.n - len(np.unique(inst.src_idx))
    f_host = torch.from_numpy(np.ascontiguousarray(inst.f)).pin_memory()
    f_dev = f_host.cuda()
    src = torch.from_numpy(inst.src_idx).cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def make(mode):
        if mode == "mixed_mg":    # multigrid-preconditioned inner solve (2D)
            opt = eik.make_options(precision="mixed", tol=args.mg_tol, precond="multigrid",
                                   band_bits=args.band_bits, inner_tol=args.inner_tol)
        else:
            opt = eik.make_options(precision=mode, tol=args.tol,
                                   tile_override=args.tile_override,
                                   band_bits=args.band_bits, inner_tol=args.inner_tol)
        return eik.eik_create(inst.dims, inst.h, inst.hbar, f_dev, src, None, opt)

    if modes is None and args.modes == "mg":
        modes = ["mixed_mg"]
    if modes is None:
        modes = [args.precision]
        if args.modes == "both":
            modes += [m for m in ("fp64", "mixed") if m != args.precision]
        if not args.no_mg:
            modes.append("mixed_mg")
    results = {}
    S_dev = torch.empty(inst.dims[::-1], dtype=torch.float64, device="cuda")
    for mode in modes:
        try:
            hd = make(mode)
        except Exception as e:  # a mode the build cannot run
            results[mode] = {"error": str(e).splitlines()[0]}
            continue
        if args.per_launch:
            eik.eik_set_profiling(hd, True)
        for _ in range(args.warmup):
            eik.eik_set_f(hd, f_dev)
            eik.eik_solve(hd, S_out=S_dev)
        torch.cuda.synchronize()
        eik.eik_reset_kernel_stats(hd)
        times, iters = [], []
        if ws > 1:
            dist.barrier()
        with Clocks(local) as clk:
            for _ in range(args.steps):
                flush_l2(flush)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                eik.eik_set_f(hd, f_dev)
                _, _, st = eik.eik_solve(hd, S_out=S_dev)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
                iters.append(st["inner_iters"])
        kst = eik.eik_kernel_stats(hd)
        launches = sum(v[0] for v in kst.values())
        total_t, units = job_totals(sum(times), n_unk * sum(iters), ws, "cuda")
        res = {"glups": units / total_t / 1e9, "ms_per_step": 1e3 * total_t / args.steps,
               "cg_iters_per_step": statistics.mean(iters), "gpu_launches": launches,
               "clocks": clk.summary(), "stats_last": st}
        # end to end through host buffers (pinned), copies inside the timed region
        if not args.no_e2e:
            S_host = torch.empty(inst.dims[::-1], dtype=torch.float64).pin_memory()
            eik.eik_set_f(hd, f_host.numpy())
            eik.eik_solve(hd, S_out=S_host.numpy())
            t0 = time.perf_counter()
            e_iters = 0
            for _ in range(args.steps):
                eik.eik_set_f(hd, f_host.numpy())
                _, _, st2 = eik.eik_solve(hd, S_out=S_host.numpy())
                e_iters += st2["inner_iters"]
            e_t, e_units = job_totals(time.perf_counter() - t0, n_unk * e_iters, ws, "cuda")
            res["e2e"] = {"value": e_units / e_t / 1e9, "unit": UNIT,
                          "h2d_bytes_per_step": int(inst.n * 8),
                          "d2h_bytes_per_step": int(inst.n * 8)}
        # one more identical step with per-launch CUDA-event timing
        eik.eik_reset_kernel_stats(hd)
        eik.eik_set_profiling(hd, True)
        eik.eik_set_f(hd, f_dev)
        eik.eik_solve(hd, S_out=S_dev)
        eik.eik_set_profiling(hd, False)
        prof = eik.eik_kernel_stats(hd)
        res["kernel_ms"] = {k: (v[2] / v[1] if v[1] else None, v[1], v[2])
                            for k, v in prof.items() if v[0]}
        results[mode] = res
        eik.eik_destroy(hd)
    return inst, desc, n_unk, results


def kernel_table(res, inst):
    """Per-kernel figures of the timed step: average launch time and, where
    the algorithmic bytes per node are known, achieved GB/s and the fraction
    of the measured HBM bandwidth."""
    peak, _ = measured_peaks()
    out = {}
    for k, (avg_ms, n, tot) in sorted(res.get("kernel_ms", {}).items()):
        if avg_ms is None:
            continue
        e = {"avg_us": round(avg_ms * 1e3, 2), "timed_launches": n}
        if k in ALGO_BYTES_PER_NODE:
            gbs = algo_bytes(k, inst) * inst.n / (avg_ms * 1e-3) / 1e9
            e["achieved_gbs"] = round(gbs, 1)
            e["frac_of_hbm"] = round(gbs / peak, 4)
        out[k] = e
    return out


def secondary_block(args, ws, local):
    """The 3D 256^3 workload timed in the same run as the headline 2D one:
    both precision modes, their ratio and the rooflines of the inner-CG
    kernels (no CPU baseline, no e2e)."""
    saved = args.no_e2e
    args.no_e2e = True
    modes = ["mixed", "fp64"] + ([] if args.no_mg else ["mixed_mg"])
    inst, desc, n_unk, res = measure(args, "c3", ws, local, modes=modes)
    args.no_e2e = saved
    out = {"workload": desc["workload"]}
    for mode, r in res.items():
        if "glups" in r:
            out[mode] = {"glups": round(r["glups"], 3), "ms_per_step": round(r["ms_per_step"], 3),
                         "cg_iters_per_step": r["cg_iters_per_step"],
                         "res_cw": r["stats_last"]["res_cw"],
                         "kernels": kernel_table(r, inst)}
        else:
            out[mode] = r
    if "glups" in res.get("fp64", {}) and "glups" in res.get("mixed", {}):
        out["mixed_speedup_vs_fp64"] = round(
            res["fp64"]["ms_per_step"] / res["mixed"]["ms_per_step"], 3)
        out["roofline"] = roofline(res["mixed"], inst, "c3")
        out["clocks"] = res["mixed"]["clocks"]
    if "glups" in res.get("mixed_mg", {}):
        out["mixed_mg"]["tol_componentwise"] = args.mg_tol
        out["mixed_mg"]["roofline_iteration"] = roofline(res["mixed_mg"], inst, "c3",
                                                         only="mixed_mg")
        for ref in ("fp64", "mixed"):
            if "glups" in res.get(ref, {}):
                out[f"mixed_mg_speedup_vs_{ref}"] = round(
                    res[ref]["ms_per_step"] / res["mixed_mg"]["ms_per_step"], 3)
    return out


def run_diff(args, emit=True):
    """Differentiation workload (config 5): 32 instances of 512^2, one source
    each; a step is the forward solve of the batch, dL/dS = 2 (S - T) on 4096
    receivers per instance, and the adjoint solve giving dL/df.  The targets
    T = S_ref + noise come from a solve of the separately seeded reference
    fields with this library (synthetic input data, made before timing)."""
    import torch
    from paper_1403_1937_gb300 import build as _build
    if not _build.up_to_date():
        _build.build()
    from paper_1403_1937_gb300 import eik
    from paper_1403_1937_gb300 import workloads as wl
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    data = wl.config5()
    mine = shard_instances([d[0].n for d in data], ws)[rank]
    data = [data[k] for k in mine]
    insts = [d[0] for d in data]
    opt = eik.make_options(precision=args.precision, tol=args.tol,
                           tile_override=args.tile_override, band_bits=args.band_bits,
                           inner_tol=args.inner_tol)
    b = eik.eik_create_batch(insts, opt, workers=args.workers)
    offs = np.cumsum([0] + [i.n for i in insts])
    # targets from the reference fields
    f_ref = torch.from_numpy(np.concatenate([d[2].ravel() for d in data])).cuda()
    eik.eik_set_f_batch(b, f_ref)
    S_ref, _ = eik.eik_solve_batch(b)
    recv = torch.from_numpy(np.concatenate([d[1] + offs[k] for k, d in enumerate(data)])).cuda()
    noise = torch.from_numpy(np.concatenate([d[3] for d in data])).cuda()
    T = S_ref[recv] + noise
    f_all = torch.from_numpy(np.concatenate([i.f.ravel() for i in insts])).cuda()
    n_unk = [i.n - len(np.unique(i.src_idx)) for i in insts]
    S = torch.empty(b.n, dtype=torch.float64, device="cuda")
    dLdS = torch.zeros(b.n, dtype=torch.float64, device="cuda")
    dLdf = torch.empty(b.n, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def step():
        eik.eik_set_f_batch(b, f_all)
        _, st_f = eik.eik_solve_batch(b, S_out=S)
        dLdS.index_copy_(0, recv, 2.0 * (S[recv] - T))
        _, st_a = eik.eik_grad_batch(b, dLdS, dLdf_out=dLdf)
        return st_f, st_a

    for _ in range(args.warmup):
        step()
    times, units, fwd_it, adj_it = [], 0, 0, 0
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush_l2(flush)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            st_f, st_a = step()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            fwd_it += sum(s_["inner_iters"] for s_ in st_f)
            adj_it += sum(s_["inner_iters"] for s_ in st_a)
            units += sum(u * (a["inner_iters"] + c["inner_iters"])
                         for u, a, c in zip(n_unk, st_f, st_a))
    total, units = job_totals(sum(times), units, ws, "cuda")
    if rank != 0:
        return
    loss = float(((S[recv] - T) ** 2).sum())
    line = {"metric": METRIC, "value": round(units / total / 1e9, 4), "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * total / args.steps, 3), "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64 forward, f64 adjoint",
            "data": "synthetic",
            "config": {"workload": "differentiation: 32 x 512^2 Fourier f, 1 source, hbar=0.01, "
                                   "4096 receivers each; forward + adjoint solve per step",
                       "instances": 32, "instances_rank0": len(insts),
                       "precision": args.precision, "tol_componentwise": args.tol,
                       "l2": "flushed between steps (256 MiB write)"},
            "clocks": clk.summary(),
            "iterations_per_step": {"forward": fwd_it / args.steps,
                                    "adjoint": adj_it / args.steps},
            "loss": loss}
    eik.eik_destroy_batch(b)
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_batch(args, emit=True):
    """Batched workload: independent 2D instances of uneven size, f, sources
    and hbar (config 4), solved together through eik_solve_batch."""
    import torch
    from paper_1403_1937_gb300 import build as _build
    if not _build.up_to_date():
        _build.build()
    from paper_1403_1937_gb300 import eik
    from paper_1403_1937_gb300 import workloads as wl
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    all_insts = wl.config4(count=args.c4_count)
    # independent instances: each rank solves its own share, no collective
    # on the data path
    mine = shard_instances([i.n for i in all_insts], ws)[rank]
    insts = [all_insts[k] for k in mine]
    n_unk = [i.n - len(np.unique(i.src_idx)) for i in insts]
    opt = eik.make_options(precision=args.precision, tol=args.tol,
                           tile_override=args.tile_override, band_bits=args.band_bits,
                           inner_tol=args.inner_tol, batch_pack=args.batch_pack,
                           batch_tile_rows=args.batch_tile_rows)
    b = eik.eik_create_batch(insts, opt, workers=args.workers)
    S = torch.empty(b.n, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        eik.eik_solve_batch(b, S_out=S)
    times, units = [], 0
    info0 = eik.eik_batch_info(b)
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush_l2(flush)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            _, stats = eik.eik_solve_batch(b, S_out=S)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            units += sum(u * st["inner_iters"] for u, st in zip(n_unk, stats))
    info1 = eik.eik_batch_info(b)
    total, units = job_totals(sum(times), units, ws, "cuda")
    roof = None
    if info1["packed"] and info1["pass_ms"] > info0["pass_ms"]:
        # the packed pass: 28 B per covered node (the single-grid pass's 7
        # words) over the device time of the graphs that ran the passes
        peak, peak_src = measured_peaks()
        work = info1["node_passes"] - info0["node_passes"]
        sec = (info1["pass_ms"] - info0["pass_ms"]) * 1e-3
        npass = info1["passes"] - info0["passes"]
        achieved = ALGO_BYTES_PER_NODE["mixed_cg"] * work / sec / 1e9
        # DRAM bytes per node from the committed ncu capture of an all-active
        # pass, times the nodes an average pass covered
        per_node = ncu_traffic_field("mixed_cg_packed", "c4", "dram_bytes_per_node")
        traffic = round(per_node * work / max(npass, 1)) if per_node else None
        roof = {"bound": "hbm", "kernel": "mixed_cg_packed (k_cg2d_batch)",
                "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": peak_src,
                "algorithmic_bytes_per_launch": round(ALGO_BYTES_PER_NODE["mixed_cg"] * work
                                                      / max(npass, 1)),
                "avg_launch_us": round(1e6 * sec / max(npass, 1), 2),
                "passes": npass, "node_passes": work,
                "share_of_step": round(sec / sum(times), 4)}
    if rank != 0:
        return
    line = {"metric": METRIC, "value": round(units / total / 1e9, 4), "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * total / args.steps, 3), "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": f"batched 2D: {len(all_insts)} instances, sides 64..1024, "
                                   "Fourier f in [0.5,1.5], 1-8 sources, hbar in {2h,4h,8h}",
                       "instances": len(all_insts), "instances_rank0": len(insts),
                       "nodes_rank0": int(b.n), "precision": args.precision,
                       "tol_componentwise": args.tol,
                       "l2": "flushed between steps (256 MiB write)"},
            "clocks": clk.summary(),
            "iterations": {"min": min(s_["inner_iters"] for s_ in stats),
                           "max": max(s_["inner_iters"] for s_ in stats)},
            "batch": {k: info1[k] for k in ("packed", "variant", "tile_rows", "tuned")},
            "roofline": roof}
    eik.eik_destroy_batch(b)
    if emit:
        print(json.dumps(line), flush=True)
    return line


def fft_flops(n, terms):
    """FP64 operations of the 1D transforms eik_fft_series runs on an n x n
    grid with `terms` terms, at the usual 5 N log2 N per complex transform of
    length N: transform length P = the smallest 2^a 3^b 5^c >= 2n - 1; the
    kernels' transforms (G~, and G when terms > 0) take 2P row transforms, a
    grid function's forward transform n + P and its inverse P + n."""
    P = max(2 * n - 1, 2)
    while True:
        q = P
        for fct in (2, 3, 5):
            while q % fct == 0:
                q //= fct
        if q == 1:
            break
        P += 1
    per = 5 * P * np.log2(P)
    kernels = 2 * P * (1 + (1 if terms > 0 else 0))
    data = (1 + terms) * 2 * (n + P)
    return float(per * (kernels + data))


def run_fft(args):
    """Second workload: the FFT perturbation series (Sec. 5, Table 1) on
    Example 1 of Sec. 5.4 (257^2, hbar = 0.006, T = 6) and on the same
    domain at 4x the resolution (1025^2, hbar scaled with h), timed with CUDA
    events around eik_fft_series with device-resident inputs."""
    import torch
    from paper_1403_1937_gb300 import build as _build
    if not _build.up_to_date():
        _build.build()
    from paper_1403_1937_gb300 import eik
    from paper_1403_1937_gb300 import workloads as wl
    torch.cuda.set_device(0)
    rows = []
    with Clocks(0) as clk:
        for scale in (1, 4):
            inst = wl.example1(h=2.0 ** -10 / scale, hbar=0.006 / scale)
            n = inst.dims[0]
            f = torch.from_numpy(inst.f).cuda()
            for _ in range(args.warmup):
                eik.fft_series(inst.dims, inst.h, inst.hbar, f, inst.src_idx, 6)
            ts = []
            for _ in range(args.steps):
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                eik.fft_series(inst.dims, inst.h, inst.hbar, f, inst.src_idx, 6)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            fl = fft_flops(n, 6)
            rows.append({"grid": [n, n], "hbar": inst.hbar, "terms": 6, "ms": round(ms, 3),
                         "transform_tflops": round(fl / (ms * 1e-3) / 1e12, 4)})
    peak = FP64_PEAK_TFLOPS
    # the oracle (numpy transforms, host cores) on Example 1, as it stands
    from oracle import fft_series as _fs
    inst = wl.example1()
    t0 = time.perf_counter()
    _fs.series(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx, 6)
    t_cpu = time.perf_counter() - t0
    cpu = {"value": round(1e3 * t_cpu, 1), "unit": "ms", "cores": os.cpu_count(),
           "kind": "oracle", "sample": "one evaluation of the series on Example 1 (257^2, 6 "
                                       "terms) by the oracle (numpy FFT)"}
    line = {"metric": "FFT perturbation series (Sec. 5, Table 1): time per evaluation",
            "value": rows[0]["ms"], "unit": "ms", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rows[0]["ms"], "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "Sec. 5.4 Example 1: f = exp(r) on [-0.125, 0.125]^2, "
                                   "one source at the origin, 6 terms",
                       "grids": rows},
            "roofline": {"bound": "fp64", "kernel": "k_fft_rows (all transforms)",
                         "achieved": rows[-1]["transform_tflops"], "peak": peak,
                         "unit": "TFLOP/s",
                         "frac": round(rows[-1]["transform_tflops"] / peak, 4),
                         "traffic": None, "peak_source": "nominal FP64 rate (no measured "
                                                         "FP64 peak on this pool)",
                         "note": "5 N log2 N per transform over the whole call (pointwise "
                                 "kernels and the Green's function samples included in the "
                                 "time)"},
            "cpu_baseline": cpu,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_paths(args):
    """The path-planning and shape-from-shading kernels: nodal gradient of S
    (eik_grad_S) and backtracking of 4096 paths (eik_backtrack) on the
    mixed-precision solution of the 2048^2 workload, and the forcing of a
    2048^2 Lambertian image of a paraboloid (eik_sfs_forcing); CUDA events
    around each call, device-resident inputs.  The oracle (oracle/paths.py,
    oracle/sfs.py) is timed on the same inputs (gradient, forcing) and on 64
    of the paths."""
    import torch
    from paper_1403_1937_gb300 import build as _build
    if not _build.up_to_date():
        _build.build()
    from paper_1403_1937_gb300 import eik
    from paper_1403_1937_gb300 import workloads as wl
    from oracle import paths as opaths, sfs as osfs
    torch.cuda.set_device(0)
    inst = wl.config2()
    n = inst.n
    f = torch.from_numpy(np.ascontiguousarray(inst.f)).cuda()
    h = eik.eik_create(inst.dims, inst.h, inst.hbar, f, inst.src_idx, None,
                       eik.make_options(precision="mixed", tol=1e-6))
    S, _, _ = eik.eik_solve(h)
    eik.eik_destroy(h)
    rng = np.random.default_rng(1937)
    hi = np.array([(d - 1) * inst.h for d in inst.dims])
    starts = rng.uniform(0, 1, (4096, 2)) * hi
    step, eps, ms = 0.5 * inst.h, 2.0 * inst.h, 8192
    nx = inst.dims[0]
    X, Y = np.meshgrid(np.arange(nx) * inst.h, np.arange(inst.dims[1]) * inst.h)
    Pimg = torch.from_numpy(osfs.image_of_height(
        ((1.4 * (X - 0.5)) ** 2 + (1.4 * (Y - 0.5)) ** 2)).ravel()).cuda()

    def timed(fn, reps):
        for _ in range(max(1, args.warmup)):
            out = fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    peak, peak_src = measured_peaks()
    with Clocks(0) as clk:
        ms_g, G = timed(lambda: eik.grad_S(S, inst.dims, inst.h), 20)
        ms_b, (P, L, st) = timed(lambda: eik.backtrack(G, inst.dims, inst.h, starts,
                                                       inst.src_idx, step, ms, eps), 3)
        ms_f, _ = timed(lambda: eik.sfs_forcing(Pimg, 1e-3), 20)
    steps = int(L.sum().item())
    gbs_g = 24.0 * n / (ms_g * 1e-3) / 1e9      # read S, write 2 gradient components
    gbs_f = 16.0 * n / (ms_f * 1e-3) / 1e9      # read P, write f
    # oracle, as it stands, on the host cores
    S_h, G_h, P_h = S.cpu().numpy(), G.cpu().numpy(), Pimg.cpu().numpy()
    t0 = time.perf_counter()
    opaths.grad_S(S_h, inst.dims, inst.h)
    t_g = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, L_ref, _ = opaths.backtrack(G_h, inst.dims, inst.h, starts[:64], step, ms, inst.src_idx,
                                   eps)
    t_b = time.perf_counter() - t0
    t0 = time.perf_counter()
    osfs.forcing(P_h, 1e-3)
    t_f = time.perf_counter() - t0
    line = {"metric": "path planning (nodal grad S + Euler backtracking) and shape-from-shading "
                      "forcing: path steps per second",
            "value": round(steps / (ms_b * 1e-3), 1), "unit": "path steps/s", "n_gpus": 1,
            "steps": 3, "warmup": max(1, args.warmup), "ms_per_step": round(ms_b, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "2048^2 mixed solution of the 2D workload; 4096 uniformly "
                                   "random start points, step h/2, stop within 2h of a source; "
                                   "2048^2 image of a paraboloid",
                       "paths": 4096, "path_steps": steps, "reached": int((st == 0).sum().item())},
            "kernels": {
                "grad_S": {"ms": round(ms_g, 4), "achieved_gbs": round(gbs_g, 1),
                           "frac_of_hbm": round(gbs_g / peak, 4), "bytes_per_node": 24},
                "backtrack": {"ms": round(ms_b, 3), "path_steps": steps},
                "sfs_forcing": {"ms": round(ms_f, 4), "achieved_gbs": round(gbs_f, 1),
                                "frac_of_hbm": round(gbs_f / peak, 4), "bytes_per_node": 16}},
            # grad S does two correctly rounded FP64 divisions and two
            # subtractions per node (bit-identical to the oracle's arithmetic),
            # and GB300's FP64 unit, not HBM, bounds it
            "roofline": {"bound": "alu", "kernel": "grad_S",
                         "achieved": round(4.0 * n / (ms_g * 1e-3) / 1e12, 4),
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": round(4.0 * n / (ms_g * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, 4),
                         "traffic": None, "peak_source": "nominal FP64 rate",
                         "note": "4 FP64 operations per node, a division counted as one; "
                                 f"the same pass moves {gbs_g:.0f} GB/s of its 24 B per node"},
            "cpu_baseline": {"value": round(int(L_ref.sum()) / t_b, 1), "unit": "path steps/s",
                             "cores": 1, "kind": "oracle",
                             "sample": f"64 of the paths ({t_b:.1f} s); grad S {1e3 * t_g:.0f} ms, "
                                       f"forcing {1e3 * t_f:.0f} ms on the full grids"},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def roofline(res, inst, wname, only=None):
    peak, peak_src = measured_peaks()
    km = {k: v for k, v in res["kernel_ms"].items() if v[0] is not None}
    cand = {k: v for k, v in km.items() if k in ALGO_BYTES_PER_NODE and
            (only is None or k == only) and (only is not None or k != "mixed_mg")}
    if not cand:
        return None
    dom = max(cand, key=lambda k: cand[k][2])
    avg_ms = cand[dom][0]
    total = sum(v[2] for v in km.values())
    if dom.startswith("cg_"):
        flops = ALGO_FLOPS_PER_NODE[(dom, len(inst.dims))] * inst.n
        achieved = flops / (avg_ms * 1e-3) / 1e12
        return {"bound": "alu", "kernel": dom, "achieved": round(achieved, 4),
                "peak": FP64_PEAK_TFLOPS,
                "peak_source": "nominal FP64 rate (152 SMs x 2.07 GHz x 4 FLOP/clock)",
                "unit": "TFLOP/s", "frac": round(achieved / FP64_PEAK_TFLOPS, 4),
                "traffic": ncu_traffic(dom, wname),
                "algorithmic_flops_per_launch": flops,
                "algorithmic_bytes_per_launch": ALGO_BYTES_PER_NODE[dom] * inst.n,
                "avg_launch_ms": avg_ms,
                "share_of_kernel_time": round(cand[dom][2] / total, 3) if total else None}
    algo = algo_bytes(dom, inst) * inst.n
    achieved = algo / (avg_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1),
            "peak": peak, "peak_source": peak_src, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": ncu_traffic(dom, wname),
            "algorithmic_bytes_per_launch": algo, "avg_launch_ms": avg_ms,
            "share_of_kernel_time": round(cand[dom][2] / total, 3) if total else None}


def cpu_baseline(inst, iters):
    from oracle import cg, fd
    sysm = fd.assemble(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    thr = cg.threads()
    if iters <= 0:
        t1 = cg.time_iterations(sysm, 5)
        iters = int(max(10, min(2000, 15.0 / max(t1 / 5, 1e-6))))
    t = cg.time_iterations(sysm, iters)
    n_unk = len(sysm.unk)
    return {"value": n_unk * iters / t / 1e9, "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": f"{iters} Jacobi-PCG iterations of the C/OpenMP oracle on the full "
                      f"{'x'.join(map(str, inst.dims))} system ({n_unk} unknowns), "
                      f"{t:.1f} s"}


def run_reference(args):
    """Reference arm: the CPU oracle timed on the host cores (rank 0 only)."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import cg, fd
    inst, desc = workload(args.workload)
    sysm = fd.assemble(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    n_unk = len(sysm.unk)
    thr = cg.threads()
    t1 = cg.time_iterations(sysm, 3) / 3
    per_step = int(max(5, min(500, 4.0 / max(t1, 1e-6))))
    for _ in range(args.warmup):
        cg.time_iterations(sysm, per_step)
    times = [cg.time_iterations(sysm, per_step) for _ in range(args.steps)]
    total = sum(times)
    value = n_unk * per_step * args.steps / total / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(desc, sample=f"{per_step} CG iterations per step"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                             "sample": f"{per_step} Jacobi-PCG iterations per step of the "
                                       f"C/OpenMP oracle on the full system ({n_unk} "
                                       f"unknowns)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def other_blocks(args):
    """The batched workload (packed, autotuned; 1 warm-up + 2 timed solves)
    and the differentiation workload (1 + 1 steps), each as a compact summary
    of its own bench line, for the default single-GPU run."""
    import copy
    out = {}
    a4 = copy.copy(args)
    a4.workload, a4.tol, a4.steps, a4.warmup = "c4", 1e-7, 2, 1
    a4.tile_override, a4.batch_pack, a4.batch_tile_rows = 0, 0, 0
    l4 = run_batch(a4, emit=False)
    out["c4"] = {k: l4[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup", "iterations",
                                    "batch", "roofline", "clocks")}
    out["c4"]["workload"] = l4["config"]["workload"]
    a5 = copy.copy(args)
    a5.workload, a5.tol, a5.steps, a5.warmup = "c5", 1e-6, 1, 1
    a5.tile_override, a5.batch_pack, a5.batch_tile_rows = 0, 0, 0
    l5 = run_diff(a5, emit=False)
    out["c5"] = {k: l5[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup",
                                    "iterations_per_step", "dtype", "clocks")}
    out["c5"]["workload"] = l5["config"]["workload"]
    return out


def main():
    args = parse()
    if args.tol is None:
        args.tol = 1e-7 if args.workload == "c4" else 1e-6
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "c4":
        run_batch(args)
        return
    if args.workload == "c5":
        run_diff(args)
        return
    if args.workload == "fft":
        run_fft(args)
        return
    if args.workload == "paths":
        run_paths(args)
        return
    inst, desc, n_unk, results, ws, rank = run_ours(args)
    c3 = None
    if args.workload == "c2" and not args.no_c3_block:
        c3 = secondary_block(args, ws, int(os.environ.get("LOCAL_RANK", "0")))
    batch_blocks = {}
    if args.workload == "c2" and not args.no_c3_block and ws == 1:
        # the batched and differentiation workloads, briefly, in the same run
        batch_blocks = other_blocks(args)
    if rank != 0:
        return
    head_mode = "mixed_mg" if args.modes == "mg" else args.precision
    head = results.get(head_mode, {})
    if "glups" not in head:
        print(json.dumps({"metric": METRIC, "error": head.get("error", "failed")}), flush=True)
        sys.exit(1)
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(inst, args.cpu_iters)
    comparison = {}
    for mode, r in results.items():
        if "glups" in r:
            comparison[mode] = {"glups": round(r["glups"], 3),
                                "ms_per_step": round(r["ms_per_step"], 3),
                                "cg_iters_per_step": r["cg_iters_per_step"],
                                "res_cw": r["stats_last"]["res_cw"]}
        else:
            comparison[mode] = r
    if "glups" in results.get("fp64", {}) and "glups" in results.get("mixed", {}):
        comparison["mixed_speedup_vs_fp64"] = round(
            results["fp64"]["ms_per_step"] / results["mixed"]["ms_per_step"], 3)
    mg = results.get("mixed_mg", {})
    if "glups" in mg:
        # time to solution of the multigrid-preconditioned mixed solve; its
        # GLUPS counts multigrid iterations, so the comparison is by time
        comparison["mixed_mg"]["tol_componentwise"] = args.mg_tol
        comparison["mixed_mg"]["roofline_iteration"] = roofline(mg, inst, args.workload,
                                                                only="mixed_mg")
        for ref in ("fp64", "mixed"):
            if "glups" in results.get(ref, {}):
                comparison[f"mixed_mg_speedup_vs_{ref}"] = round(
                    results[ref]["ms_per_step"] / mg["ms_per_step"], 3)
    line = {
        "metric": METRIC, "value": round(head["glups"], 4), "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(head["ms_per_step"], 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if head_mode == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": dict(desc, precision=head_mode,
                       tol_componentwise=args.mg_tol if head_mode == "mixed_mg" else args.tol,
                       l2="flushed between steps (256 MiB write)",
                       parallelism="replicas" if ws > 1 else "single GPU"),
        "e2e": head.get("e2e"),
        "gpu_launches": head["gpu_launches"],
        "clocks": head["clocks"],
        "roofline": roofline(head, inst, args.workload,
                             only="mixed_mg" if head_mode == "mixed_mg" else None),
        "cpu_baseline": cpu,
        "comparison": comparison,
        "kernels": kernel_table(head, inst),
    }
    if c3 is not None:
        line["c3"] = c3
    line.update(batch_blocks)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
