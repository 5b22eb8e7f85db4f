#!/usr/bin/env python
"""Benchmark of the domain-wall solver on one GB300 (or N, one process each).

One step = one full pass of the solver's hot path for one 4D source on the
16^3x32, Ls=16 Mobius workload (b=1.5, c=0.5, M0=1.8, m=0.01, links
exp(0.3 i H) + 3 stout/APE smearing steps, rho=0.1): 5D source, FP64 even-odd
set-up, mixed-precision CG with FP64 reliable updates, reconstruction, FP64
full-residual check, 4D projection.  The JSON line reports the time to
solution at ||b5 - D x5|| / ||b5|| <= 1e-10 (lower is better), the hop
kernel's HBM roofline, the oracle's CPU time on a bounded sample, the
end-to-end time through the host-buffer C-ABI call and the SM clocks seen.

Ranks (torchrun) solve independent sources (weak scaling, no collective);
--impl reference times the FP64 oracle on the host cores instead.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "c2_16^3x32_ls16_mobius"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
METRIC = "DWF CG time-to-solution @1e-10 residual; 5D Dslash GB/s vs HBM peak"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--inner", default="f16", choices=["f16", "f32", "f64"])
    ap.add_argument("--form", default="neff", choices=["neff", "standard"])
    ap.add_argument("--alpha", type=float, default=0.5)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-cg", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def source_seed(w, rank):
    """Each rank solves its own source (independent systems, weak scaling)."""
    return w["src_seed"] + rank


def max_over_ranks(x):
    """The largest x over the ranks of the process group (x itself without one);
    the only collective of the benchmark (timing, not data)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, n in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(rows)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


HOP_SOURCES = ("hop.cu", "stencil.cuh", "fields.cuh", "dwf_internal.h")


def hop_source_key():
    """sha256 (16 hex digits) of every source file the hop kernel is compiled from."""
    h = hashlib.sha256()
    for f in HOP_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2602_14454_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def hop_traffic(prec):
    """DRAM bytes per hop launch from the committed ncu summary, if it was taken
    from the current hop kernel sources (else null)."""
    path = os.path.join(ROOT, "profiles", "hop_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    e = d.get(prec)
    if not e or e.get("hop_sources_sha256_16") != hop_source_key():
        return None
    return e.get("dram_bytes_per_launch_full_size")


def cpu_baseline(w, U, fp64_iters, form, alpha):
    """The FP64 oracle as it stands, on the host cores: one application of the
    even-odd matrix and one of its adjoint on the same workload (one CG
    iteration), extrapolated to the iteration count of FP64 CG on it."""
    import numpy as np
    from oracle import dwf as orc
    from paper_2602_14454_gb300 import inputs
    ref = orc.DWF(U, w["dims"], w["Ls"], w["M0"], w["mf"], w["b"], w["c"], form=form, alpha=alpha)
    x = ref.to_eo(inputs.gaussian_5d(w["dims"], w["Ls"], 1), 0)
    t0 = time.perf_counter()
    y = ref.d_pc(x)
    ref.d_pc(y, dag=True)
    t_it = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": t_it * fp64_iters, "unit": "s", "cores": cores, "kind": "oracle",
            "sample": "one CG iteration (D and D^dag of the even-odd matrix, %.1f s) on the full "
                      "workload, times the %d iterations FP64 CG needs on it" % (t_it, fp64_iters),
            "seconds_per_iteration": t_it}


def reference_arm(args):
    """--impl reference: the FP64 oracle on the host cores, same workload."""
    import numpy as np  # noqa: F401
    from paper_2602_14454_gb300 import inputs
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    w = inputs.WORKLOADS[WORKLOAD]
    U = inputs.workload_links(w)
    from oracle import dwf as orc
    ref = orc.DWF(U, w["dims"], w["Ls"], w["M0"], w["mf"], w["b"], w["c"], form=args.form, alpha=args.alpha)
    x = ref.to_eo(inputs.gaussian_5d(w["dims"], w["Ls"], 1), 0)
    iters = fp64_iteration_count()
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        y = ref.d_pc(x)
        ref.d_pc(y, dag=True)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    t_it = sum(times) / len(times)
    val = t_it * iters
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t_it,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "dims": list(w["dims"]), "Ls": w["Ls"],
                                            "form": args.form, "alpha": args.alpha},
            "cpu_baseline": {"value": val, "unit": "s", "cores": cores, "kind": "oracle",
                             "sample": "each step: one CG iteration (D and D^dag of the even-odd matrix) "
                                       "on the full workload; value = mean step time x %d FP64 CG "
                                       "iterations" % iters},
            "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def fp64_iteration_count():
    """Iterations of plain FP64 CG on the workload to 1e-10 (from profiles/, else a
    conservative default stated in the line)."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "iteration_counts.json")))
        return int(d[WORKLOAD]["fp64_cg_iterations"])
    except Exception:
        return 300


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2602_14454_gb300 import build, dwf, inputs
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    w = inputs.WORKLOADS[WORKLOAD]
    U = inputs.workload_links(w)
    op = dwf.Operator(w["dims"], w["Ls"], w["M0"], w["mf"], w["b"], w["c"], form=args.form, alpha=args.alpha)
    op.set_gauge(torch.from_numpy(U).cuda())
    b4_host = inputs.gaussian_4d(w["dims"], source_seed(w, rank))
    b4 = torch.from_numpy(b4_host).cuda()
    st = torch.cuda.current_stream()
    kw = dict(inner_prec=args.inner, tol=args.tol)

    def step():
        b5 = op.source_5d(b4)
        x5, s = op.solve(b5, **kw)
        x4 = op.project_4d(x5)
        return x4, s

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    stats = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    l0 = op.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        x4, s = step()
        stats.append(s)
    e1.record(st)
    torch.cuda.synchronize()
    launches = op.launch_count() - l0
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
        ms = max_over_ranks(ms)
    worst_res = max(s["true_residual"] for s in stats)
    iters = stats[-1]["iterations"]

    # end to end: host buffers through the public C-ABI call
    e2e_times = []
    for _ in range(2):
        t0 = time.perf_counter()
        x4h, s2 = op.propagator_host(b4_host, **kw)
        e2e_times.append(time.perf_counter() - t0)
    e2e = min(e2e_times)

    # roofline of the dominant kernel (the hop), CUDA events around each launch, L2 flushed
    hop_prec = args.inner
    us, nbytes = op.time_hop(hop_prec, reps=30, flush_l2=True)
    iteration = op.time_iteration(hop_prec, reps=10, flush_l2=True)
    pk = peaks()
    peak = pk["hbm_gbs"] if pk else 6800.0
    achieved = nbytes / (us * 1e-6) / 1e9
    hop_flops = float(op.V // 2) * w["Ls"] * (1320 + 48 * w["Ls"])

    out = None
    if rank == 0:
        fp64 = None
        if not args.no_fp64_cg:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b5 = op.source_5d(b4)
            _, s64 = op.solve(b5, inner_prec="f64", tol=args.tol)
            torch.cuda.synchronize()
            fp64 = {"tts_s": time.perf_counter() - t0, "iterations": s64["iterations"],
                    "true_residual": s64["true_residual"]}
        base = None
        if world == 1 and not args.no_cpu_baseline:
            its = fp64["iterations"] if fp64 else fp64_iteration_count()
            base = cpu_baseline(w, U, its, args.form, args.alpha)
        out = {
            "metric": METRIC,
            "value": ms / 1000.0,
            "unit": "s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": max(3, args.warmup),
            "ms_per_step": ms,
            "higher_is_better": False,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "%s+f64" % args.inner,
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "dims": list(w["dims"]), "Ls": w["Ls"], "b": w["b"], "c": w["c"],
                       "M0": w["M0"], "mf": w["mf"], "form": args.form, "alpha": args.alpha,
                       "inner_precision": args.inner, "tol": args.tol,
                       "l2": "inputs larger than L2 (solve working set %.1f GB)" % (op.device_bytes() / 1e9)},
            "solve": {"iterations": iters, "true_residual_max": worst_res,
                      "reliable_updates": stats[-1]["reliable_updates"],
                      "d_applications": stats[-1]["d_applications"], "solves_per_s_all_ranks":
                          world * 1000.0 / ms},
            "fp64_cg": fp64,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": hop_traffic(hop_prec),
                         "kernel": "hop_kernel<%s> (even-odd hop + fused Ls mixing)" % hop_prec,
                         "us_per_launch": us, "algorithmic_bytes_per_launch": nbytes,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy), of measured" if pk
                         else "fallback 6.8 TB/s"},
            # cross-check: the same launch against the FP32 arithmetic peak derived from the
            # unit counts (152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz = 80.5 TFLOP/s); the
            # hop's useful flops per 5D site are 1320 (Wilson hop) + 48 Ls (dense Ls mixing)
            "roofline_alu": {"bound": "alu", "achieved": hop_flops / (us * 1e-6) / 1e12,
                             "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": hop_flops / (us * 1e-6) / 1e12 / FP32_PEAK_TFLOPS,
                             "flops_per_launch": hop_flops},
            # the five launches of one inner CG iteration (back to back, L2 flushed before
            # each iteration): device time and algorithmic bytes per launch
            "iteration_kernels": {
                "kernels": {k: {"us": round(v[0], 2), "bytes": v[1], "gbs": round(v[1] / (v[0] * 1e-6) / 1e9, 1)}
                            for k, v in iteration.items()},
                "us": sum(v[0] for v in iteration.values()),
                "frac_of_hbm_peak": sum(v[1] for v in iteration.values()) /
                                    (sum(v[0] for v in iteration.values()) * 1e-6) / 1e9 / peak},
            "cpu_baseline": base,
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": int(b4_host.nbytes),
                    "d2h_bytes_per_step": int(b4_host.nbytes), "true_residual": s2["true_residual"]},
            "gpu_launches": int(launches),
            "gpu_launches_per_step": int(launches // args.steps),
            "clocks": clk,
        }
        print(json.dumps(out))
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
