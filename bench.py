#!/usr/bin/env python
"""Benchmark of the domain-wall solver on one GB300 (or N, one process each).

One step = one full pass of the solver's hot path for one 4D source on the
32^3x64, Ls=16 Mobius workload (b=1.5, c=0.5, M0=1.8, m=0.005, links
exp(0.3 i H) + 3 stout/APE smearing steps, rho=0.1; Neff form, alpha 0.5):
5D source, FP64 even-odd set-up, CG on the normal equation in FP32 (the
paper's single-precision solver) with FP64 reliable updates, reconstruction,
FP64 full-residual check, 4D projection.  The JSON line reports the time to
solution at ||b5 - D x5|| / ||b5|| <= 1e-10 (lower is better), the hop
kernel's HBM roofline, the measured FP32 arithmetic peak, the oracle's CPU
time on a bounded sample, the end-to-end time through the host-buffer C-ABI
call and the SM clocks seen; beside it the FP16-inner solve, plain FP64 CG
and the 16^3x32 workload.

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

WORKLOAD = "c5_32^3x64_ls16_mobius"        # the largest single-GPU workload: the headline
SECOND = "c2_16^3x32_ls16_mobius"          # reported beside it (extra keys)
# the oracle's bounded sample: the workload's operator on an 8^3x16 lattice of
# the same link recipe (1/256 of the 32^3x64 volume); its time per CG iteration
# is scaled by the volume ratio (the oracle is a loop over sites)
SAMPLE_DIMS = (8, 8, 8, 16)
METRIC = "DWF CG time-to-solution @1e-10 residual; 5D Dslash GB/s vs HBM peak"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--inner", default="f32", choices=["f16", "f32", "f64"])
    ap.add_argument("--form", default="neff", choices=["neff", "standard"])
    ap.add_argument("--alpha", type=float, default=0.5)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-cg", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP16-inner solve and the 16^3x32 lines reported beside the headline")
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


HOP_SOURCES = ("hop.cu", "hop_kernels.cuh", "stencil.cuh", "fields.cuh", "tcgen05.cuh")


def hop_source_key():
    """sha256 (16 hex digits) of the source files the hop kernel is compiled
    from and of its argument struct (HopArgs in dwf_internal.h)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2602_14454_gb300", "csrc")
    for f in HOP_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    txt = open(os.path.join(csrc, "dwf_internal.h"), "rb").read()
    a = txt.index(b"struct HopArgs {")
    h.update(txt[a:txt.index(b"};", a) + 2])
    return h.hexdigest()[:16]


def hop_traffic(prec, workload, variant, sweep):
    """DRAM bytes per hop launch from the committed ncu summary, if it was taken
    from the current hop kernel sources on this workload with the same variant
    and sweep order (else null)."""
    path = os.path.join(ROOT, "profiles", "hop_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    e = d.get(workload, {}).get(prec)
    if not e or e.get("hop_sources_sha256_16") != hop_source_key():
        return None
    if e.get("variant") != variant or e.get("sweep_zblock") != sweep:
        return None
    return e.get("dram_bytes_per_launch")


def config_of(w, name, args):
    """The workload as both arms name it."""
    return {"workload": name, "dims": list(w["dims"]), "Ls": w["Ls"], "b": w["b"], "c": w["c"],
            "M0": w["M0"], "mf": w["mf"], "form": args.form, "alpha": args.alpha,
            "inner_precision": args.inner, "tol": args.tol,
            "links": "exp(i %.1f H), %d stout/APE steps rho 0.1, seed %d" % (w["eps"], w["smear"], w["gauge_seed"]),
            "source": "Gaussian 4D, seed %d (+ rank)" % w["src_seed"]}


def oracle_iteration_seconds(w, form, alpha):
    """The FP64 oracle as it stands, on the host cores: one CG iteration (the
    even-odd matrix and its adjoint) with the workload's operator on the
    SAMPLE_DIMS lattice of the same link and source recipe."""
    from oracle import dwf as orc
    from paper_2602_14454_gb300 import inputs
    U = inputs.smeared_links(SAMPLE_DIMS, w["eps"], 0.1, w["smear"], w["gauge_seed"])
    ref = orc.DWF(U, SAMPLE_DIMS, w["Ls"], w["M0"], w["mf"], w["b"], w["c"], form=form, alpha=alpha)
    x = ref.to_eo(inputs.gaussian_5d(SAMPLE_DIMS, w["Ls"], 1), 0)

    def one():
        t0 = time.perf_counter()
        y = ref.d_pc(x)
        ref.d_pc(y, dag=True)
        return time.perf_counter() - t0
    return one


def volume(dims):
    v = 1
    for d in dims:
        v *= int(d)
    return v


def sample_text(w, iters):
    return ("one CG iteration (D and D^dag of the even-odd matrix) of the workload's operator on a "
            "%s lattice with the same link recipe, times the volume ratio %d, times the %d iterations "
            "FP64 CG takes on the workload" % ("x".join(map(str, SAMPLE_DIMS)),
                                               volume(w["dims"]) // volume(SAMPLE_DIMS), iters))


def cpu_baseline(w, iters, form, alpha):
    one = oracle_iteration_seconds(w, form, alpha)
    one()
    t = min(one(), one())
    scale = volume(w["dims"]) / volume(SAMPLE_DIMS)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": t * scale * iters, "unit": "s", "cores": cores, "kind": "oracle",
            "sample": sample_text(w, iters), "seconds_per_sample_iteration": t}


def reference_arm(args):
    """--impl reference: the FP64 oracle on the host cores (there is no other
    implementation: the paper is the only reference), on the same workload,
    metric and config; each step times one bounded sample (cpu_baseline)."""
    from paper_2602_14454_gb300 import inputs
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    w = inputs.WORKLOADS[args.workload]
    iters = fp64_iteration_count(args.workload)
    one = oracle_iteration_seconds(w, args.form, args.alpha)
    times = []
    for k in range(args.warmup + args.steps):
        dt = one()
        if k >= args.warmup:
            times.append(dt)
    t_it = sum(times) / len(times)
    val = t_it * volume(w["dims"]) / volume(SAMPLE_DIMS) * iters
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t_it,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w, args.workload, args),
            "cpu_baseline": {"value": val, "unit": "s", "cores": cores, "kind": "oracle",
                             "sample": "each step: " + sample_text(w, iters) + "; value = mean step time "
                                       "x volume ratio x iterations"},
            "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def fp64_iteration_count(name):
    """Iterations of plain FP64 CG on the workload to 1e-10, as measured on the
    GPU and recorded in profiles/iteration_counts.json (else a default stated
    in the line)."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "iteration_counts.json")))
        return int(d[name]["fp64_cg_iterations"])
    except Exception:
        return 350


def timed_solves(op, b4, n, **kw):
    """Mean CUDA-event time (s) of n solves from a 4D source (5D source, solve,
    projection) after one untimed solve, and the last solve's statistics."""
    import torch
    st = torch.cuda.current_stream()

    def step():
        b5 = op.source_5d(b4)
        x5, s = op.solve(b5, **kw)
        op.project_4d(x5)
        return s
    step()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(n):
        s = step()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0 / n, s


KERNEL_NAMES = {0: "hop_kernel", 3: "hop_sweep_kernel", 4: "hop_block_kernel", 5: "hop_kernel_occ (FP16 projection)",
                7: "hop_lean_kernel", 9: "hop_wa_kernel (warp-autonomous)",
                10: "hop_tc_kernel (warp tiles, tcgen05 mixing)"}


def hop_roofline(op, prec, Ls, peak, reps=30):
    """The hop kernel (the dominant kernel) timed alone with CUDA events, L2
    flushed between launches, against the measured HBM peak."""
    us, nbytes = op.time_hop(prec, reps=reps, flush_l2=True)
    achieved = nbytes / (us * 1e-6) / 1e9
    var, ns, sb = op.hop_config(prec)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "us_per_launch": us, "algorithmic_bytes_per_launch": nbytes,
            "kernel": "%s<%s> variant %d (even-odd hop + fused Ls mixing)" % (KERNEL_NAMES.get(var, "hop"), prec, var),
            "config": {"variant": var, "ns": ns, "sb": sb, "sweep_zblock": op.sweep(prec)}}


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
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
    w = inputs.WORKLOADS[args.workload]
    U = inputs.workload_links(w, device="cuda")
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

    # roofline of the dominant kernel (the hop in the inner precision)
    pk = peaks()
    peak = pk["hbm_gbs"] if pk else 6800.0
    roof = hop_roofline(op, args.inner, w["Ls"], peak)
    roof["traffic"] = hop_traffic(args.inner, args.workload, roof["config"]["variant"], roof["config"]["sweep_zblock"])
    roof["peak_source"] = ("MEASURED_PEAKS.json hbm_gbs (burst copy), of measured" if pk
                           else "fallback 6.8 TB/s")
    iteration = op.time_iteration(args.inner, reps=10, flush_l2=True) if args.inner != "f64" else None
    alu = dwf.alu_peaks()
    alu_peak = max(alu["fp32_ffma_tflops"], alu["fp32_ffma2_tflops"])
    hop_flops = float(op.V // 2) * w["Ls"] * (1320 + 48 * w["Ls"])

    out = None
    if rank == 0:
        fp64 = None
        if not args.no_fp64_cg and args.inner != "f64":
            t64, s64 = timed_solves(op, b4, 1, inner_prec="f64", tol=args.tol)
            fp64 = {"tts_s": t64, "iterations": s64["iterations"], "true_residual": s64["true_residual"],
                    "speedup_of_headline": t64 / (ms / 1000.0)}
        extras = None
        if not args.no_extras:
            extras = {}
            other = "f16" if args.inner != "f16" else "f32"
            t2, s2b = timed_solves(op, b4, 2, inner_prec=other, tol=args.tol)
            extras["%s_inner" % other] = {
                "tts_s": t2, "iterations": s2b["iterations"], "true_residual": s2b["true_residual"],
                "roofline": hop_roofline(op, other, w["Ls"], peak)}
            w2 = inputs.WORKLOADS[SECOND]
            op2 = dwf.Operator(w2["dims"], w2["Ls"], w2["M0"], w2["mf"], w2["b"], w2["c"], form=args.form,
                               alpha=args.alpha)
            op2.set_gauge(torch.from_numpy(inputs.workload_links(w2, device="cuda")).cuda())
            b42 = torch.from_numpy(inputs.gaussian_4d(w2["dims"], w2["src_seed"])).cuda()
            c2 = {"config": config_of(w2, SECOND, args)}
            for prec in ("f32", "f16"):
                t, s_ = timed_solves(op2, b42, 5, inner_prec=prec, tol=args.tol)
                c2["%s_inner" % prec] = {"tts_s": t, "iterations": s_["iterations"],
                                         "true_residual": s_["true_residual"],
                                         "roofline": hop_roofline(op2, prec, w2["Ls"], peak)}
            it2 = op2.time_iteration("f32", reps=10, flush_l2=True)
            c2["iteration_kernels_f32"] = {k: {"us": round(v[0], 2), "gbs": round(v[1] / (v[0] * 1e-6) / 1e9, 1)}
                                           for k, v in it2.items()}
            extras[SECOND] = c2
            op2.close()
        base = None
        if world == 1 and not args.no_cpu_baseline:
            its = fp64["iterations"] if fp64 else fp64_iteration_count(args.workload)
            base = cpu_baseline(w, its, args.form, args.alpha)
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
            "config": dict(config_of(w, args.workload, args),
                           l2="inputs larger than L2 (solve working set %.1f GB)" % (op.device_bytes() / 1e9)),
            "solve": {"iterations": iters, "true_residual_max": worst_res,
                      "reliable_updates": stats[-1]["reliable_updates"],
                      "d_applications": stats[-1]["d_applications"], "solves_per_s_all_ranks":
                          world * 1000.0 / ms},
            "fp64_cg": fp64,
            "roofline": roof,
            # the same launch against the measured FP32 arithmetic peak (packed FP32x2
            # FMAs, dwf_alu_peaks); useful flops per 5D site: 1320 (Wilson hop) + 48 Ls
            # (one dense Ls mixing)
            "roofline_alu": {"bound": "alu", "achieved": hop_flops / (roof["us_per_launch"] * 1e-6) / 1e12,
                             "peak": alu_peak, "unit": "TFLOP/s",
                             "frac": hop_flops / (roof["us_per_launch"] * 1e-6) / 1e12 / alu_peak,
                             "flops_per_launch": hop_flops, "peak_source": "dwf_alu_peaks, measured",
                             "measured_peaks": alu},
            "iteration_kernels": None if iteration is None else {
                "kernels": {k: {"us": round(v[0], 2), "bytes": v[1], "gbs": round(v[1] / (v[0] * 1e-6) / 1e9, 1)}
                            for k, v in iteration.items()},
                "us": sum(v[0] for v in iteration.values()),
                "frac_of_hbm_peak": sum(v[1] for v in iteration.values()) /
                                    (sum(v[0] for v in iteration.values()) * 1e-6) / 1e9 / peak},
            "extras": extras,
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
