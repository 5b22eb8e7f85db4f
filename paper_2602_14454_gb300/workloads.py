"""Measurement runs of the larger workloads (one JSON line each).

    python -m paper_2602_14454_gb300.workloads batch      # 24^3x48: 12 point sources x 3 masses x Ls {8,12,16}
    python -m paper_2602_14454_gb300.workloads learned    # 16^4, Ls 16: train on 256 sources, FCG vs CG
    python -m paper_2602_14454_gb300.workloads large      # 32^3x64, Ls 16: mixed precision vs FP64 CG
    python -m paper_2602_14454_gb300.workloads alpha      # 16^3x32, Ls 16: iterations against alpha
    python -m paper_2602_14454_gb300.workloads alpha --spectrum   # ... and the condition number
    python -m paper_2602_14454_gb300.workloads delta      # 32^3x64: reliable-update threshold against time
    python -m paper_2602_14454_gb300.workloads eo5        # 16^3x32 Shamir: the 4D against the 5D even-odd split

Every run uses the seeded generators of ``inputs``; times are wall clock
around the library call after a synchronisation (device work included).
"""

import argparse
import json
import time


def _sync():
    import torch
    torch.cuda.synchronize()


def _links(w):
    import torch
    from . import inputs
    return torch.from_numpy(inputs.workload_links(w, device="cuda")).cuda()


def run_batch(args):
    import torch
    from . import dwf, inputs
    w = inputs.WORKLOADS["c3_24^3x48_batched"]
    dims = w["dims"]
    if args.small:
        dims = (8, 8, 8, 16)
        w = dict(w, dims=dims)
    U = _links(w)
    ops = {}
    for Ls in w["Ls_list"]:
        for mf in w["mf_list"]:
            op = dwf.Operator(dims, Ls, w["M0"], mf, w["b"], w["c"], form="standard")
            op.set_gauge(U)
            ops[(Ls, mf)] = op
    hs, b4s = [], []
    for spin in range(4):
        for col in range(3):
            b4 = torch.from_numpy(inputs.point_source(dims, spin=spin, colour=col)).cuda()
            for key, op in ops.items():
                hs.append(op)
                b4s.append(b4)
    _sync()
    t0 = time.perf_counter()
    x4s, st = dwf.solve_batch(hs, b4s, inner_prec=args.inner, tol=1e-10, batch_wave=args.wave)
    _sync()
    dt = time.perf_counter() - t0
    out = {"workload": "c3_24^3x48_batched" if not args.small else "batched 8^3x16 (reduced)",
           "dims": list(dims), "systems": len(hs), "inner_precision": args.inner,
           "seconds": dt, "systems_per_s": len(hs) / dt, "waves": st[0]["waves"],
           "iterations": {"min": min(s["iterations"] for s in st), "max": max(s["iterations"] for s in st)},
           "true_residual_max": max(s["true_residual"] for s in st),
           "status": sorted({s["status"] for s in st}), "kernel_launches": st[0]["kernel_launches"]}
    if args.sequential:
        # the same systems one at a time through dwf_solve (5D source, solve, 4D projection)
        n = len(hs) if args.sequential < 0 else min(args.sequential, len(hs))
        worst = 0.0
        _sync()
        t0 = time.perf_counter()
        for h, b4, xb in zip(hs[:n], b4s[:n], x4s[:n]):
            x5, s1 = h.solve(h.source_5d(b4), inner_prec=args.inner, tol=1e-10)
            x4 = h.project_4d(x5)
            worst = max(worst, float(torch.linalg.vector_norm(x4 - xb) / torch.linalg.vector_norm(x4)))
        _sync()
        ds = time.perf_counter() - t0
        out["sequential"] = {"systems": n, "seconds": ds, "systems_per_s": n / ds,
                             "batched_over_sequential": (len(hs) / dt) / (n / ds),
                             "max_rel_diff_x4_batched_vs_sequential": worst}
    print(json.dumps(out), flush=True)


def run_learned(args):
    import torch
    from . import dwf, inputs
    w = inputs.WORKLOADS["c4_16^4_ls16_neff"]
    dims = w["dims"]
    U = _links(w)
    op = dwf.Operator(dims, w["Ls"], w["M0"], w["mf"], w["b"], w["c"], form="neff", alpha=w["alpha"])
    op.set_gauge(U)
    ntrain = args.ntrain
    b4s = [torch.from_numpy(inputs.gaussian_4d(dims, s)).cuda() for s in list(w["train_seeds"])[:ntrain]]
    tests = [torch.from_numpy(inputs.gaussian_4d(dims, s)).cuda() for s in list(w["test_seeds"])[:args.ntest]]

    def solve_all(**kw):
        rows = []
        for b4 in tests:
            b5 = op.source_5d(b4)
            _sync()
            t0 = time.perf_counter()
            _, s = op.solve(b5, **kw)
            _sync()
            rows.append((s["iterations"], time.perf_counter() - t0, s["true_residual"],
                         s.get("precond_applications", 0)))
        return rows

    fp64 = solve_all(inner_prec="f64")
    mixed = solve_all(inner_prec="f32")
    op.precond_init(3, seed=1, noise=0.0)
    ident = solve_all(inner_prec="f32", precond=1)
    _sync()
    t0 = time.perf_counter()
    st = op.precond_train(b4s, epochs=args.epochs, batch=16, lr=args.lr, random_pairs=args.random_pairs)
    _sync()
    ttrain = time.perf_counter() - t0
    learned = solve_all(inner_prec="f32", precond=1)

    def summ(rows):
        return {"iterations": [r[0] for r in rows], "seconds": [round(r[1], 4) for r in rows],
                "true_residual_max": max(r[2] for r in rows), "precond_applications": [r[3] for r in rows]}
    out = {"workload": "c4_16^4_ls16_neff", "train_sources": ntrain, "random_pairs": st["pairs"] - ntrain,
           "test_sources": len(tests),
           "train_seconds": ttrain, "train_solve_seconds": st["solve_seconds"], "loss_first": st["loss_first"],
           "loss_last": st["loss_last"], "epochs": st["epochs"],
           "fp64_cg": summ(fp64), "mixed_f32_cg": summ(mixed), "fcg_identity": summ(ident),
           "fcg_learned": summ(learned)}
    print(json.dumps(out), flush=True)


def run_large(args):
    from . import dwf, inputs
    w = inputs.WORKLOADS["c5_32^3x64_ls16_mobius"]
    U = _links(w)
    op = dwf.Operator(w["dims"], w["Ls"], w["M0"], w["mf"], w["b"], w["c"], form="neff", alpha=w["alpha"])
    op.set_gauge(U)
    import torch
    b4 = torch.from_numpy(inputs.gaussian_4d(w["dims"], w["src_seed"])).cuda()
    res = {}
    for name, kw in (("mixed_f16", dict(inner_prec="f16")), ("mixed_f32", dict(inner_prec="f32")),
                     ("fp64_cg", dict(inner_prec="f64"))):
        b5 = op.source_5d(b4)
        _sync()
        t0 = time.perf_counter()
        _, s = op.solve(b5, **kw)
        _sync()
        res[name] = {"seconds": time.perf_counter() - t0, "iterations": s["iterations"],
                     "true_residual": s["true_residual"], "reliable_updates": s["reliable_updates"]}
    us, by = op.time_hop("f16", reps=10, flush_l2=True)
    res["hop_f16"] = {"us": us, "gbs": by / us / 1e3}
    us, by = op.time_hop("f32", reps=10, flush_l2=True)
    res["hop_f32"] = {"us": us, "gbs": by / us / 1e3}
    print(json.dumps({"workload": "c5_32^3x64_ls16_mobius", "device_bytes": op.device_bytes(), **res}), flush=True)


def run_alpha(args):
    """CG iterations and time against Neff's alpha (Sec. 3: the paper finds the
    fewest iterations near alpha = 0.4-0.6); alpha = 1 is the standard form.
    With --spectrum also the condition number of D^dag D (Sec. 3.2)."""
    import torch
    from . import dwf, inputs
    w = inputs.WORKLOADS["c2_16^3x32_ls16_mobius"]
    U = _links(w)
    b4 = torch.from_numpy(inputs.gaussian_4d(w["dims"], w["src_seed"])).cuda()
    rows = []
    for alpha in (0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 1.0):
        form = "standard" if alpha == 1.0 else "neff"
        op = dwf.Operator(w["dims"], w["Ls"], w["M0"], w["mf"], w["b"], w["c"], form=form, alpha=alpha)
        op.set_gauge(U)
        b5 = op.source_5d(b4)
        op.solve(b5, inner_prec=args.inner, check_every=args.check)
        _sync()
        t0 = time.perf_counter()
        x5, s = op.solve(b5, inner_prec=args.inner, check_every=args.check)
        _sync()
        secs = time.perf_counter() - t0
        x4 = op.project_4d(x5)
        row = {"alpha": alpha, "iterations": s["iterations"], "seconds": secs,
               "true_residual": s["true_residual"], "x4_norm": float(torch.linalg.vector_norm(x4))}
        if args.spectrum:
            # condition number of D^dag D (Sec. 3.2), FP64 Lanczos
            lo, hi, n = op.spectrum_bounds(max_steps=args.lanczos_steps, rtol=1e-6, seed=1)
            row.update(lambda_min=lo, lambda_max=hi, condition_number=hi / lo, lanczos_steps=n)
            # the second even-odd form, in which alpha cancels (Sec. 2.3): a control
            lo, hi, n = op.spectrum_bounds(max_steps=args.lanczos_steps, rtol=1e-6, seed=1, eo_form=1)
            row.update(condition_number_second_form=hi / lo)
        rows.append(row)
        op.close()
    print(json.dumps({"workload": "c2_16^3x32_ls16_mobius", "inner_precision": args.inner,
                      "check_every": args.check, "scan": rows}), flush=True)


def run_delta(args):
    """Time to solution against the reliable-update threshold delta (the inner
    residual falls by delta between two FP64 true-residual recomputations): a
    smaller delta means fewer FP64 hops and more drift of the iterated residual."""
    import torch
    from . import dwf, inputs
    name = "c2_16^3x32_ls16_mobius" if args.small else "c5_32^3x64_ls16_mobius"
    w = inputs.WORKLOADS[name]
    op = dwf.Operator(w["dims"], w["Ls"], w["M0"], w["mf"], w["b"], w["c"], form="neff", alpha=w["alpha"])
    op.set_gauge(_links(w))
    b4 = torch.from_numpy(inputs.gaussian_4d(w["dims"], w["src_seed"])).cuda()
    b5 = op.source_5d(b4)
    rows = []
    for delta in (0.3, 0.1, 0.03, 0.01, 0.003, 0.001):
        op.solve(b5, inner_prec=args.inner, delta=delta)
        _sync()
        t0 = time.perf_counter()
        _, s = op.solve(b5, inner_prec=args.inner, delta=delta)
        _sync()
        rows.append({"delta": delta, "seconds": time.perf_counter() - t0, "iterations": s["iterations"],
                     "reliable_updates": s["reliable_updates"], "d_applications": s["d_applications"],
                     "true_residual": s["true_residual"]})
    print(json.dumps({"workload": name, "inner_precision": args.inner, "scan": rows}), flush=True)


def run_eo5(args):
    """The two even-odd splits of Sec. 2.3 on one operator where both exist
    (standard form, c = 0: Shamir b = 1, or a scaled b): FP64 CG on the 4D
    split's normal equation (dwf_solve) against FP64 CGNR on the 5D split's
    (dwf_solve_eo5), iterations and time to the same true residual."""
    import torch
    from . import dwf, inputs
    name = "c2_16^3x32_ls16_mobius"
    w = inputs.WORKLOADS[name]
    U = _links(w)
    b4 = torch.from_numpy(inputs.gaussian_4d(w["dims"], w["src_seed"])).cuda()
    rows = []
    for bcoef in (1.0, 1.5):
        op = dwf.Operator(w["dims"], w["Ls"], w["M0"], w["mf"], bcoef, 0.0, form="standard")
        op.set_gauge(U)
        b5 = op.source_5d(b4)
        res = {"b": bcoef, "c": 0.0}
        for key, fn in (("eo4_fp64_cg", lambda: op.solve(b5, inner_prec="f64", tol=1e-10)),
                        ("eo4_fp32_mixed", lambda: op.solve(b5, inner_prec="f32", tol=1e-10)),
                        ("eo5_fp64_cgnr", lambda: op.solve_eo5(b5, tol=1e-10))):
            fn()
            _sync()
            t0 = time.perf_counter()
            out = fn()
            _sync()
            secs = time.perf_counter() - t0
            if key.startswith("eo5"):
                res[key] = {"seconds": secs, "iterations": len(out[1]) - 1, "true_residual": out[1][-1]}
            else:
                res[key] = {"seconds": secs, "iterations": out[1]["iterations"], "true_residual": out[1]["true_residual"]}
        rows.append(res)
        op.close()
    print(json.dumps({"workload": name + " (standard form, c = 0)", "scan": rows}), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["batch", "learned", "large", "alpha", "delta", "eo5"])
    ap.add_argument("--inner", default="f32", choices=["f16", "f32", "f64"])
    ap.add_argument("--wave", type=int, default=0)
    ap.add_argument("--small", action="store_true",
                    help="batch: 8^3x16 instead of 24^3x48; delta: 16^3x32 instead of 32^3x64")
    ap.add_argument("--sequential", type=int, default=0,
                    help="batch: also solve this many of the systems one by one (-1: all) and compare")
    ap.add_argument("--ntrain", type=int, default=256)
    ap.add_argument("--ntest", type=int, default=4)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--random-pairs", type=int, default=-1, help="learned: white-noise pairs (-1: as many as sources)")
    ap.add_argument("--check", type=int, default=16, help="alpha: inner iterations between convergence checks")
    ap.add_argument("--spectrum", action="store_true", help="alpha: also the extremal eigenvalues of D^dag D")
    ap.add_argument("--lanczos-steps", type=int, default=2000, help="alpha --spectrum: Lanczos step cap")
    args = ap.parse_args(argv)
    from . import build
    build.build()
    {"batch": run_batch, "learned": run_learned, "large": run_large, "alpha": run_alpha,
     "delta": run_delta, "eo5": run_eo5}[args.what](args)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
