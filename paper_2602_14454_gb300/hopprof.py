"""Time the even-odd hop kernel on one workload (for profiling runs).

    python -m paper_2602_14454_gb300.hopprof --prec f16 --reps 4
    python -m paper_2602_14454_gb300.hopprof --workload c1_4^4_ls8_shamir --prec f32
    python -m paper_2602_14454_gb300.hopprof --prec f16 --iteration   # the 5 launches of one CG iteration
    python -m paper_2602_14454_gb300.hopprof --prec f32 --time-mix --mix 2   # one stand-alone mixing launch
    python -m paper_2602_14454_gb300.hopprof --workload c5_32^3x64_ls16_mobius --prec f32 --sweep 0   # index order

Builds the operator of the named workload (links from the seeded generator of
``inputs``), optionally pins a hop configuration or a mixing mode, and times
``reps`` hop launches with CUDA events, L2 flushed between them.  Prints one
JSON line: microseconds per launch, algorithmic bytes per launch and GB/s.
With ``--iteration`` it times the five launches of one inner CG iteration of
the solver instead (p update and the four hops with their fused epilogues);
with ``--time-mix`` one stand-alone fifth-direction mixing launch in the mode
given by ``--mix`` (0 CUDA cores, 2 tensor cores).
"""

import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c2_16^3x32_ls16_mobius")
    ap.add_argument("--prec", default="f16", choices=["f64", "f32", "f16"])
    ap.add_argument("--reps", type=int, default=4)
    ap.add_argument("--form", default="neff", choices=["neff", "standard"])
    ap.add_argument("--alpha", type=float, default=0.5)
    ap.add_argument("--config", default=None, help="variant,ns,sb (default: the library's choice)")
    ap.add_argument("--mix", type=int, default=None, help="fifth-direction mixing mode")
    ap.add_argument("--sweep", type=int, default=None, help="z-planes per sweep column (0: index order, -2: automatic)")
    ap.add_argument("--iteration", action="store_true", help="time the launches of one CG iteration")
    ap.add_argument("--time-mix", action="store_true", help="time one stand-alone mixing launch (mode --mix)")
    args = ap.parse_args(argv)

    import torch
    from . import build, dwf, inputs
    build.build()
    w = inputs.WORKLOADS[args.workload]
    op = dwf.Operator(w["dims"], w["Ls"], w["M0"], w["mf"], w["b"], w["c"], form=args.form, alpha=args.alpha)
    op.set_gauge(torch.from_numpy(inputs.workload_links(w, device="cuda")).cuda())
    if args.config:
        v, ns, sb = (int(t) for t in args.config.split(","))
        op.set_hop_config(args.prec, v, ns, sb)
    if args.sweep is not None:
        op.set_sweep(args.prec, args.sweep)
    if args.time_mix:
        mode = 0 if args.mix is None else args.mix
        us, nbytes = op.time_mix(args.prec, mode, reps=args.reps, flush_l2=True)
        op.device_status()
        print(json.dumps({"workload": args.workload, "prec": args.prec, "mix_mode": mode, "us_per_launch": us,
                          "algorithmic_bytes": nbytes, "gbs": nbytes / (us * 1e-6) / 1e9}))
        return 0
    if args.mix is not None:
        op.set_mix_mode(args.prec, args.mix)
    if args.iteration:
        t = op.time_iteration(args.prec, reps=args.reps, flush_l2=True)
        op.device_status()
        tot_us = sum(v[0] for v in t.values())
        tot_by = sum(v[1] for v in t.values())
        print(json.dumps({"workload": args.workload, "prec": args.prec, "config": op.hop_config(args.prec),
                          "mix": op.mix_mode(args.prec), "sweep": op.sweep(args.prec),
                          "kernels": {k: {"us": v[0], "algorithmic_bytes": v[1], "gbs": v[1] / (v[0] * 1e-6) / 1e9}
                                      for k, v in t.items()},
                          "iteration_us": tot_us, "iteration_bytes": tot_by,
                          "iteration_gbs": tot_by / (tot_us * 1e-6) / 1e9}))
        return 0
    us, nbytes = op.time_hop(args.prec, reps=args.reps, flush_l2=True)
    op.device_status()
    print(json.dumps({"workload": args.workload, "prec": args.prec, "config": op.hop_config(args.prec),
                      "mix": op.mix_mode(args.prec), "sweep": op.sweep(args.prec), "us_per_launch": us, "algorithmic_bytes": nbytes,
                      "gbs": nbytes / (us * 1e-6) / 1e9}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
