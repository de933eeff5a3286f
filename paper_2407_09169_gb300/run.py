"""Command-line stepping of one workload through the C ABI.

    python -m paper_2407_09169_gb300.run --workload large --precision fp32 --steps 1
    python -m paper_2407_09169_gb300.run --adjoint --precision fp32 --steps 4 --ckpt 2
    python -m paper_2407_09169_gb300.run --workload large --truncate-vjp --steps 2

Builds the library if needed, creates a context for the named workload
(workload.WORKLOADS, or --paper for the paper's flow case at that grid and
chi), advances it and prints the scalar observables as one JSON line; with
--truncate-vjp it instead calls the backward of the bond truncation --steps
times on trains of the workload's sizes (workload.make_truncation_trains:
bond chi_max + 8 in left-orthonormal form, cotangent bond chi_max).  Used
as the profiled command of the ncu summaries (with QTT_GRAPHS=0 every step
runs eagerly, so every kernel launch appears individually).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import workload  # noqa: E402

from . import _binding as q  # noqa: E402
from . import build as qbuild  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="large", choices=list(workload.WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=list(workload.PRECISIONS))
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--paper", action="store_true", help="the paper's flow case at the workload's grid and chi")
    ap.add_argument("--adjoint", action="store_true",
                    help="run qtt_grad on the adjoint configuration (workload.make_adjoint_params) instead")
    ap.add_argument("--ckpt", type=int, default=0, help="checkpoint interval of --adjoint")
    ap.add_argument("--truncate-vjp", action="store_true",
                    help="call qtt_truncate_vjp --steps times at the workload's sizes instead")
    args = ap.parse_args(argv)
    qbuild.build()
    w = workload.WORKLOADS[args.workload]
    if args.truncate_vjp:
        import torch
        nsites, chi = 5 * w["bits"], w["chi_max"]
        r, xh, sy, yh = workload.make_truncation_trains(nsites, chi + 8, chi, seed=args.seed + 11)
        xd, yd = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
        cap = sum((1 if n == 0 else 2 * r[n]) * 2 * (1 if n == nsites - 1 else 2 * r[n + 1]) for n in range(nsites))
        out = torch.empty(cap, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _, kept = q.qtt_truncate_vjp(r, xd, sy, yd, chi, 1e-14, 0.0, out, cap)
        torch.cuda.synchronize()
        print(json.dumps({"sites": nsites, "bond": chi + 8, "chi": chi, "kept": kept, "calls": args.steps,
                          "wall_s": time.perf_counter() - t0}))
        return
    if args.adjoint:
        p = workload.make_adjoint_params(seed=args.seed, precision=args.precision)
        t0 = time.perf_counter()
        with q.qtt_init(p) as ctx:
            J, g = ctx.grad(args.steps, args.ckpt)
        print(json.dumps({"J": J, "grad": g.tolist(), "names": q.grad_param_names(p),
                          "wall_s": time.perf_counter() - t0}))
        return
    if args.paper:
        p = workload.make_paper_params(bits=w["bits"], chi=w["chi_max"], seed=args.seed, precision=args.precision)
    else:
        p = workload.make_params(args.workload, seed=args.seed, precision=args.precision)
    t0 = time.perf_counter()
    with q.qtt_init(p) as ctx:
        ctx.step(args.steps)
        s = ctx.scalars()
    s["wall_s"] = time.perf_counter() - t0
    print(json.dumps(s))


if __name__ == "__main__":
    main()
