"""Command line front end of the library.

    python -m paper_2410_19844_gb300 monomials --n 2 --two-d 2 [--which 1]
    python -m paper_2410_19844_gb300 solve --n N --two-d 2d --target p.npy [--A0 A0.npy]
                                     [--r R] [--tol 1e-8] [--classic] [--out A.npy]
    python -m paper_2410_19844_gb300 certify --n N --two-d 2d --target p.npy --A A.npy [--tol 1e-8]

`monomials` prints the monomial table of the plan (degree <= d rows of A with
--which 0, degree <= 2d coefficients with --which 1) in the library's order;
it needs no GPU.  `solve` runs sos_solve on a target p (a float64 .npy vector
of the M coefficients in that order) from A0 (float64 N x r .npy; N(0, 0.1^2)
seeded by --seed when absent) and prints the result as one JSON line; `--out`
saves the returned A.  `certify` evaluates ||c(A) - p|| / ||p|| in FP64.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np


def _plan(args):
    from .engine import Plan
    return Plan(args.n, args.two_d, args.r)


def cmd_monomials(args) -> int:
    pl = _plan(args)
    E = pl.monomials(args.which)
    for row in E:
        print(" ".join(str(int(v)) for v in row))
    return 0


def _load_target(pl, path):
    p = np.load(path).astype(np.float64).reshape(-1)
    if p.size != pl.M:
        raise SystemExit(f"target has {p.size} coefficients; the plan has M = {pl.M}")
    return p


def cmd_solve(args) -> int:
    import torch

    from .engine import solve
    if not torch.cuda.is_available():
        raise SystemExit("solve needs a CUDA GPU")
    pl = _plan(args)
    p = _load_target(pl, args.target)
    if args.A0:
        A0 = np.load(args.A0).astype(np.float64)
        if A0.shape != (pl.N, pl.r):
            raise SystemExit(f"A0 must be {pl.N} x {pl.r}, got {A0.shape}")
    else:
        A0 = np.random.default_rng(args.seed).normal(0.0, 0.1, size=(pl.N, pl.r))
    A = torch.from_numpy(np.ascontiguousarray(A0)).cuda()
    res = solve(pl, torch.from_numpy(p).cuda(), A, cert_tol=args.tol, tc_fp64=0 if args.classic else 1,
                max_steps=args.max_steps)
    verdict = {1: "SOS", 0: "NOT_CONVERGED", -1: "ERROR"}.get(res["verdict"], str(res["verdict"]))
    print(json.dumps({"verdict": verdict, **{k: v for k, v in res.items() if k != "verdict"}}))
    if args.out:
        np.save(args.out, A.cpu().numpy())
    return 0


def cmd_certify(args) -> int:
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("certify needs a CUDA GPU")
    pl = _plan(args)
    p = _load_target(pl, args.target)
    A = np.load(args.A).astype(np.float64)
    if A.shape != (pl.N, pl.r):
        raise SystemExit(f"A must be {pl.N} x {pl.r}, got {A.shape}")
    rel, verdict = pl.certify(torch.from_numpy(A).cuda(), torch.from_numpy(p).cuda(), args.tol)
    print(json.dumps({"rel_resid_fp64": rel, "verdict": "SOS" if verdict == 1 else "NOT_CONVERGED"}))
    return 0


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="python -m paper_2410_19844_gb300")
    sub = ap.add_subparsers(dest="cmd", required=True)

    def plan_args(sp):
        sp.add_argument("--n", type=int, required=True, help="number of variables")
        sp.add_argument("--two-d", type=int, required=True, dest="two_d", help="even degree 2d of the target")
        sp.add_argument("--r", type=int, default=None, help="number of squares (default N)")

    sp = sub.add_parser("monomials", help="print the monomial table")
    plan_args(sp)
    sp.add_argument("--which", type=int, default=0, choices=[0, 1], help="0: degree <= d, 1: degree <= 2d")
    sp.set_defaults(fn=cmd_monomials)

    sp = sub.add_parser("solve", help="run the solver on a target")
    plan_args(sp)
    sp.add_argument("--target", required=True)
    sp.add_argument("--A0", default=None)
    sp.add_argument("--seed", type=int, default=0)
    sp.add_argument("--tol", type=float, default=1e-8)
    sp.add_argument("--max-steps", type=int, default=20000, dest="max_steps")
    sp.add_argument("--classic", action="store_true", help="CUDA-core FP32 and FP64 stages after BF16")
    sp.add_argument("--out", default=None)
    sp.set_defaults(fn=cmd_solve)

    sp = sub.add_parser("certify", help="FP64 certificate of a given A")
    plan_args(sp)
    sp.add_argument("--target", required=True)
    sp.add_argument("--A", required=True)
    sp.add_argument("--tol", type=float, default=1e-8)
    sp.set_defaults(fn=cmd_certify)

    args = ap.parse_args(argv)
    return args.fn(args)


if __name__ == "__main__":
    sys.exit(main())
