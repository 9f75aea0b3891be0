"""Report: the precision ladder on the precision workload, against the FP64 oracle.

Workload: n=10, 2d=10 (N=3003 monomials, M=184,756 coefficients), r=N,
p = sum of 1000 squares of N(0,1) polynomials, A0 ~ N(0, 0.1^2), seed 0.

Runs the ladder stage by stage through sos_step (BF16 tensor-core steps until
the relative residual is below 1e-3, FP32 CUDA-core steps until they stall,
FP64 steps -- FP64 iterate, residual and update, adjoint contracted in FP32 --
until the residual is below 1e-8 or stalls), and at the end of each
stage evaluates, at that stage's iterate:
  * the stage's own loss and gradient (the precision it stepped in),
  * the library's FP64 loss and gradient,
  * the oracle's loss and gradient (FP64, CPU),
and prints their relative differences.  Then runs sos_solve from the same
start in the ladder (start BF16) and in plain FP32 (start FP32) and compares
steps, wall time and certificates, and from the BF16 start with the SOS_FP64_TC
stage (the FP64-accurate forward on tensor cores) in place of the FP32 and FP64
stages.  Needs a GPU; prints a markdown report.

    python tests/report_precision_ladder.py [--out profiles/precision_ladder_n10_2d10.md]
"""
import argparse
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import sos_inputs  # noqa: E402
from paper_2410_19844_gb300 import _lib as L  # noqa: E402
from paper_2410_19844_gb300.engine import Optimizer, Plan, _ptr, _stream_handle, solve  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--check-every", type=int, default=50)
    args = ap.parse_args()
    w = sos_inputs.PRECISION
    lines = [f"# Precision ladder, {w.name} (n={w.n}, 2d={w.two_d}, N={w.N}, M={w.M}, r={w.cols})", ""]
    t0 = time.time()
    o = oracle.Oracle(w.n, w.two_d)
    _ = o.prod
    p = o.coeffs(sos_inputs.generator(w, 0))
    A0 = sos_inputs.init_A(w, 0)
    lines.append(f"oracle set-up and target: {time.time() - t0:.1f} s on {oracle.num_threads()} host threads")
    pl = Plan(w.n, w.two_d)
    pp = float(np.dot(p, p))
    p64 = torch.from_numpy(p).cuda()
    p32 = p64.float()

    def evaluate(A_np, stage_prec, stage_loss, stage_grad):
        loss_o, g_o, _ = o.loss_grad(A_np, p)
        A64 = torch.from_numpy(A_np).cuda()
        l64, _, g64 = pl.loss_grad(A64, p64, "fp64")
        g64 = g64.cpu().numpy()
        return {"rel_resid_oracle": float(np.sqrt(2 * loss_o / pp)),
                "stage_loss_vs_oracle": abs(stage_loss - loss_o) / loss_o,
                "stage_grad_vs_oracle": rel(stage_grad, g_o),
                "fp64_loss_vs_oracle": abs(l64.item() - loss_o) / loss_o,
                "fp64_grad_vs_oracle": rel(g64, g_o)}

    A = torch.from_numpy(A0.astype(np.float32)).cuda()
    opt = Optimizer(pl, A, prec="bf16", optimizer="adam", lr=1e-2)
    rows = []
    steps = {"bf16": 0, "fp32": 0, "fp64": 0}
    # stage 1: BF16
    t_stage = time.time()
    while True:
        for _ in range(args.check_every):
            opt.step(p32)
        steps["bf16"] += args.check_every
        loss = opt.loss[0].item()
        if np.sqrt(2 * loss / pp) < 1e-3 or steps["bf16"] >= 20000:
            break
    t_bf16 = time.time() - t_stage
    l16, _, g16 = pl.loss_grad(A, p32, "bf16")
    rows.append(("end of BF16", steps["bf16"], t_bf16, evaluate(A.double().cpu().numpy(), "bf16", l16.item(),
                                                               g16.double().cpu().numpy())))
    # stage 2: FP32 with the same Adam state
    opt32 = Optimizer(pl, A, prec="fp32", optimizer="adam", lr=1e-2)
    opt32.m.copy_(opt.m)
    opt32.v.copy_(opt.v)
    opt32.state.t = opt.state.t
    best, stall = np.inf, 0
    t_stage = time.time()
    while stall < 4 and steps["fp32"] < 20000:
        for _ in range(args.check_every):
            opt32.step(p32)
        steps["fp32"] += args.check_every
        r = np.sqrt(2 * opt32.loss[0].item() / pp)
        if r < 0.99 * best:
            best, stall = r, 0
        else:
            stall += 1
    t_fp32 = time.time() - t_stage
    l32, _, g32 = pl.loss_grad(A, p32, "fp32")
    rows.append(("end of FP32", steps["fp32"], t_fp32, evaluate(A.double().cpu().numpy(), "fp32", l32.item(),
                                                               g32.double().cpu().numpy())))
    # stage 3: FP64 from the FP32 point
    A64 = A.double().contiguous()
    opt64 = Optimizer(pl, A64, prec="fp64", optimizer="adam", lr=1e-2, fp32_adjoint=True)
    opt64.m.copy_(opt32.m.double())
    opt64.v.copy_(opt32.v.double())
    opt64.state.t = opt32.state.t
    best, stall = np.inf, 0
    t_stage = time.time()
    while stall < 4 and steps["fp64"] < 4000:
        for _ in range(args.check_every):
            opt64.step(p64)
        steps["fp64"] += args.check_every
        r = np.sqrt(2 * opt64.loss[0].item() / pp)
        if r <= 0.5e-8:
            break
        if r < 0.99 * best:
            best, stall = r, 0
        else:
            stall += 1
    t_fp64 = time.time() - t_stage
    lf, _, gf = pl.loss_grad(A64, p64, "fp64")
    rows.append(("end of FP64", steps["fp64"], t_fp64, evaluate(A64.cpu().numpy(), "fp64", lf.item(),
                                                               gf.cpu().numpy())))
    rel_c, verdict = pl.certify(A64, p64)

    lines += ["", "## Stage by stage (Adam, lr 1e-2, checks every %d steps)" % args.check_every, "",
              "| stage end | steps | wall s | ||c-p||/||p|| (oracle) | stage loss vs oracle | stage grad vs oracle "
              "| GPU FP64 loss vs oracle | GPU FP64 grad vs oracle |",
              "|---|---|---|---|---|---|---|---|"]
    for name, n, t, e in rows:
        lines.append(f"| {name} | {n} | {t:.2f} | {e['rel_resid_oracle']:.3e} | {e['stage_loss_vs_oracle']:.2e} | "
                     f"{e['stage_grad_vs_oracle']:.2e} | {e['fp64_loss_vs_oracle']:.2e} | "
                     f"{e['fp64_grad_vs_oracle']:.2e} |")
    lines += ["", f"FP64 certificate of the final iterate: ||c-p||/||p|| = {rel_c:.3e}, verdict "
                  f"{'SOS' if verdict == 1 else 'not converged'}", ""]

    # sos_solve: ladder vs plain FP32
    lines += ["## sos_solve from the same start", "",
              "| start | verdict | steps bf16 / fp32 / fp64 | wall s | certificate |", "|---|---|---|---|---|"]
    runs = [("bf16", "bf16", {"tc_fp64": 0, "fp64_steps": 4000}), ("fp32", "fp32", {"tc_fp64": 0, "fp64_steps": 4000}),
            ("bf16, then SOS_FP64_TC", "bf16", {"tc_fp64": 1, "fp64_steps": 20000})]
    for label, start, extra in runs:
        A_s = torch.from_numpy(A0.copy()).cuda()
        torch.cuda.synchronize()
        t = time.time()
        res = solve(pl, p64, A_s, start_prec=start, max_steps=40000, check_every=args.check_every, **extra)
        dt = time.time() - t
        lines.append(f"| {label} | {'SOS' if res['verdict'] == 1 else 'not converged'} | {res['steps_bf16']} / "
                     f"{res['steps_fp32']} / {res['steps_fp64']} | {dt:.2f} | {res['rel_resid_fp64']:.3e} |")
    text = "\n".join(lines) + "\n"
    print(text)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)


if __name__ == "__main__":
    main()
