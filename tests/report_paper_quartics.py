"""Report: the paper's own workloads (Sec. 3.1) solved by the precision ladder.

Quartic forms in n_form = 10, 15, 20, 25, 30 (and 100) variables: p = m_2 Q m_2^T
with Q = B B^T and B uniform in [-1, 1] (l x l, l = C(n_form+1, 2) degree-2
monomials).  Dehomogenising (the last variable set to 1, Sec. 1.1) gives a
polynomial of degree <= 4 in n_form - 1 variables whose degree-<=2 monomials
are in bijection with the form's degree-2 monomials, so p = c(B) with B as the
coefficient matrix (r = l, the paper's full-rank over-parameterisation).

For each size: the target is built with the library's FP64 forward, A0 ~
N(0, 0.1^2), sos_solve runs the BF16 -> FP32 -> FP64 ladder, and the report
lists steps, wall time and the FP64 certificate, next to the paper's time to
solution (Sec. 3.1 table: Python/Jax + Adam on an i7-6500U laptop CPU; a
different optimiser set-up and hardware, so context, not a like-for-like
comparison).  For n_form <= 30 the oracle recomputes the certificate of the
returned A.  The last line fits time ~ n^k over n_form = 10..30 (the paper
reports k ~ 4.5 for its method, Sec. 3.1).

    python tests/report_paper_quartics.py [--sizes 10,15,20,25,30,100] [--out FILE]
"""
import argparse
import os
import sys
import time
from math import comb

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import sos_inputs  # noqa: E402
from paper_2410_19844_gb300.engine import Plan, solve  # noqa: E402

PAPER_SECONDS = {10: 32.7, 15: 46.0, 20: 89.0, 25: 234.0, 30: 542.0, 100: 151000.0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default="10,15,20,25,30,100")
    ap.add_argument("--out", default=None)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    sizes = [int(s) for s in args.sizes.split(",")]
    lines = ["# The paper's quartic forms (Sec. 3.1), solved by the precision ladder", "",
             "| n (form) | N = l | M | steps bf16 / fp32 / fp64 | wall s | FP64 certificate | oracle check "
             "| paper s (i7-6500U, Jax) |", "|---|---|---|---|---|---|---|---|"]
    times = {}
    for n_form in sizes:
        n = n_form - 1
        l = comb(n_form + 1, 2)
        pl = Plan(n, 4)
        assert pl.N == l and pl.M == comb(n_form + 3, 4)
        B = torch.from_numpy(sos_inputs.paper_quartic_generator(n_form, args.seed)).cuda().contiguous()
        p64 = pl.coeffs(B, "fp64")
        A = torch.from_numpy(sos_inputs.normal_matrix(l, l, args.seed + 1, sigma=0.1)).cuda()
        torch.cuda.synchronize()
        t0 = time.time()
        res = solve(pl, p64, A, max_steps=50000, check_every=50, fp64_steps=4000)
        dt = time.time() - t0
        times[n_form] = dt
        check = "-"
        if n_form <= 30:
            o = oracle.Oracle(n, 4)
            check = f"{o.certify(o.coeffs(A.cpu().numpy()), p64.cpu().numpy()):.3e}"
        lines.append(f"| {n_form} | {l} | {pl.M} | {res['steps_bf16']} / {res['steps_fp32']} / {res['steps_fp64']} "
                     f"| {dt:.2f} | {res['rel_resid_fp64']:.3e} ({'SOS' if res['verdict'] == 1 else 'not converged'}) "
                     f"| {check} | {PAPER_SECONDS.get(n_form, '-')} |")
        print(lines[-1], flush=True)
    fit = [k for k in sorted(times) if k <= 30]
    if len(fit) >= 3:
        k, _ = np.polyfit(np.log(fit), np.log([times[x] for x in fit]), 1)
        lines += ["", f"Fitted wall time ~ n^{k:.2f} over n = {fit[0]}..{fit[-1]} (the paper reports ~n^4.5 "
                      f"for its method, Sec. 3.1)."]
    text = "\n".join(lines) + "\n"
    print(text)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)


if __name__ == "__main__":
    main()
