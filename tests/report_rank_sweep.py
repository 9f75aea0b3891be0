"""Report: number of squares r below, at and above N (Sec. 1.3 and the rank
experiment of Sec. 3.2).

Workload: quartic forms in n_form = 30 variables (the paper's size for this
experiment), dehomogenised to n = 29 variables and degree <= 4: N = l = 465
degree-<=2 monomials, M = 40,920 coefficients.  Target p = c(B) with B uniform
in [-1, 1], l x l (the paper's generator, Q = B B^T, Sec. 3.1), built by the
oracle.  For every r in the sweep and three seeds: A0 ~ N(0, 0.1^2), N x r;
the precision ladder (Adam, lr 1e-2; BF16 -> FP32 -> FP64) runs until the
FP64 relative residual ||c - p|| / ||p|| is below 1e-8 or the step budget is
spent, and the report lists the steps at which the residual first fell below
1e-2, 1e-4, 1e-6 and 1e-8, the wall time and the best residual.  The oracle
recomputes the final residual of each run.

Sizes in the sweep: r = 110 (the rank the paper compares with), 286 (the
smallest r with r (r + 1) >= 2 M, the Burer-Monteiro size of Sec. 1.2; the
Pythagoras-number bound of Sec. 1.3 evaluates to 285.6 at n = 30), 465 = N
(the paper's choice) and 930 = 2N.

    python tests/report_rank_sweep.py [--ranks 110,286,465,930] [--seeds 3] [--out FILE]
"""
import argparse
import os
import sys
from math import comb

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import oracle  # noqa: E402
import sos_inputs  # noqa: E402
from paper_2410_19844_gb300.engine import Plan  # noqa: E402
from report_util import first_step_below, ladder_trace  # noqa: E402

LEVELS = (1e-2, 1e-4, 1e-6, 1e-8)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-form", type=int, default=30)
    ap.add_argument("--ranks", default="110,286,465,930")
    ap.add_argument("--seeds", type=int, default=3)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    n_form = args.n_form
    n, l = n_form - 1, comb(n_form + 1, 2)
    ranks = [int(x) for x in args.ranks.split(",")]
    o = oracle.Oracle(n, 4)
    assert o.N == l
    B = sos_inputs.paper_quartic_generator(n_form, 0)
    p = o.coeffs(B)
    p64 = torch.from_numpy(p).cuda()
    pp = float(np.dot(p, p))
    lines = [f"# Number of squares r vs convergence, quartic forms in {n_form} variables "
             f"(N = {l}, M = {o.M})", "",
             "Precision ladder (Adam, lr 1e-2, checks every 50 steps), target c(B) with B uniform l x l; "
             "steps are totals over the three stages at the first check below each level.", "",
             "| r | seed | steps to 1e-2 | 1e-4 | 1e-6 | 1e-8 | steps bf16 / fp32 / fp64 | wall s | best rel "
             "| oracle rel (final A) |", "|---|---|---|---|---|---|---|---|---|---|"]
    summary = {}
    for r in ranks:
        pl = Plan(n, 4, r)
        for seed in range(args.seeds):
            A0 = torch.from_numpy(sos_inputs.normal_matrix(l, r, 100 + seed, sigma=0.1)).cuda()
            res = ladder_trace(pl, p64, A0, max_bf16=20000, max_fp32=40000, max_fp64=6000)
            hits = [first_step_below(res["trace"], lv) for lv in LEVELS]
            A_fin = res["A"].cpu().numpy()
            c = o.coeffs(A_fin)
            rel_o = float(np.sqrt(np.dot(c - p, c - p) / pp))
            s = res["steps"]
            lines.append(f"| {r} | {seed} | " + " | ".join("-" if h is None else str(h) for h in hits)
                         + f" | {s['bf16']} / {s['fp32']} / {s['fp64']} | {res['wall_s']:.2f} "
                           f"| {res['best_rel']:.2e} | {rel_o:.2e} |")
            print(lines[-1], flush=True)
            summary.setdefault(r, []).append(hits[-1])
    lines += ["", "| r | runs reaching 1e-8 | mean steps to 1e-8 (those runs) |", "|---|---|---|"]
    for r in ranks:
        ok = [h for h in summary[r] if h is not None]
        lines.append(f"| {r} | {len(ok)} / {len(summary[r])} | {np.mean(ok):.0f} |" if ok
                     else f"| {r} | 0 / {len(summary[r])} | - |")
    text = "\n".join(lines) + "\n"
    print(text)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)


if __name__ == "__main__":
    main()
