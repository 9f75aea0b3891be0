"""Report: time to a certificate on the large workload (n = 20, 2d = 8,
N = r = 10,626, M = 3,108,105) -- the benchmark's problem taken to the end.

Target p = sum of 2000 squares of N(0, 1)/sqrt(N) polynomials (seed 0), built
with the library's FP64 forward; A0 ~ N(0, 0.1^2).  sos_solve runs with its
defaults (BF16 steps, then SOS_FP64_TC steps with slices chosen from the
residual, then the CUDA-core FP64 certificate).  The oracle then recomputes
the certificate of the returned A on the host (the full FP64 forward, about
a minute on 16 cores) and the report states both.

    python tests/report_large_solve.py [--out FILE]
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
from paper_2410_19844_gb300.engine import Plan, solve  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--max-steps", type=int, default=20000)
    args = ap.parse_args()
    w = sos_inputs.LARGE
    G = torch.from_numpy(sos_inputs.generator(w, 0)).cuda().contiguous()
    p64 = Plan(w.n, w.two_d, r=G.shape[1]).coeffs(G, "fp64")
    del G
    pl = Plan(w.n, w.two_d)
    A = torch.from_numpy(sos_inputs.init_A(w, 0)).cuda()
    torch.cuda.synchronize()
    t0 = time.time()
    res = solve(pl, p64, A, max_steps=args.max_steps, check_every=50, fp64_steps=20000)
    wall = time.time() - t0
    t1 = time.time()
    o = oracle.Oracle(w.n, w.two_d)
    p = p64.cpu().numpy()
    rel_o = o.certify(o.coeffs(A.cpu().numpy()), p)
    t_oracle = time.time() - t1
    lines = [f"# Time to a certificate, large workload (n = {w.n}, 2d = {w.two_d}, N = r = {pl.N}, M = {pl.M})", "",
             "| verdict | steps bf16 / fp64_tc | wall s | BF16 residual at the switch | FP64 certificate (GPU) "
             "| certificate recomputed by the oracle |", "|---|---|---|---|---|---|",
             f"| {'SOS' if res['verdict'] == 1 else 'not converged'} | {res['steps_bf16']} / {res['steps_fp64']} "
             f"| {wall:.1f} | {res['rel_at_switch']:.2e} | {res['rel_resid_fp64']:.3e} | {rel_o:.3e} |", "",
             f"The oracle's check took {t_oracle:.0f} s on {oracle.num_threads()} host threads."]
    text = "\n".join(lines) + "\n"
    print(text)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)


if __name__ == "__main__":
    main()
