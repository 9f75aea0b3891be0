"""Report: the first layer on targets with very unequal coefficients (Sec. 2.1,
Sec. 3.3).

Targets (quartic forms in nf variables, dehomogenised to nf - 1, built by the
oracle): the paper's uniform generator p = c(B) with B uniform in [-1, 1]
(l x l, Sec. 3.1), then
  * "one": the coefficient of x_i^4 set to 10^4 for one random i;
  * "many": every coefficient of x_i^4 and x_i^2 x_j^2 increased by an amount
    uniform in [0, 10^4].
Both stay sums of squares (the added terms are squares).

Networks (Sec. 2, k = l squares, Adam lr 1e-2):
  * A1 = I, fixed (the paper's run without the first layer; m = nf);
  * A1 general, trained, m = nf;
  * A1 general, trained, m = 2 nf (the over-parameterised first layer).
B0 ~ N(0, 0.1^2); a trained A1 starts as I (m = nf) or [I; 0] (m = 2 nf) plus
N(0, 0.1^2) noise.  Each run takes FP32 steps, then FP64 steps (FP64
iterate, FP32 adjoint, Adam state and learning rate carried over); within a
stage the learning rate drops tenfold after 6 checks without a 1% gain, at
most 3 times, and the stage ends at the next stall (or at 1e-9).  The report gives the
steps at which ||c - p|| / ||p|| first fell below 1e-3, 1e-5, 1e-7 and 1e-9,
the final relative and total squared error (recomputed by the oracle at the
final B, A1) and the wall time.

    python tests/report_first_layer.py [--nf 12] [--seeds 3] [--out FILE]
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
sys.path.insert(0, os.path.join(ROOT, "tests"))

import oracle  # noqa: E402
import sos_inputs  # noqa: E402
from paper_2410_19844_gb300.engine import Layer, LayerOptimizer, Plan  # noqa: E402
from report_util import first_step_below  # noqa: E402

LEVELS = (1e-3, 1e-5, 1e-7, 1e-9)


def targets(o, nf, seed):
    base = o.coeffs(sos_inputs.paper_quartic_generator(nf, seed))
    g = np.random.default_rng(seed + 1000)
    E = o.E2d
    full = np.concatenate([E, (4 - E.sum(axis=1))[:, None]], axis=1)   # exponents of the form
    one = base.copy()
    i = int(g.integers(nf - 1))
    one[[r for r in range(o.M) if full[r, i] == 4][0]] = 1e4
    many = base.copy()
    even = [r for r in range(o.M) if np.all(full[r] % 2 == 0) and np.count_nonzero(full[r]) <= 2]
    many[even] += g.uniform(0.0, 1e4, size=len(even))
    return {"one": one, "many": many}


def run(layer, p, B0, A10, fixed, lr=1e-2, check_every=50, max32=30000, max64=6000, tol=1e-9, stall=6,
        decays=3):
    """FP32 then FP64 Adam steps; within each stage, `stall` checks without a
    1% gain cut the learning rate tenfold (at most `decays` times per stage),
    after which the stage ends."""
    pp = float(np.dot(p, p))
    p64 = torch.from_numpy(p).cuda()
    trace, total, steps = [], 0, {"fp32": 0, "fp64": 0}
    torch.cuda.synchronize()
    t0 = time.time()

    def stage(opt, target, prec, limit, stop_rel):
        nonlocal total
        best, bad, cuts = np.inf, 0, 0
        while steps[prec] < limit:
            for _ in range(check_every):
                loss = opt.step(target)
            steps[prec] += check_every
            total += check_every
            rel = float(np.sqrt(2.0 * max(loss[0].item(), 0.0) / pp))
            trace.append((total, prec, rel))
            if not np.isfinite(rel) or rel <= stop_rel:
                return
            if rel < 0.99 * best:
                best, bad = rel, 0
                continue
            bad += 1
            if bad >= stall:
                if cuts == decays:
                    return
                cuts += 1
                bad = 0
                opt.opts.lr *= 0.1

    B32, A132 = torch.from_numpy(B0).float().cuda(), torch.from_numpy(A10).float().cuda()
    o32 = LayerOptimizer(layer, B32, A132, prec="fp32", lr=lr, fixed_A1=fixed)
    stage(o32, p64.float(), "fp32", max32, 0.25 * tol)
    B64, A164 = B32.double().contiguous(), A132.double().contiguous()
    o64 = LayerOptimizer(layer, B64, A164, prec="fp64", lr=o32.opts.lr, fixed_A1=fixed, fp32_adjoint=True)
    o64.mB.copy_(o32.mB.double())
    o64.vB.copy_(o32.vB.double())
    if not fixed:
        o64.mA1.copy_(o32.mA1.double())
        o64.vA1.copy_(o32.vA1.double())
    o64.state.t = o32.state.t
    stage(o64, p64, "fp64", max64, 0.5 * tol)
    torch.cuda.synchronize()
    return trace, steps, B64.cpu().numpy(), A164.cpu().numpy(), time.time() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nf", type=int, default=12)
    ap.add_argument("--seeds", type=int, default=3)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    nf = args.nf
    l = comb(nf + 1, 2)
    o = oracle.Oracle(nf - 1, 4)
    pl = Plan(nf - 1, 4, l)
    nets = [("A1 = I (fixed)", nf, True), ("A1 general, m = n", nf, False), ("A1 general, m = 2n", 2 * nf, False)]
    layers = {m: Layer(pl, m) for _, m, _ in nets}
    lines = [f"# First layer on non-uniform targets (Sec. 2.1, 3.3): quartic forms in {nf} variables "
             f"(N = {l}, M = {o.M}, k = {l} squares)", "",
             "Adam lr 1e-2 (cut tenfold at plateaus, at most 3 times per stage), FP32 then FP64 (FP32 adjoint) "
             "steps, checks every 50 steps; steps are totals at the first check below each level of "
             "||c - p|| / ||p||.", "",
             "| target | network | seed | 1e-3 | 1e-5 | 1e-7 | 1e-9 | steps fp32 / fp64 | wall s "
             "| best rel (checks) | final rel (oracle) | total squared error |",
             "|---|---|---|---|---|---|---|---|---|---|---|---|"]
    for seed in range(args.seeds):
        tg = targets(o, nf, seed)
        for tname, p in tg.items():
            for name, m, fixed in nets:
                B0 = sos_inputs.normal_matrix(l, nf * m, 100 + seed, sigma=0.1)
                A10 = np.zeros((m, nf))
                A10[:nf, :nf] = np.eye(nf)
                if not fixed:
                    A10 += sos_inputs.normal_matrix(m, nf, 200 + seed, sigma=0.1)
                trace, steps, Bf, A1f, wall = run(layers[m], p, B0, A10, fixed)
                hits = [first_step_below(trace, lv) for lv in LEVELS]
                c = o.layer_coeffs(Bf, A1f)
                sq = float(np.dot(c - p, c - p))
                rel = float(np.sqrt(sq / np.dot(p, p)))
                lines.append(f"| {tname} | {name} | {seed} | " + " | ".join("-" if h is None else str(h) for h in hits)
                             + f" | {steps['fp32']} / {steps['fp64']} | {wall:.2f} "
                               f"| {min(t[2] for t in trace):.2e} | {rel:.2e} | {sq:.2e} |")
                print(lines[-1], flush=True)
    text = "\n".join(lines) + "\n"
    print(text)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)


if __name__ == "__main__":
    main()
