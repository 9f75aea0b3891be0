"""Shared pieces of the GPU reports: the precision ladder run stage by stage
through Optimizer, with the relative residual recorded at every check.

The stage rules are those of sos_solve: BF16 steps until ||c - p|| / ||p|| <
switch_rel or the residual stops improving by 1% over `stall` checks; FP32
steps (same Adam state) until they stall or reach tol / 4; FP64 steps (FP64
iterate, FP32 adjoint) until tol / 2 or max_fp64 steps.  Each check reads the
loss of the step just taken (the loss before that step's update).
"""
import time

import numpy as np
import torch

from paper_2410_19844_gb300.engine import Optimizer


def ladder_trace(pl, p64, A0, lr=1e-2, check_every=50, tol=1e-8, switch_rel=1e-3, stall=4,
                 max_bf16=20000, max_fp32=20000, max_fp64=4000):
    """Runs the ladder from A0 (float64 device tensor, N x r, not modified).
    Returns {"trace": [(step, prec, rel)], "steps": {prec: count}, "A": float64
    device tensor of the last iterate, "wall_s": seconds, "best_rel": min rel}."""
    pp = float(torch.dot(p64, p64).item())
    p32 = p64.float()
    trace, steps = [], {"bf16": 0, "fp32": 0, "fp64": 0}
    total = 0
    torch.cuda.synchronize()
    t0 = time.time()

    def run(opt, p, prec, limit, stop):
        nonlocal total
        best, bad = np.inf, 0
        while steps[prec] < limit:
            for _ in range(check_every):
                loss = opt.step(p)
            steps[prec] += check_every
            total += check_every
            rel = float(np.sqrt(2.0 * max(loss[0].item(), 0.0) / pp))
            trace.append((total, prec, rel))
            if not np.isfinite(rel):
                return
            if rel < 0.99 * best:
                best, bad = rel, 0
            else:
                bad += 1
            if stop(rel, bad):
                return

    A = A0.float().contiguous()
    o16 = Optimizer(pl, A, prec="bf16", optimizer="adam", lr=lr)
    run(o16, p32, "bf16", max_bf16, lambda rel, bad: rel < switch_rel or bad >= stall)
    o32 = Optimizer(pl, A, prec="fp32", optimizer="adam", lr=lr)
    o32.m.copy_(o16.m)
    o32.v.copy_(o16.v)
    o32.state.t = o16.state.t
    run(o32, p32, "fp32", max_fp32, lambda rel, bad: bad >= stall or rel <= 0.25 * tol)
    A64 = A.double().contiguous()
    o64 = Optimizer(pl, A64, prec="fp64", optimizer="adam", lr=lr, fp32_adjoint=True)
    o64.m.copy_(o32.m.double())
    o64.v.copy_(o32.v.double())
    o64.state.t = o32.state.t
    run(o64, p64, "fp64", max_fp64, lambda rel, bad: rel <= 0.5 * tol)
    torch.cuda.synchronize()
    return {"trace": trace, "steps": steps, "A": A64, "wall_s": time.time() - t0,
            "best_rel": min(t[2] for t in trace)}


def first_step_below(trace, level):
    """First recorded step whose relative residual is <= level, or None."""
    for step, _, rel in trace:
        if rel <= level:
            return step
    return None
