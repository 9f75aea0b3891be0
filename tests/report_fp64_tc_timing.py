"""Report: one SOS_FP64_TC step, per kernel, against the tensor roofline.

Workloads: the n = 100 quartic form (n = 99 variables dehomogenised, 2d = 4,
N = r = 5050) and the large workload (n = 20, 2d = 8, N = r = 10,626); slices
s = 4, 6, 8.  Each configuration: 3 warm-up steps, 5 timed steps (Adam) with
per-kernel CUDA events.  Algorithmic work of the slice products: diagonal
units N^2 r flops each (upper triangle), cross units 2 N^2 r (every tile), s
(s+1)/2 forward passes in all; rates are compared with the measured bf16
tensor peak in MEASURED_PEAKS.json (sustained).  The CUDA-core FP64 forward
of the same A is timed beside it.

    python tests/report_fp64_tc_timing.py [--out FILE]
"""
import argparse
import json
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import sos_inputs  # noqa: E402
from paper_2410_19844_gb300 import _lib as L  # noqa: E402
from paper_2410_19844_gb300.engine import Optimizer, Plan  # noqa: E402


def peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d.get("bf16_tflops_sustained") or d.get("bf16_tflops")), "measured sustained"
    except Exception:
        return 1700.0, "fallback"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    pk, kind = peak()
    lines = ["# One SOS_FP64_TC step, per kernel", "",
             f"bf16 tensor peak for the slice products: {pk:.0f} TFLOP/s ({kind}).", "",
             "| workload | N = r | slices | step ms | slice products ms | products TFLOP/s | of peak "
             "| CUDA-core FP64 forward ms | kernels (ms per step) |", "|---|---|---|---|---|---|---|---|---|"]
    for name, n, two_d in (("quartic n=100", 99, 4), ("large n=20 2d=8", 20, 8)):
        pl = Plan(n, two_d)
        N = pl.N
        A = torch.from_numpy(sos_inputs.normal_matrix(N, N, 1, sigma=0.1)).cuda()
        p = torch.from_numpy(sos_inputs.normal_matrix(pl.M, 1, 2)[:, 0]).cuda()
        # the CUDA-core FP64 forward of the same A, for comparison
        pl.coeffs(A, "fp64")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pl.coeffs(A, "fp64")
        e1.record()
        torch.cuda.synchronize()
        native_ms = e0.elapsed_time(e1)
        for s in (4, 6, 8):
            opt = Optimizer(pl, A.clone(), prec="fp64_tc", lr=1e-6, slices=s)
            for _ in range(3):
                opt.step(p)
            torch.cuda.synchronize()
            L.sos_timing_reset()
            L.sos_timing_enable(True)
            steps = 5
            e0.record()
            for _ in range(steps):
                opt.step(p)
            e1.record()
            torch.cuda.synchronize()
            L.sos_timing_enable(False)
            rep = L.sos_timing_report()
            step_ms = e0.elapsed_time(e1) / steps
            prod_ms = sum(v[1] for k, v in rep.items() if k.startswith("tc_slices")) / steps
            units = s * (s + 1) // 2
            flops = units * float(N) * N * N
            tf = flops / (prod_ms / 1e3) / 1e12 if prod_ms > 0 else 0.0
            ks = ", ".join(f"{k} {v[1] / steps:.3f}" for k, v in sorted(rep.items(), key=lambda kv: -kv[1][1]))
            lines.append(f"| {name} | {N} | {s} | {step_ms:.2f} | {prod_ms:.2f} | {tf:.0f} | {tf / pk:.2f} "
                         f"| {native_ms:.1f} | {ks} |")
            print(lines[-1], flush=True)
            del opt
        del pl, A, p
        torch.cuda.empty_cache()
    text = "\n".join(lines) + "\n"
    print(text)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)


if __name__ == "__main__":
    main()
