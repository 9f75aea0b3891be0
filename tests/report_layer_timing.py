"""Report: time of one step of the network with its first layer (Sec. 2), per
kernel, at the paper's sizes: quartic forms in nf = 31 and nf = 101 variables
(the n = 30 and n = 100 problems of Sec. 3.1, dehomogenised), k = N squares,
first-layer width m = nf and 2 nf, FP32 and BF16 steps (Adam).

Each configuration: 3 warm-up steps, then 10 timed steps with per-kernel CUDA
events (sos_timing_*) and the whole-step time from events around the loop.
The first layer's three GEMMs do 6 k nf^2 m flops per step: on the CUDA cores
("layer_gemm"), and in BF16 steps with nf, m >= 64 two of them on the tensor
cores ("tc_gemm_diag").  Their rate is compared with the FP32 FMA peak of the
GPU, 152 SMs x 128 lanes x 2 flops x the SM clock (given on the command line,
default 1.9 GHz) -- for the mixed BF16 rows that ratio is only indicative.
The core pass does 3 N^2 k flops.

    python tests/report_layer_timing.py [--clock-ghz 1.9] [--out FILE]
"""
import argparse
import os
import sys
from math import comb

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import sos_inputs  # noqa: E402
from paper_2410_19844_gb300 import _lib as L  # noqa: E402
from paper_2410_19844_gb300.engine import Layer, LayerOptimizer, Plan  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--clock-ghz", type=float, default=1.9)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    fp32_peak = 152 * 128 * 2 * args.clock_ghz * 1e9 / 1e12
    lines = ["# One step of the network with its first layer, per kernel", "",
             f"FP32 FMA peak used for the layer GEMMs: {fp32_peak:.1f} TFLOP/s "
             f"(152 SMs x 128 lanes x 2 x {args.clock_ghz} GHz).", "",
             "| nf | m | prec | step ms | core pass TFLOP/s | layer_gemm ms/step | layer GEMM TFLOP/s "
             "| of FP32 peak | kernels (ms per step) |", "|---|---|---|---|---|---|---|---|---|"]
    for nf in (31, 101):
        N = comb(nf + 1, 2)
        pl = Plan(nf - 1, 4, N)
        p = torch.from_numpy(sos_inputs.normal_matrix(pl.M, 1, 3)[:, 0]).float().cuda()
        for m in (nf, 2 * nf):
            lay = Layer(pl, m)
            for prec in ("fp32", "bf16"):
                B = torch.from_numpy(sos_inputs.normal_matrix(N, nf * m, 1, sigma=0.05)).float().cuda()
                A1 = torch.from_numpy(sos_inputs.normal_matrix(m, nf, 2, sigma=0.3)).float().cuda()
                opt = LayerOptimizer(lay, B, A1, prec=prec, lr=1e-4)
                for _ in range(3):
                    opt.step(p)
                torch.cuda.synchronize()
                L.sos_timing_reset()
                L.sos_timing_enable(True)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                steps = 10
                e0.record()
                for _ in range(steps):
                    opt.step(p)
                e1.record()
                torch.cuda.synchronize()
                L.sos_timing_enable(False)
                rep = L.sos_timing_report()
                step_ms = e0.elapsed_time(e1) / steps
                # the layer's GEMMs: CUDA-core "layer_gemm", and in BF16 steps with nf, m >= 64 the
                # tensor-core products "tc_gemm_diag"
                gemm_ms = (rep.get("layer_gemm", (0, 0.0))[1] + rep.get("tc_gemm_diag", (0, 0.0))[1]) / steps
                core_names = [k for k in rep
                              if not k.startswith("layer_") and k not in ("update", "tc_gemm_diag")]
                core_ms = sum(rep[k][1] for k in core_names) / steps
                layer_flops = 6.0 * N * nf * nf * m
                core_flops = 3.0 * N * N * N
                gemm_tf = layer_flops / (gemm_ms / 1e3) / 1e12 if gemm_ms > 0 else 0.0
                core_tf = core_flops / (core_ms / 1e3) / 1e12 if core_ms > 0 else 0.0
                ks = ", ".join(f"{k} {v[1] / steps:.3f}" for k, v in sorted(rep.items(), key=lambda kv: -kv[1][1]))
                lines.append(f"| {nf} | {m} | {prec} | {step_ms:.3f} | {core_tf:.1f} | {gemm_ms:.3f} | {gemm_tf:.1f} "
                             f"| {gemm_tf / fp32_peak:.2f} | {ks} |")
                print(lines[-1], flush=True)
                del opt, B, A1
            del lay
        del pl
    text = "\n".join(lines) + "\n"
    print(text)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)


if __name__ == "__main__":
    main()
