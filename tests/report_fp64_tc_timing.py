"""Report: one SOS_FP64_TC step, per kernel, against the tensor roofline.

Workloads: the n = 100 quartic form (n = 99 variables dehomogenised, 2d = 4,
N = r = 5050) and the large workload (n = 20, 2d = 8, N = r = 10,626); slices
s = 4, 6, 8.  Each configuration: 3 warm-up steps, then 30 timed steps (Adam)
with per-kernel CUDA events and nvidia-smi sampling the SM clock and the
board power every 100 ms.  Algorithmic work of the slice products: diagonal
units N^2 r flops each (upper triangle), cross units 2 N^2 r (every tile), s
(s+1)/2 forward passes in all; rates are compared with the measured bf16
tensor peak in MEASURED_PEAKS.json (sustained).  The CUDA-core FP64 forward
of the same A is timed beside it.  With SOS_SLICE_FP8=1 in the environment
the slices are E4M3 bytes of 4-bit digits, s' = ceil(5 s / 4) of them: s'
(s'+1)/2 passes, against the E4M3 tensor peak (the measured bf16 peak times
the nominal ratio 2).

With --gemm-peaks the report first times cuBLAS GEMMs of 8192^3 in bf16
(torch.matmul) and E4M3 (torch._scaled_mm, bf16 output): 10 calls as a burst,
then about 4 s of calls, with the clocks and power of the long run.

    [SOS_SLICE_FP8=1|0] python tests/report_fp64_tc_timing.py [--gemm-peaks] [--workloads a,b] [--out FILE]

--workloads picks from quartic100 (n = 99, 2d = 4, N = 5050), n10 (n = 10,
2d = 10, N = 3003), medium (n = 18, 2d = 8, N = 7315) and large (n = 20,
2d = 8, N = 10,626); the default is quartic100,large.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

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


class Clocks:
    """nvidia-smi sampling of the SM clock and power while a block runs (read only)."""

    def __enter__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=clocks.sm,power.draw,clocks_event_reasons.active",
                                       "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            self.p.wait()
        self.f.seek(0)
        rows = []
        for line in self.f:
            parts = [x.strip() for x in line.split(",")]
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[2]))
            except (ValueError, IndexError):
                pass
        self.f.close()
        os.unlink(self.f.name)
        loaded = [r for r in rows if r[1] > 300] or rows
        if not loaded:
            self.text = "n/a"
            return False
        sm = sorted(r[0] for r in loaded)
        pw = sorted(r[1] for r in loaded)
        reasons = sorted({r[2] for r in loaded})
        self.text = f"{sm[len(sm) // 2]:.0f} MHz, {pw[len(pw) // 2]:.0f} W, {' '.join(reasons)}"
        return False


def gemm_peaks(lines):
    M = 8192
    a = torch.randn(M, M, device="cuda", dtype=torch.bfloat16)
    b = torch.randn(M, M, device="cuda", dtype=torch.bfloat16)
    runs = [("bf16", lambda: a @ b.t())]
    try:
        a8, b8 = a.to(torch.float8_e4m3fn), b.to(torch.float8_e4m3fn)
        one = torch.tensor(1.0, device="cuda")
        fp8 = lambda: torch._scaled_mm(a8, b8.t(), scale_a=one, scale_b=one, out_dtype=torch.bfloat16)  # noqa: E731
        fp8()
        runs.append(("E4M3", fp8))
    except Exception as ex:  # an older torch without _scaled_mm on this GPU
        lines.append(f"E4M3 GEMM unavailable: {type(ex).__name__}")
    lines += ["| cuBLAS GEMM 8192^3 | burst TFLOP/s | sustained TFLOP/s | calls | clocks (median SM, power, reasons) |",
              "|---|---|---|---|---|"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, fn in runs:
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(10):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 10
        calls = max(10, int(4000 / ms))
        with Clocks() as clk:
            e0.record()
            for _ in range(calls):
                fn()
            e1.record()
            torch.cuda.synchronize()
        sus = 2 * M ** 3 / (e0.elapsed_time(e1) / calls / 1e3) / 1e12
        lines.append(f"| {name} | {2 * M ** 3 / (ms / 1e3) / 1e12:.0f} | {sus:.0f} | {calls} | {clk.text} |")
        print(lines[-1], flush=True)
    lines.append("")
    del a, b
    torch.cuda.empty_cache()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--gemm-peaks", action="store_true")
    ap.add_argument("--workloads", default="quartic100,large")
    args = ap.parse_args()
    pk, kind = peak()
    fp8 = os.environ.get("SOS_SLICE_FP8") == "1"      # unset: bf16 slices at every size here (r <= 17,458)
    if fp8:
        pk, kind = 2 * pk, kind + " bf16 x 2"
    fmt = "E4M3 4-bit" if fp8 else "bf16 5-bit"
    lines = [f"# One SOS_FP64_TC step, per kernel ({fmt} slices)", "",
             "Command: " + ("SOS_SLICE_FP8=1 " if fp8 else "") + "python tests/report_fp64_tc_timing.py"
             + (" --gemm-peaks" if args.gemm_peaks else "")
             + (f" --workloads {args.workloads}" if args.workloads != "quartic100,large" else ""), ""]
    if args.gemm_peaks:
        gemm_peaks(lines)
    lines += [f"tensor peak for the slice products: {pk:.0f} TFLOP/s ({kind}).", "",
              "| workload | N = r | slices | step ms | slice products ms | products TFLOP/s | of peak "
              "| clocks (median SM, power, reasons) | CUDA-core FP64 forward ms | kernels (ms per step) |",
              "|---|---|---|---|---|---|---|---|---|---|"]
    known = {"quartic100": ("quartic n=100", 99, 4), "n10": ("n=10 2d=10", 10, 10),
             "medium": ("medium n=18 2d=8", 18, 8), "large": ("large n=20 2d=8", 20, 8)}
    for name, n, two_d in (known[k] for k in args.workloads.split(",")):
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
            steps = 30
            with Clocks() as clk:
                e0.record()
                for _ in range(steps):
                    opt.step(p)
                e1.record()
                torch.cuda.synchronize()
            L.sos_timing_enable(False)
            rep = L.sos_timing_report()
            step_ms = e0.elapsed_time(e1) / steps
            prod_ms = sum(v[1] for k, v in rep.items() if k.startswith("tc_slices")) / steps
            sf = (5 * s + 3) // 4 if fp8 else s
            units = sf * (sf + 1) // 2
            flops = units * float(N) * N * N
            tf = flops / (prod_ms / 1e3) / 1e12 if prod_ms > 0 else 0.0
            ks = ", ".join(f"{k} {v[1] / steps:.3f}" for k, v in sorted(rep.items(), key=lambda kv: -kv[1][1]))
            lines.append(f"| {name} | {N} | {s} | {step_ms:.2f} | {prod_ms:.2f} | {tf:.0f} | {tf / pk:.2f} "
                         f"| {clk.text} | {native_ms:.1f} | {ks} |")
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
