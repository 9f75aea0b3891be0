#!/usr/bin/env python
"""Throughput of the loss-and-gradient step with its gradient-descent update.

Workload (one step = forward c(A) = sum_k q_k^2, residual and loss, adjoint
2 H(c - p) A, GD update): n = 20 variables, degree 2d = 8, N = r = 10,626
monomials/squares, M = 3,108,105 coefficients; target p = sum of 2000 squares
of N(0, 1)/sqrt(N) polynomials; A0 ~ N(0, 0.1^2); seeded, synthetic.  Every
operand is larger than L2 (bf16 A 226 MB, bf16 H 226 MB, index table 451 MB),
so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torchrun) every rank runs its own independent problem
(replicas; the step has no cross-GPU exchange in this build) and `value` is
the sum over ranks.  `--impl reference` times the CPU oracle on the same
workload (a bounded column sample, extrapolated) on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GD iters/s at ~3.1M coeffs"
UNIT = "iters/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="large_n20_2d8")
    ap.add_argument("--lr", type=float, default=1e-7)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="steps of the end-to-end timing (default: --steps, so both run as long)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=4096)
    ap.add_argument("--latency-requests", type=int, default=512)
    ap.add_argument("--plain-sample", type=int, default=64)
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d["bf16_tflops_sustained"]),
                "hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0,
                "source": "fallback"}


# -- clocks during the timed region ------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu=timestamp,{self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self, t0: float, t1: float):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                    ts += float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                    rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
                except (ValueError, IndexError):
                    continue
        os.unlink(self.path)
        inside = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05]
        use = inside or rows
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in use for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": max(r[2] for r in use),
                "reasons": reasons, "samples_in_region": len(inside), "samples": len(use)}


# -- traffic figures committed from ncu -------------------------------------------------

def sources_sha(paths) -> str:
    """First 16 hex digits of the SHA-256 over the listed files (repo-relative)."""
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str):
    """dram bytes per launch from profiles/traffic.json, or None when the kernel
    source changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
        rec = d[kernel]
        return rec["bytes_per_launch"] if sources_sha(rec["sources"]) == rec["sources_sha"] else None
    except Exception:
        return None


# -- CPU oracle sample --------------------------------------------------------------

def linear_fit(t_small, c_small, t_big, c_big, cols):
    """Extrapolates a per-iteration time that costs a + b * columns from two
    column widths to `cols` columns; (a, b, t(cols)).  The callers take the
    widths far enough apart that timing noise cannot flatten the slope."""
    b = max(t_big - t_small, 0.0) / (c_big - c_small)
    a = max(t_small - b * c_small, 0.0)
    return a, b, a + b * cols


def oracle_sample(w, widths=(8, 32), reps=2, seed=0):
    """Times one oracle GD iteration (coefficients, residual, gradient, update) on
    column slices of A and extrapolates linearly in the number of columns: the
    oracle's cost is a + b * columns (pair-table lookups plus per-column dot
    products and axpys).  Returns (iters/s for the full workload, description)."""
    import numpy as np

    import oracle
    import sos_inputs
    t_setup = time.time()
    o = oracle.Oracle(w.n, w.two_d)
    _ = o.prod
    p = sos_inputs.normal_matrix(w.M, 1, seed)[:, 0]     # values do not change the cost
    setup_s = time.time() - t_setup
    times = {}
    for cols in widths:
        A = sos_inputs.normal_matrix(w.N, cols, seed, sigma=w.init_sigma)
        best = None
        for _ in range(reps):
            t0 = time.perf_counter()
            loss, grad, _c = o.loss_grad(A, p)
            o.gd_step(A, grad, 1e-7)
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        times[cols] = best
    (c1, t1), (c2, t2) = sorted(times.items())
    a, b, t_full = linear_fit(t1, c1, t2, c2, w.cols)
    desc = (f"oracle GD iteration on column slices of width {list(times)} of the {w.N} x {w.cols} A "
            f"(full M = {w.M}), best of {reps}: {', '.join(f'{k} cols {v:.3f} s' for k, v in times.items())}; "
            f"fit t = {a:.3f} s + {b:.4f} s/col, extrapolated to {w.cols} cols = {t_full:.1f} s/iter; "
            f"setup (tables) {setup_s:.1f} s not timed")
    return 1.0 / t_full, desc, oracle.num_threads()


def blas_sample(w, widths=(256, 512), reps=2, seed=0):
    """Times one GD iteration written as dense CPU tensor ops (torch fp32 matmuls
    plus index_add / gather through the oracle's pair table; no code shared
    with the GPU path) on column slices of A, extrapolated linearly in the
    number of columns.  Returns (iters/s for the full workload, description,
    threads)."""
    import torch

    import oracle
    import sos_inputs
    t_setup = time.time()
    o = oracle.Oracle(w.n, w.two_d)
    idx = torch.from_numpy(o.prod.astype("int64")).reshape(-1)
    p = torch.from_numpy(sos_inputs.normal_matrix(w.M, 1, seed)[:, 0]).float()
    setup_s = time.time() - t_setup
    times = {}
    for cols in widths:
        A = torch.from_numpy(sos_inputs.normal_matrix(w.N, cols, seed, sigma=w.init_sigma)).float()
        best = None
        for _ in range(reps):
            t0 = time.perf_counter()
            G = A @ A.T
            c = torch.zeros(w.M).index_add_(0, idx, G.reshape(-1))
            resid = c - p
            _loss = 0.5 * float(torch.dot(resid, resid))
            H = resid[idx].reshape(w.N, w.N)
            A -= 1e-7 * (2.0 * (H @ A))
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        times[cols] = best
    (c1, t1), (c2, t2) = sorted(times.items())
    a, b, t_full = linear_fit(t1, c1, t2, c2, w.cols)
    desc = (f"torch CPU fp32 GD iteration (A A^T, index_add into c, gather H, 2 H A) on column slices of "
            f"width {list(times)}, best of {reps}: {', '.join(f'{k} cols {v:.3f} s' for k, v in times.items())}; "
            f"fit t = {a:.3f} s + {b:.5f} s/col, extrapolated to {w.cols} cols = {t_full:.1f} s/iter; "
            f"setup (pair table) {setup_s:.1f} s not timed")
    return 1.0 / t_full, desc, torch.get_num_threads()


def run_reference(args):
    import sos_inputs
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    w = sos_inputs.WORKLOADS[args.workload]
    o = oracle.Oracle(w.n, w.two_d)
    t0 = time.time()
    _ = o.prod
    p = sos_inputs.normal_matrix(w.M, 1, 0)[:, 0]          # values do not change the cost
    setup = time.time() - t0
    cols = 8
    A = sos_inputs.normal_matrix(w.N, cols, 0, sigma=w.init_sigma)

    def step():
        loss, grad, _c = o.loss_grad(A, p)
        o.gd_step(A, grad, 1e-7)

    # a fourfold width, once, gives the per-column part of the cost
    wide = 4 * cols
    A2 = sos_inputs.normal_matrix(w.N, wide, 1, sigma=w.init_sigma)

    def step_wide():
        loss, grad, _c = o.loss_grad(A2, p)
        o.gd_step(A2, grad, 1e-7)

    for _ in range(args.warmup):
        step()
    t_2 = None
    for _ in range(2):
        t_a = time.perf_counter()
        step_wide()
        dt = time.perf_counter() - t_a
        t_2 = dt if t_2 is None else min(t_2, dt)
    t_a = time.perf_counter()
    for _ in range(args.steps):
        step()
    t_1 = (time.perf_counter() - t_a) / args.steps
    a, b, t_full = linear_fit(t_1, cols, t_2, wide, w.cols)
    value = 1.0 / t_full
    sample = (f"each timed step: one oracle GD iteration on a {w.N} x {cols} column slice of A (full M = "
              f"{w.M}); {t_1:.3f} s/step, {wide} columns {t_2:.3f} s; cost a + b*cols with a = {a:.3f} s, "
              f"b = {b:.4f} s/col; value extrapolated to {w.cols} columns = {t_full:.1f} s/iter; "
              f"table setup {setup:.1f} s untimed")
    # ms_per_step and steps describe the column-slice steps that ran; value is
    # the full-width iteration rate the fit extrapolates from them
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w, world),
            "extrapolated": True,
            "fit": {"model": "t(cols) = a + b * cols", "a_s": a, "b_s_per_col": b, "cols_timed": [cols, wide],
                    "t_timed_s": [t_1, t_2], "cols_full": w.cols, "t_full_s": t_full},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_of(w, world):
    return {"workload": w.name, "n": w.n, "two_d": w.two_d, "N": w.N, "M": w.M, "r": w.cols,
            "target_squares": w.squares, "optimizer": "gd",
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs exceed L2 (bf16 A 226 MB, bf16 H 226 MB, idx 451 MB); no flush"}


# -- serving stream ------------------------------------------------------------------

def run_serving(args):
    """Served mixed stream vs one problem at a time through the single-problem path.

    Requests: n uniform in {3..8}, 2d in {4, 6, 8}, r = N; even ids SOS (sum of
    floor(N/2) random squares), odd ids made negative at a point.  Inputs are
    built on the device before any timing.  Throughput: all requests offered at
    once.  Latency (arrival -> verdict): Poisson arrivals at 0.5x and 1.5x the
    plain path's measured capacity."""
    import numpy as np
    import torch

    from paper_2410_19844_gb300 import _lib as L
    from paper_2410_19844_gb300.server import Server, latency_stats, run_plain
    from paper_2410_19844_gb300.workloads import build_jobs

    jobs = build_jobs(args.serving_requests, 1.0, seed=0, arrivals=False)
    sample = jobs[:args.plain_sample]
    run_plain(sample[:4])                                    # warm-up (plans, graphs)
    t0 = time.perf_counter()
    plain = run_plain(sample)
    t_plain = time.perf_counter() - t0
    plain_rate = len(sample) / t_plain

    srv = Server(capacity=1024, steps_per_tick=32)
    srv.run(jobs[:8])                                          # warm-up
    srv_launch0 = srv.launches
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    served = srv.run(jobs)
    t_served = time.perf_counter() - t0
    launches = srv.launches - srv_launch0
    served_rate = len(jobs) / t_served
    by_rid = {v.rid: v for v in served}
    agree = sum(by_rid[v.rid].verdict == v.verdict for v in plain)
    counts = {"sos": 0, "not_converged": 0, "error": 0}
    names = {L.SOS_VERDICT_SOS: "sos", L.SOS_VERDICT_NOT_CONVERGED: "not_converged", L.SOS_VERDICT_ERROR: "error"}
    for v in served:
        counts[names[v.verdict]] += 1
    sos_ok = sum(1 for v in served if v.rid % 2 == 0 and v.verdict == L.SOS_VERDICT_SOS)
    neg_ok = sum(1 for v in served if v.rid % 2 == 1 and v.verdict == L.SOS_VERDICT_NOT_CONVERGED)

    latency = {}
    for mult in (0.5, 1.5):
        rate = mult * plain_rate
        stream = build_jobs(args.latency_requests, rate, seed=1)
        out = srv.run(stream)
        st = latency_stats(out)
        latency[f"{mult}x_plain"] = {"rate_per_s": rate, "requests": len(stream), **st}
    srv.close()
    return {"workload": "serving_n3-8_2d4-8", "requests": len(jobs), "served_verdicts_per_s": served_rate,
            "served_s": t_served, "plain_verdicts_per_s": plain_rate, "plain_sample": len(sample),
            "speedup_vs_plain": served_rate / plain_rate, "verdict_agreement_with_plain": f"{agree}/{len(sample)}",
            "verdicts": counts, "sos_targets_certified": f"{sos_ok}/{(len(jobs) + 1) // 2}",
            "negative_targets_not_converged": f"{neg_ok}/{len(jobs) // 2}",
            "latency": latency, "slots": srv.capacity, "steps_per_tick": 32, "gpu_launches": launches,
            "note": "grouped FP32 then FP64 (FP32 adjoint) steps, captured graphs of 32 steps; "
                    "plain = sos_step launches per problem, one problem at a time, same decision rule"}


# -- our arm -------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import sos_inputs
    from paper_2410_19844_gb300 import _lib as L
    from paper_2410_19844_gb300.engine import Optimizer, Plan

    rank, local_rank, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = sos_inputs.WORKLOADS[args.workload]
    L.lib()

    # inputs: target p = c(G) by the library's own FP64 forward; A0 ~ N(0, 0.1^2)
    G = torch.from_numpy(sos_inputs.generator(w, rank)).to(dev)
    p64 = Plan(w.n, w.two_d, r=G.shape[1]).coeffs(G.contiguous(), "fp64")
    p = p64.float().contiguous()
    del G
    A0 = torch.from_numpy(sos_inputs.init_A(w, rank).astype(np.float32))
    plan = Plan(w.n, w.two_d)
    A = A0.to(dev).contiguous()
    opt = Optimizer(plan, A, prec="bf16", optimizer="gd", lr=args.lr)
    stream = torch.cuda.current_stream()
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    for _ in range(args.warmup):
        opt.step(p)
    torch.cuda.synchronize()

    def timed_steps(per_kernel: bool):
        """K steps between a barrier and synchronisations, timed by CUDA events on
        the launching stream; with per_kernel the library also records events
        around every launch (sos_timing_*)."""
        L.sos_timing_reset()
        L.sos_timing_enable(per_kernel)
        n0 = L.sos_launch_count()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0 = time.time()
        e0.record(stream)
        for _ in range(args.steps):
            opt.step(p)
        e1.record(stream)
        torch.cuda.synchronize()
        w1 = time.time()
        if world > 1:
            dist.barrier()
        L.sos_timing_enable(False)
        rep = L.sos_timing_report() if per_kernel else {}
        L.sos_timing_reset()
        return e0.elapsed_time(e1), L.sos_launch_count() - n0, rep, w0, w1

    sampler = ClockSampler(local_rank)
    sampler.start()
    time.sleep(0.3)
    # the headline: the steps alone; then the same steps with per-kernel events
    # (the roofline's launch durations)
    elapsed_ms, launches, _, t_wall0, t_wall1 = timed_steps(False)
    inst_ms, _, kernels, _, t_wall2 = timed_steps(True)
    clocks = sampler.stop(t_wall0, t_wall2)
    status = plan.status("bf16")
    loss_now = float(opt.loss[0].item())
    if world > 1:
        t = torch.tensor([elapsed_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    ms_per_step = elapsed_ms / args.steps
    value = world * args.steps / (elapsed_ms / 1000.0)

    # roofline of the dominant kernel, from the events recorded in the timed region
    N, r = w.N, w.cols
    alg_flops = {"tc_forward": float(N) * N * r, "tc_adjoint": 2.0 * N * N * r,
                 "tc_adjoint_update": 2.0 * N * N * r}
    peaks = measured_peaks()
    dom = max(kernels.items(), key=lambda kv: kv[1][1])
    dom_name, (dom_launches, dom_ms) = dom
    avg_ms = dom_ms / dom_launches
    roof = None
    # The matching peak: the burst figure for a short timed region or one run at
    # the maximum SM clock, the sustained (power-capped) figure otherwise.
    region_s = inst_ms / 1000.0
    sm, smax = clocks.get("sm_mhz"), clocks.get("sm_max_mhz")
    burst = region_s < 1.0 or (sm is not None and smax and sm >= 0.97 * smax)
    peak_key = "bf16_tflops" if burst else "bf16_tflops_sustained"
    if dom_name in alg_flops:
        achieved = alg_flops[dom_name] / (avg_ms / 1000.0) / 1e12
        peak = peaks[peak_key]
        roof = {"bound": "tensor", "kernel": dom_name, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_kind": (f"bf16 dense {'burst' if burst else 'sustained'}, {peaks['source']} "
                              f"(timed region {region_s:.2f} s, median SM {sm} of {smax} MHz)"),
                "frac_of_burst": achieved / peaks["bf16_tflops"],
                "frac_of_sustained": achieved / peaks["bf16_tflops_sustained"],
                "alg_flops_per_launch": alg_flops[dom_name], "avg_launch_ms": avg_ms,
                "traffic": committed_traffic(dom_name)}
        if sm:
            # clock-normalised: the launch in SM cycles, and the work per SM per cycle
            roof["kcycles_per_launch"] = avg_ms * sm
            roof["flop_per_sm_cycle"] = alg_flops[dom_name] / (avg_ms * 1e-3 * sm * 1e6 * num_sms)
    step_tflops = 3.0 * N * N * r / (ms_per_step / 1000.0) / 1e12
    per_kernel = {k: {"launches": n, "ms_per_launch": ms / n} for k, (n, ms) in kernels.items()}

    # end to end through the public API: every step copies its input (the
    # target p) from pinned host memory, runs sos_step and reads the loss back
    # on the host.  The loop is pipelined as a training loop would be: step k's
    # copy runs on a copy stream into one of two device buffers while step k-1
    # computes, and the host reads step k-1's loss after enqueueing step k.  A
    # second figure also moves the state A both ways every step, synchronously.
    e2e = None
    if not args.no_e2e:
        A_host = A0.clone().pin_memory()
        p_host = p.cpu().pin_memory()
        loss_host = torch.zeros(2, dtype=torch.float64).pin_memory()
        k2 = max(1, args.e2e_steps if args.e2e_steps > 0 else args.steps)

        def timed(step_fn):
            for _ in range(2):
                step_fn()
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(k2):
                step_fn()
            f1.record(stream)
            torch.cuda.synchronize()
            ms = f0.elapsed_time(f1)
            if world > 1:
                t = torch.tensor([ms], device=dev)
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                ms = float(t.item())
            return ms

        A_dev = A0.to(dev).contiguous()
        p_dev = torch.empty_like(p)
        opt2 = Optimizer(plan, A_dev, prec="bf16", optimizer="gd", lr=args.lr)
        p_bufs = [torch.empty_like(p), torch.empty_like(p)]
        copy_stream = torch.cuda.Stream(device=dev)
        ev_copied = [torch.cuda.Event(), torch.cuda.Event()]
        ev_used = [torch.cuda.Event(), torch.cuda.Event()]
        ev_loss = [torch.cuda.Event(), torch.cuda.Event()]
        loss_ring = torch.zeros(2, 2, dtype=torch.float64).pin_memory()
        ring = {"k": 0, "pending": None, "finite": True}

        def read_pending():
            j = ring["pending"]
            if j is not None:
                ev_loss[j].synchronize()
                ring["finite"] &= bool(torch.isfinite(loss_ring[j][0]))
                ring["pending"] = None

        def e2e_step():
            s = ring["k"] % 2
            copy_stream.wait_event(ev_used[s])          # buffer s was last read by step k - 2
            with torch.cuda.stream(copy_stream):
                p_bufs[s].copy_(p_host, non_blocking=True)
            ev_copied[s].record(copy_stream)
            stream.wait_event(ev_copied[s])
            opt2.step(p_bufs[s])
            ev_used[s].record(stream)
            loss_ring[s].copy_(opt2.loss, non_blocking=True)
            ev_loss[s].record(stream)
            read_pending()                               # step k - 1's loss, on the host
            ring["pending"] = s
            ring["k"] += 1

        e2e_ms = timed(e2e_step)
        read_pending()
        if not ring["finite"]:
            raise RuntimeError("e2e: a step returned a non-finite loss")

        A_rt = torch.empty_like(A)
        opt3 = Optimizer(plan, A_rt, prec="bf16", optimizer="gd", lr=args.lr)

        def roundtrip_step():
            A_rt.copy_(A_host, non_blocking=True)
            opt3.state.flags = 0              # A changed outside sos_step
            p_dev.copy_(p_host, non_blocking=True)
            opt3.step(p_dev)
            loss_host.copy_(opt3.loss, non_blocking=True)
            A_host.copy_(A_rt, non_blocking=True)
            torch.cuda.current_stream().synchronize()

        rt_ms = timed(roundtrip_step)
        abytes = A.numel() * 4
        e2e = {"value": world * k2 / (e2e_ms / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": p.numel() * 4, "d2h_bytes_per_step": 16,
               "steps": k2, "ms_per_step": e2e_ms / k2,
               "note": "per step: target p copied host->device from pinned memory on a copy stream (two device "
                       "buffers, overlapping the previous step), sos_step through the C ABI, loss copied to "
                       "pinned host memory and read on the host after the next step is enqueued (the iterate "
                       "A stays resident, as a model's weights would)",
               "state_roundtrip": {"value": world * k2 / (rt_ms / 1000.0), "unit": UNIT,
                                   "h2d_bytes_per_step": abytes + p.numel() * 4,
                                   "d2h_bytes_per_step": abytes + 16, "ms_per_step": rt_ms / k2,
                                   "note": "A also copied host->device and back every step"}}

    cpu = cpu_blas = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, desc, cores = oracle_sample(w)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
        v, desc, cores = blas_sample(w)
        cpu_blas = {"value": v, "unit": UNIT, "cores": cores, "kind": "torch-cpu-blas", "sample": desc}

    serving = None
    if rank == 0 and not args.no_serving:
        serving = run_serving(args)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
                "config": config_of(w, world), "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
                "roofline": roof, "cpu_baseline": cpu, "cpu_blas": cpu_blas, "serving": serving,
                "step": {"alg_tflops": step_tflops,
                         "frac": step_tflops / peaks[peak_key], "peak_key": peak_key,
                         "frac_of_sustained": step_tflops / peaks["bf16_tflops_sustained"],
                         "frac_of_burst": step_tflops / peaks["bf16_tflops"],
                         "kernels": per_kernel, "status": status, "loss_after": loss_now,
                         "ms_per_step_with_kernel_events": inst_ms / args.steps,
                         "note": "value: K steps timed alone; kernels and roofline: the same K steps again with "
                                 "CUDA events around every launch"}}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
