"""Continuous-batching server for streams of sum-of-squares queries.

Each query is a target p (degree <= 2d in n variables) and a start point A0;
the answer is a verdict: SOS (an iterate with ||c(A) - p|| <= cert_tol ||p||
in FP64 -- the paper's accuracy criterion, Sec. 3), NOT_CONVERGED (a gradient
method never proves the opposite), ERROR (non-finite values) or TIMEOUT (the
request's deadline passed before a verdict).

Requests join a running FP32 group (library groups: every active problem's
tiles in one set of launches, replayed as a captured CUDA graph of K steps)
as soon as they have arrived and a slot and enough of the HBM budget are
free.  Every K steps the server reads all losses at once and moves each
problem on: to the FP64 group (with its Adam state and step count) when its
FP32 residual is small or stops improving, to a verdict when the FP64
residual of an iterate passes the certificate, or to NOT_CONVERGED when it
stalls or runs out of steps.  Finished problems free their slot for the next
arrival, so the GPU always works on a mixed batch.  A problem's iterates do
not depend on the other problems in its group.

`run_plain` serves the same jobs one at a time through the single-problem
path (sos_step per launch), with the same decision rule: the baseline the
grouped server is measured against.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np
import torch

from . import _lib as L
from .engine import Optimizer, Plan, _ptr, _stream_handle


@dataclass
class Job:
    rid: int
    arrival_s: float
    n: int
    two_d: int
    make: Callable[[], tuple]        # () -> (p64, A0_64): float64 device tensors


VERDICT_TIMEOUT = -2   # server-level verdict: the request's deadline passed


@dataclass
class Verdict:
    rid: int
    verdict: int
    rel: float                       # FP64 relative residual of the returned iterate (or best seen)
    steps_fp32: int
    steps_fp64: int
    arrival_s: float
    done_s: float

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


@dataclass
class _Active:
    job: Job
    plan: Plan
    slot: int
    phase: str                       # "fp32" or "fp64"
    bufs: dict
    pp: float = 0.0
    best: float = float("inf")
    last_gain: float = float("inf")
    stall: int = 0
    steps32: int = 0
    steps64: int = 0
    footprint: int = 0
    fresh: bool = False
    lr: float = 0.0
    decays: int = 0


@dataclass
class Policy:
    lr32: float = 1e-2
    lr64: float = 1e-2
    cert_tol: float = 1e-8
    switch_rel: float = 1e-7         # FP32 -> FP64 at once below this
    promote_rel: float = 1e-5        # ... or, when FP32 stalls, only below this: FP32 resolves
                                     # residuals far above its ~1e-7 floor, so a stall above
                                     # 1e-5 (after the step-size cuts) is the optimiser's, and
                                     # FP64 steps would not reach the certificate either
    stall_checks: int = 3            # checks without a 1% gain
    decay: float = 0.1               # on a stall above target, scale the step size by this ...
    max_decays: int = 2              # ... at most this many times per stage before deciding
    max_fp32_steps: int = 8000
    max_fp64_steps: int = 3000
    deadline_s: float = float("inf")  # arrival -> verdict budget; past it the request times out


def _footprint(plan: Plan, elt: int) -> int:
    N, M = plan.N, plan.M
    return elt * (5 * N * N + 3 * M) + 64 * 1024


class Server:
    def __init__(self, capacity: int = 256, hbm_budget: int = 16 << 30, steps_per_tick: int = 32,
                 policy: Optional[Policy] = None, optimizer: str = "adam", fp32_adjoint: bool = True,
                 fast_fp64: bool = True):
        self.capacity = capacity
        self.budget = hbm_budget
        self.K = steps_per_tick
        self.policy = policy or Policy()
        opt = L.SOS_ADAM if optimizer == "adam" else L.SOS_GD
        self.g32 = L.sos_group_create(L.SOS_FP32, capacity, opt)
        self.g64 = L.sos_group_create(L.SOS_FP64, capacity, opt,
                                      flags=(L.SOS_GROUP_FP32_ADJOINT if fp32_adjoint else 0)
                                      | (L.SOS_GROUP_FAST_FP64 if fast_fp64 else 0))
        self.plans: dict = {}
        self.free32 = list(range(capacity))[::-1]
        self.free64 = list(range(capacity))[::-1]
        self.active32: dict = {}
        self.active64: dict = {}
        self.used = 0
        self.peak_used = 0
        self.ticks = 0
        self.group_steps = 0
        self.launches = 0
        self.losses32 = np.zeros(2 * capacity)
        self.losses64 = np.zeros(2 * capacity)
        # each group ticks on its own stream, so the FP64 group's tick runs beside
        # the FP32 group's and beside the host's bookkeeping of FP32 results
        self.s32 = torch.cuda.Stream()
        self.s64 = torch.cuda.Stream()

    def close(self):
        if self.g32:
            L.sos_group_destroy(self.g32)
            L.sos_group_destroy(self.g64)
            self.g32 = self.g64 = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plan(self, n: int, two_d: int) -> Plan:
        key = (n, two_d)
        if key not in self.plans:
            self.plans[key] = Plan(n, two_d)
        return self.plans[key]

    # -- admission and phase changes ----------------------------------------------
    def _admit(self, job: Job) -> Optional[_Active]:
        plan = self.plan(job.n, job.two_d)
        need = _footprint(plan, 4)
        if not self.free32 or self.used + need > self.budget:
            return None
        st = _stream_handle()
        p64, A0 = job.make()
        N, M = plan.N, plan.M
        b = {"p64": p64}
        b["p32"] = torch.empty(M, dtype=torch.float32, device="cuda")
        b["A32"] = torch.empty(N, N, dtype=torch.float32, device="cuda")
        L.sos_convert(_ptr(p64), L.SOS_FP64, _ptr(b["p32"]), L.SOS_FP32, M, st)
        L.sos_convert(_ptr(A0), L.SOS_FP64, _ptr(b["A32"]), L.SOS_FP32, N * N, st)
        b["m32"] = torch.zeros(N, N, dtype=torch.float32, device="cuda")
        b["v32"] = torch.zeros(N, N, dtype=torch.float32, device="cuda")
        b["s32"] = torch.empty(L.sos_group_scratch_size(plan.handle, L.SOS_FP32), dtype=torch.uint8,
                               device="cuda")
        slot = self.free32.pop()
        L.sos_group_set(self.g32, slot, plan.handle, _ptr(b["A32"]), _ptr(b["m32"]), _ptr(b["v32"]),
                        _ptr(b["p32"]), _ptr(b["s32"]), self.policy.lr32, 0)
        self.used += need
        self.peak_used = max(self.peak_used, self.used)
        a = _Active(job, plan, slot, "fp32", b, footprint=need, lr=self.policy.lr32)
        self.active32[slot] = a
        return a

    def _promote(self, a: _Active) -> bool:
        """FP32 -> FP64 with the current iterate and Adam state."""
        need = _footprint(a.plan, 8)
        if not self.free64 or self.used + need > self.budget:
            return False
        st = _stream_handle()
        N = a.plan.N
        cur, _, taken = L.sos_group_state(self.g32, a.slot)
        b = a.bufs
        b["A64"] = torch.empty(N, N, dtype=torch.float64, device="cuda")
        b["m64"] = torch.empty(N, N, dtype=torch.float64, device="cuda")
        b["v64"] = torch.empty(N, N, dtype=torch.float64, device="cuda")
        L.sos_convert(cur, L.SOS_FP32, _ptr(b["A64"]), L.SOS_FP64, N * N, st)
        L.sos_convert(_ptr(b["m32"]), L.SOS_FP32, _ptr(b["m64"]), L.SOS_FP64, N * N, st)
        L.sos_convert(_ptr(b["v32"]), L.SOS_FP32, _ptr(b["v64"]), L.SOS_FP64, N * N, st)
        b["s64"] = torch.empty(L.sos_group_scratch_size(a.plan.handle, L.SOS_FP64), dtype=torch.uint8,
                               device="cuda")
        self._release32(a)
        slot = self.free64.pop()
        a.lr = self.policy.lr64 * (a.lr / self.policy.lr32)    # keep the FP32 stage's decays
        L.sos_group_set(self.g64, slot, a.plan.handle, _ptr(b["A64"]), _ptr(b["m64"]), _ptr(b["v64"]),
                        _ptr(b["p64"]), _ptr(b["s64"]), a.lr, a.steps32)
        a.slot, a.phase, a.fresh, a.decays = slot, "fp64", True, 0
        a.stall, a.last_gain = 0, float("inf")
        self.used += need
        a.footprint += need
        self.peak_used = max(self.peak_used, self.used)
        self.active64[slot] = a
        return True

    def _release32(self, a: _Active):
        L.sos_group_clear(self.g32, a.slot)
        del self.active32[a.slot]
        self.free32.append(a.slot)
        for k in ("A32", "m32", "v32", "s32", "p32"):
            a.bufs.pop(k, None)
        self.used -= _footprint(a.plan, 4)
        a.footprint -= _footprint(a.plan, 4)

    def _retire(self, a: _Active, verdict: int, rel: float, now: float, out: list):
        if a.phase == "fp32":
            self._release32(a)
        else:
            L.sos_group_clear(self.g64, a.slot)
            del self.active64[a.slot]
            self.free64.append(a.slot)
            self.used -= _footprint(a.plan, 8)
        a.bufs.clear()
        out.append(Verdict(a.job.rid, verdict, rel, a.steps32, a.steps64, a.job.arrival_s, now))

    # -- the loop ---------------------------------------------------------------
    def run(self, jobs: list, clock_start: Optional[float] = None) -> list:
        """Serves `jobs` (sorted by arrival_s, seconds from clock start) and returns
        their verdicts in completion order."""
        pol = self.policy
        pending = sorted(jobs, key=lambda j: j.arrival_s)
        pi = 0
        out: list = []
        t0 = time.perf_counter() if clock_start is None else clock_start
        cur = torch.cuda.current_stream()
        h32, h64 = _stream_handle(self.s32), _stream_handle(self.s64)
        while pi < len(pending) or self.active32 or self.active64:
            now = time.perf_counter() - t0
            while pi < len(pending) and pending[pi].arrival_s <= now:
                if self._admit(pending[pi]) is None:
                    break
                pi += 1
            if not self.active32 and not self.active64:
                if pi < len(pending):
                    time.sleep(max(0.0, min(0.01, pending[pi].arrival_s - now)))
                continue
            # both ticks follow the admissions and promotions queued on the current stream
            ran32, ran64 = bool(self.active32), bool(self.active64)
            if ran32:
                self.s32.wait_stream(cur)
                L.sos_group_sync(self.g32, h32)
                L.sos_group_run(self.g32, self.K, h32)
            if ran64:
                self.s64.wait_stream(cur)
                L.sos_group_sync(self.g64, h64)
                L.sos_group_run(self.g64, self.K, h64)
            self.ticks += 1
            self.group_steps += self.K
            self.launches += 3 * self.K * (ran32 + ran64)      # forward, residual, adjoint per step
            if ran32:
                L.sos_group_losses(self.g32, self.losses32.ctypes.data, h32)    # waits for the FP32 tick only
            now = time.perf_counter() - t0
            for slot, a in list(self.active32.items()):
                a.steps32 += self.K
                loss, pp = self.losses32[2 * slot], self.losses32[2 * slot + 1]
                a.pp = pp
                if not np.isfinite(loss) or not np.isfinite(pp):
                    self._retire(a, L.SOS_VERDICT_ERROR, float("nan"), now, out)
                    continue
                rel = float(np.sqrt(2.0 * loss / pp)) if pp > 0 else float(np.sqrt(2.0 * loss))
                if rel < 0.99 * a.last_gain:
                    a.last_gain, a.stall = rel, 0
                else:
                    a.stall += 1
                a.best = min(a.best, rel)
                stalled = a.stall >= pol.stall_checks or a.steps32 >= pol.max_fp32_steps
                if rel <= pol.switch_rel or (stalled and rel <= pol.promote_rel):
                    self._promote(a)          # waits for a FP64 slot if none is free
                elif stalled and a.decays < pol.max_decays and a.steps32 < pol.max_fp32_steps:
                    a.decays += 1
                    a.lr *= pol.decay
                    a.stall, a.last_gain = 0, rel
                    L.sos_group_set_lr(self.g32, slot, a.lr)
                elif stalled:
                    self._retire(a, L.SOS_VERDICT_NOT_CONVERGED, rel, now, out)
            if ran64:
                L.sos_group_losses(self.g64, self.losses64.ctypes.data, h64)
                now = time.perf_counter() - t0
            for slot, a in list(self.active64.items()):
                if a.fresh:                   # promoted during this tick: no FP64 step yet
                    a.fresh = False
                    continue
                a.steps64 += self.K
                loss, pp = self.losses64[2 * slot], self.losses64[2 * slot + 1]
                if not np.isfinite(loss) or not np.isfinite(pp):
                    self._retire(a, L.SOS_VERDICT_ERROR, float("nan"), now, out)
                    continue
                rel = float(np.sqrt(2.0 * loss / pp)) if pp > 0 else float(np.sqrt(2.0 * loss))
                if rel < 0.99 * a.last_gain:
                    a.last_gain, a.stall = rel, 0
                else:
                    a.stall += 1
                a.best = min(a.best, rel)
                if rel <= pol.cert_tol:
                    # the iterate whose FP64 residual this is sits in the other buffer
                    self._retire(a, L.SOS_VERDICT_SOS, rel, now, out)
                elif (a.stall >= pol.stall_checks and a.decays < pol.max_decays
                      and a.steps64 < pol.max_fp64_steps):
                    a.decays += 1
                    a.lr *= pol.decay
                    a.stall, a.last_gain = 0, rel
                    L.sos_group_set_lr(self.g64, slot, a.lr)
                elif a.stall >= pol.stall_checks or a.steps64 >= pol.max_fp64_steps:
                    self._retire(a, L.SOS_VERDICT_NOT_CONVERGED, rel, now, out)
            # requests still open past their deadline end here, between ticks
            for act in (self.active32, self.active64):
                for slot, a in list(act.items()):
                    if now - a.job.arrival_s > pol.deadline_s:
                        self._retire(a, VERDICT_TIMEOUT, a.best, now, out)
        torch.cuda.synchronize()
        return out


# -- the baseline: one problem at a time through the single-problem path -------------

def run_plain(jobs: list, policy: Optional[Policy] = None, K: int = 32, plans: Optional[dict] = None) -> list:
    """Serves jobs one after another: FP32 sos_step launches (CUDA cores), then
    FP64 sos_step launches, the same checks every K steps and the same decision
    rule as Server."""
    pol = policy or Policy()
    plans = {} if plans is None else plans
    out = []
    t0 = time.perf_counter()
    for job in sorted(jobs, key=lambda j: j.arrival_s):
        key = (job.n, job.two_d)
        if key not in plans:
            plans[key] = Plan(job.n, job.two_d)
        plan = plans[key]
        st = _stream_handle()
        p64, A0 = job.make()
        N, M = plan.N, plan.M
        p32 = torch.empty(M, dtype=torch.float32, device="cuda")
        A32 = torch.empty(N, N, dtype=torch.float32, device="cuda")
        L.sos_convert(_ptr(p64), L.SOS_FP64, _ptr(p32), L.SOS_FP32, M, st)
        L.sos_convert(_ptr(A0), L.SOS_FP64, _ptr(A32), L.SOS_FP32, N * N, st)
        opt = Optimizer(plan, A32, prec="fp32", optimizer="adam", lr=pol.lr32)
        verdict, rel, s32, s64 = None, float("nan"), 0, 0
        last_gain, stall, decays = float("inf"), 0, 0
        promote = False
        while True:
            for _ in range(K):
                opt.step(p32)
            s32 += K
            loss, pp = (float(x) for x in opt.loss.cpu().numpy())
            if not np.isfinite(loss):
                verdict = L.SOS_VERDICT_ERROR
                break
            rel = float(np.sqrt(2 * loss / pp))
            if rel < 0.99 * last_gain:
                last_gain, stall = rel, 0
            else:
                stall += 1
            stalled = stall >= pol.stall_checks or s32 >= pol.max_fp32_steps
            if rel <= pol.switch_rel or (stalled and rel <= pol.promote_rel):
                promote = True
                break
            if stalled and decays < pol.max_decays and s32 < pol.max_fp32_steps:
                decays += 1
                opt.opts.lr *= pol.decay
                stall, last_gain = 0, rel
                continue
            if stalled:
                verdict = L.SOS_VERDICT_NOT_CONVERGED
                break
        if promote:
            A64 = torch.empty(N, N, dtype=torch.float64, device="cuda")
            L.sos_convert(_ptr(A32), L.SOS_FP32, _ptr(A64), L.SOS_FP64, N * N, st)
            opt64 = Optimizer(plan, A64, prec="fp64", optimizer="adam",
                              lr=pol.lr64 * opt.opts.lr / pol.lr32)
            L.sos_convert(_ptr(opt.m), L.SOS_FP32, _ptr(opt64.m), L.SOS_FP64, N * N, st)
            L.sos_convert(_ptr(opt.v), L.SOS_FP32, _ptr(opt64.v), L.SOS_FP64, N * N, st)
            opt64.state.t = opt.state.t
            last_gain, stall, decays64 = float("inf"), 0, 0
            while True:
                for _ in range(K):
                    opt64.step(p64)
                s64 += K
                loss, pp = (float(x) for x in opt64.loss.cpu().numpy())
                rel = float(np.sqrt(2 * loss / pp))
                if rel <= pol.cert_tol:
                    verdict = L.SOS_VERDICT_SOS
                    break
                if rel < 0.99 * last_gain:
                    last_gain, stall = rel, 0
                else:
                    stall += 1
                if stall >= pol.stall_checks and decays64 < pol.max_decays and s64 < pol.max_fp64_steps:
                    decays64 += 1
                    opt64.opts.lr *= pol.decay
                    stall, last_gain = 0, rel
                    continue
                if stall >= pol.stall_checks or s64 >= pol.max_fp64_steps:
                    verdict = L.SOS_VERDICT_NOT_CONVERGED
                    break
        out.append(Verdict(job.rid, verdict, rel, s32, s64, 0.0, time.perf_counter() - t0))
    torch.cuda.synchronize()
    return out


def latency_stats(verdicts: list) -> dict:
    lat = np.array([v.latency_s for v in verdicts])
    if len(lat) == 0:
        return {}
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}
