"""Python front end of the C ABI.  torch provides device memory and streams;
every computation is a call into ``libsos_gb300.so``.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L

_DTYPE = {L.SOS_BF16: torch.float32, L.SOS_FP32: torch.float32, L.SOS_FP64: torch.float64,
          L.SOS_FP64_TC: torch.float64}


def _prec(prec) -> int:
    return L.PREC[prec] if isinstance(prec, str) else int(prec)


def _stream_handle(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


class Plan:
    """Monomial tables and device state for degree <= two_d in n variables with
    r squares (default r = N, the paper's full-rank over-parameterisation)."""

    def __init__(self, n: int, two_d: int, r: int | None = None):
        from math import comb
        N = comb(n + two_d // 2, two_d // 2)
        self.n, self.two_d = n, two_d
        self.handle = L.sos_plan(n, two_d, int(r if r is not None else N))
        self.N, self.M, self.r = L.sos_plan_sizes(self.handle)
        self._ws = {}

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                L.sos_plan_destroy(h)
            except Exception:
                pass
            self.handle = None

    # -- host tables ----------------------------------------------------------
    def monomials(self, which: int = 0) -> np.ndarray:
        rows = self.N if which == 0 else self.M
        out = np.zeros((rows, self.n), dtype=np.uint8)
        L.sos_plan_monomials(self.handle, which, out.ctypes.data)
        return out

    def idx(self) -> np.ndarray:
        out = np.zeros((self.N, self.N), dtype=np.int32)
        L.sos_plan_idx(self.handle, out.ctypes.data)
        return out

    def device_idx(self, row0: int = 0, rows: int | None = None) -> np.ndarray:
        """Rows of the index table the kernels read, copied back from the device."""
        rows = self.N - row0 if rows is None else rows
        out = np.zeros((rows, self.N), dtype=np.int32)
        L.sos_plan_device_idx(self.handle, row0, rows, out.ctypes.data)
        return out

    # -- workspace ------------------------------------------------------------
    def workspace(self, prec, device=None) -> torch.Tensor:
        prec = _prec(prec)
        device = torch.device(device or "cuda")
        key = prec
        ws = self._ws.get(key)
        if ws is None:
            nbytes = L.sos_workspace_size(self.handle, prec)
            ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
            L.sos_workspace_init(self.handle, prec, _ptr(ws), _stream_handle())
            self._ws[key] = ws
        return ws

    def _check(self, A: torch.Tensor, prec: int):
        if not A.is_cuda or A.dtype != _DTYPE[prec] or not A.is_contiguous():
            raise ValueError(f"A must be a contiguous CUDA {_DTYPE[prec]} tensor")
        if tuple(A.shape[-2:]) != (self.N, self.r):
            raise ValueError(f"A must be {self.N} x {self.r}, got {tuple(A.shape)}")

    # -- one pass ---------------------------------------------------------------
    def coeffs(self, A: torch.Tensor, prec="fp32") -> torch.Tensor:
        prec = _prec(prec)
        self._check(A, prec)
        c = torch.empty(self.M, dtype=_DTYPE[prec] if prec != L.SOS_BF16 else torch.float32, device=A.device)
        L.sos_coeffs(self.handle, prec, _ptr(A), _ptr(c), _ptr(self.workspace(prec, A.device)),
                     _stream_handle())
        return c

    def loss_grad(self, A: torch.Tensor, p: torch.Tensor, prec="fp32", want_grad=True):
        """(loss, ||p||^2, grad) with loss = 1/2 ||c(A) - p||^2; device tensors."""
        prec = _prec(prec)
        self._check(A, prec)
        out = torch.empty(2, dtype=torch.float64, device=A.device)
        grad = torch.empty_like(A) if want_grad else None
        L.sos_loss_grad(self.handle, prec, _ptr(A), _ptr(p), _ptr(grad), _ptr(out),
                        _ptr(self.workspace(prec, A.device)), _stream_handle())
        return out[0], out[1], grad

    def loss_grad_batched(self, A: torch.Tensor, p: torch.Tensor, prec="fp32", want_grad=True):
        prec = _prec(prec)
        batch = A.shape[0]
        self._check(A, prec)
        nbytes = L.sos_workspace_size_batched(self.handle, prec, batch)
        ws = torch.empty(nbytes, dtype=torch.uint8, device=A.device)
        L.sos_workspace_init(self.handle, prec, _ptr(ws), _stream_handle())
        out = torch.empty(batch, 2, dtype=torch.float64, device=A.device)
        grad = torch.empty_like(A) if want_grad else None
        L.sos_loss_grad_batched(self.handle, prec, batch, _ptr(A), _ptr(p), _ptr(grad), _ptr(out),
                                _ptr(ws), _stream_handle())
        return out[:, 0], out[:, 1], grad

    def status(self, prec) -> int:
        prec = _prec(prec)
        ws = self._ws.get(prec)
        if ws is None:
            return L.SOS_OK
        return L.sos_read_status(self.handle, prec, _ptr(ws), _stream_handle())

    def certify(self, A: torch.Tensor, p64: torch.Tensor, tol: float = 1e-8):
        """(relative FP64 residual, verdict)."""
        if A.dtype not in (torch.float32, torch.float64):
            raise ValueError("A must be float32 or float64")
        return L.sos_certify(self.handle, _ptr(A), A.dtype == torch.float64, _ptr(p64), tol,
                             _stream_handle())


def solve(plan: Plan, p64: torch.Tensor, A: torch.Tensor, **opts) -> dict:
    """Runs sos_solve on A (float64, in place): BF16 steps, then SOS_FP64_TC
    steps (or, with tc_fp64=0, FP32 then FP64 CUDA-core steps), then the FP64
    certificate; keyword arguments override fields of the default options."""
    if A.dtype != torch.float64 or p64.dtype != torch.float64:
        raise ValueError("A and p must be float64 device tensors")
    o = L.sos_solve_opts_default()
    for k, v in opts.items():
        if k in ("optimizer",) and isinstance(v, str):
            v = L.SOS_ADAM if v == "adam" else L.SOS_GD
        if k == "start_prec" and isinstance(v, str):
            v = L.PREC[v]
        setattr(o, k, v)
    return L.sos_solve(plan.handle, _ptr(p64), _ptr(A), o, _stream_handle()).as_dict()


class Optimizer:
    """Adam (the paper's optimiser, Sec. 3) or GD state for one A, stepping
    through sos_step."""

    def __init__(self, plan: Plan, A: torch.Tensor, prec="bf16", optimizer="adam", lr=1e-2,
                 beta1=0.9, beta2=0.999, eps=1e-8, fp32_adjoint=False, slices=0):
        self.plan, self.prec = plan, _prec(prec)
        plan._check(A, self.prec)
        self.A = A
        self.opts = L.sos_step_opts(L.SOS_ADAM if optimizer == "adam" else L.SOS_GD, lr, beta1,
                                    beta2, eps, L.SOS_STEP_FP32_ADJOINT if fp32_adjoint else 0, slices)
        if optimizer == "adam":
            # SOS_FP64_TC keeps the moments in FP32 next to the FP64 iterate
            mdt = torch.float32 if self.prec == L.SOS_FP64_TC else A.dtype
            self.m = torch.zeros_like(A, dtype=mdt)
            self.v = torch.zeros_like(A, dtype=mdt)
        else:
            self.m = self.v = None
        self.state = L.sos_state(_ptr(A), _ptr(self.m), _ptr(self.v), 0)
        self.loss = torch.zeros(2, dtype=torch.float64, device=A.device)

    @property
    def t(self) -> int:
        return self.state.t

    def state_dict(self) -> dict:
        """Everything needed to continue the iteration: A, m, v, the step count and
        the optimiser settings (the bf16 copy of A is rebuilt on resume)."""
        d = {"A": self.A.detach().clone(), "t": int(self.state.t), "prec": self.prec,
             "opts": {f: getattr(self.opts, f) for f, _ in self.opts._fields_}}
        if self.m is not None:
            d["m"], d["v"] = self.m.detach().clone(), self.v.detach().clone()
        return d

    def load_state_dict(self, d: dict) -> None:
        self.A.copy_(d["A"])
        if self.m is not None:
            self.m.copy_(d["m"])
            self.v.copy_(d["v"])
        for f, v in d["opts"].items():
            setattr(self.opts, f, v)
        self.state.t = int(d["t"])
        self.state.flags = 0

    def step(self, p: torch.Tensor) -> torch.Tensor:
        """One iteration; returns the device tensor {loss before the step, ||p||^2}."""
        L.sos_step(self.plan.handle, self.prec, self.state, _ptr(p), self.opts, _ptr(self.loss),
                   _ptr(self.plan.workspace(self.prec, self.A.device)), _stream_handle())
        return self.loss


class Layer:
    """The network of Sec. 2 with its first layer: the quartic form
    ||B Z A1 x||^2 in n + 1 variables (A1: m x (n+1), B: k x (n+1) m), on a
    plan with two_d = 4 and r = k.  Every computation is a call into the
    library (sos_layer_*)."""

    def __init__(self, plan: Plan, m: int):
        if plan.two_d != 4:
            raise ValueError("the first layer produces quartics: the plan needs two_d = 4")
        self.plan, self.m, self.nf, self.k = plan, int(m), plan.n + 1, plan.r
        self._ws = {}

    def workspace(self, prec, device=None) -> torch.Tensor:
        prec = _prec(prec)
        ws = self._ws.get(prec)
        if ws is None:
            nbytes = L.sos_layer_workspace_size(self.plan.handle, prec, self.m)
            ws = torch.empty(nbytes, dtype=torch.uint8, device=torch.device(device or "cuda"))
            L.sos_workspace_init(self.plan.handle, prec, _ptr(ws), _stream_handle())
            self._ws[prec] = ws
        return ws

    def _check(self, B: torch.Tensor, A1: torch.Tensor, prec: int):
        dt = _DTYPE[prec]
        for name, t, shape in (("B", B, (self.k, self.nf * self.m)), ("A1", A1, (self.m, self.nf))):
            if not t.is_cuda or t.dtype != dt or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous CUDA {dt} tensor")
            if tuple(t.shape) != shape:
                raise ValueError(f"{name} must be {shape}, got {tuple(t.shape)}")

    def expand(self, B: torch.Tensor, A1: torch.Tensor, prec="fp32") -> torch.Tensor:
        """The plan's coefficient matrix A_hat (N x k) of the network."""
        prec = _prec(prec)
        self._check(B, A1, prec)
        A_hat = torch.empty(self.plan.N, self.k, dtype=_DTYPE[prec], device=B.device)
        L.sos_layer_expand(self.plan.handle, prec, self.m, _ptr(B), _ptr(A1), _ptr(A_hat),
                           _ptr(self.workspace(prec, B.device)), _stream_handle())
        return A_hat

    def loss_grad(self, B: torch.Tensor, A1: torch.Tensor, p: torch.Tensor, prec="fp32", want_grad=True):
        """(loss, ||p||^2, grad_B, grad_A1) with loss = 1/2 ||c - p||^2."""
        prec = _prec(prec)
        self._check(B, A1, prec)
        out = torch.empty(2, dtype=torch.float64, device=B.device)
        gB = torch.empty_like(B) if want_grad else None
        gA1 = torch.empty_like(A1) if want_grad else None
        L.sos_layer_loss_grad(self.plan.handle, prec, self.m, _ptr(B), _ptr(A1), _ptr(p), _ptr(gB), _ptr(gA1),
                              _ptr(out), _ptr(self.workspace(prec, B.device)), _stream_handle())
        return out[0], out[1], gB, gA1


class LayerOptimizer:
    """Adam (or GD) on the network's B and A1 through sos_layer_step; with
    fixed_A1 the first layer stays as it is (the paper's A = I comparison)."""

    def __init__(self, layer: Layer, B: torch.Tensor, A1: torch.Tensor, prec="fp32", optimizer="adam", lr=1e-2,
                 beta1=0.9, beta2=0.999, eps=1e-8, fixed_A1=False, fp32_adjoint=False):
        self.layer, self.prec = layer, _prec(prec)
        layer._check(B, A1, self.prec)
        self.B, self.A1 = B, A1
        self.opts = L.sos_step_opts(L.SOS_ADAM if optimizer == "adam" else L.SOS_GD, lr, beta1, beta2, eps,
                                    L.SOS_STEP_FP32_ADJOINT if fp32_adjoint else 0)
        adam = optimizer == "adam"
        self.mB = torch.zeros_like(B) if adam else None
        self.vB = torch.zeros_like(B) if adam else None
        self.mA1 = torch.zeros_like(A1) if adam and not fixed_A1 else None
        self.vA1 = torch.zeros_like(A1) if adam and not fixed_A1 else None
        self.state = L.sos_layer_state(_ptr(B), _ptr(self.mB), _ptr(self.vB), _ptr(A1), _ptr(self.mA1),
                                       _ptr(self.vA1), 0, L.SOS_LAYER_FIXED_A1 if fixed_A1 else 0, 0)
        self.loss = torch.zeros(2, dtype=torch.float64, device=B.device)

    @property
    def t(self) -> int:
        return self.state.t

    def params_changed(self) -> None:
        """Call after changing B in place outside step(): the next BF16 step then
        casts B again instead of reusing the bf16 copy its update left."""
        self.state.flags &= ~L.SOS_LAYER_BF16_CURRENT

    def step(self, p: torch.Tensor) -> torch.Tensor:
        """One iteration; returns the device tensor {loss before the step, ||p||^2}."""
        L.sos_layer_step(self.layer.plan.handle, self.prec, self.layer.m, self.state, _ptr(p), self.opts,
                         _ptr(self.loss), _ptr(self.layer.workspace(self.prec, self.B.device)), _stream_handle())
        return self.loss
