"""ctypes binding of ``libsos_gb300.so``: the C ABI of ``include/sos_gb300.h``
under the same names, argument marshalling only.  Every computation runs in
the library; a missing library raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

SOS_OK = 0
SOS_E_INVALID = -1
SOS_E_CUDA = -2
SOS_E_NOMEM = -3
SOS_E_TIMEOUT = -4
SOS_E_NONFINITE = -5
SOS_E_UNSUPPORTED = -6

SOS_BF16, SOS_FP32, SOS_FP64, SOS_FP64_TC = 0, 1, 2, 3
SOS_ADAM, SOS_GD = 0, 1
SOS_VERDICT_ERROR, SOS_VERDICT_NOT_CONVERGED, SOS_VERDICT_SOS = -1, 0, 1

PREC = {"bf16": SOS_BF16, "fp32": SOS_FP32, "fp64": SOS_FP64, "fp64_tc": SOS_FP64_TC}

EXPORTS = [
    "sos_plan", "sos_plan_create", "sos_plan_destroy", "sos_plan_sizes", "sos_plan_monomials", "sos_plan_idx",
    "sos_workspace_size", "sos_workspace_init", "sos_coeffs", "sos_loss_grad",
    "sos_workspace_size_batched", "sos_loss_grad_batched", "sos_step", "sos_read_status",
    "sos_certify", "sos_diag_gemm_bf16", "sos_launch_count", "sos_timing_enable",
    "sos_timing_reset", "sos_timing_report", "sos_loss_from_coeffs_static", "sos_solve_opts_default",
    "sos_solve", "sos_group_create", "sos_group_destroy", "sos_group_scratch_size", "sos_group_set",
    "sos_group_clear", "sos_group_sync", "sos_group_run", "sos_group_losses", "sos_group_state",
    "sos_convert", "sos_group_set_lr", "sos_diag_bounded_wait", "sos_layer_workspace_size",
    "sos_layer_expand", "sos_layer_loss_grad", "sos_layer_step", "sos_last_error", "sos_plan_device_idx",
]


class SOSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


SOS_STEP_FP32_ADJOINT = 1


class sos_step_opts(ctypes.Structure):
    _fields_ = [("optimizer", ctypes.c_int), ("lr", ctypes.c_double), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double), ("eps", ctypes.c_double), ("flags", ctypes.c_int),
                ("slices", ctypes.c_int)]


class sos_layer_state(ctypes.Structure):
    _fields_ = [("B", ctypes.c_void_p), ("mB", ctypes.c_void_p), ("vB", ctypes.c_void_p),
                ("A1", ctypes.c_void_p), ("mA1", ctypes.c_void_p), ("vA1", ctypes.c_void_p),
                ("t", ctypes.c_int64), ("flags", ctypes.c_int32), ("reserved", ctypes.c_int32)]


SOS_LAYER_FIXED_A1 = 1
SOS_LAYER_BF16_CURRENT = 2


class sos_state(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_void_p), ("v", ctypes.c_void_p),
                ("t", ctypes.c_int64), ("flags", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class sos_solve_opts(ctypes.Structure):
    _fields_ = [("optimizer", ctypes.c_int), ("lr_bf16", ctypes.c_double), ("lr_fp32", ctypes.c_double),
                ("lr_fp64", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("max_steps", ctypes.c_int64), ("check_every", ctypes.c_int64),
                ("switch_rel", ctypes.c_double), ("stall_checks", ctypes.c_int64),
                ("fp64_steps", ctypes.c_int64), ("fp64_fp32_adjoint", ctypes.c_int),
                ("cert_tol", ctypes.c_double), ("start_prec", ctypes.c_int), ("tc_fp64", ctypes.c_int)]


class sos_result(ctypes.Structure):
    _fields_ = [("verdict", ctypes.c_int), ("steps", ctypes.c_int64), ("steps_bf16", ctypes.c_int64),
                ("steps_fp32", ctypes.c_int64), ("steps_fp64", ctypes.c_int64),
                ("rel_start_fp64", ctypes.c_double), ("rel_at_switch", ctypes.c_double),
                ("min_rel", ctypes.c_double), ("min_rel_fp64", ctypes.c_double),
                ("rel_resid_fp64", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def library_path() -> str:
    """The in-tree build, or the file named by SOS_LIBRARY_PATH (another build
    of the same sources, e.g. with different tile constants)."""
    return os.environ.get("SOS_LIBRARY_PATH") or _build.LIB


def lib(auto_build: bool = True):
    """The loaded library; builds it in-tree first when missing or stale."""
    global _lib
    if _lib is not None:
        return _lib
    if os.environ.get("SOS_LIBRARY_PATH"):
        path = os.environ["SOS_LIBRARY_PATH"]
    else:
        path = _build.build() if auto_build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library missing at {path}; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "sos_plan": [i32, i32, i64, P(vp)],
        "sos_plan_create": [i32, i32, i64, P(vp)],
        "sos_plan_device_idx": [vp, i64, i64, vp],
        "sos_plan_destroy": [vp],
        "sos_plan_sizes": [vp, P(i64), P(i64), P(i64)],
        "sos_plan_monomials": [vp, i32, vp],
        "sos_plan_idx": [vp, vp],
        "sos_workspace_size": [vp, i32, P(ctypes.c_size_t)],
        "sos_workspace_init": [vp, i32, vp, vp],
        "sos_coeffs": [vp, i32, vp, vp, vp, vp],
        "sos_loss_grad": [vp, i32, vp, vp, vp, vp, vp, vp],
        "sos_workspace_size_batched": [vp, i32, i64, P(ctypes.c_size_t)],
        "sos_loss_grad_batched": [vp, i32, i64, vp, vp, vp, vp, vp, vp],
        "sos_step": [vp, i32, P(sos_state), vp, P(sos_step_opts), vp, vp, vp],
        "sos_read_status": [vp, i32, vp, vp],
        "sos_certify": [vp, vp, i32, vp, dbl, P(dbl), P(i32), vp, vp],
        "sos_diag_gemm_bf16": [i32, vp, vp, vp, i64, i64, i64, i64, i64, vp, vp],
        "sos_loss_from_coeffs_static": [i32, i64, i64, vp, vp, vp, vp, vp],
        "sos_solve_opts_default": [P(sos_solve_opts)],
        "sos_solve": [vp, vp, vp, P(sos_solve_opts), P(sos_result), vp],
        "sos_group_create": [i32, i32, i32, dbl, dbl, dbl, i32, P(vp)],
        "sos_group_destroy": [vp],
        "sos_group_scratch_size": [vp, i32, P(ctypes.c_size_t)],
        "sos_group_set": [vp, i32, vp, vp, vp, vp, vp, vp, dbl, i64],
        "sos_group_clear": [vp, i32],
        "sos_group_set_lr": [vp, i32, dbl],
        "sos_group_sync": [vp, vp],
        "sos_group_run": [vp, i32, vp],
        "sos_group_losses": [vp, vp, vp],
        "sos_group_state": [vp, i32, P(vp), P(vp), P(i64)],
        "sos_convert": [vp, i32, vp, i32, i64, vp],
        "sos_diag_bounded_wait": [ctypes.c_uint64, vp, vp],
        "sos_layer_workspace_size": [vp, i32, i32, P(ctypes.c_size_t)],
        "sos_layer_expand": [vp, i32, i32, vp, vp, vp, vp, vp],
        "sos_layer_loss_grad": [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp],
        "sos_layer_step": [vp, i32, i32, P(sos_layer_state), vp, P(sos_step_opts), vp, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = i32
    L.sos_launch_count.argtypes = []
    L.sos_launch_count.restype = i64
    L.sos_timing_enable.argtypes = [i32]
    L.sos_timing_enable.restype = i32
    L.sos_timing_reset.argtypes = []
    L.sos_timing_reset.restype = i32
    L.sos_timing_report.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    L.sos_timing_report.restype = i32
    L.sos_last_error.argtypes = []
    L.sos_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc: int) -> int:
    if rc != SOS_OK:
        raise SOSError(rc, lib().sos_last_error().decode(errors="replace"))
    return rc


# ---- same-named wrappers ---------------------------------------------------------

def sos_plan(n: int, two_d: int, r: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().sos_plan(n, two_d, r, ctypes.byref(h)))
    return h.value


def sos_plan_create(n: int, two_d: int, r: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().sos_plan_create(n, two_d, r, ctypes.byref(h)))
    return h.value


def sos_plan_destroy(plan: int) -> None:
    _check(lib().sos_plan_destroy(plan))


def sos_plan_sizes(plan: int):
    N, M, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().sos_plan_sizes(plan, ctypes.byref(N), ctypes.byref(M), ctypes.byref(r)))
    return N.value, M.value, r.value


def sos_plan_monomials(plan: int, which: int, out_ptr: int) -> None:
    _check(lib().sos_plan_monomials(plan, which, out_ptr))


def sos_plan_idx(plan: int, out_ptr: int) -> None:
    _check(lib().sos_plan_idx(plan, out_ptr))


def sos_plan_device_idx(plan: int, row0: int, rows: int, out_ptr: int) -> None:
    _check(lib().sos_plan_device_idx(plan, row0, rows, out_ptr))


def sos_workspace_size(plan: int, prec: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().sos_workspace_size(plan, prec, ctypes.byref(b)))
    return b.value


def sos_workspace_init(plan: int, prec: int, ws: int, stream: int) -> None:
    _check(lib().sos_workspace_init(plan, prec, ws, stream))


def sos_coeffs(plan, prec, A, c, ws, stream) -> None:
    _check(lib().sos_coeffs(plan, prec, A, c, ws, stream))


def sos_loss_grad(plan, prec, A, p, grad, loss, ws, stream) -> None:
    _check(lib().sos_loss_grad(plan, prec, A, p, grad, loss, ws, stream))


def sos_workspace_size_batched(plan: int, prec: int, batch: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().sos_workspace_size_batched(plan, prec, batch, ctypes.byref(b)))
    return b.value


def sos_loss_grad_batched(plan, prec, batch, A, p, grad, loss, ws, stream) -> None:
    _check(lib().sos_loss_grad_batched(plan, prec, batch, A, p, grad, loss, ws, stream))


def sos_step(plan, prec, state: sos_state, p, opts: sos_step_opts, loss, ws, stream) -> None:
    _check(lib().sos_step(plan, prec, ctypes.byref(state), p, ctypes.byref(opts), loss, ws, stream))


def sos_read_status(plan, prec, ws, stream) -> int:
    """Returns the status code (does not raise) and clears it."""
    return int(lib().sos_read_status(plan, prec, ws, stream))


def sos_certify(plan, A, a_is_double, p64, tol_rel, stream):
    rel, verdict = ctypes.c_double(), ctypes.c_int()
    _check(lib().sos_certify(plan, A, int(a_is_double), p64, tol_rel, ctypes.byref(rel),
                             ctypes.byref(verdict), None, stream))
    return rel.value, verdict.value


def sos_diag_gemm_bf16(b_mn_major, X, Y, D, m, n, k, ldx, ldy, status, stream) -> None:
    _check(lib().sos_diag_gemm_bf16(int(b_mn_major), X, Y, D, m, n, k, ldx, ldy, status, stream))


def sos_last_error() -> str:
    return lib().sos_last_error().decode(errors="replace")


def sos_launch_count() -> int:
    return int(lib().sos_launch_count())


def sos_timing_enable(on: bool) -> None:
    _check(lib().sos_timing_enable(1 if on else 0))


def sos_timing_reset() -> None:
    _check(lib().sos_timing_reset())


def sos_timing_report() -> dict:
    """{kernel name: (launches, total ms)} since the last reset."""
    buf = ctypes.create_string_buffer(1 << 16)
    _check(lib().sos_timing_report(buf, len(buf)))
    out = {}
    for line in buf.value.decode().splitlines():
        name, count, ms = line.split()
        out[name] = (int(count), float(ms))
    return out


def sos_loss_from_coeffs_static(prec, batch, M, c, p, resid, loss, stream) -> None:
    _check(lib().sos_loss_from_coeffs_static(prec, batch, M, c, p, resid, loss, stream))


def sos_solve_opts_default() -> sos_solve_opts:
    o = sos_solve_opts()
    _check(lib().sos_solve_opts_default(ctypes.byref(o)))
    return o


def sos_solve(plan, p64, A, opts: sos_solve_opts, stream) -> sos_result:
    r = sos_result()
    _check(lib().sos_solve(plan, p64, A, ctypes.byref(opts), ctypes.byref(r), stream))
    return r


SOS_GROUP_FP32_ADJOINT = 1
SOS_GROUP_FAST_FP64 = 2


def sos_group_create(prec, capacity, optimizer, beta1=0.9, beta2=0.999, eps=1e-8, flags=0) -> int:
    h = ctypes.c_void_p()
    _check(lib().sos_group_create(prec, capacity, optimizer, beta1, beta2, eps, flags, ctypes.byref(h)))
    return h.value


def sos_group_destroy(group) -> None:
    _check(lib().sos_group_destroy(group))


def sos_group_scratch_size(plan, prec) -> int:
    b = ctypes.c_size_t()
    _check(lib().sos_group_scratch_size(plan, prec, ctypes.byref(b)))
    return b.value


def sos_group_set(group, slot, plan, A, m, v, p, scratch, lr, t0=0) -> None:
    _check(lib().sos_group_set(group, slot, plan, A, m, v, p, scratch, lr, t0))


def sos_group_clear(group, slot) -> None:
    _check(lib().sos_group_clear(group, slot))


def sos_group_sync(group, stream) -> None:
    _check(lib().sos_group_sync(group, stream))


def sos_group_run(group, steps, stream) -> None:
    _check(lib().sos_group_run(group, steps, stream))


def sos_group_losses(group, out_ptr, stream) -> None:
    _check(lib().sos_group_losses(group, out_ptr, stream))


def sos_group_state(group, slot):
    """(pointer of the current A, pointer of the previous A, steps taken)."""
    a, b, t = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64()
    _check(lib().sos_group_state(group, slot, ctypes.byref(a), ctypes.byref(b), ctypes.byref(t)))
    return a.value, b.value, t.value


def sos_convert(x, x_prec, y, y_prec, count, stream) -> None:
    _check(lib().sos_convert(x, x_prec, y, y_prec, count, stream))


def sos_group_set_lr(group, slot, lr) -> None:
    _check(lib().sos_group_set_lr(group, slot, lr))


def sos_diag_bounded_wait(limit_ns, status, stream) -> None:
    _check(lib().sos_diag_bounded_wait(limit_ns, status, stream))


def sos_layer_workspace_size(plan, prec, m) -> int:
    n = ctypes.c_size_t()
    _check(lib().sos_layer_workspace_size(plan, prec, m, ctypes.byref(n)))
    return n.value


def sos_layer_expand(plan, prec, m, B, A1, A_hat, ws, stream) -> None:
    _check(lib().sos_layer_expand(plan, prec, m, B, A1, A_hat, ws, stream))


def sos_layer_loss_grad(plan, prec, m, B, A1, p, grad_B, grad_A1, loss, ws, stream) -> None:
    _check(lib().sos_layer_loss_grad(plan, prec, m, B, A1, p, grad_B, grad_A1, loss, ws, stream))


def sos_layer_step(plan, prec, m, state: sos_layer_state, p, opts: sos_step_opts, loss, ws, stream) -> None:
    _check(lib().sos_layer_step(plan, prec, m, ctypes.byref(state), p, ctypes.byref(opts), loss, ws, stream))
