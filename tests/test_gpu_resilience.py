"""GPU checks of failure detection and checkpoint / resume.

Failure detection: every wait in the tensor-core kernels is an mbarrier wait
bounded on the global timer; sos_diag_bounded_wait runs that wait on a barrier
nothing arrives at, and the test checks that the kernel returns with
SOS_E_TIMEOUT in its status word and that the context keeps working (no GPU
fault is involved).  Checkpoint / resume: an optimiser state saved after k
steps and loaded into fresh buffers continues like the uninterrupted run --
bit for bit on the grouped path, which has no atomics, and up to the
run-to-run spread of the forward's atomics on the single-problem path.
"""
import time

import numpy as np
import pytest
import torch

import oracle
import sos_inputs
from paper_2410_19844_gb300 import _lib as L
from paper_2410_19844_gb300.engine import Optimizer, Plan, _ptr, _stream_handle

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_the_context_survives():
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L.sos_diag_bounded_wait(50_000_000, _ptr(status), _stream_handle())
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert status.item() == L.SOS_E_TIMEOUT
    assert 0.05 <= waited < 5.0
    # the context still computes
    o = oracle.Oracle(4, 6)
    A = sos_inputs.normal_matrix(o.N, o.N, 3, sigma=0.3)
    pl = Plan(4, 6)
    c = pl.coeffs(torch.from_numpy(A).cuda(), "fp64").cpu().numpy()
    np.testing.assert_allclose(c, o.coeffs(A), rtol=1e-12, atol=1e-12)


def test_bounded_wait_rejects_bad_arguments():
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(L.SOSError):
        L.sos_diag_bounded_wait(10 ** 10, _ptr(status), _stream_handle())
    with pytest.raises(L.SOSError):
        L.sos_diag_bounded_wait(1000, 0, _stream_handle())


@pytest.mark.parametrize("prec", ["bf16", "fp32", "fp64"])
@pytest.mark.parametrize("optimizer", ["adam", "gd"])
def test_checkpoint_resume_continues_the_run(prec, optimizer, tmp_path):
    """The restored state equals the saved one exactly; the continued run then
    follows the uninterrupted one up to the run-to-run spread of the forward's
    floating-point atomics (relative 1e-12 in FP64, 1e-6 in FP32, 1e-4 in BF16)."""
    n, two_d = 6, 8
    o = oracle.Oracle(n, two_d)
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = {"fp64": 1e-12, "fp32": 1e-6, "bf16": 1e-4}[prec]
    A0 = torch.from_numpy(sos_inputs.normal_matrix(o.N, o.N, 5, sigma=0.1)).to(dt).cuda()
    p = torch.from_numpy(o.coeffs(sos_inputs.normal_matrix(o.N, 20, 6))).to(dt).cuda()
    lr = 1e-3 if optimizer == "adam" else 1e-5
    pl = Plan(n, two_d)

    A_ref = A0.clone()
    ref = Optimizer(pl, A_ref, prec=prec, optimizer=optimizer, lr=lr)
    losses_ref = [ref.step(p)[0].item() for _ in range(12)]

    A_a = A0.clone()
    first = Optimizer(pl, A_a, prec=prec, optimizer=optimizer, lr=lr)
    losses = [first.step(p)[0].item() for _ in range(5)]
    torch.save(first.state_dict(), tmp_path / "state.pt")
    del first
    ckpt = torch.load(tmp_path / "state.pt")
    A_b = torch.empty_like(A0)
    second = Optimizer(pl, A_b, prec=prec, optimizer=optimizer, lr=lr * 7)   # settings come from ckpt
    second.load_state_dict(ckpt)
    assert second.t == 5 and second.opts.lr == lr
    assert torch.equal(A_b, ckpt["A"])
    if optimizer == "adam":
        assert torch.equal(second.m, ckpt["m"]) and torch.equal(second.v, ckpt["v"])
    losses += [second.step(p)[0].item() for _ in range(7)]
    torch.cuda.synchronize()
    np.testing.assert_allclose(losses, losses_ref, rtol=tol)
    assert (A_b - A_ref).abs().max().item() <= tol * A_ref.abs().max().item()


@pytest.mark.parametrize("prec", [L.SOS_FP32, L.SOS_FP64])
def test_group_checkpoint_resume_is_bitwise(prec):
    """The grouped path has no atomics: a problem stopped after 5 steps and put
    back into a new group with its (A, m, v, t) continues bit for bit."""
    n, two_d = 5, 6
    o = oracle.Oracle(n, two_d)
    dt = torch.float64 if prec == L.SOS_FP64 else torch.float32
    pl = Plan(n, two_d)
    st = _stream_handle()
    A0 = torch.from_numpy(sos_inputs.normal_matrix(o.N, o.N, 8, sigma=0.1)).to(dt).cuda()
    p = torch.from_numpy(o.coeffs(sos_inputs.normal_matrix(o.N, 10, 9))).to(dt).cuda()
    nbytes = L.sos_group_scratch_size(pl.handle, prec)

    def run(A, m, v, t0, steps):
        g = L.sos_group_create(prec, 1, L.SOS_ADAM)
        scratch = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        L.sos_group_set(g, 0, pl.handle, _ptr(A), _ptr(m), _ptr(v), _ptr(p), _ptr(scratch), 1e-2, t0)
        L.sos_group_sync(g, st)
        L.sos_group_run(g, steps, st)
        cur, _, taken = L.sos_group_state(g, 0)
        assert taken == steps                  # steps in this group, t0 not included
        out = torch.empty_like(A)
        L.sos_convert(cur, prec, _ptr(out), prec, A.numel(), st)
        torch.cuda.synchronize()
        L.sos_group_destroy(g)
        return out

    m, v = torch.zeros_like(A0), torch.zeros_like(A0)
    whole = run(A0.clone(), m, v, 0, 10)
    m1, v1 = torch.zeros_like(A0), torch.zeros_like(A0)
    half = run(A0.clone(), m1, v1, 0, 5)
    rest = run(half.clone(), m1, v1, 5, 5)
    assert torch.equal(rest, whole)
    assert torch.equal(m1, m) and torch.equal(v1, v)
