"""GPU checks of failure detection and checkpoint / resume.

Failure detection: every wait in the tensor-core kernels is an mbarrier wait
bounded on the global timer; sos_diag_bounded_wait runs that wait on a barrier
nothing arrives at, and the test checks that the kernel returns with
SOS_E_TIMEOUT in its status word and that the context keeps working (no GPU
fault is involved).  Checkpoint / resume: an optimiser state saved after k
steps and loaded into fresh buffers continues bit for bit like the
uninterrupted run.
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
def test_checkpoint_resume_is_bitwise(prec, optimizer):
    n, two_d = 6, 8
    o = oracle.Oracle(n, two_d)
    dt = torch.float64 if prec == "fp64" else torch.float32
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
    ckpt = first.state_dict()
    del first
    A_b = torch.empty_like(A0)
    second = Optimizer(pl, A_b, prec=prec, optimizer=optimizer, lr=lr * 7)   # settings come from ckpt
    second.load_state_dict(ckpt)
    assert second.t == 5
    losses += [second.step(p)[0].item() for _ in range(7)]
    torch.cuda.synchronize()
    assert losses == losses_ref
    assert torch.equal(A_b, A_ref)
    if optimizer == "adam":
        assert torch.equal(second.m, ref.m) and torch.equal(second.v, ref.v)
