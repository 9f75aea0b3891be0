"""The loss entry point that allocates nothing (sos_loss_from_coeffs_static).

It serves callers that cannot allocate device memory at call time: its
scratch lives in a fixed array inside the library.  Here it must give the
same losses as the allocating path (sos_coeffs, then sos_loss_grad_batched
without a gradient) on two calls in a row, since the fixed array keeps the
previous call's contents, and it must refuse a call that would not fit.
"""
import numpy as np
import pytest
import torch

import sos_inputs
from paper_2410_19844_gb300 import _lib as L
from paper_2410_19844_gb300.engine import Plan

pytestmark = pytest.mark.gpu


def _stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("prec,dtype,tol", [(L.SOS_FP32, torch.float32, 1e-5),
                                            (L.SOS_FP64, torch.float64, 1e-12)])
def test_matches_allocating_path_on_two_calls(prec, dtype, tol):
    pl = Plan(6, 8)                      # N = 210, M = 3003
    batch = 5
    for call in range(2):                # the second call sees the first call's leftovers
        A = torch.from_numpy(np.stack([sos_inputs.normal_matrix(pl.N, pl.r, seed=10 * call + s, sigma=0.3)
                                       for s in range(batch)])).to("cuda", dtype)
        p = torch.from_numpy(np.stack([sos_inputs.normal_matrix(pl.M, 1, seed=100 + 10 * call + s)[:, 0]
                                       for s in range(batch)])).to("cuda", dtype)
        prec_name = "fp64" if prec == L.SOS_FP64 else "fp32"
        want_loss, want_pp, _ = pl.loss_grad_batched(A.contiguous(), p.contiguous(), prec_name,
                                                     want_grad=False)
        c = torch.stack([pl.coeffs(A[s].contiguous(), prec_name) for s in range(batch)]).contiguous()
        resid = torch.full_like(c, float("nan"))
        loss = torch.full((batch, 2), float("nan"), dtype=torch.float64, device="cuda")
        L.sos_loss_from_coeffs_static(prec, batch, pl.M, c.data_ptr(), p.data_ptr(), resid.data_ptr(),
                                      loss.data_ptr(), _stream())
        torch.cuda.synchronize()
        assert torch.equal(resid, c - p)
        np.testing.assert_allclose(loss[:, 0].cpu().numpy(), want_loss.cpu().numpy(), rtol=tol)
        np.testing.assert_allclose(loss[:, 1].cpu().numpy(), want_pp.cpu().numpy(), rtol=tol)


def test_multiblock_problem_matches():
    """M large enough that each problem is reduced by several blocks, whose
    ticket counters must start from zero on every call."""
    pl = Plan(10, 10, r=64)             # M = 184,756: 181 blocks per problem
    A = torch.from_numpy(sos_inputs.normal_matrix(pl.N, pl.r, seed=3, sigma=0.2)).float().cuda()
    p = torch.from_numpy(sos_inputs.normal_matrix(pl.M, 1, seed=4)[:, 0]).float().cuda()
    want_loss, _, _ = pl.loss_grad(A, p, "fp32", want_grad=False)
    c = pl.coeffs(A, "fp32")
    for _ in range(2):
        loss = torch.zeros(2, dtype=torch.float64, device="cuda")
        L.sos_loss_from_coeffs_static(L.SOS_FP32, 1, pl.M, c.data_ptr(), p.data_ptr(), 0, loss.data_ptr(),
                                      _stream())
        torch.cuda.synchronize()
        assert abs(loss[0].item() - want_loss.item()) <= 1e-5 * want_loss.item()


def test_rejects_calls_beyond_the_fixed_scratch():
    c = torch.zeros(4, device="cuda")
    loss = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(L.SOSError) as e:
        L.sos_loss_from_coeffs_static(L.SOS_FP32, 2000, 1, c.data_ptr(), c.data_ptr(), 0, loss.data_ptr(),
                                      _stream())
    assert e.value.code == L.SOS_E_INVALID
    with pytest.raises(L.SOSError):
        # 200 problems of 512 blocks each: 102,400 partial sums > 65,280
        L.sos_loss_from_coeffs_static(L.SOS_FP32, 200, 600_000, c.data_ptr(), c.data_ptr(), 0,
                                      loss.data_ptr(), _stream())
