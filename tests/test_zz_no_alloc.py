"""The loss entry point that allocates nothing (sos_loss_from_coeffs_static).

Some callers cannot allocate device memory when they call into a library: a
host framework that only hands it buffers it allocated itself, or a loop held
to a fixed memory budget.  For them this entry point keeps its scratch in a
fixed array inside the library.  Here it must give the same residual and
losses as the oracle's residual on the same c and p (FP64 within 1e-12, FP32
within 1e-5 relative) and as the allocating path (sos_coeffs, then
sos_loss_grad_batched without a gradient), on two calls in a row, since the
fixed array keeps the previous call's contents.  It must report a non-finite
input as a non-finite loss and refuse a call that would not fit.

This file is collected last, so that a run stopping at the first failure has
run every other test before it; it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

import oracle
import sos_inputs
from paper_2410_19844_gb300 import _lib as L
from paper_2410_19844_gb300.engine import Plan

pytestmark = pytest.mark.gpu


def _stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("prec,dtype,tol", [(L.SOS_FP32, torch.float32, 1e-5),
                                            (L.SOS_FP64, torch.float64, 1e-12)])
def test_matches_oracle_and_allocating_path_on_two_calls(prec, dtype, tol):
    pl = Plan(6, 8)                      # N = 210, M = 3003
    o = oracle.Oracle(6, 8)
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
        got = loss.cpu().numpy()
        c_h, p_h = c.double().cpu().numpy(), p.double().cpu().numpy()
        for s in range(batch):
            # the oracle's residual and loss on the very same c and p
            loss_ref, resid_ref = o.residual(c_h[s], p_h[s])
            np.testing.assert_allclose(resid[s].double().cpu().numpy(), resid_ref, rtol=tol,
                                       atol=tol * np.abs(resid_ref).max())
            assert abs(got[s, 0] - loss_ref) <= tol * loss_ref
            assert abs(got[s, 1] - np.dot(p_h[s], p_h[s])) <= tol * np.dot(p_h[s], p_h[s])
        np.testing.assert_allclose(got[:, 0], want_loss.cpu().numpy(), rtol=tol)
        np.testing.assert_allclose(got[:, 1], want_pp.cpu().numpy(), rtol=tol)


def test_multiblock_problem_matches():
    """M large enough that each problem is reduced by several blocks, whose
    ticket counters must start from zero on every call."""
    pl = Plan(10, 10, r=64)             # M = 184,756: 181 blocks per problem
    o = oracle.Oracle(10, 10)
    A = torch.from_numpy(sos_inputs.normal_matrix(pl.N, pl.r, seed=3, sigma=0.2)).float().cuda()
    p = torch.from_numpy(sos_inputs.normal_matrix(pl.M, 1, seed=4)[:, 0]).float().cuda()
    want_loss, _, _ = pl.loss_grad(A, p, "fp32", want_grad=False)
    c = pl.coeffs(A, "fp32")
    loss_ref, _ = o.residual(c.double().cpu().numpy(), p.double().cpu().numpy())
    for _ in range(2):
        loss = torch.zeros(2, dtype=torch.float64, device="cuda")
        L.sos_loss_from_coeffs_static(L.SOS_FP32, 1, pl.M, c.data_ptr(), p.data_ptr(), 0, loss.data_ptr(),
                                      _stream())
        torch.cuda.synchronize()
        assert abs(loss[0].item() - loss_ref) <= 1e-5 * loss_ref
        assert abs(loss[0].item() - want_loss.item()) <= 1e-5 * want_loss.item()


def test_non_finite_input_gives_a_non_finite_loss():
    """An Inf in c (p finite) gives an infinite loss for that problem only; the
    next call, on finite data, is finite again."""
    M = 3003
    c = torch.from_numpy(np.stack([sos_inputs.normal_matrix(M, 1, seed=s)[:, 0] for s in (1, 2)])).float().cuda()
    p = torch.from_numpy(np.stack([sos_inputs.normal_matrix(M, 1, seed=s)[:, 0] for s in (3, 4)])).float().cuda()
    c_bad = c.clone()
    c_bad[1, 17] = float("inf")
    loss = torch.zeros(2, 2, dtype=torch.float64, device="cuda")
    L.sos_loss_from_coeffs_static(L.SOS_FP32, 2, M, c_bad.data_ptr(), p.data_ptr(), 0, loss.data_ptr(), _stream())
    torch.cuda.synchronize()
    got = loss.cpu().numpy()
    assert np.isfinite(got[0, 0]) and not np.isfinite(got[1, 0])
    L.sos_loss_from_coeffs_static(L.SOS_FP32, 2, M, c.data_ptr(), p.data_ptr(), 0, loss.data_ptr(), _stream())
    torch.cuda.synchronize()
    assert np.all(np.isfinite(loss.cpu().numpy()))


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
