"""GPU checks of whole workloads: the tiny FP64 problem stepped 2000 times
against the oracle one step at a time, and the autograd Function."""
import numpy as np
import pytest
import torch

import oracle
import sos_inputs
from paper_2410_19844_gb300.autograd import SOSLossGrad, sos_loss
from paper_2410_19844_gb300.engine import Optimizer, Plan

pytestmark = pytest.mark.gpu


def test_tiny_fp64_2000_adam_steps_track_the_oracle():
    """n=3, 2d=4, N=r=10, p = sum of 5 random squares, A0 ~ N(0, 0.1^2):
    every GPU step equals the oracle's step from the same A (1e-10), and the
    two independent trajectories stay together (drift reported)."""
    w = sos_inputs.TINY
    o = oracle.Oracle(w.n, w.two_d)
    p = o.coeffs(sos_inputs.generator(w, 0))
    A0 = sos_inputs.init_A(w, 0)
    pl = Plan(w.n, w.two_d)
    A = torch.from_numpy(A0.copy()).cuda()
    opt = Optimizer(pl, A, prec="fp64", optimizer="adam", lr=1e-2)
    p_dev = torch.from_numpy(p).cuda()
    A_ind, m_ind, v_ind = A0.copy(), np.zeros_like(A0), np.zeros_like(A0)   # oracle trajectory
    prev = A0.copy()
    m_prev, v_prev = np.zeros_like(A0), np.zeros_like(A0)
    worst_step, losses = 0.0, []
    for t in range(1, 2001):
        losses.append(opt.step(p_dev)[0].item())
        got = A.cpu().numpy()
        # one oracle step from the GPU's previous state
        Aref, m, v = prev.copy(), m_prev.copy(), v_prev.copy()
        _, g, _ = o.loss_grad(Aref, p)
        o.adam_step(Aref, m, v, g, t, lr=1e-2)
        worst_step = max(worst_step, np.linalg.norm(got - Aref) / np.linalg.norm(Aref))
        prev, m_prev, v_prev = got, opt.m.cpu().numpy(), opt.v.cpu().numpy()
        _, g2, _ = o.loss_grad(A_ind, p)
        o.adam_step(A_ind, m_ind, v_ind, g2, t, lr=1e-2)
    drift = np.linalg.norm(prev - A_ind) / np.linalg.norm(A_ind)
    print(f"tiny FP64: worst one-step deviation {worst_step:.2e}, trajectory drift after 2000 steps "
          f"{drift:.2e}, loss {losses[0]:.3e} -> {min(losses):.3e}")
    assert worst_step <= 1e-10
    assert min(losses) < 1e-3 * losses[0]


def test_autograd_gradcheck_fp64():
    pl = Plan(3, 4, r=4)
    o = oracle.Oracle(3, 4)
    p = torch.from_numpy(o.coeffs(sos_inputs.normal_matrix(o.N, 3, seed=1))).cuda()
    A = torch.from_numpy(sos_inputs.normal_matrix(o.N, 4, seed=2, sigma=0.5)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda X: SOSLossGrad.apply(X, p, pl, "fp64"), (A,), eps=1e-6,
                                    atol=1e-6, rtol=1e-6)


def test_autograd_matches_oracle_fp32():
    o = oracle.Oracle(5, 6)
    pl = Plan(5, 6)
    A_np = sos_inputs.normal_matrix(o.N, o.N, seed=4, sigma=0.3).astype(np.float32)
    p_np = o.coeffs(sos_inputs.normal_matrix(o.N, 4, seed=5)).astype(np.float32)
    A = torch.from_numpy(A_np).cuda().requires_grad_(True)
    loss = sos_loss(A, torch.from_numpy(p_np).cuda(), pl, "fp32")
    (3.0 * loss).backward()
    loss_ref, g_ref, _ = o.loss_grad(A_np.astype(np.float64), p_np.astype(np.float64))
    assert abs(loss.item() - loss_ref) <= 1e-5 * loss_ref
    g = A.grad.double().cpu().numpy()
    assert np.linalg.norm(g - 3.0 * g_ref) <= 1e-5 * np.linalg.norm(3.0 * g_ref)
