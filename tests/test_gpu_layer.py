"""GPU parity of the network with its first layer (Sec. 2, Eq. 4, Sec. 2.1),
called through the C ABI (sos_layer_*), against the oracle.

Tolerances (from the arithmetic):
  * FP64: 1e-12 relative for A_hat, 1e-11 for loss and gradients (the layer's
    GEMMs and the core pass differ from the oracle only in summation order);
  * FP32: A_hat within 1e-6 relative, loss and gradients within 1e-5
    (normwise), the core path's FP32 tolerance;
  * BF16: the core contractions see A_hat rounded to bf16 and the residual
    rounded to bf16 (2^-8 each), and with nf, m >= 64 the layer's GEMMs read
    bf16 B, A1 and S too, so loss and gradients are compared normwise at 2e-2
    -- the core BF16 path itself is checked elementwise elsewhere.
Shapes cover m < nf, m = nf, m = 2 nf, k not a multiple of 64, and a
(k nf)-deep reduction that is split over many blocks.
"""
import numpy as np
import pytest
import torch

import oracle
import sos_inputs
from paper_2410_19844_gb300 import _lib as L
from paper_2410_19844_gb300.engine import Layer, LayerOptimizer, Plan

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 10), (5, 3, 15), (6, 12, 21), (8, 8, 36), (11, 22, 200), (16, 16, 136)]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def case(nf, m, k, seed=0):
    o = oracle.Oracle(nf - 1, 4)
    B = sos_inputs.normal_matrix(k, nf * m, seed, sigma=0.3)
    A1 = sos_inputs.normal_matrix(m, nf, seed + 1, sigma=0.3)
    p = o.coeffs(sos_inputs.normal_matrix(o.N, 3, seed + 2))
    return o, B, A1, p


@pytest.mark.parametrize("nf,m,k", SHAPES)
def test_layer_expand(nf, m, k):
    o, B, A1, _ = case(nf, m, k)
    lay = Layer(Plan(nf - 1, 4, k), m)
    want = o.layer_expand(B, A1)
    got64 = lay.expand(torch.from_numpy(B).cuda(), torch.from_numpy(A1).cuda(), "fp64").cpu().numpy()
    assert rel(got64, want) < 1e-12
    got32 = lay.expand(torch.from_numpy(B).float().cuda(), torch.from_numpy(A1).float().cuda(), "fp32")
    assert rel(got32.cpu().numpy(), o.layer_expand(B.astype(np.float32), A1.astype(np.float32))) < 1e-6


@pytest.mark.parametrize("nf,m,k", SHAPES)
def test_layer_loss_grad_fp64(nf, m, k):
    o, B, A1, p = case(nf, m, k)
    lay = Layer(Plan(nf - 1, 4, k), m)
    loss, pp, gB, gA1 = lay.loss_grad(torch.from_numpy(B).cuda(), torch.from_numpy(A1).cuda(),
                                      torch.from_numpy(p).cuda(), "fp64")
    loss_ref, gB_ref, gA1_ref, _ = o.layer_loss_grad(B, A1, p)
    assert abs(loss.item() - loss_ref) <= 1e-11 * loss_ref
    assert abs(pp.item() - np.dot(p, p)) <= 1e-12 * np.dot(p, p)
    assert rel(gB.cpu().numpy(), gB_ref) < 1e-11
    assert rel(gA1.cpu().numpy(), gA1_ref) < 1e-11


@pytest.mark.parametrize("nf,m,k", SHAPES)
def test_layer_loss_grad_fp32(nf, m, k):
    o, B, A1, p = case(nf, m, k)
    B32, A132, p32 = B.astype(np.float32), A1.astype(np.float32), p.astype(np.float32)
    lay = Layer(Plan(nf - 1, 4, k), m)
    loss, _, gB, gA1 = lay.loss_grad(torch.from_numpy(B32).cuda(), torch.from_numpy(A132).cuda(),
                                     torch.from_numpy(p32).cuda(), "fp32")
    loss_ref, gB_ref, gA1_ref, _ = o.layer_loss_grad(B32.astype(np.float64), A132.astype(np.float64),
                                                     p32.astype(np.float64))
    assert abs(loss.item() - loss_ref) <= 1e-5 * loss_ref
    assert rel(gB.cpu().numpy(), gB_ref) < 1e-5
    assert rel(gA1.cpu().numpy(), gA1_ref) < 1e-5


@pytest.mark.parametrize("nf,m,k", [(6, 12, 21), (11, 22, 200),
                                    (64, 70, 20)])     # nf, m >= 64: P and dL/dB on the tensor cores
def test_layer_loss_grad_bf16(nf, m, k):
    o, B, A1, p = case(nf, m, k)
    B32, A132, p32 = B.astype(np.float32), A1.astype(np.float32), p.astype(np.float32)
    lay = Layer(Plan(nf - 1, 4, k), m)
    loss, _, gB, gA1 = lay.loss_grad(torch.from_numpy(B32).cuda(), torch.from_numpy(A132).cuda(),
                                     torch.from_numpy(p32).cuda(), "bf16")
    loss_ref, gB_ref, gA1_ref, _ = o.layer_loss_grad(B32.astype(np.float64), A132.astype(np.float64),
                                                     p32.astype(np.float64))
    assert abs(loss.item() - loss_ref) <= 2e-2 * loss_ref
    assert rel(gB.cpu().numpy(), gB_ref) < 2e-2
    assert rel(gA1.cpu().numpy(), gA1_ref) < 2e-2


@pytest.mark.parametrize("fixed", [False, True])
def test_layer_adam_steps_fp64(fixed):
    nf, m, k = 6, 12, 21
    o, B, A1, p = case(nf, m, k, seed=4)
    lay = Layer(Plan(nf - 1, 4, k), m)
    Bd, A1d = torch.from_numpy(B.copy()).cuda(), torch.from_numpy(A1.copy()).cuda()
    opt = LayerOptimizer(lay, Bd, A1d, prec="fp64", lr=1e-2, fixed_A1=fixed)
    pd = torch.from_numpy(p).cuda()
    Br, A1r = B.copy(), A1.copy()
    mB, vB, mA, vA = (np.zeros_like(B), np.zeros_like(B), np.zeros_like(A1), np.zeros_like(A1))
    for t in range(1, 6):
        loss = opt.step(pd)[0].item()
        loss_ref, gB, gA1, _ = o.layer_loss_grad(Br, A1r, p)
        assert abs(loss - loss_ref) <= 1e-11 * loss_ref
        o.adam_step(Br, mB, vB, gB, t, 1e-2)
        if not fixed:
            o.adam_step(A1r, mA, vA, gA1, t, 1e-2)
        assert rel(Bd.cpu().numpy(), Br) < 1e-10
        assert rel(A1d.cpu().numpy(), A1r) < 1e-10
    if fixed:
        assert np.array_equal(A1d.cpu().numpy(), A1)
    assert opt.t == 5


def test_layer_gd_step_fp32():
    nf, m, k = 8, 8, 36
    o, B, A1, p = case(nf, m, k, seed=6)
    B32, A132, p32 = B.astype(np.float32), A1.astype(np.float32), p.astype(np.float32)
    lay = Layer(Plan(nf - 1, 4, k), m)
    Bd, A1d = torch.from_numpy(B32.copy()).cuda(), torch.from_numpy(A132.copy()).cuda()
    lr = 1e-4
    opt = LayerOptimizer(lay, Bd, A1d, prec="fp32", optimizer="gd", lr=lr)
    opt.step(torch.from_numpy(p32).cuda())
    _, gB, gA1, _ = o.layer_loss_grad(B32.astype(np.float64), A132.astype(np.float64), p32.astype(np.float64))
    # the moves themselves, against -lr grad (rounding of B - lr g is 2^-24 |B|, far below the move)
    assert rel(Bd.cpu().numpy() - B32, -lr * gB) < 1e-3
    assert rel(A1d.cpu().numpy() - A132, -lr * gA1) < 1e-3


def test_layer_bf16_steps_reuse_the_updated_bf16_copy():
    # nf, m >= 64: the layer's GEMMs run on the tensor cores, and each BF16 step's
    # update writes the bf16 copy of the new B that the next step reads
    # (SOS_LAYER_BF16_CURRENT).  The loss a step reports is the loss at the B
    # it starts from: it must equal a fresh evaluation at that B, which casts B
    # itself (the core forward's float atomics allow 1e-5).
    nf, m, k = 64, 70, 20
    _, B, A1, p = case(nf, m, k, seed=8)
    lay = Layer(Plan(nf - 1, 4, k), m)
    Bd, A1d = torch.from_numpy(B).float().cuda(), torch.from_numpy(A1).float().cuda()
    pd = torch.from_numpy(p).float().cuda()
    opt = LayerOptimizer(lay, Bd, A1d, prec="bf16", optimizer="gd", lr=1e-9)   # about 0.5% less loss a step
    assert not opt.state.flags & L.SOS_LAYER_BF16_CURRENT
    first = opt.step(pd)[0].item()
    assert opt.state.flags & L.SOS_LAYER_BF16_CURRENT
    probe = Layer(Plan(nf - 1, 4, k), m)
    for _ in range(3):
        fresh = probe.loss_grad(Bd.clone(), A1d.clone(), pd, "bf16", want_grad=False)[0].item()
        assert abs(fresh - first) > 1e-3 * first          # the step moved B
        got = opt.step(pd)[0].item()
        assert abs(got - fresh) <= 1e-5 * fresh
        first = got
    # B changed outside the library: params_changed() makes the next step cast it again
    Bd.mul_(1.05)
    opt.params_changed()
    fresh = probe.loss_grad(Bd.clone(), A1d.clone(), pd, "bf16", want_grad=False)[0].item()
    got = opt.step(pd)[0].item()
    assert abs(got - fresh) <= 1e-5 * fresh
    # an FP32 step on the same state leaves no claim on the bf16 copy
    opt32 = LayerOptimizer(lay, Bd, A1d, prec="fp32", optimizer="gd", lr=1e-9)
    opt32.state.flags = opt.state.flags
    opt32.step(pd)
    assert not opt32.state.flags & L.SOS_LAYER_BF16_CURRENT


def test_layer_rejects_bad_arguments():
    with pytest.raises(ValueError):
        Layer(Plan(3, 6), 4)
    pl = Plan(3, 4, 5)
    with pytest.raises(L.SOSError):
        L.sos_layer_workspace_size(pl.handle, L.SOS_FP32, 0)
    lay = Layer(pl, 4)
    with pytest.raises(ValueError):
        lay.expand(torch.zeros(5, 15, device="cuda"), torch.zeros(4, 4, device="cuda"))
