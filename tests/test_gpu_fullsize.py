"""GPU parity at the full benchmark size, in the launch configuration the
benchmark times: n = 20 variables, degree 2d = 8, N = r = 10,626, M = 3,108,105.

The oracle cannot form c(A) over all M coefficients and the whole N x r
gradient in a test's time, so it computes samples one at a time:
  * coefficients c_g (oracle.coeff_at) at 64 positions: both ends and random;
  * gradient rows a (oracle.resid_row: h_b = (c - p)_{a+b} for every b, then
    grad_a = 2 h A) at both ends, both sides of the 256-row tile seam and one
    random row;
  * one BF16 gradient-descent step (the fused adjoint + update kernel the
    benchmark times) checked on the same rows.

Bounds (elementwise, from the arithmetic; u = 2^-23 allows the tensor core's
FP32 accumulation to truncate, 2^-24 on the CUDA cores):
  c:    |dc_g| <= (r + N) u |c|_g,   |c|_g = the coefficient at |A|
  h:    |dh_b| <= |dc| + u_r (|h_b| + |dc|),  u_r = 2^-8 for the BF16 residual
        the adjoint reads, 2^-24 in FP32
  grad: |dg_k| <= 2 sum_b |dh_b| |A_bk| + 2 N u sum_b (|h_b| + |dh_b|) |A_bk|
and, normwise over the coefficient samples, 1e-5 for FP32 (round to nearest:
the errors of the r additions largely cancel) and (r/16 + 64) 2^-23 |c| for
BF16: the tensor core may truncate its FP32 accumulator once per 16-deep MMA
step, so a sum of positive products drifts down by up to 2^-23 of itself per
step (measured at this size: 4e-5 relative on the coefficients that are sums
of squares, below the exact value, as truncation predicts).
"""
import numpy as np
import pytest
import torch

import bounds
import oracle
import sos_inputs
from paper_2410_19844_gb300.engine import Optimizer, Plan

pytestmark = pytest.mark.gpu

W = sos_inputs.LARGE


@pytest.fixture(scope="module")
def full():
    o = oracle.Oracle(W.n, W.two_d)
    pl = Plan(W.n, W.two_d)
    assert (pl.N, pl.M, pl.r) == (10626, 3108105, 10626)
    A32 = sos_inputs.init_A(W, 0).astype(np.float32)
    p32 = (sos_inputs.normal_matrix(pl.M, 1, 7)[:, 0] * 0.05).astype(np.float32)
    g = np.random.default_rng(11)
    coeffs = np.unique(np.concatenate([[0, 1, pl.M - 2, pl.M - 1], g.integers(0, pl.M, 60)]))
    rows = [0, 255, 256, int(g.integers(257, pl.N - 1)), pl.N - 1]
    return o, pl, A32, p32, coeffs, rows


_rows_ref = bounds.rows_ref
_coeffs_ref = bounds.coeffs_ref


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_full_size_coefficients_and_gradient_rows(full, prec):
    o, pl, A32, p32, cidx, rows = full
    A_eff = (torch.from_numpy(A32).bfloat16().double().numpy() if prec == "bf16"
             else A32.astype(np.float64))
    u = 2.0 ** -23 if prec == "bf16" else 2.0 ** -24
    u_r = 2.0 ** -8 if prec == "bf16" else 2.0 ** -24
    gamma_c = (pl.r + pl.N) * u
    A_dev = torch.from_numpy(A32).cuda()
    p_dev = torch.from_numpy(p32).cuda()

    c = pl.coeffs(A_dev, prec)[torch.from_numpy(cidx).cuda()].double().cpu().numpy()
    c_ref, c_abs = _coeffs_ref(o, A_eff, cidx)
    assert np.all(np.abs(c - c_ref) <= gamma_c * c_abs + 1e-30)
    if prec == "bf16":
        assert np.linalg.norm(c - c_ref) <= (pl.r / 16 + 64) * 2.0 ** -23 * np.linalg.norm(c_abs)
    else:
        assert np.linalg.norm(c - c_ref) <= 1e-5 * np.linalg.norm(c_ref)

    _, _, g = pl.loss_grad(A_dev, p_dev, prec)
    g_rows = g[rows].double().cpu().numpy()
    ref = _rows_ref(o, A_eff, p32.astype(np.float64), rows, u, u_r, gamma_c)
    for i, a in enumerate(rows):
        want, bound = ref[a]
        assert np.all(np.abs(g_rows[i] - want) <= bound), f"row {a}"


def test_full_size_bf16_gd_step(full):
    """One sos_step (BF16, plain GD, the fused adjoint + update kernel) at the
    benchmark's size: sampled rows of the new A against A - lr grad."""
    o, pl, A32, p32, _, rows = full
    lr = 1e-4
    A_dev = torch.from_numpy(A32).cuda()
    opt = Optimizer(pl, A_dev, prec="bf16", optimizer="gd", lr=lr)
    opt.step(torch.from_numpy(p32).cuda())
    new_rows = A_dev[rows].double().cpu().numpy()
    A16 = torch.from_numpy(A32).bfloat16().double().numpy()
    u = 2.0 ** -23
    ref = _rows_ref(o, A16, p32.astype(np.float64), rows, u, 2.0 ** -8, (pl.r + pl.N) * u)
    for i, a in enumerate(rows):
        g, bound = ref[a]
        want = A32[a].astype(np.float64) - lr * g
        tol = lr * bound + 2.0 ** -24 * (np.abs(want) + lr * np.abs(g)) + 1e-30
        assert np.all(np.abs(new_rows[i] - want) <= tol), f"row {a}"


def test_full_size_fp64_tc_coefficients(full):
    """SOS_FP64_TC at the benchmark's size (r = 10,626 <= 17,458, so every slice
    product is exact): sampled coefficients within 10 2^-40 of the same sums
    over the rows' power-of-two scales (8 slices; see test_gpu_fp64_tc.py)."""
    o, pl, A32, _, cidx, _ = full
    A64 = A32.astype(np.float64)
    c = pl.coeffs(torch.from_numpy(A64).cuda(), "fp64_tc")[torch.from_numpy(cidx).cuda()].cpu().numpy()
    c_ref, c_abs = _coeffs_ref(o, A64, cidx)
    e = np.frexp(np.abs(A64).max(axis=1))[1].astype(np.float64)
    E = np.repeat(np.exp2(e)[:, None], A64.shape[1], axis=1)
    scale = np.array([o.coeff_at(E, int(g)) for g in cidx])
    assert np.all(np.abs(c - c_ref) <= 10 * 2.0 ** -40 * scale + 1e-15 * c_abs)
