"""GPU parity over a seeded sweep of shapes: n in 1..12, 2d in 2..10, r from 1
to 2N, in every precision, through the C ABI, against the oracle.

Each shape is drawn from a fixed seed, so the sweep is the same on every run.
Tolerances are those of the focused tests: FP64 1e-12, FP32 1e-5 (normwise),
BF16 the elementwise bound (2^-8 + 4 N 2^-24) 2|H(r)||A| on the gradient and
1e-5 on the forward at the bf16-rounded A, SOS_FP64_TC the slicing bound
(s + 2) 2^(-5 s) on the sums over the rows' power-of-two scales.
"""
from math import comb

import numpy as np
import pytest
import torch

import oracle
import sos_inputs
from paper_2410_19844_gb300.engine import Plan

pytestmark = pytest.mark.gpu

DEV = "cuda"


def shapes(count=24, seed=2024):
    g = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        n = int(g.integers(1, 13))
        two_d = int(2 * g.integers(1, 6))
        N, M = comb(n + two_d // 2, two_d // 2), comb(n + two_d, two_d)
        if N > 500 or M > 60000:
            continue
        r = int(g.integers(1, 2 * N + 1))
        out.append((n, two_d, r))
    return out


SHAPES = shapes()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def case(n, two_d, r):
    o = oracle.Oracle(n, two_d)
    seed = 1000 * n + 10 * two_d + r
    A = sos_inputs.normal_matrix(o.N, r, seed, sigma=0.3)
    p = o.coeffs(sos_inputs.normal_matrix(o.N, 3, seed + 1))
    return o, A, p


@pytest.mark.parametrize("n,two_d,r", SHAPES)
def test_sweep_fp64_and_fp32(n, two_d, r):
    o, A, p = case(n, two_d, r)
    pl = Plan(n, two_d, r)
    loss, _, g = pl.loss_grad(torch.from_numpy(A).to(DEV), torch.from_numpy(p).to(DEV), "fp64")
    loss_ref, g_ref, _ = o.loss_grad(A, p)
    assert abs(loss.item() - loss_ref) <= 1e-12 * loss_ref
    assert rel(g.cpu().numpy(), g_ref) < 1e-12
    A32, p32 = A.astype(np.float32), p.astype(np.float32)
    loss, _, g = pl.loss_grad(torch.from_numpy(A32).to(DEV), torch.from_numpy(p32).to(DEV), "fp32")
    loss_ref, g_ref, _ = o.loss_grad(A32.astype(np.float64), p32.astype(np.float64))
    assert abs(loss.item() - loss_ref) <= 1e-5 * loss_ref
    assert rel(g.cpu().numpy(), g_ref) < 1e-5


@pytest.mark.parametrize("n,two_d,r", SHAPES)
def test_sweep_bf16(n, two_d, r):
    o, A, p = case(n, two_d, r)
    pl = Plan(n, two_d, r)
    A16 = torch.from_numpy(A).float().bfloat16().double().numpy()
    p32 = p.astype(np.float32).astype(np.float64)
    c = pl.coeffs(torch.from_numpy(A).float().to(DEV), "bf16").cpu().numpy()
    assert rel(c, o.coeffs(A16)) < 1e-5
    _, _, g = pl.loss_grad(torch.from_numpy(A).float().to(DEV), torch.from_numpy(p32).float().to(DEV), "bf16")
    _, resid = o.residual(o.coeffs(A16), p32)
    g_ref = o.grad_from_resid(A16, resid)
    bound = (2.0 ** -8 + 4 * o.N * 2.0 ** -24) * o.grad_from_resid(np.abs(A16), np.abs(resid)) + 1e-30
    assert np.all(np.abs(g.cpu().numpy() - g_ref) <= bound)


@pytest.mark.parametrize("n,two_d,r", SHAPES)
def test_sweep_fp64_tc(n, two_d, r):
    o, A, _ = case(n, two_d, r)
    pl = Plan(n, two_d, r)
    c = pl.coeffs(torch.from_numpy(A).to(DEV), "fp64_tc").cpu().numpy()
    e = np.frexp(np.abs(A).max(axis=1))[1].astype(np.float64)
    E = np.repeat(np.exp2(e)[:, None], r, axis=1)
    bound = 10 * 2.0 ** -40 * o.coeffs(E) + 1e-15 * o.coeffs(np.abs(A))
    assert np.all(np.abs(c - o.coeffs(A)) <= bound)
