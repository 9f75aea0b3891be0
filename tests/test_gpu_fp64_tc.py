"""GPU checks of SOS_FP64_TC: the forward c(A) to FP64 accuracy on tensor cores
by exact 5-bit slices (Ozaki et al., error-free splitting of a matrix
product), through the C ABI, against the oracle.

  * The premise: a tcgen05 product of integer matrices with entries in
    [-31, 31] is exact in its FP32 accumulator while k 31^2 < 2^24, in either
    kernel (single CTA, CTA pairs) -- compared bit for bit with int64 matmul.
  * The forward with s slices: every coefficient within (s + 2) 2^(-5 s) of
    the same sum taken over 2^(e_a + e_b) -- the rows' power-of-two scales --
    in place of A[a][k] A[b][k].  Per term, the dropped slice products (i + j
    >= s) add at most s 2^(-5 s) 2^(e_a + e_b) and the truncated tails of the
    two rows 2 2^(-5 s) 2^(e_a + e_b); the FP64 sums add rounding far below.
  * Fewer slices: the loss error shrinks about 32-fold per slice.
  * Past r = 17,458, where bf16 slice products would not be exact, the plan
    takes E4M3 slices of 4-bit digits (exact up to r = 74,565); r = 74,566 is
    refused.
  * The adjoint reads bf16 H(r) and bf16 A: inside (2^-7 + 4 N 2^-24) 2|H(r)||A|.
  * Steps converge: the solver with tc_fp64 certifies an SOS target below
    1e-8, the oracle agreeing.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import sos_inputs
from paper_2410_19844_gb300 import _lib as L
from paper_2410_19844_gb300.engine import Optimizer, Plan, solve

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.mark.parametrize("k", [64, 1000, 4096, 17000])
@pytest.mark.parametrize("pairs", [0, 1])
def test_tc_gemm_is_exact_on_small_integers(k, pairs):
    m, n = 256, 512
    g = np.random.default_rng(k + pairs)
    X = g.integers(-31, 32, size=(m, k))
    Y = g.integers(-31, 32, size=(n, k))
    X[0] = 31                                  # one row and column at the largest sums
    Y[0] = 31
    ref = X.astype(np.int64) @ Y.astype(np.int64).T
    assert np.abs(ref).max() < 2 ** 24
    ld = (k + 63) // 64 * 64
    Xd = torch.zeros(m, ld, dtype=torch.bfloat16, device=DEV)
    Xd[:, :k] = torch.from_numpy(X).to(torch.bfloat16).to(DEV)
    Yd = torch.zeros(n, ld, dtype=torch.bfloat16, device=DEV)
    Yd[:, :k] = torch.from_numpy(Y).to(torch.bfloat16).to(DEV)
    D = torch.full((m, n), float("nan"), dtype=torch.float32, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    L.sos_diag_gemm_bf16(2 * pairs, Xd.data_ptr(), Yd.data_ptr(), D.data_ptr(), m, n, k, ld, ld,
                         status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert int(status.item()) == 0
    assert np.array_equal(D.cpu().numpy().astype(np.int64), ref)


def scale_bound(o, A, slices=8, bits=5):
    """(s + 2) 2^(-b s) times the coefficients of the matrix whose row a is
    2^e_a everywhere (e_a: exponent of the row's largest entry, frexp), for s
    slices of b-bit digits."""
    e = np.frexp(np.abs(A).max(axis=1))[1].astype(np.float64)
    E = np.repeat(np.exp2(e)[:, None], A.shape[1], axis=1)
    return (slices + 2) * 2.0 ** (-bits * slices) * o.coeffs(E), E


def problem(n, two_d, r, seed=0, sigma=0.3, spread=True):
    o = oracle.Oracle(n, two_d)
    A = sos_inputs.normal_matrix(o.N, r, seed, sigma=sigma)
    if spread:                                 # rows of very different scales
        A[1] *= 1e-3
        A[-1] *= 1e3
    p = o.coeffs(sos_inputs.normal_matrix(o.N, 4, seed + 1))
    return o, A, p


# r decides the form of the slice products: k = floor((2^24 - 1) / (31^2 r)) products
# share an accumulator (k >= 2: grouped, upper triangle), or each pair alone (k = 1)
@pytest.mark.parametrize("n,two_d,r", [(3, 4, 10), (4, 6, 35), (6, 8, 210), (5, 6, 300), (9, 6, 700),
                                       (2, 10, 21),
                                       (7, 8, 5000),     # k = 3: a cross pair and the diagonal together
                                       (2, 4, 6000),     # k = 2: one cross pair per group
                                       (7, 8, 9000)])    # k = 1: one pair per product, cross pairs on all tiles
def test_fp64_tc_forward_matches_oracle(n, two_d, r):
    o, A, _ = problem(n, two_d, r)
    pl = Plan(n, two_d, r)
    c = pl.coeffs(torch.from_numpy(A).to(DEV), "fp64_tc").cpu().numpy()
    c_ref = o.coeffs(A)
    bound, _ = scale_bound(o, A)
    assert np.all(np.abs(c - c_ref) <= bound + 1e-15 * o.coeffs(np.abs(A)))


def test_fp64_tc_error_shrinks_with_slices():
    n, two_d = 6, 8
    o, A, p = problem(n, two_d, 210, seed=3, spread=False)
    pl = Plan(n, two_d, 210)
    loss_ref = o.loss(A, p)
    Ad = torch.from_numpy(A).to(DEV)
    pd = torch.from_numpy(p).to(DEV)
    errs = []
    for s in range(2, 9):
        opt = Optimizer(pl, Ad.clone(), prec="fp64_tc", optimizer="gd", lr=0.0, slices=s)
        loss = opt.step(pd)[0].item()              # the loss before the (zero) update
        errs.append(abs(loss - loss_ref) / loss_ref)
    for s, e in zip(range(2, 9), errs):
        assert e <= 2.0 ** (-5 * s + 12), (s, errs)
    assert errs[-1] <= 1e-10


@pytest.mark.parametrize("n,two_d,r", [(4, 6, 35), (6, 8, 210), (9, 6, 700)])
def test_fp64_tc_loss_and_gradient(n, two_d, r):
    o, A, p = problem(n, two_d, r, seed=5)
    pl = Plan(n, two_d, r)
    loss, pp, g = pl.loss_grad(torch.from_numpy(A).to(DEV), torch.from_numpy(p).to(DEV), "fp64_tc")
    loss_ref, g_ref, c_ref = o.loss_grad(A, p)
    _, resid = o.residual(c_ref, p)
    cb, _ = scale_bound(o, A)                   # |dc| per coefficient, as in the forward test
    assert abs(loss.item() - loss_ref) <= np.dot(np.abs(resid), cb) + np.dot(cb, cb) + 1e-14 * loss_ref
    assert abs(pp.item() - np.dot(p, p)) <= 1e-12 * np.dot(p, p)
    terms = o.grad_from_resid(np.abs(A), np.abs(resid))       # 2 |H(r)| |A|
    bound = (2.0 ** -7 + 4 * o.N * 2.0 ** -24) * terms + 1e-300
    assert np.all(np.abs(g.cpu().numpy() - g_ref) <= bound)


def test_solver_with_tc_fp64_certifies():
    n, two_d = 5, 6
    o = oracle.Oracle(n, two_d)
    p = o.coeffs(sos_inputs.normal_matrix(o.N, o.N // 2, 11))
    pl = Plan(n, two_d)
    A = torch.from_numpy(sos_inputs.normal_matrix(o.N, o.N, 12, sigma=0.1)).to(DEV)
    res = solve(pl, torch.from_numpy(p).to(DEV), A, tc_fp64=1, max_steps=20000, fp64_steps=6000)
    assert res["verdict"] == L.SOS_VERDICT_SOS, res
    assert res["steps_fp32"] == 0 and res["steps_fp64"] > 0
    assert o.certify(o.coeffs(A.cpu().numpy()), p) <= 1e-8


def test_fp64_tc_rejects_what_it_cannot_do_exactly():
    pl = Plan(2, 4, 74566)                     # r 15^2 >= 2^24: neither slice format is exact
    A = torch.zeros(pl.N, 74566, dtype=torch.float64, device=DEV)
    with pytest.raises(L.SOSError):
        pl.coeffs(A, "fp64_tc")
    with pytest.raises(L.SOSError):
        L.sos_loss_grad_batched(pl.handle, L.SOS_FP64_TC, 1, 0, 0, 0, 0, 0, 0)


@pytest.mark.parametrize("r", [17459, 30000])
def test_fp64_tc_past_the_bf16_limit_takes_e4m3_slices(r):
    """r 31^2 >= 2^24: bf16 slice products would not be exact, so the plan takes
    E4M3 slices of 4-bit digits (10 for the default 8 five-bit ones), inside
    their bound (s' + 2) 2^(-4 s') per term (the default process, SOS_SLICE_FP8
    unset, unless the environment forces a format)."""
    if os.environ.get("SOS_SLICE_FP8"):
        pytest.skip("SOS_SLICE_FP8 forces one format for every plan")
    o, A, _ = problem(2, 4, r)
    pl = Plan(2, 4, r)
    L.sos_timing_reset()
    L.sos_timing_enable(True)
    c = pl.coeffs(torch.from_numpy(A).to(DEV), "fp64_tc").cpu().numpy()
    torch.cuda.synchronize()
    L.sos_timing_enable(False)
    assert "tc_slices_e4m3" in L.sos_timing_report()
    c_ref = o.coeffs(A)
    bound, _ = scale_bound(o, A, slices=10, bits=4)
    assert np.all(np.abs(c - c_ref) <= bound + 1e-15 * o.coeffs(np.abs(A)))


def extreme_rows(o, r, seed=7):
    """A with rows the slicing treats specially: all zeros, subnormal entries
    only, a single entry, entries spanning 1e-200 .. 1, and huge entries."""
    g = np.random.default_rng(seed)
    A = g.normal(0.0, 0.3, size=(o.N, r))
    A[0] = 0.0
    A[1] = g.integers(-1000, 1000, size=r) * 5e-324          # subnormal (and zero) entries
    A[2] = 0.0
    A[2, r // 2] = -0.75
    A[3] = g.normal(0.0, 1.0, size=r) * 10.0 ** g.uniform(-200, 0, size=r)
    A[4] *= 1e150
    return A


@pytest.mark.parametrize("n,two_d,r", [(4, 6, 35), (6, 8, 210)])
def test_fp64_tc_extreme_rows(n, two_d, r):
    """Zero, subnormal, single-entry, wide-range and huge rows: the forward stays
    inside the slicing bound (plus a few subnormal units, where FP64 itself
    rounds products into the subnormal range)."""
    o = oracle.Oracle(n, two_d)
    A = extreme_rows(o, r)
    pl = Plan(n, two_d, r)
    c = pl.coeffs(torch.from_numpy(A).to(DEV), "fp64_tc").cpu().numpy()
    c_ref = o.coeffs(A)
    bound, _ = scale_bound(o, A)
    assert np.all(np.isfinite(c))
    assert np.all(np.abs(c - c_ref) <= bound + 1e-15 * o.coeffs(np.abs(A)) + 1e-320)


def test_fp64_tc_nonfinite_entry_sets_status():
    """A NaN in A reaches the coefficients (its slices carry NaN) and the status word."""
    o, A, p = problem(4, 6, 35, spread=False)
    A[2, 3] = np.nan
    pl = Plan(4, 6, 35)
    pl.loss_grad(torch.from_numpy(A).to(DEV), torch.from_numpy(p).to(DEV), "fp64_tc")
    assert pl.status("fp64_tc") == L.SOS_E_NONFINITE
    assert pl.status("fp64_tc") == L.SOS_OK
