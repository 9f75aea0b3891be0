"""GPU parity on the paper's own inputs, and the index table the kernels read.

  * The quartic forms of Sec. 3.1: p = m_2 Q m_2^T with Q = B B^T and B
    uniform in [-1, 1] (l x l, l = C(n_form + 1, 2)).  Dehomogenised (the last
    variable set to 1, Sec. 1.1) this is a polynomial of degree <= 4 in
    n_form - 1 variables whose degree-<=2 monomials match the form's, so the
    oracle builds p as c(B).  At n_form = 10 (N = 55, M = 715) every
    precision is compared with the oracle element by element at a random start
    A0 ~ N(0, 0.1^2), and the generator itself must give a zero residual.  At
    n_form = 100 (N = r = 5050, M = 4,421,275, the paper's largest case)
    sampled coefficients of c(B) and gradient rows at A0 are compared with the
    oracle computed one at a time.
  * The fine-structure target of Sec. 3.4 at n_form = 8 (N = 36, M = 330):
    10 (x_1^2 + ... + x_8^2)^2 plus U[-0.01, 0.01] on every coefficient,
    dehomogenised.  Coefficients near 10 carry a residual near 1e-2, so the
    FP64 paths are checked where the residual is a small difference of large
    coefficients, against the forward error bound the oracle computes.
  * The device index table (built on the GPU from the closed-form rank) is
    compared bit for bit with the oracle's enumerate-and-sort product table.

Tolerances are the ones of tests/test_gpu_parity.py, tests/test_gpu_fp64_tc.py
and tests/test_gpu_fullsize.py (derived there and in tests/bounds.py).
"""
from math import comb

import numpy as np
import pytest
import torch

import bounds
import oracle
import sos_inputs
from paper_2410_19844_gb300 import _lib as L
from paper_2410_19844_gb300.engine import Plan, solve

pytestmark = pytest.mark.gpu

DEV = "cuda"
U64 = 2.0 ** -53


def bf16_round(x):
    return torch.from_numpy(np.asarray(x, dtype=np.float64)).float().bfloat16().double().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def fp64_loss_grad_bounds(o, A, p, gamma):
    """Forward error bound of an FP64 pass at A, both sides' rounding counted
    (a factor 2 over the first-order terms): |dc| <= gamma |c|(|A|) per
    coefficient; |dloss| <= sum |r| |dc| + 1/2 sum dc^2 + (M + 2) u loss for
    the reduction; the gradient within 2 |H(dc)| |A| + (N + 2) u 2 |H(r)| |A|
    elementwise (u = 2^-53)."""
    loss_ref, g_ref, c_ref = o.loss_grad(A, p)
    _, resid = o.residual(c_ref, p)
    dc = 2.0 * gamma * o.coeffs(np.abs(A))
    dloss = float(np.dot(np.abs(resid), dc) + 0.5 * np.dot(dc, dc)) + (o.M + 2) * U64 * loss_ref
    dgrad = 2.0 * (o.grad_from_resid(np.abs(A), dc)
                   + (o.N + 2) * U64 * o.grad_from_resid(np.abs(A), np.abs(resid)))
    return loss_ref, g_ref, c_ref, resid, dloss, dgrad


# -- Sec. 3.1: the quartic forms ------------------------------------------------------

def quartic(n_form, seed=0):
    n = n_form - 1
    o = oracle.Oracle(n, 4)
    assert o.N == comb(n_form + 1, 2) and o.M == comb(n_form + 3, 4)
    B = sos_inputs.paper_quartic_generator(n_form, seed)
    A0 = sos_inputs.normal_matrix(o.N, o.N, seed + 1, sigma=0.1)
    return o, B, o.coeffs(B), A0


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "fp64_tc"])
def test_paper_quartic_n10_matches_oracle(prec):
    o, B, p, A = quartic(10)
    pl = Plan(9, 4)
    assert (pl.N, pl.M) == (55, 715)
    if prec in ("fp64", "fp64_tc"):
        loss, pp, g = pl.loss_grad(torch.from_numpy(A).to(DEV), torch.from_numpy(p).to(DEV), prec)
        g = g.cpu().numpy()
        if prec == "fp64":
            loss_ref, g_ref, _ = o.loss_grad(A, p)
            assert abs(loss.item() - loss_ref) <= 1e-12 * loss_ref
            assert rel(g, g_ref) < 1e-12
        else:
            cb = bounds.slice_scale_bound(o, A)
            loss_ref, g_ref, c_ref = o.loss_grad(A, p)
            _, resid = o.residual(c_ref, p)
            assert abs(loss.item() - loss_ref) <= np.dot(np.abs(resid), cb) + np.dot(cb, cb) + 1e-14 * loss_ref
            terms = o.grad_from_resid(np.abs(A), np.abs(resid))
            assert np.all(np.abs(g - g_ref) <= (2.0 ** -7 + 4 * o.N * 2.0 ** -24) * terms + 1e-300)
        assert abs(pp.item() - np.dot(p, p)) <= 1e-12 * np.dot(p, p)
    elif prec == "fp32":
        A32, p32 = A.astype(np.float32), p.astype(np.float32)
        loss, _, g = pl.loss_grad(torch.from_numpy(A32).to(DEV), torch.from_numpy(p32).to(DEV), "fp32")
        loss_ref, g_ref, _ = o.loss_grad(A32.astype(np.float64), p32.astype(np.float64))
        assert abs(loss.item() - loss_ref) <= 1e-5 * loss_ref
        assert rel(g.cpu().numpy(), g_ref) < 1e-5
    else:
        A16 = bf16_round(A)
        p32 = p.astype(np.float32).astype(np.float64)
        c = pl.coeffs(torch.from_numpy(A).float().to(DEV), "bf16").cpu().numpy()
        assert rel(c, o.coeffs(A16)) < 1e-5
        loss, _, g = pl.loss_grad(torch.from_numpy(A).float().to(DEV), torch.from_numpy(p32).float().to(DEV),
                                  "bf16")
        loss_ref, resid = o.residual(o.coeffs(A16), p32)
        g_ref = o.grad_from_resid(A16, resid)
        assert abs(loss.item() - loss_ref) <= 1e-5 * loss_ref
        terms = o.grad_from_resid(np.abs(A16), np.abs(resid))
        assert np.all(np.abs(g.cpu().numpy() - g_ref) <= (2.0 ** -8 + 4 * o.N * 2.0 ** -24) * terms + 1e-30)


@pytest.mark.parametrize("prec", ["fp64", "fp64_tc"])
def test_paper_quartic_n10_generator_has_zero_residual(prec):
    """At A = B the target is met exactly: the FP64-accurate paths must give a
    residual inside their forward error bound, far below the 1e-8 certificate."""
    o, B, p, _ = quartic(10)
    pl = Plan(9, 4)
    loss, _, _ = pl.loss_grad(torch.from_numpy(B).to(DEV), torch.from_numpy(p).to(DEV), prec, want_grad=False)
    # |c_gpu - p| <= the GPU's forward error + the oracle's own (both FP64 sums)
    fp64 = (pl.r + pl.N + 2) * U64 * o.coeffs(np.abs(B))
    dc = fp64 + (bounds.slice_scale_bound(o, B) if prec == "fp64_tc" else fp64)
    assert loss.item() <= 0.5 * float(np.dot(dc, dc)) + 1e-300
    assert np.sqrt(2.0 * loss.item()) <= 1e-10 * np.linalg.norm(p)


@pytest.fixture(scope="module")
def quartic100():
    """n_form = 100: the target p = c(B) by the oracle (a full product table and
    Gram sums, tens of seconds on the host), sample positions and rows."""
    o, B, p, A0 = quartic(100)
    pl = Plan(99, 4)
    assert (pl.N, pl.M, pl.r) == (5050, 4421275, 5050)
    g = np.random.default_rng(100)
    cidx = np.unique(np.concatenate([[0, 1, pl.M - 2, pl.M - 1], g.integers(0, pl.M, 60)]))
    rows = [0, 255, 256, int(g.integers(257, pl.N - 1)), pl.N - 1]
    return o, pl, B, p, A0, cidx, rows


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp64_tc"])
def test_paper_quartic_n100_sampled_coefficients(quartic100, prec):
    """c(B) at 64 sampled coefficients: for FP64_TC against p itself (the
    oracle's c(B)); for FP32 and BF16 against the oracle at the rounded B,
    within the bounds of tests/test_gpu_fullsize.py."""
    o, pl, B, p, _, cidx, _ = quartic100
    sel = torch.from_numpy(cidx).to(DEV)
    if prec == "fp64_tc":
        c = pl.coeffs(torch.from_numpy(B).to(DEV), "fp64_tc")[sel].cpu().numpy()
        E = bounds.row_scales(B)
        scale = np.array([o.coeff_at(E, int(g)) for g in cidx])
        c_abs = np.array([o.coeff_at(np.abs(B), int(g)) for g in cidx])
        assert np.all(np.abs(c - p[cidx]) <= 10 * 2.0 ** -40 * scale + 1e-15 * c_abs)
        return
    B32 = B.astype(np.float32)
    B_eff = bf16_round(B32) if prec == "bf16" else B32.astype(np.float64)
    u = 2.0 ** -23 if prec == "bf16" else 2.0 ** -24
    c = pl.coeffs(torch.from_numpy(B32).to(DEV), prec)[sel].double().cpu().numpy()
    c_ref, c_abs = bounds.coeffs_ref(o, B_eff, cidx)
    assert np.all(np.abs(c - c_ref) <= (pl.r + pl.N) * u * c_abs + 1e-30)
    if prec == "bf16":
        assert np.linalg.norm(c - c_ref) <= (pl.r / 16 + 64) * 2.0 ** -23 * np.linalg.norm(c_abs)
    else:
        assert np.linalg.norm(c - c_ref) <= 1e-5 * np.linalg.norm(c_ref)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_paper_quartic_n100_gradient_rows(quartic100, prec):
    """Rows of the gradient at A0 for the paper's target, against the oracle's
    rows 2 h A with h_b = (c(A0) - p)_{a+b}."""
    o, pl, _, p, A0, _, rows = quartic100
    A32 = A0.astype(np.float32)
    p32 = p.astype(np.float32)
    A_eff = bf16_round(A32) if prec == "bf16" else A32.astype(np.float64)
    u = 2.0 ** -23 if prec == "bf16" else 2.0 ** -24
    u_r = 2.0 ** -8 if prec == "bf16" else 2.0 ** -24
    _, _, g = pl.loss_grad(torch.from_numpy(A32).to(DEV), torch.from_numpy(p32).to(DEV), prec)
    g_rows = g[rows].double().cpu().numpy()
    ref = bounds.rows_ref(o, A_eff, p32.astype(np.float64), rows, u, u_r, (pl.r + pl.N) * u)
    for i, a in enumerate(rows):
        want, bound = ref[a]
        assert np.all(np.abs(g_rows[i] - want) <= bound), f"row {a}"


# -- Sec. 3.4: fine structure ---------------------------------------------------------

def fine_structure(n_form=8, seed=0):
    """10 (x_1^2 + ... + x_{n_form}^2)^2 + U[-0.01, 0.01] noise, dehomogenised;
    the smooth part is c(q) for the single square q = sqrt(10) (sum x_i^2 + 1)."""
    n = n_form - 1
    o = oracle.Oracle(n, 4)
    q = np.zeros((o.N, 1))
    for a in range(o.N):
        e = o.Ed[a].astype(int)
        if e.sum() == 0 or (e.sum() == 2 and e.max() == 2):
            q[a, 0] = np.sqrt(10.0)
    noise = sos_inputs.fine_structure_noise(o.M, seed)
    return o, q, o.coeffs(q) + noise, noise


def near_solution(o, q, seed=3):
    """The generating square in column 0 and small N(0, 0.01^2) columns: the
    residual is then of the size of the noise, on coefficients up to ~80."""
    A = sos_inputs.normal_matrix(o.N, o.N, seed, sigma=0.01)
    A[:, 0] += q[:, 0]
    return A


@pytest.mark.parametrize("prec", ["fp64", "fp64_tc"])
@pytest.mark.parametrize("where", ["start", "near_solution"])
def test_fine_structure_matches_oracle(prec, where):
    o, q, p, noise = fine_structure()
    pl = Plan(7, 4)
    assert (pl.N, pl.M) == (36, 330)
    A = (sos_inputs.normal_matrix(o.N, o.N, 1, sigma=0.1) if where == "start" else near_solution(o, q))
    loss, _, g = pl.loss_grad(torch.from_numpy(A).to(DEV), torch.from_numpy(p).to(DEV), prec)
    g = g.cpu().numpy()
    c = pl.coeffs(torch.from_numpy(A).to(DEV), prec).cpu().numpy()
    if prec == "fp64":
        gamma = (pl.r + pl.N + 2) * U64
        loss_ref, g_ref, c_ref, resid, dloss, dgrad = fp64_loss_grad_bounds(o, A, p, gamma)
        assert np.all(np.abs(c - c_ref) <= gamma * o.coeffs(np.abs(A)) + 1e-300)
        assert abs(loss.item() - loss_ref) <= dloss + 1e-300
        assert np.all(np.abs(g - g_ref) <= dgrad + 1e-300)
    else:
        cb = bounds.slice_scale_bound(o, A)
        loss_ref, g_ref, c_ref = o.loss_grad(A, p)
        _, resid = o.residual(c_ref, p)
        assert np.all(np.abs(c - c_ref) <= cb + 1e-15 * o.coeffs(np.abs(A)))
        assert abs(loss.item() - loss_ref) <= np.dot(np.abs(resid), cb) + np.dot(cb, cb) + 1e-14 * loss_ref
        terms = o.grad_from_resid(np.abs(A), np.abs(resid))
        assert np.all(np.abs(g - g_ref) <= (2.0 ** -7 + 4 * o.N * 2.0 ** -24) * terms + 1e-300)
    if where == "near_solution":
        # the residual is the noise's size: a check that cancels ~3 digits
        assert np.linalg.norm(resid) < 0.05 * np.linalg.norm(p)


def test_fine_structure_solve_certifies():
    """The default ladder (BF16, then SOS_FP64_TC steps) fits the perturbed
    target to the 1e-8 certificate; the oracle recomputes the error at the
    returned A."""
    o, _, p, _ = fine_structure()
    pl = Plan(7, 4)
    A = torch.from_numpy(sos_inputs.normal_matrix(o.N, o.N, 1, sigma=0.1)).to(DEV)
    res = solve(pl, torch.from_numpy(p).to(DEV), A, max_steps=20000, fp64_steps=20000)
    assert res["verdict"] == L.SOS_VERDICT_SOS, res
    assert o.certify(o.coeffs(A.cpu().numpy()), p) <= 1e-8


# -- the index table the kernels read ---------------------------------------------------

@pytest.mark.parametrize("n,two_d", [(6, 8), (10, 10), (3, 4), (1, 12)])
def test_device_index_table_is_bit_exact(n, two_d):
    o = oracle.Oracle(n, two_d)
    pl = Plan(n, two_d, r=4)
    dev = pl.device_idx()
    assert dev.shape == (o.N, o.N)
    assert np.array_equal(dev, o.prod)
    assert np.array_equal(pl.idx(), o.prod)


def test_device_index_table_rows_at_the_benchmark_size():
    """n = 20, 2d = 8 (N = 10,626): three full rows -- the first, one past the
    256-row tile seam, the last -- against the oracle's rank of each product
    monomial (enumerate-and-sort, binary search)."""
    o = oracle.Oracle(20, 8)
    pl = Plan(20, 8)
    for a in (0, 257, pl.N - 1):
        got = pl.device_idx(a, 1)[0]
        want = np.array([o.rank(o.Ed[a].astype(np.int64) + o.Ed[b]) for b in range(o.N)], dtype=np.int64)
        assert np.array_equal(got.astype(np.int64), want), f"row {a}"
