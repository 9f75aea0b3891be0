"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle
on the same seeded inputs.

Tolerances (written here, derived from the arithmetic):
  * FP64 path: 1e-12 relative (normwise) -- only summation order differs.
  * FP32 path (CUDA cores, no TF32): loss and gradient within 1e-5 relative,
    normwise, at a random A -- the accuracy the method is asked to hold.
  * BF16 path: the contractions see A rounded to bf16 and, in the adjoint,
    the residual rounded to bf16 (unit roundoff 2^-8: bf16 keeps 8 bits of
    significand).  The forward is compared with the oracle at the
    bf16-rounded A (1e-5 normwise: FP32 accumulation only); the gradient
    with the oracle at the same A, inside the elementwise bound
    (2^-8 + 4 N 2^-24) * 2 |H(r)| |A| that the rounding of r and the FP32
    accumulation over N terms imply.
"""
import numpy as np
import pytest
import torch

import oracle
import sos_inputs
from paper_2410_19844_gb300 import _lib as L
from paper_2410_19844_gb300.engine import Optimizer, Plan

pytestmark = pytest.mark.gpu

DEV = "cuda"


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def bf16_round(x: np.ndarray) -> np.ndarray:
    return torch.from_numpy(x).float().bfloat16().double().numpy()


def problem(n, two_d, r=None, seed=0, squares=5):
    o = oracle.Oracle(n, two_d)
    r = o.N if r is None else r
    A = sos_inputs.normal_matrix(o.N, r, seed=seed, sigma=0.3)
    G = sos_inputs.normal_matrix(o.N, squares, seed=seed + 1)
    p = o.coeffs(G)
    return o, A, p


# -- the tcgen05 GEMM core ------------------------------------------------------------

@pytest.mark.parametrize("m,n,k", [(128, 256, 64), (256, 512, 128), (200, 300, 100), (384, 256, 1000),
                                   (640, 520, 320)])
@pytest.mark.parametrize("b_mn", [0, 1])
@pytest.mark.parametrize("pairs", [0, 1])
def test_tc_gemm_matches_fp64_matmul(m, n, k, b_mn, pairs):
    g = torch.Generator().manual_seed(m * 7 + n * 3 + k + b_mn)
    X = torch.randn(m, k, generator=g).bfloat16()
    Y = torch.randn(k, n, generator=g).bfloat16() if b_mn else torch.randn(n, k, generator=g).bfloat16()
    ref = X.double() @ (Y.double() if b_mn else Y.double().T)
    ldx = (k + 63) // 64 * 64
    ldy = ((n if b_mn else k) + 63) // 64 * 64
    Xd = torch.zeros(m, ldx, dtype=torch.bfloat16, device=DEV)
    Xd[:, :k] = X.to(DEV)
    Yd = torch.zeros(Y.shape[0], ldy, dtype=torch.bfloat16, device=DEV)
    Yd[:, :Y.shape[1]] = Y.to(DEV)
    D = torch.full((m, n), float("nan"), dtype=torch.float32, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    L.sos_diag_gemm_bf16(b_mn | (2 * pairs), Xd.data_ptr(), Yd.data_ptr(), D.data_ptr(), m, n, k, ldx, ldy,
                         status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert int(status.item()) == 0
    got = D.double().cpu().numpy()
    # FP32 accumulation of exact bf16 products: 4 k 2^-24 sum|x||y| (a layout
    # mistake gives errors of the size of the entries themselves)
    bound = 4 * k * 2.0 ** -24 * (X.double().abs() @ (Y.double().abs() if b_mn else Y.double().abs().T)).numpy()
    assert np.all(np.abs(got - ref.numpy()) <= bound + 1e-30)


# -- forward --------------------------------------------------------------------

@pytest.mark.parametrize("n,two_d,r", [(3, 4, 10), (4, 6, 9), (6, 8, 210), (5, 6, 300), (2, 10, 21)])
def test_forward_fp64(n, two_d, r):
    o, A, _ = problem(n, two_d, r)
    pl = Plan(n, two_d, r)
    c = pl.coeffs(torch.from_numpy(A).to(DEV), "fp64").cpu().numpy()
    assert rel(c, o.coeffs(A)) < 1e-12


@pytest.mark.parametrize("n,two_d,r", [(6, 8, 210), (5, 6, 300), (7, 6, 50), (8, 4, 45)])
def test_forward_fp32(n, two_d, r):
    o, A, _ = problem(n, two_d, r)
    pl = Plan(n, two_d, r)
    c = pl.coeffs(torch.from_numpy(A).float().to(DEV), "fp32").cpu().numpy()
    assert rel(c, o.coeffs(A.astype(np.float32).astype(np.float64))) < 1e-5


@pytest.mark.parametrize("n,two_d,r", [(6, 8, 210), (5, 6, 300), (7, 8, 130), (9, 6, 700), (3, 4, 10)])
def test_forward_bf16(n, two_d, r):
    o, A, _ = problem(n, two_d, r)
    pl = Plan(n, two_d, r)
    c = pl.coeffs(torch.from_numpy(A).float().to(DEV), "bf16").cpu().numpy()
    assert rel(c, o.coeffs(bf16_round(A))) < 1e-5


# -- loss and gradient ---------------------------------------------------------------

@pytest.mark.parametrize("n,two_d,r", [(3, 4, 10), (4, 6, 35), (6, 8, 210), (5, 6, 77)])
def test_loss_grad_fp64(n, two_d, r):
    o, A, p = problem(n, two_d, r)
    pl = Plan(n, two_d, r)
    loss, pp, g = pl.loss_grad(torch.from_numpy(A).to(DEV), torch.from_numpy(p).to(DEV), "fp64")
    loss_ref, g_ref, _ = o.loss_grad(A, p)
    assert abs(loss.item() - loss_ref) <= 1e-12 * loss_ref
    assert abs(pp.item() - np.dot(p, p)) <= 1e-12 * np.dot(p, p)
    assert rel(g.cpu().numpy(), g_ref) < 1e-12


@pytest.mark.parametrize("n,two_d,r", [(6, 8, 210), (5, 6, 300), (7, 6, 50), (4, 10, 1001), (8, 4, 45)])
def test_loss_grad_fp32(n, two_d, r):
    o, A, p = problem(n, two_d, r)
    A32 = A.astype(np.float32)
    p32 = p.astype(np.float32)
    pl = Plan(n, two_d, r)
    loss, _, g = pl.loss_grad(torch.from_numpy(A32).to(DEV), torch.from_numpy(p32).to(DEV), "fp32")
    loss_ref, g_ref, _ = o.loss_grad(A32.astype(np.float64), p32.astype(np.float64))
    assert abs(loss.item() - loss_ref) <= 1e-5 * loss_ref
    assert rel(g.cpu().numpy(), g_ref) < 1e-5


@pytest.mark.parametrize("n,two_d,r", [(6, 8, 210), (5, 6, 300), (7, 8, 130), (9, 6, 700)])
def test_loss_grad_bf16(n, two_d, r):
    o, A, p = problem(n, two_d, r)
    A16 = bf16_round(A)
    p32 = p.astype(np.float32).astype(np.float64)
    pl = Plan(n, two_d, r)
    loss, _, g = pl.loss_grad(torch.from_numpy(A).float().to(DEV), torch.from_numpy(p32).float().to(DEV),
                              "bf16")
    c_ref = o.coeffs(A16)
    loss_ref, resid = o.residual(c_ref, p32)
    g_ref = o.grad_from_resid(A16, resid)
    assert abs(loss.item() - loss_ref) <= 1e-5 * loss_ref
    terms = o.grad_from_resid(np.abs(A16), np.abs(resid))      # 2 |H(r)| |A|
    bound = (2.0 ** -8 + 4 * o.N * 2.0 ** -24) * terms + 1e-30
    assert np.all(np.abs(g.cpu().numpy() - g_ref) <= bound)


def test_loss_only_skips_gradient():
    o, A, p = problem(4, 6)
    pl = Plan(4, 6)
    loss, _, g = pl.loss_grad(torch.from_numpy(A).to(DEV), torch.from_numpy(p).to(DEV), "fp64",
                              want_grad=False)
    assert g is None
    assert abs(loss.item() - o.loss(A, p)) <= 1e-12 * o.loss(A, p)


# -- batched FP32 (64 instances of n=6, 2d=8, 50 squares each) ------------------------------

def test_batched_fp32_matches_oracle_and_differences():
    w = sos_inputs.BATCH
    o = oracle.Oracle(w.n, w.two_d)
    pl = Plan(w.n, w.two_d)
    batch = 64
    As = np.stack([sos_inputs.init_A(w, s) for s in range(batch)]).astype(np.float32)
    ps = np.stack([o.coeffs(sos_inputs.generator(w, s)) for s in range(batch)]).astype(np.float32)
    loss, _, g = pl.loss_grad_batched(torch.from_numpy(As).to(DEV), torch.from_numpy(ps).to(DEV), "fp32")
    loss, g = loss.cpu().numpy(), g.cpu().numpy()
    rng = np.random.default_rng(5)
    for s in [0, 1, 31, 63]:
        A64, p64 = As[s].astype(np.float64), ps[s].astype(np.float64)
        loss_ref, g_ref, _ = o.loss_grad(A64, p64)
        assert abs(loss[s] - loss_ref) <= 1e-5 * loss_ref
        assert rel(g[s], g_ref) < 1e-5
        # central differences with h = 1e-3 in FP64, Richardson-combined (exact for a quartic)
        for _ in range(32):
            e = (int(rng.integers(o.N)), int(rng.integers(o.N)))
            E = np.zeros_like(A64)
            E[e] = 1.0

            def D(h):
                return (o.loss(A64 + h * E, p64) - o.loss(A64 - h * E, p64)) / (2 * h)
            fd = (4 * D(0.5e-3) - D(1e-3)) / 3
            assert abs(g[s][e] - fd) <= 1e-5 * np.abs(g_ref).max()


# -- optimiser step -------------------------------------------------------------------

@pytest.mark.parametrize("optimizer", ["adam", "gd"])
def test_step_fp64_matches_oracle(optimizer):
    o, A, p = problem(3, 4)
    A_dev = torch.from_numpy(A.copy()).to(DEV)
    pl = Plan(3, 4)
    opt = Optimizer(pl, A_dev, prec="fp64", optimizer=optimizer, lr=1e-2)
    p_dev = torch.from_numpy(p).to(DEV)
    Aref, m, v = A.copy(), np.zeros_like(A), np.zeros_like(A)
    for t in range(1, 6):
        loss = opt.step(p_dev)[0].item()
        loss_ref, g, _ = o.loss_grad(Aref, p)
        assert abs(loss - loss_ref) <= 1e-12 * loss_ref
        if optimizer == "adam":
            o.adam_step(Aref, m, v, g, t, lr=1e-2)
        else:
            o.gd_step(Aref, g, 1e-2)
        assert rel(A_dev.cpu().numpy(), Aref) < 1e-12


# -- the 128 x 128 CUDA-core tiles (N >= about 2100) --------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_large_simt_tiles(prec):
    """n = 13, 2d = 8: N = 2380 takes the 128 x 128 SIMT kernels (r = 300 keeps
    the oracle quick; the tile grid depends on N only)."""
    o, A, p = problem(13, 8, 300, squares=3)
    pl = Plan(13, 8, 300)
    dt = np.float64 if prec == "fp64" else np.float32
    A_ = A.astype(dt)
    p_ = p.astype(dt)
    loss, _, g = pl.loss_grad(torch.from_numpy(A_).to(DEV), torch.from_numpy(p_).to(DEV), prec)
    loss_ref, g_ref, _ = o.loss_grad(A_.astype(np.float64), p_.astype(np.float64))
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert abs(loss.item() - loss_ref) <= tol * loss_ref
    assert rel(g.cpu().numpy(), g_ref) < tol
    if prec == "fp32":    # the certificate's forward: FP32 A, FP64 sums
        rel_c, _ = pl.certify(torch.from_numpy(A_).to(DEV), torch.from_numpy(p).to(DEV))
        c = o.coeffs(A_.astype(np.float64))
        assert abs(rel_c - o.certify(c, p)) <= 1e-10 * o.certify(c, p)


# -- degenerate shapes -------------------------------------------------------------------

DEGENERATE = [(1, 2, 1),      # one variable, quadratic, one square: N = 2, M = 3
              (1, 20, 11),    # univariate: H(r) is a true Hankel matrix
              (1, 40, 21),
              (2, 2, 1),      # a single square of an affine form
              (5, 2, 1),
              (30, 2, 6),     # many variables, degree 2: N = 31, M = 496
              (4, 8, 1)]      # rank one at a larger degree


@pytest.mark.parametrize("n,two_d,r", DEGENERATE)
def test_degenerate_shapes_fp64(n, two_d, r):
    o, A, p = problem(n, two_d, r, squares=2)
    pl = Plan(n, two_d, r)
    loss, _, g = pl.loss_grad(torch.from_numpy(A).to(DEV), torch.from_numpy(p).to(DEV), "fp64")
    loss_ref, g_ref, _ = o.loss_grad(A, p)
    assert abs(loss.item() - loss_ref) <= 1e-12 * loss_ref
    assert rel(g.cpu().numpy(), g_ref) < 1e-12


@pytest.mark.parametrize("n,two_d,r", DEGENERATE)
def test_degenerate_shapes_fp32_and_bf16(n, two_d, r):
    o, A, p = problem(n, two_d, r, squares=2)
    pl = Plan(n, two_d, r)
    A32 = A.astype(np.float32)
    p32 = p.astype(np.float32).astype(np.float64)
    loss, _, g = pl.loss_grad(torch.from_numpy(A32).to(DEV), torch.from_numpy(p32).float().to(DEV), "fp32")
    loss_ref, g_ref, _ = o.loss_grad(A32.astype(np.float64), p32)
    assert abs(loss.item() - loss_ref) <= 1e-5 * loss_ref
    assert rel(g.cpu().numpy(), g_ref) < 1e-5
    A16 = bf16_round(A)
    c = pl.coeffs(torch.from_numpy(A32).to(DEV), "bf16").cpu().numpy()
    assert rel(c, o.coeffs(A16)) < 1e-5


# -- certificate and status ---------------------------------------------------------------

def test_certify_generating_matrix():
    o = oracle.Oracle(4, 6)
    A0 = sos_inputs.normal_matrix(o.N, o.N, seed=3)
    p = o.coeffs(A0)
    pl = Plan(4, 6)
    rel_res, verdict = pl.certify(torch.from_numpy(A0).to(DEV), torch.from_numpy(p).to(DEV))
    assert rel_res <= 1e-14 and verdict == L.SOS_VERDICT_SOS
    A1 = sos_inputs.normal_matrix(o.N, o.N, seed=4)
    rel_res, verdict = pl.certify(torch.from_numpy(A1).float().to(DEV), torch.from_numpy(p).to(DEV))
    want = o.certify(o.coeffs(A1.astype(np.float32).astype(np.float64)), p)
    assert abs(rel_res - want) <= 1e-12 * want and verdict == L.SOS_VERDICT_NOT_CONVERGED


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_nonfinite_target_sets_status(prec):
    o, A, p = problem(4, 6)
    p[3] = np.nan
    pl = Plan(4, 6)
    pl.loss_grad(torch.from_numpy(A).float().to(DEV), torch.from_numpy(p).float().to(DEV), prec)
    assert pl.status(prec) == L.SOS_E_NONFINITE
    assert pl.status(prec) == L.SOS_OK      # read-and-clear


# -- the fused BF16 step (update inside the adjoint epilogue) --------------------------------

@pytest.mark.parametrize("r", [4750, 4900])
def test_bf16_adjoint_narrow_tail_tiles(r):
    # N = 1001 (4 row blocks of 256) and r = 4750 or 4900 (19 or 20 column blocks):
    # 76 or 80 adjoint tiles.  With 72 to 76 resident CTA pairs one of the two
    # lists ends in a short last round, whose tiles run as 128-column halves;
    # the last column block is 142 (two halves) or 36 (one half) wide.
    # At this depth the forward's FP32 accumulation may truncate once per
    # 16-deep MMA step, so the bounds are those of tests/test_gpu_fullsize.py:
    # |dc| <= (r + N) u |c|(|A|) elementwise and (r / 16 + 64) u ||c(|A|)||
    # normwise, u = 2^-23, carried through the BF16 residual into the gradient.
    o, A, p = problem(10, 8, r)
    A16 = bf16_round(A)
    absA = np.abs(A16)
    p32 = p.astype(np.float32).astype(np.float64)
    pl = Plan(10, 8, r)
    A_dev = torch.from_numpy(A).float().to(DEV)
    p_dev = torch.from_numpy(p32).float().to(DEV)
    loss, _, g = pl.loss_grad(A_dev, p_dev, "bf16")
    loss_ref, resid = o.residual(o.coeffs(A16), p32)
    g_ref = o.grad_from_resid(A16, resid)
    u = 2.0 ** -23
    c_abs = o.coeffs(absA)
    dnorm = (r / 16 + 64) * u * np.linalg.norm(c_abs)
    assert abs(loss.item() - loss_ref) <= np.linalg.norm(resid) * dnorm + 0.5 * dnorm ** 2 + 1e-6 * loss_ref
    dc = (r + o.N) * u * c_abs
    dh = dc + 2.0 ** -8 * (np.abs(resid) + dc)
    bound = o.grad_from_resid(absA, dh) + o.N * u * o.grad_from_resid(absA, np.abs(resid) + dh) + 1e-30
    assert np.all(np.abs(g.cpu().numpy() - g_ref) <= bound)
    lr = 1e-4
    opt = Optimizer(pl, A_dev, prec="bf16", optimizer="gd", lr=lr)
    opt.step(p_dev)
    want = A.astype(np.float32).astype(np.float64) - lr * g_ref
    assert np.all(np.abs(A_dev.double().cpu().numpy() - want) <= lr * bound + 4 * 2.0 ** -24 * np.abs(want) + 1e-30)


@pytest.mark.parametrize("n,two_d,r", [(6, 8, 210), (7, 8, 130), (9, 6, 700)])
def test_fused_bf16_gd_steps(n, two_d, r):
    o, A, p = problem(n, two_d, r)
    p32 = p.astype(np.float32).astype(np.float64)
    pl = Plan(n, two_d, r)
    A_dev = torch.from_numpy(A).float().to(DEV)
    lr = 1e-4
    opt = Optimizer(pl, A_dev, prec="bf16", optimizer="gd", lr=lr)
    p_dev = torch.from_numpy(p32).float().to(DEV)
    A_prev = A.astype(np.float32).astype(np.float64)
    for step in range(3):
        loss = opt.step(p_dev)[0].item()
        A16 = bf16_round(A_prev)                 # what the contractions saw
        loss_ref, resid = o.residual(o.coeffs(A16), p32)
        assert abs(loss - loss_ref) <= 1e-5 * loss_ref, step
        g_ref = o.grad_from_resid(A16, resid)
        bound = (2.0 ** -8 + 4 * o.N * 2.0 ** -24) * o.grad_from_resid(np.abs(A16), np.abs(resid))
        A_new = A_dev.double().cpu().numpy()
        want = A_prev - lr * g_ref
        assert np.all(np.abs(A_new - want) <= lr * bound + 4 * 2.0 ** -24 * np.abs(want) + 1e-30), step
        A_prev = A_new                          # next step's loss: at bf16 of the updated A


def test_fused_bf16_adam_moments():
    o, A, p = problem(6, 8, 210)
    p32 = p.astype(np.float32).astype(np.float64)
    pl = Plan(6, 8, 210)
    A_dev = torch.from_numpy(A).float().to(DEV)
    opt = Optimizer(pl, A_dev, prec="bf16", optimizer="adam", lr=1e-3)
    opt.step(torch.from_numpy(p32).float().to(DEV))
    A16 = bf16_round(A.astype(np.float32).astype(np.float64))
    _, resid = o.residual(o.coeffs(A16), p32)
    g_ref = o.grad_from_resid(A16, resid)
    bound = (2.0 ** -8 + 4 * o.N * 2.0 ** -24) * o.grad_from_resid(np.abs(A16), np.abs(resid))
    m = opt.m.double().cpu().numpy()
    v = opt.v.double().cpu().numpy()
    f1 = float(np.float32(1) - np.float32(0.9))     # (1 - beta1) as the kernel forms it in FP32
    f2 = float(np.float32(1) - np.float32(0.999))
    assert np.all(np.abs(m - f1 * g_ref) <= f1 * bound * 1.001 + 1e-7 * np.abs(g_ref))
    assert np.all(np.abs(np.sqrt(v / f2) - np.abs(g_ref)) <= bound * 1.001 + 1e-6 * np.abs(g_ref))


@pytest.mark.parametrize("optimizer", ["adam", "gd"])
def test_step_fp32_matches_oracle(optimizer):
    o, A, p = problem(5, 6, 56)
    A32 = A.astype(np.float32)
    p32 = p.astype(np.float32)
    pl = Plan(5, 6, 56)
    A_dev = torch.from_numpy(A32.copy()).to(DEV)
    opt = Optimizer(pl, A_dev, prec="fp32", optimizer=optimizer, lr=1e-3)
    p_dev = torch.from_numpy(p32).to(DEV)
    Aref = A32.astype(np.float64)
    m, v = np.zeros_like(Aref), np.zeros_like(Aref)
    for t in range(1, 4):
        opt.step(p_dev)
        _, g, _ = o.loss_grad(Aref, p32.astype(np.float64))
        if optimizer == "adam":
            o.adam_step(Aref, m, v, g, t, lr=1e-3)
        else:
            o.gd_step(Aref, g, 1e-3)
        got = A_dev.double().cpu().numpy()
        assert rel(got, Aref) < 1e-5
        Aref = got.copy()                        # compare one step at a time
        if optimizer == "adam":
            m = opt.m.double().cpu().numpy().copy()
            v = opt.v.double().cpu().numpy().copy()


def test_fp64_step_with_fp32_adjoint():
    """FP64 iterate, residual and update; the adjoint contracted in FP32: the
    gradient a GD step applies is the oracle's to FP32 accuracy."""
    o, A, p = problem(6, 8, 210)
    pl = Plan(6, 8, 210)
    A_dev = torch.from_numpy(A.copy()).to(DEV)
    lr = 1e-3
    opt = Optimizer(pl, A_dev, prec="fp64", optimizer="gd", lr=lr, fp32_adjoint=True)
    loss = opt.step(torch.from_numpy(p).to(DEV))[0].item()
    loss_ref, g_ref, _ = o.loss_grad(A, p)
    assert abs(loss - loss_ref) <= 1e-12 * loss_ref          # the forward is still FP64
    g_applied = (A - A_dev.cpu().numpy()) / lr
    assert rel(g_applied, g_ref) < 1e-5
