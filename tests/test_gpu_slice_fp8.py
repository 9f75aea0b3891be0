"""SOS_FP64_TC with E4M3 slices (SOS_SLICE_FP8=1): each row of A, scaled by a
power of two, is cut into 4-bit integer digits held exactly in E4M3 bytes
(|d| <= 15 needs four significant bits, E4M3 has 1 + 3), and the slice
products run as tcgen05 kind::f8f6f4 MMAs.  Every inner sum is an integer
below r 15^2, exact in the FP32 accumulator while r <= 74,565.  For s 5-bit
slices the library takes s' = ceil(5 s / 4) 4-bit ones, so each term A_ak A_bk
is off by at most (s' + 2) 2^(-4 s') 2^(e_a + e_b) (the bound of
tests/test_gpu_fp64_tc.py with 4-bit digits).  The library reads the switch
once per process, so the checks run in child processes, against the oracle:

  * the forward at small plans, in both tile-list forms -- k = floor((2^24 -
    1) / (15^2 r)) products per accumulator, grouped when k >= 2, one pair per
    launch unit when k = 1 (r > 37,282) -- and at r = 20,000, beyond the bf16
    slices' limit;
  * the loss error shrinking with the slice count, loss and gradient, a NaN
    reaching the status word, and r = 74,566 rejected;
  * the benchmark size (N = r = 10,626): sampled coefficients one at a time.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SMALL = r'''
import numpy as np, torch
import bounds, oracle, sos_inputs
from paper_2410_19844_gb300 import _lib as L
from paper_2410_19844_gb300.engine import Optimizer, Plan

def problem(n, two_d, r, seed=0, spread=True):
    o = oracle.Oracle(n, two_d)
    A = sos_inputs.normal_matrix(o.N, r, seed, sigma=0.3)
    if spread:
        A[1] *= 1e-3
        A[-1] *= 1e3
    p = o.coeffs(sos_inputs.normal_matrix(o.N, 4, seed + 1))
    return o, A, p

L.sos_timing_reset()
L.sos_timing_enable(True)
# (n, 2d, r): grouped with k capped at 8, k = 3 at r = 20,000, and k = 1 (one pair per unit)
for n, two_d, r in [(3, 4, 10), (4, 6, 35), (6, 8, 210), (5, 6, 300), (9, 6, 700), (2, 10, 21),
                    (7, 8, 5000), (2, 4, 20000), (6, 6, 40000), (2, 4, 74565)]:
    o, A, _ = problem(n, two_d, r)
    pl = Plan(n, two_d, r)
    c = pl.coeffs(torch.from_numpy(A).cuda(), "fp64_tc").cpu().numpy()
    c_ref = o.coeffs(A)
    cb = bounds.slice_scale_bound(o, A, slices=10, bits=4)
    err = np.abs(c - c_ref) - (cb + 1e-15 * o.coeffs(np.abs(A)))
    assert np.all(err <= 0), (n, two_d, r, float(err.max()))
    print("forward", n, two_d, r, "worst error / bound", float(np.max(np.abs(c - c_ref) / (cb + 1e-300))))
    del pl

# rows the slicing treats specially: zeros, subnormals only, one entry, 1e-200 .. 1, huge
from test_gpu_fp64_tc import extreme_rows
for n, two_d, r in [(4, 6, 35), (6, 8, 210)]:
    o = oracle.Oracle(n, two_d)
    A = extreme_rows(o, r)
    c = Plan(n, two_d, r).coeffs(torch.from_numpy(A).cuda(), "fp64_tc").cpu().numpy()
    c_ref = o.coeffs(A)
    cb = bounds.slice_scale_bound(o, A, slices=10, bits=4)
    assert np.all(np.isfinite(c)), (n, two_d, r)
    assert np.all(np.abs(c - c_ref) <= cb + 1e-15 * o.coeffs(np.abs(A)) + 1e-320), (n, two_d, r)

# fewer slices: s 5-bit slices -> ceil(5 s / 4) 4-bit ones, the loss error shrinking accordingly
o, A, p = problem(6, 8, 210, seed=3, spread=False)
pl = Plan(6, 8, 210)
loss_ref = o.loss(A, p)
Ad, pd = torch.from_numpy(A).cuda(), torch.from_numpy(p).cuda()
errs = []
for s in range(2, 9):
    opt = Optimizer(pl, Ad.clone(), prec="fp64_tc", optimizer="gd", lr=0.0, slices=s)
    loss = opt.step(pd)[0].item()
    errs.append(abs(loss - loss_ref) / loss_ref)
for s, e in zip(range(2, 9), errs):
    sf = (5 * s + 3) // 4
    assert e <= 2.0 ** (-4 * sf + 12), (s, errs)
assert errs[-1] <= 1e-10, errs
print("slice errors", errs)

# loss and gradient: the forward's bound carried through the residual; the adjoint's bf16 bound
for n, two_d, r in [(4, 6, 35), (6, 8, 210), (9, 6, 700)]:
    o, A, p = problem(n, two_d, r, seed=5)
    pl = Plan(n, two_d, r)
    loss, pp, g = pl.loss_grad(torch.from_numpy(A).cuda(), torch.from_numpy(p).cuda(), "fp64_tc")
    loss_ref, g_ref, c_ref = o.loss_grad(A, p)
    _, resid = o.residual(c_ref, p)
    cb = bounds.slice_scale_bound(o, A, slices=10, bits=4)
    assert abs(loss.item() - loss_ref) <= np.dot(np.abs(resid), cb) + np.dot(cb, cb) + 1e-14 * loss_ref
    terms = o.grad_from_resid(np.abs(A), np.abs(resid))
    bound = (2.0 ** -7 + 4 * o.N * 2.0 ** -24) * terms + 1e-300
    assert np.all(np.abs(g.cpu().numpy() - g_ref) <= bound), (n, two_d, r)

# a NaN in A: its E4M3 slices carry NaN into the coefficients and the status word
o, A, p = problem(4, 6, 35, spread=False)
A[2, 3] = np.nan
pl = Plan(4, 6, 35)
pl.loss_grad(torch.from_numpy(A).cuda(), torch.from_numpy(p).cuda(), "fp64_tc")
assert pl.status("fp64_tc") == L.SOS_E_NONFINITE
assert pl.status("fp64_tc") == L.SOS_OK

# r 15^2 >= 2^24: rejected
pl = Plan(2, 4, 74566)
try:
    pl.coeffs(torch.zeros(pl.N, 74566, dtype=torch.float64, device="cuda"), "fp64_tc")
    raise SystemExit("r = 74,566 was accepted")
except L.SOSError:
    pass
torch.cuda.synchronize()
L.sos_timing_enable(False)
names = L.sos_timing_report()
assert "tc_slices_e4m3" in names and "tc_slices" not in names, names
print("e4m3 slices ok")
'''

FULL = r'''
import numpy as np, torch
import bounds, oracle, sos_inputs
from paper_2410_19844_gb300 import _lib as L
from paper_2410_19844_gb300.engine import Plan

W = sos_inputs.LARGE
o = oracle.Oracle(W.n, W.two_d)
pl = Plan(W.n, W.two_d)
A64 = sos_inputs.init_A(W, 0).astype(np.float32).astype(np.float64)
g = np.random.default_rng(9)
sq = [o.rank(2 * o.Ed[a].astype(np.int64)) for a in (0, 1, pl.N - 1, 5000)]
cidx = np.unique(np.concatenate([sq, [0, pl.M - 1], g.integers(0, pl.M, 60)]))
L.sos_timing_reset()
L.sos_timing_enable(True)
c = pl.coeffs(torch.from_numpy(A64).cuda(), "fp64_tc")[torch.from_numpy(cidx).cuda()].cpu().numpy()
torch.cuda.synchronize()
L.sos_timing_enable(False)
assert "tc_slices_e4m3" in L.sos_timing_report()
c_ref, c_abs = bounds.coeffs_ref(o, A64, cidx)
E = bounds.row_scales(A64)
scale = np.array([o.coeff_at(E, int(k)) for k in cidx])
bound = 12 * 2.0 ** -40 * scale + 1e-15 * c_abs          # s' = 10 four-bit slices
assert np.all(np.abs(c - c_ref) <= bound), float(np.max(np.abs(c - c_ref) / bound))
print("worst error / bound", float(np.max(np.abs(c - c_ref) / bound)))
print("e4m3 full size ok")
'''


def _run(code, marker):
    env = dict(os.environ, SOS_SLICE_FP8="1",
               PYTHONPATH=os.pathsep.join([ROOT, os.path.join(ROOT, "tests"), os.environ.get("PYTHONPATH", "")]))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=1200)
    assert out.returncode == 0, out.stdout + out.stderr
    assert marker in out.stdout
    print(out.stdout)


def test_e4m3_slices_small_plans():
    _run(SMALL, "e4m3 slices ok")


def test_e4m3_slices_full_size_coefficients():
    _run(FULL, "e4m3 full size ok")
