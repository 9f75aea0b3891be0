"""The CTA-pair contractions in clusters of two pairs that share the B operand
by TMA multicast (SOS_MCAST=1): pair 0's CTAs load each half of B once into
both pairs' shared memory, every stage is released by both pairs' commits, and
a unit with an odd tile out runs a stand-in whose results are dropped.  The
library reads the switch once per process, so the checks run in child
processes, against the oracle with the tolerances of tests/test_gpu_parity.py
and tests/test_gpu_fullsize.py:

  * small plans (one unit, stand-ins, several units per column block): the BF16
    forward, loss, gradient (unfused adjoint) and one fused GD step;
  * the benchmark size (N = r = 10,626): sampled coefficients, gradient rows
    and one fused step.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SMALL = r'''
import numpy as np, torch
import oracle, sos_inputs
from paper_2410_19844_gb300 import _lib as L
from paper_2410_19844_gb300.engine import Optimizer, Plan

def bf16(x):
    return torch.from_numpy(x).float().bfloat16().double().numpy()

for n, two_d, r in [(10, 8, 300), (13, 8, 64), (6, 8, 210), (9, 6, 700), (3, 4, 10)]:
    o = oracle.Oracle(n, two_d)
    A = sos_inputs.normal_matrix(o.N, r, 0, sigma=0.3)
    p = o.coeffs(sos_inputs.normal_matrix(o.N, 5, 1)).astype(np.float32).astype(np.float64)
    pl = Plan(n, two_d, r)
    A16 = bf16(A)
    c_ref = o.coeffs(A16)
    c = pl.coeffs(torch.from_numpy(A).float().cuda(), "bf16").cpu().numpy()
    assert np.linalg.norm(c - c_ref) <= 1e-5 * np.linalg.norm(c_ref), (n, two_d, r)
    loss_ref, resid = o.residual(c_ref, p)
    g_ref = o.grad_from_resid(A16, resid)
    bound = (2.0 ** -8 + 4 * o.N * 2.0 ** -24) * o.grad_from_resid(np.abs(A16), np.abs(resid)) + 1e-30
    for _ in range(2):      # a second pass on the same workspace
        loss, _, g = pl.loss_grad(torch.from_numpy(A).float().cuda(), torch.from_numpy(p).float().cuda(), "bf16")
        assert abs(loss.item() - loss_ref) <= 1e-5 * loss_ref, (n, two_d, r)
        assert np.all(np.abs(g.cpu().numpy() - g_ref) <= bound), (n, two_d, r)
    A_dev = torch.from_numpy(A).float().cuda()
    opt = Optimizer(pl, A_dev, prec="bf16", optimizer="gd", lr=1e-4)
    opt.step(torch.from_numpy(p).float().cuda())
    want = A.astype(np.float32).astype(np.float64) - 1e-4 * g_ref
    tol = 1e-4 * bound + 2.0 ** -24 * (np.abs(want) + 1e-4 * np.abs(g_ref)) + 1e-30
    assert np.all(np.abs(A_dev.double().cpu().numpy() - want) <= tol), (n, two_d, r)
    assert pl.status("bf16") == L.SOS_OK
print("mcast ok")
'''

FULL = r'''
import numpy as np, torch
import bounds, oracle, sos_inputs
from paper_2410_19844_gb300 import _lib as L
from paper_2410_19844_gb300.engine import Optimizer, Plan

W = sos_inputs.LARGE
o = oracle.Oracle(W.n, W.two_d)
pl = Plan(W.n, W.two_d)
A32 = sos_inputs.init_A(W, 0).astype(np.float32)
p32 = (sos_inputs.normal_matrix(pl.M, 1, 7)[:, 0] * 0.05).astype(np.float32)
rows = [0, 255, 256, 6000, pl.N - 1]
A16 = torch.from_numpy(A32).bfloat16().double().numpy()
u = 2.0 ** -23
ref = bounds.rows_ref(o, A16, p32.astype(np.float64), rows, u, 2.0 ** -8, (pl.r + pl.N) * u)
gen = np.random.default_rng(11)
cidx = np.unique(np.concatenate([[0, 1, pl.M - 2, pl.M - 1], gen.integers(0, pl.M, 60)]))
c = pl.coeffs(torch.from_numpy(A32).cuda(), "bf16")[torch.from_numpy(cidx).cuda()].double().cpu().numpy()
c_ref, c_abs = bounds.coeffs_ref(o, A16, cidx)
assert np.all(np.abs(c - c_ref) <= (pl.r + pl.N) * u * c_abs + 1e-30)
_, _, g = pl.loss_grad(torch.from_numpy(A32).cuda(), torch.from_numpy(p32).cuda(), "bf16")
g_rows = g[rows].double().cpu().numpy()
lr = 1e-4
A_dev = torch.from_numpy(A32).cuda()
opt = Optimizer(pl, A_dev, prec="bf16", optimizer="gd", lr=lr)
opt.step(torch.from_numpy(p32).cuda())
new_rows = A_dev[rows].double().cpu().numpy()
for i, a in enumerate(rows):
    want, bound = ref[a]
    assert np.all(np.abs(g_rows[i] - want) <= bound), f"gradient row {a}"
    step = A32[a].astype(np.float64) - lr * want
    tol = lr * bound + 2.0 ** -24 * (np.abs(step) + lr * np.abs(want)) + 1e-30
    assert np.all(np.abs(new_rows[i] - step) <= tol), f"stepped row {a}"
assert pl.status("bf16") == L.SOS_OK
print("mcast full size ok")
'''


def _run(code, marker, **env_extra):
    env = dict(os.environ, SOS_MCAST="1",
               PYTHONPATH=os.pathsep.join([ROOT, os.path.join(ROOT, "tests"), os.environ.get("PYTHONPATH", "")]))
    env.update(env_extra)
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=900)
    assert out.returncode == 0, out.stdout + out.stderr
    assert marker in out.stdout


@pytest.mark.parametrize("band", ["8", "3"])
def test_mcast_small_plans(band):
    _run(SMALL, "mcast ok", SOS_BAND_ADJ=band)


def test_mcast_full_size():
    _run(FULL, "mcast full size ok")
