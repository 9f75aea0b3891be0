"""The single-CTA tensor-core kernels (128 x 256 tiles, one SM per tile), which
run in place of the CTA pairs when the environment sets SOS_CTA_PAIRS=0.  The
library reads that switch once per process, so these checks run in a child
process: the BF16 forward, loss and gradient and one fused GD step, against
the oracle with the tolerances of tests/test_gpu_parity.py.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
import oracle, sos_inputs
from paper_2410_19844_gb300.engine import Optimizer, Plan

def bf16(x):
    return torch.from_numpy(x).float().bfloat16().double().numpy()

for n, two_d, r in [(6, 8, 210), (9, 6, 700), (7, 8, 130)]:
    o = oracle.Oracle(n, two_d)
    A = sos_inputs.normal_matrix(o.N, r, 0, sigma=0.3)
    p = o.coeffs(sos_inputs.normal_matrix(o.N, 5, 1)).astype(np.float32).astype(np.float64)
    pl = Plan(n, two_d, r)
    A16 = bf16(A)
    c = pl.coeffs(torch.from_numpy(A).float().cuda(), "bf16").cpu().numpy()
    c_ref = o.coeffs(A16)
    assert np.linalg.norm(c - c_ref) <= 1e-5 * np.linalg.norm(c_ref), (n, two_d, r)
    loss, _, g = pl.loss_grad(torch.from_numpy(A).float().cuda(), torch.from_numpy(p).float().cuda(), "bf16")
    loss_ref, resid = o.residual(c_ref, p)
    g_ref = o.grad_from_resid(A16, resid)
    assert abs(loss.item() - loss_ref) <= 1e-5 * loss_ref
    bound = (2.0 ** -8 + 4 * o.N * 2.0 ** -24) * o.grad_from_resid(np.abs(A16), np.abs(resid)) + 1e-30
    assert np.all(np.abs(g.cpu().numpy() - g_ref) <= bound)
    A_dev = torch.from_numpy(A).float().cuda()
    opt = Optimizer(pl, A_dev, prec="bf16", optimizer="gd", lr=1e-4)
    opt.step(torch.from_numpy(p).float().cuda())
    want = A.astype(np.float32).astype(np.float64) - 1e-4 * g_ref
    tol = 1e-4 * bound + 2.0 ** -24 * (np.abs(want) + 1e-4 * np.abs(g_ref)) + 1e-30
    assert np.all(np.abs(A_dev.double().cpu().numpy() - want) <= tol)
    assert pl.status("bf16") == 0
print("single-CTA kernels ok")
'''


def test_single_cta_kernels_match_the_oracle():
    env = dict(os.environ, SOS_CTA_PAIRS="0", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    out = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "single-CTA kernels ok" in out.stdout
