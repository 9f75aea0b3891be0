"""GPU checks of sos_solve against the oracle: the BF16 -> FP32 -> FP64
ladder (tc_fp64 = 0) and BF16 -> SOS_FP64_TC (tc_fp64 = 1, the default), and
the certificate."""
import numpy as np
import pytest
import torch

import oracle
import sos_inputs
from paper_2410_19844_gb300 import _lib as L
from paper_2410_19844_gb300.engine import Plan, solve

pytestmark = pytest.mark.gpu


def _sos_problem(n, two_d, squares, seed):
    o = oracle.Oracle(n, two_d)
    p = o.coeffs(sos_inputs.normal_matrix(o.N, squares, seed=seed))
    A0 = sos_inputs.normal_matrix(o.N, o.N, seed=seed + 1, sigma=0.1)
    return o, p, A0


@pytest.mark.parametrize("start,tc", [("bf16", 0), ("bf16", 1), ("fp32", 0)])
def test_ladder_certifies_an_sos_target(start, tc):
    o, p, A0 = _sos_problem(4, 6, 17, seed=0)
    pl = Plan(4, 6)
    A = torch.from_numpy(A0.copy()).cuda()
    res = solve(pl, torch.from_numpy(p).cuda(), A, start_prec=start, max_steps=3000, check_every=25,
                fp64_steps=3000, tc_fp64=tc)
    print(res)
    assert res["verdict"] == L.SOS_VERDICT_SOS
    assert res["rel_resid_fp64"] <= 1e-8
    # the oracle agrees on the returned A
    rel_ref = o.certify(o.coeffs(A.cpu().numpy()), p)
    assert rel_ref <= 1e-8
    assert abs(rel_ref - res["rel_resid_fp64"]) <= 1e-3 * rel_ref + 1e-15
    if start == "bf16":
        assert res["steps_bf16"] > 0 and res["rel_at_switch"] > 0


@pytest.mark.parametrize("tc", [0, 1])
def test_ladder_never_certifies_a_negative_target(tc):
    """p' = p - (p(x0) + 1) is negative at x0, hence not SOS; its residual
    cannot go below 1 / ||m_2d(x0)|| (Cauchy-Schwarz)."""
    o, p, A0 = _sos_problem(3, 4, 5, seed=3)
    x0 = sos_inputs.normal_matrix(1, 3, seed=4)[0]
    p[o.rank([0, 0, 0])] -= o.eval(p, x0) + 1.0
    mvec = np.array([np.prod(x0 ** e.astype(np.int64)) for e in o.E2d])
    bound = 1.0 / np.linalg.norm(mvec) / np.linalg.norm(p)
    pl = Plan(3, 4)
    A = torch.from_numpy(A0.copy()).cuda()
    res = solve(pl, torch.from_numpy(p).cuda(), A, max_steps=1500, check_every=50, fp64_steps=500, tc_fp64=tc)
    assert res["verdict"] == L.SOS_VERDICT_NOT_CONVERGED
    assert res["rel_resid_fp64"] >= bound
    assert abs(o.certify(o.coeffs(A.cpu().numpy()), p) - res["rel_resid_fp64"]) <= 1e-9
