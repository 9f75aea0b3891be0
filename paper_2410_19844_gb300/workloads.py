"""Device-resident request streams for the serving benchmark (config of the
serving workload: Poisson arrivals, n uniform in {3..8}, 2d uniform in
{4, 6, 8}, r = N; even ids a sum of floor(N/2) random squares, odd ids that
target minus (p(x0) + 1) at a point x0 where it is then negative).

Targets are built with the library's own FP64 forward; the shift at x0 is a
host-side polynomial evaluation.  x0 is taken from seeded candidates until
the residual lower bound 1 / ||m_2d(x0)|| exceeds 1e-6 ||p'||, so that no
iterate can reach the 1e-8 certificate on a negative target.
"""
from __future__ import annotations

import numpy as np
import torch

import sos_inputs

from .engine import Plan
from .server import Job


def build_jobs(count: int, rate_per_s: float, seed: int = 0, arrivals: bool = True):
    reqs = sos_inputs.request_stream(count, rate_per_s, seed)
    gen_plans, mono = {}, {}
    jobs = []
    for req in reqs:
        key = (req.n, req.two_d)
        if key not in gen_plans:
            gen_plans[key] = Plan(req.n, req.two_d, r=max(1, req.N // 2))
            mono[key] = gen_plans[key].monomials(1).astype(np.int64)
        G = torch.from_numpy(sos_inputs.request_generator(req)).cuda()
        p = gen_plans[key].coeffs(G.contiguous(), "fp64")
        if not req.sos:
            ph = p.cpu().numpy()
            E = mono[key]
            for x0 in sos_inputs.request_points(req):
                mv = np.prod(x0[None, :] ** E, axis=1)
                q = ph.copy()
                q[-1] -= float(np.dot(ph, mv)) + 1.0          # the constant monomial is last
                if 1.0 / np.linalg.norm(mv) > 1e-6 * np.linalg.norm(q):
                    p = torch.from_numpy(q).cuda()
                    break
            else:
                raise RuntimeError(f"request {req.rid}: no admissible point")
        A0 = torch.from_numpy(sos_inputs.request_init(req)).cuda()
        jobs.append(Job(req.rid, req.arrival_s if arrivals else 0.0, req.n, req.two_d,
                        (lambda p=p, A0=A0: (p, A0))))
    torch.cuda.synchronize()
    return jobs
