"""GPU checks of the grouped step and the continuous-batching server."""
import numpy as np
import pytest
import torch

import oracle
import sos_inputs
from paper_2410_19844_gb300 import _lib as L
from paper_2410_19844_gb300.engine import Optimizer, Plan, _ptr, _stream_handle
from paper_2410_19844_gb300.server import Job, Policy, Server, latency_stats, run_plain

pytestmark = pytest.mark.gpu

_ORACLES = {}


def _oracle(n, two_d):
    if (n, two_d) not in _ORACLES:
        _ORACLES[(n, two_d)] = oracle.Oracle(n, two_d)
    return _ORACLES[(n, two_d)]


def make_request(rid, n, two_d, sos, arrival=0.0):
    """SOS: p = sum of floor(N/2) random squares; otherwise p - (p(x0) + 1) at a
    point x0 resampled until the Cauchy-Schwarz bound 1 / ||m_2d(x0)|| exceeds
    1e-6 ||p'|| (so a certificate at 1e-8 is impossible)."""
    o = _oracle(n, two_d)
    g = np.random.default_rng(rid)
    p = o.coeffs(g.standard_normal((o.N, max(1, o.N // 2))))
    if not sos:
        for _ in range(100):
            x0 = g.standard_normal(n)
            q = p.copy()
            q[o.rank([0] * n)] -= o.eval(p, x0) + 1.0
            mvec = np.prod(x0[None, :] ** o.E2d.astype(np.int64), axis=1)
            if 1.0 / np.linalg.norm(mvec) > 1e-6 * np.linalg.norm(q):
                p = q
                break
        else:
            raise RuntimeError("no admissible point")
    A0 = g.normal(0.0, 0.1, size=(o.N, o.N))

    def make():
        return torch.from_numpy(p).cuda(), torch.from_numpy(A0).cuda()
    return Job(rid, arrival, n, two_d, make)


def _group_run(prec, jobs, steps, flags=0):
    """Runs `jobs` together in one group; returns each one's current A."""
    dt = torch.float64 if prec == L.SOS_FP64 else torch.float32
    g = L.sos_group_create(prec, len(jobs), L.SOS_ADAM, flags=flags)
    keep, plans = [], {}
    st = _stream_handle()
    for s, job in enumerate(jobs):
        plans.setdefault((job.n, job.two_d), Plan(job.n, job.two_d))
        pl = plans[(job.n, job.two_d)]
        p64, A0 = job.make()
        A = A0.to(dt).contiguous()
        p = p64.to(dt).contiguous()
        m, v = torch.zeros_like(A), torch.zeros_like(A)
        scratch = torch.empty(L.sos_group_scratch_size(pl.handle, prec), dtype=torch.uint8, device="cuda")
        L.sos_group_set(g, s, pl.handle, _ptr(A), _ptr(m), _ptr(v), _ptr(p), _ptr(scratch), 1e-2, 0)
        keep.append((A, m, v, p, scratch))
    L.sos_group_sync(g, st)
    L.sos_group_run(g, steps, st)
    losses = np.zeros(2 * len(jobs))
    L.sos_group_losses(g, losses.ctypes.data, st)
    out = []
    for s, job in enumerate(jobs):
        cur, _, taken = L.sos_group_state(g, s)
        assert taken == steps
        N = plans[(job.n, job.two_d)].N
        buf = torch.empty(N, N, dtype=dt, device="cuda")
        torch.cuda.synchronize()
        L.sos_convert(cur, prec, _ptr(buf), prec, N * N, st)
        torch.cuda.synchronize()
        out.append(buf.cpu().numpy())
    L.sos_group_destroy(g)
    return out, losses


@pytest.mark.parametrize("prec", [L.SOS_FP32, L.SOS_FP64])
def test_iterates_identical_alone_and_mixed(prec):
    target = make_request(7, 5, 6, True)
    others = [make_request(10 + i, n, d, i % 2 == 0) for i, (n, d) in
              enumerate([(3, 4), (8, 8), (6, 8), (4, 6), (7, 4)])]
    alone, _ = _group_run(prec, [target], 40)
    mixed, _ = _group_run(prec, others[:2] + [target] + others[2:], 40)
    assert np.array_equal(alone[0], mixed[2])


FAST = L.SOS_GROUP_FP32_ADJOINT | L.SOS_GROUP_FAST_FP64


def test_fast_fp64_iterates_identical_alone_and_mixed():
    target = make_request(7, 5, 6, True)
    others = [make_request(10 + i, n, d, i % 2 == 0) for i, (n, d) in
              enumerate([(3, 4), (8, 8), (6, 8), (4, 6), (7, 4)])]
    alone, _ = _group_run(L.SOS_FP64, [target], 40, FAST)
    mixed, _ = _group_run(L.SOS_FP64, others[:2] + [target] + others[2:], 40, FAST)
    assert np.array_equal(alone[0], mixed[2])


@pytest.mark.parametrize("n,two_d", [(4, 6), (8, 8)])
def test_fast_fp64_loss_matches_oracle(n, two_d):
    """The double-float forward: the loss of the start point within 1e-11 of the
    oracle's FP64 loss (about 2^-46 per coefficient, relative to its |products|)."""
    job = make_request(21, n, two_d, True)
    o = _oracle(n, two_d)
    p64, A0 = job.make()
    _, losses = _group_run(L.SOS_FP64, [job], 1, FAST)
    loss_ref = o.loss(A0.cpu().numpy(), p64.cpu().numpy())
    assert abs(losses[0] - loss_ref) <= 1e-11 * loss_ref


def test_group_fp64_step_matches_oracle():
    job = make_request(3, 4, 6, True)
    o = _oracle(4, 6)
    p64, A0 = job.make()
    A_ref, m, v = A0.cpu().numpy().copy(), np.zeros((o.N, o.N)), np.zeros((o.N, o.N))
    got, losses = _group_run(L.SOS_FP64, [job], 3)
    p = p64.cpu().numpy()
    for t in range(1, 4):
        loss_ref, g, _ = o.loss_grad(A_ref, p)
        o.adam_step(A_ref, m, v, g, t, lr=1e-2)
    assert np.linalg.norm(got[0] - A_ref) <= 1e-12 * np.linalg.norm(A_ref)
    assert abs(losses[0] - loss_ref) <= 1e-12 * loss_ref     # loss of the third iterate


def test_group_fp32_matches_single_problem_path():
    job = make_request(5, 6, 8, True)
    pl = Plan(6, 8)
    p64, A0 = job.make()
    A = A0.float().contiguous()
    p32 = p64.float().contiguous()
    loss_single, _, _ = pl.loss_grad(A, p32, "fp32", want_grad=False)
    _, losses = _group_run(L.SOS_FP32, [job], 1)
    assert abs(losses[0] - loss_single.item()) <= 1e-5 * loss_single.item()


def _stream(count, seed, rate, shapes):
    g = np.random.default_rng(seed)
    t = np.cumsum(g.exponential(1.0 / rate, size=count))
    t -= t[0]
    jobs = []
    for i in range(count):
        n, d = shapes[int(g.integers(len(shapes)))]
        jobs.append(make_request(1000 + i, n, d, i % 2 == 0, arrival=float(t[i])))
    return jobs


def test_server_verdicts_match_construction_and_plain_path():
    jobs = _stream(16, 0, 200.0, [(3, 4), (4, 4), (3, 6), (4, 6), (5, 4)])
    srv = Server(capacity=8, steps_per_tick=32)
    served = {v.rid: v for v in srv.run(jobs)}
    plain = {v.rid: v for v in run_plain(jobs)}
    srv.close()
    assert len(served) == len(jobs) == len(plain)
    for j in jobs:
        want = L.SOS_VERDICT_SOS if (j.rid % 2 == 0) else L.SOS_VERDICT_NOT_CONVERGED
        assert served[j.rid].verdict == want, (j.rid, served[j.rid])
        assert plain[j.rid].verdict == want, (j.rid, plain[j.rid])
        if want == L.SOS_VERDICT_SOS:
            assert served[j.rid].rel <= 1e-8
    stats = latency_stats(list(served.values()))
    assert stats["p99_s"] >= stats["p50_s"] > 0


def test_admission_respects_the_hbm_budget():
    jobs = _stream(6, 1, 1000.0, [(4, 6), (5, 6)])
    one = Plan(5, 6)
    budget = 2 * (4 * (5 * one.N ** 2 + 3 * one.M) + 64 * 1024)     # two FP32 problems at most
    srv = Server(capacity=8, hbm_budget=budget + 8 * (5 * one.N ** 2 + 3 * one.M) + 64 * 1024,
                 steps_per_tick=32)
    out = srv.run(jobs)
    srv.close()
    assert len(out) == len(jobs)
    assert srv.peak_used <= srv.budget


def test_nonfinite_request_fails_alone():
    good = _stream(4, 2, 1000.0, [(3, 4), (4, 6)])
    bad = make_request(99, 4, 6, True)
    p64, A0 = bad.make()
    p64[5] = float("nan")
    bad.make = lambda: (p64, A0)
    srv = Server(capacity=8, steps_per_tick=32)
    out = {v.rid: v for v in srv.run(good + [bad])}
    srv.close()
    assert out[99].verdict == L.SOS_VERDICT_ERROR
    for j in good:
        want = L.SOS_VERDICT_SOS if j.rid % 2 == 0 else L.SOS_VERDICT_NOT_CONVERGED
        assert out[j.rid].verdict == want


def test_deadline_times_requests_out_and_frees_their_slots():
    """A request past its deadline is answered TIMEOUT between ticks and its
    slot and memory go back to the pool; the same server then serves the
    same requests to their normal verdicts."""
    from paper_2410_19844_gb300.server import VERDICT_TIMEOUT
    jobs = _stream(6, 3, 1000.0, [(4, 4), (4, 6)])
    srv = Server(capacity=8, steps_per_tick=32, policy=Policy(deadline_s=0.0))
    out = srv.run(jobs)
    assert sorted(v.rid for v in out) == sorted(j.rid for j in jobs)
    assert all(v.verdict == VERDICT_TIMEOUT for v in out)
    assert srv.used == 0 and not srv.active32 and not srv.active64
    assert len(srv.free32) == len(srv.free64) == 8
    srv.policy = Policy()
    again = {v.rid: v for v in srv.run(jobs)}
    srv.close()
    for j in jobs:
        want = L.SOS_VERDICT_SOS if j.rid % 2 == 0 else L.SOS_VERDICT_NOT_CONVERGED
        assert again[j.rid].verdict == want
