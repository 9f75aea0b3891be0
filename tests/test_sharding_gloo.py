"""The column split of the step, on CPU with two gloo ranks.

Each rank owns half of the columns (squares) of A.  c(A) is additive over
columns, so the ranks' partial c sum to the full c with one all-reduce of M
values; the residual is then replicated and each rank's gradient columns are
local: grad[:, cols] = 2 H(r) A[:, cols].  This is the one exchange a
multi-GPU step would need; here the algebra is checked with the oracle."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import sos_inputs


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    o = oracle.Oracle(4, 6)
    A = sos_inputs.normal_matrix(o.N, o.N, seed=7, sigma=0.3)
    p = o.coeffs(sos_inputs.normal_matrix(o.N, 5, seed=8))
    cols = np.array_split(np.arange(o.N), world)[rank]
    A_local = np.ascontiguousarray(A[:, cols])
    c = torch.from_numpy(o.coeffs(A_local))
    dist.all_reduce(c, op=dist.ReduceOp.SUM)             # the one exchange per step
    loss, resid = o.residual(c.numpy(), p)
    g_local = o.grad_from_resid(A_local, resid)
    out[rank] = (loss, cols, g_local)
    dist.destroy_process_group()


def test_column_split_matches_full_step():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    o = oracle.Oracle(4, 6)
    A = sos_inputs.normal_matrix(o.N, o.N, seed=7, sigma=0.3)
    p = o.coeffs(sos_inputs.normal_matrix(o.N, 5, seed=8))
    loss_ref, g_ref, _ = o.loss_grad(A, p)
    for r in range(world):
        loss, cols, g_local = out[r]
        assert abs(loss - loss_ref) <= 1e-12 * loss_ref
        np.testing.assert_allclose(g_local, g_ref[:, cols], rtol=1e-11, atol=1e-11)
