"""Host-side checks of the library (no GPU): the plan's monomial tables and
index table against the oracle (bit-exact), sizes and edge cases, argument
validation, and that the shared library exports every symbol of the header."""
import ctypes
import os
import re
from math import comb

import numpy as np
import pytest

import oracle
from paper_2410_19844_gb300 import _lib as L
from paper_2410_19844_gb300.engine import Plan

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("n,two_d", [(1, 2), (1, 8), (2, 4), (3, 4), (4, 6), (6, 8), (5, 10), (10, 4)])
def test_tables_match_oracle_bit_exact(n, two_d):
    pl = Plan(n, two_d)
    o = oracle.Oracle(n, two_d)
    assert (pl.N, pl.M) == (comb(n + two_d // 2, two_d // 2), comb(n + two_d, two_d))
    assert np.array_equal(pl.monomials(0), o.Ed)
    assert np.array_equal(pl.monomials(1), o.E2d)
    assert np.array_equal(pl.idx(), o.prod)


def test_idx_symmetric_and_in_range():
    pl = Plan(7, 6)
    idx = pl.idx()
    assert np.array_equal(idx, idx.T)
    assert idx.min() >= 0 and idx.max() < pl.M
    # x^0 * x^a = x^a: the constant monomial is last in degree <= d
    E2 = pl.monomials(1)
    Ed = pl.monomials(0)
    const = pl.N - 1
    for a in range(pl.N):
        assert tuple(E2[idx[a, const]]) == tuple(Ed[a])


def test_rank_r_differs_from_N():
    pl = Plan(3, 4, r=7)
    assert (pl.N, pl.M, pl.r) == (10, 35, 7)


@pytest.mark.parametrize("args", [(0, 4, 1), (3, 3, 1), (3, 0, 1), (3, 4, 0), (250, 8, 1)])
def test_invalid_plans_rejected(args):
    with pytest.raises(L.SOSError) as e:
        L.sos_plan_create(*args)
    assert e.value.code == L.SOS_E_INVALID


def test_sos_plan_is_plan_create_under_its_short_name():
    h = L.sos_plan(20, 8, 10626)
    try:
        assert L.sos_plan_sizes(h) == (10626, 3108105, 10626)
    finally:
        L.sos_plan_destroy(h)
    with pytest.raises(L.SOSError) as e:
        L.sos_plan(3, 3, 1)
    assert e.value.code == L.SOS_E_INVALID


def test_too_many_coefficients_rejected():
    with pytest.raises(L.SOSError) as e:
        L.sos_plan_create(60, 12, 1)     # C(72, 12) > 2^31
    assert e.value.code == L.SOS_E_NOMEM


def test_workspace_sizes_grow_with_precision():
    pl = Plan(6, 8)
    b16 = L.sos_workspace_size(pl.handle, L.SOS_BF16)
    f32 = L.sos_workspace_size(pl.handle, L.SOS_FP32)
    f64 = L.sos_workspace_size(pl.handle, L.SOS_FP64)
    assert f64 > f32 and b16 > f32


def _header_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:int|int64_t|const char\*)\s+(sos_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L.lib()
    lib = ctypes.CDLL(L.library_path())
    names = _header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(L.EXPORTS)


def test_host_calls_validate_arguments():
    pl = Plan(3, 4)
    with pytest.raises(L.SOSError):
        L.sos_workspace_size(pl.handle, 7)
    with pytest.raises(L.SOSError):
        L.sos_plan_monomials(pl.handle, 2, 0)
    with pytest.raises(L.SOSError):
        L.sos_loss_grad(pl.handle, L.SOS_FP32, 0, 0, 0, 0, 0, 0)   # NULL A: rejected on the host
    with pytest.raises(L.SOSError):
        L.sos_plan_device_idx(pl.handle, 8, 5, 0)                 # rows beyond N: rejected on the host


def test_e4m3_slices_change_the_fp64_tc_workspace():
    """With SOS_SLICE_FP8=1 (read once per process, hence child processes) the
    SOS_FP64_TC workspace holds 10 byte-wide slice matrices with rows padded to
    16 bytes instead of 8 bf16 ones with rows padded to 64 elements; nothing
    else in it changes."""
    import subprocess
    import sys
    code = ("from paper_2410_19844_gb300 import _lib as L\n"
            "from paper_2410_19844_gb300.engine import Plan\n"
            "pl = Plan(2, 4, 1000)\n"
            "print(L.sos_workspace_size(pl.handle, L.SOS_FP64_TC))\n")
    sizes = {}
    for fp8 in ("0", "1"):
        env = dict(os.environ, SOS_SLICE_FP8=fp8, PYTHONPATH=ROOT)
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                             timeout=600)
        assert out.returncode == 0, out.stderr
        sizes[fp8] = int(out.stdout.split()[-1])
    NP = 256                                     # N = 6 rows, padded to a 256-row tile
    bf16_slices = 8 * NP * 1024 * 2              # r = 1000: 1024 bf16 per row
    e4m3_slices = 10 * NP * 1008                 # 1008 bytes per row
    assert sizes["1"] - sizes["0"] == e4m3_slices - bf16_slices


def test_slice_format_is_chosen_per_plan():
    """With SOS_SLICE_FP8 unset a plan takes bf16 slices where their products
    are exact (r <= 17,458) and E4M3 slices above: the workspace of the unset
    case equals the forced bf16 one at r = 1000 and the forced E4M3 one at
    r = 20,000."""
    import subprocess
    import sys

    def size(r, fp8):
        code = ("from paper_2410_19844_gb300 import _lib as L\n"
                "from paper_2410_19844_gb300.engine import Plan\n"
                f"pl = Plan(2, 4, {r})\n"
                "print(L.sos_workspace_size(pl.handle, L.SOS_FP64_TC))\n")
        env = dict(os.environ, PYTHONPATH=ROOT)
        env.pop("SOS_SLICE_FP8", None)
        if fp8 is not None:
            env["SOS_SLICE_FP8"] = fp8
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                             timeout=600)
        assert out.returncode == 0, out.stderr
        return int(out.stdout.split()[-1])

    assert size(1000, None) == size(1000, "0") != size(1000, "1")
    assert size(20000, None) == size(20000, "1") != size(20000, "0")
