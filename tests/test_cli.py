"""The command line front end (python -m paper_2410_19844_gb300): the monomial
table on CPU against the oracle's, and solve / certify on a GPU."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import sos_inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_cli(*args):
    out = subprocess.run([sys.executable, "-m", "paper_2410_19844_gb300", *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    return out.stdout


@pytest.mark.parametrize("which", [0, 1])
def test_cli_monomials_match_the_oracle(which):
    text = run_cli("monomials", "--n", "3", "--two-d", "4", "--which", str(which))
    got = np.array([[int(v) for v in line.split()] for line in text.strip().splitlines()])
    o = oracle.Oracle(3, 4)
    want = o.Ed if which == 0 else o.E2d
    assert np.array_equal(got, want)


@pytest.mark.gpu
def test_cli_solve_and_certify(tmp_path):
    o = oracle.Oracle(4, 6)
    p = o.coeffs(sos_inputs.normal_matrix(o.N, 10, 3))
    np.save(tmp_path / "p.npy", p)
    line = run_cli("solve", "--n", "4", "--two-d", "6", "--target", str(tmp_path / "p.npy"),
                   "--out", str(tmp_path / "A.npy"))
    res = json.loads(line.strip().splitlines()[-1])
    assert res["verdict"] == "SOS" and res["rel_resid_fp64"] <= 1e-8
    A = np.load(tmp_path / "A.npy")
    assert o.certify(o.coeffs(A), p) <= 1e-8
    cert = json.loads(run_cli("certify", "--n", "4", "--two-d", "6", "--target", str(tmp_path / "p.npy"),
                              "--A", str(tmp_path / "A.npy")).strip().splitlines()[-1])
    assert cert["verdict"] == "SOS" and abs(cert["rel_resid_fp64"] - res["rel_resid_fp64"]) <= 1e-12
