"""Pins of the CPU oracle against what the paper and mathematics fix.

Every check here is independent of the oracle's own arithmetic: fixtures from
the paper (tests/golden/, each with its citation), closed forms, the quartic
identities of Sec. 2, the univariate case (numpy.convolve), evaluation at
points, exact Richardson differences, invariances.  The last group plants
plausible mistakes in a copy of the oracle and checks that a pin catches each.
"""
from math import comb

import numpy as np
import pytest

import oracle
import sos_inputs
from pins import (directional_coeff_derivative, general_rule_coeff, golden_path,
                  load_closed_forms, load_rows, point_eval_error,
                  quartic_identity_coeffs, richardson_derivative)


def paper_order_key(e):
    # higher degree first, then larger tuple first (Sec. 1.1 example)
    return (-int(sum(e)), tuple(-int(v) for v in e))


# -- monomial tables ----------------------------------------------------------

def test_paper_example_order():
    want = [tuple(int(v) for v in r) for r in load_rows(golden_path("monomials_n2_d2.txt"))]
    got = [tuple(int(v) for v in r) for r in oracle.monomials(2, 2)]
    assert got == want


@pytest.mark.parametrize("n,deg", [(1, 0), (1, 5), (2, 4), (3, 6), (5, 4), (6, 8), (4, 10)])
def test_monomial_tables_complete_and_ordered(n, deg):
    E = oracle.monomials(n, deg)
    assert len(E) == comb(n + deg, deg)
    rows = [tuple(int(v) for v in e) for e in E]
    assert len(set(rows)) == len(rows)
    assert all(sum(r) <= deg for r in rows)
    keys = [paper_order_key(r) for r in rows]
    assert keys == sorted(keys)


def test_paper_counts():
    for n_form, deg, count, *cite in load_rows(golden_path("paper_counts.txt")):
        n_form, deg, count = int(n_form), int(deg), int(count)
        # homogenisation: forms in n_form variables <-> degree <= deg in n_form - 1
        assert oracle.count_monomials(n_form - 1, deg) == count, " ".join(cite)


def test_workload_sizes():
    for n, two_d, N, M in [(3, 4, 10, 35), (6, 8, 210, 3003), (10, 10, 3003, 184756),
                           (20, 8, 10626, 3108105)]:
        assert oracle.count_monomials(n, two_d // 2) == N
        assert oracle.count_monomials(n, two_d) == M


def test_rank_roundtrip_and_product_table():
    o = oracle.Oracle(4, 6)
    for g in range(o.M):
        assert o.rank(o.E2d[g]) == g
    prod = o.prod
    for a in range(o.N):
        for b in range(o.N):
            assert tuple(o.E2d[prod[a, b]]) == tuple(o.Ed[a] + o.Ed[b])
    assert np.array_equal(prod, prod.T)


# -- c(A) -----------------------------------------------------------------------

def build_A(o, form):
    r = 1 + max(k for k, _, _ in form["q"])
    A = np.zeros((o.N, r))
    for k, e, v in form["q"]:
        A[o.rank(e, "d"), k] = v * np.sqrt(form["scale"])
    return A


@pytest.mark.parametrize("form", load_closed_forms(golden_path("closed_forms.txt")),
                         ids=lambda f: f["name"])
def test_closed_forms(form):
    o = oracle.Oracle(form["n"], form["two_d"])
    c = o.coeffs(build_A(o, form))
    want = np.zeros(o.M)
    for e, v in form["c"].items():
        want[o.rank(e)] = v
    np.testing.assert_allclose(c, want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n,two_d,r", [(2, 4, 3), (3, 4, 10), (4, 6, 7), (6, 8, 12), (3, 10, 5)])
def test_point_evaluation(n, two_d, r):
    o = oracle.Oracle(n, two_d)
    A = sos_inputs.normal_matrix(o.N, r, seed=11)
    X = sos_inputs.points(n, 8, seed=12)
    assert point_eval_error(o.coeffs, o.Ed, o.E2d, A, X) < 1e-12


def test_sum_of_coefficients_is_value_at_ones():
    o = oracle.Oracle(5, 6)
    A = sos_inputs.normal_matrix(o.N, 9, seed=3)
    q1 = A.sum(axis=0)                      # q_k(1, ..., 1)
    assert np.isclose(o.coeffs(A).sum(), np.dot(q1, q1), rtol=1e-12)


@pytest.mark.parametrize("n", [4, 5])
def test_quartic_identities_of_section_2(n):
    """Homogeneous quadratics q_k: the quartic coefficients equal the five
    identities of Sec. 2 and the general rule stated after them."""
    o = oracle.Oracle(n, 4)
    A = sos_inputs.normal_matrix(o.N, 6, seed=5)
    A[o.Ed.sum(axis=1) < 2] = 0.0           # keep only the degree-2 rows
    c = o.coeffs(A)
    want = quartic_identity_coeffs(o.Ed, o.E2d, A)
    np.testing.assert_allclose(c, want, rtol=1e-12, atol=1e-12)
    for g in range(o.M):
        if o.E2d[g].sum() == 4:
            assert np.isclose(c[g], general_rule_coeff(o.Ed, A, o.E2d[g]), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("two_d", [2, 4, 8, 12])
def test_univariate_is_convolution(two_d):
    """n = 1: coefficients (highest power first) are sum_k convolve(q_k, q_k)."""
    o = oracle.Oracle(1, two_d)
    A = sos_inputs.normal_matrix(o.N, 4, seed=7)
    want = sum(np.convolve(A[:, k], A[:, k]) for k in range(A.shape[1]))
    np.testing.assert_allclose(o.coeffs(A), want, rtol=1e-13, atol=1e-13)


def test_orthogonal_invariance():
    o = oracle.Oracle(4, 6)
    A = sos_inputs.normal_matrix(o.N, o.N, seed=8)
    Q = sos_inputs.orthogonal(o.N, seed=9)
    np.testing.assert_allclose(o.coeffs(A @ Q), o.coeffs(A), rtol=1e-11, atol=1e-11)


def test_coeff_at_matches_full():
    o = oracle.Oracle(5, 6)
    A = sos_inputs.normal_matrix(o.N, 6, seed=13)
    c = o.coeffs(A)
    for g in [0, 1, 17, o.M // 2, o.M - 1]:
        assert np.isclose(o.coeff_at(A, g), c[g], rtol=1e-12, atol=1e-12)


# -- loss and gradient --------------------------------------------------------------

def _problem(n=3, two_d=4, r=5, seed=21):
    o = oracle.Oracle(n, two_d)
    A = sos_inputs.normal_matrix(o.N, r, seed=seed)
    G = sos_inputs.normal_matrix(o.N, 3, seed=seed + 1)
    p = o.coeffs(G)
    return o, A, p


def test_gradient_matches_exact_richardson_differences():
    o, A, p = _problem()
    _, g, _ = o.loss_grad(A, p)
    for entry in [(0, 0), (3, 2), (o.N - 1, 4), (5, 1)]:
        fd = richardson_derivative(lambda X: o.loss(X, p), A, entry, 1e-2)
        assert abs(fd - g[entry]) <= 1e-9 * max(1.0, np.abs(g).max())


def test_adjoint_identity():
    """<r, Dc[A].E> = <grad, E> for the loss 1/2 ||r||^2."""
    o, A, p = _problem(4, 6, 6)
    loss, g, c = o.loss_grad(A, p)
    resid = c - p
    E = sos_inputs.normal_matrix(*A.shape, seed=99)
    lhs = float(np.dot(resid, directional_coeff_derivative(o.coeffs, A, E)))
    assert np.isclose(lhs, float(np.sum(g * E)), rtol=1e-10)


def test_zero_at_generating_matrix():
    o = oracle.Oracle(3, 6)
    A0 = sos_inputs.normal_matrix(o.N, o.N, seed=4)
    p = o.coeffs(A0)
    loss, g, _ = o.loss_grad(A0, p)
    scale = float(np.dot(p, p))
    assert loss <= 1e-28 * scale
    assert np.abs(g).max() <= 1e-13 * np.sqrt(scale) * np.abs(A0).max()
    assert o.certify(o.coeffs(A0), p) <= 1e-14


def test_gradient_equivariance():
    o, A, p = _problem(3, 4, 10)
    Q = sos_inputs.orthogonal(10, seed=31)
    _, g, _ = o.loss_grad(A, p)
    _, gq, _ = o.loss_grad(A @ Q, p)
    np.testing.assert_allclose(gq, g @ Q, rtol=1e-10, atol=1e-10)


def test_gradient_linear_in_residual():
    o, A, p = _problem(3, 4, 4)
    r1 = sos_inputs.normal_matrix(o.M, 1, seed=1)[:, 0]
    r2 = sos_inputs.normal_matrix(o.M, 1, seed=2)[:, 0]
    g = o.grad_from_resid
    np.testing.assert_allclose(g(A, 2 * r1 - 3 * r2), 2 * g(A, r1) - 3 * g(A, r2),
                               rtol=1e-12, atol=1e-12)


def test_grad_row_matches_full():
    o, A, p = _problem(4, 6, 5)
    _, g, _ = o.loss_grad(A, p)
    for a in [0, 7, o.N - 1]:
        np.testing.assert_allclose(o.grad_row(A, p, a), g[a], rtol=1e-11, atol=1e-11)


def test_resid_row_is_the_residual_at_monomial_sums():
    """h_b = (c - p) at the monomial E_a + E_b, looked up in the full residual."""
    o, A, p = _problem(4, 6, 5)
    _, resid = o.residual(o.coeffs(A), p)
    for a in [0, 11, o.N - 1]:
        want = np.array([resid[o.rank(o.Ed[a].astype(int) + o.Ed[b].astype(int))] for b in range(o.N)])
        np.testing.assert_allclose(o.resid_row(A, p, a), want, rtol=1e-12, atol=1e-12)


# -- optimiser ------------------------------------------------------------------

def test_adam_hand_worked_steps():
    rows = load_rows(golden_path("adam_hand.txt"))
    A, m, v = np.ones(1), np.zeros(1), np.zeros(1)
    for t, g, m_want, v_want, theta_want in rows:
        oracle.Oracle.adam_step(A, m, v, np.array([float(g)]), int(t), lr=0.1)
        assert np.isclose(m[0], float(m_want), rtol=1e-14, atol=1e-16)
        assert np.isclose(v[0], float(v_want), rtol=1e-14, atol=1e-16)
        assert np.isclose(A[0], float(theta_want), rtol=1e-14)


def test_adam_constant_gradient_moves_lr_per_step():
    """With a constant gradient, bias correction makes mhat = g and vhat = g^2
    at every step, so every coordinate moves lr * |g| / (|g| + eps)."""
    g = np.array([3.0, -0.25, 1e-3])
    A, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 6):
        oracle.Oracle.adam_step(A, m, v, g, t, lr=0.01)
    np.testing.assert_allclose(A, -5 * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_gd_step():
    A = np.array([1.0, 2.0])
    oracle.Oracle.gd_step(A, np.array([0.5, -1.0]), 0.1)
    np.testing.assert_allclose(A, [0.95, 2.1], rtol=1e-15)


# -- evaluation and certificate ------------------------------------------------------

def test_eval_closed_form():
    o = oracle.Oracle(2, 4)
    form = [f for f in load_closed_forms(golden_path("closed_forms.txt"))
            if f["name"] == "mixed_degree"][0]
    c = o.coeffs(build_A(o, form))
    for x, y in [(0.3, -1.2), (2.0, 0.5), (-1.0, -1.0)]:
        assert np.isclose(o.eval(c, [x, y]), (x * x - x * y + 2) ** 2, rtol=1e-13)


def test_nonsos_lower_bound():
    """p' = p - (p(x0) + 1) is negative at x0, and every SOS c satisfies
    ||c - p'||_2 >= 1 / ||m_2d(x0)||_2 (Cauchy-Schwarz), so no A can certify it."""
    o = oracle.Oracle(3, 4)
    G = sos_inputs.normal_matrix(o.N, 5, seed=1)
    p = o.coeffs(G)
    x0 = sos_inputs.normal_matrix(1, 3, seed=2)[0]
    const = o.rank([0, 0, 0])
    p[const] -= o.eval(p, x0) + 1.0
    assert np.isclose(o.eval(p, x0), -1.0)
    mvec = np.array([o.eval(np.eye(o.M)[g], x0) for g in range(o.M)])
    bound = 1.0 / np.linalg.norm(mvec)
    for seed in range(5):
        A = sos_inputs.normal_matrix(o.N, o.N, seed=100 + seed)
        c = o.coeffs(A)
        assert np.linalg.norm(c - p) >= bound


# -- planted mistakes: each must be caught by one of the pins above ---------------

class _Mutant:
    def __init__(self, o, kind):
        self.o, self.kind = o, kind

    def coeffs(self, A):
        c = self.o.coeffs(A)
        if self.kind == "upper_pairs_only":
            # forgets that B_ab and B_ba both contribute: halves off-diagonal pairs
            c = self.o.coeffs(A)
            diag = np.zeros_like(c)
            for a in range(self.o.N):
                diag[self.o.prod[a, a]] += np.dot(A[a], A[a])
            c = 0.5 * (c + diag)
        elif self.kind == "shifted_rank":
            c = np.roll(c, 1)
        return c

    def loss(self, A, p):
        c = self.coeffs(A)
        return 0.5 * float(np.sum((c - p) ** 2))

    def grad(self, A, p):
        _, g, _ = self.o.loss_grad(A, p)
        if self.kind == "grad_missing_factor_2":
            return 0.5 * g
        if self.kind == "grad_transposed_operand":
            return g[:, ::-1].copy()
        return g


@pytest.mark.parametrize("kind", ["upper_pairs_only", "shifted_rank"])
def test_planted_forward_mistakes_are_caught(kind):
    o = oracle.Oracle(3, 4)
    A = sos_inputs.normal_matrix(o.N, 4, seed=2)
    X = sos_inputs.points(3, 8, seed=3)
    assert point_eval_error(o.coeffs, o.Ed, o.E2d, A, X) < 1e-12
    assert point_eval_error(_Mutant(o, kind).coeffs, o.Ed, o.E2d, A, X) > 1e-6


@pytest.mark.parametrize("kind", ["grad_missing_factor_2", "grad_transposed_operand"])
def test_planted_gradient_mistakes_are_caught(kind):
    o, A, p = _problem()
    mut = _Mutant(o, kind)
    g = mut.grad(A, p)
    worst = 0.0
    for entry in [(0, 0), (3, 2), (o.N - 1, 4)]:
        fd = richardson_derivative(lambda X: o.loss(X, p), A, entry, 1e-2)
        worst = max(worst, abs(fd - g[entry]) / max(1.0, abs(fd)))
    assert worst > 1e-3
