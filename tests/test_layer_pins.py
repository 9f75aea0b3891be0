"""CPU pins of the oracle's network with its first layer (Sec. 2, Eq. 4,
Sec. 2.1): the quartic form ||B Z A1 x||^2.

  * the coefficients evaluate to the network's value at random points, with
    Z built literally as blocks x_i I (dehomogenised table, x_nf = 1);
  * on the homogeneous table, the quartic coefficients equal the five
    identities of Sec. 2 with f_{x_i x_j} from sub-blocks of B and columns of
    A1, as the paper computes them;
  * a change of basis v -> G v of the first layer's output, undone in B, leaves
    the form unchanged;
  * the gradients with respect to B and A1 equal exact Richardson differences
    (the loss is a quartic polynomial along any line in B or in A1);
  * mistakes planted in a copy of the expansion and of the chain rule are
    caught by these pins.
"""
import numpy as np
import pytest

import oracle
import sos_inputs
from pins import network_second_derivative, network_value, quartic_identities, richardson_derivative


def net(nf, m, k, seed):
    B = sos_inputs.normal_matrix(k, nf * m, seed, sigma=0.5)
    A1 = sos_inputs.normal_matrix(m, nf, seed + 1, sigma=0.5)
    return B, A1


@pytest.mark.parametrize("nf,m,k", [(3, 3, 2), (5, 5, 7), (5, 10, 4), (6, 4, 9)])
def test_coefficients_evaluate_to_the_network(nf, m, k):
    o = oracle.Oracle(nf - 1, 4)
    B, A1 = net(nf, m, k, 3)
    c = o.layer_coeffs(B, A1)
    for y in sos_inputs.points(nf - 1, 8, 4):
        x = np.append(y, 1.0)
        want = network_value(B, A1, x)
        assert abs(o.eval(c, y) - want) <= 1e-12 * max(1.0, abs(want))


@pytest.mark.parametrize("nf,m,k", [(3, 3, 4), (4, 6, 5), (5, 5, 3)])
def test_section_2_identities_for_the_network(nf, m, k):
    o = oracle.Oracle(nf, 4)               # homogeneous table: the form itself
    B, A1 = net(nf, m, k, 5)
    c = o.coeffs(o.layer_expand(B, A1))
    want = quartic_identities(o.E2d, lambda i, j: network_second_derivative(B, A1, i, j))
    quartic = o.E2d.sum(axis=1) == 4
    np.testing.assert_allclose(c[quartic], want[quartic], rtol=1e-12, atol=1e-12)
    assert np.all(c[~quartic] == 0.0)


def test_change_of_basis_of_the_first_layer():
    nf, m, k = 5, 7, 6
    o = oracle.Oracle(nf - 1, 4)
    B, A1 = net(nf, m, k, 7)
    G = sos_inputs.normal_matrix(m, m, 8) + 3.0 * np.eye(m)
    B2 = B @ np.kron(np.eye(nf), np.linalg.inv(G))
    np.testing.assert_allclose(o.layer_coeffs(B2, G @ A1), o.layer_coeffs(B, A1), rtol=1e-10, atol=1e-10)


def test_layer_gradients_match_exact_differences():
    nf, m, k = 4, 5, 3
    o = oracle.Oracle(nf - 1, 4)
    B, A1 = net(nf, m, k, 9)
    p = o.coeffs(sos_inputs.normal_matrix(o.N, 2, 10))
    _, gB, gA1, _ = o.layer_loss_grad(B, A1, p)
    g = np.random.default_rng(11)
    for _ in range(6):
        e = (int(g.integers(k)), int(g.integers(nf * m)))
        d = richardson_derivative(lambda X: o.layer_loss_grad(X, A1, p)[0], B, e, 1e-3)
        assert abs(d - gB[e]) <= 1e-8 * np.abs(gB).max()
        e = (int(g.integers(m)), int(g.integers(nf)))
        d = richardson_derivative(lambda X: o.layer_loss_grad(B, X, p)[0], A1, e, 1e-3)
        assert abs(d - gA1[e]) <= 1e-8 * np.abs(gA1).max()


# -- planted mistakes ------------------------------------------------------------------

def _expand_planted(Ed, nf, B, A1, kind):
    m = A1.shape[0]
    rows = oracle.form_rows(Ed, nf)
    out = np.zeros((len(Ed), B.shape[0]))
    for k in range(B.shape[0]):
        Mk = B[k].reshape(m, nf).T if kind == "transposed_block" else B[k].reshape(nf, m)
        P = Mk @ A1
        for i in range(nf):
            for j in range(i, nf):
                if i == j:
                    v = 2.0 * P[i, i] if kind == "doubled_diagonal" else P[i, i]
                else:
                    v = P[i, j] if kind == "one_sided" else P[i, j] + P[j, i]
                out[rows[i, j], k] = v
    return out


@pytest.mark.parametrize("kind", ["transposed_block", "one_sided", "doubled_diagonal"])
def test_planted_expansion_mistakes_are_caught(kind):
    nf, m, k = 4, 4, 3
    o = oracle.Oracle(nf - 1, 4)
    B, A1 = net(nf, m, k, 12)
    c = o.coeffs(_expand_planted(o.Ed, nf, B, A1, kind))
    worst = 0.0
    for y in sos_inputs.points(nf - 1, 8, 13):
        want = network_value(B, A1, np.append(y, 1.0))
        worst = max(worst, abs(o.eval(c, y) - want) / max(1.0, abs(want)))
    assert worst > 1e-6


def test_planted_chain_rule_mistake_is_caught():
    """dL/dA1 with M_k in place of M_k^T fails the difference check."""
    nf, m, k = 4, 4, 3
    o = oracle.Oracle(nf - 1, 4)
    B, A1 = net(nf, m, k, 14)
    p = o.coeffs(sos_inputs.normal_matrix(o.N, 2, 15))
    _, g_hat, _ = o.loss_grad(o.layer_expand(B, A1), p)
    rows = oracle.form_rows(o.Ed, nf)
    wrong = sum(B[kk].reshape(nf, m) @ g_hat[rows, kk] for kk in range(k))   # should be M_k^T S_k
    e = (1, 2)
    d = richardson_derivative(lambda X: o.layer_loss_grad(B, X, p)[0], A1, e, 1e-3)
    assert abs(d - wrong[e]) > 1e-6 * np.abs(wrong).max()
