"""Independent checks that pin the CPU oracle to the paper and to mathematics.

Each check takes the function under test as an argument, so the same check
runs on the real oracle (must pass) and on an oracle with a planted mistake
(must fail).  None of these helpers calls the oracle's own rank lookup or its
product table: polynomials are evaluated here with numpy powers.
"""
from __future__ import annotations

import os
from math import factorial

import numpy as np


# -- fixtures ---------------------------------------------------------------

def load_closed_forms(path):
    forms = []
    cur = None
    with open(path) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "form":
                kv = dict(t.split("=") for t in tok[2:])
                cur = {"name": tok[1], "n": int(kv["n"]), "two_d": int(kv["two_d"]),
                       "q": [], "c": {}, "scale": 1.0}
            elif tok[0] == "q":
                cur["q"].append((int(tok[1]), tuple(int(e) for e in tok[2].split(",")),
                                 float(tok[3])))
            elif tok[0] == "c":
                cur["c"][tuple(int(e) for e in tok[1].split(","))] = float(tok[2])
            elif tok[0] == "scale":
                cur["scale"] = float(tok[1])
            elif tok[0] == "end":
                forms.append(cur)
                cur = None
    return forms


def load_rows(path):
    rows = []
    with open(path) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


# -- independent polynomial evaluation -------------------------------------

def monomial_values(E: np.ndarray, x: np.ndarray) -> np.ndarray:
    """x^e for every row e of E (numpy powers, no tables)."""
    return np.prod(np.power(x[None, :], E.astype(np.int64)), axis=1)


def point_eval_error(coeffs_fn, Ed, E2d, A, X) -> float:
    """max over points of |sum_g c_g x^g - sum_k q_k(x)^2| / sum_k q_k(x)^2."""
    c = coeffs_fn(A)
    worst = 0.0
    for x in X:
        q = A.T @ monomial_values(Ed, x)          # q_k(x) for every k
        lhs = float(np.dot(q, q))
        rhs = float(np.dot(c, monomial_values(E2d, x)))
        worst = max(worst, abs(lhs - rhs) / max(abs(lhs), 1e-300))
    return worst


# -- the paper's quartic identities (Sec. 2) --------------------------------

def quartic_identity_coeffs(Ed, E2d, A) -> np.ndarray:
    """Coefficients of the quartic part of sum_k q_k^2 from the five identities
    of Sec. 2, for q_k homogeneous quadratics.  f_{x_i x_j} is the vector
    (over k) of second partial derivatives of q_k; for a quadratic it is the
    x_i x_j coefficient when i != j and twice the x_i^2 coefficient when
    i == j.  Returns a vector over E2d; entries for degree != 4 are 0."""
    n = Ed.shape[1]
    row = {tuple(int(v) for v in e): a for a, e in enumerate(Ed)}

    def f(i, j):
        e = [0] * n
        e[i] += 1
        e[j] += 1
        v = A[row[tuple(e)]]
        return 2.0 * v if i == j else v

    return quartic_identities(E2d, f)


def quartic_identities(E2d, f) -> np.ndarray:
    """The five identities of Sec. 2 for the degree-4 entries of E2d, given
    f(i, j) = the vector of second derivatives of the outputs by x_i, x_j."""
    n = E2d.shape[1]

    def ip(u, w):
        return float(np.dot(u, w))

    out = np.zeros(len(E2d))
    for g, e in enumerate(E2d):
        if int(e.sum()) != 4:
            continue
        vars_ = [i for i in range(n) for _ in range(int(e[i]))]   # with repetition
        powers = sorted((int(p) for p in e if p > 0), reverse=True)
        if powers == [4]:
            i = vars_[0]
            out[g] = 0.25 * ip(f(i, i), f(i, i))
        elif powers == [3, 1]:
            i = [v for v in range(n) if e[v] == 3][0]
            j = [v for v in range(n) if e[v] == 1][0]
            out[g] = ip(f(i, i), f(i, j))
        elif powers == [2, 2]:
            i, j = [v for v in range(n) if e[v] == 2]
            out[g] = ip(f(i, j), f(i, j)) + 0.5 * ip(f(i, i), f(j, j))
        elif powers == [2, 1, 1]:
            i = [v for v in range(n) if e[v] == 2][0]
            j, k = [v for v in range(n) if e[v] == 1]
            out[g] = ip(f(i, i), f(j, k)) + 2.0 * ip(f(i, j), f(i, k))
        elif powers == [1, 1, 1, 1]:
            i, j, k, l = vars_
            out[g] = 2.0 * (ip(f(i, j), f(k, l)) + ip(f(i, k), f(j, l))
                            + ip(f(i, l), f(j, k)))
    return out


def network_second_derivative(B, A1, i, j) -> np.ndarray:
    """f_{x_i x_j} of the network f = B Z A1 x (Sec. 2): B Z_{x_i} A1 x_{x_j} +
    B Z_{x_j} A1 x_{x_i}, where Z_{x_i} keeps only the i-th identity block, so
    each term is the i-th block of columns of B times column j of A1."""
    m = A1.shape[0]
    return B[:, i * m:(i + 1) * m] @ A1[:, j] + B[:, j * m:(j + 1) * m] @ A1[:, i]


def network_value(B, A1, x) -> float:
    """||B Z A1 x||^2 evaluated literally: Z stacks x_i times the m x m identity."""
    m = A1.shape[0]
    Z = np.kron(x[:, None], np.eye(m))          # (nf m) x m, block i = x_i I
    f = B @ (Z @ (A1 @ x))
    return float(np.dot(f, f))


def general_rule_coeff(Ed, A, gamma) -> float:
    """The general rule stated after the identities in Sec. 2: the coefficient
    of x^gamma (degree 4) sums the products of second derivatives of f over
    the ways of splitting the four differentiation variables into two pairs,
    divided by the product of the factorials of the powers in gamma.  For a
    quadratic f, d^4 ||f||^2 / dx_a dx_b dx_c dx_d equals
    2 (<f_ab, f_cd> + <f_ac, f_bd> + <f_ad, f_bc>)."""
    n = Ed.shape[1]
    row = {tuple(int(v) for v in e): a for a, e in enumerate(Ed)}

    def f(i, j):
        e = [0] * n
        e[i] += 1
        e[j] += 1
        v = A[row[tuple(e)]]
        return 2.0 * v if i == j else v

    vars_ = [i for i in range(n) for _ in range(int(gamma[i]))]
    total = 0.0
    # d^4 ||f||^2 / dx_{v0} dx_{v1} dx_{v2} dx_{v3} = 2 * sum over the three
    # pairings {ab|cd} of <f_ab, f_cd> (f is quadratic, so only second
    # derivatives survive); the Taylor coefficient divides by prod(gamma_i!).
    for (a, b), (c, d) in [((0, 1), (2, 3)), ((0, 2), (1, 3)), ((0, 3), (1, 2))]:
        total += 2.0 * float(np.dot(f(vars_[a], vars_[b]), f(vars_[c], vars_[d])))
    denom = 1
    for p in gamma:
        denom *= factorial(int(p))
    return total / denom


# -- gradient ---------------------------------------------------------------

def richardson_derivative(loss_fn, A, entry, h) -> float:
    """(4 D(h/2) - D(h)) / 3 with D the central difference along one entry.
    L(A + tE) is a polynomial of degree 4 in t, so this is exact up to
    rounding: the h^2 terms cancel and there is no h^4 term."""
    E = np.zeros_like(A)
    E[entry] = 1.0

    def D(s):
        return (loss_fn(A + s * E) - loss_fn(A - s * E)) / (2.0 * s)

    return (4.0 * D(h / 2.0) - D(h)) / 3.0


def directional_coeff_derivative(coeffs_fn, A, E) -> np.ndarray:
    """D c[A] . E = (c(A + E) - c(A - E)) / 2, exact because c is quadratic."""
    return 0.5 * (coeffs_fn(A + E) - coeffs_fn(A - E))


def golden_path(name: str) -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
