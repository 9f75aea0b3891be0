"""CPU oracle for the over-parameterised sum-of-squares objective.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never imports it, and it imports nothing from
the product: it has its own C source (``sos_oracle.c``), compiled here with
gcc, and shares no tables, constants or helpers with the CUDA path.

Paper: Keren, Osadchy, Poranne, arXiv 2410.19844.
  * monomial vector m_d and its order ............ Sec. 1.1, Eq. 1 (n = d = 2 example)
  * c(A) = coefficients of m_d A A^T m_d^T ........ Eq. 1 with B = P P^T, Eq. 2
  * loss = 1/2 ||c(A) - p||^2 ..................... Eq. 2 (1/2 is our scale)
  * gradient by the chain rule .................... derived from Eq. 2
  * Adam, random init, best-error tracking ........ Sec. 3 (experimental set-up)
  * the network ||B Z A1 x||^2 with its first layer  Sec. 2, Eq. 4, Sec. 2.1
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from math import comb

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sos_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    lib.oracle_count_monomials.argtypes = [i32, i32]
    lib.oracle_count_monomials.restype = i64
    lib.oracle_monomials.argtypes = [i32, i32, vp, i64]
    lib.oracle_monomials.restype = i64
    lib.oracle_rank.argtypes = [i32, vp, i64, vp]
    lib.oracle_rank.restype = i64
    lib.oracle_product_table.argtypes = [i32, vp, i64, vp, i64, vp]
    lib.oracle_product_table.restype = i32
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = i32
    lib.oracle_coeffs.argtypes = [i64, i64, i64, vp, vp, vp]
    lib.oracle_coeffs.restype = i32
    lib.oracle_residual.argtypes = [i64, vp, vp, vp]
    lib.oracle_residual.restype = dbl
    lib.oracle_grad.argtypes = [i64, i64, vp, vp, vp, vp]
    lib.oracle_grad.restype = i32
    lib.oracle_coeff_at.argtypes = [i32, vp, i64, i64, vp, vp]
    lib.oracle_coeff_at.restype = dbl
    lib.oracle_grad_row.argtypes = [i32, vp, i64, vp, i64, i64, vp, vp, i64, vp]
    lib.oracle_grad_row.restype = i32
    lib.oracle_resid_row.argtypes = [i32, vp, i64, vp, i64, i64, vp, vp, i64, vp]
    lib.oracle_resid_row.restype = i32
    lib.oracle_gd_step.argtypes = [i64, dbl, vp, vp]
    lib.oracle_gd_step.restype = None
    lib.oracle_adam_step.argtypes = [i64, i64, dbl, dbl, dbl, dbl, vp, vp, vp, vp]
    lib.oracle_adam_step.restype = None
    lib.oracle_eval.argtypes = [i32, vp, i64, vp, vp]
    lib.oracle_eval.restype = dbl
    _lib = lib
    return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def num_threads() -> int:
    """OpenMP threads the oracle's heavy loops use."""
    return int(_load().oracle_num_threads())


def count_monomials(n: int, deg: int) -> int:
    """Number of monomials of degree <= deg in n variables, by enumeration."""
    return int(_load().oracle_count_monomials(n, deg))


def monomials(n: int, deg: int) -> np.ndarray:
    """All exponent tuples of degree <= deg, in the paper's order (Sec. 1.1)."""
    lib = _load()
    rows = lib.oracle_count_monomials(n, deg)
    out = np.zeros((rows, n), dtype=np.uint8)
    got = lib.oracle_monomials(n, deg, _ptr(out), rows)
    assert got == rows
    return out


class Oracle:
    """The objective of Eq. 2 for polynomials of degree <= 2d in n variables.

    ``N`` rows of A are the monomials of degree <= d, ``M`` entries of c and p
    are the monomials of degree <= 2d, both in the paper's order.
    """

    def __init__(self, n: int, two_d: int):
        if two_d < 2 or two_d % 2:
            raise ValueError("two_d must be even and >= 2")
        self.n, self.two_d, self.d = n, two_d, two_d // 2
        self.Ed = monomials(n, self.d)
        self.E2d = monomials(n, two_d)
        self.N, self.M = len(self.Ed), len(self.E2d)
        self._prod = None

    # -- tables -------------------------------------------------------
    def rank(self, mono, table: str = "2d") -> int:
        E = self.E2d if table == "2d" else self.Ed
        m = np.ascontiguousarray(np.asarray(mono, dtype=np.uint8))
        return int(_load().oracle_rank(self.n, _ptr(E), len(E), _ptr(m)))

    @property
    def prod(self) -> np.ndarray:
        """prod[a, b] = position of x^a x^b among the monomials of degree <= 2d."""
        if self._prod is None:
            p = np.empty((self.N, self.N), dtype=np.int32)
            rc = _load().oracle_product_table(self.n, _ptr(self.Ed), self.N,
                                              _ptr(self.E2d), self.M, _ptr(p))
            assert rc == 0
            self._prod = p
        return self._prod

    # -- objective ----------------------------------------------------
    def coeffs(self, A) -> np.ndarray:
        """c(A): coefficients of sum_k q_k^2 (Eq. 1 with B = A A^T)."""
        A = np.ascontiguousarray(A, dtype=np.float64)
        assert A.ndim == 2 and A.shape[0] == self.N
        c = np.empty(self.M, dtype=np.float64)
        rc = _load().oracle_coeffs(self.N, self.M, A.shape[1], _ptr(self.prod),
                                   _ptr(A), _ptr(c))
        assert rc == 0
        return c

    def residual(self, c, p):
        """(loss, resid) with resid = c - p and loss = 1/2 ||resid||^2 (Eq. 2)."""
        c = np.ascontiguousarray(c, dtype=np.float64)
        p = np.ascontiguousarray(p, dtype=np.float64)
        resid = np.empty(self.M, dtype=np.float64)
        loss = _load().oracle_residual(self.M, _ptr(c), _ptr(p), _ptr(resid))
        return float(loss), resid

    def grad_from_resid(self, A, resid) -> np.ndarray:
        A = np.ascontiguousarray(A, dtype=np.float64)
        resid = np.ascontiguousarray(resid, dtype=np.float64)
        g = np.empty_like(A)
        _load().oracle_grad(self.N, A.shape[1], _ptr(self.prod), _ptr(A),
                            _ptr(resid), _ptr(g))
        return g

    def loss_grad(self, A, p):
        """(loss, grad, c) at A for target p."""
        c = self.coeffs(A)
        loss, resid = self.residual(c, p)
        return loss, self.grad_from_resid(A, resid), c

    def loss(self, A, p) -> float:
        return self.residual(self.coeffs(A), p)[0]

    # -- one-at-a-time samples (for problems too large for prod) -------
    def coeff_at(self, A, g: int) -> float:
        A = np.ascontiguousarray(A, dtype=np.float64)
        gamma = np.ascontiguousarray(self.E2d[g])
        return float(_load().oracle_coeff_at(self.n, _ptr(self.Ed), self.N, A.shape[1],
                                             _ptr(A), _ptr(gamma)))

    def grad_row(self, A, p, a: int) -> np.ndarray:
        A = np.ascontiguousarray(A, dtype=np.float64)
        p = np.ascontiguousarray(p, dtype=np.float64)
        row = np.empty(A.shape[1], dtype=np.float64)
        rc = _load().oracle_grad_row(self.n, _ptr(self.Ed), self.N, _ptr(self.E2d),
                                     self.M, A.shape[1], _ptr(A), _ptr(p), a, _ptr(row))
        assert rc == 0
        return row

    def resid_row(self, A, p, a: int) -> np.ndarray:
        """h_b = (c(A) - p)_{a+b} for every b: row a of the matrix whose
        contraction with A gives half the gradient."""
        A = np.ascontiguousarray(A, dtype=np.float64)
        p = np.ascontiguousarray(p, dtype=np.float64)
        h = np.empty(self.N, dtype=np.float64)
        rc = _load().oracle_resid_row(self.n, _ptr(self.Ed), self.N, _ptr(self.E2d),
                                      self.M, A.shape[1], _ptr(A), _ptr(p), a, _ptr(h))
        assert rc == 0
        return h

    # -- optimiser (Sec. 3: "basic ADAM") ------------------------------
    @staticmethod
    def gd_step(A, grad, lr: float) -> None:
        assert A.dtype == np.float64 and A.flags.c_contiguous
        g = np.ascontiguousarray(grad, dtype=np.float64)
        _load().oracle_gd_step(A.size, lr, _ptr(g), _ptr(A))

    @staticmethod
    def adam_step(A, m, v, grad, t: int, lr: float, b1: float = 0.9,
                  b2: float = 0.999, eps: float = 1e-8) -> None:
        for x in (A, m, v):
            assert x.dtype == np.float64 and x.flags.c_contiguous
        g = np.ascontiguousarray(grad, dtype=np.float64)
        _load().oracle_adam_step(A.size, t, lr, b1, b2, eps, _ptr(g), _ptr(A),
                                 _ptr(m), _ptr(v))

    # -- evaluation ---------------------------------------------------
    def eval(self, c, x) -> float:
        """sum_g c_g x^g over the monomials of degree <= 2d."""
        c = np.ascontiguousarray(c, dtype=np.float64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        return float(_load().oracle_eval(self.n, _ptr(self.E2d), self.M, _ptr(c), _ptr(x)))

    def eval_d(self, q, x) -> float:
        """sum_a q_a x^a over the monomials of degree <= d."""
        q = np.ascontiguousarray(q, dtype=np.float64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        return float(_load().oracle_eval(self.n, _ptr(self.Ed), self.N, _ptr(q), _ptr(x)))

    # -- the network with its first layer (Sec. 2, Eq. 4) -----------------
    def layer_expand(self, B, A1) -> np.ndarray:
        """A_hat of the network on this table (dehomogenised when the table
        has n = nf - 1 variables, homogeneous when it has nf)."""
        nf = B.shape[1] // A1.shape[0]
        return layer_expand(self.Ed, nf, B, A1)

    def layer_coeffs(self, B, A1) -> np.ndarray:
        return self.coeffs(self.layer_expand(B, A1))

    def layer_loss_grad(self, B, A1, p):
        """(loss, grad_B, grad_A1, c) of 1/2 ||c(A_hat(B, A1)) - p||^2: the
        gradient with respect to A_hat, then the chain rule through
        P_k = M_k A1 and the symmetrisation of P_k."""
        B = np.asarray(B, dtype=np.float64)
        A1 = np.asarray(A1, dtype=np.float64)
        m = A1.shape[0]
        nf = B.shape[1] // m
        loss, g_hat, c = self.loss_grad(self.layer_expand(B, A1), p)
        rows = form_rows(self.Ed, nf)
        gB = np.zeros_like(B)
        gA1 = np.zeros_like(A1)
        for k in range(B.shape[0]):
            S = g_hat[rows, k]                    # dL/dP_k, symmetric
            Mk = B[k].reshape(nf, m)
            gB[k] = (S @ A1.T).reshape(-1)
            gA1 += Mk.T @ S
        return loss, gB, gA1, c

    def certify(self, c, p) -> float:
        """Relative residual ||c - p||_2 / ||p||_2 in double precision."""
        c = np.asarray(c, dtype=np.float64)
        p = np.asarray(p, dtype=np.float64)
        return float(np.sqrt(2.0 * self.residual(c, p)[0]) / np.linalg.norm(p))


def form_rows(Ed, nf: int) -> np.ndarray:
    """rows[i, j] = row of the monomial x_i x_j (0 <= i, j < nf) in Ed.  Ed
    with nf columns holds the form's monomials themselves; with nf - 1 columns
    the form is dehomogenised: x_nf = 1, its exponent is 2 - |e|."""
    Ed = np.asarray(Ed)
    rows = np.full((nf, nf), -1, dtype=np.int64)
    for a, e in enumerate(Ed):
        e = [int(v) for v in e]
        if len(e) == nf - 1:
            e = e + [2 - sum(e)]
        elif sum(e) != 2:
            continue
        i, j = [v for v in range(nf) for _ in range(e[v])]
        rows[i, j] = rows[j, i] = a
    assert (rows >= 0).all()
    return rows


def layer_expand(Ed, nf: int, B, A1) -> np.ndarray:
    """Coefficient matrix A_hat (rows of Ed x k) of the network's form
    ||B Z A1 x||^2 (Sec. 2, Eq. 4): Z A1 x stacks x_i (A1 x) for i = 1..nf, so
    output k is x^T M_k A1 x with M_k = B[k] read as nf x m.  With P_k = M_k A1,
    the coefficient of x_i x_j in output k is P_k[i][j] + P_k[j][i] (i < j) and
    P_k[i][i] (i = j).  Rows of Ed that are no degree-2 form monomial stay 0."""
    B = np.asarray(B, dtype=np.float64)
    A1 = np.asarray(A1, dtype=np.float64)
    m = A1.shape[0]
    assert A1.shape[1] == nf and B.shape[1] == nf * m
    rows = form_rows(Ed, nf)
    iu, ju = np.triu_indices(nf)
    out = np.zeros((len(Ed), B.shape[0]))
    for k in range(B.shape[0]):
        P = B[k].reshape(nf, m) @ A1
        sym = P + P.T
        vals = np.where(iu == ju, np.diag(P)[iu], sym[iu, ju])
        out[rows[iu, ju], k] = vals
    return out


def sizes(n: int, two_d: int):
    """(N, M) from the closed forms C(n+d, d) and C(n+2d, 2d)."""
    d = two_d // 2
    return comb(n + d, d), comb(n + two_d, two_d)
