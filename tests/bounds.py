"""Error bounds shared by the GPU parity tests, each derived from the
arithmetic of the kernel it checks and computed with the oracle.

  * rows_ref: oracle rows of the gradient 2 H(c - p) A and their elementwise
    bounds, for a forward that accumulates with unit roundoff u (2^-23 when
    the tensor core may truncate its FP32 accumulator, 2^-24 on CUDA cores)
    and an adjoint that reads the residual rounded to unit roundoff u_r
    (2^-8 for bf16):
        |dc_g| <= gamma_c |c|_g,   |c|_g = the coefficient at |A|
        |dh_b| <= |dc| + u_r (|h_b| + |dc|)
        |dg_k| <= 2 sum_b |dh_b| |A_bk| + 2 N u sum_b (|h_b| + |dh_b|) |A_bk|
  * coeffs_ref: sampled coefficients c_g and |c|_g, one at a time.
  * slice_scale_bound: SOS_FP64_TC with s slices of b-bit digits -- every
    term A_ak A_bk is off by at most (s + 2) 2^(-b s) 2^(e_a + e_b), e_a the exponent of row
    a's largest entry; summed over the pairs of each coefficient that is the
    coefficient of the matrix whose row a is 2^e_a everywhere.
"""
import numpy as np


def rows_ref(o, A, p, rows, u, u_r, gamma_c):
    """{row a: (oracle gradient row, elementwise bound)} at A for target p."""
    absA = np.abs(A)
    out = {}
    for a in rows:
        h = o.resid_row(A, p, a)
        absc = o.resid_row(absA, np.zeros_like(p), a)          # |c| at the monomials a + b
        dc = gamma_c * absc
        dh = dc + u_r * (np.abs(h) + dc)
        g = 2.0 * (h @ A)
        bound = 2.0 * (dh @ absA) + 2.0 * o.N * u * ((np.abs(h) + dh) @ absA) + 1e-30
        out[a] = (g, bound)
    return out


def coeffs_ref(o, A, idx):
    """(c_g, |c|_g) at the sampled positions idx, each computed on its own."""
    absA = np.abs(A)
    return (np.array([o.coeff_at(A, int(g)) for g in idx]),
            np.array([o.coeff_at(absA, int(g)) for g in idx]))


def row_scales(A):
    """The matrix whose row a is 2^e_a everywhere (e_a from frexp of the row's largest |entry|)."""
    e = np.frexp(np.abs(A).max(axis=1))[1].astype(np.float64)
    return np.repeat(np.exp2(e)[:, None], A.shape[1], axis=1)


def slice_scale_bound(o, A, slices=8, bits=5):
    """(s + 2) 2^(-b s) times the coefficients of row_scales(A): the bound on
    every coefficient of the SOS_FP64_TC forward with s slices of b-bit digits
    (b = 5 in bf16, 4 in E4M3)."""
    return (slices + 2) * 2.0 ** (-bits * slices) * o.coeffs(row_scales(A))
