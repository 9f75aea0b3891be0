"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module draws random numbers and nothing else: it holds none of the
method's arithmetic (no polynomial products, no losses, no gradients), so that
the CUDA library and the CPU oracle can both consume the same arrays without
sharing any code.  A target p that is a sum of squares is produced by whoever
needs it, by applying that side's own c(.) to the generating matrix returned
here.

Workload recipes (all float64, numpy ``default_rng(seed)``):

* tiny FP64 problem: n=3, 2d=4, r=N=10; target generator G has 5 columns
  of i.i.d. N(0, 1); A0 ~ N(0, 0.1^2).
* batch FP32 problems: n=6, 2d=8, r=N=210; 64 instances with seeds 0..63,
  target generator 50 columns of N(0, 1); A0 ~ N(0, 0.1^2).
* precision problem: n=10, 2d=10, r=N=3003; generator 1000 columns of N(0, 1).
* large problem: n=20, 2d=8, r=N=10626; generator 2000 columns of
  N(0, 1)/sqrt(N); A0 ~ N(0, 0.1^2).
* medium problem (profiling stand-in for the large one): n=18, 2d=8,
  r=N=7315, same recipe.
* serving stream: Poisson arrivals, n uniform in {3..8}, 2d uniform in
  {4, 6, 8}, r=N; even ids are sums of floor(N/2) random squares, odd ids are
  the same minus (p(x0) + 1) at x0 ~ N(0, I_n).
* the paper's quartic forms (Sec. 3.1): p = m_2 Q m_2^T with Q = B B^T and B
  uniform in [-1, 1], i.e. a sum of squares whose generator is B.
"""
from __future__ import annotations

from dataclasses import dataclass
from math import comb

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def sizes(n: int, two_d: int):
    """(N, M): monomials of degree <= d and of degree <= 2d in n variables."""
    d = two_d // 2
    return comb(n + d, d), comb(n + two_d, two_d)


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    two_d: int
    r: int            # columns of A (number of squares); 0 means r = N
    squares: int      # columns of the target's generator
    gen_scale: str    # "unit" -> N(0,1); "inv_sqrt_n" -> N(0,1)/sqrt(N)
    init_sigma: float = 0.1

    @property
    def N(self) -> int:
        return sizes(self.n, self.two_d)[0]

    @property
    def M(self) -> int:
        return sizes(self.n, self.two_d)[1]

    @property
    def cols(self) -> int:
        return self.r if self.r else self.N


TINY = Workload("tiny_fp64_n3_2d4", 3, 4, 0, 5, "unit")
BATCH = Workload("batch_fp32_n6_2d8", 6, 8, 0, 50, "unit")
PRECISION = Workload("precision_n10_2d10", 10, 10, 0, 1000, "unit")
LARGE = Workload("large_n20_2d8", 20, 8, 0, 2000, "inv_sqrt_n")
# a smaller case of the same kernels whose operands still exceed L2 (profiling)
MEDIUM = Workload("medium_n18_2d8", 18, 8, 0, 2000, "inv_sqrt_n")
WORKLOADS = {w.name: w for w in (TINY, BATCH, PRECISION, LARGE, MEDIUM)}


def generator(w: Workload, seed: int) -> np.ndarray:
    """N x squares matrix whose columns generate the SOS target (float64)."""
    g = rng(seed).standard_normal((w.N, w.squares))
    if w.gen_scale == "inv_sqrt_n":
        g /= np.sqrt(w.N)
    return g


def init_A(w: Workload, seed: int) -> np.ndarray:
    """N x r starting point, i.i.d. N(0, sigma^2) (float64)."""
    return rng(seed + 1_000_003).normal(0.0, w.init_sigma, size=(w.N, w.cols))


def normal_matrix(rows: int, cols: int, seed: int, sigma: float = 1.0) -> np.ndarray:
    return rng(seed).normal(0.0, sigma, size=(rows, cols))


def uniform_matrix(rows: int, cols: int, seed: int, lo: float = -1.0, hi: float = 1.0):
    return rng(seed).uniform(lo, hi, size=(rows, cols))


def points(n: int, count: int, seed: int, lo: float = -1.0, hi: float = 1.0):
    """count x n evaluation points, uniform in [lo, hi]^n."""
    return rng(seed).uniform(lo, hi, size=(count, n))


def orthogonal(r: int, seed: int) -> np.ndarray:
    """A Haar-ish random orthogonal r x r matrix (QR of a Gaussian)."""
    q, rr = np.linalg.qr(rng(seed).standard_normal((r, r)))
    return q * np.sign(np.diag(rr))


# -- serving stream ------------------------------------------------------

@dataclass(frozen=True)
class Request:
    rid: int
    arrival_s: float
    n: int
    two_d: int
    sos: bool          # even ids are SOS by construction, odd ids are not

    @property
    def N(self) -> int:
        return sizes(self.n, self.two_d)[0]

    @property
    def M(self) -> int:
        return sizes(self.n, self.two_d)[1]


def request_stream(count: int, rate_per_s: float, seed: int = 0,
                   n_range=(3, 8), two_d_choices=(4, 6, 8)):
    """Poisson arrivals (exponential gaps) with uniform (n, 2d)."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate_per_s, size=count)
    arrivals = np.cumsum(gaps) - gaps[0]
    ns = g.integers(n_range[0], n_range[1] + 1, size=count)
    ds = g.choice(np.asarray(two_d_choices), size=count)
    return [Request(i, float(arrivals[i]), int(ns[i]), int(ds[i]), i % 2 == 0)
            for i in range(count)]


def request_generator(req: Request) -> np.ndarray:
    """N x floor(N/2) generator of the request's SOS part, N(0, 1)."""
    N = req.N
    return rng(req.rid).standard_normal((N, max(1, N // 2)))


def request_points(req: Request, count: int = 64) -> np.ndarray:
    """Candidate points x0 ~ N(0, I_n) at which an odd request is made negative
    (the first admissible one is used)."""
    return rng(10_000_019 + req.rid).standard_normal((count, req.n))


def request_init(req: Request, sigma: float = 0.1) -> np.ndarray:
    return rng(20_000_003 + req.rid).normal(0.0, sigma, size=(req.N, req.N))


# -- the paper's own workloads (Sec. 3) ----------------------------------

def paper_quartic_generator(n_form: int, seed: int) -> np.ndarray:
    """B uniform in [-1, 1] with one row per degree-2 monomial of a quartic form
    in n_form variables and as many columns, so Q = B B^T (Sec. 3.1)."""
    l = comb(n_form + 1, 2)
    return rng(seed).uniform(-1.0, 1.0, size=(l, l))


def fine_structure_noise(count: int, seed: int) -> np.ndarray:
    """Coefficients uniform in [-0.01, 0.01] (Sec. 3.4)."""
    return rng(seed).uniform(-0.01, 0.01, size=count)
