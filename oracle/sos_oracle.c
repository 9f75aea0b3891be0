/*
 * sos_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, double-precision CPU statement of the over-parameterised
 * sum-of-squares objective of Keren, Osadchy and Poranne, "A practical, fast
 * method for solving sum-of-squares problems for very large polynomials"
 * (arXiv 2410.19844).  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  It shares no code,
 * header, table or constant with the CUDA library: it enumerates and sorts
 * its own monomials, looks ranks up by binary search, and multiplies
 * polynomials monomial by monomial.
 *
 * What it computes (paper sections in brackets):
 *   - m_d: every exponent tuple of total degree <= d, in the order the paper
 *     prints for n = d = 2, (x1^2, x1x2, x2^2, x1, x2, 1)  [Sec. 1.1, Eq. 1]:
 *     higher total degree first, then lexicographically larger tuple first.
 *   - c(A): coefficients of m_d (A A^T) m_d^T = sum_k q_k^2, where column k of
 *     A holds the coefficients of q_k over m_d  [Eq. 1 with B = P P^T, Eq. 2].
 *   - loss = 1/2 ||c(A) - p||^2 over the plain coefficient vectors  [Eq. 2;
 *     the factor 1/2 is this library's scale convention].
 *   - gradient by the chain rule: d c_g / d A_{a,k} = 2 A_{g-a,k}, hence
 *     grad_{a,k} = 2 sum_b (c-p)_{a+b} A_{b,k}  [derived from Eq. 2].
 *   - one step of Adam with bias correction (the paper's optimiser, Sec. 3)
 *     and of plain gradient descent.
 *   - evaluation sum_g c_g x^g at a point.
 *
 * Everything is double precision; the heavy loops use OpenMP over rows.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Monomial enumeration and ordering                                   */
/* ------------------------------------------------------------------ */

static int total_degree(const uint8_t* e, int n) {
    int s = 0;
    for (int i = 0; i < n; ++i) s += e[i];
    return s;
}

/* Paper order (Sec. 1.1): a before b when deg(a) > deg(b); for equal degree,
 * a before b when a is lexicographically larger (x1 compared first).
 * Returns <0 when a comes first, >0 when b comes first, 0 when equal. */
static int paper_order(const uint8_t* a, const uint8_t* b, int n) {
    int da = total_degree(a, n), db = total_degree(b, n);
    if (da != db) return da > db ? -1 : 1;
    for (int i = 0; i < n; ++i)
        if (a[i] != b[i]) return a[i] > b[i] ? -1 : 1;
    return 0;
}

static int cmp_with_n(const void* a, const void* b, void* n_ptr) {
    return paper_order((const uint8_t*)a, (const uint8_t*)b, *(int*)n_ptr);
}

/* Recursively writes every tuple e with e_0 + ... + e_{n-1} <= deg. */
static void enumerate_rec(int n, int i, int remaining, uint8_t* cur,
                          uint8_t* out, int64_t* count) {
    if (i == n) {
        if (out) memcpy(out + (*count) * n, cur, (size_t)n);
        (*count)++;
        return;
    }
    for (int e = 0; e <= remaining; ++e) {
        cur[i] = (uint8_t)e;
        enumerate_rec(n, i + 1, remaining - e, cur, out, count);
    }
}

int64_t oracle_count_monomials(int n, int deg) {
    if (n < 1 || deg < 0 || n > 255) return -1;
    uint8_t cur[256];
    int64_t count = 0;
    enumerate_rec(n, 0, deg, cur, NULL, &count);
    return count;
}

/* Fills out (rows x n, row-major) with all monomials of degree <= deg in the
 * paper's order.  Returns the number of rows, or -1 when cap is too small. */
int64_t oracle_monomials(int n, int deg, uint8_t* out, int64_t cap) {
    int64_t rows = oracle_count_monomials(n, deg);
    if (rows < 0 || rows > cap) return -1;
    uint8_t cur[256];
    int64_t count = 0;
    enumerate_rec(n, 0, deg, cur, out, &count);
    qsort_r(out, (size_t)rows, (size_t)n, cmp_with_n, &n);
    return rows;
}

/* Binary search of mono in a table sorted in the paper's order.
 * Returns its row, or -1 when absent. */
int64_t oracle_rank(int n, const uint8_t* table, int64_t rows, const uint8_t* mono) {
    int64_t lo = 0, hi = rows - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int c = paper_order(table + mid * n, mono, n);
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* prod[a*N + b] = row of (E_d[a] + E_d[b]) in E_2d: the position of the
 * product monomial x^a x^b in the coefficient vector of degree <= 2d. */
int oracle_product_table(int n, const uint8_t* Ed, int64_t N,
                         const uint8_t* E2d, int64_t M, int32_t* prod) {
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 16) reduction(+:bad)
    for (int64_t a = 0; a < N; ++a) {
        uint8_t sum[256];
        for (int64_t b = 0; b < N; ++b) {
            for (int i = 0; i < n; ++i) sum[i] = (uint8_t)(Ed[a * n + i] + Ed[b * n + i]);
            int64_t g = oracle_rank(n, E2d, M, sum);
            if (g < 0) bad++;
            prod[a * N + b] = (int32_t)g;
        }
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Objective, gradient, optimiser                                      */
/* ------------------------------------------------------------------ */

static int nthreads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int oracle_num_threads(void) { return nthreads(); }

/* c = coefficients of sum_k q_k^2 (Eq. 1 with B = A A^T): for every ordered
 * pair of monomials (a, b), B_ab = sum_k A_ak A_bk is added to the
 * coefficient of x^a x^b.  A is N x r row-major; c has M entries. */
int oracle_coeffs(int64_t N, int64_t M, int64_t r, const int32_t* prod,
                  const double* A, double* c) {
    memset(c, 0, (size_t)M * sizeof(double));
    int T = nthreads();
    double* part = (double*)calloc((size_t)T * (size_t)M, sizeof(double));
    if (!part) return -1;
    #pragma omp parallel
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double* mine = part + (size_t)t * (size_t)M;
        #pragma omp for schedule(static)
        for (int64_t a = 0; a < N; ++a) {
            const double* Aa = A + a * r;
            for (int64_t b = 0; b < N; ++b) {
                const double* Ab = A + b * r;
                double B = 0.0;
                for (int64_t k = 0; k < r; ++k) B += Aa[k] * Ab[k];
                mine[prod[a * N + b]] += B;
            }
        }
    }
    for (int t = 0; t < T; ++t)
        for (int64_t g = 0; g < M; ++g) c[g] += part[(size_t)t * (size_t)M + g];
    free(part);
    return 0;
}

/* resid = c - p; returns loss = 1/2 ||c - p||^2 (Eq. 2, scaled by 1/2). */
double oracle_residual(int64_t M, const double* c, const double* p, double* resid) {
    double s = 0.0;
    for (int64_t g = 0; g < M; ++g) {
        double e = c[g] - p[g];
        if (resid) resid[g] = e;
        s += e * e;
    }
    return 0.5 * s;
}

/* Chain rule: grad_{a,k} = sum_g resid_g * d c_g / d A_{a,k}
 *                         = 2 * sum_b resid[prod(a, b)] * A_{b,k}. */
int oracle_grad(int64_t N, int64_t r, const int32_t* prod, const double* A,
                const double* resid, double* grad) {
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t a = 0; a < N; ++a) {
        double* ga = grad + a * r;
        for (int64_t k = 0; k < r; ++k) ga[k] = 0.0;
        for (int64_t b = 0; b < N; ++b) {
            double h = 2.0 * resid[prod[a * N + b]];
            const double* Ab = A + b * r;
            for (int64_t k = 0; k < r; ++k) ga[k] += h * Ab[k];
        }
    }
    return 0;
}

/* One coefficient c_g computed on its own: the sum over every ordered pair
 * (a, b) with x^a x^b = x^g of sum_k A_ak A_bk.  Pairs are found by walking
 * the monomials a of degree <= d that divide x^g and looking up g - a. */
double oracle_coeff_at(int n, const uint8_t* Ed, int64_t N, int64_t r,
                       const double* A, const uint8_t* gamma) {
    double c = 0.0;
    uint8_t rest[256];
    for (int64_t a = 0; a < N; ++a) {
        const uint8_t* ea = Ed + a * n;
        int ok = 1;
        for (int i = 0; i < n; ++i) {
            if (ea[i] > gamma[i]) { ok = 0; break; }
            rest[i] = (uint8_t)(gamma[i] - ea[i]);
        }
        if (!ok) continue;
        int64_t b = oracle_rank(n, Ed, N, rest);
        if (b < 0) continue;
        const double* Aa = A + a * r;
        const double* Ab = A + b * r;
        double B = 0.0;
        for (int64_t k = 0; k < r; ++k) B += Aa[k] * Ab[k];
        c += B;
    }
    return c;
}

/* Row a of the residual Hankel-like matrix, computed on its own (for samples
 * of problems too large for the full product table):  h_b = (c - p)_{a+b}
 * for every degree-<=d monomial b, each c_{a+b} from oracle_coeff_at. */
int oracle_resid_row(int n, const uint8_t* Ed, int64_t N, const uint8_t* E2d, int64_t M,
                     int64_t r, const double* A, const double* p, int64_t a, double* h) {
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 8) reduction(+:bad)
    for (int64_t b = 0; b < N; ++b) {
        uint8_t sum[256];
        for (int i = 0; i < n; ++i) sum[i] = (uint8_t)(Ed[a * n + i] + Ed[b * n + i]);
        int64_t g = oracle_rank(n, E2d, M, sum);
        if (g < 0) { bad++; h[b] = 0.0; continue; }
        h[b] = oracle_coeff_at(n, Ed, N, r, A, sum) - p[g];
    }
    return bad ? -1 : 0;
}

/* One row a of the gradient (derived from Eq. 2):
 *   grad_{a,k} = 2 sum_b (c - p)_{a+b} A_{b,k}. */
int oracle_grad_row(int n, const uint8_t* Ed, int64_t N, const uint8_t* E2d, int64_t M,
                    int64_t r, const double* A, const double* p, int64_t a, double* row) {
    double* h = (double*)malloc((size_t)N * sizeof(double));
    if (!h) return -1;
    int rc = oracle_resid_row(n, Ed, N, E2d, M, r, A, p, a, h);
    for (int64_t k = 0; k < r; ++k) row[k] = 0.0;
    for (int64_t b = 0; b < N; ++b) {
        const double* Ab = A + b * r;
        for (int64_t k = 0; k < r; ++k) row[k] += 2.0 * h[b] * Ab[k];
    }
    free(h);
    return rc;
}

/* Plain gradient descent: A <- A - lr * grad. */
void oracle_gd_step(int64_t count, double lr, const double* grad, double* A) {
    for (int64_t i = 0; i < count; ++i) A[i] -= lr * grad[i];
}

/* Adam (Kingma and Ba), step number t >= 1, with bias correction:
 *   m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2
 *   A <- A - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
void oracle_adam_step(int64_t count, int64_t t, double lr, double b1, double b2,
                      double eps, const double* grad, double* A, double* m, double* v) {
    double c1 = 1.0 - pow(b1, (double)t);
    double c2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = 0; i < count; ++i) {
        double g = grad[i];
        m[i] = b1 * m[i] + (1.0 - b1) * g;
        v[i] = b2 * v[i] + (1.0 - b2) * g * g;
        double mhat = m[i] / c1;
        double vhat = v[i] / c2;
        A[i] -= lr * mhat / (sqrt(vhat) + eps);
    }
}

/* sum_g c_g x^g for the monomials of E (rows x n). */
double oracle_eval(int n, const uint8_t* E, int64_t rows, const double* c, const double* x) {
    double s = 0.0;
    for (int64_t g = 0; g < rows; ++g) {
        double term = c[g];
        for (int i = 0; i < n; ++i)
            for (int e = 0; e < E[g * n + i]; ++e) term *= x[i];
        s += term;
    }
    return s;
}
