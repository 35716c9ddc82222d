/*
 * bchol_oracle.c -- the parity oracle for the banded Cholesky library.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, serial FP64 CPU
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Paper: F. Liu, A. Fredriksson, S. Markidis, "Parallel Cholesky
 * Factorization for Banded Matrices using OpenMP Tasks" (arXiv 2305.04635).
 *
 * Storage (Sec. 3 and Sec. 3.1 of the paper keep the standard LAPACK band
 * format): a symmetric positive-definite matrix A of order n with
 * half-bandwidth k is held by its lower band in a column-major array `ab`
 * with leading dimension ldab >= k+1:  A(i,j) = ab[(i-j) + j*ldab] for
 * 0 <= j <= i <= min(n-1, j+k).  The factor L overwrites the same slots.
 * Slots with i-j > k, rows d >= k+1 of the array (when ldab > k+1) and the
 * slots past row n-1 in the last k columns are never read or written.
 *
 * Compiled with -O2 -ffp-contract=off so that no multiply-add is fused: the
 * results do not depend on the compiler's contraction choices.
 *
 * Parity pins (each checked by the CPU test suite, none by re-running this
 * code): the closed form of the [-1,2,-1] factor, numpy's dense LAPACK
 * Cholesky on n <= 64, the exact factor L0 of the generated A = L0 L0^T,
 * dense numpy inverses/solves, central finite differences, and the brute-
 * force evaluation of Eq. (1) against its closed form.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#define BAND(p, ld, d, j) (p)[(size_t)(j) * (size_t)(ld) + (size_t)(d)]

/* L(i,j), i >= j, i - j <= k: the band slot (i-j, j). */
static double lget(const double* ab, int ldab, int i, int j) { return BAND(ab, ldab, i - j, j); }

static int imax(int a, int b) { return a > b ? a : b; }
static int imin(int a, int b) { return a < b ? a : b; }

/*
 * oracle_pbtrf -- A = L L^T in place, by the left-looking band Cholesky of
 * Algorithm 2 (Sec. 3.2, "Performance Model").
 *
 * Row i is formed from rows r..i-1, r = max(0, i-k) (0-based), one entry at a
 * time in increasing column order:
 *     t        = sum_{l=r}^{j-1} L(i,l) L(j,l)        (ascending l)
 *     L(i,j)   = (A(i,j) - t) / L(j,j)                 j < i
 *     L(i,i)   = sqrt(A(i,i) - t)
 * The printed inner loop runs l up to j inclusive; that would read L(i,j)
 * before it is formed (and L(i,i) inside its own square root).  The textbook
 * definition, which the paper's uniqueness statement (Sec. 2.1) fixes, stops
 * at l = j-1; this routine follows that reading.  Eq. (1) keeps the printed
 * bound and is only used to count flops.
 *
 * Non-SPD input (the paper is silent): the LAPACK convention.  The first row
 * i whose pivot A(i,i) - t is not > 0 (NaN included) stops the routine and it
 * returns i+1 (the order of the leading minor that is not positive definite).
 * Returns 0 on success, -1 on an argument error.  k >= n is treated as k = n-1.
 */
int oracle_pbtrf(int n, int k, double* ab, int ldab) {
  if (n < 0 || k < 0 || ldab < k + 1 || (n > 0 && ab == NULL)) return -1;
  if (n == 0) return 0;
  if (k > n - 1) k = n - 1;
  for (int i = 0; i < n; ++i) {
    const int r = imax(0, i - k);
    for (int j = r; j <= i; ++j) {
      double t = 0.0;
      for (int l = r; l < j; ++l) t += lget(ab, ldab, i, l) * lget(ab, ldab, j, l);
      if (i == j) {
        const double d = BAND(ab, ldab, 0, i) - t;
        if (!(d > 0.0)) return i + 1;
        BAND(ab, ldab, 0, i) = sqrt(d);
      } else {
        BAND(ab, ldab, i - j, j) = (BAND(ab, ldab, i - j, j) - t) / lget(ab, ldab, j, j);
      }
    }
  }
  return 0;
}

/*
 * oracle_pbtrs -- X = A^{-1} B with A = L L^T held in `ab` (LAPACK pbtrs
 * semantics, uplo = 'L').  The paper solves nothing itself; its motivation is
 * the linear systems of an interior-point method (Sec. 1, Sec. 2).  B is n x
 * nrhs column-major with leading dimension ldb >= n and is overwritten.
 *     forward:  y_i = (b_i - sum_{l=max(0,i-k)}^{i-1} L(i,l) y_l) / L(i,i),   i ascending
 *     backward: x_i = (y_i - sum_{l=i+1}^{min(n-1,i+k)} L(l,i) x_l) / L(i,i), i descending
 * Sums run in ascending l.  Returns 0, or -1 on an argument error.
 */
int oracle_pbtrs(int n, int k, int nrhs, const double* ab, int ldab, double* b, int ldb) {
  if (n < 0 || k < 0 || nrhs < 0 || ldab < k + 1 || ldb < imax(1, n)) return -1;
  if (n == 0 || nrhs == 0) return 0;
  if (k > n - 1) k = n - 1;
  for (int c = 0; c < nrhs; ++c) {
    double* x = b + (size_t)c * (size_t)ldb;
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int l = imax(0, i - k); l < i; ++l) s += lget(ab, ldab, i, l) * x[l];
      x[i] = (x[i] - s) / lget(ab, ldab, i, i);
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = 0.0;
      for (int l = i + 1; l <= imin(n - 1, i + k); ++l) s += lget(ab, ldab, l, i) * x[l];
      x[i] = (x[i] - s) / lget(ab, ldab, i, i);
    }
  }
  return 0;
}

/* oracle_logdet -- log det A = 2 sum_i log L(i,i) for A = L L^T. */
double oracle_logdet(int n, const double* ab, int ldab) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += log(BAND(ab, ldab, 0, i));
  return 2.0 * s;
}

/*
 * oracle_sbmv -- y = A x for the symmetric band matrix held by its lower band
 * (the definition of the product; A(i,j) = A(j,i)).  nrhs columns, leading
 * dimensions ldx, ldy >= n.  Sums run in ascending j.
 */
int oracle_sbmv(int n, int k, int nrhs, const double* ab, int ldab, const double* x, int ldx,
                double* y, int ldy) {
  if (n < 0 || k < 0 || nrhs < 0 || ldab < k + 1) return -1;
  if (n == 0) return 0;
  if (k > n - 1) k = n - 1;
  for (int c = 0; c < nrhs; ++c) {
    const double* xc = x + (size_t)c * (size_t)ldx;
    double* yc = y + (size_t)c * (size_t)ldy;
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = imax(0, i - k); j <= imin(n - 1, i + k); ++j) {
        const double a = (i >= j) ? BAND(ab, ldab, i - j, j) : BAND(ab, ldab, j - i, i);
        s += a * xc[j];
      }
      yc[i] = s;
    }
  }
  return 0;
}

/*
 * Error-free transformations for the accuracy checks below: Knuth's TwoSum
 * and the FMA form of TwoProduct, combined into the compensated dot product
 * "Dot2" of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26(6), 2005), whose
 * result is as accurate as if computed in twice the working precision.
 * fma() is the C library's correctly rounded fused multiply-add.
 */
static void two_sum(double a, double b, double* s, double* e) {
  const double x = a + b;
  const double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}
static void two_prod(double a, double b, double* p, double* e) {
  const double x = a * b;
  *e = fma(a, b, -x);
  *p = x;
}

/* (A - L L^T)(i,j) for i >= j within the band, by Dot2 over l = max(0,i-k)..j. */
static double llt_residual_entry(int k, const double* a, int lda, const double* l, int ldl, int i, int j) {
  double s = BAND(a, lda, i - j, j), c = 0.0;
  for (int q = imax(0, i - k); q <= j; ++q) {
    double p, ep, t, et;
    two_prod(lget(l, ldl, i, q), lget(l, ldl, j, q), &p, &ep);
    two_sum(s, -p, &t, &et);
    s = t;
    c += et - ep;
  }
  return s + c;
}

/*
 * oracle_backward_error -- ||A - L L^T||_F / ||A||_F over the whole symmetric
 * matrix (each stored off-diagonal entry counts twice).  L L^T has the same
 * half-bandwidth as L, so only band entries can differ from zero.  Each
 * residual entry is a Dot2 sum, so the check is accurate far below 1e-13.
 */
double oracle_backward_error(int n, int k, const double* a, int lda, const double* l, int ldl) {
  if (n <= 0) return 0.0;
  if (k > n - 1) k = n - 1;
  double num = 0.0, den = 0.0;
  for (int j = 0; j < n; ++j) {
    for (int i = j; i <= imin(n - 1, j + k); ++i) {
      const double r = llt_residual_entry(k, a, lda, l, ldl, i, j);
      const double v = BAND(a, lda, i - j, j);
      const double w = (i == j) ? 1.0 : 2.0;
      num += w * r * r;
      den += w * v * v;
    }
  }
  return den > 0.0 ? sqrt(num / den) : sqrt(num);
}

/* oracle_llt_residual_sampled -- the residual entries (A - L L^T)(is[q], js[q]) for
 * m sampled band positions (is[q] >= js[q], is[q]-js[q] <= k), each by Dot2. */
void oracle_llt_residual_sampled(int n, int k, const double* a, int lda, const double* l, int ldl,
                                 int m, const int* is, const int* js, double* out) {
  if (k > n - 1) k = n - 1;
  for (int q = 0; q < m; ++q) out[q] = llt_residual_entry(k, a, lda, l, ldl, is[q], js[q]);
}

/*
 * oracle_sbmv_residual_sampled -- r_i = b_i - (A x)_i for m sampled rows is[],
 * one right-hand side, by Dot2 over the 2k+1 band terms.
 */
void oracle_sbmv_residual_sampled(int n, int k, const double* ab, int ldab, const double* x,
                                  const double* b, int m, const int* is, double* out) {
  if (k > n - 1) k = n - 1;
  for (int q = 0; q < m; ++q) {
    const int i = is[q];
    double s = b[i], c = 0.0;
    for (int j = imax(0, i - k); j <= imin(n - 1, i + k); ++j) {
      const double a = (i >= j) ? BAND(ab, ldab, i - j, j) : BAND(ab, ldab, j - i, i);
      double p, ep, t, et;
      two_prod(a, x[j], &p, &ep);
      two_sum(s, -p, &t, &et);
      s = t;
      c += et - ep;
    }
    out[q] = s + c;
  }
}

/*
 * oracle_flops_eq1 -- Eq. (1) of Sec. 3.2 summed term by term, exactly as
 * printed (1-based, r = max(1, i-k), inner l-sum up to j inclusive):
 *     sum_{i=1}^{N} sum_{j=r}^{i} sum_{l=r}^{j} 2  +  sum_{i=1}^{N} sum_{j=r}^{i} 2.
 * O(N k^2) additions; meant for the small cases that pin the closed form.
 */
uint64_t oracle_flops_eq1(int64_t N, int64_t k) {
  uint64_t total = 0;
  for (int64_t i = 1; i <= N; ++i) {
    const int64_t r = (i - k > 1) ? i - k : 1;
    for (int64_t j = r; j <= i; ++j) {
      for (int64_t l = r; l <= j; ++l) total += 2;
      total += 2;
    }
  }
  return total;
}

/*
 * oracle_inverse_band -- the lower band of Sigma = A^{-1} (Sigma(i,j) for
 * j <= i <= min(n-1, j+k)), straight from the definition: column j of Sigma is
 * the solution of A s = e_j, taken with oracle_pbtrs from the factor in `l`.
 * O(n^2 k) work; `work` holds n doubles.  Used by the adjoint checks.
 */
void oracle_inverse_band(int n, int k, const double* l, int ldl, double* sig, int ldsig, double* work) {
  if (n <= 0) return;
  if (k > n - 1) k = n - 1;
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) work[i] = 0.0;
    work[j] = 1.0;
    oracle_pbtrs(n, k, 1, l, ldl, work, n);
    for (int i = j; i <= imin(n - 1, j + k); ++i) BAND(sig, ldsig, i - j, j) = work[i];
  }
}

/*
 * oracle_band_grad_sampled -- the gradient of a loss f(x, log det A), with
 * x = A^{-1} b, with respect to m stored band entries ab(is[q]-js[q], js[q]).
 * A stored off-diagonal entry is both A(i,j) and A(j,i) of the symmetric
 * matrix, so it moves two entries of A.  With xbar = df/dx, ldbar =
 * df/dlogdet, bbar = A^{-1} xbar and Sigma = A^{-1}:
 *     d f / d A(i,j) (one entry of a general matrix) = -bbar_i x_j + ldbar Sigma(j,i)
 *   and summing the two entries a stored off-diagonal slot drives,
 *     gbar(i,j) = -(bbar_i x_j + bbar_j x_i) + 2 ldbar Sigma(i,j)     (i > j)
 *     gbar(i,i) = -bbar_i x_i + ldbar Sigma(i,i).
 * Sigma(i,j) is formed per entry as (A^{-1} e_j)_i by oracle_pbtrs.  `bbar`
 * is given (n doubles), `work` holds n doubles.
 */
void oracle_band_grad_sampled(int n, int k, const double* l, int ldl, const double* x, const double* bbar,
                              double ldbar, int m, const int* is, const int* js, double* out, double* work) {
  if (k > n - 1) k = n - 1;
  for (int q = 0; q < m; ++q) {
    const int i = is[q], j = js[q];
    for (int t = 0; t < n; ++t) work[t] = 0.0;
    work[j] = 1.0;
    oracle_pbtrs(n, k, 1, l, ldl, work, n);
    const double sig = work[i];
    if (i == j) out[q] = -bbar[i] * x[i] + ldbar * sig;
    else out[q] = -(bbar[i] * x[j] + bbar[j] * x[i]) + 2.0 * ldbar * sig;
  }
}
