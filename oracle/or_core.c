/*
 * or_core.c -- univariate building blocks of the oracle (TEST INFRASTRUCTURE).
 *
 *  - B-splines by the Cox-de Boor recursion written as its definition
 *    (Sect. 2.1: knot vector, spans, p+1 non-zero functions per span).
 *  - Gauss-Legendre nodes by Newton's method on the three-term recurrence,
 *    in long double.
 *  - Minimum-norm solution of the WQ exactness system (Eq. 5) by Householder
 *    QR of A^T (the paper solves Eq. 5 "by QR-factorization"; reading R2 picks
 *    the minimum 2-norm solution among the non-unique ones).
 *  - Boehm single-knot insertion (Eq. 10).
 *  - Weighted-quadrature point layout (reading R1) and weights (Eq. 5, exactness
 *    integrals by element Gauss with p+1 points, reading R3).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* B_{i,k}(x) from the recursive definition; 0/0 := 0.  The last non-empty
 * span is closed on the right so that the end of the domain evaluates. */
static double cdb(const double *U, int nk, int i, int k, double x) {
  if (k == 0) {
    if (U[i] < U[i + 1]) {
      if (U[i] <= x && x < U[i + 1]) return 1.0;
      if (x == U[nk - 1] && U[i + 1] == U[nk - 1]) return 1.0;
    }
    return 0.0;
  }
  double left = 0.0, right = 0.0;
  double d1 = U[i + k] - U[i];
  double d2 = U[i + k + 1] - U[i + 1];
  if (d1 > 0.0) left = (x - U[i]) / d1 * cdb(U, nk, i, k - 1, x);
  if (d2 > 0.0) right = (U[i + k + 1] - x) / d2 * cdb(U, nk, i + 1, k - 1, x);
  return left + right;
}

double or_bspline(const double *U, int nk, int p, int i, double x) {
  return cdb(U, nk, i, p, x);
}

/* d/dx B_{i,p} = p/(U[i+p]-U[i]) B_{i,p-1} - p/(U[i+p+1]-U[i+1]) B_{i+1,p-1} */
double or_bspline_deriv(const double *U, int nk, int p, int i, double x) {
  if (p == 0) return 0.0;
  double a = 0.0, b = 0.0;
  double d1 = U[i + p] - U[i];
  double d2 = U[i + p + 1] - U[i + 1];
  if (d1 > 0.0) a = (double)p / d1 * cdb(U, nk, i, p - 1, x);
  if (d2 > 0.0) b = (double)p / d2 * cdb(U, nk, i + 1, p - 1, x);
  return a - b;
}

/* q-point Gauss-Legendre rule on [-1,1], nodes ascending. */
void or_gauss_legendre(int q, double *x, double *w) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < q; k++) {
    long double z = cosl(pi * ((long double)k + 0.75L) / ((long double)q + 0.5L));
    long double dp = 1.0L;
    for (int it = 0; it < 100; it++) {
      long double p0 = 1.0L, p1 = z;
      for (int m = 2; m <= q; m++) {
        long double p2 = ((2.0L * m - 1.0L) * z * p1 - (m - 1.0L) * p0) / (long double)m;
        p0 = p1;
        p1 = p2;
      }
      if (q == 1) p0 = 1.0L;
      /* p1 = P_q(z), p0 = P_{q-1}(z) */
      dp = (long double)q * (z * p1 - p0) / (z * z - 1.0L);
      long double dz = p1 / dp;
      z -= dz;
      if (fabsl(dz) < 1e-30L) break;
    }
    {
      long double p0 = 1.0L, p1 = z;
      for (int m = 2; m <= q; m++) {
        long double p2 = ((2.0L * m - 1.0L) * z * p1 - (m - 1.0L) * p0) / (long double)m;
        p0 = p1;
        p1 = p2;
      }
      if (q == 1) p0 = 1.0L;
      dp = (long double)q * (z * p1 - p0) / (z * z - 1.0L);
    }
    x[k] = (double)(-z);
    w[k] = (double)(2.0L / ((1.0L - z * z) * dp * dp));
  }
}

/* Minimum 2-norm solution of A w = b; A is m x N row-major, m <= N, full row
 * rank.  Householder QR of A^T = Q R, then R^T y = b and w = Q [y; 0]. */
int or_minnorm(int m, int N, const double *A, const double *b, double *w) {
  double *T = (double *)malloc(sizeof(double) * (size_t)N * m);
  double *V = (double *)calloc((size_t)N * m, sizeof(double));
  double *beta = (double *)calloc((size_t)m, sizeof(double));
  double *y = (double *)malloc(sizeof(double) * (size_t)m);
  int rc = 0;
  for (int r = 0; r < N; r++)
    for (int c = 0; c < m; c++) T[r * m + c] = A[c * N + r];
  for (int k = 0; k < m; k++) {
    double nrm = 0.0;
    for (int r = k; r < N; r++) nrm += T[r * m + k] * T[r * m + k];
    nrm = sqrt(nrm);
    if (nrm == 0.0) { rc = -1; goto done; }
    double alpha = T[k * m + k] > 0.0 ? -nrm : nrm;
    double vn = 0.0;
    for (int r = k; r < N; r++) {
      double v = T[r * m + k] - (r == k ? alpha : 0.0);
      V[r * m + k] = v;
      vn += v * v;
    }
    beta[k] = vn > 0.0 ? 2.0 / vn : 0.0;
    for (int c = k; c < m; c++) {
      double s = 0.0;
      for (int r = k; r < N; r++) s += V[r * m + k] * T[r * m + c];
      s *= beta[k];
      for (int r = k; r < N; r++) T[r * m + c] -= s * V[r * m + k];
    }
  }
  /* R^T y = b (forward substitution); R = upper triangle of T[0:m,0:m] */
  for (int k = 0; k < m; k++) {
    double s = b[k];
    for (int j = 0; j < k; j++) s -= T[j * m + k] * y[j];
    if (T[k * m + k] == 0.0) { rc = -1; goto done; }
    y[k] = s / T[k * m + k];
  }
  for (int r = 0; r < N; r++) w[r] = r < m ? y[r] : 0.0;
  for (int k = m - 1; k >= 0; k--) {
    double s = 0.0;
    for (int r = k; r < N; r++) s += V[r * m + k] * w[r];
    s *= beta[k];
    for (int r = k; r < N; r++) w[r] -= s * V[r * m + k];
  }
done:
  free(T);
  free(V);
  free(beta);
  free(y);
  return rc;
}

/* Eq. 10: insert t once.  New coefficients c'_k = alpha_k c_k + (1-alpha_k) c_{k-1}
 * with alpha_k = 1 (k <= s-p), (t-U_k)/(U_{k+p}-U_k) (s-p+1 <= k <= s),
 * 0 (k >= s+1), s the span with U_s <= t < U_{s+1}. */
void or_insert_knot(const double *U, int nk, int p, double t, const double *c,
                    double *Unew, double *cnew) {
  int n = nk - p - 1;
  int s = -1;
  for (int j = 0; j < nk - 1; j++)
    if (U[j] <= t && t < U[j + 1]) s = j;
  for (int k = 0; k <= n; k++) {
    double alpha;
    if (k <= s - p) alpha = 1.0;
    else if (k >= s + 1) alpha = 0.0;
    else alpha = (t - U[k]) / (U[k + p] - U[k]);
    double ck = k < n ? c[k] : 0.0;
    double ckm = k > 0 ? c[k - 1] : 0.0;
    cnew[k] = alpha * ck + (1.0 - alpha) * ckm;
  }
  for (int j = 0; j <= s; j++) Unew[j] = U[j];
  Unew[s + 1] = t;
  for (int j = s + 1; j < nk; j++) Unew[j + 1] = U[j];
}

static int mult_of(const double *U, int nk, double v) {
  int m = 0;
  for (int j = 0; j < nk; j++)
    if (U[j] == v) m++;
  return m;
}

/* Reading R1: an element touching a knot of multiplicity 2 or more (a domain
 * end, a repeated interior knot of a mixed-continuity vector, a DWQ disc in
 * its refined space) gets p+1 points, every other element 2; points uniform
 * in the element's interior.  The zero-length spans of repeated knots get
 * none. */
int or_wq_points(const double *U, int nk, int p, double *x) {
  int cnt = 0;
  for (int j = p; j < nk - p - 1; j++) {
    double a = U[j], b = U[j + 1];
    if (!(b > a)) continue;
    int m = (mult_of(U, nk, a) >= 2 || mult_of(U, nk, b) >= 2) ? p + 1 : 2;
    for (int q = 0; q < m; q++) {
      if (x) x[cnt] = a + (b - a) * (double)(q + 1) / (double)(m + 1);
      cnt++;
    }
  }
  return cnt;
}

/* int B_j B_i over the real line by element Gauss with p+1 points (R3). */
static double exact_product(const double *U, int nk, int p, int i, int j) {
  double gx[16], gw[16];
  or_gauss_legendre(p + 1, gx, gw);
  double lo = fmax(U[i], U[j]), hi = fmin(U[i + p + 1], U[j + p + 1]);
  double s = 0.0;
  for (int e = 0; e < nk - 1; e++) {
    double a = U[e], b = U[e + 1];
    if (!(b > a) || a < lo || b > hi) continue;
    for (int g = 0; g <= p; g++) {
      double xx = a + (b - a) * (gx[g] + 1.0) * 0.5;
      s += gw[g] * (b - a) * 0.5 * cdb(U, nk, i, p, xx) * cdb(U, nk, j, p, xx);
    }
  }
  return s;
}

/* Eq. 5: sum_{k in Q_i} B_{j_r}(x_k) w_k = int B_{j_r} B_i for every trial j_r
 * whose support overlaps supp B_i; Q_i = points inside supp B_i. */
int or_wq_weights(const double *U, int nk, int p, const double *x, int nx, int i,
                  double *w) {
  int n = nk - p - 1;
  int *rows = (int *)malloc(sizeof(int) * (size_t)n);
  int *cols = (int *)malloc(sizeof(int) * (size_t)nx);
  int m = 0, N = 0;
  for (int j = 0; j < n; j++) {
    double lo = fmax(U[i], U[j]), hi = fmin(U[i + p + 1], U[j + p + 1]);
    if (hi > lo) rows[m++] = j;
  }
  for (int k = 0; k < nx; k++)
    if (x[k] > U[i] && x[k] < U[i + p + 1]) cols[N++] = k;
  double *A = (double *)malloc(sizeof(double) * (size_t)m * N);
  double *b = (double *)malloc(sizeof(double) * (size_t)m);
  double *ww = (double *)malloc(sizeof(double) * (size_t)N);
  for (int r = 0; r < m; r++) {
    for (int c = 0; c < N; c++) A[r * N + c] = cdb(U, nk, rows[r], p, x[cols[c]]);
    b[r] = exact_product(U, nk, p, i, rows[r]);
  }
  int rc = or_minnorm(m, N, A, b, ww);
  for (int k = 0; k < nx; k++) w[k] = 0.0;
  for (int c = 0; c < N; c++) w[cols[c]] = ww[c];
  free(rows);
  free(cols);
  free(A);
  free(b);
  free(ww);
  return rc == 0 ? N : -1;
}
