/*
 * or_patch.c -- the oracle's patch: quadrature set-up, trimming classification,
 * cut-element rules, discontinuous weighted quadrature, formation of the mass
 * matrix row by row, right-hand side, CG and L2 error (TEST INFRASTRUCTURE).
 *
 * Formation follows the paper literally: every active row i owns one
 * quadrature rule Q_i = {(xi_q, omega_q)} with the test function folded into
 * the weights (Eq. 4), and m_ij = sum_q omega_q c(xi_q) B_j(xi_q) (Eq. 6).
 * Which rule a row uses:
 *   interior row            tensor WQ rule Q_{i1} x Q_{i2} (Sect. 2.1, Eqs. 5, 7)
 *   cut row, hybrid Gauss   Gauss on the regular elements of the support plus the
 *                           cut-element rule on the cut elements (Sect. 3.2, Eq. 8)
 *   cut row, DWQ            DWQ rule on a rectangle R of regular elements, Gauss on
 *                           the other regular elements, cut rule on cut elements
 *                           (Sect. 3.3; region choice = reading R7)
 *   cut row, naive WQ       tensor WQ rule with c = 0 off S^r plus the cut rule
 *                           (the negative control of Table 1)
 *   method GAUSS            element Gauss for every row (the paper's reference)
 * Differentiation with respect to a density spline rho = sum_k d_k N_k in
 * c = rho det J (reading R12): or_loss gives L = sum_q omega_q detJ (u_h - g)^2
 * over Omega^v and dL/du; or_density_grad gives dL/dd_k for u and the adjoint
 * lambda = M_s^{-1} dL/du by walking every row's rule point by point, with c
 * replaced by N_k det J (each rule is linear in c).
 * No sum factorisation, blocking or reordering is applied here: the point of
 * the oracle is that each step can be checked by eye against the paper.
 *
 * Parity unpinned (no test outside the oracle can tell the alternatives
 * apart, since every admissible choice is exact at c = 1): the tie between
 * regions with the same element count and fewer discs in or_dwq_choice
 * (reading R7), and the test of the curve's first point inside the element
 * in classify (reading R8; redundant for every curve that crosses a knot
 * line).  The GPU path is held to the same choices by the parity tests.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int or_curve_folds(const or_desc *d, int o, double *pts, int cap);
int or_curve_joints(const or_desc *d, double *pts, int cap);
void or_curve_point0(const or_desc *d, double *xy);

#define MAXP1 8
#define HITCAP 512
/* relative tolerances of readings R6 and R8 */
#define CORNER 1e-12
#define TIE 1e-9

typedef struct {
  int p, nk, n, nel;
  double *U;  /* knots */
  double *bp; /* nel+1 breakpoints */
  int nq;     /* WQ points */
  double *xq;
  int *qel;   /* element of each point */
  double *W;  /* n x nq WQ weights (zero outside the support) */
  int *qlo, *qhi; /* points of supp B_i: qlo[i]..qhi[i] (points are sorted) */
  double *Bv; /* nq x (p+1): B_{qel+a}(x_k) */
  double *Bd; /* nq x (p+1): derivatives */
  double *gx, *gw; /* reference Gauss rule with p+1 points */
  double *GBv, *GBd; /* nel x (p+1) x (p+1): B_{e+a} at Gauss point g */
} dirdata;

typedef struct {
  double x[2];
  double wc; /* weight (with the test function folded in) times c */
  double w;  /* the same weight without c (0 where c is masked)   */
  int e[2];
  double bv[2][MAXP1];
} rpoint;

struct or_patch {
  or_desc d;
  int ncurves;            /* trimming curves: cd[k] is the descriptor with curve k */
  or_desc cd[OR_MAXCURVES];
  dirdata D[2];
  double *own[32];
  int nown;
  uint8_t *estate, *fstate;
  int32_t *act;
  int64_t nrows, nnz;
  int64_t *rowg;
  double *C; /* nq2 x nq1 */
  int qc;
  int64_t *cut_off; /* per element: offset (in points) into cut_pts */
  double *cut_pts;  /* x, y, w */
  double *cut_c;
  double *gc;       /* c at the element Gauss points, lazily filled */
  uint8_t *gc_done;
  int *choice;      /* per function g: k1, s1, k2, s2 (k1 = -1: none) */
};

/* ------------------------------------------------------------------ */

static double *dup(or_patch *P, const double *src, size_t n) {
  if (!src || n == 0) return NULL;
  double *d = (double *)malloc(sizeof(double) * n);
  memcpy(d, src, sizeof(double) * n);
  P->own[P->nown++] = d;
  return d;
}

static int elem_of(const dirdata *D, double x) {
  int lo = 0, hi = D->nel - 1;
  if (x >= D->bp[D->nel]) return D->nel - 1;
  if (x <= D->bp[0]) return 0;
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    if (D->bp[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

/* values (and derivatives) of the p+1 functions e..e+p that live on element e */
static void basis_at(const dirdata *D, int e, double x, double *v, double *dv) {
  for (int a = 0; a <= D->p; a++) {
    v[a] = or_bspline(D->U, D->nk, D->p, e + a, x);
    if (dv) dv[a] = or_bspline_deriv(D->U, D->nk, D->p, e + a, x);
  }
}

static double density_at(const or_patch *P, double x1, double x2) {
  const or_desc *d = &P->d;
  double s = 0.0;
  int m1 = d->dens_nknots[0] - d->dens_p[0] - 1;
  int m2 = d->dens_nknots[1] - d->dens_p[1] - 1;
  for (int k2 = 0; k2 < m2; k2++) {
    double b2 = or_bspline(d->dens_knots[1], d->dens_nknots[1], d->dens_p[1], k2, x2);
    if (b2 == 0.0) continue;
    for (int k1 = 0; k1 < m1; k1++) {
      double b1 = or_bspline(d->dens_knots[0], d->dens_nknots[0], d->dens_p[0], k1, x1);
      s += d->dens_coef[k2 * m1 + k1] * b1 * b2;
    }
  }
  return s;
}

/* c at a point given the basis values/derivatives of the element functions:
 * det J of x(xi) = sum_{i1,i2} P_{i1 i2} B_{i1}(xi1) B_{i2}(xi2) (Eq. 6's c),
 * times the density for OR_COEF_DENSITY. */
static double coef_from(const or_patch *P, double x1, double x2, int e1, const double *v1,
                        const double *d1, int e2, const double *v2, const double *d2) {
  const or_desc *d = &P->d;
  if (d->coef_kind == OR_COEF_ONE) return 1.0;
  double detj = 1.0;
  if (d->geom_kind == OR_GEOM_SPLINE) {
    int n1 = P->D[0].n;
    double xa = 0, xb = 0, ya = 0, yb = 0;
    for (int b = 0; b <= P->D[1].p; b++)
      for (int a = 0; a <= P->D[0].p; a++) {
        const double *pt = d->geom_ctrl + 2 * ((size_t)(e2 + b) * n1 + (e1 + a));
        xa += pt[0] * d1[a] * v2[b];
        ya += pt[1] * d1[a] * v2[b];
        xb += pt[0] * v1[a] * d2[b];
        yb += pt[1] * v1[a] * d2[b];
      }
    detj = xa * yb - xb * ya;
  }
  if (d->coef_kind == OR_COEF_DENSITY) return density_at(P, x1, x2) * detj;
  return detj;
}

static double coef_at(const or_patch *P, double x1, double x2) {
  double v1[MAXP1], d1[MAXP1], v2[MAXP1], d2[MAXP1];
  int e1 = elem_of(&P->D[0], x1), e2 = elem_of(&P->D[1], x2);
  basis_at(&P->D[0], e1, x1, v1, d1);
  basis_at(&P->D[1], e2, x2, v2, d2);
  return coef_from(P, x1, x2, e1, v1, d1, e2, v2, d2);
}

static void phys_from(const or_patch *P, double x1, double x2, int e1, const double *v1,
                      int e2, const double *v2, double *X) {
  if (P->d.geom_kind != OR_GEOM_SPLINE) {
    X[0] = x1;
    X[1] = x2;
    return;
  }
  int n1 = P->D[0].n;
  X[0] = X[1] = 0.0;
  for (int b = 0; b <= P->D[1].p; b++)
    for (int a = 0; a <= P->D[0].p; a++) {
      const double *pt = P->d.geom_ctrl + 2 * ((size_t)(e2 + b) * n1 + (e1 + a));
      X[0] += pt[0] * v1[a] * v2[b];
      X[1] += pt[1] * v1[a] * v2[b];
    }
}

/* the visible domain is the intersection of every curve's kept side */
static int visible(const or_patch *P, double x, double y) {
  for (int k = 0; k < P->ncurves; k++) {
    const or_desc *c = &P->cd[k];
    if (c->trim_kind == OR_TRIM_NONE) continue;
    int in = or_curve_inside(c, x, y);
    if (c->trim_keep_inside ? !in : in) return 0;
  }
  return 1;
}

static int cmpd(const void *a, const void *b);

/* crossings of every curve with the line xi_o = s inside (lo, hi), ascending */
static int set_line_hits(const or_patch *P, int o, double s, double lo, double hi, double *out,
                         int cap) {
  int n = 0;
  for (int k = 0; k < P->ncurves; k++) {
    if (P->cd[k].trim_kind == OR_TRIM_NONE) continue;
    n += or_curve_line_hits(&P->cd[k], o, s, lo, hi, out + n, cap - n);
  }
  qsort(out, (size_t)n, sizeof(double), cmpd);
  return n;
}

static int set_folds(const or_patch *P, int o, double *pts, int cap) {
  int n = 0;
  for (int k = 0; k < P->ncurves; k++)
    if (P->cd[k].trim_kind != OR_TRIM_NONE) n += or_curve_folds(&P->cd[k], o, pts + 2 * n, cap - n);
  return n;
}

static int set_joints(const or_patch *P, double *pts, int cap) {
  int n = 0;
  for (int k = 0; k < P->ncurves; k++)
    if (P->cd[k].trim_kind != OR_TRIM_NONE) n += or_curve_joints(&P->cd[k], pts + 2 * n, cap - n);
  return n;
}

/* ------------------------------------------------------------------ */
/* one direction: knots, WQ points (R1), WQ weights (Eq. 5), tables     */

static void setup_dir(or_patch *P, int dir) {
  dirdata *D = &P->D[dir];
  const or_desc *d = &P->d;
  D->p = d->p[dir];
  D->nk = d->nknots[dir];
  D->U = dup(P, d->knots[dir], (size_t)D->nk);
  D->n = D->nk - D->p - 1;
  D->nel = D->n - D->p;
  D->bp = (double *)malloc(sizeof(double) * (size_t)(D->nel + 1));
  for (int e = 0; e <= D->nel; e++) D->bp[e] = D->U[D->p + e];
  D->nq = or_wq_points(D->U, D->nk, D->p, NULL);
  D->xq = (double *)malloc(sizeof(double) * (size_t)D->nq);
  or_wq_points(D->U, D->nk, D->p, D->xq);
  D->qel = (int *)malloc(sizeof(int) * (size_t)D->nq);
  int p1 = D->p + 1;
  D->Bv = (double *)malloc(sizeof(double) * (size_t)D->nq * p1);
  D->Bd = (double *)malloc(sizeof(double) * (size_t)D->nq * p1);
  for (int k = 0; k < D->nq; k++) {
    D->qel[k] = elem_of(D, D->xq[k]);
    basis_at(D, D->qel[k], D->xq[k], D->Bv + (size_t)k * p1, D->Bd + (size_t)k * p1);
  }
  D->qlo = (int *)malloc(sizeof(int) * (size_t)D->n);
  D->qhi = (int *)malloc(sizeof(int) * (size_t)D->n);
  for (int i = 0; i < D->n; i++) {
    D->qlo[i] = D->nq;
    D->qhi[i] = -1;
    for (int k = 0; k < D->nq; k++)
      if (D->xq[k] > D->U[i] && D->xq[k] < D->U[i + D->p + 1]) {
        if (k < D->qlo[i]) D->qlo[i] = k;
        D->qhi[i] = k;
      }
  }
  D->W = (double *)malloc(sizeof(double) * (size_t)D->n * D->nq);
#pragma omp parallel for schedule(dynamic, 8)
  for (int i = 0; i < D->n; i++)
    or_wq_weights(D->U, D->nk, D->p, D->xq, D->nq, i, D->W + (size_t)i * D->nq);
  D->gx = (double *)malloc(sizeof(double) * p1);
  D->gw = (double *)malloc(sizeof(double) * p1);
  or_gauss_legendre(p1, D->gx, D->gw);
  D->GBv = (double *)malloc(sizeof(double) * (size_t)D->nel * p1 * p1);
  D->GBd = (double *)malloc(sizeof(double) * (size_t)D->nel * p1 * p1);
  for (int e = 0; e < D->nel; e++)
    for (int g = 0; g < p1; g++) {
      double a = D->bp[e], b = D->bp[e + 1];
      double x = a + (b - a) * 0.5 * (D->gx[g] + 1.0);
      double *v = D->GBv + ((size_t)e * p1 + g) * p1, *dv = D->GBd + ((size_t)e * p1 + g) * p1;
      if (b > a) {
        basis_at(D, e, x, v, dv);
      } else { /* the zero-length span of a repeated knot: nothing lives on it */
        for (int k = 0; k < p1; k++) v[k] = dv[k] = 0.0;
      }
    }
}

static void free_dir(dirdata *D) {
  free(D->bp);
  free(D->xq);
  free(D->qel);
  free(D->W);
  free(D->qlo);
  free(D->qhi);
  free(D->Bv);
  free(D->Bd);
  free(D->gx);
  free(D->gw);
  free(D->GBv);
  free(D->GBd);
}

/* ------------------------------------------------------------------ */
/* classification (Sect. 2.2, reading R8)                               */

static int any_in(const double *v, int n, double lo, double hi) {
  for (int k = 0; k < n; k++)
    if (v[k] > lo && v[k] < hi) return 1;
  return 0;
}

static void classify(or_patch *P) {
  dirdata *A = &P->D[0], *B = &P->D[1];
  int ne = A->nel * B->nel;
  P->estate = (uint8_t *)malloc((size_t)ne);
  if (P->ncurves == 1 && P->d.trim_kind == OR_TRIM_NONE) {
    for (int e2 = 0; e2 < B->nel; e2++)
      for (int e1 = 0; e1 < A->nel; e1++)
        P->estate[e2 * A->nel + e1] =
            (A->bp[e1 + 1] > A->bp[e1] && B->bp[e2 + 1] > B->bp[e2]) ? OR_ELEM_REGULAR
                                                                     : OR_ELEM_EMPTY;
  } else {
    /* crossings of the curve with every knot line */
    double *vh = (double *)malloc(sizeof(double) * (size_t)(A->nel + 1) * HITCAP);
    int *vn = (int *)malloc(sizeof(int) * (size_t)(A->nel + 1));
    double *hh = (double *)malloc(sizeof(double) * (size_t)(B->nel + 1) * HITCAP);
    int *hn = (int *)malloc(sizeof(int) * (size_t)(B->nel + 1));
    for (int e = 0; e <= A->nel; e++)
      vn[e] = set_line_hits(P, 0, A->bp[e], -1e300, 1e300, vh + (size_t)e * HITCAP, HITCAP);
    for (int e = 0; e <= B->nel; e++)
      hn[e] = set_line_hits(P, 1, B->bp[e], -1e300, 1e300, hh + (size_t)e * HITCAP, HITCAP);
    double p0[OR_MAXCURVES][2];
    for (int k = 0; k < P->ncurves; k++) or_curve_point0(&P->cd[k], p0[k]);
    for (int e2 = 0; e2 < B->nel; e2++)
      for (int e1 = 0; e1 < A->nel; e1++) {
        double a1 = A->bp[e1], b1 = A->bp[e1 + 1], a2 = B->bp[e2], b2 = B->bp[e2 + 1];
        if (!(b1 > a1) || !(b2 > a2)) { /* R1, R8: an empty span has no measure */
          P->estate[e2 * A->nel + e1] = OR_ELEM_EMPTY;
          continue;
        }
        /* R8: a crossing within TW_CORNER of an edge's end is a corner touch,
         * not a cut (keeps the decision off rounding at curves through corners) */
        double d1 = CORNER * (b1 - a1), d2 = CORNER * (b2 - a2);
        int cut = any_in(vh + (size_t)e1 * HITCAP, vn[e1], a2 + d2, b2 - d2) ||
                  any_in(vh + (size_t)(e1 + 1) * HITCAP, vn[e1 + 1], a2 + d2, b2 - d2) ||
                  any_in(hh + (size_t)e2 * HITCAP, hn[e2], a1 + d1, b1 - d1) ||
                  any_in(hh + (size_t)(e2 + 1) * HITCAP, hn[e2 + 1], a1 + d1, b1 - d1);
        /* a whole curve inside the element */
        for (int k = 0; k < P->ncurves && !cut; k++)
          cut = p0[k][0] > a1 && p0[k][0] < b1 && p0[k][1] > a2 && p0[k][1] < b2;
        uint8_t st;
        if (cut) st = OR_ELEM_CUT;
        else st = visible(P, 0.5 * (a1 + b1), 0.5 * (a2 + b2)) ? OR_ELEM_REGULAR : OR_ELEM_INVISIBLE;
        P->estate[e2 * A->nel + e1] = st;
      }
    free(vh);
    free(vn);
    free(hh);
    free(hn);
  }
  int nf = A->n * B->n;
  P->fstate = (uint8_t *)malloc((size_t)nf);
  P->act = (int32_t *)malloc(sizeof(int32_t) * (size_t)nf);
  P->nrows = 0;
  for (int i2 = 0; i2 < B->n; i2++)
    for (int i1 = 0; i1 < A->n; i1++) {
      int nreg = 0, ninv = 0, tot = 0;
      for (int e2 = i2 - B->p; e2 <= i2; e2++)
        for (int e1 = i1 - A->p; e1 <= i1; e1++) {
          if (e1 < 0 || e2 < 0 || e1 >= A->nel || e2 >= B->nel) continue;
          uint8_t s = P->estate[e2 * A->nel + e1];
          if (s == OR_ELEM_EMPTY) continue; /* R8: the states of the elements with measure */
          tot++;
          if (s == OR_ELEM_REGULAR) nreg++;
          if (s == OR_ELEM_INVISIBLE) ninv++;
        }
      int g = i2 * A->n + i1;
      P->fstate[g] = ninv == tot ? OR_FUNC_EXTERIOR : (nreg == tot ? OR_FUNC_INTERIOR : OR_FUNC_CUT);
      P->act[g] = P->fstate[g] == OR_FUNC_EXTERIOR ? -1 : (int32_t)P->nrows++;
    }
  P->rowg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(P->nrows + 1));
  P->nnz = 0;
  for (int g = 0; g < nf; g++) {
    if (P->act[g] < 0) continue;
    P->rowg[P->act[g]] = g;
    int i1 = g % A->n, i2 = g / A->n;
    for (int j2 = i2 - B->p; j2 <= i2 + B->p; j2++)
      for (int j1 = i1 - A->p; j1 <= i1 + A->p; j1++) {
        if (j1 < 0 || j2 < 0 || j1 >= A->n || j2 >= B->n) continue;
        if (P->act[j2 * A->n + j1] >= 0) P->nnz++;
      }
  }
}

/* ------------------------------------------------------------------ */
/* cut-element rule (Sect. 3.1; reading R6)                             */

typedef struct {
  double *v;
  int n, cap;
} dbuf;

static void push(dbuf *b, double x) {
  if (b->n == b->cap) {
    b->cap = b->cap ? 2 * b->cap : 256;
    b->v = (double *)realloc(b->v, sizeof(double) * (size_t)b->cap);
  }
  b->v[b->n++] = x;
}

static int cmpd(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Points (xi1, xi2, w) of a rule for the visible part of element (e1, e2):
 *  1. outer direction o: the axis along which the curve's part in the element
 *     extends more (bounding box of edge crossings and tangent points, each
 *     counted up to CORNER beyond the element's edges; extents equal within
 *     TIE times the element size count as a tie, which goes to o = 0);
 *  2. breakpoints along o: the element ends, the crossings of the curve with the
 *     two element edges parallel to o, the curve's tangent points that would
 *     fold the lines xi_o = const, and the spline's segment joints;
 *  3. q Gauss points per piece; on each line xi_o = s the crossings split the
 *     inner range into intervals, the visible ones (midpoint test) get q Gauss
 *     points each. */
static void cut_rule_build(const or_patch *P, int e1, int e2, dbuf *out) {
  double a[2] = {P->D[0].bp[e1], P->D[1].bp[e2]};
  double b[2] = {P->D[0].bp[e1 + 1], P->D[1].bp[e2 + 1]};
  int q = P->qc;
  double gx[64], gw[64];
  or_gauss_legendre(q, gx, gw);
  double hits[HITCAP], pts[2 * HITCAP];
  double lo[2] = {1e300, 1e300}, hi[2] = {-1e300, -1e300};
#define BBOX(X, Y)                            \
  do {                                        \
    double _x = (X), _y = (Y);                \
    if (_x < lo[0]) lo[0] = _x;               \
    if (_x > hi[0]) hi[0] = _x;               \
    if (_y < lo[1]) lo[1] = _y;               \
    if (_y > hi[1]) hi[1] = _y;               \
  } while (0)
  double del[2] = {CORNER * (b[0] - a[0]), CORNER * (b[1] - a[1])};
  for (int o = 0; o < 2; o++)
    for (int side = 0; side < 2; side++) {
      double s = side ? b[o] : a[o];
      int n = set_line_hits(P, o, s, a[1 - o] - del[1 - o], b[1 - o] + del[1 - o], hits, HITCAP);
      for (int k = 0; k < n; k++) {
        if (o == 0) BBOX(s, hits[k]);
        else BBOX(hits[k], s);
      }
    }
  for (int o = 0; o < 2; o++) {
    int n = set_folds(P, o, pts, HITCAP);
    for (int k = 0; k < n; k++) {
      double x = pts[2 * k], y = pts[2 * k + 1];
      if (x >= a[0] - del[0] && x <= b[0] + del[0] && y >= a[1] - del[1] && y <= b[1] + del[1])
        BBOX(x, y);
    }
  }
#undef BBOX
  /* ties (within TIE of the element size) go to o = 0 */
  double hmax = fmax(b[0] - a[0], b[1] - a[1]);
  int o = (hi[0] - lo[0] >= hi[1] - lo[1] - TIE * hmax) ? 0 : 1;
  int in = 1 - o;
  dbuf br = {0};
  push(&br, a[o]);
  push(&br, b[o]);
  for (int side = 0; side < 2; side++) {
    double s = side ? b[in] : a[in];
    int n = set_line_hits(P, in, s, a[o], b[o], hits, HITCAP);
    for (int k = 0; k < n; k++) push(&br, hits[k]);
  }
  {
    int n = set_folds(P, o, pts, HITCAP);
    for (int k = 0; k < n; k++) {
      double xo = pts[2 * k + o], xi = pts[2 * k + in];
      if (xo > a[o] && xo < b[o] && xi >= a[in] && xi <= b[in]) push(&br, xo);
    }
    n = set_joints(P, pts, HITCAP);
    for (int k = 0; k < n; k++) {
      double xo = pts[2 * k + o], xi = pts[2 * k + in];
      if (xo > a[o] && xo < b[o] && xi >= a[in] && xi <= b[in]) push(&br, xo);
    }
  }
  qsort(br.v, (size_t)br.n, sizeof(double), cmpd);
  double ends[HITCAP + 2];
  for (int pc = 0; pc + 1 < br.n; pc++) {
    double s0 = br.v[pc], s1 = br.v[pc + 1];
    if (!(s1 > s0)) continue;
    for (int g = 0; g < q; g++) {
      double s = s0 + (s1 - s0) * 0.5 * (gx[g] + 1.0);
      double ws = gw[g] * 0.5 * (s1 - s0);
      int n = set_line_hits(P, o, s, a[in], b[in], hits, HITCAP);
      ends[0] = a[in];
      for (int k = 0; k < n; k++) ends[k + 1] = hits[k];
      ends[n + 1] = b[in];
      for (int k = 0; k <= n; k++) {
        double u0 = ends[k], u1 = ends[k + 1];
        if (!(u1 > u0)) continue;
        double mid = 0.5 * (u0 + u1);
        double X = o == 0 ? s : mid, Y = o == 0 ? mid : s;
        if (!visible(P, X, Y)) continue;
        for (int h = 0; h < q; h++) {
          double u = u0 + (u1 - u0) * 0.5 * (gx[h] + 1.0);
          double w = ws * gw[h] * 0.5 * (u1 - u0);
          push(out, o == 0 ? s : u);
          push(out, o == 0 ? u : s);
          push(out, w);
        }
      }
    }
  }
  free(br.v);
}

static void build_cut_rules(or_patch *P) {
  int nel1 = P->D[0].nel, nel2 = P->D[1].nel;
  P->cut_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nel1 * nel2 + 1));
  dbuf all = {0};
  for (int e = 0; e < nel1 * nel2; e++) {
    P->cut_off[e] = all.n / 3;
    if (P->estate[e] == OR_ELEM_CUT) cut_rule_build(P, e % nel1, e / nel1, &all);
  }
  P->cut_off[nel1 * nel2] = all.n / 3;
  P->cut_pts = all.v;
  int64_t np = all.n / 3;
  P->cut_c = (double *)malloc(sizeof(double) * (size_t)(np > 0 ? np : 1));
  for (int64_t k = 0; k < np; k++)
    P->cut_c[k] = coef_at(P, all.v[3 * k], all.v[3 * k + 1]);
}

int or_cut_rule(const or_patch *P, int e1, int e2, double *pts, int cap) {
  int e = e2 * P->D[0].nel + e1;
  int64_t n = P->cut_off[e + 1] - P->cut_off[e];
  for (int64_t k = 0; k < n && k < cap; k++) {
    pts[3 * k] = P->cut_pts[3 * (P->cut_off[e] + k)];
    pts[3 * k + 1] = P->cut_pts[3 * (P->cut_off[e] + k) + 1];
    pts[3 * k + 2] = P->cut_pts[3 * (P->cut_off[e] + k) + 2];
  }
  return (int)n;
}

/* ------------------------------------------------------------------ */
/* discontinuous weighted quadrature (Sect. 3.3, Eqs. 9-10; R4, R5)      */

/* Reading R5: nested points for element e next to the disc t.  The element
 * keeps its base points; it needs p+1 points in all (the refined space has a
 * knot of multiplicity p+1 at t, reading R1).  The new points go one at a time
 * into the gap (a,x1), (x1,x2), (x2,b) whose spacing len/(q+1) is largest;
 * the base gaps are equal thirds, so "largest" is "fewest points so far", with
 * ties to the middle gap, then the gap next to t. */
static int nested_points(const dirdata *D, int e, int t_at_right, double *out) {
  int idx[MAXP1 + 2], m = 0;
  for (int k = 0; k < D->nq; k++)
    if (D->qel[k] == e) idx[m++] = k;
  int add = D->p + 1 - m;
  if (add <= 0) return 0;
  /* m == 2 here */
  double edge[4] = {D->bp[e], D->xq[idx[0]], D->xq[idx[1]], D->bp[e + 1]};
  int cnt[3] = {0, 0, 0};
  int pref[3] = {1, t_at_right ? 2 : 0, t_at_right ? 0 : 2};
  for (int r = 0; r < add; r++) {
    int best = pref[0];
    for (int k = 1; k < 3; k++)
      if (cnt[pref[k]] < cnt[best]) best = pref[k];
    cnt[best]++;
  }
  int n = 0;
  for (int gp = 0; gp < 3; gp++)
    for (int j = 0; j < cnt[gp]; j++)
      out[n++] = edge[gp] + (edge[gp + 1] - edge[gp]) * (double)(j + 1) / (double)(cnt[gp] + 1);
  return n;
}

/* DWQ rule of coarse function i, disc at breakpoint s (t = bp[s]), side 0
 * (left of t) or 1 (right of t).  Steps 1-4 of Sect. 3.3:
 *  1. insert t p times (C^{-1} at t) and keep S (Eq. 10);
 *  2. add nested points next to t (R5);
 *  3. WQ weights of the refined functions (Eq. 5);
 *  4. w = S^T w~ restricted to the refined functions on the chosen side (R4). */
int or_dwq_rule(const or_patch *P, int dir, int s, int side, int i, double *pts, int cap) {
  const dirdata *D = &P->D[dir];
  int p = D->p;
  double t = D->bp[s];
  int nk = D->nk;
  double *U = (double *)malloc(sizeof(double) * (size_t)(nk + p));
  double *Un = (double *)malloc(sizeof(double) * (size_t)(nk + p));
  double *c = (double *)calloc((size_t)(D->n + p), sizeof(double));
  double *cn = (double *)calloc((size_t)(D->n + p), sizeof(double));
  memcpy(U, D->U, sizeof(double) * (size_t)nk);
  c[i] = 1.0;
  for (int r = 0; r < p; r++) {
    or_insert_knot(U, nk, p, t, c, Un, cn);
    nk++;
    double *tmp = U; U = Un; Un = tmp;
    tmp = c; c = cn; cn = tmp;
  }
  int nr = nk - p - 1;
  double extra[2 * MAXP1];
  int ne = 0;
  ne += nested_points(D, s - 1, 1, extra + ne);
  ne += nested_points(D, s, 0, extra + ne);
  int nx = D->nq + ne;
  double *x = (double *)malloc(sizeof(double) * (size_t)nx);
  memcpy(x, D->xq, sizeof(double) * (size_t)D->nq);
  memcpy(x + D->nq, extra, sizeof(double) * (size_t)ne);
  qsort(x, (size_t)nx, sizeof(double), cmpd);
  double *w = (double *)calloc((size_t)nx, sizeof(double));
  double *wl = (double *)malloc(sizeof(double) * (size_t)nx);
  for (int l = 0; l < nr; l++) {
    if (c[l] == 0.0) continue;
    int on_side = side == 0 ? (U[l + p + 1] <= t) : (U[l] >= t);
    if (!on_side) continue;
    or_wq_weights(U, nk, p, x, nx, l, wl);
    for (int k = 0; k < nx; k++) w[k] += c[l] * wl[k];
  }
  int n = 0;
  double lo = D->U[i], hi = D->U[i + p + 1];
  for (int k = 0; k < nx; k++) {
    if (!(x[k] > lo && x[k] < hi)) continue;
    if (side == 0 ? !(x[k] < t) : !(x[k] > t)) continue;
    if (n < cap) {
      pts[2 * n] = x[k];
      pts[2 * n + 1] = w[k];
    }
    n++;
  }
  free(U);
  free(Un);
  free(c);
  free(cn);
  free(x);
  free(w);
  free(wl);
  return n;
}

/* Reading R7: the candidate regions R = R1 x R2, each R_d the whole support
 * (kind 0), its part left of an interior support knot bp[s] (kind 1) or right
 * of it (kind 2).  Valid if every element of R is regular (or empty: the
 * zero-length span of a repeated knot has no measure) and every disc bp[s]
 * is a simple knot (elements s-1 and s not empty: inserting t p times must
 * give multiplicity p+1); the valid one with most elements wins, then fewer
 * discs, then the first in the order (kind 0; kind 1 with s ascending; kind 2
 * with s ascending), direction 1 outer. */
static void opt_range(int kind, int s, int lo, int hi, int *r0, int *r1) {
  if (kind == 0) { *r0 = lo; *r1 = hi; }
  else if (kind == 1) { *r0 = lo; *r1 = s - 1; }
  else { *r0 = s; *r1 = hi; }
}

int or_dwq_choice(const or_patch *P, int i1, int i2, int *out) {
  const dirdata *A = &P->D[0], *B = &P->D[1];
  int lo[2] = {i1 - A->p < 0 ? 0 : i1 - A->p, i2 - B->p < 0 ? 0 : i2 - B->p};
  int hi[2] = {i1 < A->nel - 1 ? i1 : A->nel - 1, i2 < B->nel - 1 ? i2 : B->nel - 1};
  int opts[2][2 * MAXP1 + 1][2], no[2];
  for (int dd = 0; dd < 2; dd++) {
    int n = 0;
    opts[dd][n][0] = 0; opts[dd][n][1] = -1; n++;
    for (int s = lo[dd] + 1; s <= hi[dd]; s++) { opts[dd][n][0] = 1; opts[dd][n][1] = s; n++; }
    for (int s = lo[dd] + 1; s <= hi[dd]; s++) { opts[dd][n][0] = 2; opts[dd][n][1] = s; n++; }
    no[dd] = n;
  }
  int best = -1, bestel = 0, bestdisc = 0;
  for (int a = 0; a < no[0]; a++)
    for (int b = 0; b < no[1]; b++) {
      int r0[2], r1[2];
      opt_range(opts[0][a][0], opts[0][a][1], lo[0], hi[0], &r0[0], &r1[0]);
      opt_range(opts[1][b][0], opts[1][b][1], lo[1], hi[1], &r0[1], &r1[1]);
      int ok = 1;
      for (int dd = 0; dd < 2 && ok; dd++) {
        const dirdata *D = &P->D[dd];
        int kind = dd == 0 ? opts[0][a][0] : opts[1][b][0], s = dd == 0 ? opts[0][a][1] : opts[1][b][1];
        if (kind != 0 && !(D->bp[s - 1] < D->bp[s] && D->bp[s] < D->bp[s + 1])) ok = 0;
      }
      for (int e2 = r0[1]; e2 <= r1[1] && ok; e2++)
        for (int e1 = r0[0]; e1 <= r1[0] && ok; e1++) {
          uint8_t st = P->estate[e2 * A->nel + e1];
          if (st != OR_ELEM_REGULAR && st != OR_ELEM_EMPTY) ok = 0;
        }
      if (!ok) continue;
      int nel = (r1[0] - r0[0] + 1) * (r1[1] - r0[1] + 1);
      int disc = (opts[0][a][0] != 0) + (opts[1][b][0] != 0);
      if (best < 0 || nel > bestel || (nel == bestel && disc < bestdisc)) {
        best = a * 64 + b;
        bestel = nel;
        bestdisc = disc;
        out[0] = opts[0][a][0];
        out[1] = opts[0][a][1];
        out[2] = opts[1][b][0];
        out[3] = opts[1][b][1];
      }
    }
  if (best < 0) {
    out[0] = -1; out[1] = out[2] = out[3] = -1;
    return 0;
  }
  return 1;
}

/* ------------------------------------------------------------------ */
/* row rules                                                            */

enum { ROW_WQ = 0, ROW_GAUSS = 1, ROW_DWQ = 2, ROW_NAIVE = 3 };

static int row_kind(const or_patch *P, int g) {
  int m = P->d.method;
  if (m == OR_METHOD_GAUSS) return ROW_GAUSS;
  if (P->fstate[g] == OR_FUNC_INTERIOR) return ROW_WQ;
  if (m == OR_METHOD_HYBRID) return ROW_GAUSS;
  if (m == OR_METHOD_NAIVE) return ROW_NAIVE;
  return P->choice[4 * g] >= 0 ? ROW_DWQ : ROW_GAUSS;
}

static const double *gauss_c(or_patch *P, int e1, int e2) {
  const dirdata *A = &P->D[0], *B = &P->D[1];
  int p1 = A->p + 1, p2 = B->p + 1;
  size_t e = (size_t)e2 * A->nel + e1;
  double *c = P->gc + e * p1 * p2;
  if (!P->gc_done[e]) {
    for (int g2 = 0; g2 < p2; g2++)
      for (int g1 = 0; g1 < p1; g1++) {
        double x1 = A->bp[e1] + (A->bp[e1 + 1] - A->bp[e1]) * 0.5 * (A->gx[g1] + 1.0);
        double x2 = B->bp[e2] + (B->bp[e2 + 1] - B->bp[e2]) * 0.5 * (B->gx[g2] + 1.0);
        c[g2 * p1 + g1] = coef_from(P, x1, x2, e1, A->GBv + ((size_t)e1 * p1 + g1) * p1,
                                    A->GBd + ((size_t)e1 * p1 + g1) * p1, e2,
                                    B->GBv + ((size_t)e2 * p2 + g2) * p2,
                                    B->GBd + ((size_t)e2 * p2 + g2) * p2);
      }
    P->gc_done[e] = 1;
  }
  return c;
}

typedef struct {
  rpoint *v;
  int n, cap;
} rbuf;

static rpoint *rnew(rbuf *b) {
  if (b->n == b->cap) {
    b->cap = b->cap ? 2 * b->cap : 1024;
    b->v = (rpoint *)realloc(b->v, sizeof(rpoint) * (size_t)b->cap);
  }
  return &b->v[b->n++];
}

/* Gauss on a regular element (tensor, p+1 points per direction): the test
 * function B_i is folded into the weight. */
static void add_gauss_elem(or_patch *P, int i1, int i2, int e1, int e2, rbuf *R) {
  const dirdata *A = &P->D[0], *B = &P->D[1];
  int p1 = A->p + 1, p2 = B->p + 1;
  const double *c = gauss_c(P, e1, e2);
  for (int g2 = 0; g2 < p2; g2++)
    for (int g1 = 0; g1 < p1; g1++) {
      const double *v1 = A->GBv + ((size_t)e1 * p1 + g1) * p1;
      const double *v2 = B->GBv + ((size_t)e2 * p2 + g2) * p2;
      double h1 = A->bp[e1 + 1] - A->bp[e1], h2 = B->bp[e2 + 1] - B->bp[e2];
      rpoint *r = rnew(R);
      r->x[0] = A->bp[e1] + h1 * 0.5 * (A->gx[g1] + 1.0);
      r->x[1] = B->bp[e2] + h2 * 0.5 * (B->gx[g2] + 1.0);
      r->e[0] = e1;
      r->e[1] = e2;
      for (int a = 0; a < p1; a++) r->bv[0][a] = v1[a];
      for (int b = 0; b < p2; b++) r->bv[1][b] = v2[b];
      double w = A->gw[g1] * 0.5 * h1 * B->gw[g2] * 0.5 * h2;
      r->wc = w * v1[i1 - e1] * v2[i2 - e2] * c[g2 * p1 + g1];
      r->w = w * v1[i1 - e1] * v2[i2 - e2];
    }
}

static void add_cut_elem(or_patch *P, int i1, int i2, int e1, int e2, rbuf *R) {
  const dirdata *A = &P->D[0], *B = &P->D[1];
  int e = e2 * A->nel + e1;
  for (int64_t k = P->cut_off[e]; k < P->cut_off[e + 1]; k++) {
    rpoint *r = rnew(R);
    r->x[0] = P->cut_pts[3 * k];
    r->x[1] = P->cut_pts[3 * k + 1];
    r->e[0] = e1;
    r->e[1] = e2;
    basis_at(A, e1, r->x[0], r->bv[0], NULL);
    basis_at(B, e2, r->x[1], r->bv[1], NULL);
    r->wc = P->cut_pts[3 * k + 2] * r->bv[0][i1 - e1] * r->bv[1][i2 - e2] * P->cut_c[k];
    r->w = P->cut_pts[3 * k + 2] * r->bv[0][i1 - e1] * r->bv[1][i2 - e2];
  }
}

/* the whole quadrature rule of row g; returns the number of points */
static int row_rule(or_patch *P, int g, rbuf *R) {
  const dirdata *A = &P->D[0], *B = &P->D[1];
  int i1 = g % A->n, i2 = g / A->n;
  int kind = row_kind(P, g);
  int lo1 = i1 - A->p < 0 ? 0 : i1 - A->p, hi1 = i1 < A->nel - 1 ? i1 : A->nel - 1;
  int lo2 = i2 - B->p < 0 ? 0 : i2 - B->p, hi2 = i2 < B->nel - 1 ? i2 : B->nel - 1;
  int rg0[2] = {1, 1}, rg1[2] = {0, 0}; /* region R (empty by default) */
  R->n = 0;
  int p1 = A->p + 1, p2 = B->p + 1;
  if (kind == ROW_WQ || kind == ROW_NAIVE) {
    for (int k2 = B->qlo[i2]; k2 <= B->qhi[i2]; k2++) {
      double w2 = B->W[(size_t)i2 * B->nq + k2];
      for (int k1 = A->qlo[i1]; k1 <= A->qhi[i1]; k1++) {
        double w1 = A->W[(size_t)i1 * A->nq + k1];
        double c = P->C[(size_t)k2 * A->nq + k1];
        int masked = kind == ROW_NAIVE &&
                     P->estate[B->qel[k2] * A->nel + A->qel[k1]] != OR_ELEM_REGULAR;
        if (masked) c = 0.0;
        rpoint *r = rnew(R);
        r->x[0] = A->xq[k1];
        r->x[1] = B->xq[k2];
        r->e[0] = A->qel[k1];
        r->e[1] = B->qel[k2];
        for (int a = 0; a < p1; a++) r->bv[0][a] = A->Bv[(size_t)k1 * p1 + a];
        for (int b = 0; b < p2; b++) r->bv[1][b] = B->Bv[(size_t)k2 * p2 + b];
        r->wc = w1 * w2 * c;
        r->w = masked ? 0.0 : w1 * w2;
      }
    }
    if (kind == ROW_NAIVE) {
      for (int e2 = lo2; e2 <= hi2; e2++)
        for (int e1 = lo1; e1 <= hi1; e1++)
          if (P->estate[e2 * A->nel + e1] == OR_ELEM_CUT) add_cut_elem(P, i1, i2, e1, e2, R);
    }
    return R->n;
  }
  if (kind == ROW_DWQ) {
    const int *ch = P->choice + 4 * g;
    int rlo[2] = {lo1, lo2}, rhi[2] = {hi1, hi2}, ii[2] = {i1, i2};
    double *rp[2];
    int rn[2];
    for (int dd = 0; dd < 2; dd++) {
      const dirdata *D = &P->D[dd];
      opt_range(ch[2 * dd], ch[2 * dd + 1], rlo[dd], rhi[dd], &rg0[dd], &rg1[dd]);
      rp[dd] = (double *)malloc(sizeof(double) * 2 * (size_t)(D->nq + 2 * MAXP1));
      if (ch[2 * dd] == 0) {
        int n = 0;
        for (int k = 0; k < D->nq; k++)
          if (D->xq[k] > D->U[ii[dd]] && D->xq[k] < D->U[ii[dd] + D->p + 1]) {
            rp[dd][2 * n] = D->xq[k];
            rp[dd][2 * n + 1] = D->W[(size_t)ii[dd] * D->nq + k];
            n++;
          }
        rn[dd] = n;
      } else {
        rn[dd] = or_dwq_rule(P, dd, ch[2 * dd + 1], ch[2 * dd] == 1 ? 0 : 1, ii[dd], rp[dd],
                             D->nq + 2 * MAXP1);
      }
    }
    for (int b = 0; b < rn[1]; b++)
      for (int a = 0; a < rn[0]; a++) {
        rpoint *r = rnew(R);
        r->x[0] = rp[0][2 * a];
        r->x[1] = rp[1][2 * b];
        r->e[0] = elem_of(A, r->x[0]);
        r->e[1] = elem_of(B, r->x[1]);
        double d1[MAXP1], d2[MAXP1];
        basis_at(A, r->e[0], r->x[0], r->bv[0], d1);
        basis_at(B, r->e[1], r->x[1], r->bv[1], d2);
        double c = coef_from(P, r->x[0], r->x[1], r->e[0], r->bv[0], d1, r->e[1], r->bv[1], d2);
        r->wc = rp[0][2 * a + 1] * rp[1][2 * b + 1] * c;
        r->w = rp[0][2 * a + 1] * rp[1][2 * b + 1];
      }
    free(rp[0]);
    free(rp[1]);
  }
  /* Gauss on the regular elements outside R, cut rule on cut elements */
  for (int e2 = lo2; e2 <= hi2; e2++)
    for (int e1 = lo1; e1 <= hi1; e1++) {
      uint8_t st = P->estate[e2 * A->nel + e1];
      int inR = e1 >= rg0[0] && e1 <= rg1[0] && e2 >= rg0[1] && e2 <= rg1[1];
      if (st == OR_ELEM_REGULAR && !inR) add_gauss_elem(P, i1, i2, e1, e2, R);
      else if (st == OR_ELEM_CUT) add_cut_elem(P, i1, i2, e1, e2, R);
    }
  return R->n;
}

static double rule_apply(const rbuf *R, int p1, int p2, int j1, int j2) {
  double s = 0.0;
  for (int k = 0; k < R->n; k++) {
    const rpoint *r = &R->v[k];
    int a = j1 - r->e[0], b = j2 - r->e[1];
    if (a < 0 || b < 0 || a > p1 || b > p2) continue;
    s += r->wc * r->bv[0][a] * r->bv[1][b];
  }
  return s;
}

/* ------------------------------------------------------------------ */

or_patch *or_create(const or_desc *d) {
  or_patch *P = (or_patch *)calloc(1, sizeof(or_patch));
  P->d = *d;
  int n[2];
  for (int dd = 0; dd < 2; dd++) n[dd] = d->nknots[dd] - d->p[dd] - 1;
  P->d.trim_ctrl = dup(P, d->trim_ctrl, d->trim_kind == OR_TRIM_BSPLINE3 ? 2 * (size_t)d->trim_nctrl : 0);
  /* the curves, each as a copy of the descriptor with that curve in the trim fields */
  P->ncurves = 1;
  P->cd[0] = P->d;
  for (int k = 0; k < d->trim_nextra && P->ncurves < OR_MAXCURVES; k++) {
    const or_trim *t = &d->trim_extra[k];
    or_desc c = P->d;
    c.trim_kind = t->kind;
    c.trim_keep_inside = t->keep_inside;
    for (int m = 0; m < 6; m++) c.trim_params[m] = t->params[m];
    c.trim_nctrl = t->nctrl;
    c.trim_ctrl = dup(P, t->ctrl, t->kind == OR_TRIM_BSPLINE3 ? 2 * (size_t)t->nctrl : 0);
    P->cd[P->ncurves++] = c;
  }
  P->d.trim_nextra = 0;
  P->d.trim_extra = NULL;
  P->d.geom_ctrl = dup(P, d->geom_ctrl, d->geom_kind == OR_GEOM_SPLINE ? 2 * (size_t)n[0] * n[1] : 0);
  if (d->coef_kind == OR_COEF_DENSITY) {
    for (int dd = 0; dd < 2; dd++) P->d.dens_knots[dd] = dup(P, d->dens_knots[dd], (size_t)d->dens_nknots[dd]);
    size_t m = (size_t)(d->dens_nknots[0] - d->dens_p[0] - 1) * (d->dens_nknots[1] - d->dens_p[1] - 1);
    P->d.dens_coef = dup(P, d->dens_coef, m);
  }
  for (int dd = 0; dd < 2; dd++) setup_dir(P, dd);
  for (int dd = 0; dd < 2; dd++) P->d.knots[dd] = P->D[dd].U;
  P->qc = d->cut_order > 0 ? d->cut_order : (d->p[0] > d->p[1] ? d->p[0] : d->p[1]) + 1;
  const dirdata *A = &P->D[0], *B = &P->D[1];
  P->C = (double *)malloc(sizeof(double) * (size_t)A->nq * B->nq);
#pragma omp parallel for schedule(static)
  for (int k2 = 0; k2 < B->nq; k2++)
    for (int k1 = 0; k1 < A->nq; k1++)
      P->C[(size_t)k2 * A->nq + k1] =
          coef_from(P, A->xq[k1], B->xq[k2], A->qel[k1], A->Bv + (size_t)k1 * (A->p + 1),
                    A->Bd + (size_t)k1 * (A->p + 1), B->qel[k2], B->Bv + (size_t)k2 * (B->p + 1),
                    B->Bd + (size_t)k2 * (B->p + 1));
  classify(P);
  build_cut_rules(P);
  size_t ne = (size_t)A->nel * B->nel;
  P->gc = (double *)malloc(sizeof(double) * ne * (A->p + 1) * (B->p + 1));
  P->gc_done = (uint8_t *)calloc(ne, 1);
  P->choice = (int *)malloc(sizeof(int) * 4 * (size_t)A->n * B->n);
#pragma omp parallel for schedule(dynamic, 64)
  for (int g = 0; g < A->n * B->n; g++) {
    P->choice[4 * g] = -1;
    if (d->method == OR_METHOD_DWQ && P->fstate[g] == OR_FUNC_CUT)
      or_dwq_choice(P, g % A->n, g / A->n, P->choice + 4 * g);
  }
  return P;
}

void or_destroy(or_patch *P) {
  if (!P) return;
  for (int dd = 0; dd < 2; dd++) free_dir(&P->D[dd]);
  for (int k = 0; k < P->nown; k++) free(P->own[k]);
  free(P->estate);
  free(P->fstate);
  free(P->act);
  free(P->rowg);
  free(P->C);
  free(P->cut_off);
  free(P->cut_pts);
  free(P->cut_c);
  free(P->gc);
  free(P->gc_done);
  free(P->choice);
  free(P);
}

int or_dims(const or_patch *P, int64_t *out) {
  out[0] = P->D[0].n;
  out[1] = P->D[1].n;
  out[2] = P->D[0].nel;
  out[3] = P->D[1].nel;
  out[4] = P->D[0].nq;
  out[5] = P->D[1].nq;
  out[6] = P->nrows;
  out[7] = P->nnz;
  return 0;
}

void or_states(const or_patch *P, uint8_t *estate, uint8_t *fstate, int32_t *act) {
  size_t ne = (size_t)P->D[0].nel * P->D[1].nel, nf = (size_t)P->D[0].n * P->D[1].n;
  if (estate) memcpy(estate, P->estate, ne);
  if (fstate) memcpy(fstate, P->fstate, nf);
  if (act) memcpy(act, P->act, nf * sizeof(int32_t));
}

void or_wq_grid(const or_patch *P, int dir, double *x) {
  memcpy(x, P->D[dir].xq, sizeof(double) * (size_t)P->D[dir].nq);
}

void or_cgrid(const or_patch *P, double *C) {
  memcpy(C, P->C, sizeof(double) * (size_t)P->D[0].nq * P->D[1].nq);
}

/* one CSR row: columns = active j with |i_d - j_d| <= p_d, ascending (R11) */
int or_form_row(const or_patch *Pc, int64_t row, int32_t *col, double *val) {
  or_patch *P = (or_patch *)Pc;
  const dirdata *A = &P->D[0], *B = &P->D[1];
  int g = (int)P->rowg[row];
  int i1 = g % A->n, i2 = g / A->n;
  rbuf R = {0};
  row_rule(P, g, &R);
  int n = 0;
  for (int j2 = i2 - B->p; j2 <= i2 + B->p; j2++)
    for (int j1 = i1 - A->p; j1 <= i1 + A->p; j1++) {
      if (j1 < 0 || j2 < 0 || j1 >= A->n || j2 >= B->n) continue;
      int32_t a = P->act[j2 * A->n + j1];
      if (a < 0) continue;
      if (col) col[n] = a;
      if (val) val[n] = rule_apply(&R, A->p, B->p, j1, j2);
      n++;
    }
  free(R.v);
  return n;
}

/* Remark 1 of Sect. 3.2: the Gauss part of a cut row written as one tensor rule
 * over the whole support, the element Gauss points of every support element
 * with the coefficient c set to zero at the points outside S^r (the regular
 * elements); the cut elements keep their cut rule.  For rows without a region
 * part (hybrid Gauss rows, Gauss-method rows, DWQ rows without a region) the
 * result is the row of or_form_row summed in another order.  Returns the
 * number of entries, or -1 for a row with a region part. */
int or_form_row_remark1(const or_patch *Pc, int64_t row, int32_t *col, double *val) {
  or_patch *P = (or_patch *)Pc;
  const dirdata *A = &P->D[0], *B = &P->D[1];
  int g = (int)P->rowg[row];
  int kind = row_kind(P, g);
  if (kind != ROW_GAUSS) return -1;
  int i1 = g % A->n, i2 = g / A->n;
  int lo1 = i1 - A->p < 0 ? 0 : i1 - A->p, hi1 = i1 < A->nel - 1 ? i1 : A->nel - 1;
  int lo2 = i2 - B->p < 0 ? 0 : i2 - B->p, hi2 = i2 < B->nel - 1 ? i2 : B->nel - 1;
  int p1 = A->p + 1, p2 = B->p + 1;
  rbuf R = {0};
  for (int e2 = lo2; e2 <= hi2; e2++)
    for (int e1 = lo1; e1 <= hi1; e1++) {
      const int reg = P->estate[e2 * A->nel + e1] == OR_ELEM_REGULAR;
      const double *c = reg ? gauss_c(P, e1, e2) : NULL;
      double h1 = A->bp[e1 + 1] - A->bp[e1], h2 = B->bp[e2 + 1] - B->bp[e2];
      for (int g2 = 0; g2 < p2; g2++)
        for (int g1 = 0; g1 < p1; g1++) {
          const double *v1 = A->GBv + ((size_t)e1 * p1 + g1) * p1;
          const double *v2 = B->GBv + ((size_t)e2 * p2 + g2) * p2;
          rpoint *r = rnew(&R);
          r->x[0] = A->bp[e1] + h1 * 0.5 * (A->gx[g1] + 1.0);
          r->x[1] = B->bp[e2] + h2 * 0.5 * (B->gx[g2] + 1.0);
          r->e[0] = e1;
          r->e[1] = e2;
          for (int a = 0; a < p1; a++) r->bv[0][a] = v1[a];
          for (int b = 0; b < p2; b++) r->bv[1][b] = v2[b];
          double w = A->gw[g1] * 0.5 * h1 * B->gw[g2] * 0.5 * h2 * v1[i1 - e1] * v2[i2 - e2];
          r->wc = reg ? w * c[g2 * p1 + g1] : 0.0; /* c set to zero off S^r */
          r->w = reg ? w : 0.0;
        }
    }
  for (int e2 = lo2; e2 <= hi2; e2++)
    for (int e1 = lo1; e1 <= hi1; e1++)
      if (P->estate[e2 * A->nel + e1] == OR_ELEM_CUT) add_cut_elem(P, i1, i2, e1, e2, &R);
  int n = 0;
  for (int j2 = i2 - B->p; j2 <= i2 + B->p; j2++)
    for (int j1 = i1 - A->p; j1 <= i1 + A->p; j1++) {
      if (j1 < 0 || j2 < 0 || j1 >= A->n || j2 >= B->n) continue;
      int32_t a = P->act[j2 * A->n + j1];
      if (a < 0) continue;
      if (col) col[n] = a;
      if (val) val[n] = rule_apply(&R, A->p, B->p, j1, j2);
      n++;
    }
  free(R.v);
  return n;
}

/* Rows rows[0..n) of the matrix, row k's values at val + k * (2p+1)^2 and its
 * entry count in cnt[k].  The rows are independent: with OpenMP (the oracle's
 * all-cores build) they are formed in parallel.  The lazily filled table of c
 * at the element Gauss points is filled first for the regular elements that
 * these rows' Gauss parts use (the ones row-by-row formation would fill), so
 * that the rows only read shared state. */
void or_form_rows(const or_patch *Pc, const int64_t *rows, int64_t n, double *val, int *cnt) {
  or_patch *P = (or_patch *)Pc;
  const dirdata *A = &P->D[0], *B = &P->D[1];
  const int ne = A->nel * B->nel;
  uint8_t *need = (uint8_t *)calloc((size_t)ne, 1);
  for (int64_t k = 0; k < n; k++) {
    const int g = (int)P->rowg[rows[k]];
    const int kind = row_kind(P, g);
    if (kind != ROW_GAUSS && kind != ROW_DWQ) continue;
    const int i1 = g % A->n, i2 = g / A->n;
    for (int e2 = i2 - B->p; e2 <= i2; e2++)
      for (int e1 = i1 - A->p; e1 <= i1; e1++)
        if (e1 >= 0 && e2 >= 0 && e1 < A->nel && e2 < B->nel &&
            P->estate[e2 * A->nel + e1] == OR_ELEM_REGULAR)
          need[e2 * A->nel + e1] = 1;
  }
#pragma omp parallel for schedule(dynamic, 64)
  for (int e = 0; e < ne; e++)
    if (need[e]) gauss_c(P, e % A->nel, e / A->nel);
  free(need);
  const int64_t w = (int64_t)(2 * A->p + 1) * (2 * B->p + 1);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < n; k++) cnt[k] = or_form_row(P, rows[k], NULL, val + k * w);
}

/* threads the parallel loops use (1 in the single-thread build) */
int or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_form(const or_patch *P, int64_t *row_ptr, int32_t *col, double *val) {
  int64_t pos = 0;
  row_ptr[0] = 0;
  for (int64_t r = 0; r < P->nrows; r++) {
    pos += or_form_row(P, r, col + pos, val + pos);
    row_ptr[r + 1] = pos;
  }
}

/* ------------------------------------------------------------------ */
/* L2 projection (Sect. 4.2; readings R9, R10)                         */

static double func_eval(const or_func *f, const double *xi, const double *X) {
  switch (f->kind) {
    case OR_FUNC_SPLINE: {
      int m1 = f->nknots[0] - f->p[0] - 1, m2 = f->nknots[1] - f->p[1] - 1;
      double s = 0.0;
      for (int k2 = 0; k2 < m2; k2++) {
        double b2 = or_bspline(f->knots[1], f->nknots[1], f->p[1], k2, xi[1]);
        if (b2 == 0.0) continue;
        for (int k1 = 0; k1 < m1; k1++)
          s += f->coef[k2 * m1 + k1] * or_bspline(f->knots[0], f->nknots[0], f->p[0], k1, xi[0]) * b2;
      }
      return s;
    }
    case OR_FUNC_SINSIN: return sin(f->prm[0] * X[0]) * sin(f->prm[1] * X[1]);
    case OR_FUNC_SINCOS: return sin(f->prm[0] * X[0]) * cos(f->prm[1] * X[1]);
    case OR_FUNC_GAUSS: {
      double dx = X[0] - f->prm[1], dy = X[1] - f->prm[2];
      return exp(-f->prm[0] * (dx * dx + dy * dy));
    }
  }
  return 0.0;
}

/* R9: b_i is the row's own rule applied to f (times c) */
void or_rhs(const or_patch *Pc, const or_func *f, double *b) {
  or_patch *P = (or_patch *)Pc;
  rbuf R = {0};
  for (int64_t r = 0; r < P->nrows; r++) {
    row_rule(P, (int)P->rowg[r], &R);
    double s = 0.0;
    for (int k = 0; k < R.n; k++) {
      const rpoint *q = &R.v[k];
      double X[2];
      phys_from(P, q->x[0], q->x[1], q->e[0], q->bv[0], q->e[1], q->bv[1], X);
      s += q->wc * func_eval(f, q->x, X);
    }
    b[r] = s;
  }
  free(R.v);
}

int or_row_points(const or_patch *Pc, int64_t row, double *out, int cap) {
  or_patch *P = (or_patch *)Pc;
  rbuf R = {0};
  int n = row_rule(P, (int)P->rowg[row], &R);
  for (int k = 0; k < n && k < cap; k++) {
    const rpoint *q = &R.v[k];
    double X[2];
    phys_from(P, q->x[0], q->x[1], q->e[0], q->bv[0], q->e[1], q->bv[1], X);
    out[5 * k] = q->x[0];
    out[5 * k + 1] = q->x[1];
    out[5 * k + 2] = X[0];
    out[5 * k + 3] = X[1];
    out[5 * k + 4] = q->wc;
  }
  free(R.v);
  return n;
}

static int64_t find_pos(const int64_t *rp, const int32_t *col, int64_t r, int32_t c) {
  int64_t lo = rp[r], hi = rp[r + 1] - 1;
  while (lo <= hi) {
    int64_t m = (lo + hi) / 2;
    if (col[m] == c) return m;
    if (col[m] < c) lo = m + 1;
    else hi = m - 1;
  }
  return -1;
}

static double dotv(const double *a, const double *b, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
  return s;
}

/* R10: Jacobi-preconditioned CG on M_s = (M + M^T)/2 until ||r||/||b|| <= tol */
int or_cg(const or_patch *P, const int64_t *rp, const int32_t *col, const double *val,
          const double *b, double *u, double tol, int maxit, double *relres) {
  int64_t N = P->nrows, nnz = rp[N];
  double *ms = (double *)malloc(sizeof(double) * (size_t)nnz);
  double *dg = (double *)malloc(sizeof(double) * (size_t)N);
  for (int64_t r = 0; r < N; r++)
    for (int64_t k = rp[r]; k < rp[r + 1]; k++) {
      int64_t t = find_pos(rp, col, col[k], (int32_t)r);
      ms[k] = 0.5 * (val[k] + val[t]);
      if (col[k] == r) dg[r] = ms[k];
    }
  double *r = (double *)malloc(sizeof(double) * (size_t)N);
  double *z = (double *)malloc(sizeof(double) * (size_t)N);
  double *pv = (double *)malloc(sizeof(double) * (size_t)N);
  double *q = (double *)malloc(sizeof(double) * (size_t)N);
  for (int64_t i = 0; i < N; i++) {
    u[i] = 0.0;
    r[i] = b[i];
    z[i] = r[i] / dg[i];
    pv[i] = z[i];
  }
  double bn = sqrt(dotv(b, b, N));
  double rz = dotv(r, z, N);
  int it = 0;
  double rel = bn > 0 ? sqrt(dotv(r, r, N)) / bn : 0.0;
  while (rel > tol && it < maxit) {
    for (int64_t i = 0; i < N; i++) {
      double s = 0.0;
      for (int64_t k = rp[i]; k < rp[i + 1]; k++) s += ms[k] * pv[col[k]];
      q[i] = s;
    }
    double alpha = rz / dotv(pv, q, N);
    for (int64_t i = 0; i < N; i++) {
      u[i] += alpha * pv[i];
      r[i] -= alpha * q[i];
      z[i] = r[i] / dg[i];
    }
    double rz2 = dotv(r, z, N);
    for (int64_t i = 0; i < N; i++) pv[i] = z[i] + rz2 / rz * pv[i];
    rz = rz2;
    it++;
    rel = sqrt(dotv(r, r, N)) / bn;
  }
  if (relres) *relres = rel;
  free(ms);
  free(dg);
  free(r);
  free(z);
  free(pv);
  free(q);
  return it;
}

/* Relative L2(Omega^v) error of u_h = sum_j u_j B_j against f, measured with
 * Gauss (p+2 points) on regular elements and the cut rule on cut elements,
 * in physical measure (times det J). */
double or_l2_error(const or_patch *Pc, const double *u, const or_func *f, double *fnorm) {
  or_patch *P = (or_patch *)Pc;
  const dirdata *A = &P->D[0], *B = &P->D[1];
  int q1 = A->p + 2, q2 = B->p + 2;
  double gx1[16], gw1[16], gx2[16], gw2[16];
  or_gauss_legendre(q1, gx1, gw1);
  or_gauss_legendre(q2, gx2, gw2);
  double err = 0.0, nrm = 0.0;
  for (int e2 = 0; e2 < B->nel; e2++)
    for (int e1 = 0; e1 < A->nel; e1++) {
      uint8_t st = P->estate[e2 * A->nel + e1];
      if (st == OR_ELEM_INVISIBLE || st == OR_ELEM_EMPTY) continue;
      rbuf R = {0};
      if (st == OR_ELEM_REGULAR) {
        double h1 = A->bp[e1 + 1] - A->bp[e1], h2 = B->bp[e2 + 1] - B->bp[e2];
        for (int g2 = 0; g2 < q2; g2++)
          for (int g1 = 0; g1 < q1; g1++) {
            rpoint *r = rnew(&R);
            r->x[0] = A->bp[e1] + h1 * 0.5 * (gx1[g1] + 1.0);
            r->x[1] = B->bp[e2] + h2 * 0.5 * (gx2[g2] + 1.0);
            r->wc = gw1[g1] * 0.5 * h1 * gw2[g2] * 0.5 * h2;
          }
      } else {
        int e = e2 * A->nel + e1;
        for (int64_t k = P->cut_off[e]; k < P->cut_off[e + 1]; k++) {
          rpoint *r = rnew(&R);
          r->x[0] = P->cut_pts[3 * k];
          r->x[1] = P->cut_pts[3 * k + 1];
          r->wc = P->cut_pts[3 * k + 2];
        }
      }
      for (int k = 0; k < R.n; k++) {
        rpoint *r = &R.v[k];
        double v1[MAXP1], d1[MAXP1], v2[MAXP1], d2[MAXP1];
        basis_at(A, e1, r->x[0], v1, d1);
        basis_at(B, e2, r->x[1], v2, d2);
        double uh = 0.0;
        for (int b = 0; b <= B->p; b++)
          for (int a = 0; a <= A->p; a++) {
            int32_t ac = P->act[(e2 + b) * A->n + (e1 + a)];
            if (ac >= 0) uh += u[ac] * v1[a] * v2[b];
          }
        double X[2];
        phys_from(P, r->x[0], r->x[1], e1, v1, e2, v2, X);
        double fv = func_eval(f, r->x, X);
        double dj = 1.0;
        if (P->d.geom_kind == OR_GEOM_SPLINE) {
          int sv = P->d.coef_kind;
          P->d.coef_kind = OR_COEF_DETJ;
          dj = coef_from(P, r->x[0], r->x[1], e1, v1, d1, e2, v2, d2);
          P->d.coef_kind = sv;
        }
        err += r->wc * dj * (uh - fv) * (uh - fv);
        nrm += r->wc * dj * fv * fv;
      }
      free(R.v);
    }
  if (fnorm) *fnorm = sqrt(nrm);
  return nrm > 0 ? sqrt(err / nrm) : sqrt(err);
}

/* parameter-space area of Omega^v: regular elements plus cut-rule weights */
double or_visible_area(const or_patch *P) {
  const dirdata *A = &P->D[0], *B = &P->D[1];
  double s = 0.0;
  for (int e2 = 0; e2 < B->nel; e2++)
    for (int e1 = 0; e1 < A->nel; e1++) {
      int e = e2 * A->nel + e1;
      if (P->estate[e] == OR_ELEM_REGULAR)
        s += (A->bp[e1 + 1] - A->bp[e1]) * (B->bp[e2 + 1] - B->bp[e2]);
      else if (P->estate[e] == OR_ELEM_CUT)
        for (int64_t k = P->cut_off[e]; k < P->cut_off[e + 1]; k++) s += P->cut_pts[3 * k + 2];
    }
  return s;
}

/* ------------------------------------------------------------------ */
/* differentiation of the L2 projection w.r.t. the density (reading R12) */

static double detj_at(const or_patch *P, int e1, const double *v1, const double *d1, int e2,
                      const double *v2, const double *d2) {
  if (P->d.geom_kind != OR_GEOM_SPLINE) return 1.0;
  int n1 = P->D[0].n;
  double xa = 0, xb = 0, ya = 0, yb = 0;
  for (int b = 0; b <= P->D[1].p; b++)
    for (int a = 0; a <= P->D[0].p; a++) {
      const double *pt = P->d.geom_ctrl + 2 * ((size_t)(e2 + b) * n1 + (e1 + a));
      xa += pt[0] * d1[a] * v2[b];
      ya += pt[1] * d1[a] * v2[b];
      xb += pt[0] * v1[a] * d2[b];
      yb += pt[1] * v1[a] * d2[b];
    }
  return xa * yb - xb * ya;
}

/* spline value sum_j a_j B_j(x) over the active functions j */
static double active_spline(const or_patch *P, const double *a, int e1, const double *v1, int e2,
                            const double *v2) {
  const dirdata *A = &P->D[0];
  double s = 0.0;
  for (int b = 0; b <= P->D[1].p; b++)
    for (int c = 0; c <= A->p; c++) {
      int32_t r = P->act[(e2 + b) * A->n + (e1 + c)];
      if (r >= 0) s += a[r] * v1[c] * v2[b];
    }
  return s;
}

/* L = sum_q omega_q detJ (u_h - g)^2 over Omega^v: element Gauss (p+1 per
 * direction) on regular elements, the cut rule on cut elements; and
 * dL/du_j = 2 sum_q omega_q detJ (u_h - g) B_j. */
double or_loss(const or_patch *Pc, const double *u, const or_func *g, double *dLdu) {
  or_patch *P = (or_patch *)Pc;
  const dirdata *A = &P->D[0], *B = &P->D[1];
  int p1 = A->p + 1, p2 = B->p + 1;
  double L = 0.0;
  for (int64_t r = 0; r < P->nrows; r++) dLdu[r] = 0.0;
  for (int e2 = 0; e2 < B->nel; e2++)
    for (int e1 = 0; e1 < A->nel; e1++) {
      int e = e2 * A->nel + e1;
      uint8_t st = P->estate[e];
      if (st == OR_ELEM_INVISIBLE || st == OR_ELEM_EMPTY) continue;
      int np = st == OR_ELEM_REGULAR ? p1 * p2 : (int)(P->cut_off[e + 1] - P->cut_off[e]);
      for (int q = 0; q < np; q++) {
        double x[2], om;
        if (st == OR_ELEM_REGULAR) {
          int g1 = q % p1, g2 = q / p1;
          double h1 = A->bp[e1 + 1] - A->bp[e1], h2 = B->bp[e2 + 1] - B->bp[e2];
          x[0] = A->bp[e1] + h1 * 0.5 * (A->gx[g1] + 1.0);
          x[1] = B->bp[e2] + h2 * 0.5 * (B->gx[g2] + 1.0);
          om = A->gw[g1] * 0.5 * h1 * B->gw[g2] * 0.5 * h2;
        } else {
          int64_t k = P->cut_off[e] + q;
          x[0] = P->cut_pts[3 * k];
          x[1] = P->cut_pts[3 * k + 1];
          om = P->cut_pts[3 * k + 2];
        }
        double v1[MAXP1], d1[MAXP1], v2[MAXP1], d2[MAXP1], X[2];
        basis_at(A, e1, x[0], v1, d1);
        basis_at(B, e2, x[1], v2, d2);
        double dj = detj_at(P, e1, v1, d1, e2, v2, d2);
        phys_from(P, x[0], x[1], e1, v1, e2, v2, X);
        double res = active_spline(P, u, e1, v1, e2, v2) - func_eval(g, x, X);
        L += om * dj * res * res;
        for (int b = 0; b < p2; b++)
          for (int a = 0; a < p1; a++) {
            int32_t r = P->act[(e2 + b) * A->n + (e1 + a)];
            if (r >= 0) dLdu[r] += 2.0 * om * dj * res * v1[a] * v2[b];
          }
      }
    }
  return L;
}

/* dL/dd_k = lambda^T (db/dd_k - dM_s/dd_k u) with M_s lambda = dL/du:
 * sum over rows i and their rule points q of w_q detJ N_k(x_q)
 * [lambda_i g - lambda_i U / 2 - u_i Lambda / 2](x_q), U = sum u_j B_j and
 * Lambda = sum lambda_j B_j over the active j, w_q the row's weight without c. */
void or_density_grad(const or_patch *Pc, const double *u, const double *lam, const or_func *g,
                     double *grad) {
  or_patch *P = (or_patch *)Pc;
  const dirdata *A = &P->D[0], *B = &P->D[1];
  const or_desc *d = &P->d;
  int m1 = d->dens_nknots[0] - d->dens_p[0] - 1, m2 = d->dens_nknots[1] - d->dens_p[1] - 1;
  for (int k = 0; k < m1 * m2; k++) grad[k] = 0.0;
  rbuf R = {0};
  for (int64_t row = 0; row < P->nrows; row++) {
    int gi = (int)P->rowg[row];
    row_rule(P, gi, &R);
    for (int q = 0; q < R.n; q++) {
      rpoint *r = &R.v[q];
      if (r->w == 0.0) continue;
      double v1[MAXP1], d1[MAXP1], v2[MAXP1], d2[MAXP1], X[2];
      basis_at(A, r->e[0], r->x[0], v1, d1);
      basis_at(B, r->e[1], r->x[1], v2, d2);
      double dj = detj_at(P, r->e[0], v1, d1, r->e[1], v2, d2);
      phys_from(P, r->x[0], r->x[1], r->e[0], v1, r->e[1], v2, X);
      double U = active_spline(P, u, r->e[0], v1, r->e[1], v2);
      double Lm = active_spline(P, lam, r->e[0], v1, r->e[1], v2);
      double h = lam[row] * func_eval(g, r->x, X) - 0.5 * lam[row] * U - 0.5 * u[row] * Lm;
      double wh = r->w * dj * h;
      for (int k2 = 0; k2 < m2; k2++) {
        double b2 = or_bspline(d->dens_knots[1], d->dens_nknots[1], d->dens_p[1], k2, r->x[1]);
        if (b2 == 0.0) continue;
        for (int k1 = 0; k1 < m1; k1++) {
          double b1 = or_bspline(d->dens_knots[0], d->dens_nknots[0], d->dens_p[0], k1, r->x[0]);
          if (b1 != 0.0) grad[k2 * m1 + k1] += wh * b1 * b2;
        }
      }
    }
  }
  free(R.v);
}
