/*
 * oracle.h -- plain, slow FP64 CPU oracle for the formation of trimmed
 * isogeometric mass matrices by weighted quadrature (Marussig, "Fast formation
 * and assembly of isogeometric Galerkin matrices for trimmed patches").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference arm use it.  It shares no code with the CUDA path.
 *
 * Every routine follows the paper's definitions step by step:
 *   Sect. 2.1, Eq. 1        tensor-product B-splines (Cox-de Boor recursion)
 *   Sect. 2.1, Eqs. 3-5     weighted quadrature (one rule per test function,
 *                           min-norm solution of the exactness system)
 *   Sect. 2.1, Eqs. 6-7     mass entry m_ij = int B_i B_j c
 *   Sect. 2.2               trimming curve, exterior / interior / cut functions
 *   Sect. 3, Eq. 8          splitting of the support into S^r and S^t
 *   Sect. 3.1               higher-order cut-element quadrature (own reading)
 *   Sect. 3.2               hybrid Gauss for S^r of cut functions
 *   Sect. 3.3, Eqs. 9-10    discontinuous weighted quadrature (knot insertion)
 *   Sect. 4.2               L2 projection
 * Where the paper is silent, a reading (R1..R14) is taken; each is stated at
 * the routine that applies it.
 *
 * Parity status: every function is pinned by tests/test_oracle_*.py against
 * closed forms, brute force or textbook special cases, except the c = det J
 * rules on cut functions, whose point layout is our own reading (parity
 * unpinned beyond "equals element Gauss when c = 1").
 */
#ifndef TW_ORACLE_H
#define TW_ORACLE_H

#include <stdint.h>

/* Descriptor enums: the same values as the C-ABI (an interface that has to
 * agree between the two sides; the numbers are the contract, not shared code). */
#define OR_TRIM_NONE 0
#define OR_TRIM_CIRCLE 1   /* prm: cx, cy, r                     */
#define OR_TRIM_ELLIPSE 2  /* prm: cx, cy, a, b, phi             */
#define OR_TRIM_BSPLINE3 3 /* periodic uniform cubic, nctrl x 2  */
#define OR_TRIM_LINE 4     /* prm: x0, y0, x1, y1; "inside" = the half-plane left of (x0,y0)->(x1,y1) */

#define OR_GEOM_IDENTITY 0
#define OR_GEOM_SPLINE 1   /* control net in the patch basis, (i2*n1+i1)*2+comp */

#define OR_COEF_ONE 0      /* c = 1                               */
#define OR_COEF_DETJ 1     /* c = det J                           */
#define OR_COEF_DENSITY 2  /* c = rho(xi) * det J, rho a spline   */

#define OR_METHOD_GAUSS 0  /* element-wise Gauss everywhere (reference)     */
#define OR_METHOD_HYBRID 1 /* WQ interior rows, Gauss on S^r of cut rows    */
#define OR_METHOD_DWQ 2    /* WQ interior rows, DWQ (+Gauss rest) cut rows  */
#define OR_METHOD_NAIVE 3  /* WQ with c zeroed off S^r (negative control)   */

#define OR_FUNC_SPLINE 0   /* f = sum a_k N_k(xi), own tensor spline space */
#define OR_FUNC_SINSIN 1   /* f = sin(a x) sin(b y), physical x            */
#define OR_FUNC_SINCOS 2   /* f = sin(a x) cos(b y)                        */
#define OR_FUNC_GAUSS 3    /* f = exp(-k |x - (x0,y0)|^2), prm k,x0,y0     */

#define OR_ELEM_INVISIBLE 0
#define OR_ELEM_REGULAR 1
#define OR_ELEM_CUT 2
#define OR_ELEM_EMPTY 3 /* a zero-length span of a repeated knot: no measure */
#define OR_FUNC_EXTERIOR 0
#define OR_FUNC_INTERIOR 1
#define OR_FUNC_CUT 2

/* one more trimming curve of a patch (same fields as the descriptor's first) */
typedef struct {
  int kind;
  int keep_inside;
  double params[6];
  int nctrl;
  const double *ctrl;
} or_trim;

#define OR_MAXCURVES 8

typedef struct {
  int p[2];
  int nknots[2];
  const double *knots[2];
  int trim_kind;
  int trim_keep_inside; /* 0: the curve bounds a hole, 1: keep the inside */
  double trim_params[6];
  int trim_nctrl;
  const double *trim_ctrl;
  int geom_kind;
  const double *geom_ctrl;
  int coef_kind;
  int dens_p[2];
  int dens_nknots[2];
  const double *dens_knots[2];
  const double *dens_coef; /* (k2*m1 + k1) */
  int method;
  int cut_order; /* Gauss order on cut-element pieces; 0 -> p+1 */
  /* further trimming curves (at most OR_MAXCURVES - 1): the visible domain is
   * the intersection of every curve's kept side (outside for a hole, inside
   * for keep_inside) */
  int trim_nextra;
  const or_trim *trim_extra;
} or_desc;

typedef struct {
  int kind;
  double prm[4];
  int p[2];
  int nknots[2];
  const double *knots[2];
  const double *coef;
} or_func;

typedef struct or_patch or_patch;

/* ---- univariate building blocks (pinned individually) ---- */
double or_bspline(const double *U, int nk, int p, int i, double x);
double or_bspline_deriv(const double *U, int nk, int p, int i, double x);
void or_gauss_legendre(int q, double *x, double *w);
int or_minnorm(int m, int N, const double *A, const double *b, double *w);
/* Boehm single-knot insertion (Eq. 10): c (length nk-p-1) -> cnew (length +1),
 * Unew (length nk+1). */
void or_insert_knot(const double *U, int nk, int p, double t, const double *c,
                    double *Unew, double *cnew);
/* WQ layout (reading R1) and weights (Eq. 5, reading R2) for one direction.
 * Returns the number of points; x may be NULL to query. */
int or_wq_points(const double *U, int nk, int p, double *x);
/* weights of test function i over all nx points (zeros outside supp B_i) */
int or_wq_weights(const double *U, int nk, int p, const double *x, int nx, int i,
                  double *w);

/* ---- curve primitives ---- */
int or_curve_line_hits(const or_desc *d, int o, double s, double lo, double hi,
                       double *out, int cap);
int or_curve_inside(const or_desc *d, double x, double y);
int or_curve_folds(const or_desc *d, int o, double *pts, int cap);
int or_curve_joints(const or_desc *d, double *pts, int cap);
void or_curve_point0(const or_desc *d, double *xy);
double or_curve_area(const or_desc *d, int nsub); /* shoelace/Green, for pins */

/* ---- patch ---- */
or_patch *or_create(const or_desc *d);
void or_destroy(or_patch *P);
int or_dims(const or_patch *P, int64_t *out /* 8 */);
/* n1,n2,nel1,nel2,nq1,nq2,n_rows,nnz */
void or_states(const or_patch *P, uint8_t *estate, uint8_t *fstate, int32_t *act);
void or_wq_grid(const or_patch *P, int dir, double *x);
void or_cgrid(const or_patch *P, double *C); /* c at the WQ grid, [k2][k1] */
int or_cut_rule(const or_patch *P, int e1, int e2, double *pts, int cap);
/* DWQ rule for direction dir, disc breakpoint s, side (0 left / 1 right),
 * function i: returns npts; pts[2k] = x, pts[2k+1] = w */
int or_dwq_rule(const or_patch *P, int dir, int s, int side, int i, double *pts, int cap);
int or_dwq_choice(const or_patch *P, int i1, int i2, int *out /* 4 */);
void or_form(const or_patch *P, int64_t *row_ptr, int32_t *col, double *val);
int or_form_row(const or_patch *P, int64_t row, int32_t *col, double *val);
int or_form_row_remark1(const or_patch *P, int64_t row, int32_t *col, double *val);
void or_form_rows(const or_patch *P, const int64_t *rows, int64_t n, double *val, int *cnt);
int or_threads(void);
void or_rhs(const or_patch *P, const or_func *f, double *b);
/* The quadrature rule of one row (reading R9's rule, the one or_rhs applies to
 * f c): for each point k, out[5k..5k+4] = xi1, xi2, x1, x2 (the physical point
 * x(xi)) and the weight with the test function and c folded in, so that
 * b_row = sum_k out[5k+4] f(x1, x2) for any f.  Returns the number of points;
 * writes at most cap of them. */
int or_row_points(const or_patch *P, int64_t row, double *out, int cap);
int or_cg(const or_patch *P, const int64_t *row_ptr, const int32_t *col,
          const double *val, const double *b, double *u, double tol, int maxit,
          double *relres);
double or_l2_error(const or_patch *P, const double *u, const or_func *f,
                   double *fnorm);
double or_visible_area(const or_patch *P);
/* reading R12: loss sum_q omega_q detJ (u_h - g)^2 and its gradient in u */
double or_loss(const or_patch *P, const double *u, const or_func *g, double *dLdu);
/* gradient of the loss w.r.t. the density coefficients, given u and the
 * adjoint lambda = M_s^{-1} dL/du */
void or_density_grad(const or_patch *P, const double *u, const double *lam, const or_func *g,
                     double *grad);

#endif
