/*
 * trimwq.h -- C-ABI of the GB300 (sm_103a) library that forms the Galerkin mass
 * matrix of a trimmed bi-variate B-spline patch by row-wise weighted quadrature
 * with sum factorisation, after Marussig, "Fast formation and assembly of
 * isogeometric Galerkin matrices for trimmed patches" (arXiv 2101.08053).
 *
 * Conventions
 *  - Every entry point returns 0 (TW_OK) or a negative TW_E* code; the text of
 *    the last error of the calling thread is returned by tw_last_error().
 *  - Descriptors (tw_patch_desc, tw_func) and the arrays they point to are HOST
 *    memory owned by the caller; they are copied during the call.
 *  - Output arrays passed to tw_form_mass, tw_rhs, tw_l2_project, tw_states and
 *    tw_patch_table are DEVICE memory owned by the caller (e.g. torch tensors).
 *  - A tw_patch owns its device tables (allocated in tw_patch_create, freed in
 *    tw_patch_destroy).  It is not thread-safe; distinct patches are.
 *  - The library's device memory (patch tables, per-call scratch) comes from
 *    one stream-ordered pool per device that the library creates on first use
 *    and that keeps freed memory for reuse until the process exits (it holds
 *    at most the peak of the library's live allocations).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  All work is
 *    ordered on it; calls that must size outputs synchronise it (documented).
 *  - There is no CPU fallback: without a usable sm_103a device every call that
 *    touches the GPU returns TW_ECUDA.
 */
#ifndef TRIMWQ_H
#define TRIMWQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define TW_OK 0
#define TW_EINVAL -1        /* malformed descriptor or argument              */
#define TW_EUNSUPPORTED -2  /* valid input outside what this build handles   */
#define TW_ENOMEM -3        /* device allocation failed                      */
#define TW_ECUDA -4         /* CUDA runtime error, or a kernel's error flag   */
#define TW_ENOCONV -5       /* CG did not reach the tolerance within maxit   */

/* ---- descriptor enums ---- */
/* trimming curve (Sect. 2.2): a closed curve in the parameter space */
#define TW_TRIM_NONE 0
#define TW_TRIM_CIRCLE 1   /* params: cx, cy, r                                  */
#define TW_TRIM_ELLIPSE 2  /* params: cx, cy, a, b, phi (semi-axes, rotation)    */
#define TW_TRIM_LINE 4     /* params: x0, y0, x1, y1 (distinct); "inside" is the half-plane
                              left of the directed line (x0,y0) -> (x1,y1)   */
#define TW_TRIM_BSPLINE3 3 /* periodic uniform cubic B-spline, nctrl x 2 points,
                              C(tau) = sum_m P_m N3((tau - m) mod nctrl)          */
/* geometry map x(xi) */
#define TW_GEOM_IDENTITY 0
#define TW_GEOM_SPLINE 1   /* control net in the patch basis, n2 x n1 x 2, i1 fastest */
/* the coefficient c(xi) of Eq. 6 */
#define TW_COEF_ONE 0      /* c = 1                                             */
#define TW_COEF_DETJ 1     /* c = det J (pull-back of the physical mass matrix)  */
#define TW_COEF_DENSITY 2  /* c = rho(xi) det J, rho a tensor B-spline           */
/* treatment of cut basis functions */
#define TW_METHOD_GAUSS 0  /* element-wise Gauss for every row (the paper's reference, Sect. 4) */
#define TW_METHOD_HYBRID 1 /* WQ + sum factorisation for interior rows; Gauss on S^r and the
                              cut-element rule on S^t for cut rows (Sect. 3.2, Eq. 8)           */
#define TW_METHOD_DWQ 2    /* discontinuous WQ on a regular rectangle of S^r, Gauss on the rest
                              of S^r, cut rule on S^t (Sect. 3.3)                               */
#define TW_METHOD_NAIVE 3  /* WQ with c zeroed off S^r plus the cut rule: Table 1's negative control */
/* precision of the contraction (tw_form_mass) */
#define TW_PREC_FP64 0     /* val is double*                                     */
#define TW_PREC_FP32 1     /* val is float*; interior rows: tables rounded to FP32,
                              FP32 FMA (cut rows in FP64, rounded on output)      */
#define TW_PREC_FP32X2 2   /* val is double*; interior rows in split precision: FP64
                              values as hi+lo FP32 pairs, error-free products and
                              sums on the FP32 pipes (cut rows in FP64)           */
/* target functions for the L2 projection (Sect. 4.2), evaluated at x(xi) */
#define TW_FUNC_SPLINE 0   /* sum_k a_k N_k(xi): own tensor spline (knots/p/coef) */
#define TW_FUNC_SINSIN 1   /* sin(a x) sin(b y), prm = a, b                       */
#define TW_FUNC_SINCOS 2   /* sin(a x) cos(b y), prm = a, b                       */
#define TW_FUNC_GAUSS 3    /* exp(-k |x - (x0, y0)|^2), prm = k, x0, y0           */

/* element / function states (Sect. 2.2, Eq. 8) */
#define TW_ELEM_INVISIBLE 0
#define TW_ELEM_REGULAR 1
#define TW_ELEM_CUT 2
#define TW_ELEM_EMPTY 3  /* zero-length span of a repeated knot: no measure */
#define TW_FUNC_EXTERIOR 0
#define TW_FUNC_INTERIOR 1
#define TW_FUNC_CUT 2

/* One further trimming curve of a patch (the same fields as the descriptor's
 * trim_*).  A patch may carry up to TW_MAXCURVES curves in all. */
#define TW_MAXCURVES 8
typedef struct {
  int kind;
  int keep_inside;
  double params[6];
  int nctrl;
  const double *ctrl;
} tw_trim_curve;

/* Patch descriptor.  Field layout is shared with the CPU oracle's descriptor
 * so that one seeded generator can fill both; the values are the contract.
 *  p[d]          degree per direction, 1..6; p[0] must equal p[1]
 *  knots[d]      open knot vector: p+1 equal end knots (no more), interior
 *                knots non-decreasing, each of multiplicity m <= p (continuity
 *                C^{p-m} there, Sect. 2.1: mixed continuity); nknots[d] =
 *                n_d + p + 1, >= 2 knot spans.  The elements are the knot
 *                spans; the zero-length spans of repeated knots are empty
 *                elements (no quadrature points, state TW_ELEM_EMPTY), and an
 *                element touching a knot of multiplicity >= 2 carries p+1 WQ
 *                points (else 2).  Extended B-splines need simple knots.
 *  trim_*        the trimming curve; keep_inside = 0 keeps the outside (a hole)
 *  trim_nextra,  further curves (trim_nextra <= TW_MAXCURVES - 1, host array):
 *  trim_extra    the visible domain is the intersection of every curve's kept
 *                side -- several holes, a half-plane with holes, or the ring
 *                between a kept closed curve and a hole inside it (Sect. 4's
 *                domains bounded by several curves)
 *  geom_ctrl     n2*n1*2 doubles for TW_GEOM_SPLINE, else NULL
 *  dens_*        density spline for TW_COEF_DENSITY
 *  cut_order     Gauss order on the pieces of a cut element (0 -> p+1)
 *  stream        stream for the set-up kernels */
typedef struct {
  int p[2];
  int nknots[2];
  const double *knots[2];
  int trim_kind;
  int trim_keep_inside;
  double trim_params[6];
  int trim_nctrl;
  const double *trim_ctrl;
  int geom_kind;
  const double *geom_ctrl;
  int coef_kind;
  int dens_p[2];
  int dens_nknots[2];
  const double *dens_knots[2];
  const double *dens_coef;
  int method;
  int cut_order;
  void *stream;
  int trim_nextra;
  const tw_trim_curve *trim_extra;
} tw_patch_desc;

typedef struct {
  int kind;
  double prm[4];
  int p[2];
  int nknots[2];
  const double *knots[2];
  const double *coef;
} tw_func;

typedef struct tw_patch tw_patch;

/* Build every patch table on the device (Sect. 2.1-3.3):
 *   WQ points (one rule per test function, Eq. 4) and their weights from the
 *   exactness system Eq. 5 (min-norm solution), basis tables, c at the WQ grid,
 *   classification of elements and functions (Sect. 2.2), the cut-element rules
 *   (Sect. 3.1), the DWQ rules (Sect. 3.3, Eqs. 9-10) and the CSR pattern.
 * Synchronises desc->stream between stages (table sizes read back) and at the
 * end (the device-side checks).  Returns TW_EINVAL for a
 * malformed descriptor, TW_EUNSUPPORTED for p outside 1..6, p[0] != p[1] or a
 * curve too complex for one element, TW_ENOMEM / TW_ECUDA otherwise. */
int tw_patch_create(const tw_patch_desc *desc, tw_patch **out);
/* Frees the patch's device tables, stream-ordered on the patch's stream: the
 * call does not wait for the stream, and work already queued there that reads
 * the tables completes first.  The paper has no counterpart: resource
 * management only. */
int tw_patch_destroy(tw_patch *patch);

/* Host copy of the patch sizes (the counts behind Sect. 2.2's split of the
 * basis into interior, cut and exterior functions, Eq. 8, and the sizes of the
 * rules of Sects. 2.1-3.3):
 *  [0] n1 [1] n2 [2] nel1 [3] nel2 [4] nq1 [5] nq2 [6] n_rows [7] nnz
 *  [8] cut elements [9] cut functions [10] cut-rule points [11] DWQ rows
 *  [12] disc knots (both directions) [13] interior rows [14] p [15] method */
int tw_patch_info(const tw_patch *patch, int64_t *info16);

/* Form the mass matrix (Eqs. 6-7) into caller-owned device CSR buffers:
 *   row_ptr[n_rows+1] (int64), col[nnz] (int32, active index, ascending per row),
 *   val[nnz] (double for TW_PREC_FP64 / TW_PREC_FP32X2, float for TW_PREC_FP32).
 * Rows and columns are the active (non-exterior) functions numbered by
 * ascending i2*n1 + i1; the pattern holds every active pair with
 * |i1-j1| <= p and |i2-j2| <= p.  The result is deterministic (each entry is
 * summed by one thread in a fixed order).  Asynchronous on `stream`. */
int tw_form_mass(tw_patch *patch, int precision, int64_t *row_ptr, int32_t *col, void *val,
                 void *stream);

/* The same CSR as tw_form_mass, with the Gauss part of every cut row that has
 * no region part (hybrid Gauss rows, Gauss-method rows, DWQ rows without a
 * region) formed by the row-level sum factorisation of Sect. 3.2, Remark 1:
 * one tensor rule of element Gauss points (p+1 per direction) over the whole
 * support with the coefficient c set to zero off the regular elements,
 * contracted direction by direction as in Eq. 7; cut elements are added from
 * their element matrices.  The values equal tw_form_mass's to rounding (the
 * same quadrature summed in another order); the element matrices of the
 * regular elements are not read.  Asynchronous on `stream`. */
int tw_form_mass_rowsf(tw_patch *patch, int precision, int64_t *row_ptr, int32_t *col, void *val,
                       void *stream);

/* Right-hand side b[n_rows] of the L2 projection: each row's own quadrature
 * rule applied to f * c (Sect. 4.2).  Device output, asynchronous. */
int tw_rhs(tw_patch *patch, const tw_func *f, double *b, void *stream);

/* Two-phase right-hand side, for an f the library cannot evaluate itself
 * (Sect. 4.2's L2 projection of a given f; reading R9: b_i is row i's own
 * quadrature rule applied to f c).
 * tw_rhs_points lists every point at which some row's rule evaluates f, in
 * this order:
 *   [0, nq1*nq2)        the WQ grid, index k2*nq1 + k1 (interior rows, Eq. 7,
 *                       and the masked rule of naive rows)
 *   next ng*(p+1)^2     the element Gauss points (p+1 per direction) of the ng
 *                       regular elements that cut rows integrate by Gauss
 *                       (Sect. 3.2), element by element, g1 fastest
 *   next ncutpts        the cut-element rules (Sect. 3.1), in the order of
 *                       tw_patch_table's table 5
 *   the rest            the DWQ region points of each DWQ row (Sect. 3.3), row
 *                       by row in ascending active index, direction 1 fastest
 * A point may appear more than once (shared by several rows' rules).
 * *npts (host) receives the length of the list.  xi (device, 2*npts doubles,
 * or NULL) receives the parameter points (xi1, xi2) interleaved, x (device,
 * 2*npts doubles, or NULL) the physical points x(xi); with both NULL only the
 * length is returned.  The first call on a patch sizes the list and
 * synchronises `stream`; later calls are asynchronous.
 * tw_rhs_values: b[n_rows] (device) from fvals[npts] (device), the values of
 * f at the listed points -- at the physical points x(xi) when f is a function
 * of the physical coordinates, as for tw_rhs.  The same sums, in the same
 * order, as tw_rhs computes with f evaluated itself.  Asynchronous. */
int tw_rhs_points(tw_patch *patch, int64_t *npts, double *xi, double *x, void *stream);
int tw_rhs_values(tw_patch *patch, const double *fvals, double *b, void *stream);

/* Allocation-free right-hand side.  The paper has no counterpart: this exists
 * for callers that cannot allocate device memory while they run -- a process
 * whose device memory belongs to another allocator (a framework's caching
 * allocator that has reserved almost all of it, so a foreign cudaMalloc fails),
 * or a time-critical loop that must not pay the latency and implicit device
 * synchronisation of cudaMalloc / cudaFree.  It returns the same b as tw_rhs
 * but calls no cudaMalloc, cudaFree or allocating library routine: its scratch
 * (f*c on the WQ grid, nq1*nq2 doubles, plus the knots and coefficients of a
 * TW_FUNC_SPLINE f) lives in one file-scope device array of TW_RHS_STATIC_MAX
 * doubles (16 MiB) that every GPU which loads the library holds until the
 * process exits.  Larger patches or functions are rejected with TW_EINVAL.
 *  - Call it with the patch's device current.  The first call on a device looks
 *    up the array's device address (cudaGetSymbolAddress) for that device; make
 *    that first call before any stream capture.
 *  - Every call on a device shares the one array and leaves its contents
 *    behind; nothing in it has to start at zero, since each call writes all of
 *    the scratch it reads.  Calls that overlap on the GPU (other streams, other
 *    threads) race on the array: order them on one stream.
 *  - A spline f's host arrays (knots, coefficients) are copied into the array
 *    with cudaMemcpyAsync on `stream`.  From pageable memory the copy is staged
 *    before the call returns; from pinned (page-locked) memory it runs when the
 *    stream reaches it, so pinned arrays must stay valid and unchanged until
 *    then (synchronise the stream, or record an event and wait on it, before
 *    freeing or rewriting them). */
#define TW_RHS_STATIC_MAX (1 << 21)
int tw_rhs_static(tw_patch *patch, const tw_func *f, double *b, void *stream);

/* L2 projection (Sect. 4.2; the paper names no solver, the symmetric part is
 * taken because WQ rows with a non-constant c make M non-symmetric, Sect. 2.1):
 * Jacobi-preconditioned CG on (M + M^T)/2 with the CSR produced
 * by tw_form_mass (FP64) and the rhs of f, until ||r||/||b|| <= tol or maxit
 * iterations.  u[n_rows] device output; *iters, *relres host outputs.
 * Synchronises `stream` every few iterations.  TW_ENOCONV if not converged. */
int tw_l2_project(tw_patch *patch, const tw_func *f, const int64_t *row_ptr, const int32_t *col,
                  const double *val, double *u, double tol, int maxit, int *iters,
                  double *relres, void *stream);

/* Differentiation of the L2 projection with respect to the density (Sect. 4.2's
 * projection with c = rho det J, rho = sum_k d_k N_k the patch's density
 * spline, TW_COEF_DENSITY).  The loss compares the projection u_h of f with a
 * target g on the visible part of the patch:
 *   L = sum_q omega_q detJ(x_q) (u_h(x_q) - g(x_q))^2
 * over element Gauss (p+1 points per direction) on regular elements and the
 * cut rule (Sect. 3.1) on cut elements.
 *
 * tw_loss: *loss (device, one double) and dLdu[n_rows] (device) for the
 * coefficients u[n_rows] (device).  Asynchronous; deterministic. */
int tw_loss(tw_patch *patch, const tw_func *g, const double *u, double *loss, double *dLdu,
            void *stream);

/* tw_l2_project_adjoint: given u = M_s^{-1} b(f) from tw_l2_project (same CSR,
 * FP64) and dL/du, solves M_s lambda = dL/du by the projection's CG (same tol,
 * maxit semantics; *iters, *relres host outputs) and returns
 *   grad[k2 * m1 + k1] = dL/dd_k = lambda^T db/dd_k
 *                        - (lambda^T dM/dd_k u + u^T dM/dd_k lambda) / 2
 * (m1 x m2 density coefficients, k1 fastest), computed from every row's own
 * quadrature rule.  lam[n_rows] and grad are device outputs.  The patch must
 * have been created with TW_COEF_DENSITY (else TW_EINVAL).  Synchronises
 * `stream`; TW_ENOCONV if the adjoint CG does not converge.  Deterministic. */
int tw_l2_project_adjoint(tw_patch *patch, const tw_func *f, const int64_t *row_ptr,
                          const int32_t *col, const double *val, const double *dLdu,
                          const double *u, double *lam, double *grad, double tol, int maxit,
                          int *iters, double *relres, void *stream);

/* Extended B-splines (Sect. 3 and Sect. 4.2: the paper stabilises every L2
 * projection with the extended B-splines of Hoellig, Reif and Wipper).
 * An active function is inner when an element of its support is regular,
 * outer otherwise.  Each outer j is tied to the nearest array l + {0..p}^2 of
 * inner functions (l within [j - 2p - 1, j + p + 1] per direction; nearest
 * centre, ties to the smaller l2, then l1) with the coefficients e_{i,j} that
 * carry the B-spline coefficients of every polynomial of degree <= p from the
 * array to j.  E (n_rows x n_inner) holds the identity on inner rows and
 * e_{i,j} on outer rows; the extended basis has mass matrix E^T M E and
 * right-hand side E^T b, and a coefficient vector x of it is u = E x.
 *
 * tw_extension_build: builds the patch's extension tables once (later calls
 * only report); info4 (host) = [n_inner, n_outer, nnz of E, nnz of E^T M E].
 * Synchronises the patch's stream.  TW_EUNSUPPORTED when an outer function
 * has no all-inner array within reach (the mesh is too coarse for the trim). */
int tw_extension_build(tw_patch *patch, int64_t *info4);

/* E as CSR (device, caller-owned): e_row_ptr[n_rows + 1], e_col/e_val[nnz of
 * E]; outer rows hold their (p+1)^2 array entries (a2-major, ascending
 * columns), zeros included.  Asynchronous.  TW_EINVAL before
 * tw_extension_build. */
int tw_extension_matrix(tw_patch *patch, int64_t *e_row_ptr, int32_t *e_col, double *e_val,
                        void *stream);

/* E^T M E from the FP64 CSR of tw_form_mass (device inputs) into device
 * outputs x_row_ptr[n_inner + 1], x_col/x_val[nnz of E^T M E].  Row a holds
 * every inner b reached through a stored M[r][s] with E[r][a], E[s][b]
 * stored (structural zeros kept), columns ascending; each value is a
 * fixed-order sum (deterministic).  Synchronises `stream` to check the input;
 * TW_EINVAL if the CSR does not have the patch's pattern. */
int tw_form_mass_extended(tw_patch *patch, const int64_t *row_ptr, const int32_t *col,
                          const double *val, int64_t *x_row_ptr, int32_t *x_col, double *x_val,
                          void *stream);

/* Extended L2 projection: x from Jacobi-PCG on (E^T M E + (E^T M E)^T)/2
 * x = E^T b(f) (the CSR of tw_form_mass_extended), returned as u = E x
 * (u[n_rows], device).  tol, maxit, *iters, *relres as for tw_l2_project.
 * Synchronises `stream` every few iterations; TW_ENOCONV if not converged. */
int tw_l2_project_extended(tw_patch *patch, const tw_func *f, const int64_t *x_row_ptr,
                           const int32_t *x_col, const double *x_val, double *u, double tol,
                           int maxit, int *iters, double *relres, void *stream);

/* Differentiation of the extended L2 projection (as tw_l2_project_adjoint):
 * u = E x from tw_l2_project_extended (same CSR), lam = E mu with
 * (E^T M_s E) mu = E^T dL/du solved by the same CG, and grad as for
 * tw_l2_project_adjoint with that lam (E does not depend on the density, so
 * the gradient formula is unchanged).  TW_EINVAL without TW_COEF_DENSITY or
 * before tw_extension_build.  Synchronises `stream`; deterministic. */
int tw_l2_project_adjoint_extended(tw_patch *patch, const tw_func *f, const int64_t *x_row_ptr,
                                   const int32_t *x_col, const double *x_val, const double *dLdu,
                                   const double *u, double *lam, double *grad, double tol,
                                   int maxit, int *iters, double *relres, void *stream);

/* Device copies of the classification of Sect. 2.2 (elements regular, cut or
 * invisible; functions interior, cut or exterior, Eq. 8): estate[nel1*nel2], fstate[n1*n2]
 * (uint8, TW_ELEM_* / TW_FUNC_*), act[n1*n2] (int32 active index or -1). */
int tw_states(const tw_patch *patch, uint8_t *estate, uint8_t *fstate, int32_t *act,
              void *stream);

/* Device copy of an internal table, for parity tests (the tables of Sects.
 * 2.1-3.3: WQ points and weights, Eqs. 4-5; c at the grid, Eq. 6; cut-element
 * rules, Sect. 3.1; DWQ choices, Sect. 3.3; Gauss rules and basis values).  `which`:
 *  0/1  WQ points of direction 0/1 (double, nq)
 *  2/3  WQ weights of direction 0/1 (double, n x qmax, local point index)
 *  4    c at the WQ grid (double, nq2 x nq1, k1 fastest)
 *  5    cut-rule points (double, npts x 3: xi1, xi2, weight) in cut-element order
 *  6    cut-rule offsets (int64, ncut+1) and 7 the cut element ids (int32, ncut)
 *  8    DWQ choice per function (int32, n1*n2 x 4: kind1, s1, kind2, s2; -1 none)
 *  9/10 Gauss-Legendre nodes / weights of order p+1 (double, p+1)
 *  11/12 basis values at the WQ points of direction 0/1 (double, nq x (p+1):
 *        B_{e+a}(x_k), e the point's element)
 *  13/14 basis values at the element Gauss points of direction 0/1
 *        (double, nel x (p+1) x (p+1): [e][g][a] = B_{e+a}(x_{e,g}))
 *  15/16 knot vector of direction 0/1 (double, nknots)
 * *count receives the number of elements of the table; nothing is copied if
 * dst is NULL or cap is too small (then TW_EINVAL). */
int tw_patch_table(const tw_patch *patch, int which, void *dst, int64_t cap, int64_t *count,
                   void *stream);

/* Batched formation (many patches, one persistent launch, CUDA graph).  The
 * paper forms one patch at a time; each patch's CSR is the one of
 * tw_form_mass (Eqs. 6-7 and Sects. 3.2-3.3), only the scheduling differs.
 * tw_batch_create takes n existing patches (which must outlive the batch) and
 * their caller-owned device CSR buffers (sized as for tw_form_mass), picks the
 * interior-row tile for each degree present by timing candidate tiles on these
 * patches (cached per device, precision and degree), builds a work list of
 * interior tiles, cut rows and row-pointer copies ordered by estimated cost,
 * and captures one graph: a memset of the work counter and one persistent
 * kernel whose blocks take items until none are left.  Synchronises `stream`.
 * tw_batch_run replays the graph on `stream` (asynchronous); the CSRs equal
 * those of tw_form_mass bit for bit.  Every replay of one batch resets and
 * uses the same device work counter and writes the same CSR buffers, so two
 * replays of one batch must not overlap on the GPU: issue them on one stream
 * (or make the later stream wait on an event recorded after the earlier
 * replay).  Distinct batches are independent.
 * tw_batch_info: [0] patches [1] items [2] persistent blocks [3] dynamic
 * shared memory per block [4..9] interior tile chosen for p = 1..6. */
typedef struct tw_batch tw_batch;
int tw_batch_create(tw_patch *const *patches, int n, int precision, int64_t *const *row_ptr,
                    int32_t *const *col, void *const *val, void *stream, tw_batch **out);
int tw_batch_run(tw_batch *batch, void *stream);
int tw_batch_info(const tw_batch *batch, int64_t *info10);
int tw_batch_destroy(tw_batch *batch);

/* Many patches at once (no counterpart in the paper, which forms one patch at
 * a time; the matrices are those of tw_patch_create + tw_form_mass).  Each job
 * creates a patch from its host descriptor, with all its work ordered on the
 * descriptor's stream; if row_ptr is set it then forms the mass matrix into
 * those device buffers (capacities checked: TW_EINVAL, patch kept), and if
 * h_row_ptr / h_col / h_val are set it copies the CSR into that host memory
 * with cudaMemcpyAsync on the stream (pinned memory: the copies complete when
 * the stream does).  The jobs run on a persistent pool of native host threads
 * that the library starts on first use (nthreads threads with the calling
 * thread, 0 = one per host core, at most one per job and 64), so the set-up
 * chains of different patches overlap on the GPU.  Returns when every job's
 * host part is done (each create has synchronised its stream; formations and
 * copies may still run); the first failing job's status is returned and its
 * message is in tw_last_error.  Give each job its own stream.  The caller
 * destroys every non-NULL patch. */
typedef struct {
  const tw_patch_desc *desc; /* in */
  int precision;             /* in: TW_PREC_* of the formation */
  int64_t *row_ptr;          /* in: device CSR buffers, or NULL (set-up only) */
  int32_t *col;
  void *val;
  int64_t rows_capacity;     /* in: row_ptr holds rows_capacity + 1 entries */
  int64_t nnz_capacity;      /* in: col and val hold nnz_capacity entries */
  int64_t *h_row_ptr;        /* in: host destinations of the CSR, or NULL */
  int32_t *h_col;
  void *h_val;
  tw_patch *patch;           /* out: the created patch, or NULL */
  int status;                /* out: TW_OK or TW_E* */
} tw_job;
int tw_run_jobs(tw_job *jobs, int n, int nthreads);

/* Number of kernels this library has launched in this process.  The paper has
 * no counterpart: an instrumentation counter. */
int64_t tw_launch_count(void);

/* Read-only view of the library's device memory on the current device (no
 * counterpart in the paper: instrumentation): info3[0] = allocations the
 * library has made from its pool in this process (all devices), info3[1] =
 * bytes the pool holds reserved on the current device, info3[2] = bytes of it
 * in use.  Allocates nothing; 0 for a device the library has not used. */
int tw_pool_info(int64_t *info3);

/* Stage timing with CUDA events recorded on the launching stream around each
 * stage (off by default; the paper splits its timings the same way, Sect. 4.2.2:
 * quadrature set-up, interior rows, regular part and cut elements of cut rows).
 * tw_profile_read waits for the recorded events, returns the summed device
 * time in ms and the number of launches of `stage` since the last read, and
 * resets that stage. */
#define TW_STAGE_SETUP 0     /* tw_patch_create: all table kernels            */
#define TW_STAGE_INTERIOR 1  /* interior rows: WQ + sum factorisation kernel   */
#define TW_STAGE_CUTROWS 2   /* cut rows: region + element Gauss + cut rule   */
#define TW_STAGE_RHS 3
#define TW_STAGE_CG 4
#define TW_STAGE_LOSS 5      /* tw_loss                                       */
#define TW_STAGE_ADJOINT 6   /* tw_l2_project_adjoint's gradient kernels (its  
                                CG counts as TW_STAGE_CG)                     */
#define TW_STAGE_GAUSSMAT 7  /* inside tw_patch_create: the element matrices of
                                the regular elements near the curve           */
#define TW_STAGE_WQW 8       /* inside tw_patch_create: the WQ weight solves (Eq. 5) */
#define TW_STAGE_DWQ 9       /* inside tw_patch_create: the DWQ rules (Sect. 3.3)    */
#define TW_NSTAGES 10
int tw_profile_enable(int on);
int tw_profile_read(int stage, double *total_ms, int64_t *count);

/* Text of the calling thread's last error (no counterpart in the paper). */
const char *tw_last_error(void);

#ifdef __cplusplus
}
#endif

#endif
