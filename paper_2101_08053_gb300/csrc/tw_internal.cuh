// tw_internal.cuh -- device-side building blocks and the patch object of the
// trimmed weighted-quadrature library (sm_103a).
//
//  * B-spline values/derivatives on one span by the triangular Cox-de Boor
//    scheme (Sect. 2.1: p+1 non-zero functions per knot span).
//  * Trimming-curve primitives (Sect. 2.2): circle / ellipse in closed form
//    (angle form), periodic uniform cubic B-spline as monomial segments with
//    safeguarded Newton on monotone brackets.
//  * Minimum-norm solution of the WQ exactness system (Eq. 5) by an LQ
//    factorisation with Householder reflectors from the right.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/trimwq.h"

#define TW_MAXP 6
#define TW_MAXP1 (TW_MAXP + 1)
#define TW_WIN (2 * TW_MAXP + 1)          // band width 2p+1
#define TW_QMAX 32                        // max WQ points in one support
#define TW_LQMAX 96                       // max refined points around one disc
#define TW_BRCAP 64                       // breakpoints per cut element
#define TW_HITCAP 32                      // curve crossings per line inside one element
#define TW_RULECAP 64                     // points of one direction's region rule
#define TW_CORNER 1e-12  // relative margin: curve touching an element corner (R6, R8)
#define TW_TIE 1e-9      // relative tie of the curve's extents in a cut element (R6)
#define TW_GMAT_BUDGET ((size_t)4 << 30)  // bytes of regular-element matrices per patch

// device error flags (bit set by kernels, read by the host at sync points)
#define TWF_BRCAP 1
#define TWF_HITCAP 2
#define TWF_SINGULAR 4
#define TWF_QMAX 8
#define TWF_LQMAX 16
#define TWF_RULECAP 32
#define TWF_TIMEOUT 64  // a bounded wait on a bulk copy ran out

namespace tw {

struct Curve {
  int kind, keep_inside, nc;
  double prm[6];
  const double *seg;  // nc x 8: x(u) = a0+a1u+a2u^2+a3u^3, y(u) = b0..b3 (u in [0,1])
  const double *box;  // nc x 4: xmin xmax ymin ymax (convex hull of the 4 control points)
};

struct Dir {
  int p, n, nel, nk, nq, qmax;
  int mixed;    // the patch has a repeated interior knot (either direction)
  double *U, *bp;
  int *qoff;    // nel+1: first WQ point of each element (R1; empty spans hold none)
  uint8_t *two; // n: every element of supp B_i holds exactly two points
  double *xq;   // nq
  int *qel;     // nq
  int *qbeg;    // n
  int *qcnt;    // n
  double *Bq;   // nq x (p+1)
  double *dBq;  // nq x (p+1)
  double *W;    // n x qmax
  double *V;    // n x qmax x (2p+1)   W * B_j(x_k), r = j - i + p
  int *crange;  // n x (2p+1): lo | (hi << 16) local point range where V != 0
  const double *gx, *gw;  // Gauss-Legendre on [-1,1], p+1 points (cached, not owned)
  double *GB, *dGB; // nel x (p+1) x (p+1): B_{e+a}(x_{e,g}) at [e][g][a]
  double *GW;       // nel x (p+1)^3: w_g h_e B_{e+a}(x_{e,g}) B_{e+b}(x_{e,g}) at [e][g][a][b]
};

struct Geo {
  int geom_kind, coef_kind;
  const double *ctrl;  // n2 x n1 x 2
  int n1;
  // density spline
  int dp[2], dnk[2];
  const double *dU[2];
  const double *dcoef;
};

struct DwqSlot {  // one disc knot of one direction
  int dir, s, npts, pad;
};

// ---------------------------------------------------------------------------
// B-splines

// values N[a] = B_{span-p+a}(x), a = 0..p, span with U[span] <= x < U[span+1].
// Kept out of line: two inlined copies of this variable-trip triangle in one
// function were mis-optimised by nvcc 13.0 for sm_103a at -O3.
static __device__ __noinline__ void basis_vals(const double *U, int span, double x, int p, double *N) {
  double left[TW_MAXP1], right[TW_MAXP1];
  N[0] = 1.0;
  for (int j = 1; j <= p; j++) {
    left[j] = x - U[span + 1 - j];
    right[j] = U[span + j] - x;
    double saved = 0.0;
    for (int r = 0; r < j; r++) {
      double t = N[r] / (right[r + 1] + left[j - r]);
      N[r] = saved + right[r + 1] * t;
      saved = left[j - r] * t;
    }
    N[j] = saved;
  }
}

// values and first derivatives on span, in one pass of the triangle: the
// degree p-1 row is kept when the last level starts, then
//   B'_{i,p} = p B_{i,p-1}/(U[i+p]-U[i]) - p B_{i+1,p-1}/(U[i+p+1]-U[i+1]).
// (Two separate passes for degree p-1 and p were mis-optimised by nvcc 13.0
// for sm_103a at -O3: the values came out wrong while the derivatives did
// not; the one-pass form is correct at every optimisation level.)
__device__ __forceinline__ void basis_ders(const double *U, int span, double x, int p, double *N,
                                           double *dN) {
  double left[TW_MAXP1], right[TW_MAXP1], Nm[TW_MAXP1];
  N[0] = 1.0;
  Nm[0] = 1.0;
  for (int j = 1; j <= p; j++) {
    left[j] = x - U[span + 1 - j];
    right[j] = U[span + j] - x;
    if (j == p)
      for (int r = 0; r < p; r++) Nm[r] = N[r];
    double saved = 0.0;
    for (int r = 0; r < j; r++) {
      double t = N[r] / (right[r + 1] + left[j - r]);
      N[r] = saved + right[r + 1] * t;
      saved = left[j - r] * t;
    }
    N[j] = saved;
  }
  for (int a = 0; a <= p; a++) {
    double l = 0.0, r = 0.0;
    if (a >= 1) {
      double d = U[span + a] - U[span + a - p];
      if (d > 0.0) l = Nm[a - 1] / d;
    }
    if (a <= p - 1) {
      double d = U[span + a + 1] - U[span + a + 1 - p];
      if (d > 0.0) r = Nm[a] / d;
    }
    dN[a] = p * (l - r);
  }
}

// The Cox-de Boor denominators right[r+1] + left[j-r] equal the knot
// differences U[span+r+1] - U[span+1-j+r], which do not depend on x: for many
// points on one span their reciprocals are formed once.
//   rc[j*(j-1)/2 + r]  1 / (U[span+r+1] - U[span+1-j+r]),  j = 1..p, r < j
//   rd[a]              1 / (U[span+a] - U[span+a-p]) (0 if equal), a = 1..p
#define TW_SPAN_RC (TW_MAXP * TW_MAXP1 / 2)
__device__ __forceinline__ void span_recips(const double *U, int span, int p, double *rc,
                                            double *rd) {
  for (int j = 1; j <= p; j++)
    for (int r = 0; r < j; r++) rc[j * (j - 1) / 2 + r] = 1.0 / (U[span + r + 1] - U[span + 1 - j + r]);
  rd[0] = 0.0;
  for (int a = 1; a <= p; a++) {
    const double d = U[span + a] - U[span + a - p];
    rd[a] = d > 0.0 ? 1.0 / d : 0.0;
  }
}
// entry t of the same tables (t < p(p+1)/2: rc[t]; then rd[t - p(p+1)/2]), so
// that the lanes of a warp share the divisions of one span
__device__ __forceinline__ void span_recip_entry(const double *U, int span, int p, int t,
                                                 double *rc, double *rd) {
  const int nrc = p * (p + 1) / 2;
  if (t < nrc) {
    int j = 1, r = t;
    while (r >= j) {
      r -= j;
      j++;
    }
    rc[t] = 1.0 / (U[span + r + 1] - U[span + 1 - j + r]);
  } else {
    const int a = t - nrc;
    if (a == 0) {
      rd[0] = 0.0;
    } else {
      const double d = U[span + a] - U[span + a - p];
      rd[a] = d > 0.0 ? 1.0 / d : 0.0;
    }
  }
}

// basis_ders with the span's reciprocals (span_recips): products only
static __device__ __noinline__ void basis_ders_rc(const double *U, int span, double x, int p,
                                                  const double *rc, const double *rd, double *N,
                                                  double *dN) {
  double left[TW_MAXP1], right[TW_MAXP1], Nm[TW_MAXP1];
  N[0] = 1.0;
  Nm[0] = 1.0;
  for (int j = 1; j <= p; j++) {
    left[j] = x - U[span + 1 - j];
    right[j] = U[span + j] - x;
    if (j == p)
      for (int r = 0; r < p; r++) Nm[r] = N[r];
    double saved = 0.0;
    for (int r = 0; r < j; r++) {
      const double t = N[r] * rc[j * (j - 1) / 2 + r];
      N[r] = saved + right[r + 1] * t;
      saved = left[j - r] * t;
    }
    N[j] = saved;
  }
  for (int a = 0; a <= p; a++) {
    const double l = a >= 1 ? Nm[a - 1] * rd[a] : 0.0;
    const double r = a <= p - 1 ? Nm[a] * rd[a + 1] : 0.0;
    dN[a] = p * (l - r);
  }
}

// span of x in a knot vector (binary search over [lo, hi))
__device__ __forceinline__ int find_span(const double *U, int lo, int hi, double x) {
  // returns s in [lo, hi-1] with U[s] <= x < U[s+1]; clamps at the ends
  if (x >= U[hi]) {
    int s = hi - 1;
    while (s > lo && !(U[s] < U[s + 1])) s--;
    return s;
  }
  int a = lo, b = hi - 1;
  while (a < b) {
    int m = (a + b + 1) >> 1;
    if (U[m] <= x) a = m;
    else b = m - 1;
  }
  return a;
}

// element index of x in breakpoints bp[0..nel]
__device__ __forceinline__ int elem_of(const double *bp, int nel, double x) {
  if (x <= bp[0]) return 0;
  if (x >= bp[nel]) return nel - 1;
  int a = 0, b = nel - 1;
  while (a < b) {
    int m = (a + b + 1) >> 1;
    if (bp[m] <= x) a = m;
    else b = m - 1;
  }
  return a;
}

// ---------------------------------------------------------------------------
// trimming curve

__device__ __forceinline__ double horner3(const double *c, double u) {
  return ((c[3] * u + c[2]) * u + c[1]) * u + c[0];
}

// roots u in [0,1) of c0 + c1 u + c2 u^2 + c3 u^3 = v; returns count (<= 3)
static __device__ int cubic_roots01(const double *c, double v, double *out) {
  double br[4];
  int nb = 0;
  br[nb++] = 0.0;
  {
    // critical points: c1 + 2 c2 u + 3 c3 u^2 = 0
    double A = 3.0 * c[3], B = 2.0 * c[2], Cc = c[1];
    double sc = fabs(A) + fabs(B) + fabs(Cc);
    double r[2];
    int nr = 0;
    if (sc > 0.0) {
      if (fabs(A) <= 1e-14 * sc) {
        if (B != 0.0) r[nr++] = -Cc / B;
      } else {
        double disc = B * B - 4.0 * A * Cc;
        if (disc >= 0.0) {
          double sq = sqrt(disc);
          double q = -0.5 * (B + copysign(sq, B));
          if (q != 0.0) {
            r[nr++] = q / A;
            r[nr++] = Cc / q;
          } else {
            r[nr++] = 0.0;
          }
        }
      }
    }
    if (nr == 2 && r[0] > r[1]) {
      double t = r[0];
      r[0] = r[1];
      r[1] = t;
    }
    for (int k = 0; k < nr; k++)
      if (r[k] > 0.0 && r[k] < 1.0 && (nb == 1 || r[k] > br[nb - 1])) br[nb++] = r[k];
  }
  br[nb++] = 1.0;
  int n = 0;
  for (int k = 0; k + 1 < nb; k++) {
    double a = br[k], b = br[k + 1];
    double fa = horner3(c, a) - v, fb = horner3(c, b) - v;
    if (fa == 0.0) {
      if (a == 0.0) out[n++] = a;
      continue;
    }
    if (fb == 0.0) {
      if (b < 1.0) out[n++] = b;
      continue;
    }
    if ((fa < 0.0) == (fb < 0.0)) continue;
    // safeguarded Newton on the monotone bracket [a, b]
    double lo = a, hi = b, flo = fa;
    double u = 0.5 * (a + b);
    for (int it = 0; it < 200; it++) {
      double fu = horner3(c, u) - v;
      if (fu == 0.0) {
        lo = hi = u;
        break;
      }
      if ((fu < 0.0) == (flo < 0.0)) {
        lo = u;
        flo = fu;
      } else {
        hi = u;
      }
      double d = (3.0 * c[3] * u + 2.0 * c[2]) * u + c[1];
      double un = d != 0.0 ? u - fu / d : 0.5 * (lo + hi);
      if (!(un > lo && un < hi)) un = 0.5 * (lo + hi);
      if (un == u || hi - lo <= 4.0 * 2.220446049250313e-16 * fmax(1.0, fabs(u))) {
        u = un;
        break;
      }
      u = un;
    }
    out[n++] = fmin(fmax(u, a), b);
  }
  return n;
}

// other coordinate of the points of the curve with coordinate o equal to s,
// strictly inside (lo, hi); ascending; returns count or -1 on overflow
static __device__ int curve_line_hits(const Curve &C, int o, double s, double lo, double hi, double *out,
                               int cap) {
  int n = 0;
  if (C.kind == TW_TRIM_LINE) {
    // the point p0 + t (p1 - p0) with coordinate o equal to s
    const double p0o = C.prm[o], p0i = C.prm[1 - o];
    const double dro = C.prm[2 + o] - C.prm[o], dri = C.prm[3 - o] - C.prm[1 - o];
    if (dro == 0.0) return 0;
    const double t = (s - p0o) / dro;
    const double v = fma(t, dri, p0i);
    if (v > lo && v < hi && cap > 0) out[n++] = v;
    return n;
  }
  if (C.kind == TW_TRIM_CIRCLE) {
    double c0 = o == 0 ? C.prm[0] : C.prm[1], c1 = o == 0 ? C.prm[1] : C.prm[0];
    double r = C.prm[2];
    double d = s - c0;
    double h = r * r - d * d;
    if (h <= 0.0) return 0;
    double sq = sqrt(h);
    double v0 = c1 - sq, v1 = c1 + sq;
    if (v0 > lo && v0 < hi) out[n++] = v0;
    if (v1 > lo && v1 < hi) out[n++] = v1;
    return n;
  }
  if (C.kind == TW_TRIM_ELLIPSE) {
    double cx = C.prm[0], cy = C.prm[1], a = C.prm[2], b = C.prm[3];
    double cp = cos(C.prm[4]), sp = sin(C.prm[4]);
    double R, del, th0, th1, v0, v1;
    if (o == 0) {
      // a cos(th) cp - b sin(th) sp = R cos(th + del)
      R = sqrt(a * a * cp * cp + b * b * sp * sp);
      del = atan2(b * sp, a * cp);
      double q = (s - cx) / R;
      if (!(q > -1.0 && q < 1.0)) return 0;
      double ac = acos(q);
      th0 = ac - del;
      th1 = -ac - del;
      v0 = cy + a * cos(th0) * sp + b * sin(th0) * cp;
      v1 = cy + a * cos(th1) * sp + b * sin(th1) * cp;
    } else {
      // a cos(th) sp + b sin(th) cp = R cos(th - del)
      R = sqrt(a * a * sp * sp + b * b * cp * cp);
      del = atan2(b * cp, a * sp);
      double q = (s - cy) / R;
      if (!(q > -1.0 && q < 1.0)) return 0;
      double ac = acos(q);
      th0 = del + ac;
      th1 = del - ac;
      v0 = cx + a * cos(th0) * cp - b * sin(th0) * sp;
      v1 = cx + a * cos(th1) * cp - b * sin(th1) * sp;
    }
    if (v0 > v1) {
      double t = v0;
      v0 = v1;
      v1 = t;
    }
    if (v0 > lo && v0 < hi) out[n++] = v0;
    if (v1 > lo && v1 < hi) out[n++] = v1;
    return n;
  }
  if (C.kind == TW_TRIM_BSPLINE3) {
    for (int sg = 0; sg < C.nc; sg++) {
      const double *bx = C.box + 4 * sg;
      if (s < bx[2 * o] || s > bx[2 * o + 1]) continue;
      const double *co = C.seg + 8 * sg + 4 * o;
      const double *ci = C.seg + 8 * sg + 4 * (1 - o);
      double u[3];
      int m = cubic_roots01(co, s, u);
      for (int k = 0; k < m; k++) {
        double v = horner3(ci, u[k]);
        if (v > lo && v < hi) {
          if (n >= cap) return -1;
          // insertion sort
          int j = n++;
          while (j > 0 && out[j - 1] > v) {
            out[j] = out[j - 1];
            j--;
          }
          out[j] = v;
        }
      }
    }
  }
  return n;
}

// 1 if (x, y) is inside the closed curve
static __device__ int curve_inside(const Curve &C, double x, double y) {
  if (C.kind == TW_TRIM_LINE) {
    // left of the directed line: (p1 - p0) x (p - p0) > 0
    const double dx = C.prm[2] - C.prm[0], dy = C.prm[3] - C.prm[1];
    return fma(dx, y - C.prm[1], -(dy * (x - C.prm[0]))) > 0.0;
  }
  if (C.kind == TW_TRIM_CIRCLE) {
    double dx = x - C.prm[0], dy = y - C.prm[1];
    return dx * dx + dy * dy < C.prm[2] * C.prm[2];
  }
  if (C.kind == TW_TRIM_ELLIPSE) {
    double cp = cos(C.prm[4]), sp = sin(C.prm[4]);
    double dx = x - C.prm[0], dy = y - C.prm[1];
    double u = (cp * dx + sp * dy) / C.prm[2], v = (-sp * dx + cp * dy) / C.prm[3];
    return u * u + v * v < 1.0;
  }
  if (C.kind == TW_TRIM_BSPLINE3) {
    int cnt = 0;
    for (int sg = 0; sg < C.nc; sg++) {
      const double *bx = C.box + 4 * sg;
      if (y < bx[2] || y > bx[3] || bx[1] <= x) continue;
      double u[3];
      int m = cubic_roots01(C.seg + 8 * sg + 4, y, u);
      for (int k = 0; k < m; k++)
        if (horner3(C.seg + 8 * sg, u[k]) > x) cnt++;
    }
    return cnt & 1;
  }
  return 0;
}

__device__ __forceinline__ int visible(const Curve &C, double x, double y) {
  if (C.kind == TW_TRIM_NONE) return 1;
  int in = curve_inside(C, x, y);
  return C.keep_inside ? in : !in;
}

// the trimming curves of a patch (kind != TW_TRIM_NONE; n = 0: untrimmed); the
// visible domain is the intersection of every curve's kept side
struct CurveSet {
  int n;
  Curve c[TW_MAXCURVES];
};

// crossings of every curve with the line xi_o = s inside (lo, hi), ascending;
// -1 when more than cap
static __device__ int set_line_hits(const CurveSet &S, int o, double s, double lo, double hi,
                                    double *out, int cap) {
  int n = 0;
  for (int k = 0; k < S.n; k++) {
    if (cap - n < 2) return -1;  // a conic writes up to two crossings unchecked
    const int m = curve_line_hits(S.c[k], o, s, lo, hi, out + n, cap - n);
    if (m < 0) return -1;
    n += m;
  }
  if (S.n > 1)
    for (int i = 1; i < n; i++) {
      const double x = out[i];
      int j = i - 1;
      while (j >= 0 && out[j] > x) {
        out[j + 1] = out[j];
        j--;
      }
      out[j + 1] = x;
    }
  return n;
}

__device__ __forceinline__ int set_visible(const CurveSet &S, double x, double y) {
  for (int k = 0; k < S.n; k++)
    if (!visible(S.c[k], x, y)) return 0;
  return 1;
}

// the fold points of segment sg of a cubic spline curve (d(coordinate o)/du = 0
// for u in (0, 1)), in root order; returns their count (at most 2)
__device__ __forceinline__ int seg_folds(const Curve &C, int sg, int o, double *pts) {
  const double *co = C.seg + 8 * sg + 4 * o;
  double A = 3.0 * co[3], B = 2.0 * co[2], Cc = co[1];
  double sc = fabs(A) + fabs(B) + fabs(Cc);
  double r[2];
  int nr = 0;
  if (sc == 0.0) return 0;
  if (fabs(A) <= 1e-14 * sc) {
    if (B != 0.0) r[nr++] = -Cc / B;
  } else {
    double disc = B * B - 4.0 * A * Cc;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    double q = -0.5 * (B + copysign(sq, B));
    if (q != 0.0) {
      r[nr++] = q / A;
      r[nr++] = Cc / q;
    }
  }
  if (nr == 2 && r[0] == r[1]) nr = 1;
  int n = 0;
  for (int k = 0; k < nr; k++) {
    if (!(r[k] > 0.0 && r[k] < 1.0)) continue;
    pts[2 * n] = horner3(C.seg + 8 * sg, r[k]);
    pts[2 * n + 1] = horner3(C.seg + 8 * sg + 4, r[k]);
    n++;
  }
  return n;
}

// curve points where d(coordinate o)/d(param) = 0; returns count (pts as x,y)
static __device__ int curve_folds(const Curve &C, int o, double *pts, int cap) {
  if (C.kind == TW_TRIM_CIRCLE) {
    double r = C.prm[2];
    pts[0] = C.prm[0] - (o == 0 ? r : 0.0);
    pts[1] = C.prm[1] - (o == 0 ? 0.0 : r);
    pts[2] = C.prm[0] + (o == 0 ? r : 0.0);
    pts[3] = C.prm[1] + (o == 0 ? 0.0 : r);
    return 2;
  }
  if (C.kind == TW_TRIM_ELLIPSE) {
    double a = C.prm[2], b = C.prm[3], cp = cos(C.prm[4]), sp = sin(C.prm[4]);
    double th = o == 0 ? -atan2(b * sp, a * cp) : atan2(b * cp, a * sp);
    for (int k = 0; k < 2; k++) {
      double t = th + k * 3.141592653589793;
      pts[2 * k] = C.prm[0] + a * cos(t) * cp - b * sin(t) * sp;
      pts[2 * k + 1] = C.prm[1] + a * cos(t) * sp + b * sin(t) * cp;
    }
    return 2;
  }
  int n = 0;
  if (C.kind == TW_TRIM_BSPLINE3) {
    for (int sg = 0; sg < C.nc; sg++) {
      double f[4];
      const int m = seg_folds(C, sg, o, f);
      if (n + m > cap) return -1;
      for (int k = 0; k < 2 * m; k++) pts[2 * n + k] = f[k];
      n += m;
    }
  }
  return n;
}

// ---------------------------------------------------------------------------
// min-norm solution of A w = b (m x N, m <= N, full row rank), A row-major
// with leading dimension lda, overwritten.  LQ with Householder from the
// right: A = L Q, w = Q^T [L^{-1} b; 0].  Returns 0, or 1 if singular.
static __device__ int minnorm_lq(int m, int N, double *A, int lda, const double *b, double *w,
                          double *beta) {
  for (int k = 0; k < m; k++) {
    double *row = A + k * lda;
    double nrm2 = 0.0;
    for (int c = k; c < N; c++) nrm2 += row[c] * row[c];
    double nrm = sqrt(nrm2);
    if (nrm == 0.0) return 1;
    double alpha = row[k] >= 0.0 ? -nrm : nrm;
    double v0 = row[k] - alpha;
    // reflector v = (v0, row[k+1..N-1]); beta = 2 / |v|^2
    double vn2 = v0 * v0 + (nrm2 - row[k] * row[k]);
    beta[k] = vn2 > 0.0 ? 2.0 / vn2 : 0.0;
    row[k] = v0;  // store v in place (row k, columns k..N-1)
    for (int r = k + 1; r < m; r++) {
      double *x = A + r * lda;
      double s = 0.0;
      for (int c = k; c < N; c++) s += x[c] * row[c];
      s *= beta[k];
      for (int c = k; c < N; c++) x[c] -= s * row[c];
    }
    // diagonal of L: alpha (kept in w scratch via beta trick) -> store separately
    w[k] = alpha;
  }
  // forward substitution L y = b, L[r][c] = A[r][c] (c < r), L[k][k] = w[k]
  double y[2 * TW_MAXP + 2];
  for (int r = 0; r < m; r++) {
    double s = b[r];
    for (int c = 0; c < r; c++) s -= A[r * lda + c] * y[c];
    if (w[r] == 0.0) return 1;
    y[r] = s / w[r];
  }
  for (int c = 0; c < N; c++) w[c] = c < m ? y[c] : 0.0;
  // w = H_0 H_1 ... H_{m-1} [y; 0]
  for (int k = m - 1; k >= 0; k--) {
    const double *v = A + k * lda;
    double s = 0.0;
    for (int c = k; c < N; c++) s += v[c] * w[c];
    s *= beta[k];
    for (int c = k; c < N; c++) w[c] -= s * v[c];
  }
  return 0;
}

// ---------------------------------------------------------------------------
// c at points (Eq. 6): det J of the spline geometry, times a density spline

__device__ __forceinline__ double density_at(const Geo &G, double x1, double x2) {
  double N1[TW_MAXP1], N2[TW_MAXP1];
  int q1 = G.dp[0], q2 = G.dp[1];
  int m1 = G.dnk[0] - q1 - 1;
  int s1 = find_span(G.dU[0], q1, m1, x1), s2 = find_span(G.dU[1], q2, G.dnk[1] - q2 - 1, x2);
  basis_vals(G.dU[0], s1, x1, q1, N1);
  basis_vals(G.dU[1], s2, x2, q2, N2);
  double s = 0.0;
  for (int b = 0; b <= q2; b++)
    for (int a = 0; a <= q1; a++) s += G.dcoef[(s2 - q2 + b) * m1 + (s1 - q1 + a)] * N1[a] * N2[b];
  return s;
}

// c from the element's basis values/derivatives (functions e_d .. e_d+p)
__device__ __forceinline__ double coef_from(const Geo &G, int p, double x1, double x2, int e1, const double *v1,
                            const double *d1, int e2, const double *v2, const double *d2) {
  if (G.coef_kind == TW_COEF_ONE) return 1.0;
  double dj = 1.0;
  if (G.geom_kind == TW_GEOM_SPLINE) {
    double xa = 0, ya = 0, xb = 0, yb = 0;
    for (int b = 0; b <= p; b++) {
      double sxa = 0, sya = 0, sxb = 0, syb = 0;
      for (int a = 0; a <= p; a++) {
        const double *pt = G.ctrl + 2 * ((size_t)(e2 + b) * G.n1 + (e1 + a));
        sxa += pt[0] * d1[a];
        sya += pt[1] * d1[a];
        sxb += pt[0] * v1[a];
        syb += pt[1] * v1[a];
      }
      xa += sxa * v2[b];
      ya += sya * v2[b];
      xb += sxb * d2[b];
      yb += syb * d2[b];
    }
    dj = xa * yb - xb * ya;
  }
  if (G.coef_kind == TW_COEF_DENSITY) dj *= density_at(G, x1, x2);
  return dj;
}

__device__ __forceinline__ double coef_at(const Geo &G, const Dir &A, const Dir &B, double x1, double x2) {
  if (G.coef_kind == TW_COEF_ONE) return 1.0;
  int e1 = elem_of(A.bp, A.nel, x1), e2 = elem_of(B.bp, B.nel, x2);
  double v1[TW_MAXP1], d1[TW_MAXP1], v2[TW_MAXP1], d2[TW_MAXP1];
  basis_ders(A.U, e1 + A.p, x1, A.p, v1, d1);
  basis_ders(B.U, e2 + B.p, x2, B.p, v2, d2);
  return coef_from(G, A.p, x1, x2, e1, v1, d1, e2, v2, d2);
}

struct RowArgs {
  Dir A, B;
  Geo G;
  const uint8_t *estate, *fstate;
  const int32_t *act;
  const int64_t *rp;
  const double *C;
  const int32_t *gslot;
  const double *gc;
  const int32_t *cut_slot;
  const int64_t *cut_off;
  const double *cut_B;
  const double *cut_wc;
  const double *cut_pts;
  const double *cut_M;
  const int32_t *choice;
  const int32_t *disc_slot[2];
  const double *dwq_x[2];
  const int32_t *dwq_np[2];
  const double *dwq_w[2];
  const int32_t *dwq_k[2];
  const int32_t *dwq_e[2];
  const double *dwq_B[2];
  const double *dwq_dB[2];
  const int32_t *dwq_r[2];
  const double *gmat;
  int method;
  int *flag;
};

// ---------------------------------------------------------------------------
// warp reductions by a fixed shuffle tree (deterministic)
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum over the G consecutive lanes of one group (G a power of two <= 32)
template <int G>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Minimum-norm solutions of 32/G small systems at once (Eq. 5, reading R2),
// one per group of G consecutive lanes: an LQ factorisation A = L Q by
// Householder reflectors applied from the right (reflector k from row k,
// applied to the rows below), then L y = b by forward substitution and
// w = H_0 ... H_{m-1} [y; 0].  Every FP64 instruction serves all the warp's
// systems (GB300 issues one FP64 warp instruction per 16 cycles per SM).
// The group's system: A (m x N, row stride lda) in shared memory, b (m) in
// shared memory; lane gl of the group owns the columns (and the rows of the
// triangular solve) gl + G u, u < CPL.  Loop bounds are the warp's largest m
// and N; a group past its own m idles.  On return w[u] is the weight of
// column gl + G u (0 beyond N), A holds the reflectors, diag / beta (m, shared
// per group) their data; *singular (per group) is set when a reflector's norm
// vanishes (the group's weights are then 0).  Called by the whole warp.
template <int G, int CPL>
__device__ void group_minnorm(int m, int N, double *A, int lda, const double *b, double *diag,
                              double *beta, int gl, int *singular, double (&w)[CPL]) {
  const unsigned FULL = 0xffffffffu;
  const int M = __reduce_max_sync(FULL, (unsigned)m);
  const int NN = __reduce_max_sync(FULL, (unsigned)N);
  const int U = (NN + G - 1) / G;  // <= CPL
  bool ok = m > 0 && N > 0;
  for (int k = 0; k < M; k++) {
    const bool act = ok && k < m;
    double part = 0.0;
#pragma unroll
    for (int u = 0; u < CPL; u++) {
      if (u >= U) break;  // warp-uniform
      const int c = gl + G * u;
      const double x = (act && c >= k && c < N) ? A[k * lda + c] : 0.0;
      part = fma(x, x, part);
    }
    const double nrm2 = group_sum<G>(part);
    const double akk = act ? A[k * lda + k] : 0.0;
    const double nrm = sqrt(nrm2);
    if (act && nrm == 0.0) {
      ok = false;
      if (gl == 0) *singular = 1;
    }
    const bool go = act && ok;
    const double alpha = akk >= 0.0 ? -nrm : nrm;
    const double v0 = akk - alpha;
    const double vn2 = v0 * v0 + (nrm2 - akk * akk);
    const double bk = (go && vn2 > 0.0) ? 2.0 / vn2 : 0.0;
    __syncwarp();
    // the reflector v (columns k..N-1) replaces row k: only column k changes
    if (go && gl == (k & (G - 1))) A[k * lda + k] = v0;
    if (go && gl == 0) {
      diag[k] = alpha;
      beta[k] = bk;
    }
    __syncwarp();
    // rows below: r -= bk (r . v) v
    for (int r = k + 1; r < M; r++) {
      const bool ra = go && r < m;
      double sr = 0.0;
#pragma unroll
      for (int u = 0; u < CPL; u++) {
        if (u >= U) break;  // warp-uniform
        const int c = gl + G * u;
        if (ra && c >= k && c < N) sr = fma(A[r * lda + c], A[k * lda + c], sr);
      }
      sr = group_sum<G>(sr) * bk;
#pragma unroll
      for (int u = 0; u < CPL; u++) {
        if (u >= U) break;  // warp-uniform
        const int c = gl + G * u;
        if (ra && c >= k && c < N) A[r * lda + c] = fma(-sr, A[k * lda + c], A[r * lda + c]);
      }
    }
    __syncwarp();
  }
  // forward substitution L y = b (L below the diagonal of A, diagonal in
  // diag); y_j lives on its owner lane, slot j / G
  double y[CPL];
#pragma unroll
  for (int u = 0; u < CPL; u++) y[u] = 0.0;
  for (int j = 0; j < M; j++) {
    const bool ja = ok && j < m;
    double part = 0.0;
#pragma unroll
    for (int u = 0; u < CPL; u++) {
      if (u >= U) break;  // warp-uniform
      const int i = gl + G * u;
      if (ja && i < j) part = fma(A[j * lda + i], y[u], part);
    }
    const double s = group_sum<G>(part);
    const double yj = ja ? (b[j] - s) * (1.0 / diag[j]) : 0.0;
#pragma unroll
    for (int u = 0; u < CPL; u++)
      if (gl + G * u == j) y[u] = yj;
  }
  // w = H_0 ... H_{m-1} [y; 0]
#pragma unroll
  for (int u = 0; u < CPL; u++) w[u] = (ok && gl + G * u < m) ? y[u] : 0.0;
  for (int k = M - 1; k >= 0; k--) {
    const bool go = ok && k < m;
    double part = 0.0;
#pragma unroll
    for (int u = 0; u < CPL; u++) {
      if (u >= U) break;  // warp-uniform
      const int c = gl + G * u;
      if (go && c >= k && c < N) part = fma(A[k * lda + c], w[u], part);
    }
    const double tot = group_sum<G>(part);  // every lane takes part in the shuffles
    const double sd = go ? tot * beta[k] : 0.0;
#pragma unroll
    for (int u = 0; u < CPL; u++) {
      if (u >= U) break;  // warp-uniform
      const int c = gl + G * u;
      if (go && c >= k && c < N) w[u] = fma(-sd, A[k * lda + c], w[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < CPL; u++)
    if (!ok || gl + G * u >= N) w[u] = 0.0;
}

}  // namespace tw

// ---------------------------------------------------------------------------
// the patch object (host struct with device pointers)
struct tw_patch {
  int p, method, qc;
  int ktile[7];  // most WQ points of direction 0 under a tile of 2^k test functions i1
  int mixed;     // some knot span is empty (a repeated interior knot)
  int32_t *cnt32;  // set-up counters and 32-bit scan totals (24, zeroed at creation)
  int64_t *cnt64;  // 64-bit scan totals (4, zeroed at creation)
  tw::Dir d[2];
  const double *qrule;  // cut-piece Gauss rule (cached, not owned)
  tw::CurveSet curves;
  double *curve_ctrl[TW_MAXCURVES];  // device copies of spline curves' control points
  tw::Geo geo;
  cudaStream_t stream;
  // owned device allocations
  void *allocs[512];
  int nallocs;
  // classification
  uint8_t *estate, *fstate;
  int32_t *act;      // n1*n2
  int32_t *rowg;     // n_rows: active row -> g
  int64_t *row_ptr;  // n_rows+1
  int64_t n_rows, nnz, n_interior;
  double *C;         // nq2 x nq1
  // cut elements
  int ncut;
  int32_t *cut_list;
  int64_t *cut_off;  // ncut+1 (points)
  int64_t ncutpts;
  double *cut_pts;   // npts x 3 (xi1, xi2, w)
  double *cut_wc;    // npts: w * c
  double *cut_B;     // npts x 2 x (p+1)
  int32_t *cut_o;    // ncut: outer direction of each cut element's rule
  double *cut_M;     // ncut x (p+1)^4: element matrices of the cut elements
  int32_t *cut_slot; // nel1*nel2 -> cut index or -1
  // rows formed by the cut-row kernel
  int ncutrows;
  int32_t *cutrows;  // g
  int ncutfns;
  // element Gauss c tables
  int32_t *gslot;    // nel1*nel2 -> slot or -1
  int ngslot;
  double *gc;        // ngslot x (p+1)^2  [g2][g1]
  // DWQ
  int32_t *choice;   // n1*n2 x 4
  int32_t *disc_slot[2];  // per direction, per breakpoint s: slot or -1
  int ndisc[2];
  double *dwq_x[2];  // ndisc x TW_LQMAX points
  int32_t *dwq_np[2];
  double *dwq_w[2];  // ndisc x p x 2 x TW_LQMAX
  int32_t *dwq_k[2]; // ndisc x TW_LQMAX: base WQ point index of each window point, -1 nested
  int32_t *dwq_e[2]; // ndisc x TW_LQMAX: coarse element of each window point
  double *dwq_B[2];  // ndisc x TW_LQMAX x (p+1): coarse basis values there
  double *dwq_dB[2]; // ndisc x TW_LQMAX x (p+1): and their derivatives
  int32_t *dwq_r[2]; // ndisc x p x 2: window point run of (function, side)
  double *gmat;      // ngslot x (p+1)^4 element matrices of the Gauss elements (or NULL)
  float2 *Cf;        // c on the WQ grid as hi/lo FP32 pairs (created on first FP32 form)
  float2 *Vf[2];     // weighted basis tables as hi/lo FP32 pairs
  float *Ch;         // c rounded to float, rows padded to ldh (a multiple of 4)
  int ldh, ldf;      // ldf: the row stride of Cf in pairs (even)
  float2 *Vcf;       // direction-1 band values per (function, point) as pairs ((n1+1) rows)
  float *Vch;        // the same rounded to float
  int ndwqrows;
  // scratch
  int32_t *flag;     // error flags (device)
  // while the patch is created its small tables are carved from slabs
  char *arena;
  size_t arena_left;
  int arena_on;
  int64_t *i64tmp;
  // rule points of the rhs for an f given by values (built on first use):
  // per cut row the offset of its DWQ region points, their device total, and
  // the length of the whole list (-1 until read back)
  int64_t *pt_roff;
  int64_t *pt_dtot;
  int64_t pt_total;
  // extended B-spline tables (host struct with device pointers), built on
  // demand by tw_extension_build
  void *ext;
};

// host helpers shared by the translation units
namespace tw {
extern std::atomic<int64_t> g_launches;
extern std::atomic<int64_t> g_pool_allocs;  // allocations made from the library pool
int prof_start(cudaStream_t s);                  // -1 when profiling is off
void prof_stop(int slot, int stage, cudaStream_t s);
void set_error(const char *fmt, ...);
int check_cuda(cudaError_t e, const char *what);
void *dalloc(tw_patch *P, size_t bytes);
void release_to(tw_patch *P, int mark);  // free allocations made after `mark`
int exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total, cudaStream_t s,
                       tw_patch *P);
int exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total, cudaStream_t s,
                       tw_patch *P);
int build_tables(tw_patch *P);
// q-point Gauss-Legendre rule (x then w, 2q doubles) on the current device,
// computed once per process and device and kept until exit
int gauss_rule(int q, cudaStream_t s, const double **out);
int form_mass_launch(tw_patch *P, int precision, int64_t *row_ptr, int32_t *col, void *val,
                     cudaStream_t s, bool rowsf = false);
int launch_interior32(tw_patch *P, int precision, int32_t *col, void *val, cudaStream_t s);
int rhs_launch(tw_patch *P, const tw_func *f, double *b, cudaStream_t s);
int rhs_points_run(tw_patch *P, int64_t *npts, double *xi, double *X, cudaStream_t s);
int rhs_values_run(tw_patch *P, const double *FV, double *b, cudaStream_t s);
int l2_project_run(tw_patch *P, const tw_func *f, const int64_t *rp, const int32_t *col,
                   const double *val, double *u, double tol, int maxit, int *iters,
                   double *relres, cudaStream_t s);
RowArgs row_args(tw_patch *P);
// CG on M_s x = b for a device b; temporary allocations released before return
int cg_solve(tw_patch *P, const int64_t *rp, const int32_t *col, const double *val,
             const double *b, double *x, double tol, int maxit, int *iters, double *relres,
             cudaStream_t s);
// the same for an n x n system with nnz entries (e.g. the extended mass matrix)
int cg_solve_n(tw_patch *P, int64_t n, int64_t nnz, const int64_t *rp, const int32_t *col,
               const double *val, const double *b, double *x, double tol, int maxit, int *iters,
               double *relres, cudaStream_t s);
int loss_run(tw_patch *P, const tw_func *g, const double *u, double *loss, double *dLdu,
             cudaStream_t s);
int adjoint_run(tw_patch *P, const tw_func *f, const int64_t *rp, const int32_t *col,
                const double *val, const double *dLdu, const double *u, double *lam,
                double *grad, double tol, int maxit, int *iters, double *relres, cudaStream_t s);
// dL/dd from u and a given lambda (the patch's stream must be s)
int adjoint_grad(tw_patch *P, const tw_func *f, const double *u, const double *lam, double *grad,
                 cudaStream_t s);
}  // namespace tw

#define TW_LAUNCH() (tw::g_launches++)
