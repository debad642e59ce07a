/*
 * or_curve.c -- trimming-curve primitives of the oracle (TEST INFRASTRUCTURE).
 *
 * Sect. 2.2: the trimming curve lives in the parameter space, is closed, and
 * its side decides which part of the patch is visible.  The paper lets the
 * representation be chosen freely; three kinds are supported:
 *   circle   (cx, cy, r)                x = c + r (cos th, sin th)
 *   ellipse  (cx, cy, a, b, phi)        x = c + a cos th e1 + b sin th e2
 *   periodic uniform cubic B-spline     C(tau) = sum_m P_m N((tau - m) mod nc)
 * with N the cardinal cubic B-spline on the knots 0,1,2,3,4 (closed form of
 * its four polynomial pieces).  Everything here is plain FP64: closed forms for
 * the conics, and for the spline: critical points of each cubic coordinate in
 * closed form, then bisection on every monotone piece.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>

/* cardinal cubic B-spline and its derivative on [0,4] */
static double card3(double t) {
  if (t < 0.0 || t > 4.0) return 0.0;
  if (t <= 1.0) return t * t * t / 6.0;
  if (t <= 2.0) return (-3.0 * t * t * t + 12.0 * t * t - 12.0 * t + 4.0) / 6.0;
  if (t <= 3.0) return (3.0 * t * t * t - 24.0 * t * t + 60.0 * t - 44.0) / 6.0;
  return (4.0 - t) * (4.0 - t) * (4.0 - t) / 6.0;
}
static double card3d(double t) {
  if (t < 0.0 || t > 4.0) return 0.0;
  if (t <= 1.0) return t * t / 2.0;
  if (t <= 2.0) return (-3.0 * t * t + 8.0 * t - 4.0) / 2.0;
  if (t <= 3.0) return (3.0 * t * t - 16.0 * t + 20.0) / 2.0;
  return -(4.0 - t) * (4.0 - t) / 2.0;
}

/* segment s, local u in [0,1]: C(s+u) = sum_{r=0..3} P_{(s-r) mod nc} N(r+u) */
static double seg_coord(const or_desc *d, int s, double u, int o) {
  int nc = d->trim_nctrl;
  double v = 0.0;
  for (int r = 0; r < 4; r++) {
    int m = ((s - r) % nc + nc) % nc;
    v += d->trim_ctrl[2 * m + o] * card3((double)r + u);
  }
  return v;
}
static double seg_dcoord(const or_desc *d, int s, double u, int o) {
  int nc = d->trim_nctrl;
  double v = 0.0;
  for (int r = 0; r < 4; r++) {
    int m = ((s - r) % nc + nc) % nc;
    v += d->trim_ctrl[2 * m + o] * card3d((double)r + u);
  }
  return v;
}

/* real roots of a u^2 + b u + c in the open interval (0,1), ascending */
static int quad_roots01(double a, double b, double c, double *r) {
  int n = 0;
  double t[2];
  double scale = fabs(a) + fabs(b) + fabs(c);
  if (scale == 0.0) return 0;
  if (fabs(a) <= 1e-14 * scale) {
    if (b != 0.0) t[n++] = -c / b;
  } else {
    double disc = b * b - 4.0 * a * c;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    double q = -0.5 * (b + (b >= 0.0 ? sq : -sq));
    if (q != 0.0) {
      t[n++] = q / a;
      t[n++] = c / q;
    } else {
      t[n++] = 0.0;
    }
  }
  int m = 0;
  for (int k = 0; k < n; k++)
    if (t[k] > 0.0 && t[k] < 1.0) r[m++] = t[k];
  if (m == 2 && r[0] > r[1]) {
    double z = r[0];
    r[0] = r[1];
    r[1] = z;
  }
  if (m == 2 && r[0] == r[1]) m = 1;
  return m;
}

/* critical points of coordinate o on segment s (roots of a quadratic) */
static int seg_crit(const or_desc *d, int s, int o, double *r) {
  double q0 = seg_dcoord(d, s, 0.0, o), qh = seg_dcoord(d, s, 0.5, o),
         q1 = seg_dcoord(d, s, 1.0, o);
  double A = 2.0 * q0 - 4.0 * qh + 2.0 * q1;
  double B = -3.0 * q0 + 4.0 * qh - q1;
  double C = q0;
  return quad_roots01(A, B, C, r);
}

/* roots u in [0,1) of coordinate o on segment s equal to val */
static int seg_roots(const or_desc *d, int s, int o, double val, double *out) {
  int nc = d->trim_nctrl;
  double mn = 1e300, mx = -1e300;
  for (int r = 0; r < 4; r++) {
    int m = ((s - r) % nc + nc) % nc;
    double v = d->trim_ctrl[2 * m + o];
    if (v < mn) mn = v;
    if (v > mx) mx = v;
  }
  if (val < mn || val > mx) return 0; /* convex-hull property */
  double cr[2];
  int nb = seg_crit(d, s, o, cr);
  double br[4];
  br[0] = 0.0;
  for (int k = 0; k < nb; k++) br[k + 1] = cr[k];
  br[nb + 1] = 1.0;
  int n = 0;
  for (int k = 0; k <= nb; k++) {
    double a = br[k], b = br[k + 1];
    double fa = seg_coord(d, s, a, o) - val, fb = seg_coord(d, s, b, o) - val;
    if (fa == 0.0) {
      if (a == 0.0) out[n++] = a;
      continue;
    }
    if (fb == 0.0) {
      if (b < 1.0) out[n++] = b;
      continue;
    }
    if ((fa < 0.0) == (fb < 0.0)) continue;
    for (int it = 0; it < 200; it++) {
      double m = 0.5 * (a + b);
      if (m <= a || m >= b) break;
      double fm = seg_coord(d, s, m, o) - val;
      if (fm == 0.0) {
        a = b = m;
        break;
      }
      if ((fm < 0.0) == (fa < 0.0)) {
        a = m;
        fa = fm;
      } else {
        b = m;
      }
    }
    out[n++] = 0.5 * (a + b);
  }
  return n;
}

static int cmp_dbl(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* conic: the other coordinate where the line xi_o = s meets the conic */
static int conic_line(const or_desc *d, int o, double s, double *out) {
  const double *q = d->trim_params;
  if (d->trim_kind == OR_TRIM_CIRCLE) {
    double cx[2] = {q[0], q[1]};
    double r = q[2];
    double dd = s - cx[o];
    double h = r * r - dd * dd;
    if (h <= 0.0) return 0;
    double sq = sqrt(h);
    out[0] = cx[1 - o] - sq;
    out[1] = cx[1 - o] + sq;
    return 2;
  }
  /* ellipse: ((d.e1)/a)^2 + ((d.e2)/b)^2 = 1, e1 = (cos phi, sin phi),
   * e2 = (-sin phi, cos phi); one coordinate of d fixed to D */
  double cx[2] = {q[0], q[1]};
  double a = q[2], b = q[3], cp = cos(q[4]), sp = sin(q[4]);
  double D = s - cx[o];
  /* write d = (dx, dy); e1.d = cp dx + sp dy, e2.d = -sp dx + cp dy */
  double e1o = o == 0 ? cp : sp, e1i = o == 0 ? sp : cp;
  double e2o = o == 0 ? -sp : cp, e2i = o == 0 ? cp : -sp;
  double A = e1i * e1i / (a * a) + e2i * e2i / (b * b);
  double B = 2.0 * D * (e1o * e1i / (a * a) + e2o * e2i / (b * b));
  double C = D * D * (e1o * e1o / (a * a) + e2o * e2o / (b * b)) - 1.0;
  double disc = B * B - 4.0 * A * C;
  if (disc <= 0.0) return 0;
  double sq = sqrt(disc);
  double y1 = (-B - sq) / (2.0 * A), y2 = (-B + sq) / (2.0 * A);
  out[0] = cx[1 - o] + (y1 < y2 ? y1 : y2);
  out[1] = cx[1 - o] + (y1 < y2 ? y2 : y1);
  return 2;
}

/* All points of the curve with xi_o = s and xi_{1-o} in (lo, hi), ascending. */
int or_curve_line_hits(const or_desc *d, int o, double s, double lo, double hi,
                       double *out, int cap) {
  int n = 0;
  if (d->trim_kind == OR_TRIM_NONE) return 0;
  if (d->trim_kind == OR_TRIM_LINE) {
    /* the point p0 + t (p1 - p0) with coordinate o equal to s */
    const double *q = d->trim_params;
    double p0o = q[o], p0i = q[1 - o], dro = q[2 + o] - q[o], dri = q[3 - o] - q[1 - o];
    if (dro == 0.0) return 0;
    double t = (s - p0o) / dro;
    double v = fma(t, dri, p0i);
    if (v > lo && v < hi && cap > 0) out[n++] = v;
    return n;
  }
  if (d->trim_kind == OR_TRIM_CIRCLE || d->trim_kind == OR_TRIM_ELLIPSE) {
    double v[2];
    int m = conic_line(d, o, s, v);
    for (int k = 0; k < m; k++)
      if (v[k] > lo && v[k] < hi && n < cap) out[n++] = v[k];
    return n;
  }
  for (int sg = 0; sg < d->trim_nctrl; sg++) {
    double u[4];
    int m = seg_roots(d, sg, o, s, u);
    for (int k = 0; k < m; k++) {
      double v = seg_coord(d, sg, u[k], 1 - o);
      if (v > lo && v < hi && n < cap) out[n++] = v;
    }
  }
  qsort(out, (size_t)n, sizeof(double), cmp_dbl);
  return n;
}

/* Points where d(xi_o)/d(param) = 0 (tangent parallel to the other axis). */
int or_curve_folds(const or_desc *d, int o, double *pts, int cap) {
  const double *q = d->trim_params;
  int n = 0;
  if (d->trim_kind == OR_TRIM_CIRCLE) {
    double r = q[2];
    if (o == 0) {
      pts[0] = q[0] - r; pts[1] = q[1];
      pts[2] = q[0] + r; pts[3] = q[1];
    } else {
      pts[0] = q[0]; pts[1] = q[1] - r;
      pts[2] = q[0]; pts[3] = q[1] + r;
    }
    return 2;
  }
  if (d->trim_kind == OR_TRIM_ELLIPSE) {
    double a = q[2], b = q[3], cp = cos(q[4]), sp = sin(q[4]);
    double th = o == 0 ? atan2(-b * sp, a * cp) : atan2(b * cp, a * sp);
    for (int k = 0; k < 2; k++) {
      double t = th + k * 3.14159265358979323846;
      pts[2 * k] = q[0] + a * cos(t) * cp - b * sin(t) * sp;
      pts[2 * k + 1] = q[1] + a * cos(t) * sp + b * sin(t) * cp;
    }
    return 2;
  }
  if (d->trim_kind == OR_TRIM_BSPLINE3) {
    for (int sg = 0; sg < d->trim_nctrl; sg++) {
      double r[2];
      int m = seg_crit(d, sg, o, r);
      for (int k = 0; k < m && n < cap; k++) {
        pts[2 * n] = seg_coord(d, sg, r[k], 0);
        pts[2 * n + 1] = seg_coord(d, sg, r[k], 1);
        n++;
      }
    }
  }
  return n;
}

/* segment junctions of the spline curve (where its smoothness drops to C^2) */
int or_curve_joints(const or_desc *d, double *pts, int cap) {
  if (d->trim_kind != OR_TRIM_BSPLINE3) return 0;
  int n = 0;
  for (int sg = 0; sg < d->trim_nctrl && n < cap; sg++, n++) {
    pts[2 * n] = seg_coord(d, sg, 0.0, 0);
    pts[2 * n + 1] = seg_coord(d, sg, 0.0, 1);
  }
  return n;
}

void or_curve_point0(const or_desc *d, double *xy) {
  const double *q = d->trim_params;
  if (d->trim_kind == OR_TRIM_CIRCLE) {
    xy[0] = q[0] + q[2];
    xy[1] = q[1];
  } else if (d->trim_kind == OR_TRIM_ELLIPSE) {
    xy[0] = q[0] + q[2] * cos(q[4]);
    xy[1] = q[1] + q[2] * sin(q[4]);
  } else if (d->trim_kind == OR_TRIM_BSPLINE3) {
    xy[0] = seg_coord(d, 0, 0.0, 0);
    xy[1] = seg_coord(d, 0, 0.0, 1);
  } else {
    xy[0] = xy[1] = -1e300;
  }
}

/* 1 if (x, y) lies inside the closed curve (ray casting for the spline) */
int or_curve_inside(const or_desc *d, double x, double y) {
  const double *q = d->trim_params;
  if (d->trim_kind == OR_TRIM_LINE) {
    /* left of the directed line: (p1 - p0) x (p - p0) > 0 */
    double dx = q[2] - q[0], dy = q[3] - q[1];
    return fma(dx, y - q[1], -(dy * (x - q[0]))) > 0.0;
  }
  if (d->trim_kind == OR_TRIM_CIRCLE) {
    double dx = x - q[0], dy = y - q[1];
    return dx * dx + dy * dy < q[2] * q[2];
  }
  if (d->trim_kind == OR_TRIM_ELLIPSE) {
    double cp = cos(q[4]), sp = sin(q[4]);
    double dx = x - q[0], dy = y - q[1];
    double u = (cp * dx + sp * dy) / q[2], v = (-sp * dx + cp * dy) / q[3];
    return u * u + v * v < 1.0;
  }
  if (d->trim_kind == OR_TRIM_BSPLINE3) {
    int cnt = 0;
    for (int sg = 0; sg < d->trim_nctrl; sg++) {
      double u[4];
      int m = seg_roots(d, sg, 1, y, u);
      for (int k = 0; k < m; k++)
        if (seg_coord(d, sg, u[k], 0) > x) cnt++;
    }
    return cnt & 1;
  }
  return 0;
}

/* Enclosed area by Green's theorem: 1/2 |oint x dy - y dx|; conics in closed
 * form, the spline with nsub Gauss points per segment (exact for nsub >= 3). */
double or_curve_area(const or_desc *d, int nsub) {
  const double *q = d->trim_params;
  const double pi = 3.14159265358979323846;
  if (d->trim_kind == OR_TRIM_CIRCLE) return pi * q[2] * q[2];
  if (d->trim_kind == OR_TRIM_ELLIPSE) return pi * q[2] * q[3];
  if (d->trim_kind != OR_TRIM_BSPLINE3) return 0.0;
  double gx[64], gw[64];
  if (nsub > 64) nsub = 64;
  or_gauss_legendre(nsub, gx, gw);
  double s = 0.0;
  for (int sg = 0; sg < d->trim_nctrl; sg++)
    for (int g = 0; g < nsub; g++) {
      double u = 0.5 * (gx[g] + 1.0);
      double x = seg_coord(d, sg, u, 0), y = seg_coord(d, sg, u, 1);
      double dx = seg_dcoord(d, sg, u, 0), dy = seg_dcoord(d, sg, u, 1);
      s += 0.5 * gw[g] * (x * dy - y * dx);
    }
  return 0.5 * fabs(s);
}
