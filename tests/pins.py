"""Independent reference computations used to pin the oracle.

Built only on numpy / scipy library routines and closed forms -- never on the
oracle's own code -- so that a dropped term, a wrong index or a transposed
operand in the oracle fails one of them:

* B-spline values / integrals through scipy.interpolate.BSpline;
* Gauss-Legendre nodes through numpy.polynomial.legendre.leggauss;
* entries int_{Omega^v} B_i B_j for a domain with a hole D, by Green's theorem:
      int_D B_i1(x) B_j1(x) B_i2(y) B_j2(y) dx dy
        = oint_{dD} G(x) B_i2(y) B_j2(y) dy,   G(x) = int_{-inf}^x B_i1 B_j1,
  the line integral split at every crossing of the curve with a knot line (so
  that each piece is smooth) and integrated with many Gauss points.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.interpolate import BSpline


def bsp(U, p, i):
    c = np.zeros(len(U) - p - 1)
    c[i] = 1.0
    return BSpline(np.asarray(U, float), c, p, extrapolate=False)


def bvals(U, p, i, x):
    v = bsp(U, p, i)(np.asarray(x, float))
    return np.nan_to_num(v, nan=0.0)


def line_product_integral(U, p, i, j):
    """int B_i B_j over the real line, by numpy Gauss with p+1 points per span."""
    gx, gw = np.polynomial.legendre.leggauss(p + 1)
    s = 0.0
    for a, b in zip(U[:-1], U[1:]):
        if b <= a:
            continue
        x = a + (b - a) * (gx + 1) / 2
        s += np.sum(gw * (b - a) / 2 * bvals(U, p, i, x) * bvals(U, p, j, x))
    return s


def product_antiderivative(U, p, i, j, x):
    """G(x) = int_{-inf}^x B_i B_j (exact: Gauss on every span, partial span
    mapped onto [a, x])."""
    U = np.asarray(U, float)
    x = np.atleast_1d(np.asarray(x, float))
    gx, gw = np.polynomial.legendre.leggauss(p + 1)
    out = np.zeros_like(x)
    for a, b in zip(U[:-1], U[1:]):
        if b <= a:
            continue
        hi = np.clip(x, a, b)
        L = hi - a
        pts = a + L[:, None] * (gx[None, :] + 1) / 2
        f = bvals(U, p, i, pts.ravel()).reshape(pts.shape) * bvals(U, p, j, pts.ravel()).reshape(pts.shape)
        out += np.sum(gw[None, :] * L[:, None] / 2 * f, axis=1)
    return out


def _circle_pieces(cx, cy, r, U1, U2):
    th = [0.0, 2 * math.pi]
    for k in np.unique(U1):
        v = (k - cx) / r
        if -1 < v < 1:
            a = math.acos(v)
            th += [a, 2 * math.pi - a]
    for k in np.unique(U2):
        v = (k - cy) / r
        if -1 < v < 1:
            a = math.asin(v)
            th += [a % (2 * math.pi), (math.pi - a) % (2 * math.pi)]
    return np.unique(np.array(th))


def circle_boundary_points(cx, cy, r, U1, U2, q=40):
    """Parameter points on the circle (counter-clockwise) with Gauss weights,
    split at knot-line crossings: returns x, y, dy/dth * w."""
    br = _circle_pieces(cx, cy, r, U1, U2)
    gx, gw = np.polynomial.legendre.leggauss(q)
    X, Y, W = [], [], []
    for a, b in zip(br[:-1], br[1:]):
        t = a + (b - a) * (gx + 1) / 2
        X.append(cx + r * np.cos(t))
        Y.append(cy + r * np.sin(t))
        W.append(gw * (b - a) / 2 * r * np.cos(t))
    return np.concatenate(X), np.concatenate(Y), np.concatenate(W)


def periodic_curve(ctrl):
    """The closed curve C(tau) = sum_m P_m N(tau - m), tau in [0, nc], as a
    scipy BSpline on the integer knots -3 .. nc+3 with wrapped coefficients."""
    ctrl = np.asarray(ctrl, float)
    nc = len(ctrl)
    t = np.arange(-3, nc + 4, dtype=float)
    c = np.array([ctrl[(j - 3) % nc] for j in range(len(t) - 4)])
    return BSpline(t, c, 3)


def bspline_curve_segment_poly(ctrl, s):
    """Monomial coefficients of x(u), y(u) on segment s (tau = s + u, u in
    [0, 1]) from 4 samples of the scipy curve (a cubic is fixed by them)."""
    cv = periodic_curve(ctrl)
    us = np.array([0.0, 1 / 3, 2 / 3, 1.0])
    xy = cv(s + us)
    return np.polyfit(us, xy[:, 0], 3), np.polyfit(us, xy[:, 1], 3)


def line_removed_boundary_points(x0, y0, x1, y1, U1, U2, q=40):
    """Points / weights of oint (.) dy around the part of the unit square
    ABOVE the line through (x0, 0) .. (x1, 1)-spanning points (x0, y0) and
    (x1, y1) with x0 = 0, x1 = 1 and 0 < y0, y1 < 1, counter-clockwise: the
    line from left to right, then the right edge x = 1 upwards (the top edge
    has dy = 0 and the left edge x = 0 contributes nothing, because the
    x-antiderivatives vanish at 0).  Every piece is split at the knot lines."""
    assert x0 == 0.0 and x1 == 1.0 and 0.0 < y0 < 1.0 and 0.0 < y1 < 1.0
    gx, gw = np.polynomial.legendre.leggauss(q)
    X, Y, W = [], [], []
    # the line, t in [0, 1]: x = t, y = y0 + t (y1 - y0); split where x or y
    # crosses a knot
    br = {0.0, 1.0}
    for k in np.unique(U1):
        if 0.0 < k < 1.0:
            br.add(float(k))
    for k in np.unique(U2):
        t = (k - y0) / (y1 - y0) if y1 != y0 else -1.0
        if 0.0 < t < 1.0:
            br.add(float(t))
    br = sorted(br)
    for a, b in zip(br[:-1], br[1:]):
        t = a + (b - a) * (gx + 1) / 2
        X.append(t)
        Y.append(y0 + t * (y1 - y0))
        W.append(gw * (b - a) / 2 * (y1 - y0))
    # right edge, y from y1 to 1, split at the knots of U2
    br = sorted({y1, 1.0} | {float(k) for k in np.unique(U2) if y1 < k < 1.0})
    for a, b in zip(br[:-1], br[1:]):
        yy = a + (b - a) * (gx + 1) / 2
        X.append(np.ones_like(yy))
        Y.append(yy)
        W.append(gw * (b - a) / 2)
    return np.concatenate(X), np.concatenate(Y), np.concatenate(W)


def bspline_boundary_points(ctrl, U1, U2, q=40):
    """Points / weights of the line integral oint (.) dy along the periodic
    cubic B-spline curve, each segment split where it crosses a knot line."""
    gx, gw = np.polynomial.legendre.leggauss(q)
    X, Y, W = [], [], []
    for s in range(len(ctrl)):
        px, py = bspline_curve_segment_poly(ctrl, s)
        br = [0.0, 1.0]
        for poly, knots in ((px, U1), (py, U2)):
            for k in np.unique(knots):
                rts = np.roots(poly - np.array([0, 0, 0, k]))
                for rt in rts:
                    if abs(rt.imag) < 1e-12 and 0 < rt.real < 1:
                        br.append(rt.real)
        br = np.unique(br)
        dpy = np.polyder(py)
        for a, b in zip(br[:-1], br[1:]):
            u = a + (b - a) * (gx + 1) / 2
            X.append(np.polyval(px, u))
            Y.append(np.polyval(py, u))
            W.append(gw * (b - a) / 2 * np.polyval(dpy, u))
    return np.concatenate(X), np.concatenate(Y), np.concatenate(W)


def hole_entry(U1, U2, p, i1, i2, j1, j2, bnd):
    """int_D B_i B_j over the region D enclosed by the boundary samples bnd
    (signed: counter-clockwise positive)."""
    X, Y, W = bnd
    G = product_antiderivative(U1, p, i1, j1, X)
    H = bvals(U2, p, i2, Y) * bvals(U2, p, j2, Y)
    return float(np.sum(G * H * W))


def exact_entry_hole(U1, U2, p, i1, i2, j1, j2, bnd):
    """int_{[0,1]^2 minus D} B_i B_j (c = 1) for a hole D inside the square,
    boundary samples counter-clockwise."""
    full = line_product_integral(U1, p, i1, j1) * line_product_integral(U2, p, i2, j2)
    return full - hole_entry(U1, U2, p, i1, i2, j1, j2, bnd)


def polygon_area(bnd):
    X, Y, W = bnd
    # oint x dy
    return float(np.sum(X * W))


class GreenEntries:
    """Cached exact c = 1 entries int_{[0,1]^2 minus D} B_i B_j via Green's
    theorem (G and H tabulated once per index pair)."""

    def __init__(self, U1, U2, p, bnd):
        self.U1, self.U2, self.p, self.bnd = np.asarray(U1, float), np.asarray(U2, float), p, bnd
        self._G, self._H, self._I1, self._I2 = {}, {}, {}, {}
        X, Y, W = bnd
        self._B2 = {}

    def _b2(self, i):
        if i not in self._B2:
            self._B2[i] = bvals(self.U2, self.p, i, self.bnd[1])
        return self._B2[i]

    def entry(self, i1, i2, j1, j2):
        k1, k2 = (min(i1, j1), max(i1, j1)), (min(i2, j2), max(i2, j2))
        if k1 not in self._G:
            self._G[k1] = product_antiderivative(self.U1, self.p, k1[0], k1[1], self.bnd[0])
            self._I1[k1] = line_product_integral(self.U1, self.p, k1[0], k1[1])
        if k2 not in self._H:
            self._H[k2] = self._b2(k2[0]) * self._b2(k2[1])
            self._I2[k2] = line_product_integral(self.U2, self.p, k2[0], k2[1])
        hole = float(np.sum(self._G[k1] * self._H[k2] * self.bnd[2]))
        return self._I1[k1] * self._I2[k2] - hole


def ellipse_boundary_points(cx, cy, a, b, phi, U1, U2, q=40):
    """Points / weights of oint (.) dy along the ellipse (counter-clockwise in
    its parameter t), split where it crosses a knot line.  With c = cos phi,
    s = sin phi: x - cx = Rx cos(t + dx), y - cy = Ry cos(t - dy)."""
    cp, sp = math.cos(phi), math.sin(phi)
    Rx, dx = math.hypot(a * cp, b * sp), math.atan2(b * sp, a * cp)
    Ry, dy = math.hypot(a * sp, b * cp), math.atan2(b * cp, a * sp)
    th = [0.0, 2 * math.pi]
    for k in np.unique(U1):
        v = (k - cx) / Rx
        if -1 < v < 1:
            ac = math.acos(v)
            th += [(ac - dx) % (2 * math.pi), (-ac - dx) % (2 * math.pi)]
    for k in np.unique(U2):
        v = (k - cy) / Ry
        if -1 < v < 1:
            ac = math.acos(v)
            th += [(ac + dy) % (2 * math.pi), (-ac + dy) % (2 * math.pi)]
    br = np.unique(np.array(th))
    gx, gw = np.polynomial.legendre.leggauss(q)
    X, Y, W = [], [], []
    for t0, t1 in zip(br[:-1], br[1:]):
        t = t0 + (t1 - t0) * (gx + 1) / 2
        X.append(cx + a * np.cos(t) * cp - b * np.sin(t) * sp)
        Y.append(cy + a * np.cos(t) * sp + b * np.sin(t) * cp)
        W.append(gw * (t1 - t0) / 2 * (-a * np.sin(t) * sp + b * np.cos(t) * cp))
    return np.concatenate(X), np.concatenate(Y), np.concatenate(W)
