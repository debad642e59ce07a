"""Pins of the oracle's univariate building blocks (no GPU).

Each check compares against something other than the oracle itself: scipy's
B-splines, numpy's Gauss-Legendre and least-squares routines, closed forms
(integral of a B-spline, exactness of Gauss rules), and the defining
properties of knot insertion (Eq. 10) and weighted quadrature (Eq. 5).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from pins import bvals, line_product_integral


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_bspline_matches_scipy_and_partition_of_unity(p):
    rng = np.random.default_rng(p)
    inner = np.sort(rng.uniform(0.05, 0.95, size=7))
    U = np.concatenate([[0.0] * (p + 1), inner, [1.0] * (p + 1)])
    n = len(U) - p - 1
    xs = rng.uniform(0, 1, size=40)
    for x in xs:
        vals = [oracle.bspline(U, p, i, x) for i in range(n)]
        ref = [bvals(U, p, i, x)[()] for i in range(n)]
        assert np.allclose(vals, ref, atol=1e-14)
        assert abs(sum(vals) - 1.0) < 1e-14
        # derivative against scipy's derivative
        d = [oracle.bspline(U, p, i, x, deriv=True) for i in range(n)]
        from pins import bsp
        dref = [np.nan_to_num(bsp(U, p, i).derivative()(x)) for i in range(n)]
        assert np.allclose(d, dref, atol=1e-10)


@pytest.mark.parametrize("p", [1, 3, 6])
def test_bspline_integral_closed_form(p):
    U = synth.open_uniform_knots(p, 9)
    n = len(U) - p - 1
    gx, gw = np.polynomial.legendre.leggauss(p + 2)
    for i in range(n):
        s = 0.0
        for a, b in zip(U[:-1], U[1:]):
            if b > a:
                for x, w in zip(a + (b - a) * (gx + 1) / 2, gw * (b - a) / 2):
                    s += w * oracle.bspline(U, p, i, x)
        assert abs(s - (U[i + p + 1] - U[i]) / (p + 1)) < 1e-15


@pytest.mark.parametrize("q", [1, 2, 3, 5, 7, 12, 20])
def test_gauss_legendre_against_numpy_and_exactness(q):
    x, w = oracle.gauss_legendre(q)
    xr, wr = np.polynomial.legendre.leggauss(q)
    assert np.allclose(x, xr, atol=1e-15)
    assert np.allclose(w, wr, atol=1e-15)
    for k in range(2 * q):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14


def test_minnorm_against_numpy():
    rng = np.random.default_rng(0)
    for m, N in [(3, 3), (5, 6), (9, 10), (13, 14), (7, 19)]:
        A = rng.normal(size=(m, N))
        b = rng.normal(size=m)
        w = oracle.minnorm(A, b)
        assert np.allclose(A @ w, b, atol=1e-12)
        assert np.allclose(w, np.linalg.pinv(A) @ b, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_knot_insertion_preserves_the_spline(p):
    """Eq. 10: sum_j c_j B_j == sum_k c'_k B'_k pointwise (scipy evaluation)."""
    rng = np.random.default_rng(10 + p)
    U = synth.open_uniform_knots(p, 8)
    c = rng.normal(size=len(U) - p - 1)
    from scipy.interpolate import BSpline
    for t in [U[p + 3], 0.37, U[p + 5]]:
        Un, cn = oracle.insert_knot(U, p, t, c)
        assert np.all(np.diff(Un) >= 0) and np.sum(Un == t) == np.sum(U == t) + 1
        xs = rng.uniform(0, 1, 50)
        assert np.allclose(BSpline(U, c, p)(xs), BSpline(Un, cn, p)(xs), atol=1e-13)


@pytest.mark.parametrize("p,nel", [(1, 5), (2, 6), (3, 8), (4, 3), (5, 9), (6, 2), (6, 11)])
def test_wq_layout_and_exactness(p, nel):
    """Reading R1 point counts; Eq. 5 exactness against scipy-integrated
    products for every trial function overlapping the test function."""
    U = synth.open_uniform_knots(p, nel)
    x = oracle.wq_points(U, p)
    nq_expected = 2 * (p + 1) + 2 * (nel - 2) if nel >= 2 else p + 1
    assert len(x) == nq_expected
    assert np.all(np.diff(x) > 0)
    assert not np.any(np.isin(x, U))
    n = len(U) - p - 1
    for i in range(n):
        w = oracle.wq_weights(U, p, x, i)
        outside = (x <= U[i]) | (x >= U[i + p + 1])
        assert np.all(w[outside] == 0)
        for j in range(max(0, i - p), min(n, i + p + 1)):
            lhs = np.sum(w * bvals(U, p, j, x))
            assert abs(lhs - line_product_integral(U, p, i, j)) < 1e-15


def test_wq_minimum_norm():
    """Reading R2: the weights are the minimum-norm solution (numpy pinv)."""
    p = 3
    U = synth.open_uniform_knots(p, 7)
    x = oracle.wq_points(U, p)
    n = len(U) - p - 1
    for i in range(n):
        cols = np.where((x > U[i]) & (x < U[i + p + 1]))[0]
        rows = [j for j in range(n) if min(U[i + p + 1], U[j + p + 1]) > max(U[i], U[j])]
        A = np.array([[bvals(U, p, j, x[k]) for k in cols] for j in rows])
        b = np.array([line_product_integral(U, p, i, j) for j in rows])
        w = oracle.wq_weights(U, p, x, i)
        assert np.allclose(w[cols], np.linalg.pinv(A) @ b, atol=1e-14)


def test_curve_primitives_against_brute_force():
    rng = np.random.default_rng(3)
    trims = [synth.circle(0.5, 0.5, 0.27), synth.ellipse(0.45, 0.55, 0.3, 0.15, 0.7),
             synth.bspline_curve(rng)]
    from pins import periodic_curve
    for t in trims:
        # dense polygon of the curve
        if t["kind"] == "circle":
            th = np.linspace(0, 2 * math.pi, 200001)
            P = np.stack([0.5 + 0.27 * np.cos(th), 0.5 + 0.27 * np.sin(th)], 1)
        elif t["kind"] == "ellipse":
            th = np.linspace(0, 2 * math.pi, 200001)
            cx, cy, a, b, ph = t["params"]
            P = np.stack([cx + a * np.cos(th) * math.cos(ph) - b * np.sin(th) * math.sin(ph),
                          cy + a * np.cos(th) * math.sin(ph) + b * np.sin(th) * math.cos(ph)], 1)
        else:
            tau = np.linspace(0, len(t["ctrl"]), 200001)
            P = periodic_curve(t["ctrl"])(tau)
        for o in (0, 1):
            for s in rng.uniform(0.15, 0.85, size=6):
                hits = oracle.curve_line_hits(t, o, s)
                v = P[:, o] - s
                idx = np.where(np.sign(v[:-1]) != np.sign(v[1:]))[0]
                ref = np.sort(P[idx, 1 - o])
                assert len(hits) == len(ref)
                assert np.allclose(hits, ref, atol=1e-4)
    # area by Green / closed form
    for t in trims:
        if t["kind"] == "bspline3":
            from pins import bspline_boundary_points, polygon_area
            ref = polygon_area(bspline_boundary_points(t["ctrl"], [0, 1], [0, 1]))
        elif t["kind"] == "circle":
            ref = math.pi * 0.27 ** 2
        else:
            ref = math.pi * 0.3 * 0.15
        assert abs(oracle.curve_area(t, 4) - ref) < 1e-14


def test_curve_inside_against_winding_number():
    rng = np.random.default_rng(4)
    t = synth.bspline_curve(rng, nc=8, radius=0.3, jitter=0.15, relative_jitter=True)
    from pins import periodic_curve
    P = periodic_curve(t["ctrl"])(np.linspace(0, 8, 40001))
    for x, y in rng.uniform(0.1, 0.9, size=(200, 2)):
        d = P - np.array([x, y])
        ang = np.arctan2(d[:, 1], d[:, 0])
        wind = np.sum(np.angle(np.exp(1j * np.diff(ang)))) / (2 * math.pi)
        assert oracle.curve_inside(t, x, y) == (abs(round(wind)) == 1)
