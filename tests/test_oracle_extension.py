"""Pins of the oracle's extended B-splines (readings R15-R17) against what the
mathematics fixes independently of oracle/extension.py:

- on uniform knots the extension coefficients are Hoellig's Lagrange form
  prod_{mu != a} (j - l - mu) / (a - mu) (a closed form, not the blossom route);
- the extended space reproduces polynomials: the B-spline coefficients of a
  tensor polynomial, fitted by scipy's spline interpolation, satisfy
  c_active = E c_inner (uniform and graded knots, different per direction;
  circle, straight-line and cubic B-spline trims);
- every chosen array is all-inner and no all-inner array anywhere in the patch
  is nearer (brute force over all arrays, no search window);
- the extended L2 projection of a polynomial returns its coefficients exactly;
- E^T M E equals the dense product, and its condition number stays bounded as
  the trim cuts ever thinner slivers while that of M_s grows without bound.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.interpolate import make_interp_spline

import oracle
import synth
from oracle.extension import Extension


def _lagrange(t, a, p):
    v = 1.0
    for mu in range(p + 1):
        if mu != a:
            v *= (t - mu) / (a - mu)
    return v


@pytest.mark.parametrize("p,nel,r", [(2, 16, 0.27), (3, 18, 0.3), (4, 24, 0.31), (6, 30, 0.28)])
def test_uniform_coefficients_are_lagrange(p, nel, r):
    spec = synth.make_spec(p, nel, synth.circle(0.5, 0.5, r))
    P = oracle.Patch(spec)
    X = Extension(P)
    assert X.n_outer > 0
    U = spec["knots"][0]
    h = 1.0 / nel
    checked = 0
    for g, (l1, l2) in X.arrays.items():
        j1, j2 = g % P.n1, g // P.n1
        e1, e2 = X.coefs[g]
        for j, l, e in ((j1, l1, e1), (j2, l2, e2)):
            lo, hi = min(j, l) + 1, max(j, l + p) + p
            if not np.allclose(np.diff(U[lo:hi + 1]), h, rtol=0, atol=1e-15):
                continue  # the closed form holds on uniform knots only
            ref = np.array([_lagrange(j - l, a, p) for a in range(p + 1)])
            assert np.max(np.abs(e - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref))), (j, l, e, ref)
            checked += 1
    assert checked == 2 * X.n_outer


def _poly_coefs(U, p, poly):
    """B-spline coefficients of the 1-D polynomial `poly` (numpy.polynomial
    coefficients, lowest first) by scipy's interpolation at the Greville points."""
    x = synth.greville(np.asarray(U), p)
    y = np.polynomial.polynomial.polyval(x, poly)
    return make_interp_spline(x, y, k=p, t=np.asarray(U)).c


def _graded_spec(p, nel, r, ratios=(1.12, 0.9)):
    spec = synth.make_spec(p, nel, synth.circle(0.5, 0.5, r))
    return synth.with_knots(spec, synth.graded_knots(p, nel, ratios[0]),
                            synth.graded_knots(p, nel, ratios[1]))


@pytest.mark.parametrize("p,nel,r,graded", [
    (2, 16, 0.27, False), (3, 18, 0.3, True), (4, 20, 0.31, True), (5, 24, 0.29, True),
    (3, 12, "line", False), (4, 22, "bspline", True),
])
def test_extension_reproduces_polynomials(p, nel, r, graded):
    if r == "line":
        spec = synth.line_trim_spec(p, nel=nel)
    elif r == "bspline":
        tr = synth.bspline_curve(np.random.default_rng(7), nc=8, radius=0.28, jitter=0.15,
                                 relative_jitter=True)
        spec = synth.with_knots(synth.make_spec(p, nel, tr), synth.graded_knots(p, nel, 1.1),
                                synth.graded_knots(p, nel, 0.92))
    elif graded:
        spec = _graded_spec(p, nel, r)
    else:
        spec = synth.make_spec(p, nel, synth.circle(0.5, 0.5, r))
    P = oracle.Patch(spec)
    X = Extension(P)
    es, fs, act = P.states()
    rng = np.random.default_rng(5)
    U1, U2 = spec["knots"]
    for deg1, deg2 in ((p, p), (p, 0), (1, p), (0, 0)):
        c1 = _poly_coefs(U1, p, rng.standard_normal(deg1 + 1))
        c2 = _poly_coefs(U2, p, rng.standard_normal(deg2 + 1))
        c = np.outer(c2, c1).ravel()  # g = i2 * n1 + i1
        cA = c[act >= 0]
        cI = c[X.inner]
        assert np.max(np.abs(X.E @ cI - cA)) <= 1e-11 * np.max(np.abs(c))


def test_arrays_are_inner_and_nearest_by_brute_force():
    spec = _graded_spec(3, 20, 0.31)
    P = oracle.Patch(spec)
    X = Extension(P)
    p, n1, n2 = P.p, P.n1, P.n2
    I = X.inner.reshape(n2, n1)
    # every array of the patch, all-inner flag by a sliding window product
    L2, L1 = np.meshgrid(np.arange(n2 - p), np.arange(n1 - p), indexing="ij")
    allin = np.ones_like(L1, dtype=bool)
    for a2 in range(p + 1):
        for a1 in range(p + 1):
            allin &= I[L2 + a2, L1 + a1]
    for g, (l1, l2) in X.arrays.items():
        j1, j2 = g % n1, g // n1
        assert allin[l2, l1]
        d = (2 * L1 + p - 2 * j1) ** 2 + (2 * L2 + p - 2 * j2) ** 2
        d = np.where(allin, d, np.iinfo(np.int64).max)
        dmin = d.min()
        assert d[l2, l1] == dmin
        cand = np.argwhere(d == dmin)  # rows (l2, l1) in ascending order
        assert tuple(cand[0]) == (l2, l1)
    # the outer functions are exactly the active ones with no regular element
    es, fs, act = P.states()
    for g in range(n1 * n2):
        if act[g] < 0:
            assert not X.inner[g] and not X.outer[g]
            continue
        i1, i2 = g % n1, g // n1
        regs = [es[e2 * P.nel1 + e1] == oracle.extension.ELEM_REGULAR
                for e2 in range(max(0, i2 - p), min(P.nel2 - 1, i2) + 1)
                for e1 in range(max(0, i1 - p), min(P.nel1 - 1, i1) + 1)]
        assert X.inner[g] == any(regs) and X.outer[g] == (not any(regs))


@pytest.mark.parametrize("method", ["hybrid", "dwq"])
def test_extended_projection_of_a_polynomial_is_exact(method):
    p, nel = 3, 14
    spec = synth.make_spec(p, nel, synth.circle(0.5, 0.5, 0.29), method=method)
    P = oracle.Patch(spec)
    X = Extension(P)
    U1, U2 = spec["knots"]
    rng = np.random.default_rng(3)
    c = np.outer(_poly_coefs(U2, p, rng.standard_normal(p + 1)),
                 _poly_coefs(U1, p, rng.standard_normal(p + 1)))
    f = {"kind": "spline", "prm": [0.0] * 4, "p": p, "knots": [U1, U2], "coef": c}
    rp, col, val = P.form()
    es, fs, act = P.states()
    u, x = X.project(f, rp, col, val)
    cA = c.ravel()[act >= 0]
    assert np.max(np.abs(u - cA)) <= 1e-10 * np.max(np.abs(cA))
    # a spline outside the extended space is not reproduced
    f2 = dict(f)
    f2["coef"] = rng.uniform(-1, 1, size=c.shape)
    u2, _ = X.project(f2, rp, col, val)
    assert np.max(np.abs(u2 - f2["coef"].ravel()[act >= 0])) > 1e-3


def test_extended_mass_matches_dense_product():
    spec = synth.config2(p=3, nel=12)
    P = oracle.Patch(spec)
    X = Extension(P)
    rp, col, val = P.form()
    xr, xc, xv = X.mass(rp, col, val)
    n, m = P.n_rows, X.n_inner
    M = sp.csr_matrix((val, col, rp), shape=(n, n)).toarray()
    E = X.E.toarray()
    ref = E.T @ M @ E
    got = sp.csr_matrix((xv, xc, xr), shape=(m, m)).toarray()
    assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref)
    # the pattern holds every numerically nonzero entry, each row ascending
    assert np.count_nonzero(ref[got == 0]) == 0
    for a in range(m):
        assert np.all(np.diff(xc[xr[a]:xr[a + 1]]) > 0)


@pytest.mark.parametrize("p,nel", [(2, 16), (3, 16)])
def test_extended_mass_is_well_conditioned_for_every_sliver(p, nel):
    P0 = oracle.Patch(synth.make_spec(p, nel, {"kind": "none"}))
    r0, c0, v0 = P0.form()
    cond0 = np.linalg.cond(sp.csr_matrix((v0, c0, r0), shape=(P0.n_rows,) * 2).toarray())
    worst_plain = 0.0
    for r in (0.2, 0.27, 0.2713, 0.305, 0.31):
        P = oracle.Patch(synth.make_spec(p, nel, synth.circle(0.5, 0.5, r)))
        X = Extension(P)
        rp, col, val = P.form()
        M = sp.csr_matrix((val, col, rp), shape=(P.n_rows,) * 2).toarray()
        Ms = 0.5 * (M + M.T)
        Me = np.asarray(X.E.T @ Ms @ X.E)
        assert np.allclose(Me, Me.T, rtol=0, atol=1e-15 * np.abs(Me).max())
        assert np.linalg.eigvalsh(Me).min() > 0
        assert np.linalg.cond(Me) <= 100.0 * cond0
        worst_plain = max(worst_plain, np.linalg.cond(Ms))
    assert worst_plain >= 1e12 * cond0
