"""Pins of the oracle's row rules at a NON-constant coefficient c (no GPU).

Every rule of the paper is linear in c (Eq. 6 with the weights of Eqs. 4-5,
the DWQ rules of Sect. 3.3, element Gauss and the cut-element rule of
Sect. 3.1).  With identity geometry and a density spline whose coefficients
are an outer product, d_{k1 k2} = a_{k1} b_{k2}, the coefficient separates:

    c(xi1, xi2) = c1(xi1) c2(xi2),   c1 = sum a_k N_k,  c2 = sum b_k N_k,

and c1 != c2.  Then each tensor part of a row rule factors into two 1-D sums:

  * interior (WQ) row, Eq. 7:
        m_ij = [sum_k1 w1_k1 c1(x_k1) B_j1(x_k1)] [sum_k2 w2_k2 c2(x_k2) B_j2(x_k2)]
  * DWQ region R = R1 x R2 (Sect. 3.3): the same product over the two 1-D
    DWQ rules (or full WQ rules in a direction without a disc);
  * element Gauss on a regular element (p+1 points per direction): a product
    of two 1-D Gauss sums;
  * cut elements: sum over the cut rule's points of w B_i B_j c1 c2.

The 1-D sums are computed here from scipy B-splines, numpy Gauss-Legendre and
scipy's own evaluation of c1, c2; the only oracle pieces used are the 1-D
points and weights (pinned on their own by exactness and minimum norm in
test_oracle_core.py and by DWQ one-sided exactness in test_oracle_patch.py)
and the cut-rule point sets (pinned by Green's theorem at c = 1).  So a
transposed read of the c grid, c taken at another point of a DWQ rule, a
transposed c at the element Gauss points or a cut-rule c paired with the
wrong point each fail here, which no c = 1 pin can see.  The right-hand side
(reading R9: the row's own rule applied to f c) is pinned the same way with a
separable f = sin(a x) sin(b y).
"""
import numpy as np
import pytest
from scipy.interpolate import BSpline

import oracle
import synth
from pins import bvals


def separable_density(rng, q=2, m=7):
    V = synth.open_uniform_knots(q, m - q)
    a = rng.uniform(0.5, 2.0, size=m)
    b = rng.uniform(0.5, 2.0, size=m)
    # keep the two factors far apart, so that c1 != c2 everywhere it matters
    b = b[::-1] * 0.7 + 0.3
    coef = np.outer(b, a)  # [k2, k1]
    c1 = BSpline(V, a, q, extrapolate=False)
    c2 = BSpline(V, b, q, extrapolate=False)
    dens = {"kind": "density", "p": q, "knots": [V, V.copy()], "coef": coef}
    return dens, c1, c2


def _ev(f, x):
    return np.nan_to_num(f(np.asarray(x, float)), nan=0.0)


class Sums:
    """1-D sums of a test function against trial functions with c_d folded in."""

    def __init__(self, U, p, cd):
        self.U, self.p, self.cd = np.asarray(U, float), p, cd
        self.n = len(U) - p - 1
        self.nel = self.n - p
        self.x = oracle.wq_points(self.U, p)
        self.W = [oracle.wq_weights(self.U, p, self.x, i) for i in range(self.n)]
        self.gx, self.gw = np.polynomial.legendre.leggauss(p + 1)

    def rule_sum(self, x, w, j):
        return float(np.sum(w * _ev(self.cd, x) * bvals(self.U, self.p, j, x)))

    def wq(self, i, j):
        return self.rule_sum(self.x, self.W[i], j)

    def gauss_elem(self, e, i, j):
        a, b = self.U[self.p + e], self.U[self.p + e + 1]
        xx = a + (b - a) * (self.gx + 1) / 2
        w = self.gw * (b - a) / 2 * bvals(self.U, self.p, i, xx)
        return self.rule_sum(xx, w, j)


def region_range(kind, s, lo, hi):
    if kind == 0:
        return lo, hi
    if kind == 1:
        return lo, s - 1
    return s, hi


def expected_row(P, S, c1, c2, i1, i2, method, f=None):
    """Expected entries {(j1, j2): m_ij} (or, with f = (f1, f2), the rhs b_i)
    of row i = (i1, i2), from the tensor structure alone."""
    p = P.p
    es, fs, act = P.states()
    E = es.reshape(P.nel2, P.nel1)
    n1 = P.n1
    g = i2 * n1 + i1
    f1, f2 = (None, None) if f is None else f
    lo = [max(0, i1 - p), max(0, i2 - p)]
    hi = [min(i1, P.nel1 - 1), min(i2, P.nel2 - 1)]
    trials = [(j1, j2) for j2 in range(max(0, i2 - p), min(P.n2, i2 + p + 1))
              for j1 in range(max(0, i1 - p), min(n1, i1 + p + 1))
              if act[j2 * n1 + j1] >= 0]
    if f is not None:
        trials = [None]
    out = {t: 0.0 for t in trials}

    if fs[g] == 1 and method != "gauss":
        for t in trials:
            if t is None:
                out[t] = (float(np.sum(S[0].W[i1] * _ev(c1, S[0].x) * f1(S[0].x)))
                          * float(np.sum(S[1].W[i2] * _ev(c2, S[1].x) * f2(S[1].x))))
            else:
                out[t] = S[0].wq(i1, t[0]) * S[1].wq(i2, t[1])
        return out
    rg = [(1, 0), (1, 0)]  # empty region
    if method == "dwq":
        ch = P.dwq_choice(i1, i2)
        if ch[0] >= 0:
            rules = []
            for d, (kind, s) in enumerate([(ch[0], ch[1]), (ch[2], ch[3])]):
                i = (i1, i2)[d]
                rg[d] = region_range(kind, s, lo[d], hi[d])
                if kind == 0:
                    m = S[d].W[i] != 0
                    rules.append((S[d].x[m], S[d].W[i][m]))
                else:
                    r = P.dwq_rule(d, s, 0 if kind == 1 else 1, i)
                    rules.append((r[:, 0], r[:, 1]))
            cd, fd = (c1, c2), (f1, f2)
            for t in trials:
                prod = 1.0
                for d in range(2):
                    x, w = rules[d]
                    v = w * _ev(cd[d], x)
                    v = v * (fd[d](x) if t is None else bvals(S[d].U, p, t[d], x))
                    prod *= float(np.sum(v))
                out[t] += prod
    for e2 in range(lo[1], hi[1] + 1):
        for e1 in range(lo[0], hi[0] + 1):
            st = E[e2, e1]
            inR = rg[0][0] <= e1 <= rg[0][1] and rg[1][0] <= e2 <= rg[1][1]
            if st == 1 and not inR:
                for t in trials:
                    if t is None:
                        out[t] += _gauss_f(S[0], e1, i1, c1, f1) * _gauss_f(S[1], e2, i2, c2, f2)
                    else:
                        out[t] += S[0].gauss_elem(e1, i1, t[0]) * S[1].gauss_elem(e2, i2, t[1])
            elif st == 2:
                r = P.cut_rule(e1, e2)
                x, y, w = r[:, 0], r[:, 1], r[:, 2]
                base = (w * bvals(S[0].U, p, i1, x) * bvals(S[1].U, p, i2, y)
                        * _ev(c1, x) * _ev(c2, y))
                for t in trials:
                    if t is None:
                        out[t] += float(np.sum(base * f1(x) * f2(y)))
                    else:
                        out[t] += float(np.sum(base * bvals(S[0].U, p, t[0], x)
                                               * bvals(S[1].U, p, t[1], y)))
    return out


def _gauss_f(Sd, e, i, cd, fd):
    a, b = Sd.U[Sd.p + e], Sd.U[Sd.p + e + 1]
    xx = a + (b - a) * (Sd.gx + 1) / 2
    return float(np.sum(Sd.gw * (b - a) / 2 * bvals(Sd.U, Sd.p, i, xx) * _ev(cd, xx) * fd(xx)))


def _patch(p, nel, method, seed, trim=None):
    rng = np.random.default_rng(seed)
    dens, c1, c2 = separable_density(rng)
    spec = synth.make_spec(p, nel, trim or synth.circle(0.47, 0.53, 0.29), coef=dens,
                           method=method)
    P = oracle.Patch(spec)
    S = [Sums(spec["knots"][d], p, (c1, c2)[d]) for d in range(2)]
    return spec, P, S, c1, c2


def _rows_by_kind(P, method):
    es, fs, act = P.states()
    rows = np.where(act >= 0)[0]
    interior = [g for g in rows if fs[g] == 1]
    cut = [g for g in rows if fs[g] == 2]
    if method == "dwq":
        dwq = [g for g in cut if P.dwq_choice(g % P.n1, g // P.n1)[0] >= 0]
        other = [g for g in cut if g not in set(dwq)]
        return interior, dwq, other, act
    return interior, cut, [], act


def _check_rows(P, S, c1, c2, rows, act, method, tol=1e-14):
    inv = {int(a): int(g) for g, a in enumerate(act) if a >= 0}
    worst = 0.0
    for g in rows:
        i1, i2 = g % P.n1, g // P.n1
        col, val = P.form_row(int(act[g]))
        exp = expected_row(P, S, c1, c2, i1, i2, method)
        assert len(col) == len(exp)
        scale = max(abs(v) for v in exp.values())
        for c, v in zip(col, val):
            gj = inv[int(c)]
            err = abs(v - exp[(gj % P.n1, gj // P.n1)])
            worst = max(worst, err / scale)
    assert worst < tol, worst


@pytest.mark.parametrize("p,nel", [(2, 9), (3, 10), (4, 11)])
def test_wq_rows_factor_at_separable_c(p, nel):
    """Interior rows (Eq. 7): each entry is the product of two 1-D sums,
    direction 1 with c1 and direction 2 with c2."""
    spec, P, S, c1, c2 = _patch(p, nel, "hybrid", 31 + p)
    interior, _, _, act = _rows_by_kind(P, "hybrid")
    rng = np.random.default_rng(p)
    pick = rng.choice(interior, size=min(40, len(interior)), replace=False)
    _check_rows(P, S, c1, c2, pick, act, "hybrid")


@pytest.mark.parametrize("p,nel", [(2, 9), (3, 10), (4, 11), (5, 12)])
def test_dwq_rows_factor_at_separable_c(p, nel):
    """DWQ rows (Sect. 3.3): region part = product of the two 1-D DWQ rules
    with c1, c2; plus element Gauss on the other regular elements and the cut
    rule on cut elements, each with c = c1 c2 evaluated here."""
    spec, P, S, c1, c2 = _patch(p, nel, "dwq", 41 + p)
    _, dwq, other, act = _rows_by_kind(P, "dwq")
    assert len(dwq) > 0
    # every region shape: a disc in direction 1, in direction 2, in both
    kinds = {}
    for g in dwq:
        ch = P.dwq_choice(g % P.n1, g // P.n1)
        kinds.setdefault((ch[0] != 0, ch[2] != 0), []).append(g)
    assert (True, False) in kinds and (False, True) in kinds, kinds.keys()
    pick = []
    for k, v in kinds.items():
        pick += v[:6]
    _check_rows(P, S, c1, c2, pick + other[:4], act, "dwq")


@pytest.mark.parametrize("p", [2, 4])
def test_hybrid_rows_factor_at_separable_c(p):
    """Hybrid Gauss rows (Sect. 3.2): element Gauss per regular element (a
    product of 1-D Gauss sums) plus the cut rule."""
    spec, P, S, c1, c2 = _patch(p, 10, "hybrid", 51 + p)
    _, cut, _, act = _rows_by_kind(P, "hybrid")
    _check_rows(P, S, c1, c2, cut[::3], act, "hybrid")


@pytest.mark.parametrize("method", ["hybrid", "dwq"])
def test_rhs_factors_at_separable_c_and_f(method):
    """Reading R9 at c = c1 c2 and f = sin(a x) sin(b y): interior rows give
    b_i = [sum w1 c1 f1][sum w2 c2 f2]; cut rows the same decomposition as
    their matrix rows."""
    p = 3
    spec, P, S, c1, c2 = _patch(p, 10, method, 61)
    fa, fb = 2.3, 1.1
    f1 = lambda x: np.sin(fa * np.asarray(x))  # noqa: E731
    f2 = lambda y: np.sin(fb * np.asarray(y))  # noqa: E731
    b = P.rhs({"kind": "sinsin", "prm": [fa, fb, 0.0, 0.0]})
    es, fs, act = P.states()
    worst = 0.0
    rows = np.where(act >= 0)[0]
    for g in rows[::5]:
        i1, i2 = g % P.n1, g // P.n1
        exp = expected_row(P, S, c1, c2, i1, i2, method, f=(f1, f2))[None]
        worst = max(worst, abs(b[act[g]] - exp) / max(abs(exp), 1e-300) if abs(exp) > 1e-12
                    else abs(b[act[g]] - exp))
    assert worst < 5e-14, worst
