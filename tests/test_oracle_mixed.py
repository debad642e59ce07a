"""Pins of the oracle on mixed-continuity knot vectors (no GPU).

A knot of multiplicity m lowers the continuity there to C^{p-m} (Sect. 2.1);
the paper defers the WQ point layout to Hiemstra et al.  Reading R1 for such
vectors: elements are the knot spans, the zero-length spans of repeated knots
are empty (no points, no measure), and a non-empty element touching a knot of
multiplicity 2 or more gets p+1 points, every other one 2.

Anchors, none of them the oracle's own code:
  * the exactness of every WQ rule (Eq. 5) against scipy B-spline products
    integrated by numpy Gauss, for random multiplicity patterns p = 1..6 (a
    layout with too few points leaves the systems without an exact solution);
  * every entry of an untrimmed c = 1 matrix against the product of 1-D scipy
    integrals (Eq. 7 exact for c = 1);
  * the entries of cut rows of a trimmed c = 1 matrix against Green's theorem;
  * the one-sided exactness of a DWQ rule next to a repeated knot (Sect. 3.3);
  * the element states against the knot spans and dense samples of the curve.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from pins import GreenEntries, bvals, circle_boundary_points, line_product_integral

PATTERNS = {
    # degree: list of {interior knot index: multiplicity}
    1: [{}],
    2: [{3: 2}, {2: 2, 3: 2}, {1: 2, 6: 2}],
    3: [{3: 2}, {2: 3, 5: 2}, {1: 3, 2: 3, 3: 3}],
    4: [{4: 2}, {2: 4, 3: 2}, {1: 2, 6: 4}],
    5: [{4: 3}, {2: 5, 6: 2}],
    6: [{4: 2}, {3: 6, 5: 3}],
}
CASES = [(p, r) for p, rs in PATTERNS.items() for r in rs]


def _support_overlaps(U, p, i):
    n = len(U) - p - 1
    return [j for j in range(n) if min(U[i + p + 1], U[j + p + 1]) > max(U[i], U[j])]


@pytest.mark.parametrize("p,reps", CASES, ids=["p%d-%s" % (p, r) for p, r in CASES])
def test_wq_rules_are_exact_on_mixed_knots(p, reps):
    """Eq. 5 on a mixed-continuity vector: sum_k w_ik B_j(x_k) = int B_i B_j for
    every test function i and every trial j whose support overlaps B_i's."""
    U = synth.mixed_knots(p, 9, reps)
    x = oracle.wq_points(U, p)
    assert np.all(np.diff(x) > 0)
    n = len(U) - p - 1
    B = np.array([bvals(U, p, j, x) for j in range(n)])
    worst = 0.0
    for i in range(n):
        w = oracle.wq_weights(U, p, x, i)
        inside = (x > U[i]) & (x < U[i + p + 1])
        assert np.all(w[~inside] == 0.0)
        for j in _support_overlaps(U, p, i):
            exact = line_product_integral(U, p, i, j)
            worst = max(worst, abs(float(np.dot(w, B[j])) - exact))
    assert worst < 1e-15, worst


@pytest.mark.parametrize("p,reps", [(2, {3: 2}), (3, {2: 3, 5: 2}), (4, {2: 4, 3: 2}),
                                    (6, {3: 6, 5: 3})])
def test_point_counts_follow_the_multiplicities(p, reps):
    """Zero-length spans carry no point; an element next to a knot of
    multiplicity >= 2 carries p+1, every other one 2 (by counting the
    oracle's points per span)."""
    U = synth.mixed_knots(p, 9, reps)
    x = oracle.wq_points(U, p)
    vals, counts = np.unique(U, return_counts=True)
    mult = dict(zip(vals, counts))
    for j in range(p, len(U) - p - 1):
        a, b = U[j], U[j + 1]
        got = int(np.sum((x > a) & (x < b)))
        if not b > a:
            assert got == 0
        else:
            assert got == (p + 1 if max(mult[a], mult[b]) >= 2 else 2), (j, got)


def _spec(p, reps1, reps2, nel, trim, method="hybrid", cut_order=0, geom=False, coef=None):
    U1 = synth.mixed_knots(p, nel, reps1)
    U2 = synth.mixed_knots(p, nel, reps2)
    g = None
    if geom:
        rng = np.random.default_rng(p + nel)
        g = {"kind": "spline", "ctrl": synth.perturbed_bilinear_net(
            rng, p, len(U1) - 2 * p - 1, knots=(U1, U2))}
    spec = synth.make_spec(p, nel, trim, geom=g, coef=coef or ({"kind": "detj"} if geom else None),
                           method=method, cut_order=cut_order)
    return synth.with_knots(spec, U1, U2), U1, U2


@pytest.mark.parametrize("p,r1,r2", [(2, {2: 2}, {4: 2}), (3, {3: 3}, {2: 2, 5: 3}),
                                     (5, {4: 5}, {3: 2})])
def test_untrimmed_matrix_equals_tensor_products(p, r1, r2):
    """No trim, c = 1: every row is a WQ row and Eq. 7 is exact, so each entry
    is the product of two 1-D integrals of scipy B-splines (including the
    structural zeros of functions whose supports only touch at a repeated
    knot)."""
    spec, U1, U2 = _spec(p, r1, r2, 8, {"kind": "none", "params": [0.0] * 6, "ctrl": None,
                                        "keep_inside": False})
    P = oracle.Patch(spec)
    rp, col, val = P.form()
    es, fs, act = P.states()
    inv = {int(a): int(g) for g, a in enumerate(act) if a >= 0}
    n1 = P.n1
    I1, I2 = {}, {}
    worst = 0.0
    for r in range(P.n_rows):
        gi = inv[r]
        i1, i2 = gi % n1, gi // n1
        for k in range(rp[r], rp[r + 1]):
            gj = inv[int(col[k])]
            j1, j2 = gj % n1, gj // n1
            if (i1, j1) not in I1:
                I1[(i1, j1)] = line_product_integral(U1, p, i1, j1)
            if (i2, j2) not in I2:
                I2[(i2, j2)] = line_product_integral(U2, p, i2, j2)
            worst = max(worst, abs(val[k] - I1[(i1, j1)] * I2[(i2, j2)]))
    assert worst < 1e-15, worst


@pytest.mark.parametrize("method,p,r1,r2", [("hybrid", 2, {3: 2}, {6: 2}),
                                            ("gauss", 3, {3: 3}, {4: 2}),
                                            ("dwq", 3, {4: 2}, {2: 3, 6: 2}),
                                            ("dwq", 4, {3: 4}, {5: 2}),
                                            ("hybrid", 5, {4: 3, 7: 5}, {3: 2})])
def test_cut_rows_against_greens_theorem(method, p, r1, r2):
    """Circle hole, c = 1, every entry of sampled cut rows (and of sampled
    interior rows) against int over the square minus the disc by Green's
    theorem over the circle."""
    cx, cy, rad = 0.5, 0.5, 0.31
    spec, U1, U2 = _spec(p, r1, r2, 9, synth.circle(cx, cy, rad), method=method, cut_order=16)
    P = oracle.Patch(spec)
    rp, col, val = P.form()
    es, fs, act = P.states()
    inv = {int(a): int(g) for g, a in enumerate(act) if a >= 0}
    n1 = P.n1
    G = GreenEntries(U1, U2, p, circle_boundary_points(cx, cy, rad, U1, U2))
    rng = np.random.default_rng(p)
    cut = [int(act[g]) for g in np.where(fs == 2)[0]]
    inner = [int(act[g]) for g in np.where(fs == 1)[0]]
    rows = list(rng.choice(cut, size=min(30, len(cut)), replace=False))
    rows += list(rng.choice(inner, size=min(10, len(inner)), replace=False))
    worst = 0.0
    for r in rows:
        gi = inv[r]
        for k in range(rp[r], rp[r + 1]):
            gj = inv[int(col[k])]
            ex = G.entry(gi % n1, gi // n1, gj % n1, gj // n1)
            worst = max(worst, abs(val[k] - ex))
    assert worst < 5e-15, worst
    assert abs(P.visible_area() - (1.0 - math.pi * rad ** 2)) < 1e-13


def test_dwq_one_sided_exactness_next_to_a_repeated_knot():
    """A disc at a simple knot t whose window holds a repeated knot: the DWQ
    rule of every coarse function across t integrates B_i B_j exactly on each
    side of t, for every coarse trial j (Sect. 3.3, steps 1-4)."""
    p = 3
    reps = {3: 2, 6: 3}
    U = synth.mixed_knots(p, 9, reps)
    spec, U1, U2 = _spec(p, reps, reps, 9, synth.circle(0.5, 0.5, 0.3), method="dwq")
    P = oracle.Patch(spec)
    bp = U[p:len(U) - p]
    gx, gw = np.polynomial.legendre.leggauss(p + 1)
    checked = 0
    for s in range(1, len(bp) - 1):
        if not (bp[s - 1] < bp[s] < bp[s + 1]):
            continue  # discs are simple knots
        t = bp[s]
        near = [k for k in range(max(0, s - p), min(len(bp) - 1, s + p)) if bp[k + 1] == bp[k]]
        if not near:
            continue
        for i in range(len(U) - p - 1):
            if not (U[i] < t < U[i + p + 1]):
                continue
            for side in (0, 1):
                pts = P.dwq_rule(0, s, side, i)
                lo, hi = (U[i], t) if side == 0 else (t, U[i + p + 1])
                for j in _support_overlaps(U, p, i):
                    ex = 0.0
                    edges = np.unique(np.concatenate([[lo, hi], U[(U > lo) & (U < hi)]]))
                    for a, b in zip(edges[:-1], edges[1:]):
                        xx = a + (b - a) * (gx + 1) / 2
                        ex += np.sum(gw * (b - a) / 2 * bvals(U, p, i, xx) * bvals(U, p, j, xx))
                    got = float(np.sum(pts[:, 1] * bvals(U, p, j, pts[:, 0])))
                    assert abs(got - ex) < 1e-15, (s, i, side, j, got, ex)
                checked += 1
    assert checked > 0


def test_states_on_mixed_knots():
    """Zero-length spans are empty elements and nothing else is; the other
    elements are cut iff a dense sampling of the circle meets their open box,
    otherwise regular iff their centre is outside the disc; a function is
    exterior / interior / cut by the states of its non-empty support elements."""
    p = 3
    r1, r2 = {2: 3, 5: 2}, {4: 2}
    spec, U1, U2 = _spec(p, r1, r2, 12, synth.circle(0.47, 0.52, 0.29))
    P = oracle.Patch(spec)
    es, fs, act = P.states()
    b1, b2 = U1[p:len(U1) - p], U2[p:len(U2) - p]
    nel1, nel2 = len(b1) - 1, len(b2) - 1
    E = es.reshape(nel2, nel1)
    th = np.linspace(0, 2 * math.pi, 400001)
    X, Y = 0.47 + 0.29 * np.cos(th), 0.52 + 0.29 * np.sin(th)
    for e2 in range(nel2):
        for e1 in range(nel1):
            empty = not (b1[e1 + 1] > b1[e1] and b2[e2 + 1] > b2[e2])
            if empty:
                assert E[e2, e1] == 3
                continue
            hit = np.any((X > b1[e1]) & (X < b1[e1 + 1]) & (Y > b2[e2]) & (Y < b2[e2 + 1]))
            if hit:
                assert E[e2, e1] == 2
            else:
                xc, yc = (b1[e1] + b1[e1 + 1]) / 2, (b2[e2] + b2[e2 + 1]) / 2
                assert E[e2, e1] == (1 if math.hypot(xc - 0.47, yc - 0.52) > 0.29 else 0)
    n1 = len(U1) - p - 1
    for g in range(len(fs)):
        i1, i2 = g % n1, g // n1
        sts = [E[e2, e1] for e2 in range(max(0, i2 - p), min(nel2 - 1, i2) + 1)
               for e1 in range(max(0, i1 - p), min(nel1 - 1, i1) + 1) if E[e2, e1] != 3]
        want = 0 if all(s == 0 for s in sts) else (1 if all(s == 1 for s in sts) else 2)
        assert fs[g] == want


def test_reproduction_and_remark1_on_mixed_knots():
    """R9 on a C^0 / C^1 vector with c = det J and DWQ: f = sum a_j B_j in the
    patch's own basis gives b = M a; Remark 1's rows equal the element rows."""
    p = 3
    spec, U1, U2 = _spec(p, {3: 3, 6: 2}, {4: 2}, 10, synth.circle(0.5, 0.5, 0.3),
                         method="dwq", geom=True)
    P = oracle.Patch(spec)
    rp, col, val = P.form()
    f = synth.func_spline(spec, np.random.default_rng(4))
    b = P.rhs(f)
    es, fs, act = P.states()
    a = np.array([f["coef"].ravel()[g] for g in range(len(act)) if act[g] >= 0])
    Ma = np.array([np.dot(val[rp[r]:rp[r + 1]], a[col[rp[r]:rp[r + 1]]]) for r in range(P.n_rows)])
    assert np.max(np.abs(Ma - b)) <= 1e-14 * max(1.0, np.max(np.abs(b)))
    spec_h = dict(spec, method="hybrid")
    H = oracle.Patch(spec_h)
    es, fs, act = H.states()
    for g in np.where(fs == 2)[0][:40]:
        r = int(act[g])
        c1, v1 = H.form_row_remark1(r)
        c0, v0 = H.form_row(r)
        assert np.array_equal(c0, c1)
        assert np.max(np.abs(v1 - v0)) <= 1e-15 * max(1.0, 10 * np.max(np.abs(v0)))


def test_knot_vectors_the_reading_excludes():
    """Multiplicity p+1 inside the domain (C^-1) and non-open ends are refused;
    the extended basis (R16's arrays) is read on simple knots only."""
    p = 2
    with pytest.raises(ValueError):
        oracle.check_knots(synth.mixed_knots(p, 6, {3: 3}), p)
    with pytest.raises(ValueError):
        oracle.check_knots(np.array([0, 0, 0, 0, 0.5, 1, 1, 1.0]), p)
    oracle.check_knots(synth.mixed_knots(p, 6, {3: 2}), p)
    from oracle.extension import Extension
    spec, U1, U2 = _spec(p, {3: 2}, {}, 8, synth.circle(0.5, 0.5, 0.3))
    with pytest.raises(ValueError):
        Extension(oracle.Patch(spec))


def test_dwq_choice_by_enumeration_on_mixed_knots():
    """R7 with empty elements, by brute force over every cut function of a
    small patch: candidates R = R1 x R2 in the order (whole support; left part,
    knot ascending; right part, knot ascending), direction 1 outer; valid iff
    each element of R is regular or empty and each disc is a simple knot; the
    most elements win, then fewer discs, then the first.  Any admissible choice
    is exact at c = 1, so this pins the tie rules of the reading, not the
    mathematics."""
    p = 3
    spec, U1, U2 = _spec(p, {3: 2, 5: 3}, {4: 3}, 10, synth.circle(0.52, 0.47, 0.27), method="dwq")
    P = oracle.Patch(spec)
    es, fs, act = P.states()
    bps = [U1[p:len(U1) - p], U2[p:len(U2) - p]]
    nel = [len(b) - 1 for b in bps]
    E = es.reshape(nel[1], nel[0])
    n1 = len(U1) - p - 1
    crossing_empty = 0
    for g in np.where(fs == 2)[0]:
        i = (int(g) % n1, int(g) // n1)
        lo = [max(0, i[d] - p) for d in range(2)]
        hi = [min(nel[d] - 1, i[d]) for d in range(2)]
        opts = []
        for d in range(2):
            o = [(0, -1, lo[d], hi[d])]
            o += [(1, s, lo[d], s - 1) for s in range(lo[d] + 1, hi[d] + 1)]
            o += [(2, s, s, hi[d]) for s in range(lo[d] + 1, hi[d] + 1)]
            opts.append(o)
        best, key = None, None
        for a in opts[0]:
            for b in opts[1]:
                ok = True
                for d, o in ((0, a), (1, b)):
                    bp = bps[d]
                    if o[0] != 0 and not (bp[o[1] - 1] < bp[o[1]] < bp[o[1] + 1]):
                        ok = False
                sub = E[b[2]:b[3] + 1, a[2]:a[3] + 1]
                ok = ok and bool(np.all((sub == 1) | (sub == 3)))
                if not ok:
                    continue
                k = (sub.size, -((a[0] != 0) + (b[0] != 0)))
                if key is None or k > key:
                    best, key = (a[0], a[1], b[0], b[1]), k
        got = tuple(int(v) for v in P.dwq_choice(*i))
        want = best if best is not None else (-1, -1, -1, -1)
        assert got == want, (i, got, want)
        if best is not None:
            a_rng = [x for x in opts[0] if x[:2] == best[:2]][0]
            b_rng = [x for x in opts[1] if x[:2] == best[2:]][0]
            if np.any(E[b_rng[2]:b_rng[3] + 1, a_rng[2]:a_rng[3] + 1] == 3):
                crossing_empty += 1
    assert crossing_empty > 0  # some chosen regions span an empty element
