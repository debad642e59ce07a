"""Pins of the oracle's patch-level results (no GPU).

Anchors, none of them the oracle's own code:
  * the CSR pattern and classification against brute force (dense curve
    sampling, closed-form inside tests);
  * every entry of the c = 1 matrix against int_{Omega^v} B_i B_j computed by
    Green's theorem on the hole boundary (tests/pins.py) -- this pins the
    cut-element rule (Sect. 3.1), hybrid Gauss (Sect. 3.2) and DWQ (Sect. 3.3)
    at once, and Table 1's "equal to standard Gauss up to machine precision";
  * WQ exactness for constant c on untrimmed patches (Sect. 2.1) and the
    closed-form row sums int B_i;
  * the visible area 1 - pi r^2 (and Green's area for the spline hole);
  * DWQ one-sided exactness (Sect. 3.3, the statement after step 4);
  * det J of the geometry against scipy derivatives of the control net;
  * L2 projection reproducing a function of the spline space (reading R9).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import synth
from pins import (GreenEntries, bspline_boundary_points, bvals, circle_boundary_points)


def dense(P, rp, col, val):
    return sp.csr_matrix((val, col, rp), shape=(P.n_rows, P.n_rows)).toarray()


def test_config1_counts_and_pattern():
    P = oracle.Patch(synth.config1())
    assert (P.n1, P.n_rows, P.nnz) == (18, 308, 6452)
    es, fs, act = P.states()
    assert np.bincount(es, minlength=3).tolist() == [44, 176, 36]
    assert np.bincount(fs, minlength=3).tolist() == [16, 200, 108]
    rp, col, _ = P.form()
    # brute-force pattern (reading R11)
    n = P.n1
    p = P.p
    act2 = act.reshape(n, n)
    k = 0
    for g in range(n * n):
        i1, i2 = g % n, g // n
        if act2[i2, i1] < 0:
            continue
        cols = [act2[j2, j1] for j2 in range(max(0, i2 - p), min(n, i2 + p + 1))
                for j1 in range(max(0, i1 - p), min(n, i1 + p + 1)) if act2[j2, j1] >= 0]
        assert list(col[rp[k]:rp[k + 1]]) == sorted(cols)
        k += 1


@pytest.mark.parametrize("trim", ["circle", "ellipse", "bspline3"])
def test_classification_against_dense_curve_samples(trim):
    rng = np.random.default_rng(7)
    if trim == "circle":
        t = synth.circle(0.5, 0.5, 0.27)
        th = np.linspace(0, 2 * math.pi, 400001)
        pts = np.stack([0.5 + 0.27 * np.cos(th), 0.5 + 0.27 * np.sin(th)], 1)
    elif trim == "ellipse":
        t = synth.ellipse(0.5, 0.5, 0.35, 0.2, 0.6)
        th = np.linspace(0, 2 * math.pi, 400001)
        pts = np.stack([0.5 + 0.35 * np.cos(th) * math.cos(0.6) - 0.2 * np.sin(th) * math.sin(0.6),
                        0.5 + 0.35 * np.cos(th) * math.sin(0.6) + 0.2 * np.sin(th) * math.cos(0.6)], 1)
    else:
        t = synth.bspline_curve(rng)
        from pins import periodic_curve
        pts = periodic_curve(t["ctrl"])(np.linspace(0, 12, 400001))
    nel = 23
    P = oracle.Patch(synth.make_spec(3, nel, t))
    es, fs, act = P.states()
    cut = np.zeros(nel * nel, bool)
    e1 = np.minimum((pts[:, 0] * nel).astype(int), nel - 1)
    e2 = np.minimum((pts[:, 1] * nel).astype(int), nel - 1)
    cut[e2 * nel + e1] = True
    assert np.array_equal(es == 2, cut)
    # non-cut elements: visible iff the centre is outside the hole
    for e in np.where(~cut)[0]:
        cx, cy = ((e % nel) + 0.5) / nel, ((e // nel) + 0.5) / nel
        assert (es[e] == 1) == (not oracle.curve_inside(t, cx, cy))
    # function states from element states
    n = nel + 3
    E = es.reshape(nel, nel)
    for g in range(n * n):
        i1, i2 = g % n, g // n
        sub = E[max(0, i2 - 3):min(nel, i2 + 1), max(0, i1 - 3):min(nel, i1 + 1)]
        ref = 0 if np.all(sub == 0) else (1 if np.all(sub == 1) else 2)
        assert fs[g] == ref
        assert (act[g] >= 0) == (ref != 0)


@pytest.mark.parametrize("p,nel", [(1, 6), (2, 5), (3, 7), (4, 4), (5, 6), (6, 3)])
def test_untrimmed_wq_exact_for_constant_c(p, nel):
    """WQ is exact when c is constant: interior-row WQ == element Gauss, and
    row sums equal int B_i = (U[i+p+1] - U[i]) / (p + 1) * ... in 2-D."""
    trim = {"kind": "none", "params": [], "ctrl": None}
    W = oracle.Patch(synth.make_spec(p, nel, trim, method="hybrid"))
    G = oracle.Patch(synth.make_spec(p, nel, trim, method="gauss"))
    rp, col, vw = W.form()
    _, _, vg = G.form()
    assert np.max(np.abs(vw - vg)) < 1e-16
    U = synth.open_uniform_knots(p, nel)
    n = len(U) - p - 1
    I = (U[p + 1:] - U[:n]) / (p + 1)
    rows = np.add.reduceat(vw, rp[:-1])
    ref = np.array([I[g % n] * I[g // n] for g in range(n * n)])
    assert np.max(np.abs(rows - ref)) < 1e-16
    assert abs(vw.sum() - 1.0) < 1e-14


@pytest.mark.parametrize("p,nel", [(2, 7), (3, 9), (5, 8)])
def test_graded_knots_wq_exact_and_green(p, nel):
    """Non-uniform simple knots (reading R1 admits them): WQ on an untrimmed
    graded patch equals element Gauss for constant c, row sums equal
    int B_i1 * int B_i2 = (U[i+p+1] - U[i]) / (p + 1) per direction, and on a
    trimmed graded patch every c = 1 entry of the hybrid matrix matches
    Green's theorem."""
    U1 = synth.graded_knots(p, nel, 1.2)
    U2 = synth.graded_knots(p, nel + 2, 0.85)
    trim = {"kind": "none", "params": [], "ctrl": None}
    W = oracle.Patch(synth.with_knots(synth.make_spec(p, 4, trim, method="hybrid"), U1, U2))
    G = oracle.Patch(synth.with_knots(synth.make_spec(p, 4, trim, method="gauss"), U1, U2))
    rp, col, vw = W.form()
    _, _, vg = G.form()
    assert np.max(np.abs(vw - vg)) < 1e-16
    n1, n2 = len(U1) - p - 1, len(U2) - p - 1
    I1 = (U1[p + 1:] - U1[:n1]) / (p + 1)
    I2 = (U2[p + 1:] - U2[:n2]) / (p + 1)
    rows = np.add.reduceat(vw, rp[:-1])
    ref = np.array([I1[g % n1] * I2[g // n1] for g in range(n1 * n2)])
    assert np.max(np.abs(rows - ref)) < 1e-16
    cx, cy, r = 0.47, 0.52, 0.29
    spec = synth.with_knots(synth.make_spec(p, 4, synth.circle(cx, cy, r), method="hybrid",
                                            cut_order=16), U1, U2)
    P = oracle.Patch(spec)
    rp, col, val = P.form()
    es, fs, act = P.states()
    Gr = GreenEntries(U1, U2, p, circle_boundary_points(cx, cy, r, U1, U2))
    gof = {int(act[g]): int(g) for g in np.flatnonzero(act >= 0)}
    worst = 0.0
    for row in range(P.n_rows):
        g = gof[row]
        for k in range(rp[row], rp[row + 1]):
            j = gof[int(col[k])]
            worst = max(worst, abs(val[k] - Gr.entry(g % n1, g // n1, j % n1, j // n1)))
    assert worst < 2e-15, worst


@pytest.mark.parametrize("method", ["gauss", "hybrid", "dwq"])
@pytest.mark.parametrize("p,nel", [(1, 7), (2, 6), (3, 5), (4, 8), (6, 6)])
def test_entries_against_greens_theorem_circle(method, p, nel):
    """Every entry int_{Omega^v} B_i B_j (c = 1) against Green's theorem on the
    circle; a high cut order makes the cut-element rule converge."""
    spec = synth.make_spec(p, nel, synth.circle(0.5, 0.5, 0.27), method=method, cut_order=16)
    P = oracle.Patch(spec)
    rp, col, val = P.form()
    es, fs, act = P.states()
    n = P.n1
    inv = np.full(P.n_rows, -1)
    inv[act[act >= 0]] = np.where(act >= 0)[0]
    U = spec["knots"][0]
    ge = GreenEntries(U, U, p, circle_boundary_points(0.5, 0.5, 0.27, U, U, q=40))
    err = 0.0
    for r in range(P.n_rows):
        gi = inv[r]
        for k in range(rp[r], rp[r + 1]):
            gj = inv[col[k]]
            ref = ge.entry(gi % n, gi // n, gj % n, gj // n)
            err = max(err, abs(val[k] - ref))
    assert err < 2e-15


@pytest.mark.parametrize("method", ["hybrid", "dwq"])
def test_entries_against_greens_theorem_spline_hole(method):
    rng = np.random.default_rng(synth.BASE_SEED + 2)
    t = synth.bspline_curve(rng)
    p, nel = 3, 9
    spec = synth.make_spec(p, nel, t, method=method, cut_order=16)
    P = oracle.Patch(spec)
    rp, col, val = P.form()
    es, fs, act = P.states()
    n = P.n1
    inv = np.full(P.n_rows, -1)
    inv[act[act >= 0]] = np.where(act >= 0)[0]
    U = spec["knots"][0]
    ge = GreenEntries(U, U, p, bspline_boundary_points(t["ctrl"], U, U, q=40))
    err = 0.0
    for r in range(P.n_rows):
        gi = inv[r]
        for k in range(rp[r], rp[r + 1]):
            gj = inv[col[k]]
            ref = ge.entry(gi % n, gi // n, gj % n, gj // n)
            err = max(err, abs(val[k] - ref))
    assert err < 5e-15


def test_visible_area_converges_with_cut_order():
    """Sum of all entries (c = 1) = |Omega^v| = 1 - pi r^2; the error is the
    cut rule's and vanishes as its order grows."""
    exact = 1.0 - math.pi * 0.27 ** 2
    errs = []
    for q in (3, 5, 8, 12):
        P = oracle.Patch(synth.make_spec(2, 16, synth.circle(0.5, 0.5, 0.27), cut_order=q))
        _, _, v = P.form()
        errs.append(abs(v.sum() - exact))
    assert errs[0] < 1e-7
    assert errs[-1] < 1e-13
    assert errs[1] < errs[0]


def test_table1_behaviour_naive_wq():
    """Table 1: hybrid Gauss and DWQ equal element Gauss to roundoff; naive WQ
    (c zeroed off S^r) does not (errors 1e-4 .. 1e-3 in the paper).  At p = 1
    the min-norm WQ rule of reading R2 on the R1 layout is element-local, so
    naive WQ is exact there too: the control starts at p = 2."""
    for p in (1, 2, 3, 4, 5, 6):
        mats = {}
        for m in ("gauss", "hybrid", "dwq", "naive"):
            P = oracle.Patch(synth.make_spec(p, 10, synth.circle(0.5, 0.5, 0.3), method=m))
            mats[m] = P.form()[2]
        ref = np.linalg.norm(mats["gauss"])
        assert np.linalg.norm(mats["hybrid"] - mats["gauss"]) / ref < 1e-14
        assert np.linalg.norm(mats["dwq"] - mats["gauss"]) / ref < 1e-14
        if p >= 2:
            assert np.linalg.norm(mats["naive"] - mats["gauss"]) / ref > 1e-6


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_dwq_one_sided_exactness(p):
    """After step 4 of Sect. 3.3 the rule of B_i restricted to one side of the
    disc integrates B_i B_j over that side exactly, for every coarse j."""
    nel = 9
    spec = synth.make_spec(p, nel, synth.circle(0.5, 0.5, 0.3), method="dwq")
    P = oracle.Patch(spec)
    U = spec["knots"][0]
    n = len(U) - p - 1
    gx, gw = np.polynomial.legendre.leggauss(p + 1)
    for s in (1, 4, nel - 1):
        t = U[p + s]
        for i in range(s, min(s + p, n)):
            for side in (0, 1):
                rule = P.dwq_rule(0, s, side, i)
                x, w = rule[:, 0], rule[:, 1]
                assert np.all(x < t) if side == 0 else np.all(x > t)
                for j in range(max(0, i - p), min(n, i + p + 1)):
                    ref = 0.0
                    for a, b in zip(U[:-1], U[1:]):
                        if b <= a or (side == 0 and a >= t) or (side == 1 and b <= t):
                            continue
                        xx = a + (b - a) * (gx + 1) / 2
                        ref += np.sum(gw * (b - a) / 2 * bvals(U, p, i, xx) * bvals(U, p, j, xx))
                    assert abs(np.sum(w * bvals(U, p, j, x)) - ref) < 1e-15


def test_dwq_choice_is_a_valid_regular_rectangle():
    P = oracle.Patch(synth.make_spec(4, 20, synth.circle(0.5, 0.5, 0.3), method="dwq"))
    es, fs, act = P.states()
    E = es.reshape(20, 20)
    n = P.n1
    nfound = 0
    for g in np.where(fs == 2)[0]:
        i1, i2 = g % n, g // n
        ch = P.dwq_choice(i1, i2)
        if ch[0] < 0:
            continue
        nfound += 1
        rng_ = []
        for d, (kind, s) in enumerate([(ch[0], ch[1]), (ch[2], ch[3])]):
            i = (i1, i2)[d]
            lo, hi = max(0, i - 4), min(19, i)
            rng_.append((lo, hi) if kind == 0 else ((lo, s - 1) if kind == 1 else (s, hi)))
            if kind:
                assert lo < s <= hi
        sub = E[rng_[1][0]:rng_[1][1] + 1, rng_[0][0]:rng_[0][1] + 1]
        assert sub.size > 0 and np.all(sub == 1)
        assert ch[0] != 0 or ch[2] != 0
    assert nfound > 0


def test_detj_against_scipy_and_greville_identity():
    rng = np.random.default_rng(11)
    p, nel = 3, 8
    net = synth.perturbed_bilinear_net(rng, p, nel)
    spec = synth.make_spec(p, nel, synth.circle(0.5, 0.5, 0.27),
                           geom={"kind": "spline", "ctrl": net}, coef={"kind": "detj"})
    P = oracle.Patch(spec)
    C = P.cgrid()
    x1, x2 = P.wq_grid(0), P.wq_grid(1)
    from scipy.interpolate import NdBSpline
    U = spec["knots"][0]
    geo = NdBSpline((U, U), np.transpose(net, (1, 0, 2)), p)
    X1, X2 = np.meshgrid(x1, x2, indexing="xy")
    pts = np.stack([X1.ravel(), X2.ravel()], 1)
    da = geo(pts, nu=(1, 0))
    db = geo(pts, nu=(0, 1))
    dj = (da[:, 0] * db[:, 1] - db[:, 0] * da[:, 1]).reshape(C.shape)
    assert np.max(np.abs(C - dj)) < 1e-12
    assert np.all(C > 0)
    # Greville net of the identity map: det J = 1, so the matrix equals c = 1
    g = synth.greville(U, p)
    G1, G2 = np.meshgrid(g, g, indexing="xy")
    ident = np.stack([G1, G2], 2)
    A = oracle.Patch(synth.make_spec(p, nel, synth.circle(0.5, 0.5, 0.27),
                                     geom={"kind": "spline", "ctrl": ident}, coef={"kind": "detj"}))
    B = oracle.Patch(synth.make_spec(p, nel, synth.circle(0.5, 0.5, 0.27)))
    assert np.max(np.abs(A.form()[2] - B.form()[2])) < 1e-15


def test_density_scales_linearly():
    rng = np.random.default_rng(5)
    dens = synth.density(rng, q=2, m=8)
    dens["coef"][:] = 2.5
    A = oracle.Patch(synth.make_spec(3, 8, synth.circle(0.5, 0.5, 0.25), coef=dens))
    B = oracle.Patch(synth.make_spec(3, 8, synth.circle(0.5, 0.5, 0.25)))
    assert np.max(np.abs(A.form()[2] - 2.5 * B.form()[2])) < 1e-15


@pytest.mark.parametrize("method", ["hybrid", "dwq", "gauss"])
def test_rhs_and_l2_projection_reproduce_spline(method):
    """Reading R9: f = sum a_j B_j gives b = M a exactly; with c = 1 M is
    symmetric and CG recovers a (CG pinned against scipy's sparse solver)."""
    rng = np.random.default_rng(2)
    spec = synth.make_spec(2, 12, synth.circle(0.5, 0.5, 0.27), method=method)
    P = oracle.Patch(spec)
    rp, col, val = P.form()
    f = synth.func_spline(spec, rng)
    b = P.rhs(f)
    es, fs, act = P.states()
    a = f["coef"].ravel()[act >= 0]
    M = sp.csr_matrix((val, col, rp), shape=(P.n_rows, P.n_rows))
    assert np.max(np.abs(b - M @ a)) < 1e-16
    u, it, rel = P.cg(rp, col, val, b, tol=1e-13)
    assert rel <= 1e-13
    Ms = 0.5 * (M + M.T)
    ref = spla.spsolve(Ms.tocsc(), b)
    assert np.max(np.abs(u - ref)) < 1e-8 * np.max(np.abs(ref))
    assert np.max(np.abs(u - a)) < 1e-8
    err, fn = P.l2_error(u, f)
    assert err < 1e-9


def test_l2_projection_converges():
    """Sect. 4.2: optimal rates; the error of projecting sin(2x)cos(3y) drops
    by about 2^(p+1) per refinement."""
    errs = []
    for nel in (8, 16, 32):
        spec = synth.make_spec(2, nel, synth.circle(0.5, 0.5, 0.27), method="hybrid")
        P = oracle.Patch(spec)
        rp, col, val = P.form()
        f = synth.func_sincos(2.0, 3.0)
        u, it, rel = P.cg(rp, col, val, P.rhs(f), tol=1e-13)
        errs.append(P.l2_error(u, f)[0])
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(rates) > 2.5


def test_density_grid_against_scipy():
    """c = rho(xi) (identity geometry) on the WQ grid against scipy's NdBSpline."""
    from scipy.interpolate import NdBSpline
    spec = synth.config5(nel=20)
    P = oracle.Patch(spec)
    C = P.cgrid()
    c = spec["coef"]
    dens = NdBSpline(tuple(c["knots"]), c["coef"].T, c["p"])
    X1, X2 = np.meshgrid(P.wq_grid(0), P.wq_grid(1), indexing="xy")
    ref = dens(np.stack([X1.ravel(), X2.ravel()], 1)).reshape(C.shape)
    assert np.max(np.abs(C - ref)) < 1e-14


def test_cg_solves_the_symmetric_part_of_a_nonsymmetric_matrix():
    """Reading R10: with c = det J the WQ rows give m_ij != m_ji; CG solves
    (M + M^T)/2 u = b (against scipy's direct solve of that system), not M."""
    rng = np.random.default_rng(6)
    p, nel = 3, 10
    net = synth.perturbed_bilinear_net(rng, p, nel)
    spec = synth.make_spec(p, nel, {"kind": "none"}, geom={"kind": "spline", "ctrl": net},
                           coef={"kind": "detj"}, method="hybrid")
    P = oracle.Patch(spec)
    rp, col, val = P.form()
    n = P.n_rows
    M = sp.csr_matrix((val, col, rp), shape=(n, n))
    asym = spla.norm(M - M.T) / spla.norm(M)
    assert asym > 1e-6  # the rule really is non-symmetric here
    b = P.rhs(synth.func_sincos(2.0, 3.0))
    u, it, rel = P.cg(rp, col, val, b, tol=1e-14)
    Ms = 0.5 * (M + M.T)
    ref = spla.spsolve(Ms.tocsc(), b)
    assert np.max(np.abs(u - ref)) <= 1e-10 * np.max(np.abs(ref))
    plain = spla.spsolve(M.tocsc(), b)
    assert np.max(np.abs(plain - ref)) > 1e3 * np.max(np.abs(u - ref))


@pytest.mark.parametrize("p,i,side,expected", [
    # p = 3, disc t = 1/2 on 8 uniform elements (h = 1/8).  The element left of
    # t holds its 2 base points at 1/3, 2/3 and gets p + 1 - 2 = 2 nested
    # points: the first in the middle gap (1/2), the second in the gap next to
    # t (5/6).  Right of t the gap next to t is the first one (1/6).
    (3, 4, 0, [1 + 1 / 3, 1 + 2 / 3, 2 + 1 / 3, 2 + 2 / 3, 3 + 1 / 3, 3 + 1 / 2, 3 + 2 / 3,
               3 + 5 / 6]),
    (3, 4, 1, [4 + 1 / 6, 4 + 1 / 3, 4 + 1 / 2, 4 + 2 / 3]),
    # p = 5: 4 nested points, one per gap (middle, next to t, far), the fourth
    # again in the middle (ties go to the middle gap): middle gap at its thirds
    (5, 6, 0, [1 + 1 / 3, 1 + 2 / 3, 2 + 1 / 3, 2 + 2 / 3, 3 + 1 / 6, 3 + 1 / 3, 3 + 4 / 9,
               3 + 5 / 9, 3 + 2 / 3, 3 + 5 / 6]),
])
def test_dwq_nested_points_by_hand(p, i, side, expected):
    """Reading R5 on a hand-worked case: the points of the DWQ rule of B_i on
    one side of the disc knot t = 1/2 (in units of h, from 0)."""
    spec = synth.make_spec(p, 8, synth.circle(0.5, 0.5, 0.2), method="dwq")
    P = oracle.Patch(spec)
    x = P.dwq_rule(0, 4, side, i)[:, 0]
    assert np.allclose(x, np.array(expected) / 8.0, rtol=0, atol=1e-15)


def test_l2_error_of_zero_is_the_norm_of_f():
    """or_l2_error at u = 0: relative error 1 and ||f|| = sqrt(int f^2), a
    closed form for sin(2x) cos(3y) on the untrimmed square."""
    import math
    P = oracle.Patch(synth.make_spec(3, 16, {"kind": "none"}))
    e, fn = P.l2_error(np.zeros(P.n_rows), synth.func_sincos(2.0, 3.0))
    ref = math.sqrt((0.5 - math.sin(4.0) / 8.0) * (0.5 + math.sin(6.0) / 12.0))
    assert abs(fn - ref) <= 1e-12 and abs(e - 1.0) <= 1e-14


@pytest.mark.parametrize("method", ["hybrid", "dwq", "naive", "gauss"])
def test_row_points_carry_the_rhs_rule(method):
    """or_row_points lists the rule that or_rhs applies (reading R9): summing
    w c f over the listed physical points gives or_rhs's b for the built-in
    kinds, so the pins of or_rhs carry over to an f given only as values."""
    rng = np.random.default_rng(9)
    spec = synth.make_spec(3, 9, synth.bspline_curve(rng, nc=12, radius=0.3, jitter=0.05),
                           geom={"kind": "spline", "ctrl": synth.perturbed_bilinear_net(rng, 3, 9)},
                           coef={"kind": "detj"}, method=method)
    P = oracle.Patch(spec)
    for fk, fn in [(synth.func_sinsin(), lambda x, y: np.sin(math.pi * x) * np.sin(math.pi * y)),
                   (synth.func_gauss(), lambda x, y: np.exp(-10 * ((x - 0.3) ** 2 + (y - 0.7) ** 2)))]:
        b = P.rhs(fk)
        b2 = P.rhs_from(fn)
        assert np.max(np.abs(b - b2)) <= 1e-15 * np.max(np.abs(b)) * 10
    if method == "gauss":
        return
    # the points of an interior row are its tensor WQ rule
    es, fs, act = P.states()
    g = [g for g in np.where(fs == 1)[0]][len(np.where(fs == 1)[0]) // 2]
    q = P.row_points(act[g])
    x1, x2 = P.wq_grid(0), P.wq_grid(1)
    assert set(np.round(q[:, 0], 15)) <= set(np.round(x1, 15))
    assert set(np.round(q[:, 1], 15)) <= set(np.round(x2, 15))


@pytest.mark.parametrize("method,geom", [("hybrid", "identity"), ("hybrid", "spline"),
                                         ("gauss", "spline"), ("dwq", "spline")])
def test_remark1_rows_equal_element_gauss_rows(method, geom):
    """Remark 1 of Sect. 3.2: the Gauss part of a cut row as one tensor rule over
    the whole support with c set to zero off the regular elements is the same
    quadrature as element Gauss on the regular elements, so every row without a
    region part equals or_form_row to rounding (c = 1 and c = det J)."""
    rng = np.random.default_rng(21)
    p, nel = 3, 12
    g = ({"kind": "spline", "ctrl": synth.perturbed_bilinear_net(rng, p, nel)}
         if geom == "spline" else None)
    spec = synth.make_spec(p, nel, synth.bspline_curve(rng, nc=12, radius=0.3, jitter=0.05),
                           geom=g, coef={"kind": "detj" if g else "one"}, method=method)
    P = oracle.Patch(spec)
    es, fs, act = P.states()
    rows = [int(act[g_]) for g_ in np.where(fs == 2)[0]]
    if method == "gauss":
        rows = list(range(P.n_rows))
    nchecked = 0
    for r in rows:
        res = P.form_row_remark1(r)
        if res is None:  # a DWQ row with a region part
            continue
        c1, v1 = res
        c0, v0 = P.form_row(r)
        assert np.array_equal(c0, c1)
        assert np.max(np.abs(v1 - v0)) <= 1e-15 * max(1.0, np.max(np.abs(v0)) * 10), r
        nchecked += 1
    assert nchecked > 0
