"""Pins of the oracle on patches trimmed by several curves (no GPU).

The paper's trimming examples (Sect. 4, the domains of its figures) bound the
visible domain by one or more curves; here the visible domain is the
intersection of every curve's kept side.  Two cases: two disjoint holes (a
circle and a cubic B-spline), and an annulus (the inside of a circle kept, an
ellipse inside it removed), a domain bounded by two loops.

Anchors, none of them the oracle's own code:
  * every c = 1 entry int_{Omega^v} B_i B_j by Green's theorem over every
    boundary loop (tests/pins.py): full square minus both holes, or disc
    minus ellipse;
  * the visible area against its closed form, converging with the cut order;
  * the classification against dense samples of every curve.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from pins import (GreenEntries, bspline_boundary_points, circle_boundary_points,
                  ellipse_boundary_points)


class LoopEntries:
    """Exact c = 1 entries over the visible domain of several loops, each
    loop's boundary integral cached (GreenEntries gives full - int_loop)."""

    def __init__(self, kind, U, p, loops):
        self.kind = kind
        self.G = [GreenEntries(U, U, p, b) for b in loops]
        self.U, self.p = U, p

    def entry(self, i1, i2, j1, j2):
        e = [g.entry(i1, i2, j1, j2) for g in self.G]  # full - int_D for each loop D
        if self.kind == "holes":  # full - int_D1 - int_D2
            return e[0] + e[1] - (self.G[0]._I1[(min(i1, j1), max(i1, j1))]
                                  * self.G[0]._I2[(min(i2, j2), max(i2, j2))])
        return e[1] - e[0]  # int_disc - int_ellipse


def _case(kind, p, nel, method, cut_order=0):
    if kind == "holes":
        trims = synth.two_holes()
    else:
        trims = synth.annulus()
    spec = synth.make_spec(p, nel, trims[0], extra_trims=trims[1:], method=method,
                           cut_order=cut_order)
    U = spec["knots"][0]
    if kind == "holes":
        c = trims[0]["params"]
        loops = [circle_boundary_points(c[0], c[1], c[2], U, U),
                 bspline_boundary_points(trims[1]["ctrl"], U, U)]
    else:
        c = trims[0]["params"]
        e = trims[1]["params"]
        loops = [circle_boundary_points(c[0], c[1], c[2], U, U),
                 ellipse_boundary_points(e[0], e[1], e[2], e[3], e[4], U, U)]
    return spec, U, loops


@pytest.mark.parametrize("kind", ["holes", "annulus"])
@pytest.mark.parametrize("method,p", [("hybrid", 2), ("dwq", 3), ("gauss", 2), ("hybrid", 4)])
def test_entries_against_greens_theorem_over_all_loops(kind, method, p):
    nel = 14
    spec, U, loops = _case(kind, p, nel, method, cut_order=16)
    ex_ = LoopEntries(kind, U, p, loops)
    P = oracle.Patch(spec)
    rp, col, val = P.form()
    es, fs, act = P.states()
    inv = {int(a): int(g) for g, a in enumerate(act) if a >= 0}
    n = P.n1
    rng = np.random.default_rng(p)
    cut_rows = [int(act[g]) for g in np.where(fs == 2)[0]]
    rows = list(rng.choice(cut_rows, size=min(40, len(cut_rows)), replace=False))
    worst = 0.0
    for r in rows:
        gi = inv[r]
        i1, i2 = gi % n, gi // n
        for k in range(rp[r], rp[r + 1]):
            gj = inv[int(col[k])]
            ex = ex_.entry(i1, i2, gj % n, gj // n)
            worst = max(worst, abs(val[k] - ex))
    assert worst < 5e-15, worst


def test_visible_areas_converge_to_the_closed_forms():
    for kind in ("holes", "annulus"):
        spec, U, loops = _case(kind, 2, 20, "hybrid", cut_order=16)
        P = oracle.Patch(spec)
        if kind == "holes":
            X, Y, W = loops[1]
            exact = 1.0 - math.pi * 0.17 ** 2 - abs(float(np.sum(X * W)))
        else:
            exact = math.pi * 0.44 ** 2 - math.pi * 0.2 * 0.13
        assert abs(P.visible_area() - exact) < 1e-13, (kind, P.visible_area() - exact)
        # at the default order the rule is an approximation that converges
        P3 = oracle.Patch(dict(spec, cut_order=0))
        assert abs(P3.visible_area() - exact) < 1e-6


def test_classification_against_dense_samples_of_every_curve():
    from pins import periodic_curve
    for kind in ("holes", "annulus"):
        spec, U, loops = _case(kind, 2, 24, "hybrid")
        P = oracle.Patch(spec)
        es, fs, act = P.states()
        E = es.reshape(24, 24)
        trims = [spec["trim"]] + spec["extra_trims"]
        cut = np.zeros((24, 24), bool)
        for t in trims:
            if t["kind"] == "circle":
                th = np.linspace(0, 2 * math.pi, 400001)
                pts = np.stack([t["params"][0] + t["params"][2] * np.cos(th),
                                t["params"][1] + t["params"][2] * np.sin(th)], 1)
            elif t["kind"] == "ellipse":
                cx, cy, a, b, ph = t["params"][:5]
                th = np.linspace(0, 2 * math.pi, 400001)
                pts = np.stack([cx + a * np.cos(th) * math.cos(ph) - b * np.sin(th) * math.sin(ph),
                                cy + a * np.cos(th) * math.sin(ph) + b * np.sin(th) * math.cos(ph)], 1)
            else:
                cv = periodic_curve(t["ctrl"])
                pts = cv(np.linspace(0, len(t["ctrl"]), 400001))
            idx = np.clip((pts * 24).astype(int), 0, 23)
            cut[idx[:, 1], idx[:, 0]] = True
        assert np.array_equal(E == 2, cut), kind
        # an element away from every curve is visible iff its centre is
        xc = (np.arange(24) + 0.5) / 24
        X1, X2 = np.meshgrid(xc, xc, indexing="xy")
        for e2 in range(24):
            for e1 in range(24):
                if cut[e2, e1]:
                    continue
                x, y = X1[e2, e1], X2[e2, e1]
                vis = True
                for t in trims:
                    inside = oracle.curve_inside(t, x, y)
                    vis = vis and (inside if t.get("keep_inside") else not inside)
                assert (E[e2, e1] == 1) == vis
