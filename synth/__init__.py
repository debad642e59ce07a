"""Seeded synthetic patch generators shared by the oracle tests, the GPU tests
and the benchmark.

This module only draws inputs -- knot vectors, trimming curves, geometry control
nets, density coefficients, target functions -- shaped like the paper's
examples (Sect. 4: trimmed bi-variate B-spline patches with line, circle and
curvy trims, degrees up to 6).  It contains none of the method's arithmetic:
no basis evaluation, quadrature, classification or formation.

A *patch spec* is a plain dict:
    p        degree (same in both directions)
    nel      (nel1, nel2) elements per direction
    knots    [U1, U2] open uniform knot vectors (float64 arrays)
    trim     {"kind": "none"|"circle"|"ellipse"|"bspline3", "params": [...],
              "ctrl": (nc, 2) array or None, "keep_inside": bool}
    geom     {"kind": "identity"} or {"kind": "spline", "ctrl": (n2, n1, 2)}
    coef     {"kind": "one"|"detj"} or {"kind": "density", "p": q,
              "knots": [V1, V2], "coef": (m2, m1)}
    method   "gauss" | "hybrid" | "dwq" | "naive"
    cut_order  Gauss order on cut-element pieces (0 -> p + 1)
    extra_trims  (optional) further trimming curves, each a dict like trim; the
             visible domain is the intersection of every curve's kept side
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 20210108

TRIM_KINDS = {"none": 0, "circle": 1, "ellipse": 2, "bspline3": 3}
GEOM_KINDS = {"identity": 0, "spline": 1}
COEF_KINDS = {"one": 0, "detj": 1, "density": 2}
METHODS = {"gauss": 0, "hybrid": 1, "dwq": 2, "naive": 3}
FUNC_KINDS = {"spline": 0, "sinsin": 1, "sincos": 2, "gauss": 3}


def open_uniform_knots(p: int, nel: int, a: float = 0.0, b: float = 1.0) -> np.ndarray:
    """p+1 copies of each end, nel-1 equally spaced simple interior knots."""
    inner = [a + (b - a) * k / nel for k in range(1, nel)]
    return np.array([a] * (p + 1) + inner + [b] * (p + 1), dtype=np.float64)


def graded_knots(p: int, nel: int, ratio: float = 1.15, a: float = 0.0, b: float = 1.0) -> np.ndarray:
    """Open knot vector with simple interior knots graded geometrically (each
    element `ratio` times the previous one), for non-uniform parity cases."""
    h = ratio ** np.arange(nel)
    x = np.concatenate([[0.0], np.cumsum(h)])
    x = a + (b - a) * x / x[-1]
    x[-1] = b
    return np.array([a] * (p + 1) + list(x[1:-1]) + [b] * (p + 1), dtype=np.float64)


def mixed_knots(p: int, nel: int, reps: dict, a: float = 0.0, b: float = 1.0) -> np.ndarray:
    """Open knot vector over nel equal elements whose k-th interior knot
    (k = 1 .. nel-1) appears reps.get(k, 1) times: continuity C^{p-m} at a
    knot of multiplicity m (mixed-continuity cases)."""
    U = [a] * (p + 1)
    for k in range(1, nel):
        U += [a + (b - a) * k / nel] * int(reps.get(k, 1))
    U += [b] * (p + 1)
    return np.array(U, dtype=np.float64)


def with_knots(spec, U1, U2):
    """The spec on other knot vectors (same degree; nel from the knots)."""
    s = dict(spec)
    s["knots"] = [np.asarray(U1, dtype=np.float64), np.asarray(U2, dtype=np.float64)]
    p = spec["p"]
    s["nel"] = (len(U1) - 2 * p - 1, len(U2) - 2 * p - 1)
    return s


def greville(U: np.ndarray, p: int) -> np.ndarray:
    n = len(U) - p - 1
    return np.array([U[i + 1:i + p + 1].mean() for i in range(n)], dtype=np.float64)


def circle(cx=0.5, cy=0.5, r=0.27, keep_inside=False):
    return {"kind": "circle", "params": [cx, cy, r], "ctrl": None, "keep_inside": keep_inside}


def line(x0, y0, x1, y1, keep_inside=False):
    """Half-plane trim by the straight line through (x0, y0) and (x1, y1);
    "inside" is the side left of the direction (x0, y0) -> (x1, y1)."""
    return {"kind": "line", "params": [x0, y0, x1, y1], "ctrl": None, "keep_inside": keep_inside}


# The line trim of the paper's mass-matrix example (its figure is not part of
# the text): the line through (0, 0.31) and (1, 0.77), the part below it kept.
LINE_TRIM = (0.0, 0.31, 1.0, 0.77)


def line_trim_spec(p, nel=10, method="hybrid", cut_order=0):
    """Unit square, identity geometry, c = 1, the straight-line trim above."""
    return make_spec(p, nel, line(*LINE_TRIM, keep_inside=False), method=method,
                     cut_order=cut_order)


def ellipse(cx, cy, a, b, phi, keep_inside=False):
    return {"kind": "ellipse", "params": [cx, cy, a, b, phi], "ctrl": None,
            "keep_inside": keep_inside}


def bspline_curve(rng: np.random.Generator, nc=12, radius=0.3, jitter=0.05,
                  center=(0.5, 0.5), relative_jitter=False, keep_inside=False):
    """Closed periodic cubic B-spline: nc control points at angles 2 pi k / nc,
    counter-clockwise, radius `radius` + U(-jitter, jitter) (or times
    1 + U(-jitter, jitter) with relative_jitter)."""
    ang = 2.0 * math.pi * np.arange(nc) / nc
    u = rng.uniform(-1.0, 1.0, size=nc)
    rad = radius * (1.0 + jitter * u) if relative_jitter else radius + jitter * u
    ctrl = np.stack([center[0] + rad * np.cos(ang), center[1] + rad * np.sin(ang)], axis=1)
    return {"kind": "bspline3", "params": [0.0] * 6, "ctrl": ctrl.astype(np.float64),
            "keep_inside": keep_inside}


def perturbed_bilinear_net(rng: np.random.Generator, p: int, nel: int, amplitude_h=0.05,
                           knots=None):
    """Control net P_ij = A(gamma_i1, gamma_i2) + delta_ij: A the bilinear map
    with corners (0,0), (1,0), (1.15,1.1), (0.05,0.95); gamma the Greville
    abscissae (of open uniform knots, or of knots = (U1, U2)); delta a smooth
    seeded field of three Fourier modes scaled so that max |delta| =
    amplitude_h / nel."""
    if knots is None:
        ga = gb = greville(open_uniform_knots(p, nel), p)
    else:
        ga, gb = greville(np.asarray(knots[0]), p), greville(np.asarray(knots[1]), p)
    g1, g2 = np.meshgrid(ga, gb, indexing="xy")  # [i2, i1]
    c00, c10, c11, c01 = map(np.array, ([0.0, 0.0], [1.0, 0.0], [1.15, 1.1], [0.05, 0.95]))
    A = ((1 - g1)[..., None] * (1 - g2)[..., None] * c00 + g1[..., None] * (1 - g2)[..., None] * c10
         + g1[..., None] * g2[..., None] * c11 + (1 - g1)[..., None] * g2[..., None] * c01)
    delta = np.zeros_like(A)
    for comp in range(2):
        for m in range(1, 4):
            a, b = rng.uniform(-1, 1, size=2)
            phi, psi = rng.uniform(0, 2 * math.pi, size=2)
            delta[..., comp] += a * np.sin(2 * math.pi * m * g1 + phi) * b * np.cos(2 * math.pi * m * g2 + psi)
    mx = np.max(np.linalg.norm(delta, axis=2))
    if mx > 0:
        delta *= (amplitude_h / nel) / mx
    return (A + delta).astype(np.float64)


def density(rng: np.random.Generator, q=2, m=32, lo=0.5, hi=2.0):
    V = open_uniform_knots(q, m - q)
    return {"kind": "density", "p": q, "knots": [V, V.copy()],
            "coef": rng.uniform(lo, hi, size=(m, m)).astype(np.float64)}


def make_spec(p, nel, trim, geom=None, coef=None, method="hybrid", cut_order=0, extra_trims=None):
    nel = (nel, nel) if np.isscalar(nel) else tuple(nel)
    spec = {
        "p": int(p),
        "nel": nel,
        "knots": [open_uniform_knots(p, nel[0]), open_uniform_knots(p, nel[1])],
        "trim": trim,
        "geom": geom or {"kind": "identity"},
        "coef": coef or {"kind": "one"},
        "method": method,
        "cut_order": int(cut_order),
    }
    if extra_trims:
        spec["extra_trims"] = list(extra_trims)
    return spec


def two_holes(rng=None):
    """A circular hole and a seeded 10-point spline hole, disjoint."""
    rng = rng or np.random.default_rng(BASE_SEED + 6)
    return [circle(0.3, 0.32, 0.17),
            bspline_curve(rng, nc=10, radius=0.16, jitter=0.02, center=(0.68, 0.66))]


def annulus():
    """The ring between an ellipse (a hole) and the circle around it (the
    inside kept): a visible domain bounded by two loops."""
    return [circle(0.5, 0.5, 0.44, keep_inside=True),
            ellipse(0.52, 0.47, 0.2, 0.13, 0.4)]


# ---------------------------------------------------------------------------
# the workloads (shapes of the paper's examples, Sect. 4)

def config1(method="hybrid"):
    """p = 2, 16 x 16 elements, unit square, identity geometry, c = 1, circular
    hole r = 0.27 at (0.5, 0.5)."""
    return make_spec(2, 16, circle(0.5, 0.5, 0.27), method=method)


def config2(p=4, nel=512, method="hybrid", seed=None):
    """Perturbed bilinear geometry (c = det J) with a seeded 12-point cubic
    B-spline hole of radius 0.3 +- 0.05."""
    rng = np.random.default_rng(BASE_SEED + 2 if seed is None else seed)
    trim = bspline_curve(rng, nc=12, radius=0.3, jitter=0.05)
    net = perturbed_bilinear_net(rng, p, nel)
    return make_spec(p, nel, trim, geom={"kind": "spline", "ctrl": net},
                     coef={"kind": "detj"}, method=method)


def config3(p=4, nel=1024, method="hybrid", seed=None):
    rng = np.random.default_rng(BASE_SEED + 3 if seed is None else seed)
    net = perturbed_bilinear_net(rng, p, nel)
    return make_spec(p, nel, circle(0.5, 0.5, 0.3), geom={"kind": "spline", "ctrl": net},
                     coef={"kind": "detj"}, method=method)


def config4_patch(rng: np.random.Generator, method="hybrid"):
    p = int(rng.integers(2, 7))
    nel = (int(rng.integers(16, 257)), int(rng.integers(16, 257)))
    if rng.uniform() < 0.5:
        trim = ellipse(0.5, 0.5, float(rng.uniform(0.1, 0.4)), float(rng.uniform(0.1, 0.4)),
                       float(rng.uniform(0.0, math.pi)))
    else:
        trim = bspline_curve(rng, nc=8, radius=float(rng.uniform(0.15, 0.35)), jitter=0.15,
                             relative_jitter=True)
    return make_spec(p, nel, trim, method=method)


def config5(nel=256, method="hybrid", seed=None):
    rng = np.random.default_rng(BASE_SEED + 5 if seed is None else seed)
    return make_spec(3, nel, circle(0.5, 0.5, 0.25), coef=density(rng), method=method)


def func_spline(spec, rng: np.random.Generator):
    """f = sum_j a_j B_j in the patch's own basis (for reproduction tests)."""
    U1, U2 = spec["knots"]
    p = spec["p"]
    n1, n2 = len(U1) - p - 1, len(U2) - p - 1
    return {"kind": "spline", "prm": [0.0] * 4, "p": p, "knots": [U1, U2],
            "coef": rng.uniform(-1.0, 1.0, size=(n2, n1)).astype(np.float64)}


def func_sinsin(a=math.pi, b=math.pi):
    return {"kind": "sinsin", "prm": [a, b, 0.0, 0.0]}


def func_sincos(a=2.0, b=3.0):
    return {"kind": "sincos", "prm": [a, b, 0.0, 0.0]}


def func_gauss(k=10.0, x0=0.3, y0=0.7):
    return {"kind": "gauss", "prm": [k, x0, y0, 0.0]}
