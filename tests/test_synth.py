"""The synthetic inputs follow the stated recipe (seeds, sizes, value ranges,
geometry and curve shapes of the paper's examples, Sect. 4), independently of
the oracle: the control net is compared with the bilinear map of the Greville
abscissae, det J is evaluated with scipy's B-splines on a dense grid, the
hole's control points are read back in polar form."""
import math

import numpy as np
import pytest
from scipy.interpolate import BSpline

import synth


def _bilinear(g1, g2):
    c00, c10, c11, c01 = map(np.array, ([0.0, 0.0], [1.0, 0.0], [1.15, 1.1], [0.05, 0.95]))
    return ((1 - g1)[..., None] * (1 - g2)[..., None] * c00
            + g1[..., None] * (1 - g2)[..., None] * c10
            + g1[..., None] * g2[..., None] * c11 + (1 - g1)[..., None] * g2[..., None] * c01)


@pytest.mark.parametrize("p,nel", [(3, 24), (4, 40), (5, 32)])
def test_config2_geometry_recipe(p, nel):
    spec = synth.config2(p=p, nel=nel)
    assert spec["p"] == p and spec["nel"] == (nel, nel)
    assert spec["coef"] == {"kind": "detj"}
    U = spec["knots"][0]
    assert np.allclose(U, np.r_[[0.0] * (p + 1), np.arange(1, nel) / nel, [1.0] * (p + 1)])
    net = spec["geom"]["ctrl"]  # [i2, i1, 2]
    g = np.array([U[i + 1:i + p + 1].mean() for i in range(nel + p)])
    G1, G2 = np.meshgrid(g, g, indexing="xy")
    delta = net - _bilinear(G1, G2)
    # the perturbation is rescaled so that its largest displacement is 0.05 h
    assert np.max(np.linalg.norm(delta, axis=2)) == pytest.approx(0.05 / nel, rel=1e-12)
    # det J > 0 on a dense grid of the parameter square (scipy's B-splines)
    x = np.linspace(0.0, 1.0, 101)[1:-1]
    n = nel + p
    B = np.array([BSpline(U, np.eye(n)[i], p)(x) for i in range(n)])          # [i][x]
    dB = np.array([BSpline(U, np.eye(n)[i], p).derivative()(x) for i in range(n)])
    xa = dB.T @ net[..., 0].T @ B      # d x / d xi1 at (x_a, x_b): [a][b]
    ya = dB.T @ net[..., 1].T @ B
    xb = B.T @ net[..., 0].T @ dB
    yb = B.T @ net[..., 1].T @ dB
    assert np.min(xa * yb - xb * ya) > 0.0


def test_config2_hole_recipe():
    spec = synth.config2(p=4, nel=16)
    t = spec["trim"]
    assert t["kind"] == "bspline3" and not t["keep_inside"]
    c = t["ctrl"] - 0.5
    r = np.hypot(c[:, 0], c[:, 1])
    ang = np.mod(np.arctan2(c[:, 1], c[:, 0]), 2 * math.pi)
    assert len(r) == 12
    assert np.all(r >= 0.25) and np.all(r <= 0.35)
    assert np.allclose(ang, 2 * math.pi * np.arange(12) / 12, atol=1e-12)  # counter-clockwise


def test_seeds_are_base_plus_config_number():
    assert synth.BASE_SEED == 20210108
    a = synth.config2(p=3, nel=8)["trim"]["ctrl"]
    rng = np.random.default_rng(20210108 + 2)
    b = synth.bspline_curve(rng, nc=12, radius=0.3, jitter=0.05)["ctrl"]
    assert np.array_equal(a, b)


def test_config1_config3_config5():
    s1 = synth.config1()
    assert (s1["p"], s1["nel"], s1["trim"]["params"]) == (2, (16, 16), [0.5, 0.5, 0.27])
    assert s1["coef"] == {"kind": "one"} and s1["geom"] == {"kind": "identity"}
    s3 = synth.config3(p=6, nel=32)
    assert s3["trim"]["params"] == [0.5, 0.5, 0.3] and s3["coef"] == {"kind": "detj"}
    s5 = synth.config5(nel=24)
    assert s5["p"] == 3 and s5["trim"]["params"] == [0.5, 0.5, 0.25]
    d = s5["coef"]
    assert d["kind"] == "density" and d["p"] == 2 and d["coef"].shape == (32, 32)
    assert np.all(d["coef"] >= 0.5) and np.all(d["coef"] <= 2.0)
    # 32 coefficients of a degree-2 open uniform spline: 30 density elements
    assert len(d["knots"][0]) == 32 + 2 + 1


def test_config4_ranges():
    rng = np.random.default_rng(synth.BASE_SEED + 4)
    kinds = []
    for _ in range(200):
        s = synth.config4_patch(rng)
        assert 2 <= s["p"] <= 6
        assert all(16 <= n <= 256 for n in s["nel"])
        t = s["trim"]
        kinds.append(t["kind"])
        if t["kind"] == "ellipse":
            cx, cy, a, b, phi = t["params"]
            assert (cx, cy) == (0.5, 0.5) and 0.1 <= a <= 0.4 and 0.1 <= b <= 0.4
            assert 0.0 <= phi <= math.pi
        else:
            c = t["ctrl"] - 0.5
            r = np.hypot(c[:, 0], c[:, 1])
            assert len(r) == 8 and np.all(r >= 0.15 * 0.85 - 1e-12) and np.all(r <= 0.35 * 1.15 + 1e-12)
    frac = kinds.count("ellipse") / len(kinds)
    assert 0.35 <= frac <= 0.65
