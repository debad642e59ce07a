"""Two-phase right-hand side (tw_rhs_points / tw_rhs_values) against the
oracle, for target functions the library cannot evaluate itself.

Sect. 4.2 projects a given f; reading R9 makes b_i row i's own quadrature rule
applied to f c.  The library lists every point its rules evaluate f at, the
caller fills the values, and tw_rhs_values applies the rules.  The oracle lists
the rule of each of its rows (or_row_points) and the test sums w c f there, so
the same f, given only as values, meets both sides."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def f_np(x, y):
    """A target outside the built-in kinds (no product form, no spline)."""
    return np.exp(0.7 * x) * np.cos(3.0 * y) + x * x * y - 0.3 * np.sin(5.0 * x * y)


def f_torch(X):
    x, y = X[:, 0], X[:, 1]
    return torch.exp(0.7 * x) * torch.cos(3.0 * y) + x * x * y - 0.3 * torch.sin(5.0 * x * y)


def _specs():
    rng = np.random.default_rng(23)
    return [
        ("config1-hybrid", synth.config1("hybrid")),
        ("spline-geometry-dwq", synth.config2(p=3, nel=24, method="dwq", seed=11)),
        ("spline-geometry-hybrid", synth.config2(p=4, nel=20, method="hybrid", seed=12)),
        ("spline-geometry-gauss", synth.config2(p=2, nel=16, method="gauss", seed=13)),
        ("naive", synth.make_spec(3, 14, synth.circle(0.5, 0.5, 0.3), method="naive")),
        ("density-dwq", synth.config5(nel=20, method="dwq")),
        ("ellipse-dwq-p5", synth.make_spec(5, 18, synth.ellipse(0.5, 0.5, 0.33, 0.21, 0.4),
                                           geom={"kind": "spline",
                                                 "ctrl": synth.perturbed_bilinear_net(rng, 5, 18)},
                                           coef={"kind": "detj"}, method="dwq")),
        ("untrimmed", synth.make_spec(3, 10, {"kind": "none", "params": [], "ctrl": None,
                                              "keep_inside": False})),
    ]


@pytest.mark.parametrize("name,spec", _specs(), ids=[n for n, _ in _specs()])
def test_rhs_values_of_an_arbitrary_f_against_the_oracle(name, spec):
    from paper_2101_08053_gb300 import api
    P = api.Patch(spec)
    xi, X = P.rhs_points()
    info = P.info
    p1 = spec["p"] + 1
    ng = P.nq1 * P.nq2
    # the list starts with the WQ grid, k1 fastest
    x1 = P.table(0).cpu().numpy()
    x2 = P.table(1).cpu().numpy()
    xin = xi.cpu().numpy()
    assert np.array_equal(xin[:ng, 0], np.tile(x1, P.nq2))
    assert np.array_equal(xin[:ng, 1], np.repeat(x2, P.nq1))
    # then Gauss points, cut-rule points (table 5's order), region points
    cut = P.table(5).cpu().numpy().reshape(-1, 3)
    assert len(cut) == info[10]
    nrest = len(xin) - ng - len(cut)
    # naive rows use the grid and the cut rule only; untrimmed patches have
    # no cut rows at all
    assert nrest >= 0
    assert (nrest > 0) == (spec["trim"]["kind"] != "none" and spec["method"] != "naive")
    ngauss = 0
    if spec["method"] != "dwq":
        assert nrest % (p1 * p1) == 0
        ngauss = nrest // (p1 * p1)
    if spec["method"] != "dwq" and len(cut):
        g0 = ng + ngauss * p1 * p1
        assert np.array_equal(xin[g0:g0 + len(cut)], cut[:, :2])
    # an f outside the built-in kinds, given only by its values
    b = P.rhs_values(f_torch(X)).cpu().numpy()
    O = oracle.Patch(spec)
    ref = O.rhs_from(f_np)
    assert b.shape == ref.shape
    rel = np.linalg.norm(b - ref) / np.linalg.norm(ref)
    assert rel <= TOL, rel
    # a built-in kind through the values path equals tw_rhs
    Xn = X.cpu().numpy()
    fs = np.sin(math.pi * Xn[:, 0]) * np.sin(math.pi * Xn[:, 1])
    b2 = P.rhs_values(torch.from_numpy(fs).cuda()).cpu().numpy()
    b3 = P.rhs(synth.func_sinsin()).cpu().numpy()
    assert np.linalg.norm(b2 - b3) <= 1e-14 * np.linalg.norm(b3)


@pytest.mark.parametrize("method", ["hybrid", "dwq", "gauss", "naive"])
def test_rhs_values_of_a_spline_reproduce_the_matrix(method):
    """Reading R9 through the values path: for f = sum_j a_j B_j in the patch's
    own basis, given only by its values at the listed points, every row's rule
    gives b_i = sum_j m_ij a_j exactly (the same rule forms M), so b = M a to
    rounding (identity geometry; f evaluated here by scipy)."""
    from scipy.interpolate import BSpline
    from paper_2101_08053_gb300 import api
    spec = synth.make_spec(3, 18, synth.circle(0.47, 0.52, 0.29), method=method)
    P = api.Patch(spec)
    rng = np.random.default_rng(8)
    U1, U2 = spec["knots"]
    p = spec["p"]
    n1, n2 = len(U1) - p - 1, len(U2) - p - 1
    a = rng.uniform(-1, 1, size=(n2, n1))
    xi, _ = P.rhs_points(physical=False)
    x = xi.cpu().numpy()
    B1 = np.stack([np.nan_to_num(BSpline(U1, np.eye(n1)[j], p, extrapolate=False)(x[:, 0]))
                   for j in range(n1)], 1)
    B2 = np.stack([np.nan_to_num(BSpline(U2, np.eye(n2)[j], p, extrapolate=False)(x[:, 1]))
                   for j in range(n2)], 1)
    fv = np.einsum("kb,ba,ka->k", B2, a, B1)
    b = P.rhs_values(torch.from_numpy(fv).cuda()).cpu().numpy()
    rp, col, val = [t.cpu().numpy() for t in P.form_mass("fp64")]
    M = sp.csr_matrix((val, col, rp), shape=(P.n_rows, P.n_rows))
    es, fs, act = [t.cpu().numpy() for t in P.states()]
    aa = np.zeros(P.n_rows)
    aa[act[act >= 0]] = a.ravel()[act >= 0]
    r = M @ aa
    assert np.linalg.norm(b - r) <= 1e-13 * np.linalg.norm(r), np.linalg.norm(b - r) / np.linalg.norm(r)
