"""Pins of the oracle's differentiation of the L2 projection with respect to
the density coefficients (no GPU).

Anchors, none of them the oracle's own gradient code:
  * the loss is quadratic in u: central differences of or_loss along random
    directions equal dL/du . v up to rounding;
  * a spline target of the patch's own space projected with u = its
    coefficients has loss 0; with u = 0 and g = 1 the loss is the visible
    area 1 - pi r^2 and sum_j dL/du_j = -2 |Omega^v| (partition of unity);
  * every row rule is linear in c (Eqs. 4, 5, 7): with u = 0 the gradient is
    lambda^T b(e_k), with f = 0 it is -(lambda^T M(e_k) u + u^T M(e_k) lambda)/2,
    where b(e_k), M(e_k) are formed with the k-th density coefficient alone;
  * the whole chain d -> M(d), b(d) -> u -> L(u) against central finite
    differences (h = 1e-4) with a dense solve of M_s = (M + M^T)/2, for every
    method (hybrid Gauss, DWQ, naive WQ, Gauss) and with a spline geometry.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth


def _density(m, seed):
    return synth.density(np.random.default_rng(seed), q=2, m=m)


def _spec(method="hybrid", nel=10, m=6, seed=11, geom=False, p=3, cut_order=0):
    dens = _density(m, seed)
    g = None
    if geom:
        rng = np.random.default_rng(seed + 1)
        g = {"kind": "spline", "ctrl": synth.perturbed_bilinear_net(rng, p, nel)}
    return synth.make_spec(p, nel, synth.circle(0.5, 0.5, 0.27), geom=g, coef=dens, method=method,
                           cut_order=cut_order)


def _with_coef(spec, coef):
    s = dict(spec)
    c = dict(spec["coef"])
    c["coef"] = np.asarray(coef, dtype=np.float64).reshape(c["coef"].shape)
    s["coef"] = c
    return s


def _msym(P):
    rp, col, val = P.form()
    M = sp.csr_matrix((val, col, rp), shape=(P.n_rows, P.n_rows)).toarray()
    return M, 0.5 * (M + M.T)


def _chain(spec, f, g):
    """L(d) through a dense solve; returns (L, u, lambda, P)."""
    P = oracle.Patch(spec)
    _, Ms = _msym(P)
    u = np.linalg.solve(Ms, P.rhs(f))
    L, dl = P.loss(u, g)
    lam = np.linalg.solve(Ms, dl)
    return L, u, lam, P


F = synth.func_sincos(2.0, 3.0)
G = synth.func_gauss(8.0, 0.3, 0.7)


def test_loss_is_quadratic_in_u():
    P = oracle.Patch(_spec())
    rng = np.random.default_rng(3)
    u = rng.standard_normal(P.n_rows)
    L, dl = P.loss(u, G)
    for _ in range(3):
        v = rng.standard_normal(P.n_rows)
        h = 0.5
        fd = (P.loss(u + h * v, G)[0] - P.loss(u - h * v, G)[0]) / (2 * h)
        assert abs(fd - dl @ v) <= 1e-12 * max(1.0, abs(fd))


def test_loss_zero_for_own_space_target():
    spec = _spec()
    P = oracle.Patch(spec)
    g = synth.func_spline(spec, np.random.default_rng(4))
    es, fs, act = P.states()
    a = g["coef"].ravel()[act >= 0]
    L, dl = P.loss(a, g)
    assert L < 1e-28
    assert np.max(np.abs(dl)) < 1e-14


def test_loss_of_zero_is_visible_area():
    """High-order cut rule (12 points) so that its own error is below 1e-13."""
    P = oracle.Patch(_spec(cut_order=12))
    one = {"kind": "spline", "p": 0, "knots": [np.array([0.0, 1.0]), np.array([0.0, 1.0])],
           "coef": np.ones((1, 1))}
    L, dl = P.loss(np.zeros(P.n_rows), one)
    area = 1.0 - math.pi * 0.27 ** 2
    assert abs(L - area) < 1e-12
    assert abs(dl.sum() + 2.0 * area) < 1e-12


@pytest.mark.parametrize("method", ["hybrid", "dwq", "naive", "gauss"])
def test_gradient_is_linear_in_the_density(method):
    """Every row rule is linear in c, so dL/dd_k splits into lambda^T b(e_k)
    and -(lambda^T M(e_k) u + u^T M(e_k) lambda)/2 exactly."""
    spec = _spec(method=method, m=5)
    P = oracle.Patch(spec)
    rng = np.random.default_rng(6)
    u = rng.standard_normal(P.n_rows)
    lam = rng.standard_normal(P.n_rows)
    zero_f = synth.func_spline(spec, rng)
    zero_f["coef"][:] = 0.0
    gb = P.density_grad(np.zeros(P.n_rows), lam, F).ravel()
    gm = P.density_grad(u, lam, zero_f).ravel()
    m = spec["coef"]["coef"].size
    for k in range(m):
        ek = np.zeros(m)
        ek[k] = 1.0
        Pk = oracle.Patch(_with_coef(spec, ek))
        Mk, _ = _msym(Pk)
        bk = Pk.rhs(F)
        ref_b = lam @ bk
        ref_m = -0.5 * (lam @ Mk @ u + u @ Mk @ lam)
        assert abs(gb[k] - ref_b) <= 1e-13 * (1 + abs(ref_b))
        assert abs(gm[k] - ref_m) <= 1e-12 * (1 + abs(ref_m))


@pytest.mark.parametrize("method,geom", [("hybrid", False), ("dwq", False), ("naive", False),
                                         ("gauss", False), ("hybrid", True)])
def test_gradient_against_finite_differences(method, geom):
    """Reading R12's loss: the projection of g itself, so L is the squared
    projection error and depends on the density at first order."""
    spec = _spec(method=method, geom=geom, nel=6)
    d0 = spec["coef"]["coef"].ravel().copy()
    L, u, lam, P = _chain(spec, G, G)
    grad = P.density_grad(u, lam, G).ravel()
    h = 1e-4  # central differences: O(h^2) error ~1e-9 relative; at h = 1e-6
    # the solve's rounding noise (~1e-14 absolute) reaches 1e-5 of the
    # smallest (Gauss method) gradient
    rng = np.random.default_rng(7)
    ks = list(rng.choice(d0.size, 4, replace=False))
    scale = np.max(np.abs(grad))
    for k in ks:
        dp, dm = d0.copy(), d0.copy()
        dp[k] += h
        dm[k] -= h
        fd = (_chain(_with_coef(spec, dp), G, G)[0] - _chain(_with_coef(spec, dm), G, G)[0]) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * scale, (k, fd, grad[k])
    v = rng.standard_normal(d0.size)
    fd = (_chain(_with_coef(spec, d0 + h * v), G, G)[0] -
          _chain(_with_coef(spec, d0 - h * v), G, G)[0]) / (2 * h)
    assert abs(fd - grad @ v) <= 1e-6 * scale * np.linalg.norm(v, 1) / math.sqrt(d0.size)


def test_targets_against_closed_forms_and_quadrature():
    """The targets f, g the projection and the loss use: at u = 0 the loss is
    the integral of g^2 over the visible domain (identity geometry), against
    closed forms on the untrimmed square (sin.cos, sin.sin) and against
    scipy's adaptive quadrature on the line-trimmed square for the Gaussian
    bump (the trim makes the domain asymmetric, so a swapped centre shows)."""
    import math
    from scipy.integrate import dblquad

    def s2(a):  # integral of sin^2(a x) over [0, 1]
        return 0.5 - math.sin(2 * a) / (4 * a)

    def c2(a):  # integral of cos^2(a x) over [0, 1]
        return 0.5 + math.sin(2 * a) / (4 * a)

    P = oracle.Patch(synth.make_spec(3, 16, {"kind": "none"}))
    u = np.zeros(P.n_rows)
    L, _ = P.loss(u, synth.func_sincos(2.0, 3.0))
    assert abs(L - s2(2.0) * c2(3.0)) <= 1e-12
    L, _ = P.loss(u, synth.func_sinsin(2.5, 1.5))
    assert abs(L - s2(2.5) * s2(1.5)) <= 1e-12
    P = oracle.Patch(synth.line_trim_spec(3, nel=16))
    u = np.zeros(P.n_rows)
    L, _ = P.loss(u, synth.func_gauss(8.0, 0.3, 0.7))
    x0, y0, x1, y1 = synth.LINE_TRIM
    ref = dblquad(lambda y, x: math.exp(-16.0 * ((x - 0.3) ** 2 + (y - 0.7) ** 2)), 0.0, 1.0,
                  lambda x: 0.0, lambda x: y0 + (y1 - y0) * x, epsabs=1e-14, epsrel=1e-13)[0]
    assert abs(L - ref) <= 1e-10 * ref
    # sin(2x) cos(3y) on the same asymmetric domain (on the square a swap of
    # x and y would integrate to the same value)
    L, _ = P.loss(u, synth.func_sincos(2.0, 3.0))
    ref = dblquad(lambda y, x: (math.sin(2.0 * x) * math.cos(3.0 * y)) ** 2, 0.0, 1.0,
                  lambda x: 0.0, lambda x: y0 + (y1 - y0) * x, epsabs=1e-14, epsrel=1e-13)[0]
    assert abs(L - ref) <= 1e-10 * ref


def test_physical_points_on_an_exact_bilinear_geometry():
    """The target is evaluated at x(xi): with an unperturbed bilinear control
    net the patch is exactly the quadrilateral (0,0), (1,0), (1.15,1.1),
    (0.05,0.95), and the loss at u = 0 (sum of w det J g(x(xi))^2) equals the
    integral of g^2 over that quadrilateral (two triangles, scipy)."""
    import math
    from scipy.integrate import dblquad

    p, nel = 3, 12
    net = synth.perturbed_bilinear_net(np.random.default_rng(0), p, nel, amplitude_h=0.0)
    spec = synth.make_spec(p, nel, {"kind": "none"}, geom={"kind": "spline", "ctrl": net},
                           coef={"kind": "detj"})
    P = oracle.Patch(spec)
    L, _ = P.loss(np.zeros(P.n_rows), synth.func_gauss(4.0, 0.6, 0.4))

    def tri(a, b, c):
        (ax, ay), (bx, by), (cx, cy) = a, b, c
        jac = abs((bx - ax) * (cy - ay) - (cx - ax) * (by - ay))

        def f(t, s):
            x = ax + s * (bx - ax) + t * (cx - ax)
            y = ay + s * (by - ay) + t * (cy - ay)
            return math.exp(-8.0 * ((x - 0.6) ** 2 + (y - 0.4) ** 2))

        return jac * dblquad(f, 0.0, 1.0, lambda s: 0.0, lambda s: 1.0 - s, epsabs=1e-14,
                             epsrel=1e-13)[0]

    corners = [(0.0, 0.0), (1.0, 0.0), (1.15, 1.1), (0.05, 0.95)]
    ref = tri(corners[0], corners[1], corners[2]) + tri(corners[0], corners[2], corners[3])
    assert abs(L - ref) <= 1e-10 * ref
