"""Parity of the sm_103a extended B-splines (tw_extension_build,
tw_extension_matrix, tw_form_mass_extended, tw_l2_project_extended, through
the C-ABI) with the oracle's restatement of readings R15-R17.

Bar: the inner/outer split, the arrays and the patterns of E and E^T M E bit
for bit; E's coefficients within 1e-12 of the largest coefficient of their row
(the GPU solves the polynomial reproduction in another basis than the oracle:
evaluations of Marsden's psi_k instead of blossoms of monomials; in exact
arithmetic both give the same coefficients, in FP64 the two (p+1) x (p+1)
solves differ by about 1e-14 of the row at p = 5 and 1e-13 at p = 6, with
coefficients up to a few hundred); E^T M E within 1e-12 relative Frobenius
of the oracle's product of its own M; the extended projection
by its residual in the oracle's own extended system (<= 1e-11 of the
right-hand side) and within 10 cond x 1e-13 of the oracle's direct solve (CG
stops at a relative residual of 1e-13; the extension bounds cond independently
of where the trim cuts, but the bound grows steeply with p: 1e2 at p = 2,
4e6 at p = 4, 3e10 at p = 5 in these cases, because an inner function may own
only a corner element of its support, where it is O(t^p) small).  At the full 512 x 512 size
the oracle builds E and the product E^T M E is checked on sampled rows with
the GPU's own M (whose parity the formation tests pin).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth
from oracle.extension import Extension

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "config1": lambda: synth.config1(),
    "p3_graded": lambda: synth.with_knots(synth.make_spec(3, 18, synth.circle(0.5, 0.5, 0.3)),
                                          synth.graded_knots(3, 18, 1.12),
                                          synth.graded_knots(3, 18, 0.9)),
    "p4_sliver": lambda: synth.make_spec(4, 20, synth.circle(0.5, 0.5, 0.31)),
    "p2_dwq": lambda: synth.make_spec(2, 16, synth.circle(0.5, 0.5, 0.27), method="dwq"),
    "p3_spline_geom": lambda: synth.config2(p=3, nel=24),
    "p6_ellipse": lambda: synth.make_spec(6, 30, synth.ellipse(0.5, 0.5, 0.3, 0.2, 0.4)),
    "p5_bspline": lambda: synth.make_spec(5, (26, 22), synth.bspline_curve(
        np.random.default_rng(7), nc=8, radius=0.28, jitter=0.15, relative_jitter=True)),
    "p3_line": lambda: synth.line_trim_spec(3, nel=12),
    "p2_coarse": lambda: synth.make_spec(2, 5, synth.circle(0.5, 0.5, 0.42)),
}


def _csr_host(t):
    return [x.cpu().numpy() for x in t]


def _e_close(ev, E):
    """E's values within 1e-12 of each row's largest coefficient."""
    rp = E.indptr
    scale = np.maximum.reduceat(np.abs(E.data), rp[:-1]) if E.nnz else np.zeros(0)
    per = np.repeat(scale, np.diff(rp))
    return np.all(np.abs(ev - E.data) <= 1e-12 * per)


def _gpu(spec):
    from paper_2101_08053_gb300 import Patch
    P = Patch(spec)
    info = P.extension()
    return P, info


@pytest.mark.parametrize("case", sorted(CASES))
def test_extension_matrix_matches_oracle(case):
    spec = CASES[case]()
    P, (ni, no, nnz_e, nnz_x) = _gpu(spec)
    O = oracle.Patch(spec)
    X = Extension(O)
    assert (ni, no) == (X.n_inner, X.n_outer)
    assert nnz_e == X.E.nnz
    erp, ecol, ev = _csr_host(P.extension_matrix())
    torch.cuda.synchronize()
    assert np.array_equal(erp, X.E.indptr)
    assert np.array_equal(ecol, X.E.indices)
    assert _e_close(ev, X.E), np.max(np.abs(ev - X.E.data))


@pytest.mark.parametrize("case", sorted(CASES))
def test_extended_mass_matches_oracle(case):
    spec = CASES[case]()
    P, (ni, no, nnz_e, nnz_x) = _gpu(spec)
    csr = P.form_mass("fp64")
    xr, xc, xv = _csr_host(P.form_mass_extended(csr))
    O = oracle.Patch(spec)
    X = Extension(O)
    orp, ocol, oval = O.form()
    rr, rc, rv = X.mass(orp, ocol, oval)
    assert nnz_x == len(rc)
    assert np.array_equal(xr, rr) and np.array_equal(xc, rc)
    assert np.linalg.norm(xv - rv) <= 1e-12 * np.linalg.norm(rv)
    # deterministic: a second formation is bitwise equal
    xr2, xc2, xv2 = _csr_host(P.form_mass_extended(csr))
    assert np.array_equal(xv, xv2)


@pytest.mark.parametrize("case", ["config1", "p3_graded", "p4_sliver", "p3_spline_geom",
                                  "p5_bspline"])
def test_extended_projection_matches_oracle(case):
    spec = CASES[case]()
    f = synth.func_sincos(2.0, 3.0)
    P, info = _gpu(spec)
    csr = P.form_mass("fp64")
    xcsr = P.form_mass_extended(csr)
    u, it, rel = P.l2_project_extended(f, xcsr, tol=1e-13)
    O = oracle.Patch(spec)
    X = Extension(O)
    orp, ocol, oval = O.form()
    uo, _ = X.project(f, orp, ocol, oval)
    uh = u.cpu().numpy()
    assert rel <= 1e-13
    # x = u on the inner rows (E is the identity there): its residual in the
    # oracle's own extended system, and u against the oracle's direct solve
    # within cond x the CG tolerance
    n = O.n_rows
    M = sp.csr_matrix((oval, ocol, orp), shape=(n, n))
    A = (X.E.T @ (0.5 * (M + M.T)) @ X.E).toarray()
    bx = X.E.T @ O.rhs(f)
    x = uh[X.act[X.inner]]  # inner functions in ascending g = ascending row
    assert np.linalg.norm(A @ x - bx) <= 1e-11 * np.linalg.norm(bx)
    kappa = np.linalg.cond(A)
    assert np.max(np.abs(uh - uo)) <= 10 * kappa * 1e-13 * np.max(np.abs(uo)), kappa
    # the projection error of the extended space matches the oracle's measure
    e_gpu, fn = O.l2_error(uh, f)
    e_or, _ = O.l2_error(uo, f)
    assert abs(e_gpu - e_or) <= 1e-9 * fn


def test_extension_reproduces_polynomials_and_bounds_coefficients():
    """A polynomial is projected exactly (it lies in the extended space), and a
    smooth target gets coefficients of the size of the target at the same L2
    accuracy, where the plain projection's coefficients on functions with tiny
    visible supports grow past 1e3 (to ~1e11 in a direct solve, whose L2 error
    roundoff then spoils).  Jacobi-PCG's iteration count is about the same with
    and without the extension: the diagonal scaling already absorbs the tiny
    functions' scale."""
    p, nel = 3, 40
    spec = synth.make_spec(p, nel, synth.circle(0.5, 0.5, 0.3037))
    P, (ni, no, nnz_e, nnz_x) = _gpu(spec)
    csr = P.form_mass("fp64")
    xcsr = P.form_mass_extended(csr)
    U1, U2 = spec["knots"]
    from scipy.interpolate import make_interp_spline
    rng = np.random.default_rng(4)

    def coefs(U):
        x = synth.greville(np.asarray(U), p)
        return make_interp_spline(x, np.polynomial.polynomial.polyval(x, rng.standard_normal(p + 1)),
                                  k=p, t=np.asarray(U)).c

    c = np.outer(coefs(U2), coefs(U1))
    f = {"kind": "spline", "prm": [0.0] * 4, "p": p, "knots": [U1, U2], "coef": c}
    u, it_ext, rel = P.l2_project_extended(f, xcsr, tol=1e-13)
    es, fs, act = [t.cpu().numpy() for t in P.states()]
    cA = c.ravel()[act >= 0]
    # exact up to CG's stopping point: within 10 cond x 1e-13
    xr, xc, xv = _csr_host(xcsr)
    A = sp.csr_matrix((xv, xc, xr), shape=(ni, ni)).toarray()
    kappa = np.linalg.cond(0.5 * (A + A.T))
    err = np.max(np.abs(u.cpu().numpy() - cA))
    assert err <= 10 * kappa * 1e-13 * np.max(np.abs(cA)), (err, kappa)
    # a smooth target (|g| <= 1)
    g = synth.func_sincos(2.0, 3.0)
    ue, _, _ = P.l2_project_extended(g, xcsr, tol=1e-13)
    u0, _, _ = P.l2_project(g, csr, tol=1e-13)
    O = oracle.Patch(spec)
    ee, gn = O.l2_error(ue.cpu().numpy(), g)
    e0, _ = O.l2_error(u0.cpu().numpy(), g)
    assert torch.max(torch.abs(ue)).item() <= 1.5
    assert torch.max(torch.abs(u0)).item() >= 1e3
    assert ee <= 1e-6 * gn and ee <= 2.0 * e0


def test_untrimmed_patch_extension_is_the_identity():
    spec = synth.make_spec(3, (11, 9), {"kind": "none"})
    P, (ni, no, nnz_e, nnz_x) = _gpu(spec)
    assert no == 0 and ni == P.n_rows and nnz_e == ni and nnz_x == P.nnz
    csr = P.form_mass("fp64")
    xr, xc, xv = P.form_mass_extended(csr)
    assert torch.equal(xr, csr[0]) and torch.equal(xc, csr[1]) and torch.equal(xv, csr[2])
    erp, ecol, ev = _csr_host(P.extension_matrix())
    assert np.array_equal(ecol, np.arange(ni)) and np.all(ev == 1.0)


def test_patch_too_coarse_for_its_trim_is_rejected():
    from paper_2101_08053_gb300 import Patch, TWError
    spec = synth.make_spec(3, 4, synth.circle(0.5, 0.5, 0.45))
    with pytest.raises(ValueError):
        Extension(oracle.Patch(spec))
    P = Patch(spec)
    with pytest.raises(TWError):
        P.extension()
    # the patch stays usable
    rp, col, val = P.form_mass("fp64")
    torch.cuda.synchronize()
    assert int(rp[-1]) == P.nnz


def test_extension_requires_build_first():
    from paper_2101_08053_gb300 import Patch, TWError, api
    import ctypes as C
    P = Patch(synth.config1())
    rp = torch.empty(P.n_rows + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(8, dtype=torch.int32, device="cuda")
    val = torch.empty(8, dtype=torch.float64, device="cuda")
    rc = api.load().tw_extension_matrix(P._h, C.c_void_p(rp.data_ptr()),
                                        C.c_void_p(col.data_ptr()), C.c_void_p(val.data_ptr()),
                                        None)
    assert rc == -1


def test_full_size_512_extension_against_oracle_e():
    spec = synth.config2(p=4, nel=512)
    P, (ni, no, nnz_e, nnz_x) = _gpu(spec)
    O = oracle.Patch(spec)
    X = Extension(O)
    assert (ni, no) == (X.n_inner, X.n_outer)
    erp, ecol, ev = _csr_host(P.extension_matrix())
    assert np.array_equal(erp, X.E.indptr) and np.array_equal(ecol, X.E.indices)
    assert _e_close(ev, X.E)
    csr = P.form_mass("fp64")
    xr, xc, xv = _csr_host(P.form_mass_extended(csr))
    rp, col, val = _csr_host(csr)
    n = P.n_rows
    M = sp.csr_matrix((val, col, rp), shape=(n, n))
    # rows next to the trim (where E differs from the identity) and a random sample
    near = np.unique(X.E.indices[np.repeat(np.diff(X.E.indptr) > 1, np.diff(X.E.indptr))])
    rng = np.random.default_rng(8)
    rows = np.unique(np.concatenate([rng.choice(near, min(300, len(near)), replace=False),
                                     rng.choice(ni, 300, replace=False)]))
    ET = X.E.T.tocsr()
    ref = (ET[rows] @ M @ X.E).tocsr()
    for k, a in enumerate(rows):
        cols = xc[xr[a]:xr[a + 1]]
        vals = xv[xr[a]:xr[a + 1]]
        r = ref.getrow(k)
        dense = np.zeros(ni)
        dense[r.indices] = r.data
        assert np.all(np.diff(cols) > 0)
        assert np.count_nonzero(dense) == np.count_nonzero(dense[cols])
        err = np.max(np.abs(vals - dense[cols]))
        assert err <= 1e-13 * np.max(np.abs(dense)), (a, err)
    f = synth.func_sincos(2.0, 3.0)
    u, it, rel = P.l2_project_extended(f, P.form_mass_extended(csr), tol=1e-12)
    u2, it2, rel2 = P.l2_project_extended(f, P.form_mass_extended(csr), tol=1e-12)
    assert torch.equal(u, u2) and it == it2


# ---------------------------------------------------------------------------
# differentiation of the extended projection (reading R12 with u = E x)

G_FN = synth.func_gauss(8.0, 0.3, 0.7)


def _density_case(seed=11, nel=(9, 8), m=6, p=3, r=0.29):
    dens = synth.density(np.random.default_rng(seed), q=2, m=m)
    return synth.make_spec(p, nel, synth.circle(0.5, 0.5, r), coef=dens)


def _with_coef(spec, coef):
    s = dict(spec)
    c = dict(spec["coef"])
    c["coef"] = np.asarray(coef, dtype=np.float64).reshape(c["coef"].shape)
    s["coef"] = c
    return s


def test_extended_adjoint_lambda_against_oracle_system():
    spec = _density_case(nel=(14, 13), m=8)
    P, (ni, no, nnz_e, nnz_x) = _gpu(spec)
    assert no > 0
    csr = P.form_mass("fp64")
    xcsr = P.form_mass_extended(csr)
    u, _, _ = P.l2_project_extended(G_FN, xcsr, tol=1e-13)
    L, dl = P.loss(u, G_FN)
    grad, lam, it, rel = P.l2_project_adjoint_extended(G_FN, xcsr, dl, u, tol=1e-13)
    O = oracle.Patch(spec)
    X = Extension(O)
    lamh = lam.cpu().numpy()
    mu = lamh[X.act[X.inner]]
    # lam = E mu on every row, and mu solves the oracle's extended adjoint system
    assert np.max(np.abs(X.E @ mu - lamh)) <= 1e-14 * np.max(np.abs(lamh))
    orp, ocol, oval = O.form()
    n = O.n_rows
    M = sp.csr_matrix((oval, ocol, orp), shape=(n, n))
    A = X.E.T @ (0.5 * (M + M.T)) @ X.E
    r = X.E.T @ dl.cpu().numpy()
    assert np.linalg.norm(A @ mu - r) <= 1e-11 * np.linalg.norm(r)
    # the gradient stage with this lam and u equals the oracle's
    Ograd = O.density_grad(u.cpu().numpy(), lamh, G_FN)
    ref = np.max(np.abs(Ograd))
    assert np.max(np.abs(grad.cpu().numpy() - Ograd)) <= 1e-12 * ref


def _dense_extended_loss(spec):
    """L(d) with the GPU's own M(d), b(d), E and tw_loss; u = E x by a dense
    solve of the extended system."""
    from paper_2101_08053_gb300 import Patch
    P = Patch(spec)
    ni = P.extension()[0]
    csr = P.form_mass("fp64")
    rp, col, val = _csr_host(csr)
    n = P.n_rows
    M = sp.csr_matrix((val, col, rp), shape=(n, n))
    erp, ecol, ev = _csr_host(P.extension_matrix())
    E = sp.csr_matrix((ev, ecol, erp), shape=(n, ni))
    A = (E.T @ (0.5 * (M + M.T)) @ E).toarray()
    b = P.rhs(G_FN).cpu().numpy()
    u = E @ np.linalg.solve(A, E.T @ b)
    L, dl = P.loss(torch.from_numpy(u).cuda(), G_FN)
    return L.item(), u, dl, P, csr


def test_extended_gradient_against_finite_differences():
    spec = _density_case(nel=(11, 10), r=0.33)  # 14 outer functions
    d0 = spec["coef"]["coef"].ravel().copy()
    L, u, dl, P, csr = _dense_extended_loss(spec)
    xcsr = P.form_mass_extended(csr)
    grad, lam, it, rel = P.l2_project_adjoint_extended(G_FN, xcsr, dl, torch.from_numpy(u).cuda(),
                                                       tol=1e-14)
    grad = grad.cpu().numpy().ravel()
    scale = np.max(np.abs(grad))
    h = 1e-4
    rng = np.random.default_rng(9)
    for k in list(rng.choice(d0.size, 4, replace=False)):
        dp, dm = d0.copy(), d0.copy()
        dp[k] += h
        dm[k] -= h
        fd = (_dense_extended_loss(_with_coef(spec, dp))[0] -
              _dense_extended_loss(_with_coef(spec, dm))[0]) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * scale, (k, fd, grad[k])


def test_extended_autograd_matches_adjoint():
    from paper_2101_08053_gb300 import Patch, projection_loss
    spec = _density_case(nel=(10, 10))
    d = torch.tensor(spec["coef"]["coef"], dtype=torch.float64, requires_grad=True)
    L = projection_loss(d, spec, G_FN, G_FN, extended=True)
    L.backward()
    P = Patch(spec)
    P.extension()
    xcsr = P.form_mass_extended(P.form_mass("fp64"))
    u, _, _ = P.l2_project_extended(G_FN, xcsr, tol=1e-13)
    L2, dl = P.loss(u, G_FN)
    grad, _, _, _ = P.l2_project_adjoint_extended(G_FN, xcsr, dl, u, tol=1e-13)
    assert L.item() == L2.item()
    assert torch.equal(d.grad, grad.cpu())
