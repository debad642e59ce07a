"""Parity of the sm_103a differentiation of the L2 projection (tw_loss,
tw_l2_project_adjoint and the autograd wrapper, through the C-ABI) with the
oracle's loss and density gradient.

Bar (FP64): the loss and dL/du for the same u, and the gradient for the same
seeded u and the adjoint lambda the GPU returns, within 1e-12 of the oracle's
(relative, max-norm over the vector); the adjoint lambda by its residual against the oracle's own matrix,
||M_s lambda - dL/du|| <= 1e-11 ||dL/du|| (CG solutions of different rounding
agree only to cond x tol); the whole chain against central differences with u
from a dense solve of the GPU's M_s and b; at the full 256 x 256 size, where
the oracle's gradient takes minutes, the linearity of every row rule in c
(gradient = lambda^T b(e_k) - (lambda^T M(e_k) u + u^T M(e_k) lambda) / 2 with
b(e_k), M(e_k) formed on the GPU for single density coefficients) on sampled
coefficients, and bitwise reproducibility.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
G_FN = synth.func_gauss(8.0, 0.3, 0.7)
F_FN = synth.func_sincos(2.0, 3.0)


def _spec(method="hybrid", nel=(13, 11), m=6, seed=11, geom=False, p=3, trim=None):
    dens = synth.density(np.random.default_rng(seed), q=2, m=m)
    g = None
    if geom:
        rng = np.random.default_rng(seed + 1)
        assert nel[0] == nel[1], "the perturbed bilinear net is square"
        g = {"kind": "spline", "ctrl": synth.perturbed_bilinear_net(rng, p, nel[0])}
    trim = trim if trim is not None else synth.circle(0.5, 0.5, 0.27)
    return synth.make_spec(p, nel, trim, geom=g, coef=dens, method=method)


def _with_coef(spec, coef):
    s = dict(spec)
    c = dict(spec["coef"])
    c["coef"] = np.asarray(coef, dtype=np.float64).reshape(c["coef"].shape)
    s["coef"] = c
    return s


def _gpu_chain(spec, f, g, tol=1e-13):
    from paper_2101_08053_gb300 import Patch
    P = Patch(spec)
    csr = P.form_mass("fp64")
    u, _, _ = P.l2_project(f, csr, tol=tol)
    L, dl = P.loss(u, g)
    grad, lam, it, rel = P.l2_project_adjoint(f, csr, dl, u, tol=tol)
    torch.cuda.synchronize()
    return P, csr, u, L, dl, grad, lam


def _rel_max(a, b):
    s = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / (s if s > 0 else 1.0)


def _msym_host(csr, n):
    rp, col, val = [t.cpu().numpy() for t in csr]
    M = sp.csr_matrix((val, col, rp), shape=(n, n))
    return 0.5 * (M + M.T)


@pytest.mark.parametrize("method,geom,nel,m", [
    ("hybrid", False, (13, 11), 6),
    ("dwq", False, (13, 11), 6),
    ("naive", False, (12, 12), 5),
    ("gauss", False, (9, 14), 6),
    ("hybrid", True, (15, 15), 8),
    ("dwq", True, (16, 16), 8),
    ("hybrid", False, (40, 33), 32),
])
def test_loss_and_gradient_against_oracle(method, geom, nel, m):
    """Loss and dL/du at the projection u; the gradient stage for a seeded
    random u (at the projection the gradient is a small difference of large
    terms -- Gauss rows give a symmetric M, whose first-order terms nearly
    cancel -- so there it is checked by finite differences instead)."""
    spec = _spec(method, nel, m, geom=geom)
    P, csr, u, L, dl, grad, lam = _gpu_chain(spec, F_FN, G_FN)
    O = oracle.Patch(spec)
    uh = u.cpu().numpy()
    OL, Odl = O.loss(uh, G_FN)
    assert abs(L.item() - OL) <= TOL * abs(OL)
    assert _rel_max(dl.cpu().numpy(), Odl) <= TOL
    rng = np.random.default_rng(21)
    ur = rng.standard_normal(P.n_rows)
    dr = Odl  # a smooth right-hand side: random ones excite the cut rows'
    # near-null directions and lambda's residual then only meets cond x tol
    grad, lam, _, _ = P.l2_project_adjoint(F_FN, csr, torch.from_numpy(dr).cuda(),
                                           torch.from_numpy(ur).cuda(), tol=1e-13)
    lamh = lam.cpu().numpy()
    Ograd = O.density_grad(ur, lamh, F_FN)
    assert grad.shape == Ograd.shape
    assert _rel_max(grad.cpu().numpy(), Ograd) <= TOL
    orp, ocol, oval = O.form()
    M = sp.csr_matrix((oval, ocol, orp), shape=(O.n_rows, O.n_rows))
    Ms = 0.5 * (M + M.T)
    r = Ms @ lamh - dr
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(dr)


def test_untrimmed_patch_has_no_cut_rows():
    spec = _spec("hybrid", (10, 12), 6, trim={"kind": "none"})
    P, csr, u, L, dl, grad, lam = _gpu_chain(spec, F_FN, G_FN)
    O = oracle.Patch(spec)
    rng = np.random.default_rng(22)
    ur = rng.standard_normal(P.n_rows)
    dr = torch.from_numpy(rng.standard_normal(P.n_rows)).cuda()
    grad, lam, _, _ = P.l2_project_adjoint(F_FN, csr, dr, torch.from_numpy(ur).cuda(), tol=1e-13)
    Ograd = O.density_grad(ur, lam.cpu().numpy(), F_FN)
    assert _rel_max(grad.cpu().numpy(), Ograd) <= TOL


def _dense_loss(spec, f, g):
    """L(d) with the GPU's own M(d), b(d) and tw_loss, u by a dense solve."""
    from paper_2101_08053_gb300 import Patch
    P = Patch(spec)
    csr = P.form_mass("fp64")
    b = P.rhs(f).cpu().numpy()
    Ms = _msym_host(csr, P.n_rows).toarray()
    u = np.linalg.solve(Ms, b)
    L, dl = P.loss(torch.from_numpy(u).cuda(), g)
    return L.item(), u, dl, P, csr


@pytest.mark.parametrize("method", ["hybrid", "dwq", "gauss"])
def test_gradient_against_finite_differences(method):
    spec = _spec(method, (7, 6), 6)
    d0 = spec["coef"]["coef"].ravel().copy()
    L, u, dl, P, csr = _dense_loss(spec, G_FN, G_FN)
    grad, lam, it, rel = P.l2_project_adjoint(G_FN, csr, dl, torch.from_numpy(u).cuda(), tol=1e-14)
    grad = grad.cpu().numpy().ravel()
    scale = np.max(np.abs(grad))
    h = 1e-4
    rng = np.random.default_rng(9)
    for k in list(rng.choice(d0.size, 3, replace=False)):
        dp, dm = d0.copy(), d0.copy()
        dp[k] += h
        dm[k] -= h
        fd = (_dense_loss(_with_coef(spec, dp), G_FN, G_FN)[0] -
              _dense_loss(_with_coef(spec, dm), G_FN, G_FN)[0]) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * scale, (k, fd, grad[k])


def test_autograd_matches_adjoint_and_oracle_chain():
    from paper_2101_08053_gb300 import projection_loss
    spec = _spec("hybrid", (8, 7), 6)
    d = torch.tensor(spec["coef"]["coef"], dtype=torch.float64, requires_grad=True)
    L = projection_loss(d, spec, G_FN, G_FN)
    L.backward()
    P, csr, u, L2, dl, grad, lam = _gpu_chain(spec, G_FN, G_FN)
    assert L.item() == L2.item()
    assert torch.equal(d.grad, grad.cpu())
    O = oracle.Patch(spec)
    orp, ocol, oval = O.form()
    M = sp.csr_matrix((oval, ocol, orp), shape=(O.n_rows, O.n_rows)).toarray()
    Ms = 0.5 * (M + M.T)
    uo = np.linalg.solve(Ms, O.rhs(G_FN))
    Lo, dlo = O.loss(uo, G_FN)
    lo = np.linalg.solve(Ms, dlo)
    go = O.density_grad(uo, lo, G_FN)
    assert abs(L.item() - Lo) <= 1e-9 * Lo
    assert _rel_max(d.grad.numpy(), go) <= 1e-8


def test_full_size_config5_linearity_and_determinism():
    from paper_2101_08053_gb300 import Patch
    spec = synth.config5()
    P, csr, u, L, dl, grad, lam = _gpu_chain(spec, G_FN, G_FN)
    O = oracle.Patch(spec)
    uh = u.cpu().numpy()
    OL, Odl = O.loss(uh, G_FN)
    assert abs(L.item() - OL) <= TOL * abs(OL)
    assert _rel_max(dl.cpu().numpy(), Odl) <= TOL
    g2, lam2, _, _ = P.l2_project_adjoint(G_FN, csr, dl, u, tol=1e-13)
    assert torch.equal(g2, grad) and torch.equal(lam2, lam)
    gh = grad.cpu().numpy().ravel()
    m = spec["coef"]["coef"].size
    lamh = lam.cpu().numpy()
    rng = np.random.default_rng(12)
    for k in list(rng.choice(m, 4, replace=False)):
        ek = np.zeros(m)
        ek[k] = 1.0
        Pk = Patch(_with_coef(spec, ek))
        rp, col, val = Pk.form_mass("fp64")
        bk = Pk.rhs(G_FN).cpu().numpy()
        Mk = sp.csr_matrix((val.cpu().numpy(), col.cpu().numpy(), rp.cpu().numpy()),
                           shape=(Pk.n_rows, Pk.n_rows))
        ref = lamh @ bk - 0.5 * (lamh @ (Mk @ uh) + uh @ (Mk @ lamh))
        terms = abs(lamh) @ abs(bk) + abs(lamh) @ (abs(Mk) @ abs(uh))
        assert abs(gh[k] - ref) <= 1e-13 * terms, (k, gh[k], ref)


def test_adjoint_rejects_patch_without_density():
    from paper_2101_08053_gb300 import Patch, TWError
    spec = synth.config1()
    P = Patch(spec)
    csr = P.form_mass("fp64")
    u, _, _ = P.l2_project(G_FN, csr)
    L, dl = P.loss(u, G_FN)
    assert math.isfinite(L.item())
    with pytest.raises(TWError):
        P.l2_project_adjoint(G_FN, csr, dl, u)
