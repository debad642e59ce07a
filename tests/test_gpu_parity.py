"""Parity of the sm_103a path (through the C-ABI) with the FP64 CPU oracle.

Bar (FP64): CSR pattern, classification, active numbering and DWQ region
choices bit-exact; WQ points/weights, cut-rule points, rhs and matrix values
within 1e-12 relative Frobenius (the tolerance the method's FP64 form is held
to); single entries within 1e-12 of the matrix's max entry.  Sizes span several
tiles and ragged tails (nel1 != nel2, odd sizes); full-size patches compare
seeded sampled rows against rows the oracle forms one by one.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def gpu_patch(spec):
    from paper_2101_08053_gb300 import Patch
    return Patch(spec)


def rel_fro(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def compare_full(spec, tol=TOL):
    G = gpu_patch(spec)
    O = oracle.Patch(spec)
    assert (G.n1, G.n2, G.nq1, G.nq2, G.n_rows, G.nnz) == (O.n1, O.n2, O.nq1, O.nq2, O.n_rows, O.nnz)
    es, fs, act = G.states()
    oes, ofs, oact = O.states()
    assert np.array_equal(es.cpu().numpy(), oes)
    assert np.array_equal(fs.cpu().numpy(), ofs)
    assert np.array_equal(act.cpu().numpy(), oact)
    rp, col, val = G.form_mass("fp64")
    torch.cuda.synchronize()
    orp, ocol, oval = O.form()
    assert np.array_equal(rp.cpu().numpy(), orp)
    assert np.array_equal(col.cpu().numpy(), ocol)
    v = val.cpu().numpy()
    assert np.all(np.isfinite(v))
    r = rel_fro(v, oval)
    assert r <= tol, r
    if oval.size:
        assert np.max(np.abs(v - oval)) <= tol * np.max(np.abs(oval))
    return G, O, (rp, col, val), (orp, ocol, oval)


@pytest.mark.parametrize("method", ["gauss", "hybrid", "dwq", "naive"])
def test_config1_all_methods(method):
    compare_full(synth.config1(method))


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("method", ["hybrid", "dwq"])
def test_degrees_circle(p, method):
    compare_full(synth.make_spec(p, (11, 14), synth.circle(0.47, 0.53, 0.3), method=method))


@pytest.mark.parametrize("p", [3, 4, 5])
@pytest.mark.parametrize("method", ["hybrid", "dwq"])
def test_spline_geometry_spline_hole(p, method):
    """Config-2 shape at 24 x 24 elements: perturbed bilinear geometry (c = det J)
    and a seeded 12-point cubic B-spline hole."""
    compare_full(synth.config2(p=p, nel=24, method=method, seed=1000 + p))


@pytest.mark.parametrize("keep_inside", [False, True])
def test_ellipse(keep_inside):
    t = synth.ellipse(0.5, 0.5, 0.33, 0.17, 0.7, keep_inside=keep_inside)
    compare_full(synth.make_spec(4, (19, 13), t, method="dwq"))


def test_density_coefficient():
    spec = synth.config5(nel=20)
    G = gpu_patch(spec)
    C = G.table(4).cpu().numpy().reshape(G.nq2, G.nq1)
    assert rel_fro(C, oracle.Patch(spec).cgrid()) < 1e-14
    compare_full(spec)


def test_untrimmed_and_high_cut_order():
    compare_full(synth.make_spec(5, 9, {"kind": "none", "params": [], "ctrl": None}))
    compare_full(synth.make_spec(3, 13, synth.circle(0.5, 0.5, 0.3), cut_order=9, method="dwq"))


DEGENERATE = {
    # a hole inside one element (the element holds the whole curve)
    "hole_in_one_element": synth.circle(0.51, 0.52, 0.003),
    # everything trimmed away: no active function, empty matrix
    "all_invisible": synth.circle(0.5, 0.5, 2.0),
    # keep the inside of a small circle: a few active functions, all cut
    "keep_inside_small": dict(synth.circle(0.5, 0.5, 0.05), keep_inside=True),
    # a circle crossing the patch boundary
    "crossing_boundary": synth.circle(0.0, 0.5, 0.3),
}


@pytest.mark.parametrize("case", sorted(DEGENERATE))
@pytest.mark.parametrize("method", ["hybrid", "dwq"])
def test_degenerate_trims(case, method):
    spec = synth.make_spec(2, (12, 11), DEGENERATE[case], method=method)
    G, O, (rp, col, val), _ = compare_full(spec)
    f = synth.func_sinsin()
    b = G.rhs(f).cpu().numpy()
    ob = O.rhs(f)
    assert b.shape == ob.shape
    if ob.size:
        assert rel_fro(b, ob) <= TOL
    u, it, rel = G.l2_project(f, (rp, col, val), check=False)
    assert u.shape[0] == G.n_rows
    if case == "all_invisible":
        assert G.n_rows == 0 and G.nnz == 0 and it == 0


@pytest.mark.parametrize("method", ["gauss", "hybrid", "dwq", "naive"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_line_trim_table1_sizes(p, method):
    """The paper's mass-matrix example: a straight-line trim on 10 x 10 elements."""
    compare_full(synth.line_trim_spec(p, 10, method))


def test_line_trim_table1_on_the_gpu():
    """Table 1 on the GPU path: hybrid Gauss and DWQ equal element Gauss to
    roundoff, naive WQ does not (p >= 2)."""
    for p in (1, 2, 3, 4, 5, 6):
        mats = {}
        for m in ("gauss", "hybrid", "dwq", "naive"):
            G = gpu_patch(synth.line_trim_spec(p, 10, m))
            mats[m] = G.form_mass("fp64")[2].cpu().numpy()
        ref = np.linalg.norm(mats["gauss"])
        assert np.linalg.norm(mats["hybrid"] - mats["gauss"]) / ref < 1e-14
        assert np.linalg.norm(mats["dwq"] - mats["gauss"]) / ref < 1e-14
        if p >= 2:
            assert np.linalg.norm(mats["naive"] - mats["gauss"]) / ref > 1e-6


def test_line_trim_ragged_and_steep():
    """A steep line (more crossings of horizontal knot lines) on a ragged
    patch, and the kept side flipped."""
    steep = synth.line(0.2, 0.0, 0.65, 1.0, keep_inside=True)
    compare_full(synth.make_spec(3, (13, 9), steep, method="hybrid"))
    compare_full(synth.make_spec(4, (11, 14), synth.line(0.0, 0.62, 1.0, 0.21), method="dwq"))


def test_config4_shaped_patches():
    rng = np.random.default_rng(synth.BASE_SEED + 4)
    for _ in range(3):
        spec = synth.config4_patch(rng)
        spec = synth.make_spec(spec["p"], (min(spec["nel"][0], 40), min(spec["nel"][1], 40)),
                               spec["trim"], method="hybrid")
        compare_full(spec)


def test_tables_against_oracle():
    spec = synth.config2(p=4, nel=20, method="dwq", seed=7)
    G = gpu_patch(spec)
    O = oracle.Patch(spec)
    for d in (0, 1):
        x = G.table(d).cpu().numpy()
        assert np.allclose(x, O.wq_grid(d), rtol=0, atol=1e-15)
    C = G.table(4).cpu().numpy().reshape(G.nq2, G.nq1)
    assert rel_fro(C, O.cgrid()) < 1e-14
    gx, _ = oracle.gauss_legendre(5)
    assert np.allclose(G.table(9).cpu().numpy(), gx, atol=1e-15)
    # cut-element rules as point sets
    off = G.table(6).cpu().numpy()
    cl = G.table(7).cpu().numpy()
    pts = G.table(5).cpu().numpy().reshape(-1, 3)
    assert len(cl) == G.n_cut_elems
    for ci, e in enumerate(cl):
        mine = pts[off[ci]:off[ci + 1]]
        ref = O.cut_rule(int(e % G.nel1), int(e // G.nel1))
        assert mine.shape == ref.shape
        a = mine[np.lexsort((mine[:, 1], mine[:, 0]))]
        b = ref[np.lexsort((ref[:, 1], ref[:, 0]))]
        assert np.allclose(a, b, rtol=0, atol=1e-14)
    # DWQ region choices
    ch = G.table(8).cpu().numpy().reshape(-1, 4)
    es, fs, act = O.states()
    for g in np.where(fs == 2)[0]:
        assert tuple(ch[g]) == O.dwq_choice(int(g % G.n1), int(g // G.n1))


def test_determinism_bitwise():
    spec = synth.config2(p=4, nel=48, method="dwq", seed=3)
    G = gpu_patch(spec)
    a = G.form_mass()[2].clone()
    b = G.form_mass()[2].clone()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    H = gpu_patch(spec)
    c = H.form_mass()[2]
    torch.cuda.synchronize()
    assert torch.equal(a, c)


def _sampled_rows_parity(spec, n_random, cut_stride, seed):
    """The whole matrix from the GPU; seeded random rows and every cut_stride-th
    cut row against the oracle's row-by-row formation (pattern bit-exact,
    values within TOL relative Frobenius over the sampled rows)."""
    G = gpu_patch(spec)
    O = oracle.Patch(spec)
    assert (G.n_rows, G.nnz) == (O.n_rows, O.nnz)
    rp, col, val = G.form_mass()
    torch.cuda.synchronize()
    rp = rp.cpu().numpy()
    col = col.cpu().numpy()
    val = val.cpu().numpy()
    assert np.all(np.isfinite(val))
    rng = np.random.default_rng(seed)
    es, fs, act = O.states()
    cut_rows = act[(fs == 2)]
    rows = np.unique(np.concatenate([rng.integers(0, G.n_rows, n_random), cut_rows[::cut_stride]]))
    num = den = 0.0
    for r in rows:
        oc, ov = O.form_row(int(r))
        assert np.array_equal(col[rp[r]:rp[r + 1]], oc)
        mv = val[rp[r]:rp[r + 1]]
        num += np.sum((mv - ov) ** 2)
        den += np.sum(ov ** 2)
    assert np.sqrt(num / den) <= TOL


@pytest.mark.parametrize("p", [4, 6])
def test_full_size_config3_sampled_rows(p):
    """1024 x 1024 elements, p = 4 and 6 (the largest patches, 61.5 M and
    129 M nonzeros), circular hole, perturbed spline geometry."""
    _sampled_rows_parity(synth.config3(p=p, nel=1024), 300, 29, p)


@pytest.mark.parametrize("p", [3, 4, 5])
@pytest.mark.parametrize("method", ["hybrid", "dwq"])
def test_benchmark_128_patches_full(p, method):
    """The six 128 x 128 patches of the benchmark sweep, whole matrices."""
    compare_full(synth.config2(p=p, nel=128, method=method))


@pytest.mark.parametrize("p,method", [(3, "hybrid"), (4, "dwq"), (5, "hybrid"),
                                      (3, "dwq"), (4, "hybrid"), (5, "dwq")])
def test_full_size_config2_sampled_rows(p, method):
    """512 x 512 elements (the benchmark's patches): the whole matrix from the
    GPU, 400 seeded rows (and every cut row among the first 100k) against the
    oracle's row-by-row formation."""
    spec = synth.config2(p=p, nel=512, method=method)
    G = gpu_patch(spec)
    O = oracle.Patch(spec)
    assert (G.n_rows, G.nnz) == (O.n_rows, O.nnz)
    rp, col, val = G.form_mass()
    torch.cuda.synchronize()
    rp = rp.cpu().numpy()
    col = col.cpu().numpy()
    val = val.cpu().numpy()
    assert np.all(np.isfinite(val))
    rng = np.random.default_rng(p)
    es, fs, act = O.states()
    cut_rows = act[(fs == 2)]
    rows = np.unique(np.concatenate([rng.integers(0, G.n_rows, 400), cut_rows[::7]]))
    num = den = 0.0
    for r in rows:
        oc, ov = O.form_row(int(r))
        assert np.array_equal(col[rp[r]:rp[r + 1]], oc)
        mv = val[rp[r]:rp[r + 1]]
        num += np.sum((mv - ov) ** 2)
        den += np.sum(ov ** 2)
    assert np.sqrt(num / den) <= TOL


@pytest.mark.parametrize("method", ["hybrid", "dwq", "gauss"])
def test_rhs_and_l2_projection(method):
    spec = synth.make_spec(3, (17, 15), synth.circle(0.5, 0.5, 0.27), method=method)
    G = gpu_patch(spec)
    O = oracle.Patch(spec)
    rng = np.random.default_rng(9)
    fspl = synth.func_spline(spec, rng)
    b = G.rhs(fspl).cpu().numpy()
    ob = O.rhs(fspl)
    assert rel_fro(b, ob) <= TOL
    f = synth.func_sinsin()
    assert rel_fro(G.rhs(f).cpu().numpy(), O.rhs(f)) <= TOL
    csr = G.form_mass()
    u, it, rel = G.l2_project(f, csr, tol=1e-12)
    assert rel <= 1e-12
    # M_s is ill-conditioned without extended B-splines (tiny cut supports),
    # so solutions are compared through the residual of the oracle's system
    import scipy.sparse as sp
    orp, ocol, oval = O.form()
    M = sp.csr_matrix((oval, ocol, orp), shape=(O.n_rows, O.n_rows))
    Ms = 0.5 * (M + M.T)
    obf = O.rhs(f)
    assert np.linalg.norm(Ms @ u.cpu().numpy() - obf) / np.linalg.norm(obf) <= 1e-11
    ou, oit, orel = O.cg(orp, ocol, oval, obf, tol=1e-12)
    assert abs(it - oit) <= 16
    # reproduction of a function of the spline space (reading R9)
    ua, _, rela = G.l2_project(fspl, csr, tol=1e-13)
    es, fs, act = O.states()
    a = fspl["coef"].ravel()[act >= 0]
    ua = ua.cpu().numpy()
    assert np.linalg.norm(Ms @ ua - ob) / np.linalg.norm(ob) <= 1e-12
    if method != "dwq":  # c = 1: M is symmetric up to roundoff, so u = a
        assert np.linalg.norm(ua - a) / np.linalg.norm(a) < 1e-3  # bounded by cond(M_s) * tol


def test_geometry_rhs_and_projection_det_j():
    spec = synth.config2(p=3, nel=20, method="hybrid", seed=5)
    G = gpu_patch(spec)
    O = oracle.Patch(spec)
    f = synth.func_sincos(2.0, 3.0)
    assert rel_fro(G.rhs(f).cpu().numpy(), O.rhs(f)) <= TOL


def test_cg_reports_non_convergence():
    spec = synth.config1("hybrid")
    G = gpu_patch(spec)
    csr = G.form_mass()
    from paper_2101_08053_gb300.api import TWError
    with pytest.raises(TWError) as ei:
        G.l2_project(synth.func_sinsin(), csr, tol=1e-14, maxit=2)
    assert ei.value.code == -5


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_basis_tables_against_scipy(p):
    """Basis values at the WQ points and at the element Gauss points (tables
    11 and 13) against scipy's B-splines, for every degree."""
    from pins import bvals
    spec = synth.make_spec(p, 9, synth.circle(0.5, 0.5, 0.3))
    G = gpu_patch(spec)
    U = spec["knots"][0]
    x = G.table(0).cpu().numpy()
    Bq = G.table(11).cpu().numpy().reshape(len(x), p + 1)
    el = np.minimum(np.searchsorted(U[p:len(U) - p], x, side="right") - 1, 8)
    for k in range(len(x)):
        ref = [bvals(U, p, el[k] + a, x[k])[()] for a in range(p + 1)]
        assert np.allclose(Bq[k], ref, atol=1e-14)
    GB = G.table(13).cpu().numpy().reshape(9, p + 1, p + 1)
    gx, _ = np.polynomial.legendre.leggauss(p + 1)
    for e in range(9):
        a, b = U[p + e], U[p + e + 1]
        for g in range(p + 1):
            xx = a + (b - a) * (gx[g] + 1) / 2
            ref = [bvals(U, p, e + q, xx)[()] for q in range(p + 1)]
            assert np.allclose(GB[e, g], ref, atol=1e-14)


@pytest.mark.parametrize("extended", [False, True])
@pytest.mark.parametrize("trim", ["circle", "line"])
@pytest.mark.parametrize("p", [2, 3])
def test_l2_projection_convergence_rates(trim, p, extended):
    """Sect. 4.2: the L2 projection of sin(2x) cos(3y) on the trimmed patch
    converges at the optimal rate p + 1 under h-refinement, in the plain and
    in the extended B-spline basis (the paper's setting); the error is
    measured by tw_loss (the same rule as the oracle's L2 error)."""
    f = synth.func_sincos(2.0, 3.0)
    errs = []
    for nel in (8, 16, 32, 64):
        tr = synth.circle(0.5, 0.5, 0.27) if trim == "circle" else synth.line(*synth.LINE_TRIM)
        spec = synth.make_spec(p, nel, tr, method="hybrid")
        G = gpu_patch(spec)
        csr = G.form_mass("fp64")
        if extended:
            u, it, rel = G.l2_project_extended(f, G.form_mass_extended(csr), tol=1e-13,
                                               check=False)
        else:
            u, it, rel = G.l2_project(f, csr, tol=1e-13, check=False)
        L, _ = G.loss(u, f)
        errs.append(float(L.item()) ** 0.5)
        if nel <= 16:  # the same rule as the oracle's loss, for the same u
            O = oracle.Patch(spec)
            L_o, _ = O.loss(u.cpu().numpy(), f)
            assert abs(L_o ** 0.5 - errs[-1]) <= 1e-10 * errs[-1]
    rates = [np.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]
    assert min(rates[1:]) > p + 0.6, rates


@pytest.mark.parametrize("method", ["gauss", "hybrid", "dwq", "naive"])
@pytest.mark.parametrize("p", [2, 3, 5])
def test_graded_knots(p, method):
    """Non-uniform simple knots (reading R1), graded geometrically and
    differently per direction, with a circular hole."""
    U1 = synth.graded_knots(p, 9, 1.2)
    U2 = synth.graded_knots(p, 12, 0.85)
    spec = synth.with_knots(synth.make_spec(p, 4, synth.circle(0.47, 0.52, 0.29), method=method),
                            U1, U2)
    compare_full(spec)


def test_graded_knots_spline_hole_density():
    rng = np.random.default_rng(31)
    U1 = synth.graded_knots(4, 14, 1.1)
    U2 = synth.graded_knots(4, 11, 0.9)
    trim = synth.bspline_curve(rng, nc=8, radius=0.3, jitter=0.1, relative_jitter=True)
    dens = synth.density(rng, q=2, m=7)
    spec = synth.with_knots(synth.make_spec(4, 4, trim, coef=dens, method="dwq"), U1, U2)
    compare_full(spec)


@pytest.mark.parametrize("method", ["hybrid", "dwq"])
def test_scans_beyond_direct_carry_at_2048(method):
    """2048 x 2048 elements, p = 2: the function, element and row-pointer
    scans run over more than 2048 blocks of 1024 entries, so the block totals
    are scanned by their own pass before the carries are added.  States, the
    active numbering and the matrix size bit-exact against the oracle, and
    sampled rows (cut and interior, the first and the last) against rows the
    oracle forms one by one, by the sampled-row bar (relative Frobenius over
    the rows)."""
    spec = synth.make_spec(2, 2048, synth.circle(0.47, 0.53, 0.29), method=method)
    G = gpu_patch(spec)
    O = oracle.Patch(spec)
    assert (G.n_rows, G.nnz) == (O.n_rows, O.nnz)
    es, fs, act = [t.cpu().numpy() for t in G.states()]
    oes, ofs, oact = O.states()
    assert np.array_equal(es, oes) and np.array_equal(fs, ofs) and np.array_equal(act, oact)
    rp, col, val = [t.cpu().numpy() for t in G.form_mass("fp64")]
    assert rp[-1] == O.nnz
    rng = np.random.default_rng(20)
    gs = list(rng.choice(np.where(ofs == 2)[0], 20, replace=False))
    gs += list(rng.choice(np.where(ofs == 1)[0], 20, replace=False))
    rows = [int(oact[g]) for g in gs] + [0, O.n_rows - 1]
    num = den = 0.0
    for row in rows:
        oc, ov = O.form_row(row)
        assert np.array_equal(col[rp[row]:rp[row + 1]], oc)
        num += np.sum((val[rp[row]:rp[row + 1]] - ov) ** 2)
        den += np.sum(ov ** 2)
    assert np.sqrt(num / den) <= TOL
