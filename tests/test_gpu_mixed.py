"""Mixed-continuity knot vectors (Sect. 2.1, reading R1) on the GPU against the
oracle: repeated interior knots of multiplicity 2..p, empty elements on their
zero-length spans, p+1 WQ points next to them.  States and CSR patterns bit
for bit, values within the parity tolerance, in every method and precision;
the WQ points and the cut-element rules point for point; the right-hand side
and the L2 projection; the batch; the extension's refusal."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _spec(p, r1, r2, nel, trim=None, method="hybrid", geom=False, coef=None, seed=0):
    U1 = synth.mixed_knots(p, nel[0], r1)
    U2 = synth.mixed_knots(p, nel[1], r2)
    g = None
    if geom:
        rng = np.random.default_rng(100 + p + seed)
        g = {"kind": "spline", "ctrl": synth.perturbed_bilinear_net(
            rng, p, len(U1) - 2 * p - 1, knots=(U1, U2))}
    if trim is None:
        trim = synth.circle(0.47, 0.53, 0.29)
    spec = synth.make_spec(p, nel, trim, geom=g, coef=coef or ({"kind": "detj"} if geom else None),
                           method=method)
    return synth.with_knots(spec, U1, U2)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CASES = [
    (2, {3: 2}, {5: 2}, (12, 11), "hybrid", False),
    (3, {2: 3, 6: 2}, {4: 2}, (13, 12), "dwq", True),
    (3, {4: 3}, {3: 3, 7: 3}, (12, 12), "gauss", False),
    (4, {3: 2, 4: 4}, {6: 3}, (14, 13), "hybrid", True),
    (4, {5: 2}, {2: 4}, (14, 14), "dwq", False),
    (5, {4: 5}, {6: 2}, (15, 14), "naive", False),
    (6, {5: 2}, {7: 3}, (16, 15), "dwq", True),
    (6, {3: 6, 8: 2}, {4: 2}, (16, 16), "hybrid", False),
]


@pytest.mark.parametrize("p,r1,r2,nel,method,geom", CASES,
                         ids=["p%d-%s%s" % (c[0], c[4], "-geo" if c[5] else "") for c in CASES])
def test_mixed_continuity_parity(p, r1, r2, nel, method, geom):
    from paper_2101_08053_gb300 import api
    spec = _spec(p, r1, r2, nel, method=method, geom=geom)
    G = api.Patch(spec)
    O = oracle.Patch(spec)
    assert (G.n1, G.n2, G.nq1, G.nq2, G.n_rows, G.nnz) == (O.n1, O.n2, O.nq1, O.nq2, O.n_rows, O.nnz)
    es, fs, act = [t.cpu().numpy() for t in G.states()]
    oes, ofs, oact = O.states()
    assert np.array_equal(es, oes) and np.array_equal(fs, ofs) and np.array_equal(act, oact)
    assert np.any(es == 3)  # empty elements present
    for d in (0, 1):
        assert np.allclose(G.table(d).cpu().numpy(), O.wq_grid(d), rtol=0, atol=1e-15)
    orp, ocol, oval = O.form()
    for prec, tol in (("fp64", TOL), ("fp32x2", TOL), ("fp32", 2e-6)):
        rp, col, val = [t.cpu().numpy() for t in G.form_mass(prec)]
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
        v = val.astype(np.float64)
        assert np.all(np.isfinite(v))
        assert _rel(v, oval) <= tol, (prec, _rel(v, oval))
    if method != "naive":
        rp, col, val = [t.cpu().numpy() for t in G.form_mass("fp64", rowsf=True)]
        assert np.array_equal(col, ocol) and _rel(val, oval) <= TOL
    # cut-element rules, element by element
    pts = G.table(5).cpu().numpy().reshape(-1, 3)
    off = G.table(6).cpu().numpy()
    ids = G.table(7).cpu().numpy()
    for ci in range(len(ids)):
        e = int(ids[ci])
        ref = O.cut_rule(e % G.nel1, e // G.nel1)
        mine = pts[off[ci]:off[ci + 1]]
        assert mine.shape == ref.shape
        assert np.max(np.abs(mine - ref)) <= 1e-14
    if method == "dwq":
        ch = G.table(8).cpu().numpy().reshape(-1, 4)
        for g in np.where(ofs == 2)[0]:
            assert tuple(ch[g]) == O.dwq_choice(int(g % G.n1), int(g // G.n1))
    # right-hand sides: a descriptor kind and an f outside the kinds (two-phase)
    f = synth.func_sincos()
    assert _rel(G.rhs(f).cpu().numpy(), O.rhs(f)) <= TOL
    xi, x = G.rhs_points()
    xy = x.cpu().numpy().reshape(-1, 2)
    fv = np.cos(3 * xy[:, 0] + xy[:, 1] ** 2) * np.exp(-xy[:, 1])
    ofn = lambda X, Y: np.cos(3 * X + Y ** 2) * np.exp(-Y)
    b = G.rhs_values(torch.tensor(fv, device="cuda")).cpu().numpy()
    assert _rel(b, O.rhs_from(ofn)) <= TOL


def test_mixed_untrimmed_exact_and_projection():
    """No trim, c = 1, C^0 and C^1 knots: the GPU matrix equals the products of
    1-D integrals (through the oracle pinned to them), and the L2 projection of
    a spline of the space reproduces its coefficients."""
    from paper_2101_08053_gb300 import api
    spec = _spec(3, {3: 3, 5: 2}, {4: 3}, (10, 9),
                 trim={"kind": "none", "params": [0.0] * 6, "ctrl": None, "keep_inside": False})
    G = api.Patch(spec)
    O = oracle.Patch(spec)
    rp, col, val = G.form_mass("fp64")
    orp, ocol, oval = O.form()
    assert np.array_equal(col.cpu().numpy(), ocol)
    assert _rel(val.cpu().numpy(), oval) <= 1e-14
    f = synth.func_spline(spec, np.random.default_rng(2))
    u, it, rel = G.l2_project(f, (rp, col, val), tol=1e-13)
    es, fs, act = O.states()
    a = f["coef"].ravel()[act >= 0]
    assert np.linalg.norm(u.cpu().numpy() - a) / np.linalg.norm(a) < 1e-10


def test_mixed_sampled_rows_at_256():
    """256 x 256 elements, p = 4, a C^0 knot and two C^2 knots per direction,
    spline geometry, DWQ: sampled rows against the oracle."""
    from paper_2101_08053_gb300 import api
    r = {60: 4, 128: 2, 200: 2}
    spec = _spec(4, r, r, (256, 256), trim=synth.bspline_curve(np.random.default_rng(8), nc=12,
                                                                radius=0.3, jitter=0.05),
                 method="dwq", geom=True)
    G = api.Patch(spec)
    O = oracle.Patch(spec)
    rp, col, val = [t.cpu().numpy() for t in G.form_mass("fp64")]
    es, fs, act = O.states()
    assert np.array_equal(G.states()[0].cpu().numpy(), es)
    rng = np.random.default_rng(6)
    rows = list(rng.choice(np.where(fs == 2)[0], size=40, replace=False))
    rows += list(rng.choice(np.where(fs == 1)[0], size=40, replace=False))
    num = den = 0.0
    for g in rows:
        row = int(act[g])
        oc, ov = O.form_row(row)
        assert np.array_equal(col[rp[row]:rp[row + 1]], oc)
        num += float(np.sum((val[rp[row]:rp[row + 1]] - ov) ** 2))
        den += float(np.sum(ov ** 2))
    assert np.sqrt(num / den) <= TOL


def test_mixed_batch_and_refusals():
    """A mixed patch in a batch forms the same CSR bit for bit; a patch with more
    points under a tile than the batch carries is refused, and so is the
    extension (R16 on simple knots); the one-patch formation takes both."""
    from paper_2101_08053_gb300 import api
    small = _spec(3, {4: 2}, {5: 2}, (12, 12), method="dwq")
    P = api.Patch(small)
    ref = [t.clone() for t in P.form_mass("fp64")]
    outs = [P.alloc_csr("fp64")]
    B = api.Batch([P], outs, precision="fp64")
    B.run()
    torch.cuda.synchronize()
    assert torch.equal(outs[0][2][:P.nnz], ref[2]) and torch.equal(outs[0][1][:P.nnz], ref[1])
    B.close()
    dense = _spec(6, {k: 2 for k in range(1, 16)}, {}, (16, 12), method="hybrid")
    Q = api.Patch(dense)
    O = oracle.Patch(dense)
    assert _rel(Q.form_mass("fp64")[2].cpu().numpy(), O.form()[2]) <= TOL
    with pytest.raises(RuntimeError):
        api.Batch([Q], [Q.alloc_csr("fp64")], precision="fp64")
    with pytest.raises(RuntimeError):
        P.extension()


def test_descriptor_refuses_multiplicity_p_plus_one():
    from paper_2101_08053_gb300 import api
    spec = synth.make_spec(2, 8, synth.circle(0.5, 0.5, 0.3))
    bad = synth.with_knots(spec, synth.mixed_knots(2, 8, {4: 3}), synth.mixed_knots(2, 8, {}))
    with pytest.raises(RuntimeError):
        api.Patch(bad)
