"""tw_form_mass_rowsf: the cut rows' Gauss part by the row-level sum
factorisation of Sect. 3.2, Remark 1 (one tensor rule over the support's
element Gauss points with c set to zero off the regular elements).

It is the same quadrature as element-wise hybrid Gauss, so the CSR must have
the pattern of tw_form_mass exactly and its values to rounding, and match the
oracle (whose or_form_row_remark1 is pinned to its element-wise rows) within
the parity tolerance."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _specs():
    rng = np.random.default_rng(31)
    out = []
    for p in (2, 3, 4, 5, 6):
        out.append(("hybrid-p%d" % p, synth.config2(p=p, nel=20 + 2 * p, method="hybrid",
                                                    seed=40 + p)))
    out.append(("dwq-p4", synth.config2(p=4, nel=24, method="dwq", seed=47)))
    out.append(("gauss-p3", synth.config2(p=3, nel=14, method="gauss", seed=48)))
    out.append(("density-p3", synth.config5(nel=24, method="hybrid")))
    out.append(("line-p5", synth.line_trim_spec(5)))
    out.append(("ellipse-graded", synth.with_knots(
        synth.make_spec(4, 20, synth.ellipse(0.5, 0.48, 0.31, 0.2, 0.6), method="hybrid"),
        synth.graded_knots(4, 20), synth.graded_knots(4, 22, ratio=0.93))))
    return out


@pytest.mark.parametrize("name,spec", _specs(), ids=[n for n, _ in _specs()])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rowsf_equals_element_form_and_oracle(name, spec, precision):
    from paper_2101_08053_gb300 import api
    P = api.Patch(spec)
    rp0, col0, val0 = [t.cpu().numpy() for t in P.form_mass(precision)]
    rp1, col1, val1 = [t.cpu().numpy() for t in P.form_mass(precision, rowsf=True)]
    assert np.array_equal(rp0, rp1) and np.array_equal(col0, col1)
    v0, v1 = val0.astype(np.float64), val1.astype(np.float64)
    tol = 1e-13 if precision == "fp64" else 2e-7
    assert np.linalg.norm(v1 - v0) <= tol * np.linalg.norm(v0)
    if precision == "fp64":
        O = oracle.Patch(spec)
        orp, ocol, oval = O.form()
        assert np.array_equal(rp1, orp) and np.array_equal(col1, ocol)
        assert np.linalg.norm(v1 - oval) <= TOL * np.linalg.norm(oval)


def test_rowsf_sampled_rows_at_512():
    """At 512^2, p = 5, sampled cut rows against the oracle's Remark 1 rows."""
    from paper_2101_08053_gb300 import api
    spec = synth.config2(p=5, nel=512, method="hybrid")
    P = api.Patch(spec)
    rp, col, val = [t.cpu().numpy() for t in P.form_mass("fp64", rowsf=True)]
    O = oracle.Patch(spec)
    es, fs, act = O.states()
    cut = np.where(fs == 2)[0]
    rng = np.random.default_rng(5)
    num = den = 0.0
    for g in rng.choice(cut, size=40, replace=False):
        r = int(act[g])
        oc, ov = O.form_row_remark1(r)
        assert np.array_equal(col[rp[r]:rp[r + 1]], oc)
        v = val[rp[r]:rp[r + 1]]
        num += float(np.sum((v - ov) ** 2))
        den += float(np.sum(ov ** 2))
    # relative Frobenius error of the sampled rows (a row of a function with a
    # sliver of visible support has entries near 1e-14 and is not held alone)
    assert np.sqrt(num / den) <= TOL, np.sqrt(num / den)
