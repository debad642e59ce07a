"""Reduced-precision forms of the interior contraction against the FP64 oracle.

TW_PREC_FP32X2 (split precision on the FP32 pipes, FP64 output) is held to the
FP64 bar, 1e-12 relative Frobenius; TW_PREC_FP32 (FP32 tables and FMA, float
output) to the stated 2e-6.  The CSR pattern is identical in every mode."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUND = {"fp32x2": 1e-12, "fp32": 2e-6}


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("mode", ["fp32x2", "fp32"])
@pytest.mark.parametrize("spec", [synth.config1("hybrid"),
                                  synth.config2(p=3, nel=24, method="dwq", seed=21),
                                  synth.config2(p=5, nel=28, method="hybrid", seed=22),
                                  synth.make_spec(6, (17, 23), synth.circle(0.5, 0.5, 0.3),
                                                  method="hybrid")],
                         ids=["config1", "p3-dwq", "p5-hybrid", "p6-ragged"])
def test_precision_modes_against_oracle(mode, spec):
    from paper_2101_08053_gb300 import Patch
    G = Patch(spec)
    O = oracle.Patch(spec)
    rp, col, val = G.form_mass(mode)
    torch.cuda.synchronize()
    orp, ocol, oval = O.form()
    assert np.array_equal(rp.cpu().numpy(), orp)
    assert np.array_equal(col.cpu().numpy(), ocol)
    v = val.double().cpu().numpy()
    assert rel(v, oval) <= BOUND[mode], rel(v, oval)


def test_precision_modes_full_size_sampled():
    """512 x 512, p = 4: split precision matches the FP64 GPU form to 1e-13
    over the whole matrix and the oracle on sampled rows to 1e-12."""
    from paper_2101_08053_gb300 import Patch
    spec = synth.config2(p=4, nel=512, method="dwq")
    G = Patch(spec)
    v64 = G.form_mass("fp64")[2].clone()
    rp, col, v2 = G.form_mass("fp32x2")
    v32 = G.form_mass("fp32")[2]
    torch.cuda.synchronize()
    n64 = torch.linalg.norm(v64)
    assert float(torch.linalg.norm(v2 - v64) / n64) <= 1e-13
    assert float(torch.linalg.norm(v32.double() - v64) / n64) <= BOUND["fp32"]
    O = oracle.Patch(spec)
    rp = rp.cpu().numpy()
    v2 = v2.cpu().numpy()
    num = den = 0.0
    for r in np.random.default_rng(4).integers(0, G.n_rows, 300):
        oc, ov = O.form_row(int(r))
        num += np.sum((v2[rp[r]:rp[r + 1]] - ov) ** 2)
        den += np.sum(ov ** 2)
    assert np.sqrt(num / den) <= 1e-12
