"""Batched formation (one persistent launch replayed from a CUDA graph, tiles
chosen by the autotuner) against one-patch formation: identical CSRs, bit for
bit, in every precision; mixed degrees, sizes, trims and methods."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def batch_specs(n=10, cap=40):
    rng = np.random.default_rng(synth.BASE_SEED + 4)
    out = []
    for k in range(n):
        s = synth.config4_patch(rng, method=("hybrid", "dwq")[k % 2])
        out.append(synth.make_spec(s["p"], (min(s["nel"][0], cap), min(s["nel"][1], cap)),
                                   s["trim"], method=s["method"]))
    return out


@pytest.mark.parametrize("mode", ["fp64", "fp32x2", "fp32"])
def test_batch_equals_single_patch_formation(mode):
    from paper_2101_08053_gb300 import Batch, Patch
    specs = batch_specs()
    patches = [Patch(s) for s in specs]
    assert len({P.p for P in patches}) >= 3
    ref = [P.form_mass(mode) for P in patches]
    ref = [(r.clone(), c.clone(), v.clone()) for r, c, v in ref]
    outs = [P.alloc_csr(mode) for P in patches]
    for o in outs:
        o[2].fill_(float("nan"))
    B = Batch(patches, outs, mode)
    assert B.items > 0 and B.blocks > 0
    assert all(t in (16, 32, 64) for t in B.tiles.values())
    for rep in range(2):
        B.run()
        torch.cuda.synchronize()
        for P, o, r in zip(patches, outs, ref):
            assert torch.equal(o[0], r[0])
            assert torch.equal(o[1][:P.nnz], r[1])
            assert torch.equal(o[2][:P.nnz], r[2])
    B.close()


def test_batch_against_oracle():
    from paper_2101_08053_gb300 import Batch, Patch
    specs = batch_specs(4, cap=24)
    patches = [Patch(s) for s in specs]
    outs = [P.alloc_csr("fp64") for P in patches]
    B = Batch(patches, outs, "fp64")
    B.run()
    torch.cuda.synchronize()
    for s, P, o in zip(specs, patches, outs):
        O = oracle.Patch(s)
        orp, ocol, oval = O.form()
        assert np.array_equal(o[0].cpu().numpy(), orp)
        v = o[2][:P.nnz].cpu().numpy()
        assert np.linalg.norm(v - oval) / np.linalg.norm(oval) <= 1e-12


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_batch_config4_full_size(mode):
    """The benchmark's batch: 512 patches of degree 2..6 and 16..256 elements
    per direction (713 M nonzeros), one persistent launch.  Every patch's CSR
    equals its one-patch formation bit for bit on 24 seeded patches, and the
    three smallest of those equal the oracle's whole matrices (FP64)."""
    from paper_2101_08053_gb300 import Batch, Patch
    rng = np.random.default_rng(synth.BASE_SEED + 4)
    specs = [synth.config4_patch(rng, method="hybrid") for _ in range(512)]
    patches = [Patch(s) for s in specs]
    outs = [P.alloc_csr(mode) for P in patches]
    B = Batch(patches, outs, mode)
    B.run()
    torch.cuda.synchronize()
    pick = np.random.default_rng(44).choice(len(patches), 24, replace=False)
    for k in pick:
        P = patches[k]
        r, c, v = P.form_mass(mode)
        torch.cuda.synchronize()
        assert torch.equal(outs[k][0], r)
        assert torch.equal(outs[k][1][:P.nnz], c)
        assert torch.equal(outs[k][2][:P.nnz], v)
    if mode == "fp64":
        for k in sorted(pick, key=lambda j: patches[j].nnz)[:3]:
            O = oracle.Patch(specs[k])
            orp, ocol, oval = O.form()
            assert np.array_equal(outs[k][0].cpu().numpy(), orp)
            assert np.array_equal(outs[k][1][:patches[k].nnz].cpu().numpy(), ocol)
            vv = outs[k][2][:patches[k].nnz].cpu().numpy()
            assert np.linalg.norm(vv - oval) <= 1e-12 * np.linalg.norm(oval)
    B.close()
    for P in patches:
        P.close()
