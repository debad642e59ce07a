"""The algorithmic FLOP count behind the bench's roofline (bench.interior_flops)
against a brute-force count on small trimmed patches: for every interior row
(i1, i2) and every output (j1, j2) of its band, one FMA per WQ point of
supp B_i1 cap supp B_j1 (stage 2); for every (i2, j2) and every WQ point k1 of
direction 1 that some interior row of i2 uses, one FMA per point of
supp B_i2 cap supp B_j2 (stage 1).  Supports come from the knot spans and the
points from the oracle's WQ layout, not from the bench's per-element counts."""
import os
import sys

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _brute(spec):
    P = oracle.Patch(spec)
    p = spec["p"]
    U = np.asarray(spec["knots"][0])
    n = len(U) - p - 1
    x = oracle.wq_points(U, p)
    es, fs, act = P.states()
    fs = fs.reshape(n, n)  # [i2, i1]
    insupp = np.array([[U[i] < xk < U[i + p + 1] for xk in x] for i in range(n)])  # [i][k]
    ov = np.zeros((n, n), dtype=np.int64)  # points of supp B_i cap supp B_j
    for i in range(n):
        for j in range(n):
            ov[i, j] = np.count_nonzero(insupp[i] & insupp[j])
    stage2 = 0
    stage1 = 0
    for i2 in range(n):
        rows = [i1 for i1 in range(n) if fs[i2, i1] == 1]
        used = np.zeros(len(x), dtype=bool)
        for i1 in rows:
            used |= insupp[i1]
            for j2 in range(max(0, i2 - p), min(n - 1, i2 + p) + 1):
                for j1 in range(max(0, i1 - p), min(n - 1, i1 + p) + 1):
                    stage2 += ov[i1, j1]
        if rows:
            for j2 in range(max(0, i2 - p), min(n - 1, i2 + p) + 1):
                stage1 += ov[i2, j2] * int(used.sum())
    return 2.0 * (stage1 + stage2), fs


@pytest.mark.parametrize("p,nel,r", [(2, 8, 0.27), (3, 10, 0.3), (4, 11, 0.25), (2, 6, 0.0)])
def test_interior_flops_matches_brute_force(p, nel, r):
    trim = synth.circle(0.5, 0.5, r) if r > 0 else {"kind": "none"}
    spec = synth.make_spec(p, nel, trim)
    ref, fs = _brute(spec)
    got = bench.interior_flops(p, nel, fs.ravel())
    assert got == ref
