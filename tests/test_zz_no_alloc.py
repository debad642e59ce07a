"""tw_rhs_static, the allocation-free right-hand side, against tw_rhs.

tw_rhs_static serves callers that cannot allocate device memory while they
run (memory owned by another allocator, time-critical loops that must not pay
for cudaMalloc / cudaFree); its scratch is a fixed file-scope device array.  It
must give the same b as tw_rhs, call after call, although every call reuses
the array the previous call left behind.  This file is collected last so that
a run stopping at the first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _lib():
    from paper_2101_08053_gb300 import api
    L = api.load()
    L.tw_rhs_static.argtypes = [C.c_void_p, C.POINTER(api.FuncDesc), C.c_void_p, C.c_void_p]
    return api, L


def _static_rhs(api, L, P, f):
    keep = []
    fd = api.make_func_desc(f, keep)
    out = torch.full((max(P.n_rows, 1),), float("nan"), dtype=torch.float64, device="cuda")
    rc = L.tw_rhs_static(P._h, C.byref(fd), C.c_void_p(out.data_ptr()),
                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, L.tw_last_error().decode()
    torch.cuda.synchronize()
    return out[:P.n_rows].cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("spec", [synth.config1("hybrid"),
                                  synth.config2(p=4, nel=24, method="dwq", seed=11),
                                  synth.config5(nel=20, method="gauss")],
                         ids=["config1-hybrid", "spline-geometry-dwq", "density-gauss"])
def test_static_rhs_equals_tw_rhs_on_consecutive_calls(spec):
    api, L = _lib()
    P = api.Patch(spec)
    rng = np.random.default_rng(17)
    fs = [synth.func_spline(spec, rng), synth.func_sinsin(), synth.func_spline(spec, rng)]
    for f in fs:
        ref = P.rhs(f).cpu().numpy()
        first = _static_rhs(api, L, P, f)
        second = _static_rhs(api, L, P, f)
        assert np.all(np.isfinite(first)) and np.all(np.isfinite(second))
        assert _rel(first, ref) <= TOL
        assert _rel(second, ref) <= TOL


def test_static_rhs_rejects_scratch_beyond_the_array():
    api, L = _lib()
    P = api.Patch(synth.make_spec(2, (1100, 1000), synth.circle(0.5, 0.5, 0.3)))
    assert P.nq1 * P.nq2 > 1 << 21
    keep = []
    fd = api.make_func_desc(synth.func_sinsin(), keep)
    out = torch.empty(P.n_rows, dtype=torch.float64, device="cuda")
    rc = L.tw_rhs_static(P._h, C.byref(fd), C.c_void_p(out.data_ptr()),
                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1
    assert b"static array" in L.tw_last_error()
