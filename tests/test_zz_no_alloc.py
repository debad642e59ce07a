"""tw_rhs_static, the allocation-free right-hand side, against tw_rhs and the
oracle.

tw_rhs_static serves callers that cannot allocate device memory while they
run (memory owned by another allocator, time-critical loops that must not pay
for cudaMalloc / cudaFree); its scratch is a fixed file-scope device array.  It
must give the same b as tw_rhs, call after call, although every call reuses
the array the previous call left behind, and the same b as the oracle within
the parity tolerance.  It must also allocate nothing: across a call the
library's pool counters and the device's free memory stay where they were.
This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _lib():
    from paper_2101_08053_gb300 import api
    L = api.load()
    L.tw_rhs_static.argtypes = [C.c_void_p, C.POINTER(api.FuncDesc), C.c_void_p, C.c_void_p]
    return api, L


def _static_call(api, L, P, f, out):
    keep = []
    fd = api.make_func_desc(f, keep)
    rc = L.tw_rhs_static(P._h, C.byref(fd), C.c_void_p(out.data_ptr()),
                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, L.tw_last_error().decode()
    torch.cuda.synchronize()  # also keeps the host arrays of `keep` alive past the copy


def _static_rhs(api, L, P, f):
    out = torch.full((max(P.n_rows, 1),), float("nan"), dtype=torch.float64, device="cuda")
    _static_call(api, L, P, f, out)
    return out[:P.n_rows].cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("spec", [synth.config1("hybrid"),
                                  synth.config2(p=4, nel=24, method="dwq", seed=11),
                                  synth.config5(nel=20, method="gauss")],
                         ids=["config1-hybrid", "spline-geometry-dwq", "density-gauss"])
def test_static_rhs_equals_tw_rhs_and_oracle_on_consecutive_calls(spec):
    api, L = _lib()
    P = api.Patch(spec)
    O = oracle.Patch(spec)
    rng = np.random.default_rng(17)
    fs = [synth.func_spline(spec, rng), synth.func_sinsin(), synth.func_spline(spec, rng)]
    for f in fs:
        ref = P.rhs(f).cpu().numpy()
        orc = O.rhs(f)
        first = _static_rhs(api, L, P, f)
        second = _static_rhs(api, L, P, f)
        assert np.all(np.isfinite(first)) and np.all(np.isfinite(second))
        assert _rel(first, ref) <= TOL
        assert _rel(second, ref) <= TOL
        assert _rel(first, orc) <= TOL
        assert _rel(second, orc) <= TOL


def test_static_rhs_allocates_nothing():
    """The first tw_rhs_static call on a freshly created patch, and the next
    one, leave the library pool (allocation count, reserved and used bytes)
    and the device's free memory unchanged."""
    api, L = _lib()
    # warm-up on another patch: module loading and the per-device address
    # lookup of the static array happen here, before anything is measured
    W = api.Patch(synth.config1("hybrid"))
    _static_rhs(api, L, W, synth.func_sinsin())
    spec = synth.config2(p=3, nel=20, method="dwq", seed=5)
    P = api.Patch(spec)
    f = synth.func_spline(spec, np.random.default_rng(3))
    out = torch.empty(P.n_rows, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    before = (api.pool_info(), torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved())
    _static_call(api, L, P, f, out)
    _static_call(api, L, P, synth.func_sinsin(), out)
    after = (api.pool_info(), torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved())
    assert before == after, (before, after)
    assert before[0][1] > 0  # the pool exists and holds the patches' tables


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
