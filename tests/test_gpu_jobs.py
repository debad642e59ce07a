"""tw_run_jobs: many patches created and formed on their own streams by the
library's native thread pool give the CSR of tw_patch_create + tw_form_mass,
bit for bit, and the host copies of it."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _specs():
    rng = np.random.default_rng(4)
    return [synth.config1("hybrid"), synth.config2(p=3, nel=24, method="dwq", seed=3),
            synth.config2(p=5, nel=20, method="hybrid", seed=4), synth.config5(nel=20),
            synth.config4_patch(rng, method="dwq"), synth.config4_patch(rng, method="hybrid"),
            synth.make_spec(4, 12, synth.circle(0.5, 0.5, 0.3), method="naive")]


@pytest.mark.parametrize("nthreads", [0, 1, 3])
def test_jobs_equal_one_patch_formation(nthreads):
    from paper_2101_08053_gb300 import api
    specs = _specs()
    ref, outs, host = [], [], []
    for s in specs:
        P = api.Patch(s)
        rp, col, val = P.form_mass("fp64")
        ref.append((rp.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()))
        outs.append(P.alloc_csr("fp64"))
        host.append(tuple(torch.empty(t.numel(), dtype=t.dtype, pin_memory=True) for t in outs[-1]))
        P.close()
    streams = [torch.cuda.Stream() for _ in specs]
    J = api.Jobs(specs, streams, outs=outs, host=host, nthreads=nthreads)
    for _ in range(2):  # the pool serves repeated batches
        for o in outs:
            o[2].fill_(float("nan"))
        J.run()
        torch.cuda.synchronize()
        for k, (r, o, h) in enumerate(zip(ref, outs, host)):
            n, z = len(r[0]) - 1, len(r[1])
            assert np.array_equal(o[0][:n + 1].cpu().numpy(), r[0]), k
            assert np.array_equal(o[1][:z].cpu().numpy(), r[1]), k
            assert np.array_equal(o[2][:z].cpu().numpy(), r[2]), k
            assert np.array_equal(h[0][:n + 1].numpy(), r[0]), k
            assert np.array_equal(h[1][:z].numpy(), r[1]), k
            assert np.array_equal(h[2][:z].numpy(), r[2]), k
        J.destroy()


def test_jobs_set_up_only_and_capacity_error():
    from paper_2101_08053_gb300 import api
    specs = _specs()[:3]
    streams = [torch.cuda.Stream() for _ in specs]
    J = api.Jobs(specs, streams)
    hs = J.run()
    assert all(hs)
    for h, s in zip(hs, specs):
        info = np.zeros(16, dtype=np.int64)
        api._check(api.load().tw_patch_info(h, info.ctypes.data_as(api.C.POINTER(api.C.c_int64))))
        assert info[6] == api.Patch(s).n_rows
    J.destroy()
    # CSR buffers one entry too small: TW_EINVAL, the patch is still returned
    P = api.Patch(specs[1])
    rp, col, val = P.alloc_csr("fp64")
    small = (rp, col[:P.nnz - 1], val[:P.nnz - 1])
    J2 = api.Jobs([specs[1]], [streams[0]], outs=[small])
    with pytest.raises(api.TWError) as ei:
        J2.run()
    assert ei.value.code == -1 and "CSR buffers" in str(ei.value)
    assert J2.handles[0]
    J2.destroy()
