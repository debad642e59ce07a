"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/trimwq.h; host-side validation rejects malformed
descriptors before any device work (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "trimwq.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|const char \*)\s*\*?\s*(tw_\w+)\s*\(", txt, re.M)))


def test_library_exports_every_declared_symbol():
    from paper_2101_08053_gb300 import api
    L = api.load()
    syms = declared_symbols()
    assert len(syms) >= 10
    for s in syms:
        assert hasattr(L, s), s


def test_header_symbols_cover_the_binding():
    syms = set(declared_symbols())
    for s in ["tw_patch_create", "tw_patch_destroy", "tw_form_mass", "tw_rhs", "tw_l2_project",
              "tw_states", "tw_patch_info", "tw_patch_table", "tw_last_error", "tw_launch_count",
              "tw_extension_build", "tw_extension_matrix", "tw_form_mass_extended",
              "tw_l2_project_extended"]:
        assert s in syms


@pytest.mark.parametrize("bad", ["degree", "mixed", "knots", "closed", "trim", "method", "cut",
                                 "extra_count", "extra_null", "extra_curve"])
def test_descriptor_validation_on_host(bad):
    from paper_2101_08053_gb300 import api
    L = api.load()
    spec = synth.config1()
    keep = []
    d = api.make_patch_desc(spec, keep)
    if bad == "degree":
        d.p[0] = d.p[1] = 9
        code = -2
    elif bad == "mixed":
        d.p[1] = 3
        code = -2
    elif bad == "knots":
        U = np.array([0, 0, 0, 0.5, 0.4, 1, 1, 1.0])
        keep.append(U)
        d.knots[0] = U.ctypes.data_as(api.PD)
        d.nknots[0] = len(U)
        code = -1
    elif bad == "closed":
        U = np.array([0, 0, 0.1, 0.5, 0.9, 1, 1, 1.0])
        keep.append(U)
        d.knots[0] = U.ctypes.data_as(api.PD)
        d.nknots[0] = len(U)
        code = -1
    elif bad == "trim":
        d.trim_params[2] = -0.1
        code = -1
    elif bad == "method":
        d.method = 7
        code = -1
    elif bad == "extra_count":  # more curves than TW_MAXCURVES
        d.trim_nextra = 8
        arr = (api.TrimCurve * 8)()
        keep.append(arr)
        d.trim_extra = C.cast(arr, C.POINTER(api.TrimCurve))
        code = -1
    elif bad == "extra_null":
        d.trim_nextra = 1
        code = -1
    elif bad == "extra_curve":  # a second curve with a negative radius
        arr = (api.TrimCurve * 1)()
        arr[0].kind = 1
        arr[0].params[2] = -0.2
        keep.append(arr)
        d.trim_nextra = 1
        d.trim_extra = C.cast(arr, C.POINTER(api.TrimCurve))
        code = -1
    else:
        d.cut_order = 1000
        code = -1
    h = C.c_void_p()
    rc = L.tw_patch_create(C.byref(d), C.byref(h))
    assert rc == code
    assert len(L.tw_last_error()) > 0
    assert not h.value


def test_extension_entry_points_reject_null_arguments_on_host():
    """The extended B-spline entry points check their arguments before any
    device work: NULL patch or buffers give TW_EINVAL and an error text."""
    from paper_2101_08053_gb300 import api
    L = api.load()
    info = np.zeros(4, dtype=np.int64)
    assert L.tw_extension_build(None, info.ctypes.data_as(C.POINTER(C.c_int64))) == -1
    assert len(L.tw_last_error()) > 0
    assert L.tw_extension_matrix(None, None, None, None, None) == -1
    assert L.tw_form_mass_extended(None, None, None, None, None, None, None, None) == -1
    keep = []
    fd = api.make_func_desc(synth.func_sincos(2.0, 3.0), keep)
    it, rel = C.c_int(0), C.c_double(0)
    assert L.tw_l2_project_extended(None, C.byref(fd), None, None, None, None, 1e-12, 10,
                                    C.byref(it), C.byref(rel), None) == -1
    assert L.tw_l2_project_adjoint_extended(None, C.byref(fd), None, None, None, None, None,
                                            None, None, 1e-12, 10, C.byref(it), C.byref(rel),
                                            None) == -1
