"""Thin Python binding of libtrimwq (include/trimwq.h): argument marshalling
only.  Every step of the method runs in the library's sm_103a kernels; PyTorch
provides device memory and streams.  There is no CPU fallback: if the library
or a CUDA device is missing, every call raises."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import _build

TRIM = {"none": 0, "circle": 1, "ellipse": 2, "bspline3": 3, "line": 4}
GEOM = {"identity": 0, "spline": 1}
COEF = {"one": 0, "detj": 1, "density": 2}
METHOD = {"gauss": 0, "hybrid": 1, "dwq": 2, "naive": 3}
PREC = {"fp64": 0, "fp32": 1, "fp32x2": 2}
FUNC = {"spline": 0, "sinsin": 1, "sincos": 2, "gauss": 3}
ERRORS = {-1: "EINVAL", -2: "EUNSUPPORTED", -3: "ENOMEM", -4: "ECUDA", -5: "ENOCONV"}

PD = C.POINTER(C.c_double)


class TWError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class TrimCurve(C.Structure):
    _fields_ = [
        ("kind", C.c_int),
        ("keep_inside", C.c_int),
        ("params", C.c_double * 6),
        ("nctrl", C.c_int),
        ("ctrl", PD),
    ]


class PatchDesc(C.Structure):
    _fields_ = [
        ("p", C.c_int * 2),
        ("nknots", C.c_int * 2),
        ("knots", PD * 2),
        ("trim_kind", C.c_int),
        ("trim_keep_inside", C.c_int),
        ("trim_params", C.c_double * 6),
        ("trim_nctrl", C.c_int),
        ("trim_ctrl", PD),
        ("geom_kind", C.c_int),
        ("geom_ctrl", PD),
        ("coef_kind", C.c_int),
        ("dens_p", C.c_int * 2),
        ("dens_nknots", C.c_int * 2),
        ("dens_knots", PD * 2),
        ("dens_coef", PD),
        ("method", C.c_int),
        ("cut_order", C.c_int),
        ("stream", C.c_void_p),
        ("trim_nextra", C.c_int),
        ("trim_extra", C.POINTER(TrimCurve)),
    ]


class JobDesc(C.Structure):
    _fields_ = [
        ("desc", C.POINTER(PatchDesc)),
        ("precision", C.c_int),
        ("row_ptr", C.c_void_p),
        ("col", C.c_void_p),
        ("val", C.c_void_p),
        ("rows_capacity", C.c_int64),
        ("nnz_capacity", C.c_int64),
        ("h_row_ptr", C.c_void_p),
        ("h_col", C.c_void_p),
        ("h_val", C.c_void_p),
        ("patch", C.c_void_p),
        ("status", C.c_int),
    ]


class FuncDesc(C.Structure):
    _fields_ = [
        ("kind", C.c_int),
        ("prm", C.c_double * 4),
        ("p", C.c_int * 2),
        ("nknots", C.c_int * 2),
        ("knots", PD * 2),
        ("coef", PD),
    ]


_lib = None


def load(build: bool = True):
    """Load libtrimwq.so (building it in-tree first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libtrimwq.so is missing; run __graft_entry__.build()")
    L = C.CDLL(path)
    vp, i64p = C.c_void_p, C.POINTER(C.c_int64)
    L.tw_patch_create.argtypes = [C.POINTER(PatchDesc), C.POINTER(C.c_void_p)]
    L.tw_patch_destroy.argtypes = [vp]
    L.tw_patch_info.argtypes = [vp, i64p]
    L.tw_form_mass.argtypes = [vp, C.c_int, vp, vp, vp, vp]
    L.tw_form_mass_rowsf.argtypes = [vp, C.c_int, vp, vp, vp, vp]
    L.tw_rhs.argtypes = [vp, C.POINTER(FuncDesc), vp, vp]
    L.tw_rhs_points.argtypes = [vp, i64p, vp, vp, vp]
    L.tw_rhs_values.argtypes = [vp, vp, vp, vp]
    L.tw_l2_project.argtypes = [vp, C.POINTER(FuncDesc), vp, vp, vp, vp, C.c_double, C.c_int,
                                C.POINTER(C.c_int), C.POINTER(C.c_double), vp]
    L.tw_loss.argtypes = [vp, C.POINTER(FuncDesc), vp, vp, vp, vp]
    L.tw_l2_project_adjoint.argtypes = [vp, C.POINTER(FuncDesc), vp, vp, vp, vp, vp, vp, vp,
                                        C.c_double, C.c_int, C.POINTER(C.c_int),
                                        C.POINTER(C.c_double), vp]
    L.tw_extension_build.argtypes = [vp, i64p]
    L.tw_extension_matrix.argtypes = [vp, vp, vp, vp, vp]
    L.tw_form_mass_extended.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    L.tw_l2_project_extended.argtypes = [vp, C.POINTER(FuncDesc), vp, vp, vp, vp, C.c_double,
                                         C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double), vp]
    L.tw_l2_project_adjoint_extended.argtypes = [vp, C.POINTER(FuncDesc), vp, vp, vp, vp, vp,
                                                 vp, vp, C.c_double, C.c_int,
                                                 C.POINTER(C.c_int), C.POINTER(C.c_double), vp]
    L.tw_states.argtypes = [vp, vp, vp, vp, vp]
    L.tw_patch_table.argtypes = [vp, C.c_int, vp, C.c_int64, i64p, vp]
    L.tw_run_jobs.argtypes = [C.POINTER(JobDesc), C.c_int, C.c_int]
    L.tw_launch_count.restype = C.c_int64
    L.tw_pool_info.argtypes = [i64p]
    L.tw_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.POINTER(C.c_void_p),
                                  C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), vp,
                                  C.POINTER(C.c_void_p)]
    L.tw_batch_run.argtypes = [vp, vp]
    L.tw_batch_info.argtypes = [vp, i64p]
    L.tw_batch_destroy.argtypes = [vp]
    L.tw_profile_enable.argtypes = [C.c_int]
    L.tw_profile_read.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    L.tw_last_error.restype = C.c_char_p
    _lib = L
    return L


def _check(rc):
    if rc != 0:
        raise TWError(rc, load().tw_last_error().decode())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("trimwq needs a CUDA device (sm_103a); none is available")
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _pd(a):
    return a.ctypes.data_as(PD)


def make_patch_desc(spec, keep):
    d = PatchDesc()
    p = spec["p"]
    for k in range(2):
        U = _f64(spec["knots"][k])
        keep.append(U)
        d.p[k] = p
        d.nknots[k] = len(U)
        d.knots[k] = _pd(U)
    t = spec["trim"]
    d.trim_kind = TRIM[t["kind"]]
    d.trim_keep_inside = int(bool(t.get("keep_inside", False)))
    prm = list(t.get("params", [])) + [0.0] * 6
    for k in range(6):
        d.trim_params[k] = prm[k]
    if t.get("ctrl") is not None:
        ctrl = _f64(t["ctrl"])
        keep.append(ctrl)
        d.trim_nctrl = ctrl.shape[0]
        d.trim_ctrl = _pd(ctrl)
    g = spec["geom"]
    d.geom_kind = GEOM[g["kind"]]
    if g["kind"] == "spline":
        net = _f64(g["ctrl"])
        keep.append(net)
        d.geom_ctrl = _pd(net)
    c = spec["coef"]
    d.coef_kind = COEF[c["kind"]]
    if c["kind"] == "density":
        for k in range(2):
            V = _f64(c["knots"][k])
            keep.append(V)
            d.dens_p[k] = c["p"]
            d.dens_nknots[k] = len(V)
            d.dens_knots[k] = _pd(V)
        dc = _f64(c["coef"])
        keep.append(dc)
        d.dens_coef = _pd(dc)
    d.method = METHOD[spec["method"]]
    d.cut_order = spec.get("cut_order", 0)
    extra = spec.get("extra_trims", [])
    if extra:
        arr = (TrimCurve * len(extra))()
        for k, t in enumerate(extra):
            arr[k].kind = TRIM[t["kind"]]
            arr[k].keep_inside = int(bool(t.get("keep_inside", False)))
            prm = list(t.get("params", [])) + [0.0] * 6
            for m in range(6):
                arr[k].params[m] = prm[m]
            if t.get("ctrl") is not None:
                ctrl = _f64(t["ctrl"])
                keep.append(ctrl)
                arr[k].nctrl = ctrl.shape[0]
                arr[k].ctrl = ctrl.ctypes.data_as(PD)
        keep.append(arr)
        d.trim_nextra = len(extra)
        d.trim_extra = C.cast(arr, C.POINTER(TrimCurve))
    return d


def make_func_desc(f, keep):
    s = FuncDesc()
    s.kind = FUNC[f["kind"]]
    prm = list(f.get("prm", [])) + [0.0] * 4
    for k in range(4):
        s.prm[k] = prm[k]
    if f["kind"] == "spline":
        for k in range(2):
            U = _f64(f["knots"][k])
            keep.append(U)
            s.p[k] = f["p"]
            s.nknots[k] = len(U)
            s.knots[k] = _pd(U)
        cf = _f64(f["coef"])
        keep.append(cf)
        s.coef = _pd(cf)
    return s


class Patch:
    """A trimmed patch with its device tables (tw_patch_create)."""

    def __init__(self, spec, stream=None):
        L = load()
        _torch()
        keep = []
        d = make_patch_desc(spec, keep)
        d.stream = _stream(stream)
        h = C.c_void_p()
        _check(L.tw_patch_create(C.byref(d), C.byref(h)))
        self._h = h
        info = np.zeros(16, dtype=np.int64)
        _check(L.tw_patch_info(self._h, info.ctypes.data_as(C.POINTER(C.c_int64))))
        self.info = info
        (self.n1, self.n2, self.nel1, self.nel2, self.nq1, self.nq2, self.n_rows, self.nnz,
         self.n_cut_elems, self.n_cut_fns, self.n_cut_pts, self.n_dwq_rows, self.n_discs,
         self.n_interior, self.p, self.method) = [int(v) for v in info]
        self.spec = spec

    def close(self):
        if getattr(self, "_h", None):
            load().tw_patch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def alloc_csr(self, precision="fp64"):
        torch = _torch()
        dt = torch.float32 if precision == "fp32" else torch.float64
        rp = torch.empty(self.n_rows + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(max(self.nnz, 1), dtype=torch.int32, device="cuda")
        val = torch.empty(max(self.nnz, 1), dtype=dt, device="cuda")
        return rp, col, val

    def form_mass(self, precision="fp64", out=None, stream=None, rowsf=False):
        """tw_form_mass (or, with rowsf, tw_form_mass_rowsf: Remark 1's row-level
        sum factorisation of the cut rows' Gauss part) into (row_ptr, col, val)
        device tensors."""
        rp, col, val = out if out is not None else self.alloc_csr(precision)
        fn = load().tw_form_mass_rowsf if rowsf else load().tw_form_mass
        _check(fn(self._h, PREC[precision], C.c_void_p(rp.data_ptr()),
                  C.c_void_p(col.data_ptr()), C.c_void_p(val.data_ptr()), _stream(stream)))
        return rp, col[:self.nnz], val[:self.nnz]

    def rhs(self, f, stream=None):
        torch = _torch()
        keep = []
        fd = make_func_desc(f, keep)
        b = torch.empty(max(self.n_rows, 1), dtype=torch.float64, device="cuda")
        _check(load().tw_rhs(self._h, C.byref(fd), C.c_void_p(b.data_ptr()), _stream(stream)))
        return b[:self.n_rows]

    def rhs_points(self, physical=True, stream=None):
        """Every point at which a row's rule evaluates f (tw_rhs_points):
        (xi, x), (npts, 2) float64 device tensors of the parameter and the
        physical points (x is None unless `physical`)."""
        torch = _torch()
        n = C.c_int64(0)
        _check(load().tw_rhs_points(self._h, C.byref(n), None, None, _stream(stream)))
        xi = torch.empty((max(n.value, 1), 2), dtype=torch.float64, device="cuda")
        x = torch.empty((max(n.value, 1), 2), dtype=torch.float64, device="cuda") if physical else None
        _check(load().tw_rhs_points(self._h, C.byref(n), C.c_void_p(xi.data_ptr()),
                                    C.c_void_p(x.data_ptr()) if physical else None,
                                    _stream(stream)))
        return xi[:n.value], (x[:n.value] if physical else None)

    def rhs_values(self, fvals, stream=None):
        """b from the values of f at the points of rhs_points (tw_rhs_values);
        fvals is a float64 device tensor of length npts."""
        torch = _torch()
        fv = fvals.contiguous()
        assert fv.dtype == torch.float64 and fv.is_cuda
        b = torch.empty(max(self.n_rows, 1), dtype=torch.float64, device="cuda")
        _check(load().tw_rhs_values(self._h, C.c_void_p(fv.data_ptr()), C.c_void_p(b.data_ptr()),
                                    _stream(stream)))
        return b[:self.n_rows]

    def l2_project(self, f, csr, tol=1e-12, maxit=None, stream=None, check=True):
        torch = _torch()
        keep = []
        fd = make_func_desc(f, keep)
        rp, col, val = csr
        u = torch.empty(max(self.n_rows, 1), dtype=torch.float64, device="cuda")
        it = C.c_int(0)
        rel = C.c_double(0)
        rc = load().tw_l2_project(self._h, C.byref(fd), C.c_void_p(rp.data_ptr()),
                                  C.c_void_p(col.data_ptr()), C.c_void_p(val.data_ptr()),
                                  C.c_void_p(u.data_ptr()), tol,
                                  int(maxit if maxit is not None else 10 * self.n_rows),
                                  C.byref(it), C.byref(rel), _stream(stream))
        if check:
            _check(rc)
        return u[:self.n_rows], it.value, rel.value

    def loss(self, u, g, stream=None):
        """tw_loss: (L as a 0-d device tensor, dL/du)."""
        torch = _torch()
        keep = []
        gd = make_func_desc(g, keep)
        u = u.contiguous()
        out = torch.empty(max(self.n_rows, 1) + 1, dtype=torch.float64, device="cuda")
        _check(load().tw_loss(self._h, C.byref(gd), C.c_void_p(u.data_ptr()),
                              C.c_void_p(out.data_ptr()), C.c_void_p(out[1:].data_ptr()),
                              _stream(stream)))
        return out[0], out[1:1 + self.n_rows]

    def density_shape(self):
        """(m2, m1) of the density spline; (0, 0) without one."""
        c = self.spec["coef"]
        if c["kind"] != "density":
            return (0, 0)
        return (len(c["knots"][1]) - c["p"] - 1, len(c["knots"][0]) - c["p"] - 1)

    def l2_project_adjoint(self, f, csr, dLdu, u, tol=1e-12, maxit=None, stream=None,
                           check=True):
        """tw_l2_project_adjoint: (dL/dd as (m2, m1), lambda, iterations, residual)."""
        torch = _torch()
        keep = []
        fd = make_func_desc(f, keep)
        rp, col, val = csr
        dLdu = dLdu.contiguous()
        u = u.contiguous()
        lam = torch.empty(max(self.n_rows, 1), dtype=torch.float64, device="cuda")
        m2, m1 = self.density_shape()
        grad = torch.empty(max(m2 * m1, 1), dtype=torch.float64, device="cuda")
        it = C.c_int(0)
        rel = C.c_double(0)
        rc = load().tw_l2_project_adjoint(
            self._h, C.byref(fd), C.c_void_p(rp.data_ptr()), C.c_void_p(col.data_ptr()),
            C.c_void_p(val.data_ptr()), C.c_void_p(dLdu.data_ptr()), C.c_void_p(u.data_ptr()),
            C.c_void_p(lam.data_ptr()), C.c_void_p(grad.data_ptr()), tol,
            int(maxit if maxit is not None else 10 * self.n_rows), C.byref(it), C.byref(rel),
            _stream(stream))
        if check:
            _check(rc)
        return grad[:m2 * m1].view(m2, m1), lam[:self.n_rows], it.value, rel.value

    def extension(self):
        """tw_extension_build: (n_inner, n_outer, nnz of E, nnz of E^T M E)."""
        info = np.zeros(4, dtype=np.int64)
        _check(load().tw_extension_build(self._h, info.ctypes.data_as(C.POINTER(C.c_int64))))
        return tuple(int(v) for v in info)

    def extension_matrix(self, stream=None):
        """E as (row_ptr, col, val) device tensors (n_rows x n_inner)."""
        torch = _torch()
        n_inner, n_outer, nnz_e, nnz_x = self.extension()
        rp = torch.empty(self.n_rows + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(max(nnz_e, 1), dtype=torch.int32, device="cuda")
        val = torch.empty(max(nnz_e, 1), dtype=torch.float64, device="cuda")
        _check(load().tw_extension_matrix(self._h, C.c_void_p(rp.data_ptr()),
                                          C.c_void_p(col.data_ptr()), C.c_void_p(val.data_ptr()),
                                          _stream(stream)))
        return rp, col[:nnz_e], val[:nnz_e]

    def form_mass_extended(self, csr, stream=None):
        """E^T M E from the FP64 CSR of form_mass, as (row_ptr, col, val)."""
        torch = _torch()
        n_inner, n_outer, nnz_e, nnz_x = self.extension()
        rp, col, val = csr
        xrp = torch.empty(n_inner + 1, dtype=torch.int64, device="cuda")
        xcol = torch.empty(max(nnz_x, 1), dtype=torch.int32, device="cuda")
        xval = torch.empty(max(nnz_x, 1), dtype=torch.float64, device="cuda")
        _check(load().tw_form_mass_extended(
            self._h, C.c_void_p(rp.data_ptr()), C.c_void_p(col.data_ptr()),
            C.c_void_p(val.data_ptr()), C.c_void_p(xrp.data_ptr()), C.c_void_p(xcol.data_ptr()),
            C.c_void_p(xval.data_ptr()), _stream(stream)))
        return xrp, xcol[:nnz_x], xval[:nnz_x]

    def l2_project_extended(self, f, xcsr, tol=1e-12, maxit=None, stream=None, check=True):
        """Extended L2 projection: (u = E x on the active basis, iterations, residual)."""
        torch = _torch()
        keep = []
        fd = make_func_desc(f, keep)
        n_inner = self.extension()[0]
        rp, col, val = xcsr
        u = torch.empty(max(self.n_rows, 1), dtype=torch.float64, device="cuda")
        it = C.c_int(0)
        rel = C.c_double(0)
        rc = load().tw_l2_project_extended(
            self._h, C.byref(fd), C.c_void_p(rp.data_ptr()), C.c_void_p(col.data_ptr()),
            C.c_void_p(val.data_ptr()), C.c_void_p(u.data_ptr()), tol,
            int(maxit if maxit is not None else 10 * max(n_inner, 1)), C.byref(it),
            C.byref(rel), _stream(stream))
        if check:
            _check(rc)
        return u[:self.n_rows], it.value, rel.value

    def l2_project_adjoint_extended(self, f, xcsr, dLdu, u, tol=1e-12, maxit=None, stream=None,
                                    check=True):
        """tw_l2_project_adjoint_extended: (dL/dd as (m2, m1), lambda = E mu,
        iterations, residual)."""
        torch = _torch()
        keep = []
        fd = make_func_desc(f, keep)
        n_inner = self.extension()[0]
        rp, col, val = xcsr
        dLdu = dLdu.contiguous()
        u = u.contiguous()
        lam = torch.empty(max(self.n_rows, 1), dtype=torch.float64, device="cuda")
        m2, m1 = self.density_shape()
        grad = torch.empty(max(m2 * m1, 1), dtype=torch.float64, device="cuda")
        it = C.c_int(0)
        rel = C.c_double(0)
        rc = load().tw_l2_project_adjoint_extended(
            self._h, C.byref(fd), C.c_void_p(rp.data_ptr()), C.c_void_p(col.data_ptr()),
            C.c_void_p(val.data_ptr()), C.c_void_p(dLdu.data_ptr()), C.c_void_p(u.data_ptr()),
            C.c_void_p(lam.data_ptr()), C.c_void_p(grad.data_ptr()), tol,
            int(maxit if maxit is not None else 10 * max(n_inner, 1)), C.byref(it),
            C.byref(rel), _stream(stream))
        if check:
            _check(rc)
        return grad[:m2 * m1].view(m2, m1), lam[:self.n_rows], it.value, rel.value

    def states(self, stream=None):
        torch = _torch()
        es = torch.empty(self.nel1 * self.nel2, dtype=torch.uint8, device="cuda")
        fs = torch.empty(self.n1 * self.n2, dtype=torch.uint8, device="cuda")
        act = torch.empty(self.n1 * self.n2, dtype=torch.int32, device="cuda")
        _check(load().tw_states(self._h, C.c_void_p(es.data_ptr()), C.c_void_p(fs.data_ptr()),
                                C.c_void_p(act.data_ptr()), _stream(stream)))
        return es, fs, act

    def table(self, which, stream=None):
        torch = _torch()
        L = load()
        n = C.c_int64(0)
        _check(L.tw_patch_table(self._h, which, None, 0, C.byref(n), _stream(stream)))
        dt = {6: torch.int64, 7: torch.int32, 8: torch.int32}.get(which, torch.float64)
        t = torch.empty(max(n.value, 1), dtype=dt, device="cuda")
        _check(L.tw_patch_table(self._h, which, C.c_void_p(t.data_ptr()), n.value, C.byref(n),
                                _stream(stream)))
        return t[:n.value]


class Jobs:
    """tw_run_jobs: create and form many patches, each on its own stream, from
    the library's native thread pool.  specs and streams (torch streams) per
    job; outs: CSR device buffers per job (Patch.alloc_csr) or None for set-up
    only; host: host CSR buffers per job (pinned tensors) or None.  The
    descriptors are built once here; run() may be called repeatedly and
    returns the created patches' handles for destroy()."""

    def __init__(self, specs, streams, outs=None, precision="fp64", host=None, nthreads=0):
        n = len(specs)
        self._keep = []
        self._descs = (PatchDesc * n)()
        self._jobs = (JobDesc * n)()
        self.n, self.nthreads = n, int(nthreads)
        for k, sp in enumerate(specs):
            d = make_patch_desc(sp, self._keep)
            d.stream = _stream(streams[k])
            self._descs[k] = d
            J = self._jobs[k]
            J.desc = C.pointer(self._descs[k])
            J.precision = PREC[precision]
            if outs is not None:
                rp, col, val = outs[k]
                J.row_ptr, J.col, J.val = rp.data_ptr(), col.data_ptr(), val.data_ptr()
                J.rows_capacity, J.nnz_capacity = rp.numel() - 1, col.numel()
            if host is not None:
                hr, hc, hv = host[k]
                J.h_row_ptr, J.h_col, J.h_val = hr.data_ptr(), hc.data_ptr(), hv.data_ptr()
        self.handles = []

    def run(self):
        rc = load().tw_run_jobs(self._jobs, self.n, self.nthreads)
        self.handles = [self._jobs[k].patch for k in range(self.n)]
        _check(rc)
        return self.handles

    def destroy(self):
        L = load()
        for h in self.handles:
            if h:
                L.tw_patch_destroy(h)
        self.handles = []


class Batch:
    """tw_batch_create / tw_batch_run: many patches formed by one persistent
    launch replayed from a CUDA graph.  `outs` are (row_ptr, col, val) device
    tensors per patch (Patch.alloc_csr); the patches must outlive the batch."""

    def __init__(self, patches, outs, precision="fp64", stream=None):
        L = load()
        n = len(patches)
        arr = lambda vals: (C.c_void_p * n)(*vals)
        self._keep = (patches, outs)
        hp = arr([P._h.value for P in patches])
        rp = arr([o[0].data_ptr() for o in outs])
        col = arr([o[1].data_ptr() for o in outs])
        val = arr([o[2].data_ptr() for o in outs])
        h = C.c_void_p()
        _check(L.tw_batch_create(hp, n, PREC[precision], rp, col, val, _stream(stream),
                                 C.byref(h)))
        self._h = h
        info = np.zeros(10, dtype=np.int64)
        _check(L.tw_batch_info(self._h, info.ctypes.data_as(C.POINTER(C.c_int64))))
        self.n, self.items, self.blocks, self.smem = [int(v) for v in info[:4]]
        self.tiles = {p: int(info[3 + p]) for p in range(1, 7)}

    def run(self, stream=None):
        _check(load().tw_batch_run(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            load().tw_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    return int(load().tw_launch_count())


def pool_info():
    """(allocations from the library pool so far, bytes reserved and bytes in
    use by the pool on the current device)."""
    out = (C.c_int64 * 3)()
    _check(load().tw_pool_info(out))
    return int(out[0]), int(out[1]), int(out[2])


STAGES = {"setup": 0, "interior": 1, "cutrows": 2, "rhs": 3, "cg": 4, "loss": 5, "adjoint": 6,
          "gaussmat": 7, "wq_weights": 8, "dwq": 9}


def profile_enable(on: bool = True):
    _check(load().tw_profile_enable(int(bool(on))))


def profile_read(stage: str):
    """(total device ms, launches) of a stage since the last read."""
    ms = C.c_double(0)
    n = C.c_int64(0)
    _check(load().tw_profile_read(STAGES[stage], C.byref(ms), C.byref(n)))
    return ms.value, n.value


def _density_spec(spec, coef):
    s = dict(spec)
    c = dict(spec["coef"])
    c["coef"] = coef
    s["coef"] = c
    return s


class ProjectionLoss(torch.autograd.Function):
    """L(d) = sum_q omega_q detJ (u_h - g)^2, u_h the L2 projection of f onto
    the trimmed patch's spline space under c = rho(d) det J, as a function of
    the density coefficients d (m2 x m1).  forward: patch setup, formation,
    CG and tw_loss; backward: tw_l2_project_adjoint.  With extended=True the
    projection and its adjoint run in the extended B-spline basis
    (tw_form_mass_extended, tw_l2_project_extended and
    tw_l2_project_adjoint_extended)."""

    @staticmethod
    def forward(ctx, dcoef, spec, f, g, tol, extended):
        d = dcoef.detach().to("cpu", torch.float64).numpy()
        P = Patch(_density_spec(spec, d))
        csr = P.form_mass("fp64")
        if extended:
            csr = P.form_mass_extended(csr)
            u, _, _ = P.l2_project_extended(f, csr, tol=tol)
        else:
            u, _, _ = P.l2_project(f, csr, tol=tol)
        L, dLdu = P.loss(u, g)
        ctx.state = (P, csr, u, dLdu, f, tol, extended)
        return L.to(dcoef.device, dcoef.dtype)

    @staticmethod
    def backward(ctx, gout):
        P, csr, u, dLdu, f, tol, extended = ctx.state
        adj = P.l2_project_adjoint_extended if extended else P.l2_project_adjoint
        grad, _, _, _ = adj(f, csr, dLdu, u, tol=tol)
        ctx.state = None
        return gout * grad.to(gout.device, gout.dtype), None, None, None, None, None


def projection_loss(dcoef, spec, f, g, tol=1e-13, extended=False):
    """Differentiable projection loss (see ProjectionLoss)."""
    _torch()
    return ProjectionLoss.apply(dcoef, spec, f, g, tol, extended)
