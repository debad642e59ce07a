"""ctypes binding of the FP64 CPU oracle (plain C in this folder).

Two builds of the same sources: liboracle.so (single thread, the oracle the
tests pin) and liboracle_omp.so (compiled with -fopenmp, so the pragmas on the
independent loops -- WQ weights per function, c per grid line, DWQ choice per
function, rows -- run on all host cores; it serves only the benchmark's
all-cores CPU baseline).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference arm are the only callers.  The product library never
imports, links or calls this package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
LIB_OMP = os.path.join(HERE, "liboracle_omp.so")
SOURCES = ["or_core.c", "or_curve.c", "or_patch.c"]

TRIM = {"none": 0, "circle": 1, "ellipse": 2, "bspline3": 3, "line": 4}
GEOM = {"identity": 0, "spline": 1}
COEF = {"one": 0, "detj": 1, "density": 2}
METHOD = {"gauss": 0, "hybrid": 1, "dwq": 2, "naive": 3}
FUNC = {"spline": 0, "sinsin": 1, "sincos": 2, "gauss": 3}


def _build_one(out, extra, force):
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    hdr = os.path.join(HERE, "oracle.h")
    if not force and os.path.exists(out):
        t = os.path.getmtime(out)
        if all(os.path.getmtime(s) <= t for s in srcs + [hdr]):
            return out
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared"] + extra + ["-o", tmp]
                          + srcs + ["-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (single-threaded, -O2, FP64) and, where
    the compiler has OpenMP, liboracle_omp.so."""
    _build_one(LIB, [], force)
    try:
        _build_one(LIB_OMP, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        pass
    return LIB


class Trim(C.Structure):
    _fields_ = [
        ("kind", C.c_int),
        ("keep_inside", C.c_int),
        ("params", C.c_double * 6),
        ("nctrl", C.c_int),
        ("ctrl", C.POINTER(C.c_double)),
    ]


class Desc(C.Structure):
    _fields_ = [
        ("p", C.c_int * 2),
        ("nknots", C.c_int * 2),
        ("knots", C.POINTER(C.c_double) * 2),
        ("trim_kind", C.c_int),
        ("trim_keep_inside", C.c_int),
        ("trim_params", C.c_double * 6),
        ("trim_nctrl", C.c_int),
        ("trim_ctrl", C.POINTER(C.c_double)),
        ("geom_kind", C.c_int),
        ("geom_ctrl", C.POINTER(C.c_double)),
        ("coef_kind", C.c_int),
        ("dens_p", C.c_int * 2),
        ("dens_nknots", C.c_int * 2),
        ("dens_knots", C.POINTER(C.c_double) * 2),
        ("dens_coef", C.POINTER(C.c_double)),
        ("method", C.c_int),
        ("cut_order", C.c_int),
        ("trim_nextra", C.c_int),
        ("trim_extra", C.POINTER(Trim)),
    ]


class Func(C.Structure):
    _fields_ = [
        ("kind", C.c_int),
        ("prm", C.c_double * 4),
        ("p", C.c_int * 2),
        ("nknots", C.c_int * 2),
        ("knots", C.POINTER(C.c_double) * 2),
        ("coef", C.POINTER(C.c_double)),
    ]


_lib = None
_lib_omp = None
PD = C.POINTER(C.c_double)
PI64 = C.POINTER(C.c_int64)
PI32 = C.POINTER(C.c_int32)
PU8 = C.POINTER(C.c_uint8)


def lib(omp=False):
    global _lib, _lib_omp
    if omp:
        if _lib_omp is None:
            build()
            if not os.path.exists(LIB_OMP):
                return None
            _lib_omp = _declare(C.CDLL(LIB_OMP))
        return _lib_omp
    if _lib is None:
        build()
        _lib = _declare(C.CDLL(LIB))
    return _lib


def _declare(L):
    if True:
        L.or_bspline.restype = C.c_double
        L.or_bspline.argtypes = [PD, C.c_int, C.c_int, C.c_int, C.c_double]
        L.or_bspline_deriv.restype = C.c_double
        L.or_bspline_deriv.argtypes = [PD, C.c_int, C.c_int, C.c_int, C.c_double]
        L.or_gauss_legendre.argtypes = [C.c_int, PD, PD]
        L.or_minnorm.argtypes = [C.c_int, C.c_int, PD, PD, PD]
        L.or_insert_knot.argtypes = [PD, C.c_int, C.c_int, C.c_double, PD, PD, PD]
        L.or_wq_points.argtypes = [PD, C.c_int, C.c_int, PD]
        L.or_wq_weights.argtypes = [PD, C.c_int, C.c_int, PD, C.c_int, C.c_int, PD]
        L.or_curve_line_hits.argtypes = [C.POINTER(Desc), C.c_int, C.c_double, C.c_double,
                                         C.c_double, PD, C.c_int]
        L.or_curve_inside.argtypes = [C.POINTER(Desc), C.c_double, C.c_double]
        L.or_curve_area.restype = C.c_double
        L.or_curve_area.argtypes = [C.POINTER(Desc), C.c_int]
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [C.POINTER(Desc)]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_dims.argtypes = [C.c_void_p, PI64]
        L.or_states.argtypes = [C.c_void_p, PU8, PU8, PI32]
        L.or_wq_grid.argtypes = [C.c_void_p, C.c_int, PD]
        L.or_cgrid.argtypes = [C.c_void_p, PD]
        L.or_cut_rule.argtypes = [C.c_void_p, C.c_int, C.c_int, PD, C.c_int]
        L.or_dwq_rule.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, PD, C.c_int]
        L.or_dwq_choice.argtypes = [C.c_void_p, C.c_int, C.c_int, PI32]
        L.or_form.argtypes = [C.c_void_p, PI64, PI32, PD]
        L.or_form_row.argtypes = [C.c_void_p, C.c_int64, PI32, PD]
        L.or_form_row_remark1.argtypes = [C.c_void_p, C.c_int64, PI32, PD]
        L.or_rhs.argtypes = [C.c_void_p, C.POINTER(Func), PD]
        L.or_row_points.argtypes = [C.c_void_p, C.c_int64, PD, C.c_int]
        L.or_cg.argtypes = [C.c_void_p, PI64, PI32, PD, PD, PD, C.c_double, C.c_int, PD]
        L.or_l2_error.restype = C.c_double
        L.or_l2_error.argtypes = [C.c_void_p, PD, C.POINTER(Func), PD]
        L.or_visible_area.restype = C.c_double
        L.or_visible_area.argtypes = [C.c_void_p]
        L.or_loss.restype = C.c_double
        L.or_loss.argtypes = [C.c_void_p, PD, C.POINTER(Func), PD]
        L.or_density_grad.argtypes = [C.c_void_p, PD, PD, C.POINTER(Func), PD]
        L.or_form_rows.argtypes = [C.c_void_p, PI64, C.c_int64, PD, PI32]
        L.or_threads.restype = C.c_int
    return L


def _pd(a):
    return a.ctypes.data_as(PD)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_desc(spec, keep):
    """Fill an or_desc from a synth patch spec; `keep` collects arrays that
    must outlive the call."""
    d = Desc()
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
        arr = (Trim * len(extra))()
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
                arr[k].ctrl = _pd(ctrl)
        keep.append(arr)
        d.trim_nextra = len(extra)
        d.trim_extra = C.cast(arr, C.POINTER(Trim))
    return d


def make_func(f, keep):
    s = Func()
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


def threads(omp=False):
    """Threads the oracle's parallel loops use in the given build."""
    L = lib(omp)
    return int(L.or_threads()) if L is not None else 0


# ---- univariate helpers ----------------------------------------------------

def bspline(U, p, i, x, deriv=False):
    U = _f64(U)
    fn = lib().or_bspline_deriv if deriv else lib().or_bspline
    return fn(_pd(U), len(U), p, i, float(x))


def gauss_legendre(q):
    x = np.zeros(q)
    w = np.zeros(q)
    lib().or_gauss_legendre(q, _pd(x), _pd(w))
    return x, w


def minnorm(A, b):
    A = _f64(A)
    b = _f64(b)
    w = np.zeros(A.shape[1])
    rc = lib().or_minnorm(A.shape[0], A.shape[1], _pd(A), _pd(b), _pd(w))
    assert rc == 0
    return w


def insert_knot(U, p, t, c):
    U = _f64(U)
    c = _f64(c)
    Un = np.zeros(len(U) + 1)
    cn = np.zeros(len(c) + 1)
    lib().or_insert_knot(_pd(U), len(U), p, float(t), _pd(c), _pd(Un), _pd(cn))
    return Un, cn


def wq_points(U, p):
    U = _f64(U)
    n = lib().or_wq_points(_pd(U), len(U), p, None)
    x = np.zeros(n)
    lib().or_wq_points(_pd(U), len(U), p, _pd(x))
    return x


def wq_weights(U, p, x, i):
    U = _f64(U)
    x = _f64(x)
    w = np.zeros(len(x))
    n = lib().or_wq_weights(_pd(U), len(U), p, _pd(x), len(x), i, _pd(w))
    assert n > 0
    return w


def _curve_desc(trim, keep):
    spec = {"p": 1, "knots": [np.array([0, 0, 1, 1.0])] * 2, "trim": trim,
            "geom": {"kind": "identity"}, "coef": {"kind": "one"}, "method": "hybrid"}
    return make_desc(spec, keep)


def curve_line_hits(trim, o, s, lo=-1e300, hi=1e300):
    keep = []
    d = _curve_desc(trim, keep)
    out = np.zeros(1024)
    n = lib().or_curve_line_hits(C.byref(d), o, float(s), float(lo), float(hi), _pd(out), 1024)
    return out[:n].copy()


def curve_inside(trim, x, y):
    keep = []
    d = _curve_desc(trim, keep)
    return bool(lib().or_curve_inside(C.byref(d), float(x), float(y)))


def curve_area(trim, nsub=8):
    keep = []
    d = _curve_desc(trim, keep)
    return lib().or_curve_area(C.byref(d), nsub)


# ---- patch -----------------------------------------------------------------


def check_knots(U, p):
    """Open knot vector (p+1 equal end knots, no more), non-decreasing, every
    interior knot of multiplicity 1..p (continuity C^{p-m}, reading R1)."""
    if len(U) < 2 * p + 3 or np.any(np.diff(U) < 0):
        raise ValueError("knots must be non-decreasing with at least two elements")
    if np.any(U[:p + 1] != U[0]) or np.any(U[-p - 1:] != U[-1]) or not (U[p + 1] > U[0]) \
            or not (U[-p - 2] < U[-1]):
        raise ValueError("knot vector is not open (exactly p+1 equal end knots)")
    inner = U[p + 1:len(U) - p - 1]
    if inner.size:
        _, counts = np.unique(inner, return_counts=True)
        if counts.max() > p:
            raise ValueError("an interior knot of multiplicity %d > p" % counts.max())

class Patch:
    def __init__(self, spec, omp=False):
        """omp=True builds the patch with the all-cores library (benchmark
        baseline only)."""
        self.spec = spec
        for U in spec["knots"]:
            check_knots(np.asarray(U, dtype=np.float64), spec["p"])
        self._L = lib(omp)
        if self._L is None:
            raise RuntimeError("the OpenMP build of the oracle is not available")
        keep = []
        d = make_desc(spec, keep)
        self._h = self._L.or_create(C.byref(d))
        dims = np.zeros(8, dtype=np.int64)
        self._L.or_dims(self._h, dims.ctypes.data_as(PI64))
        (self.n1, self.n2, self.nel1, self.nel2, self.nq1, self.nq2,
         self.n_rows, self.nnz) = [int(v) for v in dims]
        self.p = spec["p"]

    def __del__(self):
        if getattr(self, "_h", None):
            self._L.or_destroy(self._h)
            self._h = None

    def states(self):
        es = np.zeros(self.nel1 * self.nel2, dtype=np.uint8)
        fs = np.zeros(self.n1 * self.n2, dtype=np.uint8)
        act = np.zeros(self.n1 * self.n2, dtype=np.int32)
        self._L.or_states(self._h, es.ctypes.data_as(PU8), fs.ctypes.data_as(PU8),
                        act.ctypes.data_as(PI32))
        return es, fs, act

    def wq_grid(self, d):
        x = np.zeros(self.nq1 if d == 0 else self.nq2)
        self._L.or_wq_grid(self._h, d, _pd(x))
        return x

    def cgrid(self):
        c = np.zeros(self.nq1 * self.nq2)
        self._L.or_cgrid(self._h, _pd(c))
        return c.reshape(self.nq2, self.nq1)

    def cut_rule(self, e1, e2):
        cap = 1 << 16
        out = np.zeros(3 * cap)
        n = self._L.or_cut_rule(self._h, e1, e2, _pd(out), cap)
        return out[:3 * n].reshape(n, 3).copy()

    def dwq_rule(self, d, s, side, i):
        cap = 4096
        out = np.zeros(2 * cap)
        n = self._L.or_dwq_rule(self._h, d, s, side, i, _pd(out), cap)
        return out[:2 * n].reshape(n, 2).copy()

    def dwq_choice(self, i1, i2):
        out = np.zeros(4, dtype=np.int32)
        self._L.or_dwq_choice(self._h, i1, i2, out.ctypes.data_as(PI32))
        return tuple(int(v) for v in out)

    def form(self):
        rp = np.zeros(self.n_rows + 1, dtype=np.int64)
        col = np.zeros(max(self.nnz, 1), dtype=np.int32)
        val = np.zeros(max(self.nnz, 1), dtype=np.float64)
        self._L.or_form(self._h, rp.ctypes.data_as(PI64), col.ctypes.data_as(PI32), _pd(val))
        return rp, col[:self.nnz], val[:self.nnz]

    def form_row_remark1(self, r):
        """Row r with its Gauss part as Remark 1's masked tensor rule over the
        whole support; None for a row with a region part."""
        cap = (2 * self.p + 1) ** 2
        col = np.zeros(cap, dtype=np.int32)
        val = np.zeros(cap)
        n = self._L.or_form_row_remark1(self._h, int(r), col.ctypes.data_as(PI32), _pd(val))
        if n < 0:
            return None
        return col[:n].copy(), val[:n].copy()

    def form_rows(self, rows):
        """Entries of the rows `rows` (in C, in parallel with the all-cores
        library): (values, counts), values padded to (2p+1)^2 per row."""
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        w = (2 * self.p + 1) ** 2
        val = np.zeros(max(len(rows), 1) * w)
        cnt = np.zeros(max(len(rows), 1), dtype=np.int32)
        self._L.or_form_rows(self._h, rows.ctypes.data_as(PI64), len(rows), _pd(val),
                             cnt.ctypes.data_as(PI32))
        return val[:len(rows) * w].reshape(len(rows), w), cnt[:len(rows)]

    def form_row(self, r):
        cap = (2 * self.p + 1) ** 2
        col = np.zeros(cap, dtype=np.int32)
        val = np.zeros(cap)
        n = self._L.or_form_row(self._h, int(r), col.ctypes.data_as(PI32), _pd(val))
        return col[:n].copy(), val[:n].copy()

    def rhs(self, f):
        keep = []
        fs = make_func(f, keep)
        b = np.zeros(self.n_rows)
        self._L.or_rhs(self._h, C.byref(fs), _pd(b))
        return b

    def row_points(self, r):
        """The quadrature rule of active row r: an (n, 5) array of xi1, xi2,
        x1, x2 (physical point) and the weight with B_i and c folded in."""
        cap = 1 << 14
        while True:
            out = np.zeros(5 * cap)
            n = self._L.or_row_points(self._h, int(r), _pd(out), cap)
            if n <= cap:
                return out[:5 * n].reshape(n, 5).copy()
            cap = n

    def rhs_from(self, f):
        """b_i = sum over row i's rule of w c f(x) for a Python callable
        f(x1, x2) of the physical point (vectorised over numpy arrays)."""
        b = np.zeros(self.n_rows)
        for r in range(self.n_rows):
            q = self.row_points(r)
            b[r] = float(np.sum(q[:, 4] * f(q[:, 2], q[:, 3])))
        return b

    def cg(self, rp, col, val, b, tol=1e-12, maxit=None):
        u = np.zeros(self.n_rows)
        rel = C.c_double(0)
        rp = np.ascontiguousarray(rp, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = _f64(val)
        b = _f64(b)
        it = self._L.or_cg(self._h, rp.ctypes.data_as(PI64), col.ctypes.data_as(PI32), _pd(val),
                         _pd(b), _pd(u), tol, maxit or 10 * self.n_rows, C.byref(rel))
        return u, it, rel.value

    def l2_error(self, u, f):
        keep = []
        fs = make_func(f, keep)
        fn = C.c_double(0)
        u = _f64(u)
        e = self._L.or_l2_error(self._h, _pd(u), C.byref(fs), C.byref(fn))
        return e, fn.value

    def visible_area(self):
        return self._L.or_visible_area(self._h)

    def loss(self, u, g):
        """(L, dL/du) of reading R12."""
        keep = []
        gs = make_func(g, keep)
        u = _f64(u)
        dl = np.zeros(self.n_rows)
        L = self._L.or_loss(self._h, _pd(u), C.byref(gs), _pd(dl))
        return L, dl

    def density_grad(self, u, lam, g):
        keep = []
        gs = make_func(g, keep)
        c = self.spec["coef"]
        m1 = len(c["knots"][0]) - c["p"] - 1
        m2 = len(c["knots"][1]) - c["p"] - 1
        out = np.zeros(m1 * m2)
        self._L.or_density_grad(self._h, _pd(_f64(u)), _pd(_f64(lam)), C.byref(gs), _pd(out))
        return out.reshape(m2, m1)
