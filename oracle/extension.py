"""Extended B-splines of a trimmed patch -- plain numpy restatement.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference arm are the only callers.  The product library never
imports, links or calls this package.

The paper stabilises every L2 projection (Sect. 3, "extended B-spline concept",
and Sect. 4.2) with the extended B-splines of Hoellig, Reif and Wipper, and
defers their construction to that literature.  The steps below restate that
construction for a tensor-product patch; the points the paper leaves open are
fixed by these readings:

  R15  inner / outer.  An active function is *inner* when at least one element
       of its support is regular (wholly visible); every other active function
       is *outer*.
  R16  closest inner array.  Each outer j = (j1, j2) is tied to one array
       l + {0..p}^2 of inner functions: among the arrays all of whose members
       are inner, with l_v in [j_v - 2p - 1, j_v + p + 1], the one whose centre
       l + p/2 is nearest to j (squared Euclidean distance in index space);
       ties go to the smaller l2, then the smaller l1.  An outer function with
       no such array makes the extension undefined (the patch is too coarse
       for its trim).
  R17  extension coefficients.  e_{i,j} = e1 * e2 with each 1-D factor the
       unique coefficients for which sum_a e_a lambda_{l+a}(q) = lambda_j(q)
       for every polynomial q of degree <= p, lambda_k(q) being q's k-th
       B-spline coefficient (the dual functional).  The extended space thus
       reproduces polynomials; on uniform knots this is the Lagrange form
       prod_{mu != a} (j - l - mu) / (a - mu).

With E the (active x inner) matrix whose inner rows are the identity and whose
outer row j holds e_{i,j} in the columns of its array, the extended functions
are B^e_i = B_i + sum_j e_{i,j} B_j, a coefficient vector x of the extended
basis is u = E x in the active basis, and the mass matrix and the right-hand
side of the extended basis are E^T M E and E^T b.  The extended L2 projection
solves E^T M_s E x = E^T b (M_s = (M + M^T)/2) and returns u = E x.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

ELEM_REGULAR = 1
REACH = 1  # R16: l_v ranges over [j_v - 2p - REACH, j_v + p + REACH]


def support_elements(i, p, nel):
    """Elements of supp B_i for an open knot vector with simple interior knots
    (element e spans the knots e + p, e + p + 1)."""
    return range(max(0, i - p), min(nel - 1, i) + 1)


def classify(P):
    """R15: (inner, outer) boolean arrays over g = i2 * n1 + i1."""
    es, fs, act = P.states()
    n1, n2, nel1, p = P.n1, P.n2, P.nel1, P.p
    inner = np.zeros(n1 * n2, dtype=bool)
    outer = np.zeros(n1 * n2, dtype=bool)
    for g in range(n1 * n2):
        if act[g] < 0:
            continue
        i1, i2 = g % n1, g // n1
        reg = any(es[e2 * nel1 + e1] == ELEM_REGULAR
                  for e2 in support_elements(i2, p, P.nel2)
                  for e1 in support_elements(i1, p, nel1))
        inner[g] = reg
        outer[g] = not reg
    return inner, outer


def array_ok(inner, n1, n2, p):
    """ok[l2, l1]: every member of the array l + {0..p}^2 is inner."""
    I = inner.reshape(n2, n1)
    ok = np.zeros((n2 - p, n1 - p), dtype=bool)
    for l2 in range(n2 - p):
        for l1 in range(n1 - p):
            ok[l2, l1] = I[l2:l2 + p + 1, l1:l1 + p + 1].all()
    return ok


def closest_array(ok, j1, j2, p):
    """R16: (l1, l2) of the nearest all-inner array, or None."""
    n2p, n1p = ok.shape
    best = None
    for l2 in range(max(0, j2 - 2 * p - REACH), min(n2p - 1, j2 + p + REACH) + 1):
        for l1 in range(max(0, j1 - 2 * p - REACH), min(n1p - 1, j1 + p + REACH) + 1):
            if not ok[l2, l1]:
                continue
            d = (2 * l1 + p - 2 * j1) ** 2 + (2 * l2 + p - 2 * j2) ** 2
            if best is None or d < best[0]:  # scan order: l2, then l1 ascending
                best = (d, l1, l2)
    return None if best is None else (best[1], best[2])


def elementary_symmetric(u):
    """sigma_0..sigma_n of the values u: coefficients of prod_r (1 + u_r z)."""
    s = np.zeros(len(u) + 1)
    s[0] = 1.0
    for v in u:
        s[1:] = s[1:] + v * s[:-1]
    return s


def dual_of_monomials(U, p, k, c, h):
    """lambda_k(((x - c)/h)^m) for m = 0..p: the blossom of the monomial at
    the knots U[k+1..k+p] (Marsden's identity), sigma_m / binom(p, m) of the
    knots in the local coordinate (x - c)/h."""
    u = (np.asarray(U[k + 1:k + p + 1], dtype=np.float64) - c) / h
    s = elementary_symmetric(u)
    return np.array([s[m] / math.comb(p, m) for m in range(p + 1)])


def coef_1d(U, p, j, l):
    """R17, one direction: e_a (a = 0..p) with sum_a e_a lambda_{l+a} =
    lambda_j on the polynomials of degree <= p, solved in the monomial basis
    of a local coordinate spanning the knots involved."""
    lo = min(j, l) + 1
    hi = max(j, l + p) + p
    c = 0.5 * (U[lo] + U[hi])
    h = U[hi] - U[lo]
    V = np.stack([dual_of_monomials(U, p, l + a, c, h) for a in range(p + 1)], axis=1)
    rhs = dual_of_monomials(U, p, j, c, h)
    return np.linalg.solve(V, rhs)


class Extension:
    """The extension of an oracle.Patch: inner/outer sets, the array of each
    outer function and the matrix E (scipy CSR, active x inner)."""

    def __init__(self, P):
        self.P = P
        p, n1, n2 = P.p, P.n1, P.n2
        U1, U2 = [np.asarray(u, dtype=np.float64) for u in P.spec["knots"]]
        for U in (U1, U2):
            inner_knots = U[p + 1:len(U) - p - 1]
            if inner_knots.size and np.any(np.diff(inner_knots) == 0):
                # the arrays (R16) are read on simple knots: with a repeated
                # knot p+1 consecutive functions need not share an element
                raise ValueError("extended B-splines need simple interior knots")
        es, fs, act = P.states()
        self.act = act
        self.inner, self.outer = classify(P)
        self.inner_index = np.full(n1 * n2, -1, dtype=np.int64)
        self.inner_index[self.inner] = np.arange(int(self.inner.sum()))
        self.n_inner = int(self.inner.sum())
        self.n_outer = int(self.outer.sum())
        ok = array_ok(self.inner, n1, n2, p)
        self.arrays = {}
        self.coefs = {}
        rows, cols, vals = [], [], []
        for g in range(n1 * n2):
            if act[g] < 0:
                continue
            r = int(act[g])
            if self.inner[g]:
                rows.append(r)
                cols.append(int(self.inner_index[g]))
                vals.append(1.0)
                continue
            j1, j2 = g % n1, g // n1
            arr = closest_array(ok, j1, j2, p)
            if arr is None:
                raise ValueError("outer function (%d, %d) has no inner array within reach" % (j1, j2))
            l1, l2 = arr
            e1 = coef_1d(U1, p, j1, l1)
            e2 = coef_1d(U2, p, j2, l2)
            self.arrays[g] = (l1, l2)
            self.coefs[g] = (e1, e2)
            for a2 in range(p + 1):
                for a1 in range(p + 1):
                    gi = (l2 + a2) * n1 + (l1 + a1)
                    rows.append(r)
                    cols.append(int(self.inner_index[gi]))
                    vals.append(e1[a1] * e2[a2])
        self.E = sp.csr_matrix((vals, (rows, cols)), shape=(P.n_rows, self.n_inner))
        self.E.sort_indices()

    def mass(self, rp, col, val):
        """E^T M E as (row_ptr, col, val) on the structural pattern: entry
        (a, b) is present when some r, s with E[r, a] != 0, E[s, b] != 0 have a
        stored entry M[r, s] (structural zeros of M included)."""
        n = self.P.n_rows
        M = sp.csr_matrix((np.asarray(val, dtype=np.float64), col, rp), shape=(n, n))
        S = sp.csr_matrix((np.ones(len(col)), col, rp), shape=(n, n))
        Eb = sp.csr_matrix((np.ones(self.E.nnz), self.E.indices, self.E.indptr), shape=self.E.shape)
        pat = (Eb.T @ S @ Eb).tocsr()
        pat.sort_indices()
        X = (self.E.T @ M @ self.E).tocoo()
        # place the product's (numerically nonzero) entries on the pattern
        m = self.n_inner
        prow = np.repeat(np.arange(m, dtype=np.int64), np.diff(pat.indptr))
        pkey = prow * m + pat.indices
        xkey = X.row.astype(np.int64) * m + X.col
        pos = np.searchsorted(pkey, xkey)
        assert np.all(pkey[pos] == xkey)
        out = np.zeros(pat.nnz)
        out[pos] = X.data
        return pat.indptr.astype(np.int64), pat.indices.astype(np.int32), out

    def project(self, f, rp, col, val):
        """Extended L2 projection: u = E x with E^T M_s E x = E^T b(f) (sparse
        direct solve)."""
        n = self.P.n_rows
        M = sp.csr_matrix((np.asarray(val, dtype=np.float64), col, rp), shape=(n, n))
        Ms = 0.5 * (M + M.T)
        A = (self.E.T @ Ms @ self.E).tocsc()
        b = self.P.rhs(f)
        x = spla.spsolve(A, self.E.T @ b)
        return self.E @ x, x
