// tw_func.cuh -- the projected function f (Sect. 4.2's data) on the device:
// a tensor spline in its own knots, or one of the closed-form test functions of
// the physical coordinates.  Shared by the rhs and the adjoint.
#pragma once
#include <cstring>

#include "tw_internal.cuh"

namespace tw {

struct Func {
  int kind;
  double prm[4];
  int q[2], nk[2], m1;
  const double *U[2];
  const double *coef;
};

// Where the value of f at a rule point is found when f is given by its values
// at the points of tw_rhs_points: the WQ grid from 0, the element Gauss points
// from gbase, the cut-rule points from cbase and the DWQ region points of cut
// row r from dbase + roff[r].
struct PtIndex {
  const double *FV;
  const int64_t *roff;
  int64_t gbase, cbase, dbase;
};

static __device__ __forceinline__ void phys_at(const Geo &G, const Dir &A, const Dir &B, double x1,
                                        double x2, double *X) {
  if (G.geom_kind != TW_GEOM_SPLINE) {
    X[0] = x1;
    X[1] = x2;
    return;
  }
  int e1 = elem_of(A.bp, A.nel, x1), e2 = elem_of(B.bp, B.nel, x2);
  double v1[TW_MAXP1], v2[TW_MAXP1];
  basis_vals(A.U, e1 + A.p, x1, A.p, v1);
  basis_vals(B.U, e2 + B.p, x2, B.p, v2);
  X[0] = X[1] = 0.0;
  for (int b = 0; b <= B.p; b++)
    for (int a = 0; a <= A.p; a++) {
      const double *pt = G.ctrl + 2 * ((size_t)(e2 + b) * G.n1 + (e1 + a));
      X[0] += pt[0] * v1[a] * v2[b];
      X[1] += pt[1] * v1[a] * v2[b];
    }
}

static __device__ double func_at(const Func &f, double x1, double x2, const double *X) {
  switch (f.kind) {
    case TW_FUNC_SPLINE: {
      double N1[TW_MAXP1], N2[TW_MAXP1];
      int s1 = find_span(f.U[0], f.q[0], f.nk[0] - f.q[0] - 1, x1);
      int s2 = find_span(f.U[1], f.q[1], f.nk[1] - f.q[1] - 1, x2);
      basis_vals(f.U[0], s1, x1, f.q[0], N1);
      basis_vals(f.U[1], s2, x2, f.q[1], N2);
      double s = 0.0;
      for (int b = 0; b <= f.q[1]; b++)
        for (int a = 0; a <= f.q[0]; a++)
          s += f.coef[(size_t)(s2 - f.q[1] + b) * f.m1 + (s1 - f.q[0] + a)] * N1[a] * N2[b];
      return s;
    }
    case TW_FUNC_SINSIN: return sin(f.prm[0] * X[0]) * sin(f.prm[1] * X[1]);
    case TW_FUNC_SINCOS: return sin(f.prm[0] * X[0]) * cos(f.prm[1] * X[1]);
    case TW_FUNC_GAUSS: {
      double dx = X[0] - f.prm[1], dy = X[1] - f.prm[2];
      return exp(-f.prm[0] * (dx * dx + dy * dy));
    }
  }
  return 0.0;
}

static __device__ __forceinline__ double fpoint(const Func &f, const Geo &G, const Dir &A, const Dir &B,
                                         double x1, double x2) {
  double X[2];
  phys_at(G, A, B, x1, x2, X);
  return func_at(f, x1, x2, X);
}

static Func make_func(const tw_func *f, tw_patch *P, int *rc) {
  Func F;
  memset(&F, 0, sizeof(F));
  F.kind = f->kind;
  for (int k = 0; k < 4; k++) F.prm[k] = f->prm[k];
  *rc = 0;
  if (f->kind < TW_FUNC_SPLINE || f->kind > TW_FUNC_GAUSS) {
    set_error("unknown function kind %d", f->kind);
    *rc = TW_EINVAL;
    return F;
  }
  if (f->kind == TW_FUNC_SPLINE) {
    size_t m = 1;
    for (int d = 0; d < 2; d++) {
      if (!f->knots[d] || f->p[d] < 0 || f->p[d] > TW_MAXP || f->nknots[d] < 2 * f->p[d] + 2) {
        set_error("spline function: bad knots or degree");
        *rc = TW_EINVAL;
        return F;
      }
      F.q[d] = f->p[d];
      F.nk[d] = f->nknots[d];
      double *u = (double *)dalloc(P, sizeof(double) * f->nknots[d]);
      if (!u) { *rc = TW_ENOMEM; return F; }
      cudaMemcpyAsync(u, f->knots[d], sizeof(double) * f->nknots[d], cudaMemcpyHostToDevice,
                      P->stream);
      F.U[d] = u;
      m *= (size_t)(f->nknots[d] - f->p[d] - 1);
    }
    F.m1 = f->nknots[0] - f->p[0] - 1;
    double *c = (double *)dalloc(P, sizeof(double) * m);
    if (!c || !f->coef) { *rc = c ? TW_EINVAL : TW_ENOMEM; return F; }
    cudaMemcpyAsync(c, f->coef, sizeof(double) * m, cudaMemcpyHostToDevice, P->stream);
    F.coef = c;
  }
  return F;
}

}  // namespace tw
