// tw_adjoint.cu -- differentiation of the L2 projection (Sect. 4.2) with respect
// to the coefficients d_k of a density spline rho = sum_k d_k N_k, c = rho det J.
//
//   loss     L = sum_q omega_q detJ (u_h - g)^2 over the visible part of the
//            patch: element Gauss (p+1 points per direction) on regular
//            elements, the cut rule on cut elements, and
//            dL/du_j = 2 sum_q omega_q detJ (u_h - g) B_j.
//   adjoint  M_s lambda = dL/du (the projection's CG, M_s = (M + M^T)/2), then
//            dL/dd_k = lambda^T db/dd_k - (lambda^T dM/dd_k u + u^T dM/dd_k lambda)/2
//                    = sum_i sum_{q in rule(i)} w_q detJ N_k [lambda_i f - lambda_i U/2
//                                                             - u_i Lambda/2](x_q)
//            with U = sum_j u_j B_j, Lambda = sum_j lambda_j B_j and w_q row i's
//            weight without c: every row rule (WQ, DWQ, element Gauss, cut rule)
//            is linear in c (Eqs. 4, 5, 7), so d/dd_k replaces c by N_k det J.
//   WQ rows  the double sum over the rows and their tensor points is the
//            transposed sum-factorised contraction (Eq. 7 read backwards) on the
//            WQ grid: LW = sum_i lambda_i W1[i1,.] W2[i2,.], UW likewise, then
//            T = detJ [(f - U/2) LW - Lambda UW/2] and G = N1^T T N2.
//   cut rows one thread per row walks its rule's points (the same three parts
//            as the formation kernel) into a private window of coefficients; the
//            windows are added per coefficient in row order.
// Every output value has one owner thread and a fixed summation order, so the
// loss, dL/du and the gradient are bitwise reproducible.
#include "tw_func.cuh"

namespace tw {

#define ADJ_BLOCKS 256

// det J of the spline geometry from the element's basis values / derivatives
__device__ __forceinline__ double detj_of(const Geo &G, int p, int e1, const double *v1,
                                          const double *d1, int e2, const double *v2,
                                          const double *d2) {
  if (G.geom_kind != TW_GEOM_SPLINE) return 1.0;
  double xa = 0, ya = 0, xb = 0, yb = 0;
  for (int b = 0; b <= p; b++) {
    double sxa = 0, sya = 0, sxb = 0, syb = 0;
    for (int a = 0; a <= p; a++) {
      const double *pt = G.ctrl + 2 * ((size_t)(e2 + b) * G.n1 + (e1 + a));
      sxa += pt[0] * d1[a];
      sya += pt[1] * d1[a];
      sxb += pt[0] * v1[a];
      syb += pt[1] * v1[a];
    }
    xa += sxa * v2[b];
    ya += sya * v2[b];
    xb += sxb * d2[b];
    yb += syb * d2[b];
  }
  return xa * yb - xb * ya;
}

__device__ __forceinline__ void phys_of(const Geo &G, int p, double x1, double x2, int e1,
                                        const double *v1, int e2, const double *v2, double *X) {
  if (G.geom_kind != TW_GEOM_SPLINE) {
    X[0] = x1;
    X[1] = x2;
    return;
  }
  X[0] = X[1] = 0.0;
  for (int b = 0; b <= p; b++)
    for (int a = 0; a <= p; a++) {
      const double *pt = G.ctrl + 2 * ((size_t)(e2 + b) * G.n1 + (e1 + a));
      X[0] += pt[0] * v1[a] * v2[b];
      X[1] += pt[1] * v1[a] * v2[b];
    }
}

// U = sum_j u_j B_j and Lambda = sum_j lambda_j B_j over the active functions
// of element (e1, e2)
__device__ __forceinline__ void active_pair(const int32_t *act, int n1, int p, int e1,
                                            const double *v1, int e2, const double *v2,
                                            const double *u, const double *lam, double *U,
                                            double *L) {
  double su = 0.0, sl = 0.0;
  for (int b = 0; b <= p; b++) {
    double tu = 0.0, tl = 0.0;
    for (int a = 0; a <= p; a++) {
      int32_t r = act[(size_t)(e2 + b) * n1 + (e1 + a)];
      if (r >= 0) {
        tu += u[r] * v1[a];
        if (lam) tl += lam[r] * v1[a];
      }
    }
    su += tu * v2[b];
    sl += tl * v2[b];
  }
  *U = su;
  *L = sl;
}

// ---------------------------------------------------------------------------
// loss and dL/du

// one thread per element: its loss share and the (p+1)^2 local dL/du terms
__global__ void k_loss_elems(Dir A, Dir B, Geo G, Func g, const uint8_t *estate,
                             const int32_t *cut_slot, const int64_t *cut_off,
                             const double *cut_pts, const int32_t *act, const double *u,
                             double *lossE, double *loc) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= A.nel * B.nel) return;
  const int p = A.p, p1 = p + 1;
  int e1 = e % A.nel, e2 = e / A.nel;
  double *lo = loc + (size_t)e * p1 * p1;
  double acc[TW_MAXP1 * TW_MAXP1];
  for (int k = 0; k < p1 * p1; k++) acc[k] = 0.0;
  double L = 0.0;
  uint8_t st = estate[e];
  int64_t q0 = 0, q1 = 0;
  if (st == TW_ELEM_REGULAR) q1 = p1 * p1;
  else if (st == TW_ELEM_CUT) {
    int cs = cut_slot[e];
    q0 = cut_off[cs];
    q1 = cut_off[cs + 1];
  }
  double h1 = 0.5 * (A.bp[e1 + 1] - A.bp[e1]), h2 = 0.5 * (B.bp[e2 + 1] - B.bp[e2]);
  for (int64_t q = q0; q < q1; q++) {
    double x1, x2, om;
    double v1[TW_MAXP1], d1[TW_MAXP1], v2[TW_MAXP1], d2[TW_MAXP1];
    if (st == TW_ELEM_REGULAR) {
      int g1 = (int)(q % p1), g2 = (int)(q / p1);
      x1 = A.bp[e1] + h1 * (A.gx[g1] + 1.0);
      x2 = B.bp[e2] + h2 * (B.gx[g2] + 1.0);
      om = A.gw[g1] * h1 * B.gw[g2] * h2;
      for (int a = 0; a < p1; a++) {
        v1[a] = A.GB[((size_t)e1 * p1 + g1) * p1 + a];
        d1[a] = A.dGB[((size_t)e1 * p1 + g1) * p1 + a];
        v2[a] = B.GB[((size_t)e2 * p1 + g2) * p1 + a];
        d2[a] = B.dGB[((size_t)e2 * p1 + g2) * p1 + a];
      }
    } else {
      x1 = cut_pts[3 * q];
      x2 = cut_pts[3 * q + 1];
      om = cut_pts[3 * q + 2];
      basis_ders(A.U, e1 + p, x1, p, v1, d1);
      basis_ders(B.U, e2 + p, x2, p, v2, d2);
    }
    double dj = detj_of(G, p, e1, v1, d1, e2, v2, d2);
    double X[2], U, dummy;
    phys_of(G, p, x1, x2, e1, v1, e2, v2, X);
    active_pair(act, A.n, p, e1, v1, e2, v2, u, nullptr, &U, &dummy);
    double res = U - func_at(g, x1, x2, X);
    double t = om * dj * res;
    L += t * res;
    for (int b = 0; b < p1; b++)
      for (int a = 0; a < p1; a++) acc[b * p1 + a] += 2.0 * t * v1[a] * v2[b];
  }
  for (int k = 0; k < p1 * p1; k++) lo[k] = acc[k];
  lossE[e] = L;
}

// dL/du_r: the local terms of the row's support elements, e2 then e1 ascending
__global__ void k_dldu(Dir A, Dir B, const int32_t *rowg, int64_t nrows, const double *loc,
                       double *dLdu) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int p = A.p, p1 = p + 1;
  int g = rowg[r];
  int i1 = g % A.n, i2 = g / A.n;
  int lo1 = max(0, i1 - p), hi1 = min(A.nel - 1, i1);
  int lo2 = max(0, i2 - p), hi2 = min(B.nel - 1, i2);
  double s = 0.0;
  for (int e2 = lo2; e2 <= hi2; e2++)
    for (int e1 = lo1; e1 <= hi1; e1++)
      s += loc[((size_t)e2 * A.nel + e1) * p1 * p1 + (i2 - e2) * p1 + (i1 - e1)];
  dLdu[r] = s;
}

// fixed-tree sum of x[0..n): ADJ_BLOCKS partials, then one block
__global__ void k_sum_partial(const double *x, int64_t n, double *part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)ADJ_BLOCKS * 256)
    s += x[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_final(const double *part, double *out) {
  __shared__ double sh[ADJ_BLOCKS];
  sh[threadIdx.x] = part[threadIdx.x];
  __syncthreads();
  for (int o = ADJ_BLOCKS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// ---------------------------------------------------------------------------
// gradient, WQ rows: transposed contraction on the grid

// Z(k1, i2) = sum over interior rows (i1, i2) whose point range holds k1 of
// W1[i1, k1] * {lambda, u}; the rows holding k1 lie within one element of the
// point's own element's functions
__global__ void k_adj_z(Dir A, Dir B, const uint8_t *fstate, const int32_t *act,
                        const double *u, const double *lam, double *Zu, double *Zl) {
  int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)A.nq * B.n) return;
  int k1 = (int)(id % A.nq), i2 = (int)(id / A.nq);
  int e = A.qel[k1];
  double zu = 0.0, zl = 0.0;
  for (int a = -1; a <= A.p + 1; a++) {
    int i1 = e + a;
    if (i1 < 0 || i1 >= A.n) continue;
    int c = k1 - A.qbeg[i1];
    if (c < 0 || c >= A.qcnt[i1]) continue;
    int g = i2 * A.n + i1;
    if (fstate[g] != TW_FUNC_INTERIOR) continue;
    double w = A.W[(size_t)i1 * A.qmax + c];
    int32_t r = act[g];
    zu += w * u[r];
    zl += w * lam[r];
  }
  Zu[id] = zu;
  Zl[id] = zl;
}

// T(k1, k2) = detJ [(f - U/2) LW - Lambda UW / 2] at each grid point
__global__ void k_adj_t(Dir A, Dir B, Geo G, Func f, const int32_t *act, const double *u,
                        const double *lam, const double *Zu, const double *Zl, double *T) {
  int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)A.nq * B.nq) return;
  int k1 = (int)(id % A.nq), k2 = (int)(id / A.nq);
  const int p = A.p, p1 = p + 1;
  int e = B.qel[k2];
  double uw = 0.0, lw = 0.0;
  for (int b = -1; b <= p + 1; b++) {
    int i2 = e + b;
    if (i2 < 0 || i2 >= B.n) continue;
    int c = k2 - B.qbeg[i2];
    if (c < 0 || c >= B.qcnt[i2]) continue;
    double w = B.W[(size_t)i2 * B.qmax + c];
    uw += w * Zu[(size_t)i2 * A.nq + k1];
    lw += w * Zl[(size_t)i2 * A.nq + k1];
  }
  double t = 0.0;
  if (uw != 0.0 || lw != 0.0) {
    int e1 = A.qel[k1], e2 = B.qel[k2];
    const double *v1 = A.Bq + (size_t)k1 * p1, *d1 = A.dBq + (size_t)k1 * p1;
    const double *v2 = B.Bq + (size_t)k2 * p1, *d2 = B.dBq + (size_t)k2 * p1;
    double x1 = A.xq[k1], x2 = B.xq[k2];
    double dj = detj_of(G, p, e1, v1, d1, e2, v2, d2);
    double X[2], U, Lm;
    phys_of(G, p, x1, x2, e1, v1, e2, v2, X);
    active_pair(act, A.n, p, e1, v1, e2, v2, u, lam, &U, &Lm);
    double fv = func_at(f, x1, x2, X);
    t = dj * ((fv - 0.5 * U) * lw - 0.5 * Lm * uw);
  }
  T[id] = t;
}

// density basis at the WQ points of one direction: span and q+1 values
__global__ void k_dens_basis(const double *x, int nq, const double *V, int q, int m, int *span,
                             double *N) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nq) return;
  int s = find_span(V, q, m, x[k]);
  double v[TW_MAXP1];
  basis_vals(V, s, x[k], q, v);
  span[k] = s;
  for (int a = 0; a <= q; a++) N[(size_t)k * (q + 1) + a] = v[a];
}

// first index in span[0..n) with span >= s (span is non-decreasing)
__device__ __forceinline__ int lower_idx(const int *span, int n, int s) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int m = (lo + hi) >> 1;
    if (span[m] < s) lo = m + 1;
    else hi = m;
  }
  return lo;
}

// Y(m1, k2) = sum_k1 N1_{m1}(x_k1) T(k1, k2) over the points in N1_{m1}'s support
__global__ void k_adj_y(int nq1, int nq2, int m1n, int q1, const int *span1, const double *N1,
                        const double *T, double *Y) {
  int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)m1n * nq2) return;
  int m1 = (int)(id % m1n), k2 = (int)(id / m1n);
  int k0 = lower_idx(span1, nq1, m1), kend = lower_idx(span1, nq1, m1 + q1 + 1);
  const double *Tr = T + (size_t)k2 * nq1;
  double s = 0.0;
  for (int k = k0; k < kend; k++) s += N1[(size_t)k * (q1 + 1) + (m1 - span1[k] + q1)] * Tr[k];
  Y[id] = s;
}

// Gw(m1, m2) = sum_k2 N2_{m2}(x_k2) Y(m1, k2)
__global__ void k_adj_gw(int nq2, int m1n, int m2n, int q2, const int *span2, const double *N2,
                         const double *Y, double *Gw) {
  int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)m1n * m2n) return;
  int m1 = (int)(id % m1n), m2 = (int)(id / m1n);
  int k0 = lower_idx(span2, nq2, m2), kend = lower_idx(span2, nq2, m2 + q2 + 1);
  double s = 0.0;
  for (int k = k0; k < kend; k++)
    s += N2[(size_t)k * (q2 + 1) + (m2 - span2[k] + q2)] * Y[(size_t)k * m1n + m1];
  Gw[id] = s;
}

// ---------------------------------------------------------------------------
// gradient, cut rows

// the density coefficients a row's support can touch: origin and width per
// direction, from the density spans at the support's two ends
__device__ __forceinline__ void row_window(const Geo &G, const Dir &A, const Dir &B, int i1,
                                           int i2, int *o, int *w) {
  const int p = A.p;
  for (int d = 0; d < 2; d++) {
    const Dir &D = d == 0 ? A : B;
    int i = d == 0 ? i1 : i2;
    int q = G.dp[d], m = G.dnk[d] - q - 1;
    int s0 = find_span(G.dU[d], q, m, D.U[i]);
    int s1 = find_span(G.dU[d], q, m, D.U[i + p + 1]);
    o[d] = s0 - q;
    w[d] = s1 - s0 + q + 1;
  }
}

__global__ void k_adj_windows(RowArgs a, const int32_t *rows, int nrows, int2 *org, int *wmax) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  int g = rows[r];
  int o[2], w[2];
  row_window(a.G, a.A, a.B, g % a.A.n, g / a.A.n, o, w);
  org[r] = make_int2(o[0], o[1]);
  atomicMax(wmax, w[0]);
  atomicMax(wmax + 1, w[1]);
}

struct AdjRow {
  const double *u, *lam;
  double ui, li;
  double *win;
  int o1, o2, w1, w2;
  int *flag;
};

// one rule point of a cut row: weight w without c, basis values / derivatives
// of element (e1, e2) at (x1, x2)
__device__ __forceinline__ void adj_point(const RowArgs &a, const Func &f, AdjRow &R, double x1,
                                          double x2, double w, int e1, const double *v1,
                                          const double *d1, int e2, const double *v2,
                                          const double *d2) {
  const Geo &G = a.G;
  const int p = a.A.p;
  double dj = detj_of(G, p, e1, v1, d1, e2, v2, d2);
  double X[2], U, Lm;
  phys_of(G, p, x1, x2, e1, v1, e2, v2, X);
  active_pair(a.act, a.A.n, p, e1, v1, e2, v2, R.u, R.lam, &U, &Lm);
  double fv = func_at(f, x1, x2, X);
  double val = w * dj * (R.li * (fv - 0.5 * U) - 0.5 * R.ui * Lm);
  int q1 = G.dp[0], q2 = G.dp[1];
  int s1 = find_span(G.dU[0], q1, G.dnk[0] - q1 - 1, x1);
  int s2 = find_span(G.dU[1], q2, G.dnk[1] - q2 - 1, x2);
  double N1[TW_MAXP1], N2[TW_MAXP1];
  basis_vals(G.dU[0], s1, x1, q1, N1);
  basis_vals(G.dU[1], s2, x2, q2, N2);
  int c1 = s1 - q1 - R.o1, c2 = s2 - q2 - R.o2;
  if (c1 < 0 || c2 < 0 || c1 + q1 >= R.w1 || c2 + q2 >= R.w2) {
    atomicOr(R.flag, 1);
    return;
  }
  for (int b = 0; b <= q2; b++)
    for (int aa = 0; aa <= q1; aa++) R.win[(c2 + b) * R.w1 + c1 + aa] += val * N1[aa] * N2[b];
}

// one thread per cut row: region rule (WQ / DWQ), element Gauss outside the
// region, cut rule on cut elements -- the rule of the formation kernel
__global__ void k_adj_cut(RowArgs a, Func f, const int32_t *rows, int nrows, const double *u,
                          const double *lam, const int2 *org, int w1, int w2, double *part,
                          int *flag) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const Dir &A = a.A;
  const Dir &B = a.B;
  const int P = A.p, p1 = P + 1;
  int g = rows[r];
  int i1 = g % A.n, i2 = g / A.n;
  AdjRow R;
  R.u = u;
  R.lam = lam;
  R.ui = u[a.act[g]];
  R.li = lam[a.act[g]];
  R.win = part + (size_t)r * w1 * w2;
  R.o1 = org[r].x;
  R.o2 = org[r].y;
  R.w1 = w1;
  R.w2 = w2;
  R.flag = flag;
  for (int k = 0; k < w1 * w2; k++) R.win[k] = 0.0;
  int kind;
  if (a.method == TW_METHOD_GAUSS || a.method == TW_METHOD_HYBRID) kind = 0;
  else if (a.method == TW_METHOD_NAIVE) kind = 1;
  else kind = a.choice[4 * g] >= 0 ? 2 : 0;
  int lo1 = max(0, i1 - P), hi1 = min(A.nel - 1, i1);
  int lo2 = max(0, i2 - P), hi2 = min(B.nel - 1, i2);
  int r0[2] = {1, 1}, r1[2] = {0, 0};
  if (kind != 0) {
    double rx[2][32], rw[2][32];
    int rk[2][32], nr[2];
    for (int d = 0; d < 2; d++) {
      const Dir &D = d == 0 ? A : B;
      int i = d == 0 ? i1 : i2;
      int n = 0;
      int ck = kind == 2 ? a.choice[4 * g + 2 * d] : 0;
      int s = kind == 2 ? a.choice[4 * g + 2 * d + 1] : -1;
      int lo = d == 0 ? lo1 : lo2, hi = d == 0 ? hi1 : hi2;
      r0[d] = ck == 2 ? s : lo;
      r1[d] = ck == 1 ? s - 1 : hi;
      if (ck == 0) {
        for (int c = 0; c < D.qcnt[i] && n < 32; c++) {
          rx[d][n] = D.xq[D.qbeg[i] + c];
          rw[d][n] = D.W[(size_t)i * D.qmax + c];
          rk[d][n] = D.qbeg[i] + c;
          n++;
        }
      } else {
        int side = ck - 1, sl = a.disc_slot[d][s];
        double t = D.bp[s];
        const double *xs = a.dwq_x[d] + (size_t)sl * TW_LQMAX;
        const double *ws = a.dwq_w[d] + (((size_t)sl * P + (i - s)) * 2 + side) * TW_LQMAX;
        for (int k = 0; k < a.dwq_np[d][sl] && n < 32; k++) {
          double x = xs[k];
          if (!(x > D.U[i] && x < D.U[i + P + 1])) continue;
          if (side == 0 ? !(x < t) : !(x > t)) continue;
          rx[d][n] = x;
          rw[d][n] = ws[k];
          rk[d][n] = -1;
          n++;
        }
      }
      nr[d] = n;
    }
    if (kind == 1) {
      r0[0] = r0[1] = 1;
      r1[0] = r1[1] = 0;
    }
    for (int ib = 0; ib < nr[1]; ib++)
      for (int ia = 0; ia < nr[0]; ia++) {
        int k1 = rk[0][ia], k2 = rk[1][ib];
        double x1 = rx[0][ia], x2 = rx[1][ib];
        int e1, e2;
        if (k1 >= 0) e1 = A.qel[k1];
        else e1 = elem_of(A.bp, A.nel, x1);
        if (k2 >= 0) e2 = B.qel[k2];
        else e2 = elem_of(B.bp, B.nel, x2);
        if (kind == 1 && a.estate[e2 * A.nel + e1] != TW_ELEM_REGULAR) continue;
        double v1[TW_MAXP1], d1[TW_MAXP1], v2[TW_MAXP1], d2[TW_MAXP1];
        basis_ders(A.U, e1 + P, x1, P, v1, d1);
        basis_ders(B.U, e2 + P, x2, P, v2, d2);
        adj_point(a, f, R, x1, x2, rw[0][ia] * rw[1][ib], e1, v1, d1, e2, v2, d2);
      }
  }
  for (int e2 = lo2; e2 <= hi2; e2++)
    for (int e1 = lo1; e1 <= hi1; e1++) {
      int e = e2 * A.nel + e1;
      uint8_t st = a.estate[e];
      bool inR = e1 >= r0[0] && e1 <= r1[0] && e2 >= r0[1] && e2 <= r1[1];
      if (st == TW_ELEM_REGULAR && kind != 1 && !inR) {
        double h1 = 0.5 * (A.bp[e1 + 1] - A.bp[e1]), h2 = 0.5 * (B.bp[e2 + 1] - B.bp[e2]);
        for (int g2 = 0; g2 < p1; g2++)
          for (int g1 = 0; g1 < p1; g1++) {
            double v1[TW_MAXP1], d1[TW_MAXP1], v2[TW_MAXP1], d2[TW_MAXP1];
            for (int k = 0; k < p1; k++) {
              v1[k] = A.GB[((size_t)e1 * p1 + g1) * p1 + k];
              d1[k] = A.dGB[((size_t)e1 * p1 + g1) * p1 + k];
              v2[k] = B.GB[((size_t)e2 * p1 + g2) * p1 + k];
              d2[k] = B.dGB[((size_t)e2 * p1 + g2) * p1 + k];
            }
            double x1 = A.bp[e1] + h1 * (A.gx[g1] + 1.0), x2 = B.bp[e2] + h2 * (B.gx[g2] + 1.0);
            double w = A.gw[g1] * h1 * B.gw[g2] * h2 * v1[i1 - e1] * v2[i2 - e2];
            adj_point(a, f, R, x1, x2, w, e1, v1, d1, e2, v2, d2);
          }
      } else if (st == TW_ELEM_CUT) {
        int cs = a.cut_slot[e];
        for (int64_t q = a.cut_off[cs]; q < a.cut_off[cs + 1]; q++) {
          const double *xq = a.cut_pts + 3 * q;
          double v1[TW_MAXP1], d1[TW_MAXP1], v2[TW_MAXP1], d2[TW_MAXP1];
          basis_ders(A.U, e1 + P, xq[0], P, v1, d1);
          basis_ders(B.U, e2 + P, xq[1], P, v2, d2);
          double w = xq[2] * v1[i1 - e1] * v2[i2 - e2];
          adj_point(a, f, R, xq[0], xq[1], w, e1, v1, d1, e2, v2, d2);
        }
      }
    }
}

// one warp per cut row, for windows of at most ADJ_WIN coefficients: the
// lanes share the row's points, each lane sums into its own window, and the
// warp adds the lanes' windows entry by entry in a fixed order
#define ADJ_WIN 64
__global__ void __launch_bounds__(128) k_adj_cut_warp(RowArgs a, Func f, const int32_t *rows,
                                                      int nrows, const double *u,
                                                      const double *lam, const int2 *org, int w1,
                                                      int w2, double *part, int *flag) {
  const int lane = threadIdx.x & 31;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= nrows) return;  // the whole warp
  double win[ADJ_WIN];
  const Dir &A = a.A;
  const Dir &B = a.B;
  const int P = A.p, p1 = P + 1;
  int g = rows[r];
  int i1 = g % A.n, i2 = g / A.n;
  AdjRow R;
  R.u = u;
  R.lam = lam;
  R.ui = u[a.act[g]];
  R.li = lam[a.act[g]];
  R.win = win;
  R.o1 = org[r].x;
  R.o2 = org[r].y;
  R.w1 = w1;
  R.w2 = w2;
  R.flag = flag;
  for (int k = 0; k < w1 * w2; k++) R.win[k] = 0.0;
  int kind;
  if (a.method == TW_METHOD_GAUSS || a.method == TW_METHOD_HYBRID) kind = 0;
  else if (a.method == TW_METHOD_NAIVE) kind = 1;
  else kind = a.choice[4 * g] >= 0 ? 2 : 0;
  int lo1 = max(0, i1 - P), hi1 = min(A.nel - 1, i1);
  int lo2 = max(0, i2 - P), hi2 = min(B.nel - 1, i2);
  int r0[2] = {1, 1}, r1[2] = {0, 0};
  if (kind != 0) {
    double rx[2][32], rw[2][32];
    int rk[2][32], nr[2];
    for (int d = 0; d < 2; d++) {
      const Dir &D = d == 0 ? A : B;
      int i = d == 0 ? i1 : i2;
      int n = 0;
      int ck = kind == 2 ? a.choice[4 * g + 2 * d] : 0;
      int s = kind == 2 ? a.choice[4 * g + 2 * d + 1] : -1;
      int lo = d == 0 ? lo1 : lo2, hi = d == 0 ? hi1 : hi2;
      r0[d] = ck == 2 ? s : lo;
      r1[d] = ck == 1 ? s - 1 : hi;
      if (ck == 0) {
        for (int c = 0; c < D.qcnt[i] && n < 32; c++) {
          rx[d][n] = D.xq[D.qbeg[i] + c];
          rw[d][n] = D.W[(size_t)i * D.qmax + c];
          rk[d][n] = D.qbeg[i] + c;
          n++;
        }
      } else {
        int side = ck - 1, sl = a.disc_slot[d][s];
        double t = D.bp[s];
        const double *xs = a.dwq_x[d] + (size_t)sl * TW_LQMAX;
        const double *ws = a.dwq_w[d] + (((size_t)sl * P + (i - s)) * 2 + side) * TW_LQMAX;
        for (int k = 0; k < a.dwq_np[d][sl] && n < 32; k++) {
          double x = xs[k];
          if (!(x > D.U[i] && x < D.U[i + P + 1])) continue;
          if (side == 0 ? !(x < t) : !(x > t)) continue;
          rx[d][n] = x;
          rw[d][n] = ws[k];
          rk[d][n] = -1;
          n++;
        }
      }
      nr[d] = n;
    }
    if (kind == 1) {
      r0[0] = r0[1] = 1;
      r1[0] = r1[1] = 0;
    }
    for (int t = lane; t < nr[0] * nr[1]; t += 32) {
        const int ia = t % nr[0], ib = t / nr[0];
        int k1 = rk[0][ia], k2 = rk[1][ib];
        double x1 = rx[0][ia], x2 = rx[1][ib];
        int e1, e2;
        if (k1 >= 0) e1 = A.qel[k1];
        else e1 = elem_of(A.bp, A.nel, x1);
        if (k2 >= 0) e2 = B.qel[k2];
        else e2 = elem_of(B.bp, B.nel, x2);
        if (kind == 1 && a.estate[e2 * A.nel + e1] != TW_ELEM_REGULAR) continue;
        double v1[TW_MAXP1], d1[TW_MAXP1], v2[TW_MAXP1], d2[TW_MAXP1];
        basis_ders(A.U, e1 + P, x1, P, v1, d1);
        basis_ders(B.U, e2 + P, x2, P, v2, d2);
        adj_point(a, f, R, x1, x2, rw[0][ia] * rw[1][ib], e1, v1, d1, e2, v2, d2);
      }
  }
  for (int e2 = lo2; e2 <= hi2; e2++)
    for (int e1 = lo1; e1 <= hi1; e1++) {
      int e = e2 * A.nel + e1;
      uint8_t st = a.estate[e];
      bool inR = e1 >= r0[0] && e1 <= r1[0] && e2 >= r0[1] && e2 <= r1[1];
      if (st == TW_ELEM_REGULAR && kind != 1 && !inR) {
        double h1 = 0.5 * (A.bp[e1 + 1] - A.bp[e1]), h2 = 0.5 * (B.bp[e2 + 1] - B.bp[e2]);
        for (int t = lane; t < p1 * p1; t += 32) {
            const int g1 = t % p1, g2 = t / p1;
            double v1[TW_MAXP1], d1[TW_MAXP1], v2[TW_MAXP1], d2[TW_MAXP1];
            for (int k = 0; k < p1; k++) {
              v1[k] = A.GB[((size_t)e1 * p1 + g1) * p1 + k];
              d1[k] = A.dGB[((size_t)e1 * p1 + g1) * p1 + k];
              v2[k] = B.GB[((size_t)e2 * p1 + g2) * p1 + k];
              d2[k] = B.dGB[((size_t)e2 * p1 + g2) * p1 + k];
            }
            double x1 = A.bp[e1] + h1 * (A.gx[g1] + 1.0), x2 = B.bp[e2] + h2 * (B.gx[g2] + 1.0);
            double w = A.gw[g1] * h1 * B.gw[g2] * h2 * v1[i1 - e1] * v2[i2 - e2];
            adj_point(a, f, R, x1, x2, w, e1, v1, d1, e2, v2, d2);
          }
      } else if (st == TW_ELEM_CUT) {
        int cs = a.cut_slot[e];
        for (int64_t q = a.cut_off[cs] + lane; q < a.cut_off[cs + 1]; q += 32) {
          const double *xq = a.cut_pts + 3 * q;
          double v1[TW_MAXP1], d1[TW_MAXP1], v2[TW_MAXP1], d2[TW_MAXP1];
          basis_ders(A.U, e1 + P, xq[0], P, v1, d1);
          basis_ders(B.U, e2 + P, xq[1], P, v2, d2);
          double w = xq[2] * v1[i1 - e1] * v2[i2 - e2];
          adj_point(a, f, R, xq[0], xq[1], w, e1, v1, d1, e2, v2, d2);
        }
      }
    }
  double *out = part + (size_t)r * w1 * w2;
  for (int k = 0; k < w1 * w2; k++) {
    double v = warp_sum(win[k]);
    if (lane == 0) out[k] = v;
  }
}

// grad(m1, m2) = WQ part + the cut rows' windows that hold (m1, m2), row order
__global__ void k_adj_final(int m1n, int m2n, const double *Gw, int nrows, const int2 *org, int w1,
                            int w2, const double *part, double *grad) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= m1n * m2n) return;
  int m1 = id % m1n, m2 = id / m1n;
  double s = Gw ? Gw[id] : 0.0;
  for (int r = 0; r < nrows; r++) {
    int2 o = org[r];
    int c1 = m1 - o.x, c2 = m2 - o.y;
    if (c1 >= 0 && c1 < w1 && c2 >= 0 && c2 < w2) s += part[((size_t)r * w2 + c2) * w1 + c1];
  }
  grad[id] = s;
}

// ---------------------------------------------------------------------------
// host side

static int loss_impl(tw_patch *P, const tw_func *g, const double *u, double *loss, double *dLdu,
                     cudaStream_t s) {
  int rc = 0;
  Func F = make_func(g, P, &rc);
  if (rc) return rc;
  Dir &A = P->d[0];
  Dir &B = P->d[1];
  const int p1 = P->p + 1;
  int64_t ne = (int64_t)A.nel * B.nel;
  double *lossE = (double *)dalloc(P, sizeof(double) * (ne + ADJ_BLOCKS));
  double *loc = (double *)dalloc(P, sizeof(double) * ne * p1 * p1);
  if (!lossE || !loc) return TW_ENOMEM;
  double *part = lossE + ne;
  k_loss_elems<<<(unsigned)((ne + 127) / 128), 128, 0, s>>>(A, B, P->geo, F, P->estate,
                                                            P->cut_slot, P->cut_off, P->cut_pts,
                                                            P->act, u, lossE, loc);
  TW_LAUNCH();
  if (P->n_rows > 0) {
    k_dldu<<<(unsigned)((P->n_rows + 255) / 256), 256, 0, s>>>(A, B, P->rowg, P->n_rows, loc,
                                                               dLdu);
    TW_LAUNCH();
  }
  k_sum_partial<<<ADJ_BLOCKS, 256, 0, s>>>(lossE, ne, part);
  TW_LAUNCH();
  k_sum_final<<<1, ADJ_BLOCKS, 0, s>>>(part, loss);
  TW_LAUNCH();
  return check_cuda(cudaGetLastError(), "tw_loss");
}

int loss_run(tw_patch *P, const tw_func *g, const double *u, double *loss, double *dLdu,
             cudaStream_t s) {
  cudaStream_t keep = P->stream;
  P->stream = s;
  int mark = P->nallocs;
  int ps = prof_start(s);
  int rc = loss_impl(P, g, u, loss, dLdu, s);
  prof_stop(ps, TW_STAGE_LOSS, s);
  release_to(P, mark);
  P->stream = keep;
  return rc;
}

static int grad_impl(tw_patch *P, const tw_func *f, const double *u, const double *lam,
                     double *grad, cudaStream_t s) {
  int rc = 0;
  Func F = make_func(f, P, &rc);
  if (rc) return rc;
  Dir &A = P->d[0];
  Dir &B = P->d[1];
  const Geo &G = P->geo;
  const int m1n = G.dnk[0] - G.dp[0] - 1, m2n = G.dnk[1] - G.dp[1] - 1;
  const int nm = m1n * m2n;
  double *Gw = nullptr;
  if (P->method != TW_METHOD_GAUSS && P->n_interior > 0) {
    int64_t nz = (int64_t)A.nq * B.n, ng = (int64_t)A.nq * B.nq;
    int64_t ny = (int64_t)m1n * B.nq;
    double *buf = (double *)dalloc(P, sizeof(double) * (2 * nz + ng + ny + nm));
    double *N1 = (double *)dalloc(P, sizeof(double) * ((size_t)A.nq * (G.dp[0] + 1) +
                                                       (size_t)B.nq * (G.dp[1] + 1)));
    int *sp = (int *)dalloc(P, sizeof(int) * (A.nq + B.nq));
    if (!buf || !N1 || !sp) return TW_ENOMEM;
    double *Zu = buf, *Zl = Zu + nz, *T = Zl + nz, *Y = T + ng;
    Gw = Y + ny;
    double *N2 = N1 + (size_t)A.nq * (G.dp[0] + 1);
    int *sp1 = sp, *sp2 = sp + A.nq;
    k_adj_z<<<(unsigned)((nz + 255) / 256), 256, 0, s>>>(A, B, P->fstate, P->act, u, lam, Zu, Zl);
    TW_LAUNCH();
    k_adj_t<<<(unsigned)((ng + 127) / 128), 128, 0, s>>>(A, B, P->geo, F, P->act, u, lam, Zu, Zl,
                                                         T);
    TW_LAUNCH();
    k_dens_basis<<<(A.nq + 255) / 256, 256, 0, s>>>(A.xq, A.nq, G.dU[0], G.dp[0], m1n, sp1, N1);
    TW_LAUNCH();
    k_dens_basis<<<(B.nq + 255) / 256, 256, 0, s>>>(B.xq, B.nq, G.dU[1], G.dp[1], m2n, sp2, N2);
    TW_LAUNCH();
    k_adj_y<<<(unsigned)((ny + 255) / 256), 256, 0, s>>>(A.nq, B.nq, m1n, G.dp[0], sp1, N1, T, Y);
    TW_LAUNCH();
    k_adj_gw<<<(nm + 255) / 256, 256, 0, s>>>(B.nq, m1n, m2n, G.dp[1], sp2, N2, Y, Gw);
    TW_LAUNCH();
  }
  int nc = P->ncutrows;
  int2 *org = nullptr;
  double *part = nullptr;
  int w[2] = {0, 0};
  int *dflag = nullptr;
  RowArgs ra = row_args(P);
  if (nc > 0) {
    org = (int2 *)dalloc(P, sizeof(int2) * nc);
    dflag = (int *)dalloc(P, sizeof(int) * 4);
    if (!org || !dflag) return TW_ENOMEM;
    cudaMemsetAsync(dflag, 0, sizeof(int) * 4, s);
    k_adj_windows<<<(nc + 127) / 128, 128, 0, s>>>(ra, P->cutrows, nc, org, dflag + 1);
    TW_LAUNCH();
    cudaMemcpyAsync(w, dflag + 1, sizeof(w), cudaMemcpyDeviceToHost, s);
    if ((rc = check_cuda(cudaStreamSynchronize(s), "tw_l2_project_adjoint: windows"))) return rc;
    if (w[0] <= 0 || w[1] <= 0 || (int64_t)w[0] * w[1] > (int64_t)1 << 20) {
      set_error("tw_l2_project_adjoint: density window %d x %d out of range", w[0], w[1]);
      return TW_EUNSUPPORTED;
    }
    part = (double *)dalloc(P, sizeof(double) * (size_t)nc * w[0] * w[1]);
    if (!part) return TW_ENOMEM;
    if (w[0] * w[1] <= ADJ_WIN)
      k_adj_cut_warp<<<(nc + 3) / 4, 128, 0, s>>>(ra, F, P->cutrows, nc, u, lam, org, w[0], w[1],
                                                 part, dflag);
    else
      k_adj_cut<<<(nc + 63) / 64, 64, 0, s>>>(ra, F, P->cutrows, nc, u, lam, org, w[0], w[1],
                                              part, dflag);
    TW_LAUNCH();
  }
  k_adj_final<<<(nm + 255) / 256, 256, 0, s>>>(m1n, m2n, Gw, nc, org, w[0], w[1], part, grad);
  TW_LAUNCH();
  if ((rc = check_cuda(cudaGetLastError(), "tw_l2_project_adjoint"))) return rc;
  if (dflag) {
    int hf = 0;
    cudaMemcpyAsync(&hf, dflag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if ((rc = check_cuda(cudaStreamSynchronize(s), "tw_l2_project_adjoint"))) return rc;
    if (hf) {
      set_error("tw_l2_project_adjoint: a rule point fell outside its row's density window");
      return TW_ECUDA;
    }
  }
  return 0;
}

int adjoint_run(tw_patch *P, const tw_func *f, const int64_t *rp, const int32_t *col,
                const double *val, const double *dLdu, const double *u, double *lam,
                double *grad, double tol, int maxit, int *iters, double *relres, cudaStream_t s) {
  cudaStream_t keep = P->stream;
  P->stream = s;
  int mark = P->nallocs;
  int ps = prof_start(s);
  int rc = cg_solve(P, rp, col, val, dLdu, lam, tol, maxit, iters, relres, s);
  prof_stop(ps, TW_STAGE_CG, s);
  if (rc == 0) {
    ps = prof_start(s);
    rc = grad_impl(P, f, u, lam, grad, s);
    prof_stop(ps, TW_STAGE_ADJOINT, s);
  }
  release_to(P, mark);
  P->stream = keep;
  return rc;
}

// the gradient stage alone (lam given), for the extended projection's adjoint
int adjoint_grad(tw_patch *P, const tw_func *f, const double *u, const double *lam, double *grad,
                 cudaStream_t s) {
  int ps = prof_start(s);
  int rc = grad_impl(P, f, u, lam, grad, s);
  prof_stop(ps, TW_STAGE_ADJOINT, s);
  return rc;
}

}  // namespace tw
