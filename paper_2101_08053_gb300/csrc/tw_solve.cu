// tw_solve.cu -- L2 projection with the formed matrix (Sect. 4.2).
//   rhs   b_i = the row's own quadrature rule applied to f * c (reading R9):
//         interior rows  sum_{k1,k2} W1[i1,k1] W2[i2,k2] c f  (WQ, test function in W)
//         cut rows       region rule + element Gauss + cut-element rule, as in formation
//   CG    Jacobi-preconditioned CG on M_s = (M + M^T)/2 (reading R10); M^T is read
//         through a permutation of the symmetric pattern, dot products reduce in a
//         fixed order so the iteration is bitwise reproducible.
#include <cmath>
#include <cstring>
#include <mutex>

#include "tw_func.cuh"

namespace tw {

// f * c on the WQ grid
__global__ void k_fc_grid(Func f, Geo G, Dir A, Dir B, const double *C, double *FC) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= A.nq * B.nq) return;
  int k1 = id % A.nq, k2 = id / A.nq;
  FC[id] = C[id] * fpoint(f, G, A, B, A.xq[k1], B.xq[k2]);
}

__global__ void k_rhs_interior(Dir A, Dir B, const uint8_t *fstate, const int32_t *act,
                               const double *FC, double *b) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= A.n * B.n || fstate[g] != TW_FUNC_INTERIOR) return;
  int i1 = g % A.n, i2 = g / A.n;
  double s = 0.0;
  for (int c2 = 0; c2 < B.qcnt[i2]; c2++) {
    int k2 = B.qbeg[i2] + c2;
    double t = 0.0;
    for (int c1 = 0; c1 < A.qcnt[i1]; c1++)
      t += A.W[(size_t)i1 * A.qmax + c1] * FC[(size_t)k2 * A.nq + A.qbeg[i1] + c1];
    s += B.W[(size_t)i2 * B.qmax + c2] * t;
  }
  b[act[g]] = s;
}

// The region part of a cut row's rule (DWQ region, or the masked WQ rule of a
// naive row): the 1-D points rx, weights rw and base WQ indices rk (-1 for a
// DWQ window point) per direction, and the element range r0..r1 the region
// covers.  kind: 0 Gauss rows (no region), 1 naive, 2 DWQ with a region.
struct RegionRule {
  double rx[2][32], rw[2][32];
  int rk[2][32], nr[2];
  int r0[2], r1[2];
};

__device__ __forceinline__ int cut_row_kind(const RowArgs &a, int g) {
  if (a.method == TW_METHOD_GAUSS || a.method == TW_METHOD_HYBRID) return 0;
  if (a.method == TW_METHOD_NAIVE) return 1;
  return a.choice[4 * g] >= 0 ? 2 : 0;
}

__device__ void region_rule(const RowArgs &a, int g, int kind, RegionRule &R) {
  const Dir &A = a.A;
  const Dir &B = a.B;
  const int P = A.p;
  const int i1 = g % A.n, i2 = g / A.n;
  const int lo1 = max(0, i1 - P), hi1 = min(A.nel - 1, i1);
  const int lo2 = max(0, i2 - P), hi2 = min(B.nel - 1, i2);
  R.r0[0] = R.r0[1] = 1;
  R.r1[0] = R.r1[1] = 0;
  R.nr[0] = R.nr[1] = 0;
  if (kind == 0) return;
  for (int d = 0; d < 2; d++) {
    const Dir &D = d == 0 ? A : B;
    int i = d == 0 ? i1 : i2;
    int n = 0;
    int ck = kind == 2 ? a.choice[4 * g + 2 * d] : 0;
    int s = kind == 2 ? a.choice[4 * g + 2 * d + 1] : -1;
    int lo = d == 0 ? lo1 : lo2, hi = d == 0 ? hi1 : hi2;
    R.r0[d] = ck == 2 ? s : lo;
    R.r1[d] = ck == 1 ? s - 1 : hi;
    if (ck == 0) {
      for (int c = 0; c < D.qcnt[i] && n < 32; c++) {
        R.rx[d][n] = D.xq[D.qbeg[i] + c];
        R.rw[d][n] = D.W[(size_t)i * D.qmax + c];
        R.rk[d][n] = D.qbeg[i] + c;
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
        R.rx[d][n] = x;
        R.rw[d][n] = ws[k];
        R.rk[d][n] = -1;
        n++;
      }
    }
    R.nr[d] = n;
  }
  if (kind == 1) {  // region unused for element exclusion: naive uses no Gauss
    R.r0[0] = R.r0[1] = 1;
    R.r1[0] = R.r1[1] = 0;
  }
}

// one warp per cut row: the same three parts as k_cutrows, applied to f; the
// lanes share the row's points and the warp adds their sums in a fixed order.
// VALUES: f is read at the listed rule points (tw_rhs_values) instead of being
// evaluated; the index of each point follows the list of tw_rhs_points.
template <bool VALUES>
__global__ void __launch_bounds__(128) k_rhs_cut(RowArgs a, Func f, PtIndex pi,
                                                 const int32_t *rows, int nrows, const double *FC,
                                                 double *b) {
  const int lane = threadIdx.x & 31;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= nrows) return;  // the whole warp
  const Dir &A = a.A;
  const Dir &B = a.B;
  const int P = A.p, p1 = P + 1;
  int g = rows[r];
  int i1 = g % A.n, i2 = g / A.n;
  const int kind = cut_row_kind(a, g);
  int lo1 = max(0, i1 - P), hi1 = min(A.nel - 1, i1);
  int lo2 = max(0, i2 - P), hi2 = min(B.nel - 1, i2);
  RegionRule R;
  region_rule(a, g, kind, R);
  double sum = 0.0;
  if (kind != 0) {
    for (int t = lane; t < R.nr[0] * R.nr[1]; t += 32) {
      const int ia = t % R.nr[0], ib = t / R.nr[0];
      int k1 = R.rk[0][ia], k2 = R.rk[1][ib];
      double v;
      if (k1 >= 0 && k2 >= 0) {
        v = FC[(size_t)k2 * A.nq + k1];
        if (kind == 1 && a.estate[B.qel[k2] * A.nel + A.qel[k1]] != TW_ELEM_REGULAR) v = 0.0;
      } else {
        const double fv = VALUES ? pi.FV[pi.dbase + pi.roff[r] + t]
                                 : fpoint(f, a.G, A, B, R.rx[0][ia], R.rx[1][ib]);
        v = coef_at(a.G, A, B, R.rx[0][ia], R.rx[1][ib]) * fv;
      }
      sum += R.rw[0][ia] * R.rw[1][ib] * v;
    }
  }
  for (int e2 = lo2; e2 <= hi2; e2++)
    for (int e1 = lo1; e1 <= hi1; e1++) {
      int e = e2 * A.nel + e1;
      uint8_t st = a.estate[e];
      bool inR = e1 >= R.r0[0] && e1 <= R.r1[0] && e2 >= R.r0[1] && e2 <= R.r1[1];
      if (st == TW_ELEM_REGULAR && kind != 1 && !inR) {
        const double *cgp = a.gc + (size_t)a.gslot[e] * p1 * p1;
        double h1 = 0.5 * (A.bp[e1 + 1] - A.bp[e1]), h2 = 0.5 * (B.bp[e2 + 1] - B.bp[e2]);
        for (int t = lane; t < p1 * p1; t += 32) {
          const int g1 = t % p1, g2 = t / p1;
          double x1 = A.bp[e1] + h1 * (A.gx[g1] + 1.0), x2 = B.bp[e2] + h2 * (B.gx[g2] + 1.0);
          double w = A.gw[g1] * h1 * B.gw[g2] * h2 * A.GB[(e1 * p1 + g1) * p1 + (i1 - e1)] *
                     B.GB[(e2 * p1 + g2) * p1 + (i2 - e2)];
          const double fv = VALUES ? pi.FV[pi.gbase + (int64_t)a.gslot[e] * p1 * p1 + t]
                                   : fpoint(f, a.G, A, B, x1, x2);
          sum += w * cgp[g2 * p1 + g1] * fv;
        }
      } else if (st == TW_ELEM_CUT) {
        int cs = a.cut_slot[e];
        for (int64_t q = a.cut_off[cs] + lane; q < a.cut_off[cs + 1]; q += 32) {
          const double *Bv = a.cut_B + 2 * q * p1;
          const double *xq = a.cut_pts + 3 * q;
          const double fv = VALUES ? pi.FV[pi.cbase + q] : fpoint(f, a.G, A, B, xq[0], xq[1]);
          sum += a.cut_wc[q] * Bv[i1 - e1] * Bv[p1 + (i2 - e2)] * fv;
        }
      }
    }
  sum = warp_sum(sum);
  if (lane == 0) b[a.act[g]] = sum;
}

// ---------------------------------------------------------------------------
// CG on (M + M^T)/2

__global__ void k_perm(const int64_t *rp, const int32_t *col, int64_t n, int64_t *perm) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  for (int64_t k = rp[r]; k < rp[r + 1]; k++) {
    int32_t j = col[k];
    int64_t lo = rp[j], hi = rp[j + 1] - 1, pos = -1;
    while (lo <= hi) {
      int64_t m = (lo + hi) >> 1;
      if (col[m] == r) { pos = m; break; }
      if (col[m] < r) lo = m + 1;
      else hi = m - 1;
    }
    perm[k] = pos;
  }
}

__global__ void k_msym(const int64_t *rp, const int32_t *col, const double *val,
                       const int64_t *perm, int64_t n, double *ms, double *dinv) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double dg = 0.0;
  for (int64_t k = rp[r]; k < rp[r + 1]; k++) {
    double v = perm[k] >= 0 ? 0.5 * (val[k] + val[perm[k]]) : val[k];
    ms[k] = v;
    if (col[k] == r) dg = v;
  }
  dinv[r] = dg != 0.0 ? 1.0 / dg : 1.0;
}

// One CG iteration = 3 launches, each with a full grid (a warp per row for
// the product, a thread per entry for the updates):
//   k_cg_spmv     q = M_s p, p.q
//   k_cg_update1  alpha = rz / pq; u += alpha p; r -= alpha q; z = D^-1 r; r.z, r.r
//   k_cg_update2  beta = rz_new / rz; p = z + beta p
// Each block writes one partial sum; the block that takes the last ticket of
// a counter sums all partials in index order (a fixed tree inside the block)
// and writes the scalar, so every scalar is bitwise reproducible.  The r.z
// scalar is double-buffered by iteration parity.
#define CG_THREADS 256

enum { SC_PQ = 0, SC_RZ0 = 1, SC_RR0 = 3, SC_BB = 5, SC_N = 6 };

// block sum, fixed order (xor tree in the warp, then warp order); all threads
// get the result; sh has 9 doubles
__device__ __forceinline__ double block_sum(double v, double *sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();  // sh may still be read from a previous call
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < CG_THREADS / 32; k++) t += sh[k];
    sh[8] = t;
  }
  __syncthreads();
  return sh[8];
}

// publish this block's partial v of scalar `slot`; the last block to arrive
// reduces all partials in order into sc[slot] and rearms the ticket
__device__ __forceinline__ void reduce_scalar(double v, double *part, unsigned *ticket,
                                              double *sc, int slot, double *sh) {
  __shared__ int last;
  __syncthreads();  // every thread has read `last` of a previous call
  if (threadIdx.x == 0) {
    part[blockIdx.x] = v;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
#pragma unroll 4
  for (unsigned k = threadIdx.x; k < gridDim.x; k += CG_THREADS) t += __ldcg(part + k);
  t = block_sum(t, sh);
  if (threadIdx.x == 0) {
    sc[slot] = t;
    *ticket = 0u;
  }
}

__global__ void __launch_bounds__(CG_THREADS) k_cg_init(const double *b, const double *dinv,
                                                        double *u, double *r, double *z,
                                                        double *p, int64_t n, double *part,
                                                        unsigned *ticket, double *sc) {
  __shared__ double sh[9];
  int64_t i = (int64_t)blockIdx.x * CG_THREADS + threadIdx.x;
  double rz = 0.0, bb = 0.0;
  if (i < n) {
    double bi = b[i], zi = bi * dinv[i];
    u[i] = 0.0;
    r[i] = bi;
    z[i] = zi;
    p[i] = zi;
    rz = bi * zi;
    bb = bi * bi;
  }
  rz = block_sum(rz, sh);
  bb = block_sum(bb, sh);
  // r.z of "iteration -1" goes to the odd slot
  reduce_scalar(rz, part, ticket, sc, SC_RZ0 + 1, sh);
  reduce_scalar(bb, part + gridDim.x, ticket + 1, sc, SC_BB, sh);
}

// CG_LPR lanes per row (fixed shuffle tree); measured on GB300 for the banded
// (2p+1)^2 rows of these matrices, 4 lanes per row keep ~3x more loads in
// flight than a warp per row
#define CG_LPR 4
__global__ void __launch_bounds__(CG_THREADS) k_cg_spmv(const int64_t *rp, const int32_t *col,
                                                        const double *ms, const double *p,
                                                        double *q, int64_t n, double *part,
                                                        unsigned *ticket, double *sc) {
  __shared__ double sh[9];
  const int sub = threadIdx.x & (CG_LPR - 1);
  const int64_t r = ((int64_t)blockIdx.x * CG_THREADS + threadIdx.x) / CG_LPR;
  double s = 0.0, pq = 0.0;
  if (r < n) {
    const int64_t k0 = rp[r], k1 = rp[r + 1];
#pragma unroll 4
    for (int64_t k = k0 + sub; k < k1; k += CG_LPR) s += ms[k] * __ldg(p + col[k]);
  }
  for (int o = CG_LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (r < n && sub == 0) {
    q[r] = s;
    pq = p[r] * s;
  }
  pq = block_sum(pq, sh);
  reduce_scalar(pq, part, ticket, sc, SC_PQ, sh);
}

__global__ void __launch_bounds__(CG_THREADS) k_cg_update1(const double *p, const double *q,
                                                           const double *dinv, double *u,
                                                           double *r, double *z, int64_t n,
                                                           int cur, double *part,
                                                           unsigned *ticket, double *sc) {
  __shared__ double sh[9];
  const double alpha = sc[SC_RZ0 + (cur ^ 1)] / sc[SC_PQ];
  int64_t i = (int64_t)blockIdx.x * CG_THREADS + threadIdx.x;
  double rz = 0.0, rr = 0.0;
  if (i < n) {
    u[i] += alpha * p[i];
    double ri = r[i] - alpha * q[i];
    double zi = ri * dinv[i];
    r[i] = ri;
    z[i] = zi;
    rz = ri * zi;
    rr = ri * ri;
  }
  rz = block_sum(rz, sh);
  rr = block_sum(rr, sh);
  reduce_scalar(rz, part, ticket, sc, SC_RZ0 + cur, sh);
  reduce_scalar(rr, part + gridDim.x, ticket + 1, sc, SC_RR0 + cur, sh);
}

__global__ void __launch_bounds__(CG_THREADS) k_cg_update2(const double *z, double *p, int64_t n,
                                                           int cur, const double *sc) {
  const double beta = sc[SC_RZ0 + cur] / sc[SC_RZ0 + (cur ^ 1)];
  int64_t i = (int64_t)blockIdx.x * CG_THREADS + threadIdx.x;
  if (i < n) p[i] = z[i] + beta * p[i];
}

RowArgs row_args(tw_patch *Pt) {
  RowArgs ra;
  ra.A = Pt->d[0];
  ra.B = Pt->d[1];
  ra.G = Pt->geo;
  ra.estate = Pt->estate;
  ra.fstate = Pt->fstate;
  ra.act = Pt->act;
  ra.rp = Pt->row_ptr;
  ra.C = Pt->C;
  ra.gslot = Pt->gslot;
  ra.gc = Pt->gc;
  ra.cut_slot = Pt->cut_slot;
  ra.cut_off = Pt->cut_off;
  ra.cut_B = Pt->cut_B;
  ra.cut_wc = Pt->cut_wc;
  ra.cut_pts = Pt->cut_pts;
  ra.cut_M = Pt->cut_M;
  ra.choice = Pt->choice;
  for (int d = 0; d < 2; d++) {
    ra.disc_slot[d] = Pt->disc_slot[d];
    ra.dwq_x[d] = Pt->dwq_x[d];
    ra.dwq_np[d] = Pt->dwq_np[d];
    ra.dwq_w[d] = Pt->dwq_w[d];
    ra.dwq_k[d] = Pt->dwq_k[d];
    ra.dwq_e[d] = Pt->dwq_e[d];
    ra.dwq_B[d] = Pt->dwq_B[d];
    ra.dwq_dB[d] = Pt->dwq_dB[d];
    ra.dwq_r[d] = Pt->dwq_r[d];
  }
  ra.gmat = Pt->gmat;
  ra.method = Pt->method;
  ra.flag = Pt->flag;
  return ra;
}

static int rhs_impl(tw_patch *P, const tw_func *f, double *b, cudaStream_t s) {
  int rc = 0;
  Func F = make_func(f, P, &rc);
  if (rc) return rc;
  Dir &A = P->d[0];
  Dir &B = P->d[1];
  int64_t ng = (int64_t)A.nq * B.nq;
  double *FC = (double *)dalloc(P, sizeof(double) * ng);
  if (!FC) return TW_ENOMEM;
  k_fc_grid<<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(F, P->geo, A, B, P->C, FC);
  TW_LAUNCH();
  if (P->method != TW_METHOD_GAUSS) {
    int64_t nf = (int64_t)A.n * B.n;
    k_rhs_interior<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(A, B, P->fstate, P->act, FC, b);
    TW_LAUNCH();
  }
  if (P->ncutrows > 0) {
    k_rhs_cut<false><<<(P->ncutrows + 3) / 4, 128, 0, s>>>(row_args(P), F, PtIndex{}, P->cutrows,
                                                            P->ncutrows, FC, b);
    TW_LAUNCH();
  }
  return check_cuda(cudaGetLastError(), "tw_rhs");
}

// temporary allocations are made on `s` and released in stream order
int rhs_launch(tw_patch *P, const tw_func *f, double *b, cudaStream_t s) {
  cudaStream_t keep = P->stream;
  P->stream = s;
  int mark = P->nallocs;
  int ps = prof_start(s);
  int rc = rhs_impl(P, f, b, s);
  prof_stop(ps, TW_STAGE_RHS, s);
  release_to(P, mark);
  P->stream = keep;
  return rc;
}

// ---------------------------------------------------------------------------
// Rule points of the right-hand side for an f given by values (tw_rhs_points,
// tw_rhs_values).  The list: the WQ grid (k2 * nq1 + k1), the element Gauss
// points of the Gauss slots (slot, then g2, g1), the cut-rule points, the DWQ
// region points of each cut row (row, then ib, ia as k_rhs_cut walks them).
// Every point is formed by the same expression the rhs kernels use, so a value
// listed for it is the value tw_rhs would have evaluated there.

__device__ __forceinline__ void put_point(const RowArgs &a, int64_t k, double x1, double x2,
                                          double *xi, double *X) {
  if (xi) {
    xi[2 * k] = x1;
    xi[2 * k + 1] = x2;
  }
  if (X) {
    double Q[2];
    phys_at(a.G, a.A, a.B, x1, x2, Q);
    X[2 * k] = Q[0];
    X[2 * k + 1] = Q[1];
  }
}

// number of DWQ region points of each cut row; cnt[nrows] = 0 (for the scan)
__global__ void k_pts_count(RowArgs a, const int32_t *rows, int nrows, int64_t *cnt) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r > nrows) return;
  if (r == nrows) {
    cnt[r] = 0;
    return;
  }
  const int g = rows[r];
  const int kind = cut_row_kind(a, g);
  if (kind != 2) {
    cnt[r] = 0;
    return;
  }
  RegionRule R;
  region_rule(a, g, kind, R);
  cnt[r] = (int64_t)R.nr[0] * R.nr[1];
}

__global__ void k_pts_grid(RowArgs a, double *xi, double *X) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)a.A.nq * a.B.nq) return;
  const int k1 = (int)(id % a.A.nq), k2 = (int)(id / a.A.nq);
  put_point(a, id, a.A.xq[k1], a.B.xq[k2], xi, X);
}

// thread per (element, Gauss point); elements without a Gauss slot write nothing
__global__ void k_pts_gauss(RowArgs a, int64_t base, double *xi, double *X) {
  const Dir &A = a.A;
  const Dir &B = a.B;
  const int p1 = A.p + 1;
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)A.nel * B.nel * p1 * p1) return;
  const int e = (int)(id / (p1 * p1)), t = (int)(id % (p1 * p1));
  const int sl = a.gslot[e];
  if (sl < 0) return;
  const int e1 = e % A.nel, e2 = e / A.nel, g1 = t % p1, g2 = t / p1;
  const double h1 = 0.5 * (A.bp[e1 + 1] - A.bp[e1]), h2 = 0.5 * (B.bp[e2 + 1] - B.bp[e2]);
  const double x1 = A.bp[e1] + h1 * (A.gx[g1] + 1.0), x2 = B.bp[e2] + h2 * (B.gx[g2] + 1.0);
  put_point(a, base + (int64_t)sl * p1 * p1 + t, x1, x2, xi, X);
}

__global__ void k_pts_cut(RowArgs a, int64_t base, int64_t npts, double *xi, double *X) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= npts) return;
  put_point(a, base + q, a.cut_pts[3 * q], a.cut_pts[3 * q + 1], xi, X);
}

// one warp per cut row
__global__ void __launch_bounds__(128) k_pts_dwq(RowArgs a, const int32_t *rows, int nrows,
                                                 const int64_t *roff, int64_t base, double *xi,
                                                 double *X) {
  const int lane = threadIdx.x & 31;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= nrows) return;
  const int g = rows[r];
  const int kind = cut_row_kind(a, g);
  if (kind != 2) return;
  RegionRule R;
  region_rule(a, g, kind, R);
  for (int t = lane; t < R.nr[0] * R.nr[1]; t += 32) {
    const int ia = t % R.nr[0], ib = t / R.nr[0];
    put_point(a, base + roff[r] + t, R.rx[0][ia], R.rx[1][ib], xi, X);
  }
}

__global__ void k_fc_values(const double *C, const double *FV, double *FC, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) FC[i] = C[i] * FV[i];
}

// per-row offsets of the DWQ region points (patch-owned, built on first use)
static int ensure_point_index(tw_patch *P, cudaStream_t s) {
  if (P->pt_roff) return 0;
  const int64_t n = (int64_t)P->ncutrows + 1;
  int64_t *buf = (int64_t *)dalloc(P, sizeof(int64_t) * (2 * n + 1));
  if (!buf) return TW_ENOMEM;
  int64_t *cnt = buf, *roff = buf + n, *tot = buf + 2 * n;
  k_pts_count<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(row_args(P), P->cutrows, P->ncutrows,
                                                          cnt);
  TW_LAUNCH();
  int rc = exclusive_scan_i64(cnt, roff, n, tot, s, P);
  if (rc) return rc;
  P->pt_roff = roff;
  P->pt_dtot = tot;
  P->pt_total = -1;
  return check_cuda(cudaGetLastError(), "rhs point index");
}

static PtIndex point_index(const tw_patch *P, const double *FV) {
  const int64_t p1 = P->p + 1;
  PtIndex pi;
  pi.FV = FV;
  pi.roff = P->pt_roff;
  pi.gbase = (int64_t)P->d[0].nq * P->d[1].nq;
  pi.cbase = pi.gbase + (int64_t)P->ngslot * p1 * p1;
  pi.dbase = pi.cbase + P->ncutpts;
  return pi;
}

int rhs_points_run(tw_patch *P, int64_t *npts, double *xi, double *X, cudaStream_t s) {
  cudaStream_t keep = P->stream;
  P->stream = s;
  int rc = ensure_point_index(P, s);
  if (!rc && P->pt_total < 0) {
    int64_t h = 0;
    rc = check_cuda(cudaMemcpyAsync(&h, P->pt_dtot, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
                    "tw_rhs_points: count");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(s), "tw_rhs_points: count");
    if (!rc) P->pt_total = point_index(P, nullptr).dbase + h;
  }
  P->stream = keep;
  if (rc) return rc;
  *npts = P->pt_total;
  if (!xi && !X) return 0;
  const PtIndex pi = point_index(P, nullptr);
  const RowArgs ra = row_args(P);
  const int64_t ng = pi.gbase;
  const int64_t p1 = P->p + 1;
  const int64_t ngp = (int64_t)P->d[0].nel * P->d[1].nel * p1 * p1;
  k_pts_grid<<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(ra, xi, X);
  TW_LAUNCH();
  if (P->ngslot > 0) {
    k_pts_gauss<<<(unsigned)((ngp + 255) / 256), 256, 0, s>>>(ra, pi.gbase, xi, X);
    TW_LAUNCH();
  }
  if (P->ncutpts > 0) {
    k_pts_cut<<<(unsigned)((P->ncutpts + 255) / 256), 256, 0, s>>>(ra, pi.cbase, P->ncutpts, xi,
                                                                  X);
    TW_LAUNCH();
  }
  if (P->ncutrows > 0 && P->method == TW_METHOD_DWQ) {
    k_pts_dwq<<<(P->ncutrows + 3) / 4, 128, 0, s>>>(ra, P->cutrows, P->ncutrows, P->pt_roff,
                                                    pi.dbase, xi, X);
    TW_LAUNCH();
  }
  return check_cuda(cudaGetLastError(), "tw_rhs_points");
}

int rhs_values_run(tw_patch *P, const double *FV, double *b, cudaStream_t s) {
  cudaStream_t keep = P->stream;
  P->stream = s;
  int rc = ensure_point_index(P, s);
  int mark = P->nallocs;
  int ps = prof_start(s);
  Dir &A = P->d[0];
  Dir &B = P->d[1];
  const int64_t ng = (int64_t)A.nq * B.nq;
  double *FC = rc ? nullptr : (double *)dalloc(P, sizeof(double) * ng);
  if (!rc && !FC) rc = TW_ENOMEM;
  if (!rc) {
    k_fc_values<<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(P->C, FV, FC, ng);
    TW_LAUNCH();
    if (P->method != TW_METHOD_GAUSS) {
      const int64_t nf = (int64_t)A.n * B.n;
      k_rhs_interior<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(A, B, P->fstate, P->act, FC, b);
      TW_LAUNCH();
    }
    if (P->ncutrows > 0) {
      Func F;
      memset(&F, 0, sizeof(F));
      k_rhs_cut<true><<<(P->ncutrows + 3) / 4, 128, 0, s>>>(row_args(P), F, point_index(P, FV),
                                                            P->cutrows, P->ncutrows, FC, b);
      TW_LAUNCH();
    }
    rc = check_cuda(cudaGetLastError(), "tw_rhs_values");
  }
  prof_stop(ps, TW_STAGE_RHS, s);
  release_to(P, mark);
  P->stream = keep;
  return rc;
}

struct CgBufs {
  const int64_t *rp;
  const int32_t *col;
  const double *ms, *dinv;
  double *u, *r, *z, *p, *q;
  double *part, *sc;
  unsigned *ticket;
  int64_t n;
};

// iteration `it` of the three-launch CG step
static void cg_iteration(const CgBufs &B, int it, cudaStream_t s) {
  const int cur = it & 1;
  const unsigned gw = (unsigned)((B.n * CG_LPR + CG_THREADS - 1) / CG_THREADS);
  const unsigned ge = (unsigned)((B.n + CG_THREADS - 1) / CG_THREADS);
  k_cg_spmv<<<gw, CG_THREADS, 0, s>>>(B.rp, B.col, B.ms, B.p, B.q, B.n, B.part, B.ticket, B.sc);
  k_cg_update1<<<ge, CG_THREADS, 0, s>>>(B.p, B.q, B.dinv, B.u, B.r, B.z, B.n, cur, B.part,
                                         B.ticket, B.sc);
  k_cg_update2<<<ge, CG_THREADS, 0, s>>>(B.z, B.p, B.n, cur, B.sc);
}

// CG on M_s x = b for a device b (n_rows); x is overwritten.  Iterations run in
// chunks of CG_CHUNK replayed from a CUDA graph (captured once per call on a
// private stream, launched on s); the residual is read back after each chunk.
#define CG_CHUNK 8
static int cg_core(tw_patch *P, int64_t n, int64_t nnz, const int64_t *rp, const int32_t *col,
                   const double *val, const double *b, double *u, double tol, int maxit,
                   int *iters, double *relres, cudaStream_t s) {
  if (n == 0) {
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return TW_OK;
  }
  const int64_t gw = (n * CG_LPR + CG_THREADS - 1) / CG_THREADS;  // the largest grid
  double *buf = (double *)dalloc(P, sizeof(double) * (5 * n + 2 * gw + SC_N));
  int64_t *perm = (int64_t *)dalloc(P, sizeof(int64_t) * (nnz + 1));
  double *ms = (double *)dalloc(P, sizeof(double) * (nnz + 1));
  unsigned *ticket = (unsigned *)dalloc(P, sizeof(unsigned) * 2);
  if (!buf || !perm || !ms || !ticket) return TW_ENOMEM;
  CgBufs B;
  B.rp = rp;
  B.col = col;
  B.ms = ms;
  B.n = n;
  B.u = u;
  B.r = buf;
  B.z = B.r + n;
  B.p = B.z + n;
  B.q = B.p + n;
  double *dinv = B.q + n;
  B.dinv = dinv;
  B.part = dinv + n;
  B.sc = B.part + 2 * gw;
  B.ticket = ticket;
  int rc = 0;
  cudaMemsetAsync(ticket, 0, sizeof(unsigned) * 2, s);
  unsigned gb = (unsigned)((n + 255) / 256);
  k_perm<<<gb, 256, 0, s>>>(rp, col, n, perm);
  TW_LAUNCH();
  k_msym<<<gb, 256, 0, s>>>(rp, col, val, perm, n, ms, dinv);
  TW_LAUNCH();
  k_cg_init<<<(unsigned)((n + CG_THREADS - 1) / CG_THREADS), CG_THREADS, 0, s>>>(
      b, dinv, u, B.r, B.z, B.p, n, B.part, ticket, B.sc);
  TW_LAUNCH();
  double hs[SC_N];
  cudaMemcpyAsync(hs, B.sc, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if ((rc = check_cuda(cudaStreamSynchronize(s), "tw_l2_project"))) return rc;
  double bn = sqrt(hs[SC_BB]);
  double rel = bn > 0 ? 1.0 : 0.0;
  int it = 0;
  cudaGraphExec_t exec = nullptr;
  if (rel > tol && maxit >= CG_CHUNK) {
    // capture CG_CHUNK iterations starting at an even index (the parity
    // pattern of the scalars repeats every two iterations)
    cudaStream_t cap;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
      e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        for (int k = 0; k < CG_CHUNK; k++) cg_iteration(B, k, cap);
        e = cudaStreamEndCapture(cap, &graph);
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      cudaStreamDestroy(cap);
    }
    if ((rc = check_cuda(e, "tw_l2_project: CG graph"))) return rc;
  }
  while (rel > tol && it < maxit) {
    int nstep = maxit - it < CG_CHUNK ? maxit - it : CG_CHUNK;
    if (nstep == CG_CHUNK && exec && (it & 1) == 0) {
      rc = check_cuda(cudaGraphLaunch(exec, s), "tw_l2_project: CG chunk");
      g_launches += 3 * CG_CHUNK;
    } else {
      for (int k = 0; k < nstep; k++) {
        cg_iteration(B, it + k, s);
        g_launches += 3;
      }
    }
    if (rc) break;
    it += nstep;
    cudaMemcpyAsync(hs, B.sc, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if ((rc = check_cuda(cudaStreamSynchronize(s), "tw_l2_project"))) break;
    rel = bn > 0 ? sqrt(hs[SC_RR0 + ((it - 1) & 1)]) / bn : 0.0;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (rc) return rc;
  if (iters) *iters = it;
  if (relres) *relres = rel;
  if (rel > tol) {
    set_error("tw_l2_project: CG stopped at relative residual %.3e after %d iterations", rel, it);
    return TW_ENOCONV;
  }
  return TW_OK;
}

static int cg_impl(tw_patch *P, const tw_func *f, const int64_t *rp, const int32_t *col,
                   const double *val, double *u, double tol, int maxit, int *iters,
                   double *relres, cudaStream_t s) {
  double *b = (double *)dalloc(P, sizeof(double) * (P->n_rows + 1));
  if (!b) return TW_ENOMEM;
  int rc = rhs_impl(P, f, b, s);
  if (rc) return rc;
  return cg_core(P, P->n_rows, P->nnz, rp, col, val, b, u, tol, maxit, iters, relres, s);
}

int cg_solve(tw_patch *P, const int64_t *rp, const int32_t *col, const double *val,
             const double *b, double *x, double tol, int maxit, int *iters, double *relres,
             cudaStream_t s) {
  return cg_solve_n(P, P->n_rows, P->nnz, rp, col, val, b, x, tol, maxit, iters, relres, s);
}

int cg_solve_n(tw_patch *P, int64_t n, int64_t nnz, const int64_t *rp, const int32_t *col,
               const double *val, const double *b, double *x, double tol, int maxit, int *iters,
               double *relres, cudaStream_t s) {
  int mark = P->nallocs;
  int rc = cg_core(P, n, nnz, rp, col, val, b, x, tol, maxit, iters, relres, s);
  release_to(P, mark);
  return rc;
}

int l2_project_run(tw_patch *P, const tw_func *f, const int64_t *rp, const int32_t *col,
                   const double *val, double *u, double tol, int maxit, int *iters,
                   double *relres, cudaStream_t s) {
  cudaStream_t keep = P->stream;
  P->stream = s;
  int mark = P->nallocs;
  int ps = prof_start(s);
  int rc = cg_impl(P, f, rp, col, val, u, tol, maxit, iters, relres, s);
  prof_stop(ps, TW_STAGE_CG, s);
  release_to(P, mark);
  P->stream = keep;
  return rc;
}

}  // namespace tw

// ---------------------------------------------------------------------------
// tw_rhs_static: the right-hand side without any device allocation, for
// callers that cannot allocate device memory (see include/trimwq.h).  Its
// scratch is this file-scope array; host code never uses the array's name as an
// address, it asks the runtime for the device address once per device.
static __device__ __align__(256) double g_rhs_static_scratch[TW_RHS_STATIC_MAX];

namespace tw {

#define TW_STATIC_MAX_DEVICES 64
static std::mutex g_static_mu;
static double *g_static_addr[TW_STATIC_MAX_DEVICES];

// device address of the scratch array on the current device (looked up on the
// first call for that device)
static int static_scratch(double **out) {
  int dev = -1;
  if (check_cuda(cudaGetDevice(&dev), "tw_rhs_static: cudaGetDevice")) return TW_ECUDA;
  if (dev < 0 || dev >= TW_STATIC_MAX_DEVICES) {
    set_error("tw_rhs_static: device %d beyond %d", dev, TW_STATIC_MAX_DEVICES);
    return TW_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_rhs_static_scratch);
    if (e != cudaSuccess || !p) {
      set_error("tw_rhs_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return TW_ECUDA;
    }
    g_static_addr[dev] = (double *)p;
  }
  *out = g_static_addr[dev];
  return 0;
}

}  // namespace tw

extern "C" int tw_rhs_static(tw_patch *P, const tw_func *f, double *b, void *stream) {
  using namespace tw;
  if (!P || !f || !b) {
    set_error("tw_rhs_static: NULL argument");
    return TW_EINVAL;
  }
  if (f->kind < TW_FUNC_SPLINE || f->kind > TW_FUNC_GAUSS) {
    set_error("tw_rhs_static: unknown function kind %d", f->kind);
    return TW_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Dir &A = P->d[0];
  Dir &B = P->d[1];
  const int64_t ng = (int64_t)A.nq * B.nq;
  int64_t need = ng;
  int64_t m[2] = {0, 0};
  if (f->kind == TW_FUNC_SPLINE) {
    for (int d = 0; d < 2; d++) {
      if (!f->knots[d] || f->p[d] < 0 || f->p[d] > TW_MAXP || f->nknots[d] < 2 * f->p[d] + 2) {
        set_error("tw_rhs_static: spline function: bad knots or degree");
        return TW_EINVAL;
      }
      m[d] = f->nknots[d] - f->p[d] - 1;
      need += f->nknots[d];
    }
    if (!f->coef) {
      set_error("tw_rhs_static: spline function without coefficients");
      return TW_EINVAL;
    }
    need += m[0] * m[1];
  }
  if (need > TW_RHS_STATIC_MAX) {
    set_error("tw_rhs_static: needs %lld doubles of scratch, the static array holds %d",
              (long long)need, TW_RHS_STATIC_MAX);
    return TW_EINVAL;
  }
  double *scr = nullptr;
  int rc = static_scratch(&scr);
  if (rc) return rc;
  Func F;
  memset(&F, 0, sizeof(F));
  F.kind = f->kind;
  for (int k = 0; k < 4; k++) F.prm[k] = f->prm[k];
  if (f->kind == TW_FUNC_SPLINE) {
    double *dst = scr + ng;
    for (int d = 0; d < 2; d++) {
      F.q[d] = f->p[d];
      F.nk[d] = f->nknots[d];
      if (check_cuda(cudaMemcpyAsync(dst, f->knots[d], sizeof(double) * f->nknots[d],
                                     cudaMemcpyHostToDevice, s),
                     "tw_rhs_static: knots"))
        return TW_ECUDA;
      F.U[d] = dst;
      dst += f->nknots[d];
    }
    F.m1 = (int)m[0];
    if (check_cuda(cudaMemcpyAsync(dst, f->coef, sizeof(double) * m[0] * m[1],
                                   cudaMemcpyHostToDevice, s),
                   "tw_rhs_static: coefficients"))
      return TW_ECUDA;
    F.coef = dst;
  }
  k_fc_grid<<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(F, P->geo, A, B, P->C, scr);
  TW_LAUNCH();
  if (P->method != TW_METHOD_GAUSS) {
    int64_t nf = (int64_t)A.n * B.n;
    k_rhs_interior<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(A, B, P->fstate, P->act, scr, b);
    TW_LAUNCH();
  }
  if (P->ncutrows > 0) {
    k_rhs_cut<false><<<(P->ncutrows + 3) / 4, 128, 0, s>>>(row_args(P), F, PtIndex{},
                                                            P->cutrows, P->ncutrows, scr, b);
    TW_LAUNCH();
  }
  return check_cuda(cudaGetLastError(), "tw_rhs_static");
}
