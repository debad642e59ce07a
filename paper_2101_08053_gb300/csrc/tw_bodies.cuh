// tw_bodies.cuh -- the per-item bodies of the formation kernels, shared by the
// one-patch kernels (tw_form.cu, tw_form32.cu) and the persistent batched
// kernel (tw_batch.cu).  Each body is run by a whole 256-thread block and takes
// its shared memory as a carved buffer, so a persistent block can run items of
// any degree and kind one after the other.
#pragma once

#include <type_traits>

#include "tw_bulk.cuh"
#include "tw_interior.cuh"

namespace tw {

#define TW_RC 32

template <int P>
struct CutSmem {
  static constexpr int W = 2 * P + 1, P1 = P + 1;
  double acc[W * W];
  double rx[2][TW_RC], rb[2][TW_RC][W];  // rb: weight x basis value
  double cg[TW_RC * TW_RC];
  double Z[W * TW_RC];
  double Tg[P1 * P1];
  int rk[2][TW_RC];
  int rq[2][TW_RC];  // DWQ table index of each region point (-1: a WQ rule point)
  int nr[2], nnest[2], nest[2][TW_RC];
  double pv[2][TW_RC][P1], pd[2][TW_RC][P1];  // basis values / derivatives at the region points
  int pe[2][TW_RC];                            // and their elements
  // spline geometry: control net contracted over a nested point's direction,
  // [nested point][control row / column - (i - P)][x', y' along 1; x, y]
  double T0[P][W][4], T1[P][W][4];
  const double *eM[P1 * P1];  // per support element: its matrix row of this test function
  int jact[W * W];            // active index of each row entry (-1: none)
  unsigned msk[8];            // ballots of the active entries, one per 32 entries
};

// a cut row with no region part (hybrid Gauss, or DWQ without a region) whose
// element matrices are all precomputed: a plain gather of element rows
__device__ __forceinline__ bool cutrow_is_gather(const RowArgs &a, int g) {
  if (!a.gmat || a.method == TW_METHOD_NAIVE) return false;
  return a.method != TW_METHOD_DWQ || a.choice[4 * g] < 0;
}

// One warp per such row, no block barrier: lanes hold the support elements'
// matrix rows of this test function in the warp's table `tab`, then own the
// row entries (lane, lane + 32, ...) and add their elements' terms in (e2, e1)
// order -- the same sums, in the same order, as cutrow_item.
template <int P, typename OutT>
__device__ __forceinline__ void cutrow_gather_warp(const RowArgs &a, int g, int lane,
                                                   const double **tab,
                                                   int32_t *__restrict__ col,
                                                   OutT *__restrict__ val) {
  constexpr int W = 2 * P + 1, P1 = P + 1, P2 = P1 * P1, NE = (W * W + 31) / 32;
  const Dir &A = a.A;
  const Dir &B = a.B;
  const int n1 = A.n;
  const int i1 = g % n1, i2 = g / n1;
  const int lo1 = max(0, i1 - P), hi1 = min(A.nel - 1, i1);
  const int lo2 = max(0, i2 - P), hi2 = min(B.nel - 1, i2);
  for (int t = lane; t < P2; t += 32) {
    const int e1 = i1 - P + t % P1, e2 = i2 - P + t / P1;
    const double *Me = nullptr;
    if (e1 >= lo1 && e1 <= hi1 && e2 >= lo2 && e2 <= hi2) {
      const int e = e2 * A.nel + e1;
      const uint8_t st = a.estate[e];
      const size_t rowoff = (size_t)((i2 - e2) * P1 + (i1 - e1)) * P2;
      if (st == TW_ELEM_REGULAR) Me = a.gmat + (size_t)a.gslot[e] * P2 * P2 + rowoff;
      else if (st == TW_ELEM_CUT) Me = a.cut_M + (size_t)a.cut_slot[e] * P2 * P2 + rowoff;
    }
    tab[t] = Me;
  }
  __syncwarp();
  const int64_t base = a.rp[a.act[g]];
  int before = 0;  // active entries in the previous chunks of 32
#pragma unroll
  for (int k = 0; k < NE; k++) {
    const int t = k * 32 + lane;
    int jact = -1;
    double s = 0.0;
    if (t < W * W) {
      const int q2 = t / W, q1 = t % W;
      const int j1 = i1 - P + q1, j2 = i2 - P + q2;
      if (j1 >= 0 && j1 < n1 && j2 >= 0 && j2 < B.n) jact = a.act[j2 * n1 + j1];
#pragma unroll
      for (int u2 = 0; u2 <= P; u2++) {
        if (u2 < q2 - P || u2 > q2) continue;
#pragma unroll
        for (int u1 = 0; u1 <= P; u1++) {
          if (u1 < q1 - P || u1 > q1) continue;
          const double *Me = tab[u2 * P1 + u1];
          if (Me) s += Me[(q2 - u2) * P1 + (q1 - u1)];
        }
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, jact >= 0);
    if (jact >= 0) {
      const int ps = before + __popc(m & ((1u << lane) - 1u));
      val[base + ps] = (OutT)s;
      col[base + ps] = jact;
    }
    before += __popc(m);
  }
  __syncwarp();  // tab reused by the warp's next row
}

template <int P, typename OutT>
__device__ void cutrow_item(const RowArgs &a, int g, int32_t *__restrict__ col,
                            OutT *__restrict__ val, char *smem) {
  constexpr int W = 2 * P + 1, P1 = P + 1;
  CutSmem<P> &S = *reinterpret_cast<CutSmem<P> *>(smem);
  const Dir &A = a.A;
  const Dir &B = a.B;
  // (g: the row's function index)
  const int n1 = A.n;
  const int i1 = g % n1, i2 = g / n1;
  const int tid = threadIdx.x;
  int kind;  // 0: element Gauss on S^r, 1: naive WQ, 2: DWQ region + Gauss rest
  if (a.method == TW_METHOD_GAUSS || a.method == TW_METHOD_HYBRID) kind = 0;
  else if (a.method == TW_METHOD_NAIVE) kind = 1;
  else kind = a.choice[4 * g] >= 0 ? 2 : 0;
  int ch[4] = {-1, -1, -1, -1};
  if (kind == 2)
    for (int k = 0; k < 4; k++) ch[k] = a.choice[4 * g + k];
  const int lo1 = max(0, i1 - P), hi1 = min(A.nel - 1, i1);
  const int lo2 = max(0, i2 - P), hi2 = min(B.nel - 1, i2);
  int r0[2] = {1, 1}, r1[2] = {0, 0};  // region R in elements (empty unless DWQ)
  if (kind == 2) {
    int lo[2] = {lo1, lo2}, hi[2] = {hi1, hi2};
    for (int d = 0; d < 2; d++) {
      int k = ch[2 * d], s = ch[2 * d + 1];
      r0[d] = k == 2 ? s : lo[d];
      r1[d] = k == 1 ? s - 1 : hi[d];
    }
  }
  for (int t = tid; t < W * W; t += blockDim.x) S.acc[t] = 0.0;

  // ---- region part: naive WQ (full support, c masked) or DWQ rectangle ----
  // warp d assembles direction d's rule, one lane per point, from the tables
  if (kind != 0) {
    const int wd = tid >> 5, lane = tid & 31;
    if (wd < 2) {
      const int d = wd;
      const Dir &D = d == 0 ? A : B;
      const int i = d == 0 ? i1 : i2;
      int n;
      if (kind == 1 || ch[2 * d] == 0) {
        n = D.qcnt[i];
        if (lane < n) {
          const int k = D.qbeg[i] + lane;
          S.rx[d][lane] = D.xq[k];
          const double wk = D.W[(size_t)i * D.qmax + lane];
          S.rk[d][lane] = k;
          S.rq[d][lane] = -1;
          for (int r = 0; r < W; r++) {
            int aa = i - P + r - D.qel[k];
            S.rb[d][lane][r] = wk * ((aa >= 0 && aa <= P) ? D.Bq[k * P1 + aa] : 0.0);
          }
        }
      } else {
        const int s = ch[2 * d + 1], side = ch[2 * d] - 1;
        const int sl = a.disc_slot[d][s];
        const int run = a.dwq_r[d][((size_t)sl * P + (i - s)) * 2 + side];
        const int k0 = run & 0xffff, k1 = run >> 16;
        n = k1 - k0;
        if (n > TW_RC) {
          if (lane == 0) atomicOr(a.flag, TWF_RULECAP);
          n = 0;
        }
        if (lane < n) {
          const size_t k = (size_t)sl * TW_LQMAX + k0 + lane;
          S.rx[d][lane] = a.dwq_x[d][k];
          const double wk =
              a.dwq_w[d][(((size_t)sl * P + (i - s)) * 2 + side) * TW_LQMAX + k0 + lane];
          S.rk[d][lane] = a.dwq_k[d][k];  // base points read c from the grid
          S.rq[d][lane] = (int)k;
          const int e = a.dwq_e[d][k];
          const double *Bv = a.dwq_B[d] + k * P1;
          for (int r = 0; r < W; r++) {
            int aa = i - P + r - e;
            S.rb[d][lane][r] = wk * ((aa >= 0 && aa <= P) ? Bv[aa] : 0.0);
          }
        }
      }
      if (lane == 0) S.nr[d] = n;
    }
    __syncthreads();
    const int m1 = S.nr[0], m2 = S.nr[1];
    // c at the tensor points: grid pairs first, then the pairs with a nested
    // point packed densely so only a few warps evaluate c directly
    for (int t = tid; t < m1 * m2; t += blockDim.x) {
      int ia = t % m1, ib = t / m1;
      int k1 = S.rk[0][ia], k2 = S.rk[1][ib];
      if (k1 >= 0 && k2 >= 0) {
        double c = a.C[(size_t)k2 * A.nq + k1];
        if (kind == 1 && a.estate[B.qel[k2] * A.nel + A.qel[k1]] != TW_ELEM_REGULAR) c = 0.0;
        S.cg[ia * TW_RC + ib] = c;
      }
    }
    // basis values and derivatives at every region point, once per row: from
    // the WQ tables at base points, from the DWQ rule's tables at nested points
    const bool unit_c = a.G.coef_kind == TW_COEF_ONE;
    for (int t = tid; t < m1 + m2 && !unit_c; t += blockDim.x) {
      const int d = t < m1 ? 0 : 1, j = d == 0 ? t : t - m1;
      const Dir &D = d == 0 ? A : B;
      const int k = S.rk[d][j];
      if (k >= 0) {
        S.pe[d][j] = D.qel[k];
        for (int q = 0; q <= P; q++) {
          S.pv[d][j][q] = D.Bq[(size_t)k * P1 + q];
          S.pd[d][j][q] = D.dBq[(size_t)k * P1 + q];
        }
      } else {  // a nested point exists only in a DWQ rule
        const int q = S.rq[d][j];
        S.pe[d][j] = a.dwq_e[d][q];
        for (int qq = 0; qq <= P; qq++) {
          S.pv[d][j][qq] = a.dwq_B[d][(size_t)q * P1 + qq];
          S.pd[d][j][qq] = a.dwq_dB[d][(size_t)q * P1 + qq];
        }
      }
    }
    if (tid == 0) {
      int na = 0, nb = 0;
      for (int ia = 0; ia < m1; ia++)
        if (S.rk[0][ia] < 0) S.nest[0][na++] = ia;
      for (int ib = 0; ib < m2; ib++)
        if (S.rk[1][ib] < 0) S.nest[1][nb++] = ib;
      S.nnest[0] = na;
      S.nnest[1] = nb;
    }
    __syncthreads();
    {
      const int na = S.nnest[0], nb = S.nnest[1];
      const int tot = na * m2 + (m1 - na) * nb;
      // spline geometry: J at (nested x1, any x2) from the net contracted over
      // direction 0 at x1 (4 (p+1) terms per pair instead of 4 (p+1)^2; the
      // same sums in the same order as coef_from), and at (base x1, nested
      // x2) from the net contracted over direction 1 at x2
      const bool fact = !unit_c && a.G.geom_kind == TW_GEOM_SPLINE && na <= P && nb <= P;
      if (fact) {
        const int n2 = B.n;
        for (int t = tid; t < (na + nb) * W; t += blockDim.x) {
          const int n = t / W, rr = t % W;
          const bool d0 = n < na;
          const int ix = d0 ? S.nest[0][n] : S.nest[1][n - na];
          double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
          if (d0) {
            const int R = i2 - P + rr, e1 = S.pe[0][ix];
            if (R >= 0 && R < n2)
              for (int aa = 0; aa <= P; aa++) {
                const double *pt = a.G.ctrl + 2 * ((size_t)R * a.G.n1 + (e1 + aa));
                s0 += pt[0] * S.pd[0][ix][aa];
                s1 += pt[1] * S.pd[0][ix][aa];
                s2 += pt[0] * S.pv[0][ix][aa];
                s3 += pt[1] * S.pv[0][ix][aa];
              }
            double *T = S.T0[n][rr];
            T[0] = s0;
            T[1] = s1;
            T[2] = s2;
            T[3] = s3;
          } else {
            const int Cc = i1 - P + rr, e2 = S.pe[1][ix];
            if (Cc >= 0 && Cc < n1)
              for (int b = 0; b <= P; b++) {
                const double *pt = a.G.ctrl + 2 * ((size_t)(e2 + b) * a.G.n1 + Cc);
                s0 += pt[0] * S.pv[1][ix][b];
                s1 += pt[1] * S.pv[1][ix][b];
                s2 += pt[0] * S.pd[1][ix][b];
                s3 += pt[1] * S.pd[1][ix][b];
              }
            double *T = S.T1[n - na][rr];
            T[0] = s0;
            T[1] = s1;
            T[2] = s2;
            T[3] = s3;
          }
        }
        __syncthreads();
      }
      for (int t = tid; t < tot; t += blockDim.x) {
        int ia, ib;
        if (t < na * m2) {
          ia = S.nest[0][t / m2];
          ib = t % m2;
        } else {
          int u = t - na * m2;
          ib = S.nest[1][u % nb];
          // the (u / nb)-th base point of direction 0
          int want = u / nb, cntb = -1;
          ia = 0;
          for (int q = 0; q < m1; q++)
            if (S.rk[0][q] >= 0 && ++cntb == want) {
              ia = q;
              break;
            }
        }
        double c;
        if (unit_c) {
          c = 1.0;
        } else if (fact) {
          double xa = 0, ya = 0, xb = 0, yb = 0;
          if (t < na * m2) {
            // rows e2 + b of the net, contracted over direction 0 at x1
            const double(*T)[4] = S.T0[t / m2] + (S.pe[1][ib] - (i2 - P));
            for (int b = 0; b <= P; b++) {
              xa += T[b][0] * S.pv[1][ib][b];
              ya += T[b][1] * S.pv[1][ib][b];
              xb += T[b][2] * S.pd[1][ib][b];
              yb += T[b][3] * S.pd[1][ib][b];
            }
          } else {
            // columns e1 + a, contracted over direction 1 at x2
            const double(*T)[4] = S.T1[(t - na * m2) % nb] + (S.pe[0][ia] - (i1 - P));
            for (int aa = 0; aa <= P; aa++) {
              xa += T[aa][0] * S.pd[0][ia][aa];
              ya += T[aa][1] * S.pd[0][ia][aa];
              xb += T[aa][2] * S.pv[0][ia][aa];
              yb += T[aa][3] * S.pv[0][ia][aa];
            }
          }
          c = xa * yb - xb * ya;
          if (a.G.coef_kind == TW_COEF_DENSITY) c *= density_at(a.G, S.rx[0][ia], S.rx[1][ib]);
        } else {
          c = coef_from(a.G, P, S.rx[0][ia], S.rx[1][ib], S.pe[0][ia], S.pv[0][ia], S.pd[0][ia],
                        S.pe[1][ib], S.pv[1][ib], S.pd[1][ib]);
        }
        S.cg[ia * TW_RC + ib] = c;
      }
    }
    __syncthreads();
    for (int t = tid; t < W * m1; t += blockDim.x) {
      int r2 = t / m1, ia = t % m1;
      double s = 0.0;
      for (int ib = 0; ib < m2; ib++) s = fma(S.rb[1][ib][r2], S.cg[ia * TW_RC + ib], s);
      S.Z[r2 * TW_RC + ia] = s;
    }
    __syncthreads();
    for (int t = tid; t < W * W; t += blockDim.x) {
      int r2 = t / W, q1 = t % W;
      double s = 0.0;
      for (int ia = 0; ia < m1; ia++) s = fma(S.rb[0][ia][q1], S.Z[r2 * TW_RC + ia], s);
      S.acc[t] += s;
    }
    __syncthreads();
  } else {
    __syncthreads();
  }

  // ---- elements of the support: Gauss on regular (outside R), cut rule on cut ----
  const int p1 = P1;
  if (a.gmat || kind == 1) {
    // every element matrix is precomputed.  First the support elements' rows
    // of this test function (one thread per element), then one owner thread
    // per row entry adds its elements' terms in (e2, e1) order: independent
    // loads, no barrier per element
    constexpr int P2 = P1 * P1;
    for (int t = tid; t < P2; t += blockDim.x) {
      const int e1 = i1 - P + t % P1, e2 = i2 - P + t / P1;
      const double *Me = nullptr;
      if (e1 >= lo1 && e1 <= hi1 && e2 >= lo2 && e2 <= hi2) {
        const int e = e2 * A.nel + e1;
        const uint8_t st = a.estate[e];
        const bool inR = e1 >= r0[0] && e1 <= r1[0] && e2 >= r0[1] && e2 <= r1[1];
        const size_t rowoff = (size_t)((i2 - e2) * P1 + (i1 - e1)) * P2;
        if (st == TW_ELEM_REGULAR && kind != 1 && !inR)
          Me = a.gmat + (size_t)a.gslot[e] * P2 * P2 + rowoff;
        else if (st == TW_ELEM_CUT)
          Me = a.cut_M + (size_t)a.cut_slot[e] * P2 * P2 + rowoff;
      }
      S.eM[t] = Me;
    }
    __syncthreads();
    for (int t = tid; t < W * W; t += blockDim.x) {
      const int q2 = t / W, q1 = t % W;
      double s = S.acc[t];
      // support element u (offset from i - P) covers entry q iff u <= q <= u + P
#pragma unroll
      for (int u2 = 0; u2 <= P; u2++) {
        if (u2 < q2 - P || u2 > q2) continue;
#pragma unroll
        for (int u1 = 0; u1 <= P; u1++) {
          if (u1 < q1 - P || u1 > q1) continue;
          const double *Me = S.eM[u2 * P1 + u1];
          if (Me) s += Me[(q2 - u2) * P1 + (q1 - u1)];
        }
      }
      S.acc[t] = s;
    }
    __syncthreads();
  } else
  for (int e2 = lo2; e2 <= hi2; e2++)
    for (int e1 = lo1; e1 <= hi1; e1++) {
      const int e = e2 * A.nel + e1;
      const uint8_t st = a.estate[e];
      const bool inR = e1 >= r0[0] && e1 <= r1[0] && e2 >= r0[1] && e2 <= r1[1];
      if (st == TW_ELEM_REGULAR && kind != 1 && !inR && a.gmat) {
        // the regular element's matrix, formed once per element
        const double *Me = a.gmat + ((size_t)a.gslot[e] * p1 * p1 + (i2 - e2) * p1 + (i1 - e1)) * p1 * p1;
        if (tid < p1 * p1) {
          int b1 = tid % p1, b2 = tid / p1;
          S.acc[(e2 + b2 - i2 + P) * W + (e1 + b1 - i1 + P)] += Me[b2 * p1 + b1];
        }
        __syncthreads();
      } else if (st == TW_ELEM_REGULAR && kind != 1 && !inR) {
        const double *cgp = a.gc + (size_t)a.gslot[e] * p1 * p1;
        const double h1 = 0.5 * (A.bp[e1 + 1] - A.bp[e1]), h2 = 0.5 * (B.bp[e2 + 1] - B.bp[e2]);
        const double *GB1 = A.GB + (size_t)e1 * p1 * p1;
        const double *GB2 = B.GB + (size_t)e2 * p1 * p1;
        if (tid < p1 * p1) {
          int b1 = tid % p1, g2 = tid / p1;
          double s = 0.0;
          for (int g1 = 0; g1 < p1; g1++)
            s = fma(A.gw[g1] * h1 * GB1[g1 * p1 + (i1 - e1)] * GB1[g1 * p1 + b1], cgp[g2 * p1 + g1], s);
          S.Tg[g2 * p1 + b1] = s;
        }
        __syncthreads();
        if (tid < p1 * p1) {
          int b1 = tid % p1, b2 = tid / p1;
          double s = 0.0;
          for (int g2 = 0; g2 < p1; g2++)
            s = fma(S.Tg[g2 * p1 + b1], B.gw[g2] * h2 * GB2[g2 * p1 + (i2 - e2)] * GB2[g2 * p1 + b2], s);
          S.acc[(e2 + b2 - i2 + P) * W + (e1 + b1 - i1 + P)] += s;
        }
        __syncthreads();
      } else if (st == TW_ELEM_CUT) {
        // the cut element's matrix, formed once per element
        const int cs = a.cut_slot[e];
        const double *Me = a.cut_M + ((size_t)cs * p1 * p1 + (i2 - e2) * p1 + (i1 - e1)) * p1 * p1;
        if (tid < p1 * p1) {
          int b1 = tid % p1, b2 = tid / p1;
          S.acc[(e2 + b2 - i2 + P) * W + (e1 + b1 - i1 + P)] += Me[b2 * p1 + b1];
        }
        __syncthreads();
      }
    }

  // ---- write the row: active columns in ascending order (R11) ----
  // an entry's position = active entries before it, from one ballot per 32
  // entries (blockDim is a multiple of 32, so a warp's lanes share a ballot)
  constexpr int NW = (W * W + 31) / 32;
  static_assert(NW <= 8, "row entries exceed eight ballots");
  const int lane = tid & 31;
  for (int t = tid; t < NW * 32; t += blockDim.x) {
    int jact = -1;
    if (t < W * W) {
      const int r2 = t / W, q1 = t % W;
      const int j1 = i1 - P + q1, j2 = i2 - P + r2;
      if (j1 >= 0 && j1 < n1 && j2 >= 0 && j2 < B.n) jact = a.act[j2 * n1 + j1];
      S.jact[t] = jact;
    }
    const unsigned m = __ballot_sync(0xffffffffu, jact >= 0);
    if (lane == 0) S.msk[t >> 5] = m;
  }
  __syncthreads();
  const int64_t base = a.rp[a.act[g]];
  for (int t = tid; t < W * W; t += blockDim.x) {
    const int jact = S.jact[t];
    if (jact < 0) continue;
    const int w = t >> 5;
    int ps = __popc(S.msk[w] & ((1u << (t & 31)) - 1u));
    for (int k = 0; k < w; k++) ps += __popc(S.msk[k]);
    val[base + ps] = (OutT)S.acc[t];
    col[base + ps] = jact;
  }
  __syncthreads();  // smem reused by the next item
}

// One interior row whose band holds inactive neighbours (possible only with a
// repeated knot, where j may share just the empty span with B_i): the active
// entries in ascending column order, positions from one ballot per 32
// entries.  src is the row's [r2][r1] block; called by a whole warp.
template <int P, typename OutT>
__device__ __forceinline__ void band_write_compact(const OutT *src, const int32_t *__restrict__ act,
                                                   int n1, int lo1, int w1, int d1, int lo2,
                                                   int w2, int d2, int64_t rowbase, int lane,
                                                   int32_t *__restrict__ col,
                                                   OutT *__restrict__ val) {
  constexpr int W = 2 * P + 1;
  int64_t pos = rowbase;
  for (int k0 = 0; k0 < w1 * w2; k0 += 32) {
    const int k = k0 + lane;
    int ja = -1, q1 = 0, q2 = 0;
    if (k < w1 * w2) {
      q2 = k / w1;
      q1 = k - q2 * w1;
      ja = act[(lo2 + q2) * n1 + lo1 + q1];
    }
    const unsigned m = __ballot_sync(0xffffffffu, ja >= 0);
    if (ja >= 0) {
      const int64_t ps = pos + __popc(m & ((1u << lane) - 1u));
      val[ps] = src[(q2 + d2) * W + q1 + d1];
      col[ps] = ja;
    }
    pos += __popc(m);
  }
}

// s = (sh, sl) += a * b, a and b pairs; products and sums error-free in the
// leading parts (__fmul_rn / __fadd_rn are never contracted into FMAs)
__device__ __forceinline__ void df_fma(float2 a, float2 b, float &sh, float &sl) {
  float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  float t = __fadd_rn(sh, p);
  float bp = __fadd_rn(t, -sh);
  float err = __fadd_rn(__fadd_rn(sh, -__fadd_rn(t, -bp)), __fadd_rn(p, -bp));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}

// The tables of the FP32-pipe contraction.  FP32: c and the weighted basis
// rounded to float; split: (hi, lo) float pairs.  The c grid is padded to a
// row stride ldc of 16 bytes' multiple so that any 16-byte-aligned column range
// of a row can be bulk-copied; Vc1 holds, per test function of direction 1
// and point c1 of its support, the P+1 weighted basis values that can be
// nonzero there (trial functions el .. el+P of the point's support element
// el = c1 / 2; rows whose support has the two-point layout of inner
// elements), padded by one row.
struct Tables32 {
  const void *C;  // float or float2, nq2 x ldc
  int ldc;
  const void *Vc1;  // float or float2, (n1 + 1) x (2P+2) x (P+1)
  const float2 *V1f, *V2f;  // full weighted basis tables (hi, lo), n x qmax x W
  int bulk_out;             // the CSR buffers are 16-byte aligned: bulk stores allowed
};

// Shared memory of one FP32-pipe tile (16-byte-aligned regions):
//   slab  the c rows of supp B_i2 over the tile's columns (bulk-copied)
//   vc    the tile's rows of Vc1 (bulk-copied)
//   Y     stage-1 sums, W x KMAX
//   V2s   the weighted basis of row i2
//   os    the tile's outputs in CSR order (+ one 16-byte alignment shift)
//   cs    their columns (+ the same)
//   sc    the tile's scalars, the band ranges of row i2, per row the interior
//         flag and the first WQ point
// kmax bounds the WQ points under the tile's rows (odd; the static bound for
// simple knots), q those of one support (4P for simple knots); a
// mixed-continuity vector passes its own, larger bounds.
__host__ __device__ constexpr int interior32_kmax(int P, int T) { return (2 * T + 4 * P + 4) | 1; }
__host__ __device__ constexpr size_t a16(size_t x) { return (x + 15) / 16 * 16; }
__host__ __device__ constexpr size_t interior32_slab_cols(int kmax) {
  return (size_t)kmax + 8;  // columns rounded out to 16 bytes on both sides
}
struct Layout32 {
  size_t slab, vc, y, v2, os, cs, cr2, total;
};
__host__ __device__ constexpr Layout32 interior32_layout(int P, int T, bool split, int kmax,
                                                         int q) {
  const size_t e = split ? sizeof(float2) : sizeof(float);
  const size_t o = split ? sizeof(double) : sizeof(float);
  const int W = 2 * P + 1, Q = q;  // Q bounds the WQ points of one support
  Layout32 L{};
  L.slab = 0;
  L.vc = L.slab + a16(e * Q * interior32_slab_cols(kmax));
  L.y = L.vc + a16(e * (size_t)T * (2 * P + 2) * (P + 1));
  L.v2 = L.y + a16(e * (size_t)W * kmax);
  L.os = L.v2 + a16(e * (size_t)Q * W);
  L.cs = L.os + a16(o * ((size_t)T * W * W + 16 / o));
  L.cr2 = L.cs + a16(sizeof(int) * ((size_t)T * W * W + 4));
  L.total = L.cr2 + a16(sizeof(int) * (8 + W + 2 * (size_t)T));
  return L;
}
__host__ __device__ constexpr Layout32 interior32_layout(int P, int T, bool split) {
  return interior32_layout(P, T, split, interior32_kmax(P, T), 4 * P);
}
__host__ __device__ constexpr size_t interior32_smem(int P, int T, bool split = true) {
  return interior32_layout(P, T, split).total;
}

// One tile of T test functions i1a .. i1a+T-1 of row i2 on the FP32 pipes.
// One thread stages the c slab and the tile's Vc1 rows with bulk copies on
// the mbarrier *bar (phase *phase, flipped here); stage 1 and stage 2 then
// read shared memory only.  A tile whose rows are all interior with a full
// band owns one contiguous CSR range: its values and columns are staged in
// CSR order and written by bulk shared -> global copies (the unaligned head
// and tail by plain stores); other tiles write one row per warp.  A wait that
// runs out sets TWF_TIMEOUT in *flag and the block abandons the tile (the
// decision is taken by the whole block, so no thread is left at a barrier).
template <int P, bool SPLIT>
__device__ void interior_tile32(const Dir &A, const Dir &B, const Tables32 &tb,
                                const uint8_t *__restrict__ fstate,
                                const int32_t *__restrict__ act, const int64_t *__restrict__ rp,
                                int32_t *__restrict__ col, void *__restrict__ valv, int i2,
                                int i1a, int T, char *smem, uint64_t *bar, uint32_t *phase,
                                int *flag, bool mixed, int kmax = 0, int q = 0) {
  constexpr int W = 2 * P + 1, NV = (2 * P + 2) * (P + 1);
  using ET = typename std::conditional<SPLIT, float2, float>::type;
  using OutT = typename std::conditional<SPLIT, double, float>::type;
  constexpr int AE = 16 / (int)sizeof(ET);    // elements per 16 bytes of a table
  constexpr int AO = 16 / (int)sizeof(OutT);  // of the outputs
  if (kmax <= 0) kmax = interior32_kmax(P, T);
  if (q <= 0) q = 4 * P;
  const Layout32 L = interior32_layout(P, T, SPLIT, kmax, q);
  ET *slab = (ET *)(smem + L.slab);
  ET *vcs = (ET *)(smem + L.vc);
  ET *Y = (ET *)(smem + L.y);
  ET *V2s = (ET *)(smem + L.v2);
  OutT *osb = (OutT *)(smem + L.os);
  int32_t *csb = (int32_t *)(smem + L.cs);
  // [0] any interior [1] full [2] kA [3] kB [4] qb2 [5] qc2 [6..7] CSR base (8-byte aligned)
  int *sc = (int *)(smem + L.cr2);
  int *cr2 = sc + 8;
  int *rowint = cr2 + W, *rowq = rowint + T;
  const int KMAX = kmax;
  const int i1b = min(A.n, i1a + T);
  const int nr = i1b - i1a;
  const int n1 = A.n;
  // the tile's scalars, loaded once (the CSR base of a full tile included)
  if (threadIdx.x == 0) {
    const bool range = i2 >= P && i2 <= B.n - 1 - P && i1a >= P && i1b - 1 <= n1 - 1 - P;
    sc[0] = 0;
    sc[1] = range ? 1 : 0;
    sc[2] = A.qbeg[i1a];
    sc[3] = A.qbeg[i1b - 1] + A.qcnt[i1b - 1];
    sc[4] = B.qbeg[i2];
    sc[5] = B.qcnt[i2];
    const int a0 = range ? act[i2 * n1 + i1a] : -1;
    *(int64_t *)(sc + 6) = a0 >= 0 ? rp[a0] : 0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nr; t += blockDim.x) {
    const int g = i2 * n1 + i1a + t;
    const bool in = fstate[g] == TW_FUNC_INTERIOR;
    rowint[t] = in ? 1 : 0;
    rowq[t] = A.qbeg[i1a + t];
    if (in) sc[0] = 1;
    // a full tile needs every row's whole band active: always so for simple
    // knots; with a repeated knot a band neighbour may share only the empty
    // span with B_i and be exterior
    if (!in || (mixed && rp[act[g] + 1] - rp[act[g]] != (int64_t)W * W)) sc[1] = 0;
  }
  __syncthreads();
  if (!sc[0]) return;  // uniform across the block
  const bool full = sc[1] != 0;
  const int kA = sc[2], kB = sc[3], qb2 = sc[4], qc2 = sc[5];
  const int kA0 = kA & ~(AE - 1);
  const int Kp = ((kB + AE - 1) & ~(AE - 1)) - kA0;  // slab row length, whole 16-byte units
  const int off = kA - kA0;
  // bulk loads: qc2 slab rows and the tile's Vc1 rows (even row count)
  if (threadIdx.x == 0) {
    const int nvr = (nr + 1) & ~1;
    const uint32_t rowb = (uint32_t)(sizeof(ET) * Kp);
    const uint32_t vcb = (uint32_t)(sizeof(ET) * NV * nvr);
    mbar_arrive_expect(bar, rowb * qc2 + vcb);
    const ET *C = (const ET *)tb.C;
    for (int c2 = 0; c2 < qc2; c2++)
      bulk_g2s(slab + (size_t)c2 * Kp, C + (size_t)(qb2 + c2) * tb.ldc + kA0, rowb, bar);
    bulk_g2s(vcs, (const ET *)tb.Vc1 + (size_t)i1a * NV, vcb, bar);
  }
  const float2 *V2f = tb.V2f + (size_t)i2 * B.qmax * W;
  for (int t = threadIdx.x; t < qc2 * W; t += blockDim.x) {
    if constexpr (SPLIT) V2s[t] = V2f[t];
    else V2s[t] = V2f[t].x;
  }
  for (int t = threadIdx.x; t < W; t += blockDim.x) cr2[t] = B.crange[i2 * W + t];
  // one thread waits for the copies (bounded); the block barrier then orders
  // the copied data before every other thread's reads, and carries the
  // outcome to all threads
  const int ok = __syncthreads_and(threadIdx.x == 0 ? (mbar_wait_bounded(bar, *phase) ? 1 : 0) : 1);
  *phase ^= 1u;
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(flag, TWF_TIMEOUT);
    return;
  }
  const int K = kB - kA;
  // stage 1: Y[r2][k1] = sum_{k2} V2[i2][k2][r2] c[k2][k1], two columns per thread
  const int K2 = (K + 1) >> 1;
  for (int idx = threadIdx.x; idx < W * K2; idx += blockDim.x) {
    const int r2 = idx / K2, kk = 2 * (idx - r2 * K2);
    const bool two = kk + 1 < K;
    const int lo = cr2[r2] & 0xffff, hi = cr2[r2] >> 16;
    const ET *cc = slab + (size_t)lo * Kp + off + kk;
    float sh0 = 0.f, sl0 = 0.f, sh1 = 0.f, sl1 = 0.f;
#pragma unroll 4
    for (int c2 = lo; c2 < hi; c2++, cc += Kp) {
      const ET vv = V2s[c2 * W + r2];
      const ET c0 = cc[0];
      if constexpr (SPLIT) {
        const float2 c1 = two ? cc[1] : make_float2(0.f, 0.f);
        df_fma(vv, c0, sh0, sl0);
        df_fma(vv, c1, sh1, sl1);
      } else {
        const float c1 = two ? cc[1] : 0.f;
        sh0 = fmaf(vv, c0, sh0);
        sh1 = fmaf(vv, c1, sh1);
      }
    }
    if constexpr (SPLIT) {
      Y[r2 * KMAX + kk] = make_float2(sh0, sl0);
      if (two) Y[r2 * KMAX + kk + 1] = make_float2(sh1, sl1);
    } else {
      Y[r2 * KMAX + kk] = sh0;
      if (two) Y[r2 * KMAX + kk + 1] = sh1;
    }
  }
  __syncthreads();
  // the tile's CSR range (full tiles): base position and the alignment shift
  // that puts 16-byte units of the range on 16-byte units of shared memory
  const int64_t base = full ? *(const int64_t *)(sc + 6) : 0;
  const int sho = (int)(base & (AO - 1)), shc = (int)(base & 3);
  // stage 2 (point-major for rows away from the end elements, from vcs) into
  // os: full tiles at CSR position (t W + r2) W + r1 (+ shift), others at
  // [t][r2][r1].  A thread owns one (row, r2) item; in FP32 below p = 6 two
  // neighbouring r2 of one row (measured faster at p = 4, slower at p = 6)
  constexpr int NRP = (SPLIT || P >= 6) ? 1 : 2;
  constexpr int WH = (W + NRP - 1) / NRP;
  OutT *os = osb + (full ? sho : 0);
  for (int idx = threadIdx.x; idx < nr * WH; idx += blockDim.x) {
    const int t = idx / WH, r2a = NRP * (idx - t * WH), r2b = r2a + 1;
    const int i1 = i1a + t;
    if (!rowint[t]) continue;
    const int j2a = i2 - P + r2a, j2b = j2a + 1;
    const bool va = j2a >= 0 && j2a < B.n;
    const bool vb = NRP == 2 && r2b < W && j2b >= 0 && j2b < B.n;
    if (!va && !vb) continue;
    const int yo = rowq[t] - kA;
    const ET *ya = Y + r2a * KMAX + yo;
    const ET *yb = Y + (vb ? r2b : r2a) * KMAX + yo;
    OutT *oa = os + ((size_t)t * W + r2a) * W;
    OutT *ob = oa + W;
    if (i1 >= P + 1 && i1 <= A.nel - 2 && (!mixed || A.two[i1])) {
      const ET *v = vcs + (size_t)t * NV;
      float aha[W], ala[W], ahb[W], alb[W];
#pragma unroll
      for (int r = 0; r < W; r++) aha[r] = ala[r] = ahb[r] = alb[r] = 0.f;
#pragma unroll
      for (int el = 0; el <= P; el++) {
#pragma unroll
        for (int pt = 0; pt < 2; pt++) {
          const int c1 = 2 * el + pt;
          const ET yva = ya[c1], yvb = yb[c1];
#pragma unroll
          for (int a = 0; a <= P; a++) {
            const ET vv = v[c1 * (P + 1) + a];
            if constexpr (SPLIT) {
              df_fma(vv, yva, aha[el + a], ala[el + a]);
            } else {
              aha[el + a] = fmaf(vv, yva, aha[el + a]);
              ahb[el + a] = fmaf(vv, yvb, ahb[el + a]);
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < W; r++) {
        if constexpr (SPLIT) {
          if (va) oa[r] = widen_f32(aha[r]) + widen_f32(ala[r]);
        } else {
          if (va) oa[r] = aha[r];
          if (vb) ob[r] = ahb[r];
        }
      }
    } else {
      const float2 *v = tb.V1f + ((size_t)i1 * A.qmax) * W;
      for (int r1 = 0; r1 < W; r1++) {
        const int j1 = i1 - P + r1;
        if (j1 < 0 || j1 >= n1) continue;
        const int cr = A.crange[i1 * W + r1];
        const int lo = cr & 0xffff, hi = cr >> 16;
        float sha = 0.f, sla = 0.f, shb = 0.f;
        for (int c1 = lo; c1 < hi; c1++) {
          const float2 vv = v[c1 * W + r1];
          if constexpr (SPLIT) {
            df_fma(vv, ya[c1], sha, sla);
          } else {
            sha = fmaf(vv.x, ya[c1], sha);
            shb = fmaf(vv.x, yb[c1], shb);
          }
        }
        if constexpr (SPLIT) {
          if (va) oa[r1] = widen_f32(sha) + widen_f32(sla);
        } else {
          if (va) oa[r1] = sha;
          if (vb) ob[r1] = shb;
        }
      }
    }
  }
  OutT *val = (OutT *)valv;
  if (full) {
    // columns of the full band, in CSR order.  Every trial function of a full
    // tile is active (it overlaps an interior function), so along one trial
    // row j2 the active indices are consecutive: col = act(j2, i1a - P) + t + q1
    int32_t *cs = csb + shc;
    const int L2 = nr * W * W;
    for (int k = threadIdx.x; k < nr * W; k += blockDim.x) {
      const int t = k / W, q2 = k - t * W;
      const int32_t c0 = act[(i2 - P + q2) * n1 + i1a - P] + t;
      int32_t *dst = cs + (size_t)k * W;
#pragma unroll
      for (int q1 = 0; q1 < W; q1++) dst[q1] = c0 + q1;
    }
    fence_proxy_async_smem();
    __syncthreads();
    // head and tail by plain stores, the 16-byte units between by bulk copies
    const int hv = (AO - sho) & (AO - 1), hc = (4 - shc) & 3;
    const int mv = tb.bulk_out && L2 > hv ? (L2 - hv) / AO * AO : 0;
    const int mc = tb.bulk_out && L2 > hc ? (L2 - hc) / 4 * 4 : 0;
    const int tv = mv > 0 ? L2 - hv - mv : L2, tc = mc > 0 ? L2 - hc - mc : L2;
    for (int k = threadIdx.x; k < (mv > 0 ? hv + tv : L2); k += blockDim.x) {
      const int kk = k < hv || mv == 0 ? k : k + mv;
      val[base + kk] = os[kk];
    }
    for (int k = threadIdx.x; k < (mc > 0 ? hc + tc : L2); k += blockDim.x) {
      const int kk = k < hc || mc == 0 ? k : k + mc;
      col[base + kk] = cs[kk];
    }
    if (threadIdx.x == 0) {
      if (mv > 0) bulk_s2g(val + base + hv, os + hv, (uint32_t)(sizeof(OutT) * mv));
      if (mc > 0) bulk_s2g(col + base + hc, cs + hc, (uint32_t)(sizeof(int32_t) * mc));
      bulk_commit();
      bulk_wait_read();  // shared memory is free for the next tile when the block moves on
    }
  } else {
    __syncthreads();
    // one warp per row, consecutive lanes on consecutive CSR positions
    const int nw = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lo2 = max(0, i2 - P), w2 = min(B.n - 1, i2 + P) - lo2 + 1, d2 = lo2 - (i2 - P);
    for (int t = wid; t < nr; t += nw) {
      const int i1 = i1a + t, g = i2 * n1 + i1;
      if (fstate[g] != TW_FUNC_INTERIOR) continue;  // the whole warp
      const int lo1 = max(0, i1 - P), w1 = min(n1 - 1, i1 + P) - lo1 + 1, d1 = lo1 - (i1 - P);
      const int64_t rowbase = rp[act[g]];
      const OutT *src = os + (size_t)t * W * W;
      if (!mixed || rp[act[g] + 1] - rowbase == (int64_t)w1 * w2) {  // whole band active
        for (int k = lane; k < w1 * w2; k += 32) {
          const int q2 = k / w1, q1 = k - q2 * w1;
          val[rowbase + k] = src[(q2 + d2) * W + q1 + d1];
          col[rowbase + k] = act[(lo2 + q2) * n1 + lo1 + q1];
        }
      } else {
        band_write_compact<P>(src, act, n1, lo1, w1, d1, lo2, w2, d2, rowbase, lane, col, val);
      }
    }
  }
  __syncthreads();  // the tile's shared memory is reused by the next item
}

}  // namespace tw
