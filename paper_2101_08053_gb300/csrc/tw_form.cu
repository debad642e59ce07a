// tw_form.cu -- formation of the trimmed mass matrix (Sect. 2.1 Eqs. 6-7,
// Sect. 3 Eq. 8, Sects. 3.1-3.3), written straight into the caller's CSR.
//
//  k_interior<P,T>  interior test functions: weighted quadrature with sum
//                   factorisation, row-based.  One thread block per (i2, tile
//                   of T consecutive i1): stage 1 contracts direction 2 over
//                   the block's slab of c,
//                       Y[r2][k1] = sum_{k2 in Q_{i2}} W2[i2,k2] B_{j2}(x_k2) c[k2][k1],
//                   stage 2 gives every output of the tile's rows,
//                       m_{i,j} = sum_{k1 in Q_{i1}} W1[i1,k1] B_{j1}(x_k1) Y[r2][k1].
//                   Both stages skip the zero part of the band (only points in
//                   supp B_i cap supp B_j contribute).  Consecutive threads own
//                   consecutive CSR positions of a row, so writes coalesce.
//  k_cutrows<P>     one block per cut row (all rows for the Gauss method):
//                   region part (DWQ rectangle or naive masked WQ) by sum
//                   factorisation, element Gauss on regular elements (element
//                   level sum factorisation), cut-element rule on cut elements.
//                   Every output is owned by one thread and summed in a fixed
//                   order, so the matrix is bitwise reproducible.
#include "tw_internal.cuh"

namespace tw {

template <int P, int T>
__global__ void __launch_bounds__(256) k_interior(Dir A, Dir B, const double *__restrict__ C,
                                                  const uint8_t *__restrict__ fstate,
                                                  const int32_t *__restrict__ act,
                                                  const int64_t *__restrict__ rp,
                                                  int32_t *__restrict__ col,
                                                  double *__restrict__ val) {
  constexpr int W = 2 * P + 1;
  constexpr int KMAX = (2 * T + 4 * P + 4) | 1;  // odd row stride: no bank conflicts
  __shared__ double Y[W * KMAX];
  __shared__ double V2s[TW_QMAX * W];
  __shared__ int cr2[W];
  __shared__ int anyint;
  const int i2 = blockIdx.y;
  const int i1a = blockIdx.x * T;
  const int i1b = min(A.n, i1a + T);
  const int n1 = A.n;
  if (threadIdx.x == 0) anyint = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < i1b - i1a; t += blockDim.x)
    if (fstate[i2 * n1 + i1a + t] == TW_FUNC_INTERIOR) anyint = 1;
  __syncthreads();
  if (!anyint) return;
  const int kA = A.qbeg[i1a];
  const int kB = A.qbeg[i1b - 1] + A.qcnt[i1b - 1];
  const int K = kB - kA;
  const int qb2 = B.qbeg[i2], qc2 = B.qcnt[i2];
  for (int t = threadIdx.x; t < qc2 * W; t += blockDim.x)
    V2s[t] = B.V[(size_t)i2 * B.qmax * W + t];
  for (int t = threadIdx.x; t < W; t += blockDim.x) cr2[t] = B.crange[i2 * W + t];
  __syncthreads();
  // stage 1
  for (int idx = threadIdx.x; idx < W * K; idx += blockDim.x) {
    int r2 = idx / K, kk = idx - r2 * K;
    int lo = cr2[r2] & 0xffff, hi = cr2[r2] >> 16;
    const double *cc = C + (size_t)(qb2 + lo) * A.nq + kA + kk;
    double s = 0.0;
    for (int c2 = lo; c2 < hi; c2++, cc += A.nq) s = fma(V2s[c2 * W + r2], *cc, s);
    Y[r2 * KMAX + kk] = s;
  }
  __syncthreads();
  // stage 2.  Rows whose support avoids the two end elements (2 points per
  // element, full band) take the point-major path: thread (row, r2) walks the
  // 2(P+1) points of supp B_i1 and adds each point's value into the P+1
  // outputs whose trial function lives on the point's element, so every lane
  // issues the same (P+1)*2*(P+1) DFMAs.  Other rows use the per-output loop.
  const int lo2 = max(0, i2 - P);
  const int NR = (i1b - i1a) * W;
  for (int idx = threadIdx.x; idx < NR; idx += blockDim.x) {
    const int t = idx / W, r2 = idx - t * W;
    const int i1 = i1a + t;
    const int g = i2 * n1 + i1;
    const int j2 = i2 - P + r2;
    if (fstate[g] != TW_FUNC_INTERIOR || j2 < 0 || j2 >= B.n) continue;
    const double *y = Y + r2 * KMAX + (A.qbeg[i1] - kA);
    const double *v = A.V + ((size_t)i1 * A.qmax) * W;
    const int64_t rowbase = rp[act[g]];
    if (i1 >= P + 1 && i1 <= A.nel - 2) {
      double acc[W];
#pragma unroll
      for (int r = 0; r < W; r++) acc[r] = 0.0;
#pragma unroll
      for (int el = 0; el <= P; el++) {
#pragma unroll
        for (int pt = 0; pt < 2; pt++) {
          const int c1 = 2 * el + pt;
          const double yv = y[c1];
#pragma unroll
          for (int a = 0; a <= P; a++) acc[el + a] = fma(v[c1 * W + el + a], yv, acc[el + a]);
        }
      }
      double *out = val + rowbase + (int64_t)(j2 - lo2) * W;
      int32_t *oc = col + rowbase + (int64_t)(j2 - lo2) * W;
      const int32_t *arow = act + j2 * n1 + (i1 - P);
#pragma unroll
      for (int r = 0; r < W; r++) {
        out[r] = acc[r];
        oc[r] = arow[r];
      }
    } else {
      const int lo1 = max(0, i1 - P), w1 = min(n1 - 1, i1 + P) - lo1 + 1;
      for (int r1 = 0; r1 < W; r1++) {
        const int j1 = i1 - P + r1;
        if (j1 < 0 || j1 >= n1) continue;
        const int cr = A.crange[i1 * W + r1];
        const int lo = cr & 0xffff, hi = cr >> 16;
        double s = 0.0;
        for (int c1 = lo; c1 < hi; c1++) s = fma(v[c1 * W + r1], y[c1], s);
        const int64_t pos = rowbase + (int64_t)(j2 - lo2) * w1 + (j1 - lo1);
        val[pos] = s;
        col[pos] = act[j2 * n1 + j1];
      }
    }
  }
}

#define TW_RC 32

template <int P, typename OutT>
__global__ void __launch_bounds__(256) k_cutrows(RowArgs a, const int32_t *__restrict__ rows,
                                                 int32_t *__restrict__ col,
                                                 OutT *__restrict__ val) {
  constexpr int W = 2 * P + 1, P1 = P + 1;
  __shared__ double acc[W * W];
  __shared__ double rx[2][TW_RC], rw[2][TW_RC], rb[2][TW_RC][W];
  __shared__ int rk[2][TW_RC];
  __shared__ int nr[2], nnest[2], nest[2][TW_RC];
  __shared__ double cg[TW_RC * TW_RC];
  __shared__ double Z[W * TW_RC];
  __shared__ double Tg[P1 * P1];
  __shared__ int pos[W * W];
  const Dir &A = a.A;
  const Dir &B = a.B;
  const int g = rows[blockIdx.x];
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
  for (int t = tid; t < W * W; t += blockDim.x) acc[t] = 0.0;

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
          rx[d][lane] = D.xq[k];
          rw[d][lane] = D.W[(size_t)i * D.qmax + lane];
          rk[d][lane] = k;
          for (int r = 0; r < W; r++) {
            int aa = i - P + r - D.qel[k];
            rb[d][lane][r] = (aa >= 0 && aa <= P) ? D.Bq[k * P1 + aa] : 0.0;
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
          rx[d][lane] = a.dwq_x[d][k];
          rw[d][lane] = a.dwq_w[d][(((size_t)sl * P + (i - s)) * 2 + side) * TW_LQMAX + k0 + lane];
          rk[d][lane] = a.dwq_k[d][k];  // base points read c from the grid
          const int e = a.dwq_e[d][k];
          const double *Bv = a.dwq_B[d] + k * P1;
          for (int r = 0; r < W; r++) {
            int aa = i - P + r - e;
            rb[d][lane][r] = (aa >= 0 && aa <= P) ? Bv[aa] : 0.0;
          }
        }
      }
      if (lane == 0) nr[d] = n;
    }
    __syncthreads();
    const int m1 = nr[0], m2 = nr[1];
    // c at the tensor points: grid pairs first, then the pairs with a nested
    // point packed densely so only a few warps evaluate c directly
    for (int t = tid; t < m1 * m2; t += blockDim.x) {
      int ia = t % m1, ib = t / m1;
      int k1 = rk[0][ia], k2 = rk[1][ib];
      if (k1 >= 0 && k2 >= 0) {
        double c = a.C[(size_t)k2 * A.nq + k1];
        if (kind == 1 && a.estate[B.qel[k2] * A.nel + A.qel[k1]] != TW_ELEM_REGULAR) c = 0.0;
        cg[ia * TW_RC + ib] = c;
      }
    }
    if (tid == 0) {
      int na = 0, nb = 0;
      for (int ia = 0; ia < m1; ia++)
        if (rk[0][ia] < 0) nest[0][na++] = ia;
      for (int ib = 0; ib < m2; ib++)
        if (rk[1][ib] < 0) nest[1][nb++] = ib;
      nnest[0] = na;
      nnest[1] = nb;
    }
    __syncthreads();
    {
      const int na = nnest[0], nb = nnest[1];
      const int tot = na * m2 + (m1 - na) * nb;
      for (int t = tid; t < tot; t += blockDim.x) {
        int ia, ib;
        if (t < na * m2) {
          ia = nest[0][t / m2];
          ib = t % m2;
        } else {
          int u = t - na * m2;
          ib = nest[1][u % nb];
          // the (u / nb)-th base point of direction 0
          int want = u / nb, cntb = -1;
          ia = 0;
          for (int q = 0; q < m1; q++)
            if (rk[0][q] >= 0 && ++cntb == want) {
              ia = q;
              break;
            }
        }
        cg[ia * TW_RC + ib] = coef_at(a.G, A, B, rx[0][ia], rx[1][ib]);
      }
    }
    __syncthreads();
    for (int t = tid; t < W * m1; t += blockDim.x) {
      int r2 = t / m1, ia = t % m1;
      double s = 0.0;
      for (int ib = 0; ib < m2; ib++) s = fma(rw[1][ib] * rb[1][ib][r2], cg[ia * TW_RC + ib], s);
      Z[r2 * TW_RC + ia] = s;
    }
    __syncthreads();
    for (int t = tid; t < W * W; t += blockDim.x) {
      int r2 = t / W, q1 = t % W;
      double s = 0.0;
      for (int ia = 0; ia < m1; ia++) s = fma(rw[0][ia] * rb[0][ia][q1], Z[r2 * TW_RC + ia], s);
      acc[t] += s;
    }
    __syncthreads();
  } else {
    __syncthreads();
  }

  // ---- elements of the support: Gauss on regular (outside R), cut rule on cut ----
  const int p1 = P1;
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
          acc[(e2 + b2 - i2 + P) * W + (e1 + b1 - i1 + P)] += Me[b2 * p1 + b1];
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
          Tg[g2 * p1 + b1] = s;
        }
        __syncthreads();
        if (tid < p1 * p1) {
          int b1 = tid % p1, b2 = tid / p1;
          double s = 0.0;
          for (int g2 = 0; g2 < p1; g2++)
            s = fma(Tg[g2 * p1 + b1], B.gw[g2] * h2 * GB2[g2 * p1 + (i2 - e2)] * GB2[g2 * p1 + b2], s);
          acc[(e2 + b2 - i2 + P) * W + (e1 + b1 - i1 + P)] += s;
        }
        __syncthreads();
      } else if (st == TW_ELEM_CUT) {
        // the cut element's matrix, formed once per element
        const int cs = a.cut_slot[e];
        const double *Me = a.cut_M + ((size_t)cs * p1 * p1 + (i2 - e2) * p1 + (i1 - e1)) * p1 * p1;
        if (tid < p1 * p1) {
          int b1 = tid % p1, b2 = tid / p1;
          acc[(e2 + b2 - i2 + P) * W + (e1 + b1 - i1 + P)] += Me[b2 * p1 + b1];
        }
        __syncthreads();
      }
    }

  // ---- write the row: active columns in ascending order (R11) ----
  if (tid == 0) {
    int c = 0;
    for (int r2 = 0; r2 < W; r2++)
      for (int q1 = 0; q1 < W; q1++) {
        int j1 = i1 - P + q1, j2 = i2 - P + r2;
        int ok = j1 >= 0 && j1 < n1 && j2 >= 0 && j2 < B.n && a.act[j2 * n1 + j1] >= 0;
        pos[r2 * W + q1] = ok ? c++ : -1;
      }
  }
  __syncthreads();
  const int64_t base = a.rp[a.act[g]];
  for (int t = tid; t < W * W; t += blockDim.x) {
    int ps = pos[t];
    if (ps < 0) continue;
    int r2 = t / W, q1 = t % W;
    int j1 = i1 - P + q1, j2 = i2 - P + r2;
    val[base + ps] = (OutT)acc[t];
    col[base + ps] = a.act[j2 * n1 + j1];
  }
}

__global__ void k_copy_i64(const int64_t *src, int64_t *dst, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

template <int P>
static int launch_form(tw_patch *Pt, int precision, int64_t *rp, int32_t *col, void *valv,
                       cudaStream_t s) {
  constexpr int T = 32;
  Dir &A = Pt->d[0];
  Dir &B = Pt->d[1];
  double *val = (double *)valv;
  if (Pt->method != TW_METHOD_GAUSS && Pt->n_interior > 0 && precision != TW_PREC_FP64) {
    int rc = launch_interior32(Pt, precision, col, valv, s);
    if (rc) return rc;
  } else if (Pt->method != TW_METHOD_GAUSS && Pt->n_interior > 0) {
    dim3 grid((A.n + T - 1) / T, B.n);
    int ps = prof_start(s);
    k_interior<P, T><<<grid, 256, 0, s>>>(A, B, Pt->C, Pt->fstate, Pt->act, Pt->row_ptr, col, val);
    prof_stop(ps, TW_STAGE_INTERIOR, s);
    TW_LAUNCH();
  }
  if (Pt->ncutrows > 0) {
    RowArgs ra;
    ra.A = A;
    ra.B = B;
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
      ra.dwq_r[d] = Pt->dwq_r[d];
    }
    ra.gmat = Pt->gmat;
    ra.method = Pt->method;
    ra.flag = Pt->flag;
    int ps = prof_start(s);
    if (precision == TW_PREC_FP32)
      k_cutrows<P, float><<<Pt->ncutrows, 256, 0, s>>>(ra, Pt->cutrows, col, (float *)valv);
    else
      k_cutrows<P, double><<<Pt->ncutrows, 256, 0, s>>>(ra, Pt->cutrows, col, val);
    prof_stop(ps, TW_STAGE_CUTROWS, s);
    TW_LAUNCH();
  }
  return 0;
}

int form_mass_launch(tw_patch *P, int precision, int64_t *rp, int32_t *col, void *val,
                     cudaStream_t s) {
  int64_t n = P->n_rows + 1;
  k_copy_i64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P->row_ptr, rp, n);
  TW_LAUNCH();
  int rc;
  switch (P->p) {
    case 1: rc = launch_form<1>(P, precision, rp, col, val, s); break;
    case 2: rc = launch_form<2>(P, precision, rp, col, val, s); break;
    case 3: rc = launch_form<3>(P, precision, rp, col, val, s); break;
    case 4: rc = launch_form<4>(P, precision, rp, col, val, s); break;
    case 5: rc = launch_form<5>(P, precision, rp, col, val, s); break;
    case 6: rc = launch_form<6>(P, precision, rp, col, val, s); break;
    default: return TW_EUNSUPPORTED;
  }
  if (rc) return rc;
  return check_cuda(cudaGetLastError(), "tw_form_mass launch");
}

}  // namespace tw
