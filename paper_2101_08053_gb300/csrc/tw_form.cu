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
//  k_cutrows_gather rows without a region part whose element matrices are all
//                   precomputed (hybrid Gauss, Gauss method, DWQ rows without
//                   a region): one warp per row gathers the element rows.
//                   Every output is owned by one thread and summed in a fixed
//                   order, so the matrix is bitwise reproducible.
#include <algorithm>

#include "tw_bodies.cuh"

namespace tw {

__device__ __forceinline__ bool cutrow_is_rowsf(const RowArgs &a, int g) {
  if (a.method == TW_METHOD_NAIVE) return false;
  return a.method != TW_METHOD_DWQ || a.choice[4 * g] < 0;
}

// rows that need the region part or element integration (the rest go to
// k_cutrows_gather, or to k_cutrows_sf in the row-sum-factorised form)
template <int P, typename OutT>
__global__ void __launch_bounds__(128) k_cutrows(RowArgs a, const int32_t *__restrict__ rows,
                                                 int32_t *__restrict__ col,
                                                 OutT *__restrict__ val, int rowsf) {
  __shared__ __align__(16) char smem[sizeof(CutSmem<P>)];
  const int g = rows[blockIdx.x];
  if (rowsf ? cutrow_is_rowsf(a, g) : cutrow_is_gather(a, g)) return;
  cutrow_item<P, OutT>(a, g, col, val, smem);
}

// one warp per gather row; the launch also copies the patch's row pointer
// (nrp entries) into the caller's CSR, grid-stride over all its threads
template <int P, typename OutT>
__global__ void __launch_bounds__(128) k_cutrows_gather(RowArgs a,
                                                        const int32_t *__restrict__ rows,
                                                        int nrows, int32_t *__restrict__ col,
                                                        OutT *__restrict__ val,
                                                        int64_t *__restrict__ rp_out,
                                                        int64_t nrp) {
  __shared__ const double *tab[4][(P + 1) * (P + 1)];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrp;
       i += (int64_t)gridDim.x * blockDim.x)
    rp_out[i] = a.rp[i];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * 4 + wib;
  if (r >= nrows) return;  // the whole warp
  const int g = rows[r];
  if (!cutrow_is_gather(a, g)) return;
  cutrow_gather_warp<P, OutT>(a, g, lane, tab[wib], col, val);
}

// Remark 1 of Sect. 3.2 on a cut row without a region part: the Gauss part as
// one tensor rule over the element Gauss points of the whole support, with c
// set to zero off the regular elements (S^r), sum-factorised like Eq. 7 --
// stage A over the points of direction 1, stage B over direction 2 -- plus the
// cut elements' matrix rows.  One block per row; each output is summed by one
// thread in a fixed order.

template <int P>
struct SfSmem {
  static constexpr int W = 2 * P + 1, P1 = P + 1, NG = P1 * P1;
  double ct[NG * NG];     // c at the support grid, [k2][k1], zero off S^r
  double wbj[2][NG][P1];  // Gauss weight x B_i x B_{e+a} at grid point k of element e
  double X[W * NG];       // stage A, [r1][k2]
  double acc[W * W];
  const double *eM[P1 * P1];  // matrix rows of the support's cut elements
};

template <int P, typename OutT>
__global__ void __launch_bounds__(128) k_cutrows_sf(RowArgs a, const int32_t *__restrict__ rows,
                                                    int nrows, int32_t *__restrict__ col,
                                                    OutT *__restrict__ val) {
  constexpr int W = 2 * P + 1, P1 = P + 1, NG = P1 * P1, P2 = P1 * P1, NE = (W * W + 31) / 32;
  __shared__ SfSmem<P> S;
  const int r = blockIdx.x;
  if (r >= nrows) return;
  const int g = rows[r];
  if (!cutrow_is_rowsf(a, g)) return;  // the whole block
  const Dir &A = a.A;
  const Dir &B = a.B;
  const int n1 = A.n;
  const int i1 = g % n1, i2 = g / n1;
  const int lo1 = max(0, i1 - P), hi1 = min(A.nel - 1, i1);
  const int lo2 = max(0, i2 - P), hi2 = min(B.nel - 1, i2);
  const int N1 = (hi1 - lo1 + 1) * P1, N2 = (hi2 - lo2 + 1) * P1;
  // grid tables of both directions
  for (int t = threadIdx.x; t < N1 + N2; t += blockDim.x) {
    const int d = t < N1 ? 0 : 1, k = d ? t - N1 : t;
    const Dir &D = d ? B : A;
    const int e = (d ? lo2 : lo1) + k / P1, gg = k % P1, i = d ? i2 : i1;
    const double *gb = D.GB + ((size_t)e * P1 + gg) * P1;
    const double w = D.gw[gg] * 0.5 * (D.bp[e + 1] - D.bp[e]) * gb[i - e];
#pragma unroll
    for (int q = 0; q < P1; q++) S.wbj[d][k][q] = w * gb[q];
  }
  // c at the grid, masked off the regular elements
  for (int t = threadIdx.x; t < N1 * N2; t += blockDim.x) {
    const int k2 = t / N1, k1 = t - k2 * N1;
    const int e1 = lo1 + k1 / P1, e2 = lo2 + k2 / P1, ee = e2 * A.nel + e1;
    S.ct[k2 * N1 + k1] = a.estate[ee] == TW_ELEM_REGULAR
                             ? a.gc[(size_t)a.gslot[ee] * P2 + (k2 % P1) * P1 + (k1 % P1)]
                             : 0.0;
  }
  for (int t = threadIdx.x; t < P2; t += blockDim.x) {
    const int e1 = i1 - P + t % P1, e2 = i2 - P + t / P1;
    const double *Me = nullptr;
    if (e1 >= lo1 && e1 <= hi1 && e2 >= lo2 && e2 <= hi2) {
      const int e = e2 * A.nel + e1;
      if (a.estate[e] == TW_ELEM_CUT)
        Me = a.cut_M + (size_t)a.cut_slot[e] * P2 * P2 +
             (size_t)((i2 - e2) * P1 + (i1 - e1)) * P2;
    }
    S.eM[t] = Me;
  }
  __syncthreads();
  // stage A: X[r1][k2] = sum over the points k1 of the elements shared by
  // supp B_i1 and supp B_j1 of w B_i1 B_j1 c
  for (int idx = threadIdx.x; idx < W * N2; idx += blockDim.x) {
    const int r1 = idx / N2, k2 = idx - r1 * N2;
    const int j1 = i1 - P + r1;
    double s = 0.0;
    const int ulo = max(0, j1 - P - lo1), uhi = min(hi1 - lo1, j1 - lo1);
    for (int u1 = ulo; u1 <= uhi; u1++) {
      const int a1 = j1 - (lo1 + u1);
      const double *ct = S.ct + k2 * N1 + u1 * P1;
#pragma unroll
      for (int gg = 0; gg < P1; gg++) s = fma(S.wbj[0][u1 * P1 + gg][a1], ct[gg], s);
    }
    S.X[r1 * NG + k2] = s;
  }
  __syncthreads();
  // stage B, then the cut elements' rows in (u2, u1) order
  for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x) {
    const int q2 = idx / W, q1 = idx - q2 * W;
    const int j2 = i2 - P + q2;
    double s = 0.0;
    const int ulo = max(0, j2 - P - lo2), uhi = min(hi2 - lo2, j2 - lo2);
    for (int u2 = ulo; u2 <= uhi; u2++) {
      const int a2 = j2 - (lo2 + u2);
      const double *x = S.X + q1 * NG + u2 * P1;
#pragma unroll
      for (int gg = 0; gg < P1; gg++) s = fma(S.wbj[1][u2 * P1 + gg][a2], x[gg], s);
    }
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
    S.acc[idx] = s;
  }
  __syncthreads();
  // the row's active entries in ascending order, by the first warp
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const int64_t base = a.rp[a.act[g]];
    int before = 0;
#pragma unroll
    for (int k = 0; k < NE; k++) {
      const int t = k * 32 + lane;
      int jact = -1;
      if (t < W * W) {
        const int q2 = t / W, q1 = t % W;
        const int j1 = i1 - P + q1, j2 = i2 - P + q2;
        if (j1 >= 0 && j1 < n1 && j2 >= 0 && j2 < B.n) jact = a.act[j2 * n1 + j1];
      }
      const unsigned m = __ballot_sync(0xffffffffu, jact >= 0);
      if (jact >= 0) {
        const int ps = before + __popc(m & ((1u << lane) - 1u));
        val[base + ps] = (OutT)S.acc[t];
        col[base + ps] = jact;
      }
      before += __popc(m);
    }
  }
}

__global__ void k_copy_i64(const int64_t *src, int64_t *dst, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

template <int P>
static int launch_form(tw_patch *Pt, int precision, int64_t *rp, int32_t *col, void *valv,
                       cudaStream_t s, bool rowsf) {
  constexpr int T = P <= 5 ? 32 : 16;  // the tile's output buffer stays within 48 KB
  constexpr int LT = P <= 5 ? 5 : 4;   // log2 T
  Dir &A = Pt->d[0];
  Dir &B = Pt->d[1];
  double *val = (double *)valv;
  if (Pt->method != TW_METHOD_GAUSS && Pt->n_interior > 0 && precision != TW_PREC_FP64) {
    int rc = launch_interior32(Pt, precision, col, valv, s);
    if (rc) return rc;
  } else if (Pt->method != TW_METHOD_GAUSS && Pt->n_interior > 0) {
    dim3 grid((A.n + T - 1) / T, B.n);
    // the stage-1 buffer holds the WQ points under a tile: the static bound
    // for simple knots, the patch's own (odd) for a mixed-continuity vector
    const int kmax = std::max(interior_kmax(P, T), Pt->ktile[LT] | 1);
    const size_t smem = interior_smem(P, T, kmax);
    int ps = prof_start(s);
    if (!Pt->mixed) {
      k_interior<P, T, false><<<grid, 256, 0, s>>>(A, B, Pt->C, Pt->fstate, Pt->act,
                                                   Pt->row_ptr, col, val, kmax);
    } else {
      if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(
            k_interior<P, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return check_cuda(e, "interior contraction: shared memory");
      }
      k_interior<P, T, true><<<grid, 256, smem, s>>>(A, B, Pt->C, Pt->fstate, Pt->act,
                                                     Pt->row_ptr, col, val, kmax);
    }
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
      ra.dwq_dB[d] = Pt->dwq_dB[d];
      ra.dwq_r[d] = Pt->dwq_r[d];
    }
    ra.gmat = Pt->gmat;
    ra.method = Pt->method;
    ra.flag = Pt->flag;
    int ps = prof_start(s);
    const unsigned gw = (unsigned)((Pt->ncutrows + 3) / 4);
    // gather rows exist iff there are element matrices and the method is not
    // naive WQ; block rows iff not every row is a gather row
    // row-sum-factorised form (Remark 1): every row without a region part goes
    // to k_cutrows_sf, element matrices unused
    const bool sf = rowsf && Pt->method != TW_METHOD_NAIVE;
    const bool gather = !sf && Pt->gmat && Pt->method != TW_METHOD_NAIVE;
    const bool block = !(gather || sf) || Pt->method == TW_METHOD_DWQ;
    const int rsf = sf ? 1 : 0;
    if (precision == TW_PREC_FP32) {
      if (gather)
        k_cutrows_gather<P, float><<<gw, 128, 0, s>>>(ra, Pt->cutrows, Pt->ncutrows, col,
                                                      (float *)valv, rp, Pt->n_rows + 1);
      if (sf)
        k_cutrows_sf<P, float><<<Pt->ncutrows, 128, 0, s>>>(ra, Pt->cutrows, Pt->ncutrows, col,
                                                             (float *)valv);
      if (block)
        k_cutrows<P, float><<<Pt->ncutrows, 128, 0, s>>>(ra, Pt->cutrows, col, (float *)valv,
                                                          rsf);
    } else {
      if (gather)
        k_cutrows_gather<P, double><<<gw, 128, 0, s>>>(ra, Pt->cutrows, Pt->ncutrows, col, val,
                                                       rp, Pt->n_rows + 1);
      if (sf)
        k_cutrows_sf<P, double><<<Pt->ncutrows, 128, 0, s>>>(ra, Pt->cutrows, Pt->ncutrows, col,
                                                              val);
      if (block)
        k_cutrows<P, double><<<Pt->ncutrows, 128, 0, s>>>(ra, Pt->cutrows, col, val, rsf);
    }
    if (gather) TW_LAUNCH();
    if (sf) TW_LAUNCH();
    if (block) TW_LAUNCH();
    prof_stop(ps, TW_STAGE_CUTROWS, s);
    if (gather) return 0;  // the gather launch copied the row pointer
  }
  const int64_t n = Pt->n_rows + 1;
  k_copy_i64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Pt->row_ptr, rp, n);
  TW_LAUNCH();
  return 0;
}

int form_mass_launch(tw_patch *P, int precision, int64_t *rp, int32_t *col, void *val,
                     cudaStream_t s, bool rowsf) {
  int rc;
  switch (P->p) {
    case 1: rc = launch_form<1>(P, precision, rp, col, val, s, rowsf); break;
    case 2: rc = launch_form<2>(P, precision, rp, col, val, s, rowsf); break;
    case 3: rc = launch_form<3>(P, precision, rp, col, val, s, rowsf); break;
    case 4: rc = launch_form<4>(P, precision, rp, col, val, s, rowsf); break;
    case 5: rc = launch_form<5>(P, precision, rp, col, val, s, rowsf); break;
    case 6: rc = launch_form<6>(P, precision, rp, col, val, s, rowsf); break;
    default: return TW_EUNSUPPORTED;
  }
  if (rc) return rc;
  return check_cuda(cudaGetLastError(), "tw_form_mass launch");
}

}  // namespace tw
