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
#include "tw_bodies.cuh"

namespace tw {

// rows that need the region part or element integration (the rest go to
// k_cutrows_gather)
template <int P, typename OutT>
__global__ void __launch_bounds__(128) k_cutrows(RowArgs a, const int32_t *__restrict__ rows,
                                                 int32_t *__restrict__ col,
                                                 OutT *__restrict__ val) {
  __shared__ __align__(16) char smem[sizeof(CutSmem<P>)];
  const int g = rows[blockIdx.x];
  if (cutrow_is_gather(a, g)) return;
  cutrow_item<P, OutT>(a, g, col, val, smem);
}

// one warp per gather row
template <int P, typename OutT>
__global__ void __launch_bounds__(128) k_cutrows_gather(RowArgs a,
                                                        const int32_t *__restrict__ rows,
                                                        int nrows, int32_t *__restrict__ col,
                                                        OutT *__restrict__ val) {
  __shared__ const double *tab[4][(P + 1) * (P + 1)];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * 4 + wib;
  if (r >= nrows) return;  // the whole warp
  const int g = rows[r];
  if (!cutrow_is_gather(a, g)) return;
  cutrow_gather_warp<P, OutT>(a, g, lane, tab[wib], col, val);
}

__global__ void k_copy_i64(const int64_t *src, int64_t *dst, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

template <int P>
static int launch_form(tw_patch *Pt, int precision, int64_t *rp, int32_t *col, void *valv,
                       cudaStream_t s) {
  constexpr int T = P <= 5 ? 32 : 16;  // the tile's output buffer stays within static smem
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
    const unsigned gw = (unsigned)((Pt->ncutrows + 3) / 4);
    // gather rows exist iff there are element matrices and the method is not
    // naive WQ; block rows iff not every row is a gather row
    const bool gather = Pt->gmat && Pt->method != TW_METHOD_NAIVE;
    const bool block = !gather || Pt->method == TW_METHOD_DWQ;
    if (precision == TW_PREC_FP32) {
      if (gather)
        k_cutrows_gather<P, float><<<gw, 128, 0, s>>>(ra, Pt->cutrows, Pt->ncutrows, col,
                                                      (float *)valv);
      if (block)
        k_cutrows<P, float><<<Pt->ncutrows, 128, 0, s>>>(ra, Pt->cutrows, col, (float *)valv);
    } else {
      if (gather)
        k_cutrows_gather<P, double><<<gw, 128, 0, s>>>(ra, Pt->cutrows, Pt->ncutrows, col, val);
      if (block)
        k_cutrows<P, double><<<Pt->ncutrows, 128, 0, s>>>(ra, Pt->cutrows, col, val);
    }
    if (gather) TW_LAUNCH();
    if (block) TW_LAUNCH();
    prof_stop(ps, TW_STAGE_CUTROWS, s);
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
