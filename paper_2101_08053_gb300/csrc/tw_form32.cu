// tw_form32.cu -- the interior-row contraction (Eq. 7) on the FP32 pipes.
//
// On GB300 the FP32 FMA rate is ~58x the FP64 rate, so two reduced-precision
// forms of the sum-factorised WQ contraction are provided:
//   TW_PREC_FP32    tables rounded to FP32, FP32 FMA, float CSR values;
//   TW_PREC_FP32X2  split precision: every FP64 table value is kept as an
//                   unevaluated pair hi + lo of FP32 numbers, products are
//                   formed exactly (hi*hi by an FMA residual) and sums by
//                   TwoSum with the rounding errors carried in a second FP32
//                   accumulator, so the result keeps ~46 bits and is written
//                   as FP64.
// The tables (V of both directions, c on the WQ grid) are split once per
// patch, on first use.  Cut rows always run in FP64 (k_cutrows).
#include "tw_bodies.cuh"

namespace tw {

__device__ __forceinline__ float2 split_f64(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return make_float2(h, l);
}

__global__ void k_split_table(const double *src, float2 *dst, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = split_f64(src[i]);
}

template <int P, int T, bool SPLIT>
__global__ void __launch_bounds__(256) k_interior32(Dir A, Dir B, const float2 *__restrict__ Cf,
                                                    const float2 *__restrict__ V1f,
                                                    const float2 *__restrict__ V2f,
                                                    const uint8_t *__restrict__ fstate,
                                                    const int32_t *__restrict__ act,
                                                    const int64_t *__restrict__ rp,
                                                    int32_t *__restrict__ col, void *__restrict__ valv) {
  __shared__ __align__(16) char smem[interior32_smem(P, T, SPLIT)];
  interior_tile32<P, SPLIT>(A, B, Cf, V1f, V2f, fstate, act, rp, col, valv, blockIdx.y,
                            blockIdx.x * T, T, smem);
}

// split the patch's tables on first use (patch-owned)
int ensure_split_tables(tw_patch *P, cudaStream_t s) {
  if (P->Cf) return 0;
  Dir &A = P->d[0];
  Dir &B = P->d[1];
  cudaStream_t keep = P->stream;
  P->stream = s;
  const int W = 2 * P->p + 1;
  int64_t nc = (int64_t)A.nq * B.nq;
  int64_t nv[2] = {(int64_t)A.n * A.qmax * W, (int64_t)B.n * B.qmax * W};
  float2 *cf = (float2 *)dalloc(P, sizeof(float2) * nc);
  float2 *v0 = (float2 *)dalloc(P, sizeof(float2) * nv[0]);
  float2 *v1 = (float2 *)dalloc(P, sizeof(float2) * nv[1]);
  P->stream = keep;
  if (!cf || !v0 || !v1) return TW_ENOMEM;
  k_split_table<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(P->C, cf, nc);
  TW_LAUNCH();
  k_split_table<<<(unsigned)((nv[0] + 255) / 256), 256, 0, s>>>(A.V, v0, nv[0]);
  TW_LAUNCH();
  k_split_table<<<(unsigned)((nv[1] + 255) / 256), 256, 0, s>>>(B.V, v1, nv[1]);
  TW_LAUNCH();
  P->Cf = cf;
  P->Vf[0] = v0;
  P->Vf[1] = v1;
  return check_cuda(cudaGetLastError(), "split tables");
}

// tiles as large as the static shared memory allows for the staged outputs:
// split (FP64 outputs) 32 rows (16 at p = 6), FP32 64 rows (32 at p = 6)
template <int P>
static void launch32(tw_patch *Pt, bool split, int32_t *col, void *val, cudaStream_t s) {
  constexpr int TS = P <= 5 ? 32 : 16, TF = P <= 5 ? 64 : 32;
  static_assert(interior32_smem(P, TS, true) <= 48 * 1024, "split tile exceeds static smem");
  static_assert(interior32_smem(P, TF, false) <= 48 * 1024, "FP32 tile exceeds static smem");
  Dir &A = Pt->d[0];
  Dir &B = Pt->d[1];
  if (split)
    k_interior32<P, TS, true><<<dim3((A.n + TS - 1) / TS, B.n), 256, 0, s>>>(
        A, B, Pt->Cf, Pt->Vf[0], Pt->Vf[1], Pt->fstate, Pt->act, Pt->row_ptr, col, val);
  else
    k_interior32<P, TF, false><<<dim3((A.n + TF - 1) / TF, B.n), 256, 0, s>>>(
        A, B, Pt->Cf, Pt->Vf[0], Pt->Vf[1], Pt->fstate, Pt->act, Pt->row_ptr, col, val);
}

int launch_interior32(tw_patch *P, int precision, int32_t *col, void *val, cudaStream_t s) {
  int rc = ensure_split_tables(P, s);
  if (rc) return rc;
  if (P->n_interior == 0) return 0;
  bool split = precision == TW_PREC_FP32X2;
  int ps = prof_start(s);
  switch (P->p) {
    case 1: launch32<1>(P, split, col, val, s); break;
    case 2: launch32<2>(P, split, col, val, s); break;
    case 3: launch32<3>(P, split, col, val, s); break;
    case 4: launch32<4>(P, split, col, val, s); break;
    case 5: launch32<5>(P, split, col, val, s); break;
    case 6: launch32<6>(P, split, col, val, s); break;
    default: return TW_EUNSUPPORTED;
  }
  prof_stop(ps, TW_STAGE_INTERIOR, s);
  TW_LAUNCH();
  return check_cuda(cudaGetLastError(), "interior contraction (FP32 pipes)");
}

}  // namespace tw
