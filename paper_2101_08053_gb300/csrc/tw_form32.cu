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
// The tables (V of both directions, c on the WQ grid, the band values of
// direction 1 per point) are split once per patch, on first use; each tile
// stages its slab of c and its rows of band values in shared memory with bulk
// copies and, when its CSR range is contiguous, writes it with bulk copies
// (interior_tile32).  Cut rows always run in FP64 (k_cutrows).
#include <algorithm>

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

// c as (hi, lo) float pairs with rows padded to ld pairs, so that every row
// starts on 16 bytes for the bulk copies (the pad columns are zero; nq1 is odd
// for some mixed-continuity vectors)
__global__ void k_split_rows(const double *src, float2 *dst, int n1, int n2, int ld) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n2 * ld) return;
  const int k2 = (int)(i / ld), k1 = (int)(i % ld);
  dst[i] = k1 < n1 ? split_f64(src[(size_t)k2 * n1 + k1]) : make_float2(0.f, 0.f);
}

// c rounded to float with rows padded to ld (the pad columns are zero)
__global__ void k_round_rows(const double *src, float *dst, int n1, int n2, int ld) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n2 * ld) return;
  const int k2 = (int)(i / ld), k1 = (int)(i % ld);
  dst[i] = k1 < n1 ? __double2float_rn(src[(size_t)k2 * n1 + k1]) : 0.f;
}

// Vc[i][c1][a] = V[i][c1][c1 / 2 + a], a = 0..P: the band values that can be
// nonzero at point c1 of supp B_i when every support element holds two points
// (D.two: rows P+1 .. nel-2 for simple knots); zero elsewhere and in the pad
// row n
__global__ void k_band_table(Dir D, float2 *vcf, float *vch) {
  const int P = D.p, W = 2 * P + 1, NV = (2 * P + 2) * (P + 1);
  int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)(D.n + 1) * NV) return;
  const int i = (int)(id / NV), r = (int)(id % NV), c1 = r / (P + 1), a = r % (P + 1);
  double v = 0.0;
  if (i < D.n && D.two[i]) v = D.V[((size_t)i * D.qmax + c1) * W + c1 / 2 + a];
  const float2 h = split_f64(v);
  vcf[id] = h;
  vch[id] = h.x;
}

// threads of a one-patch block: one per stage-2 item of the tile (a row and
// one r2; a row and two neighbouring r2 in FP32 below p = 6), rounded to
// warps, so that no phase of the tile leaves a large part of the block waiting
__host__ __device__ constexpr int interior32_threads(int P, int T, bool split) {
  return (T * ((split || P >= 6) ? 2 * P + 1 : P + 1) + 31) / 32 * 32;
}

// MIXED: the patch has a repeated knot (runtime layout from kmax and q, the
// two-point and whole-band tests); otherwise the static layout of simple knots
template <int P, int T, bool SPLIT, bool MIXED>
__global__ void __launch_bounds__(interior32_threads(P, T, SPLIT))
    k_interior32(Dir A, Dir B, Tables32 tb,
                                                    const uint8_t *__restrict__ fstate,
                                                    const int32_t *__restrict__ act,
                                                    const int64_t *__restrict__ rp,
                                                    int32_t *__restrict__ col, void *__restrict__ valv,
                                                    int *flag, int kmax, int q) {
  extern __shared__ __align__(16) char smem[];
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  uint32_t phase = 0;
  interior_tile32<P, SPLIT>(A, B, tb, fstate, act, rp, col, valv, blockIdx.y, blockIdx.x * T, T,
                            smem, &bar, &phase, flag, MIXED, MIXED ? kmax : 0, MIXED ? q : 0);
}

// split the patch's tables on first use (patch-owned)
int ensure_split_tables(tw_patch *P, cudaStream_t s) {
  if (P->Cf) return 0;
  Dir &A = P->d[0];
  Dir &B = P->d[1];
  cudaStream_t keep = P->stream;
  P->stream = s;
  const int W = 2 * P->p + 1;
  const int NV = (2 * P->p + 2) * (P->p + 1);
  const int ldh = (A.nq + 3) & ~3, ldf = (A.nq + 1) & ~1;  // 16-byte rows
  int64_t nc = (int64_t)B.nq * ldf, nh = (int64_t)B.nq * ldh;
  int64_t nv[2] = {(int64_t)A.n * A.qmax * W, (int64_t)B.n * B.qmax * W};
  int64_t nb = (int64_t)(A.n + 1) * NV;
  float2 *cf = (float2 *)dalloc(P, sizeof(float2) * nc);
  float2 *v0 = (float2 *)dalloc(P, sizeof(float2) * nv[0]);
  float2 *v1 = (float2 *)dalloc(P, sizeof(float2) * nv[1]);
  float *ch = (float *)dalloc(P, sizeof(float) * nh);
  float2 *vcf = (float2 *)dalloc(P, sizeof(float2) * nb);
  float *vch = (float *)dalloc(P, sizeof(float) * nb);
  P->stream = keep;
  if (!cf || !v0 || !v1 || !ch || !vcf || !vch) return TW_ENOMEM;
  k_split_rows<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(P->C, cf, A.nq, B.nq, ldf);
  TW_LAUNCH();
  k_split_table<<<(unsigned)((nv[0] + 255) / 256), 256, 0, s>>>(A.V, v0, nv[0]);
  TW_LAUNCH();
  k_split_table<<<(unsigned)((nv[1] + 255) / 256), 256, 0, s>>>(B.V, v1, nv[1]);
  TW_LAUNCH();
  k_round_rows<<<(unsigned)((nh + 255) / 256), 256, 0, s>>>(P->C, ch, A.nq, B.nq, ldh);
  TW_LAUNCH();
  k_band_table<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(A, vcf, vch);
  TW_LAUNCH();
  P->Cf = cf;
  P->ldf = ldf;
  P->Vf[0] = v0;
  P->Vf[1] = v1;
  P->Ch = ch;
  P->ldh = ldh;
  P->Vcf = vcf;
  P->Vch = vch;
  return check_cuda(cudaGetLastError(), "split tables");
}

Tables32 tables32(const tw_patch *P, bool split, const void *col, const void *val) {
  Tables32 tb;
  tb.C = split ? (const void *)P->Cf : (const void *)P->Ch;
  tb.ldc = split ? P->ldf : P->ldh;
  tb.Vc1 = split ? (const void *)P->Vcf : (const void *)P->Vch;
  tb.V1f = P->Vf[0];
  tb.V2f = P->Vf[1];
  tb.bulk_out = ((uintptr_t)col % 16 == 0 && (uintptr_t)val % 16 == 0) ? 1 : 0;
  return tb;
}

// tiles of 32 rows for FP32 and 16 for split precision (half of that at
// p = 6): values and columns of a tile are staged in shared memory for its
// bulk stores, and these heights keep 6 blocks resident per SM
template <int P, bool SPLIT>
static cudaError_t launch32_t(tw_patch *Pt, int32_t *col, void *val, cudaStream_t s) {
  constexpr int T = (SPLIT ? 16 : 32) / (P <= 5 ? 1 : 2);
  constexpr int LT = (SPLIT ? 4 : 5) - (P <= 5 ? 0 : 1);  // log2 T
  static_assert(interior32_smem(P, T, SPLIT) <= 200 * 1024, "FP32-pipe tile exceeds shared memory");
  Dir &A = Pt->d[0];
  Dir &B = Pt->d[1];
  // the static bounds for simple knots; a mixed-continuity vector's own
  const int kmax = std::max(interior32_kmax(P, T), Pt->ktile[LT] | 1);
  const int q = std::max(4 * P, std::max(A.qmax, B.qmax));
  const dim3 grid((A.n + T - 1) / T, B.n);
  const int nt = interior32_threads(P, T, SPLIT);
  const Tables32 tb = tables32(Pt, SPLIT, col, val);
  if (!Pt->mixed) {
    constexpr size_t smem = interior32_smem(P, T, SPLIT);
    cudaError_t e = cudaFuncSetAttribute(k_interior32<P, T, SPLIT, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_interior32<P, T, SPLIT, false><<<grid, nt, smem, s>>>(A, B, tb, Pt->fstate, Pt->act,
                                                            Pt->row_ptr, col, val, Pt->flag, 0, 0);
    return cudaSuccess;
  }
  const size_t smem = interior32_layout(P, T, SPLIT, kmax, q).total;
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_interior32<P, T, SPLIT, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_interior32<P, T, SPLIT, true><<<grid, nt, smem, s>>>(A, B, tb, Pt->fstate, Pt->act,
                                                         Pt->row_ptr, col, val, Pt->flag, kmax, q);
  return cudaSuccess;
}

template <int P>
static cudaError_t launch32(tw_patch *Pt, bool split, int32_t *col, void *val, cudaStream_t s) {
  return split ? launch32_t<P, true>(Pt, col, val, s) : launch32_t<P, false>(Pt, col, val, s);
}

int launch_interior32(tw_patch *P, int precision, int32_t *col, void *val, cudaStream_t s) {
  int rc = ensure_split_tables(P, s);
  if (rc) return rc;
  if (P->n_interior == 0) return 0;
  bool split = precision == TW_PREC_FP32X2;
  int ps = prof_start(s);
  cudaError_t e = cudaErrorInvalidValue;
  switch (P->p) {
    case 1: e = launch32<1>(P, split, col, val, s); break;
    case 2: e = launch32<2>(P, split, col, val, s); break;
    case 3: e = launch32<3>(P, split, col, val, s); break;
    case 4: e = launch32<4>(P, split, col, val, s); break;
    case 5: e = launch32<5>(P, split, col, val, s); break;
    case 6: e = launch32<6>(P, split, col, val, s); break;
    default: return TW_EUNSUPPORTED;
  }
  prof_stop(ps, TW_STAGE_INTERIOR, s);
  TW_LAUNCH();
  if (e != cudaSuccess) return check_cuda(e, "interior contraction (FP32 pipes): attributes");
  return check_cuda(cudaGetLastError(), "interior contraction (FP32 pipes)");
}

}  // namespace tw
