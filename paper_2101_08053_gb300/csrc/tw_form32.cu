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
#include "tw_internal.cuh"

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

template <int P, int T, bool SPLIT>
__global__ void __launch_bounds__(256) k_interior32(Dir A, Dir B, const float2 *__restrict__ Cf,
                                                    const float2 *__restrict__ V1f,
                                                    const float2 *__restrict__ V2f,
                                                    const uint8_t *__restrict__ fstate,
                                                    const int32_t *__restrict__ act,
                                                    const int64_t *__restrict__ rp,
                                                    int32_t *__restrict__ col, void *__restrict__ valv) {
  constexpr int W = 2 * P + 1;
  constexpr int KMAX = (2 * T + 4 * P + 4) | 1;
  __shared__ float2 Y[W * KMAX];
  __shared__ float2 V2s[TW_QMAX * W];
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
  for (int t = threadIdx.x; t < qc2 * W; t += blockDim.x) V2s[t] = V2f[(size_t)i2 * B.qmax * W + t];
  for (int t = threadIdx.x; t < W; t += blockDim.x) cr2[t] = B.crange[i2 * W + t];
  __syncthreads();
  // stage 1: Y[r2][k1] = sum_{k2} V2[i2][k2][r2] c[k2][k1]
  for (int idx = threadIdx.x; idx < W * K; idx += blockDim.x) {
    const int r2 = idx / K, kk = idx - r2 * K;
    const int lo = cr2[r2] & 0xffff, hi = cr2[r2] >> 16;
    const float2 *cc = Cf + (size_t)(qb2 + lo) * A.nq + kA + kk;
    float sh = 0.f, sl = 0.f;
    for (int c2 = lo; c2 < hi; c2++, cc += A.nq) {
      if (SPLIT) df_fma(V2s[c2 * W + r2], *cc, sh, sl);
      else sh = fmaf(V2s[c2 * W + r2].x, cc->x, sh);
    }
    Y[r2 * KMAX + kk] = make_float2(sh, sl);
  }
  __syncthreads();
  // stage 2 (point-major for rows away from the end elements)
  const int lo2 = max(0, i2 - P);
  const int NR = (i1b - i1a) * W;
  double *vald = (double *)valv;
  float *valf = (float *)valv;
  for (int idx = threadIdx.x; idx < NR; idx += blockDim.x) {
    const int t = idx / W, r2 = idx - t * W;
    const int i1 = i1a + t;
    const int g = i2 * n1 + i1;
    const int j2 = i2 - P + r2;
    if (fstate[g] != TW_FUNC_INTERIOR || j2 < 0 || j2 >= B.n) continue;
    const float2 *y = Y + r2 * KMAX + (A.qbeg[i1] - kA);
    const float2 *v = V1f + ((size_t)i1 * A.qmax) * W;
    const int64_t rowbase = rp[act[g]];
    if (i1 >= P + 1 && i1 <= A.nel - 2) {
      float ah[W], al[W];
#pragma unroll
      for (int r = 0; r < W; r++) ah[r] = al[r] = 0.f;
#pragma unroll
      for (int el = 0; el <= P; el++) {
#pragma unroll
        for (int pt = 0; pt < 2; pt++) {
          const int c1 = 2 * el + pt;
          const float2 yv = y[c1];
#pragma unroll
          for (int a = 0; a <= P; a++) {
            if (SPLIT) df_fma(v[c1 * W + el + a], yv, ah[el + a], al[el + a]);
            else ah[el + a] = fmaf(v[c1 * W + el + a].x, yv.x, ah[el + a]);
          }
        }
      }
      const int64_t base = rowbase + (int64_t)(j2 - lo2) * W;
      const int32_t *arow = act + j2 * n1 + (i1 - P);
#pragma unroll
      for (int r = 0; r < W; r++) {
        if (SPLIT) vald[base + r] = (double)ah[r] + (double)al[r];
        else valf[base + r] = ah[r];
        col[base + r] = arow[r];
      }
    } else {
      const int lo1 = max(0, i1 - P), w1 = min(n1 - 1, i1 + P) - lo1 + 1;
      for (int r1 = 0; r1 < W; r1++) {
        const int j1 = i1 - P + r1;
        if (j1 < 0 || j1 >= n1) continue;
        const int cr = A.crange[i1 * W + r1];
        const int lo = cr & 0xffff, hi = cr >> 16;
        float sh = 0.f, sl = 0.f;
        for (int c1 = lo; c1 < hi; c1++) {
          if (SPLIT) df_fma(v[c1 * W + r1], y[c1], sh, sl);
          else sh = fmaf(v[c1 * W + r1].x, y[c1].x, sh);
        }
        const int64_t pos = rowbase + (int64_t)(j2 - lo2) * w1 + (j1 - lo1);
        if (SPLIT) vald[pos] = (double)sh + (double)sl;
        else valf[pos] = sh;
        col[pos] = act[j2 * n1 + j1];
      }
    }
  }
}

// split the patch's tables on first use (patch-owned)
static int ensure_split_tables(tw_patch *P, cudaStream_t s) {
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

template <int P>
static void launch32(tw_patch *Pt, bool split, int32_t *col, void *val, cudaStream_t s) {
  constexpr int T = 32;
  Dir &A = Pt->d[0];
  Dir &B = Pt->d[1];
  dim3 grid((A.n + T - 1) / T, B.n);
  if (split)
    k_interior32<P, T, true><<<grid, 256, 0, s>>>(A, B, Pt->Cf, Pt->Vf[0], Pt->Vf[1], Pt->fstate,
                                                   Pt->act, Pt->row_ptr, col, val);
  else
    k_interior32<P, T, false><<<grid, 256, 0, s>>>(A, B, Pt->Cf, Pt->Vf[0], Pt->Vf[1], Pt->fstate,
                                                    Pt->act, Pt->row_ptr, col, val);
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
