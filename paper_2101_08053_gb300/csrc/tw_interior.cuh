// tw_interior.cuh -- the interior-row tile of the FP64 formation (Sect. 2.1,
// Eqs. 6-7): weighted quadrature with sum factorisation, row-based, one tile of
// T consecutive test functions i1 of one i2 per item.  Used by the one-patch
// kernel k_interior (tw_form.cu) and the persistent batched kernel.
#pragma once

#include "tw_internal.cuh"

namespace tw {

// smem of one interior tile: Y[W * kmax] | V2s[TW_QMAX * W] | the tile's
// outputs [T][W][W] (written out row by row with coalesced stores) | cr2[W] | flag.
// kmax (odd) bounds the WQ points under the tile's T rows: interior_kmax for
// simple knots; a mixed-continuity vector (more points next to repeated knots)
// passes its own bound.
__host__ __device__ constexpr int interior_kmax(int P, int T) { return (2 * T + 4 * P + 4) | 1; }
__host__ __device__ constexpr size_t interior_out_off(int P, int T, int kmax) {
  return sizeof(double) * ((size_t)(2 * P + 1) * kmax + TW_QMAX * (2 * P + 1));
}
__host__ __device__ constexpr size_t interior_smem(int P, int T, int kmax) {
  return interior_out_off(P, T, kmax) + sizeof(double) * (size_t)T * (2 * P + 1) * (2 * P + 1) +
         sizeof(int) * (2 * P + 2);
}
__host__ __device__ constexpr size_t interior_smem(int P, int T) {
  return interior_smem(P, T, interior_kmax(P, T));
}

template <int P>
__device__ void interior_tile(const Dir &A, const Dir &B, const double *__restrict__ C,
                              const uint8_t *__restrict__ fstate, const int32_t *__restrict__ act,
                              const int64_t *__restrict__ rp, int32_t *__restrict__ col,
                              double *__restrict__ val, int i2, int i1a, int T, char *smem,
                              int KMAX, bool mixed) {
  constexpr int W = 2 * P + 1;
  double *Y = (double *)smem;
  double *V2s = Y + W * KMAX;
  double *os = (double *)(smem + interior_out_off(P, T, KMAX));  // [t][r2][r1]
  int *cr2 = (int *)(os + (size_t)T * W * W);
  int *anyintp = cr2 + W;
  const int i1b = min(A.n, i1a + T);
  const int n1 = A.n;
  if (threadIdx.x == 0) *anyintp = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < i1b - i1a; t += blockDim.x)
    if (fstate[i2 * n1 + i1a + t] == TW_FUNC_INTERIOR) *anyintp = 1;
  __syncthreads();
  if (!*anyintp) return;  // uniform across the block
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
  // stage 2.  Rows whose support elements all hold 2 points away from the end
  // elements (A.two; full band) take the point-major path: thread (row, r2) walks the
  // 2(P+1) points of supp B_i1 and adds each point's value into the P+1
  // outputs whose trial function lives on the point's element, so every lane
  // issues the same (P+1)*2*(P+1) DFMAs.  Other rows use the per-output loop.
  const int NR = (i1b - i1a) * W;
  for (int idx = threadIdx.x; idx < NR; idx += blockDim.x) {
    const int t = idx / W, r2 = idx - t * W;
    const int i1 = i1a + t;
    const int g = i2 * n1 + i1;
    const int j2 = i2 - P + r2;
    if (fstate[g] != TW_FUNC_INTERIOR || j2 < 0 || j2 >= B.n) continue;
    const double *y = Y + r2 * KMAX + (A.qbeg[i1] - kA);
    const double *v = A.V + ((size_t)i1 * A.qmax) * W;
    double *o = os + ((size_t)t * W + r2) * W;
    if (i1 >= P + 1 && i1 <= A.nel - 2 && (!mixed || A.two[i1])) {
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
#pragma unroll
      for (int r = 0; r < W; r++) o[r] = acc[r];
    } else {
      for (int r1 = 0; r1 < W; r1++) {
        const int j1 = i1 - P + r1;
        if (j1 < 0 || j1 >= n1) continue;
        const int cr = A.crange[i1 * W + r1];
        const int lo = cr & 0xffff, hi = cr >> 16;
        double s = 0.0;
        for (int c1 = lo; c1 < hi; c1++) s = fma(v[c1 * W + r1], y[c1], s);
        o[r1] = s;
      }
    }
  }
  __syncthreads();
  // write out: one warp per row of the tile, consecutive lanes on consecutive
  // CSR positions (j2 major, j1 minor over the valid part of the band)
  const int nw = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lo2 = max(0, i2 - P), w2 = min(B.n - 1, i2 + P) - lo2 + 1, d2 = lo2 - (i2 - P);
  for (int t = wid; t < i1b - i1a; t += nw) {
    const int i1 = i1a + t, g = i2 * n1 + i1;
    if (fstate[g] != TW_FUNC_INTERIOR) continue;  // the whole warp
    const int lo1 = max(0, i1 - P), w1 = min(n1 - 1, i1 + P) - lo1 + 1, d1 = lo1 - (i1 - P);
    const int64_t rowbase = rp[act[g]];
    const double *src = os + (size_t)t * W * W;
    // every band neighbour active (always for simple knots)
    if (!mixed || rp[act[g] + 1] - rowbase == (int64_t)w1 * w2) {
      for (int k = lane; k < w1 * w2; k += 32) {
        const int q2 = k / w1, q1 = k - q2 * w1;
        val[rowbase + k] = src[(q2 + d2) * W + q1 + d1];
        col[rowbase + k] = act[(lo2 + q2) * n1 + lo1 + q1];
      }
    } else {  // a repeated knot: some neighbour shares only the empty span
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
  }
  __syncthreads();  // the tile's smem is reused by the next item
}

// MIXED: the patch has a repeated knot (runtime bound kmax, the two-point and
// whole-band tests); otherwise the static bound and layout of simple knots
template <int P, int T, bool MIXED>
__global__ void __launch_bounds__(256) k_interior(Dir A, Dir B, const double *__restrict__ C,
                                                  const uint8_t *__restrict__ fstate,
                                                  const int32_t *__restrict__ act,
                                                  const int64_t *__restrict__ rp,
                                                  int32_t *__restrict__ col,
                                                  double *__restrict__ val, int kmax) {
  if constexpr (MIXED) {
    extern __shared__ __align__(16) char dsmem[];  // interior_smem(P, T, kmax) bytes
    interior_tile<P>(A, B, C, fstate, act, rp, col, val, blockIdx.y, blockIdx.x * T, T, dsmem,
                     kmax, true);
  } else {
    __shared__ __align__(16) char smem[interior_smem(P, T)];
    interior_tile<P>(A, B, C, fstate, act, rp, col, val, blockIdx.y, blockIdx.x * T, T, smem,
                     interior_kmax(P, T), false);
  }
}

}  // namespace tw
