// Extended B-splines of a trimmed patch (Hoellig, Reif and Wipper), which the
// paper uses to keep the mass matrix of every L2 projection well conditioned
// (Sect. 3, Sect. 4.2).  The paper defers the construction to the literature;
// these readings fix it for a tensor-product patch:
//  R15  an active function is inner when at least one element of its support
//       is regular, outer otherwise;
//  R16  outer j = (j1, j2) is tied to the all-inner array l + {0..p}^2 with
//       l_v in [j_v - 2p - 1, j_v + p + 1] whose centre l + p/2 is nearest to j
//       (squared index distance), ties to the smaller l2, then l1;
//  R17  e_{i,j} = e1 * e2, each 1-D factor the coefficients that carry the
//       B-spline coefficients of every polynomial of degree <= p from the
//       array to j (polynomial reproduction).
// With E (active x inner: identity rows for inner functions, e_{i,j} in the
// columns of j's array for outer j) the extended basis has the mass matrix
// E^T M E and the right-hand side E^T b; its L2 projection solves
// E^T M_s E x = E^T b and returns u = E x.
#include <climits>
#include <mutex>

#include "tw_internal.cuh"

namespace tw {

#define TWF_EXT_REACH 64   // an outer function has no all-inner array within reach
#define TWF_EXT_CSR 128    // the CSR passed in is not the patch's pattern
#define TW_EXT_REACH 1     // R16: arrays start within [j - 2p - 1, j + p + 1]
#define TW_EXT_THREADS 256
#define TW_EXT_WARPS (TW_EXT_THREADS / 32)
// |b - a| <= 5p + 2 per direction for an entry (a, b) of E^T M E: a's
// transposed list reaches 2p + 1, M's band p, an outer function's array 2p + 1
#define TW_EXT_MAXW (5 * TW_MAXP + 2)
#define TW_EXT_MAXSIDE (2 * TW_EXT_MAXW + 1)
#define TW_EXT_WORDS ((TW_EXT_MAXSIDE * TW_EXT_MAXSIDE + 31) / 32)

// device view of the extension tables
struct Ext {
  int n1, n2, p, pp;        // pp = (p + 1)^2
  int64_t n_rows, n_inner, n_outer;
  const int32_t *act;       // g -> active row or -1
  const int32_t *rowg;      // active row -> g
  const int32_t *inng;      // g -> inner index or -1
  const int32_t *outg;      // g -> outer index or -1
  const int32_t *inner_g;   // inner index -> g
  const int32_t *ainn;      // active row -> inner index or -1
  const int32_t *aout;      // active row -> outer index or -1
  const int32_t *arr;       // outer index -> g of its array's first member l
  const int32_t *ocol;      // outer index x pp: inner indices of the array (a2-major)
  const double *oval;       // outer index x pp: e1[a1] * e2[a2]
  const uint8_t *near;      // inner index: member of some outer function's array
  const int64_t *et_rp;     // inner index -> its transposed list (E's column)
  const int32_t *et_r;      // active rows r with E[r][a] stored, ascending
  const double *et_e;       // E[r][a]
};

// R15: 1 for inner, 1 << 32 for outer, 0 for exterior (one scan counts both)
__global__ void k_ext_flags(Dir A, Dir B, const uint8_t *estate, const int32_t *act,
                            int64_t *fl) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)A.n * B.n) return;
  int64_t v = 0;
  if (act[g] >= 0) {
    const int i1 = (int)(g % A.n), i2 = (int)(g / A.n), p = A.p;
    int reg = 0;
    for (int e2 = max(0, i2 - p); e2 <= min(B.nel - 1, i2); e2++)
      for (int e1 = max(0, i1 - p); e1 <= min(A.nel - 1, i1); e1++)
        reg |= estate[e2 * A.nel + e1] == TW_ELEM_REGULAR;
    v = reg ? (int64_t)1 : ((int64_t)1 << 32);
  }
  fl[g] = v;
}

__global__ void k_ext_index(int64_t nf, const int64_t *fl, const int64_t *pos, int32_t *inng,
                            int32_t *outg, int32_t *inner_g, int32_t *outer_g) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nf) return;
  const int32_t ib = (int32_t)(pos[g] & 0xffffffff), ob = (int32_t)(pos[g] >> 32);
  inng[g] = -1;
  outg[g] = -1;
  if (fl[g] == 1) {
    inng[g] = ib;
    inner_g[ib] = (int32_t)g;
  } else if (fl[g] != 0) {
    outg[g] = ob;
    outer_g[ob] = (int32_t)g;
  }
}

// ok[l] = 1 when every member of the array l + {0..p}^2 is inner
__global__ void k_ext_arrays(int n1, int n2, int p, const int32_t *inng, uint8_t *ok) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)n1 * n2) return;
  const int l1 = (int)(g % n1), l2 = (int)(g / n1);
  int good = l1 + p < n1 && l2 + p < n2;
  for (int a2 = 0; a2 <= p && good; a2++)
    for (int a1 = 0; a1 <= p && good; a1++) good = inng[(l2 + a2) * n1 + l1 + a1] >= 0;
  ok[g] = (uint8_t)good;
}

// R17, one direction, by Marsden's identity: B_k's coefficient of (x - y)^p
// is psi_k(y) = prod_{r=1..p} (t_{k+r} - y), and the powers (x - y)^p span the
// polynomials of degree <= p, so sum_a e_a psi_{l+a}(y) = psi_j(y) for all y
// is polynomial reproduction.  Both sides are degree-p polynomials in y: the
// identity is imposed at p + 1 points of a local coordinate spanning the
// knots involved and solved by Gaussian elimination with partial pivoting.
__device__ void ext_coef_1d(const double *U, int p, int j, int l, double *e) {
  const int lo = min(j, l) + 1, hi = max(j, l + p) + p;
  const double c = 0.5 * (U[lo] + U[hi]), h = U[hi] - U[lo];
  double S[TW_MAXP1][TW_MAXP1 + 1];
  for (int m = 0; m <= p; m++) {
    const double y = -0.5 + (double)m / (double)p;
    for (int a = 0; a <= p + 1; a++) {
      const int k = a <= p ? l + a : j;  // column p + 1: the right-hand side
      double v = 1.0;
      for (int r = 1; r <= p; r++) v *= (U[k + r] - c) / h - y;
      S[m][a] = v;
    }
  }
  for (int cc = 0; cc <= p; cc++) {
    int piv = cc;
    for (int r = cc + 1; r <= p; r++)
      if (fabs(S[r][cc]) > fabs(S[piv][cc])) piv = r;
    if (piv != cc)
      for (int a = 0; a <= p + 1; a++) {
        const double t = S[cc][a];
        S[cc][a] = S[piv][a];
        S[piv][a] = t;
      }
    for (int r = cc + 1; r <= p; r++) {
      const double f = S[r][cc] / S[cc][cc];
      for (int a = cc; a <= p + 1; a++) S[r][a] -= f * S[cc][a];
    }
  }
  for (int a = p; a >= 0; a--) {
    double v = S[a][p + 1];
    for (int b = a + 1; b <= p; b++) v -= S[a][b] * e[b];
    e[a] = v / S[a][a];
  }
}

// R16 + R17 for each outer function
__global__ void k_ext_outer(Dir A, Dir B, int64_t n_outer, const int32_t *outer_g,
                            const uint8_t *ok, const int32_t *inng, int32_t *arr, int32_t *ocol,
                            double *oval, int *flag) {
  int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_outer) return;
  const int n1 = A.n, n2 = B.n, p = A.p, pp = (p + 1) * (p + 1);
  const int g = outer_g[o], j1 = g % n1, j2 = g / n1;
  int best = INT_MAX, b1 = -1, b2 = -1;
  for (int l2 = max(0, j2 - 2 * p - TW_EXT_REACH); l2 <= min(n2 - p - 1, j2 + p + TW_EXT_REACH);
       l2++)
    for (int l1 = max(0, j1 - 2 * p - TW_EXT_REACH);
         l1 <= min(n1 - p - 1, j1 + p + TW_EXT_REACH); l1++) {
      if (!ok[l2 * n1 + l1]) continue;
      const int d1 = 2 * l1 + p - 2 * j1, d2 = 2 * l2 + p - 2 * j2;
      const int d = d1 * d1 + d2 * d2;
      if (d < best) {  // scan order: l2, then l1 ascending
        best = d;
        b1 = l1;
        b2 = l2;
      }
    }
  if (b1 < 0) {
    atomicOr(flag, TWF_EXT_REACH);
    arr[o] = -1;
    for (int k = 0; k < pp; k++) {
      ocol[o * pp + k] = 0;
      oval[o * pp + k] = 0.0;
    }
    return;
  }
  double e1[TW_MAXP1], e2[TW_MAXP1];
  ext_coef_1d(A.U, p, j1, b1, e1);
  ext_coef_1d(B.U, p, j2, b2, e2);
  arr[o] = b2 * n1 + b1;
  for (int a2 = 0; a2 <= p; a2++)
    for (int a1 = 0; a1 <= p; a1++) {
      const int k = a2 * (p + 1) + a1;
      ocol[o * pp + k] = inng[(b2 + a2) * n1 + b1 + a1];
      oval[o * pp + k] = e1[a1] * e2[a2];
    }
}

__global__ void k_ext_mark(int64_t n, const int32_t *ocol, uint8_t *near) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) near[ocol[k]] = 1;
}

// E's column a (the transposed list): a's own row and every outer r whose
// array holds a, in ascending row order.  Outer r with a in its array lie in
// [a - 2p - 1, a + 2p + 1] per direction (R16).  count only (cnt) or fill.
__global__ void k_ext_tlist(Ext X, int64_t *cnt, int32_t *et_r, double *et_e) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= X.n_inner) return;
  const int n1 = X.n1, n2 = X.n2, p = X.p, R = 2 * p + TW_EXT_REACH;
  const int g = X.inner_g[a], a1 = g % n1, a2 = g / n1;
  int64_t k = cnt ? 0 : X.et_rp[a];
  const bool own_only = !X.near[a];
  for (int r2 = own_only ? a2 : max(0, a2 - R); r2 <= (own_only ? a2 : min(n2 - 1, a2 + R)); r2++)
    for (int r1 = own_only ? a1 : max(0, a1 - R); r1 <= (own_only ? a1 : min(n1 - 1, a1 + R));
         r1++) {
      const int gr = r2 * n1 + r1;
      double e;
      if (gr == g) {
        e = 1.0;
      } else {
        const int o = X.outg[gr];
        if (o < 0) continue;
        const int l = X.arr[o], l1 = l % n1, l2 = l / n1;
        if (a1 < l1 || a1 > l1 + p || a2 < l2 || a2 > l2 + p) continue;
        e = X.oval[(int64_t)o * X.pp + (a2 - l2) * (p + 1) + (a1 - l1)];
      }
      if (!cnt) {
        et_r[k] = X.act[gr];
        et_e[k] = e;
      }
      k++;
    }
  if (cnt) cnt[a] = k;
}

// ---------------------------------------------------------------------------
// E^T M E.  Row a is a plain copy of M's row when a is no array member and
// all its active neighbours are inner ("copy rows", almost all of them);
// otherwise ("near rows", next to the trim) its columns are the inner b
// reached through a's transposed list, M's band and the neighbours' arrays.
// The pattern is counted at build time as a bitmask over the window
// |b - a| <= 5p + 2 (one warp per row; atomicOr of bits is order-independent).
// A near row's values accumulate in a dense window of shared memory:
//   row a = sum_{r in col(a)} E[r][a] sum_{s in M's row r} M[r][s] E[s][.]
// with lanes prefetching 32 entries of M's row and the entries applied one
// after another (lanes over the array of an outer s), so every value is a
// fixed-order sum.

__device__ __forceinline__ bool ext_row_is_copy(const Ext &X, int64_t a, int lane, int *count) {
  const int n1 = X.n1, n2 = X.n2, p = X.p, w = 2 * p + 1;
  const int g = X.inner_g[a], a1 = g % n1, a2 = g / n1;
  int cnt = 0, out = 0;
  for (int c = lane; c < w * w; c += 32) {
    const int s1 = a1 + c % w - p, s2 = a2 + c / w - p;
    if (s1 < 0 || s1 >= n1 || s2 < 0 || s2 >= n2) continue;
    const int gs = s2 * n1 + s1;
    if (X.act[gs] < 0) continue;
    cnt++;
    out |= X.inng[gs] < 0;
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  *count = cnt;
  return !X.near[a] && !__any_sync(0xffffffffu, out);
}

// bitmask of row a's columns; returns false (after flagging) if a column
// fell outside the window, which the bound above rules out
__device__ bool ext_row_bits(const Ext &X, int64_t a, int lane, unsigned *bm, int W, int side,
                             int *flag) {
  const int n1 = X.n1, n2 = X.n2, p = X.p, w = 2 * p + 1;
  const int g = X.inner_g[a], a1 = g % n1, a2 = g / n1;
  const int words = (side * side + 31) >> 5;
  for (int k = lane; k < words; k += 32) bm[k] = 0u;
  __syncwarp();
  int bad = 0;
  for (int64_t t = X.et_rp[a]; t < X.et_rp[a + 1]; t++) {
    const int gr = X.rowg[X.et_r[t]], r1 = gr % n1, r2 = gr / n1;
    for (int c = lane; c < w * w; c += 32) {
      const int s1 = r1 + c % w - p, s2 = r2 + c / w - p;
      if (s1 < 0 || s1 >= n1 || s2 < 0 || s2 >= n2) continue;
      const int gs = s2 * n1 + s1;
      if (X.act[gs] < 0) continue;
      if (X.inng[gs] >= 0) {
        const int d1 = s1 - a1 + W, d2 = s2 - a2 + W;
        if (d1 < 0 || d1 >= side || d2 < 0 || d2 >= side) {
          bad = 1;
          continue;
        }
        const int idx = d2 * side + d1;
        atomicOr(&bm[idx >> 5], 1u << (idx & 31));
      } else {
        const int o = X.outg[gs], l = X.arr[o], l1 = l % n1, l2 = l / n1;
        for (int b2 = l2; b2 <= l2 + p; b2++)
          for (int b1 = l1; b1 <= l1 + p; b1++) {
            const int d1 = b1 - a1 + W, d2 = b2 - a2 + W;
            if (d1 < 0 || d1 >= side || d2 < 0 || d2 >= side) {
              bad = 1;
              continue;
            }
            const int idx = d2 * side + d1;
            atomicOr(&bm[idx >> 5], 1u << (idx & 31));
          }
      }
    }
  }
  __syncwarp();
  if (__any_sync(0xffffffffu, bad)) {
    if (lane == 0) atomicOr(flag, TWF_EXT_CSR);
    return false;
  }
  return true;
}

__global__ void __launch_bounds__(TW_EXT_THREADS)
    k_ext_xcount(Ext X, int64_t *cnt, int32_t *near_row, int *flag) {
  __shared__ unsigned bm_all[TW_EXT_WARPS][TW_EXT_WORDS];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t a = (int64_t)blockIdx.x * TW_EXT_WARPS + wib;
  if (a >= X.n_inner) return;
  int c;
  const bool copy = ext_row_is_copy(X, a, lane, &c);
  if (lane == 0) near_row[a] = !copy;
  if (copy) {
    if (lane == 0) cnt[a] = c;
    return;
  }
  const int W = 5 * X.p + 2, side = 2 * W + 1;
  unsigned *bm = bm_all[wib];
  if (!ext_row_bits(X, a, lane, bm, W, side, flag)) {
    if (lane == 0) cnt[a] = 0;
    return;
  }
  const int words = (side * side + 31) >> 5;
  int n = 0;
  for (int k = lane; k < words; k += 32) n += __popc(bm[k]);
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if (lane == 0) cnt[a] = n;
}

__global__ void __launch_bounds__(TW_EXT_THREADS)
    k_ext_xcopy(Ext X, const int32_t *near_row, const int64_t *rp, const int32_t *col,
                const double *val, const int64_t *xrp, int32_t *xcol, double *xval, int *flag) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t a = (int64_t)blockIdx.x * TW_EXT_WARPS + wib;
  if (a >= X.n_inner || near_row[a]) return;
  const int64_t x0 = xrp[a], len = xrp[a + 1] - x0;
  const int32_t r = X.act[X.inner_g[a]];
  const int64_t m0 = rp[r];
  if (rp[r + 1] - m0 != len) {
    if (lane == 0) atomicOr(flag, TWF_EXT_CSR);
    return;
  }
  int bad = 0;
  for (int64_t k = lane; k < len; k += 32) {
    const int32_t s = col[m0 + k];
    const int32_t b = (s >= 0 && s < X.n_rows) ? X.ainn[s] : -1;
    bad |= b < 0;
    xcol[x0 + k] = b < 0 ? 0 : b;
    xval[x0 + k] = val[m0 + k];
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flag, TWF_EXT_CSR);
}

#define TW_EXT_NEAR_WARPS 4
// dynamic shared memory of k_ext_xnear for degree p: per warp the value
// window (side^2 doubles) and its bitmask, in 4-byte words, rounded up to an
// even count so that every warp's window starts 8-byte aligned
__host__ __device__ __forceinline__ size_t ext_near_words(int p) {
  const int side = 2 * (5 * p + 2) + 1, cells = side * side;
  const size_t w = (size_t)cells * 2 + (((size_t)cells + 31) / 32);
  return (w + 1) & ~(size_t)1;
}

__global__ void __launch_bounds__(32 * TW_EXT_NEAR_WARPS)
    k_ext_xnear(Ext X, const int32_t *near_list, int64_t n_near, const int64_t *rp,
                const int32_t *col, const double *val, const int64_t *xrp, int32_t *xcol,
                double *xval, int *flag) {
  extern __shared__ double ext_dyn[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t ni = (int64_t)blockIdx.x * TW_EXT_NEAR_WARPS + wib;
  if (ni >= n_near) return;
  const int p = X.p, p1 = p + 1, pp = X.pp, n1 = X.n1;
  const int W = 5 * p + 2, side = 2 * W + 1, cells = side * side, words = (cells + 31) >> 5;
  double *cv = (double *)((unsigned *)ext_dyn + (size_t)wib * ext_near_words(p));
  unsigned *bm = (unsigned *)(cv + cells);
  const int32_t a = near_list[ni];
  const int g = X.inner_g[a], a1 = g % n1, a2 = g / n1;
  for (int k = lane; k < cells; k += 32) cv[k] = 0.0;
  for (int k = lane; k < words; k += 32) bm[k] = 0u;
  __syncwarp();
  int bad = 0;
  for (int64_t t = X.et_rp[a]; t < X.et_rp[a + 1]; t++) {
    const int32_t r = X.et_r[t];
    const double er = X.et_e[t];
    const int64_t k_end = rp[r + 1];
    for (int64_t k0 = rp[r]; k0 < k_end; k0 += 32) {
      // lane j prefetches entry k0 + j: its weight and where it lands
      const int64_t k = k0 + lane;
      int cell = -1, o = -1;  // inner s: its cell; outer s: its index and array corner
      int c1 = 0, c2 = 0;
      double mv = 0.0;
      if (k < k_end) {
        const int32_t s = col[k];
        if (s < 0 || s >= X.n_rows) {
          bad = 1;
        } else {
          mv = er * val[k];
          const int32_t bi = X.ainn[s];
          if (bi >= 0) {
            const int gb = X.inner_g[bi];
            const int d1 = gb % n1 - a1 + W, d2 = gb / n1 - a2 + W;
            if (d1 < 0 || d1 >= side || d2 < 0 || d2 >= side) bad = 1;
            else cell = d2 * side + d1;
          } else {
            const int oo = X.aout[s];
            const int l = X.arr[oo];
            c1 = l % n1 - a1 + W;
            c2 = l / n1 - a2 + W;
            if (c1 < 0 || c1 + p >= side || c2 < 0 || c2 + p >= side) bad = 1;
            else o = oo;
          }
        }
      }
      const int nk = (int)min((int64_t)32, k_end - k0);
      for (int j = 0; j < nk; j++) {
        const double mj = __shfl_sync(0xffffffffu, mv, j);
        const int cj = __shfl_sync(0xffffffffu, cell, j);
        const int oj = __shfl_sync(0xffffffffu, o, j);
        const int q1 = __shfl_sync(0xffffffffu, c1, j), q2 = __shfl_sync(0xffffffffu, c2, j);
        if (cj >= 0) {
          if (lane == 0) {
            cv[cj] += mj;
            bm[cj >> 5] |= 1u << (cj & 31);
          }
        } else if (oj >= 0) {
          for (int q = lane; q < pp; q += 32) {
            const int c = (q2 + q / p1) * side + q1 + q % p1;
            cv[c] = fma(mj, X.oval[(int64_t)oj * pp + q], cv[c]);
            atomicOr(&bm[c >> 5], 1u << (c & 31));
          }
        }
        __syncwarp();
      }
    }
  }
  if (__any_sync(0xffffffffu, bad)) {
    if (lane == 0) atomicOr(flag, TWF_EXT_CSR);
    return;
  }
  // write the window's cells in ascending g order (row-major in (b2, b1))
  const int64_t x0 = xrp[a], len = xrp[a + 1] - x0;
  int64_t base = 0;
  for (int w0 = 0; w0 < words; w0 += 32) {
    const int wi = w0 + lane;
    unsigned bits = wi < words ? bm[wi] : 0u;
    const int nb = __popc(bits);
    int incl = nb;
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += v;
    }
    int64_t k = base + incl - nb;
    while (bits) {
      const int bit = __ffs(bits) - 1;
      bits &= bits - 1;
      const int idx = wi * 32 + bit;
      const int b1 = a1 + idx % side - W, b2 = a2 + idx / side - W;
      if (k < len) {
        xcol[x0 + k] = X.inng[b2 * n1 + b1];
        xval[x0 + k] = cv[idx];
      }
      k++;
    }
    base += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (base != len && lane == 0) atomicOr(flag, TWF_EXT_CSR);
}

__global__ void k_ext_amaps(int64_t nf, const int32_t *act, const int32_t *inng,
                            const int32_t *outg, int32_t *ainn, int32_t *aout) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nf || act[g] < 0) return;
  ainn[act[g]] = inng[g];
  aout[act[g]] = outg[g];
}

__global__ void k_ext_compact(int64_t n, const int32_t *flag, const int32_t *pos, int32_t *list) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flag[i]) list[pos[i]] = (int32_t)i;
}

// E^T y (inner) and E x (active)
__global__ void k_ext_restrict(Ext X, const double *y, double *out) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= X.n_inner) return;
  double v = 0.0;
  for (int64_t t = X.et_rp[a]; t < X.et_rp[a + 1]; t++) v += X.et_e[t] * y[X.et_r[t]];
  out[a] = v;
}

__global__ void k_ext_expand(Ext X, const double *x, double *u) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= X.n_rows) return;
  const int g = X.rowg[r];
  const int32_t i = X.inng[g];
  if (i >= 0) {
    u[r] = x[i];
    return;
  }
  const int64_t o = X.outg[g];
  double v = 0.0;
  for (int k = 0; k < X.pp; k++) v += X.oval[o * X.pp + k] * x[X.ocol[o * X.pp + k]];
  u[r] = v;
}

// E as CSR: row r holds one entry (inner) or the array's pp entries (outer)
__global__ void k_ext_ecsr(Ext X, const int64_t *pos, int64_t *erp, int32_t *ecol, double *eval) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > X.n_rows) return;
  if (r == X.n_rows) {
    erp[r] = X.n_inner + X.n_outer * X.pp;
    return;
  }
  const int g = X.rowg[r];
  const int64_t e0 = (pos[g] & 0xffffffff) + (pos[g] >> 32) * X.pp;
  erp[r] = e0;
  const int32_t i = X.inng[g];
  if (i >= 0) {
    ecol[e0] = i;
    eval[e0] = 1.0;
    return;
  }
  const int64_t o = X.outg[g];
  for (int k = 0; k < X.pp; k++) {
    ecol[e0 + k] = X.ocol[o * X.pp + k];
    eval[e0 + k] = X.oval[o * X.pp + k];
  }
}

// ---------------------------------------------------------------------------
// host side

struct ExtTables {
  Ext X;
  int64_t *pos;      // g: packed (inner before, outer before)
  int64_t *xrp;      // E^T M E row pointer (n_inner + 1)
  int32_t *near_row; // inner index: 1 for a near row (not a copy of M's row)
  int32_t *near_list;
  int64_t nnz_x, nnz_t, n_near;
};

static int ext_flag(tw_patch *P, const char *what) {
  int f = 0;
  if (check_cuda(cudaMemcpyAsync(&f, P->flag, sizeof(int), cudaMemcpyDeviceToHost, P->stream),
                 what))
    return TW_ECUDA;
  if (check_cuda(cudaStreamSynchronize(P->stream), what)) return TW_ECUDA;
  if (f & TWF_EXT_REACH) {
    set_error("%s: an outer function has no all-inner (p+1)^2 array within reach; the patch "
              "is too coarse for its trim",
              what);
    return TW_EUNSUPPORTED;
  }
  if (f & TWF_EXT_CSR) {
    set_error("%s: the CSR passed in does not have the patch's mass-matrix pattern", what);
    return TW_EINVAL;
  }
  if (f) {
    set_error("%s: device check failed (flags 0x%x)", what, f);
    return TW_ECUDA;
  }
  return TW_OK;
}

#define GX(n) (unsigned)(((n) + 255) / 256), 256, 0, st

static int ext_build_impl(tw_patch *P) {
  cudaStream_t st = P->stream;
  const Dir &A = P->d[0], &B = P->d[1];
  const int n1 = A.n, n2 = B.n, p = P->p, pp = (p + 1) * (p + 1);
  const int64_t nf = (int64_t)n1 * n2, n = P->n_rows;
  ExtTables *T = (ExtTables *)calloc(1, sizeof(ExtTables));
  if (!T) return TW_ENOMEM;
  P->ext = T;
  Ext &X = T->X;
  X.n1 = n1;
  X.n2 = n2;
  X.p = p;
  X.pp = pp;
  X.n_rows = n;
  X.act = P->act;
  X.rowg = P->rowg;
  int64_t *fl = (int64_t *)dalloc(P, sizeof(int64_t) * (nf + 1));
  T->pos = (int64_t *)dalloc(P, sizeof(int64_t) * (nf + 1));
  int32_t *inng = (int32_t *)dalloc(P, sizeof(int32_t) * nf);
  int32_t *outg = (int32_t *)dalloc(P, sizeof(int32_t) * nf);
  int32_t *inner_g = (int32_t *)dalloc(P, sizeof(int32_t) * (n + 1));
  int32_t *outer_g = (int32_t *)dalloc(P, sizeof(int32_t) * (n + 1));
  uint8_t *ok = (uint8_t *)dalloc(P, nf);
  int64_t *tot = (int64_t *)dalloc(P, sizeof(int64_t) * 4);
  if (!fl || !T->pos || !inng || !outg || !inner_g || !outer_g || !ok || !tot) return TW_ENOMEM;
  cudaMemsetAsync(P->flag, 0, sizeof(int), st);
  k_ext_flags<<<GX(nf)>>>(A, B, P->estate, P->act, fl);
  TW_LAUNCH();
  int rc = exclusive_scan_i64(fl, T->pos, nf, tot, st, P);
  if (rc) return rc;
  k_ext_index<<<GX(nf)>>>(nf, fl, T->pos, inng, outg, inner_g, outer_g);
  TW_LAUNCH();
  k_ext_arrays<<<GX(nf)>>>(n1, n2, p, inng, ok);
  TW_LAUNCH();
  int32_t *ainn = (int32_t *)dalloc(P, sizeof(int32_t) * (n + 1));
  int32_t *aout = (int32_t *)dalloc(P, sizeof(int32_t) * (n + 1));
  if (!ainn || !aout) return TW_ENOMEM;
  k_ext_amaps<<<GX(nf)>>>(nf, P->act, inng, outg, ainn, aout);
  TW_LAUNCH();
  X.ainn = ainn;
  X.aout = aout;
  int64_t htot = 0;
  cudaMemcpyAsync(&htot, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if ((rc = check_cuda(cudaStreamSynchronize(st), "tw_extension_build"))) return rc;
  X.n_inner = htot & 0xffffffff;
  X.n_outer = htot >> 32;
  X.inng = inng;
  X.outg = outg;
  X.inner_g = inner_g;
  const int64_t no = X.n_outer, ni = X.n_inner;
  int32_t *arr = (int32_t *)dalloc(P, sizeof(int32_t) * (no + 1));
  int32_t *ocol = (int32_t *)dalloc(P, sizeof(int32_t) * (no * pp + 1));
  double *oval = (double *)dalloc(P, sizeof(double) * (no * pp + 1));
  uint8_t *near = (uint8_t *)dalloc(P, ni + 1);
  int64_t *tcnt = (int64_t *)dalloc(P, sizeof(int64_t) * (ni + 1));
  int64_t *et_rp = (int64_t *)dalloc(P, sizeof(int64_t) * (ni + 1));
  int64_t *xcnt = (int64_t *)dalloc(P, sizeof(int64_t) * (ni + 1));
  T->xrp = (int64_t *)dalloc(P, sizeof(int64_t) * (ni + 1));
  T->near_row = (int32_t *)dalloc(P, sizeof(int32_t) * (ni + 1));
  int32_t *near_pos = (int32_t *)dalloc(P, sizeof(int32_t) * (ni + 1));
  T->near_list = (int32_t *)dalloc(P, sizeof(int32_t) * (ni + 1));
  if (!arr || !ocol || !oval || !near || !tcnt || !et_rp || !xcnt || !T->xrp || !T->near_row ||
      !near_pos || !T->near_list)
    return TW_ENOMEM;
  if (no > 0) {
    k_ext_outer<<<GX(no)>>>(A, B, no, outer_g, ok, inng, arr, ocol, oval, P->flag);
    TW_LAUNCH();
  }
  if ((rc = ext_flag(P, "tw_extension_build"))) return rc;
  cudaMemsetAsync(near, 0, ni + 1, st);
  // the scans below run over ni + 1 counts: the last one must be zero
  cudaMemsetAsync(tcnt, 0, sizeof(int64_t) * (ni + 1), st);
  cudaMemsetAsync(xcnt, 0, sizeof(int64_t) * (ni + 1), st);
  if (no > 0) {
    k_ext_mark<<<GX(no * pp)>>>(no * pp, ocol, near);
    TW_LAUNCH();
  }
  X.arr = arr;
  X.ocol = ocol;
  X.oval = oval;
  X.near = near;
  if (ni > 0) {
    k_ext_tlist<<<GX(ni)>>>(X, tcnt, nullptr, nullptr);
    TW_LAUNCH();
  }
  if ((rc = exclusive_scan_i64(tcnt, et_rp, ni + 1, tot + 1, st, P))) return rc;
  cudaMemcpyAsync(&T->nnz_t, tot + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if ((rc = check_cuda(cudaStreamSynchronize(st), "tw_extension_build"))) return rc;
  int32_t *et_r = (int32_t *)dalloc(P, sizeof(int32_t) * (T->nnz_t + 1));
  double *et_e = (double *)dalloc(P, sizeof(double) * (T->nnz_t + 1));
  if (!et_r || !et_e) return TW_ENOMEM;
  X.et_rp = et_rp;
  if (ni > 0) {
    k_ext_tlist<<<GX(ni)>>>(X, nullptr, et_r, et_e);
    TW_LAUNCH();
  }
  X.et_r = et_r;
  X.et_e = et_e;
  if (ni > 0) {
    k_ext_xcount<<<(unsigned)((ni + TW_EXT_WARPS - 1) / TW_EXT_WARPS), TW_EXT_THREADS, 0, st>>>(
        X, xcnt, T->near_row, P->flag);
    TW_LAUNCH();
  }
  if ((rc = exclusive_scan_i64(xcnt, T->xrp, ni + 1, tot + 2, st, P))) return rc;
  cudaMemcpyAsync(&T->nnz_x, tot + 2, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  int32_t *tot32 = (int32_t *)(tot + 3);
  if ((rc = exclusive_scan_i32(T->near_row, near_pos, ni, tot32, st, P))) return rc;
  if (ni > 0) {
    k_ext_compact<<<GX(ni)>>>(ni, T->near_row, near_pos, T->near_list);
    TW_LAUNCH();
  }
  int32_t hn = 0;
  cudaMemcpyAsync(&hn, tot32, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  rc = ext_flag(P, "tw_extension_build");
  T->n_near = hn;
  return rc;
}

void ext_free(tw_patch *P) {
  free(P->ext);
  P->ext = nullptr;
}

static int need_ext(tw_patch *P, const char *what) {
  if (!P->ext) {
    set_error("%s: call tw_extension_build first", what);
    return TW_EINVAL;
  }
  return TW_OK;
}

// out = E A^{-1} E^T y for active-length y and out, A the symmetric part of
// the extended mass matrix (CG to tol); the patch's stream must be s
static int ext_solve(tw_patch *P, const int64_t *xrp, const int32_t *xcol, const double *xval,
                     const double *y, double *out, double tol, int maxit, int *iters,
                     double *relres, cudaStream_t st) {
  const ExtTables *T = (const ExtTables *)P->ext;
  const int mark = P->nallocs;
  const int64_t n = P->n_rows, ni = T->X.n_inner;
  double *yx = (double *)dalloc(P, sizeof(double) * (2 * ni + 2));
  if (!yx) return TW_ENOMEM;
  double *x = yx + ni + 1;
  if (ni > 0) {
    k_ext_restrict<<<GX(ni)>>>(T->X, y, yx);
    TW_LAUNCH();
  }
  int rc = cg_solve_n(P, ni, T->nnz_x, xrp, xcol, xval, yx, x, tol, maxit, iters, relres, st);
  if ((!rc || rc == TW_ENOCONV) && n > 0) {
    k_ext_expand<<<GX(n)>>>(T->X, x, out);
    TW_LAUNCH();
  }
  release_to(P, mark);
  return rc;
}

}  // namespace tw

using namespace tw;

extern "C" int tw_extension_build(tw_patch *P, int64_t *info4) {
  if (!P || !info4) {
    set_error("tw_extension_build: NULL argument");
    return TW_EINVAL;
  }
  if (P->mixed) {  // R16's arrays are read on simple knots
    set_error("tw_extension_build: extended B-splines need simple interior knots");
    return TW_EUNSUPPORTED;
  }
  if (!P->ext) {
    const int mark = P->nallocs;
    int rc = ext_build_impl(P);
    if (rc) {
      cudaStreamSynchronize(P->stream);
      release_to(P, mark);
      ext_free(P);
      return rc;
    }
  }
  const ExtTables *T = (const ExtTables *)P->ext;
  info4[0] = T->X.n_inner;
  info4[1] = T->X.n_outer;
  info4[2] = T->X.n_inner + T->X.n_outer * T->X.pp;
  info4[3] = T->nnz_x;
  return TW_OK;
}

extern "C" int tw_extension_matrix(tw_patch *P, int64_t *e_row_ptr, int32_t *e_col,
                                   double *e_val, void *stream) {
  if (!P || !e_row_ptr || !e_col || !e_val) {
    set_error("tw_extension_matrix: NULL argument");
    return TW_EINVAL;
  }
  int rc = need_ext(P, "tw_extension_matrix");
  if (rc) return rc;
  const ExtTables *T = (const ExtTables *)P->ext;
  cudaStream_t st = (cudaStream_t)stream;
  k_ext_ecsr<<<GX(T->X.n_rows + 1)>>>(T->X, T->pos, e_row_ptr, e_col, e_val);
  TW_LAUNCH();
  return check_cuda(cudaGetLastError(), "tw_extension_matrix");
}

extern "C" int tw_form_mass_extended(tw_patch *P, const int64_t *row_ptr, const int32_t *col,
                                     const double *val, int64_t *x_row_ptr, int32_t *x_col,
                                     double *x_val, void *stream) {
  if (!P || !row_ptr || !col || !val || !x_row_ptr || !x_col || !x_val) {
    set_error("tw_form_mass_extended: NULL argument");
    return TW_EINVAL;
  }
  int rc = need_ext(P, "tw_form_mass_extended");
  if (rc) return rc;
  const ExtTables *T = (const ExtTables *)P->ext;
  cudaStream_t keep = P->stream, st = (cudaStream_t)stream;
  P->stream = st;
  const int64_t ni = T->X.n_inner;
  cudaMemsetAsync(P->flag, 0, sizeof(int), st);
  cudaMemcpyAsync(x_row_ptr, T->xrp, sizeof(int64_t) * (ni + 1), cudaMemcpyDeviceToDevice, st);
  if (ni > 0) {
    k_ext_xcopy<<<(unsigned)((ni + TW_EXT_WARPS - 1) / TW_EXT_WARPS), TW_EXT_THREADS, 0, st>>>(
        T->X, T->near_row, row_ptr, col, val, T->xrp, x_col, x_val, P->flag);
    TW_LAUNCH();
  }
  if (T->n_near > 0) {
    static std::once_flag near_attr[64];
    int dev = 0;
    cudaGetDevice(&dev);
    std::call_once(near_attr[dev & 63], [] {
      cudaFuncSetAttribute(k_ext_xnear, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(TW_EXT_NEAR_WARPS * ext_near_words(TW_MAXP) * 4));
    });
    const size_t smem = TW_EXT_NEAR_WARPS * ext_near_words(T->X.p) * 4;
    k_ext_xnear<<<(unsigned)((T->n_near + TW_EXT_NEAR_WARPS - 1) / TW_EXT_NEAR_WARPS),
                  32 * TW_EXT_NEAR_WARPS, smem, st>>>(T->X, T->near_list, T->n_near, row_ptr,
                                                      col, val, T->xrp, x_col, x_val, P->flag);
    TW_LAUNCH();
  }
  rc = ext_flag(P, "tw_form_mass_extended");
  P->stream = keep;
  return rc;
}

extern "C" int tw_l2_project_extended(tw_patch *P, const tw_func *f, const int64_t *x_row_ptr,
                                      const int32_t *x_col, const double *x_val, double *u,
                                      double tol, int maxit, int *iters, double *relres,
                                      void *stream) {
  if (!P || !f || !x_row_ptr || !x_col || !x_val || !u) {
    set_error("tw_l2_project_extended: NULL argument");
    return TW_EINVAL;
  }
  if (!(tol > 0) || maxit < 0) {
    set_error("tw_l2_project_extended: need tol > 0 and maxit >= 0");
    return TW_EINVAL;
  }
  int rc = need_ext(P, "tw_l2_project_extended");
  if (rc) return rc;
  cudaStream_t keep = P->stream, st = (cudaStream_t)stream;
  P->stream = st;
  const int mark = P->nallocs;
  double *b = (double *)dalloc(P, sizeof(double) * (P->n_rows + 1));
  if (!b) rc = TW_ENOMEM;
  const int ps = prof_start(st);
  if (!rc) rc = rhs_launch(P, f, b, st);
  if (!rc) rc = ext_solve(P, x_row_ptr, x_col, x_val, b, u, tol, maxit, iters, relres, st);
  prof_stop(ps, TW_STAGE_CG, st);
  release_to(P, mark);
  P->stream = keep;
  return rc;
}

extern "C" int tw_l2_project_adjoint_extended(tw_patch *P, const tw_func *f,
                                              const int64_t *x_row_ptr, const int32_t *x_col,
                                              const double *x_val, const double *dLdu,
                                              const double *u, double *lam, double *grad,
                                              double tol, int maxit, int *iters, double *relres,
                                              void *stream) {
  if (!P || !f || !x_row_ptr || !x_col || !x_val || !dLdu || !u || !lam || !grad) {
    set_error("tw_l2_project_adjoint_extended: NULL argument");
    return TW_EINVAL;
  }
  if (P->geo.coef_kind != TW_COEF_DENSITY) {
    set_error("tw_l2_project_adjoint_extended: the patch has no density spline "
              "(TW_COEF_DENSITY)");
    return TW_EINVAL;
  }
  if (!(tol > 0) || maxit < 0) {
    set_error("tw_l2_project_adjoint_extended: need tol > 0 and maxit >= 0");
    return TW_EINVAL;
  }
  int rc = need_ext(P, "tw_l2_project_adjoint_extended");
  if (rc) return rc;
  cudaStream_t keep = P->stream, st = (cudaStream_t)stream;
  P->stream = st;
  const int mark = P->nallocs;
  const int ps = prof_start(st);
  rc = ext_solve(P, x_row_ptr, x_col, x_val, dLdu, lam, tol, maxit, iters, relres, st);
  prof_stop(ps, TW_STAGE_CG, st);
  if (!rc) rc = adjoint_grad(P, f, u, lam, grad, st);
  release_to(P, mark);
  P->stream = keep;
  return rc;
}
