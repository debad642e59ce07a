// tw_setup.cu -- patch set-up kernels (everything that depends on the patch but
// not on the matrix entries' precision):
//   WQ point layout and weights            Sect. 2.1, Eqs. 4-5 (readings R1-R3)
//   trimming classification                Sect. 2.2 (reading R8)
//   c at the WQ grid (sum-factorised det J) Eqs. 6-7
//   cut-element rules                      Sect. 3.1 (reading R6)
//   DWQ region choice and rules            Sect. 3.3, Eqs. 9-10 (readings R4, R5, R7)
//   CSR pattern                            row-based assembly (reading R11)
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "tw_internal.cuh"

namespace tw {

// point offset of element e in the WQ layout (R1, the table D.qoff built
// from the knots): p+1 points in an element touching a knot of multiplicity
// >= 2 (the domain ends, repeated interior knots), none on the zero-length
// span of a repeated knot, 2 elsewhere
__device__ __forceinline__ int wq_off(const Dir &D, int e) {
  return D.qoff[e <= 0 ? 0 : (e >= D.nel ? D.nel : e)];
}

// ---------------------------------------------------------------------------
// scans of 1024-element blocks (integer sums: exact in any order).  One launch
// when the input fits one block; otherwise the block scans, then a pass in
// which every block sums the totals of the blocks before it itself (no third
// launch) while there are at most TW_SCAN_DIRECT blocks, else a one-block scan
// of the totals between the two.

#define TW_SCAN_DIRECT 2048

// inclusive scan over the 1024 threads of a block (warp shuffles, two barriers)
template <typename T>
__device__ __forceinline__ T block_scan_incl(T v, T *wsum) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T w = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  return wid > 0 ? x + wsum[wid - 1] : x;
}

// One or two independent scans per launch (blockIdx.y picks the scan; blocks
// past a scan's own count return).
template <typename T>
struct ScanJob {
  const T *in;
  T *out, *bsum, *total;
  int64_t n, nb;
  int direct;
};
template <typename T>
struct ScanJobs {
  ScanJob<T> j[2];
};

// block scan: out = exclusive scan within the block, bsum = the block's total;
// a single-block scan also writes the grand total
template <typename T>
__global__ void __launch_bounds__(1024) k_scan_block(ScanJobs<T> J) {
  __shared__ T wsum[32];
  const ScanJob<T> &S = J.j[blockIdx.y];
  if ((int64_t)blockIdx.x >= S.nb) return;  // the whole block
  const int t = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * 1024 + t;
  const T v = i < S.n ? S.in[i] : (T)0;
  const T incl = block_scan_incl(v, wsum);
  if (i < S.n) S.out[i] = incl - v;
  if (t == 1023) {
    S.bsum[blockIdx.x] = incl;
    if (S.nb == 1) *S.total = incl;
  }
}

// the totals of blocks scanned in place (exclusive), and the grand total, for
// more than TW_SCAN_DIRECT blocks
template <typename T>
__global__ void __launch_bounds__(1024) k_scan_sums(T *bsum, int64_t nb, T *total) {
  __shared__ T wsum[32];
  __shared__ T carry;
  const int t = threadIdx.x;
  if (t == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += 1024) {
    const int64_t i = base + t;
    const T v = i < nb ? bsum[i] : (T)0;
    const T incl = block_scan_incl(v, wsum);
    const T c = carry;
    if (i < nb) bsum[i] = c + incl - v;
    __syncthreads();
    if (t == 1023) carry = c + incl;
    __syncthreads();
  }
  if (t == 0) *total = carry;
}

// adds each block's carry: the sum of the totals of the blocks before it,
// formed by the block itself (direct; the last block then writes the grand
// total) or read from the scanned totals
template <typename T>
__global__ void __launch_bounds__(1024) k_scan_add(ScanJobs<T> J) {
  __shared__ T wsum[32];
  __shared__ T carry_s;
  const ScanJob<T> &S = J.j[blockIdx.y];
  const int64_t b = blockIdx.x;
  if (S.nb < 2 || b >= S.nb) return;  // the whole block
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  T carry;
  if (S.direct) {
    T s = 0;
    for (int64_t j = t; j < b; j += 1024) s += S.bsum[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) wsum[wid] = s;
    __syncthreads();
    if (wid == 0) {
      T w = wsum[lane];
      for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
      if (lane == 0) carry_s = w;
    }
    __syncthreads();
    carry = carry_s;
  } else {
    carry = S.bsum[b];
  }
  const int64_t i = b * 1024 + t;
  if (i < S.n) S.out[i] += carry;
  if (S.direct && b == S.nb - 1 && t == 0) *S.total = carry + S.bsum[b];
}

// exclusive scans of in0 (n0 entries) and, if n1 >= 0, of in1 (n1 entries),
// with their totals, in two launches at most (three past TW_SCAN_DIRECT blocks)
template <typename T>
static int scan2_impl(const T *in0, T *out0, int64_t n0, T *tot0, const T *in1, T *out1,
                      int64_t n1, T *tot1, cudaStream_t s, tw_patch *P) {
  ScanJobs<T> J;
  const int ns = n1 >= 0 ? 2 : 1;
  int64_t nbmax = 0;
  bool any_add = false;
  for (int k = 0; k < ns; k++) {
    ScanJob<T> &S = J.j[k];
    S.in = k ? in1 : in0;
    S.out = k ? out1 : out0;
    S.total = k ? tot1 : tot0;
    S.n = k ? n1 : n0;
    S.nb = (S.n + 1023) / 1024;
    S.direct = S.nb <= TW_SCAN_DIRECT;
    S.bsum = nullptr;
    if (S.n <= 0) {
      S.nb = 0;
      cudaMemsetAsync(S.total, 0, sizeof(T), s);
      continue;
    }
    S.bsum = (T *)dalloc(P, sizeof(T) * S.nb);
    if (!S.bsum) return TW_ENOMEM;
    nbmax = std::max(nbmax, S.nb);
    any_add = any_add || S.nb > 1;
  }
  if (ns == 1) J.j[1] = J.j[0];  // never read (gridDim.y = 1)
  if (nbmax == 0) return 0;
  k_scan_block<T><<<dim3((unsigned)nbmax, ns), 1024, 0, s>>>(J);
  TW_LAUNCH();
  if (any_add) {
    for (int k = 0; k < ns; k++)
      if (J.j[k].nb > 1 && !J.j[k].direct) {
        k_scan_sums<T><<<1, 1024, 0, s>>>(J.j[k].bsum, J.j[k].nb, J.j[k].total);
        TW_LAUNCH();
      }
    k_scan_add<T><<<dim3((unsigned)nbmax, ns), 1024, 0, s>>>(J);
    TW_LAUNCH();
  }
  return check_cuda(cudaGetLastError(), "scan");
}

template <typename T>
static int scan_impl(const T *in, T *out, int64_t n, T *total_dev, cudaStream_t s, tw_patch *P) {
  return scan2_impl<T>(in, out, n, total_dev, nullptr, nullptr, -1, nullptr, s, P);
}

int exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total, cudaStream_t s,
                       tw_patch *P) {
  return scan_impl<int32_t>(in, out, n, total, s, P);
}
int exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total, cudaStream_t s,
                       tw_patch *P) {
  return scan_impl<int64_t>(in, out, n, total, s, P);
}

// ---------------------------------------------------------------------------
// univariate tables

// q-point Gauss-Legendre by Newton on the Legendre recurrence (double)
__global__ void k_gauss_nodes(int q, double *x, double *w) {
  int k = threadIdx.x;
  if (k >= q) return;
  double z = cos(3.141592653589793 * (q - k - 0.25) / (q + 0.5));  // ascending order
  double dp = 1.0;
  for (int it = 0; it < 64; it++) {
    double a = 1.0, b = z;  // P0, P1
    for (int m = 2; m <= q; m++) {
      double c = ((2 * m - 1) * z * b - (m - 1) * a) / m;
      a = b;
      b = c;
    }
    if (q == 1) a = 1.0;
    dp = q * (z * b - a) / (z * z - 1.0);
    double dz = b / dp;
    z -= dz;
    if (fabs(dz) <= 1e-15) break;  // quadratic convergence: z is now exact to rounding
  }
  {
    double a = 1.0, b = z;
    for (int m = 2; m <= q; m++) {
      double c = ((2 * m - 1) * z * b - (m - 1) * a) / m;
      a = b;
      b = c;
    }
    if (q == 1) a = 1.0;
    dp = q * (z * b - a) / (z * z - 1.0);
  }
  x[k] = z;
  w[k] = 2.0 / ((1.0 - z * z) * dp * dp);
}

// The per-direction tables, both directions and all three kinds in one launch
// of one-warp blocks (blockIdx.y picks the direction; each item runs a long
// FP64 chain, so the items are spread over many SMs).  Each kind is an
// out-of-line routine, so no function holds two inlined copies of the
// Cox-de Boor triangle.

// WQ point j of element e (of its m = qoff[e+1] - qoff[e] <= p + 1 points,
// R1): uniform in the element's interior, with the basis and derivatives there
static __device__ __noinline__ void wq_point_item(const Dir &D, int e, int j) {
  const int p = D.p, k0 = D.qoff[e], m = D.qoff[e + 1] - k0;
  if (j >= m) return;
  const double a = D.bp[e], b = D.bp[e + 1];
  const int k = k0 + j;
  const double x = a + (b - a) * (double)(j + 1) / (double)(m + 1);
  D.xq[k] = x;
  D.qel[k] = e;
  double N[TW_MAXP1], dN[TW_MAXP1];
  basis_ders(D.U, e + p, x, p, N, dN);
  for (int a2 = 0; a2 <= p; a2++) {
    D.Bq[k * (p + 1) + a2] = N[a2];
    D.dBq[k * (p + 1) + a2] = dN[a2];
  }
}

// test function i: the run of WQ points of its support
__device__ __forceinline__ void wq_ranges_item(const Dir &D, int i) {
  int lo = max(0, i - D.p), hi = min(D.nel - 1, i);
  D.qbeg[i] = wq_off(D, lo);
  D.qcnt[i] = wq_off(D, hi + 1) - D.qbeg[i];
}

// Gauss point g of element e: basis values and derivatives, and the weighted
// products of the element matrices (Gauss weight x Jacobian of the span map x
// two basis values), once per element of the direction
static __device__ __noinline__ void gauss_tables_item(const Dir &D, int id) {
  int p1 = D.p + 1;
  int e = id / p1, g = id % p1;
  double a = D.bp[e], b = D.bp[e + 1];
  double x = a + (b - a) * 0.5 * (D.gx[g] + 1.0);
  double N[TW_MAXP1], dN[TW_MAXP1];
  if (b > a) {
    basis_ders(D.U, e + D.p, x, D.p, N, dN);
  } else {  // the zero-length span of a repeated knot: nothing lives on it
    for (int k = 0; k < p1; k++) N[k] = dN[k] = 0.0;
  }
  for (int k = 0; k < p1; k++) {
    D.GB[(e * p1 + g) * p1 + k] = N[k];
    D.dGB[(e * p1 + g) * p1 + k] = dN[k];
  }
  const double hw = D.gw[g] * (0.5 * (b - a));
  double *gw3 = D.GW + (size_t)(e * p1 + g) * p1 * p1;
  for (int i = 0; i < p1; i++)
    for (int k = 0; k < p1; k++) gw3[i * p1 + k] = hw * N[i] * N[k];
}

// segment s of a closed cubic B-spline trimming curve (the periodic uniform
// spline of its nc control points) in monomial form on u in [0, 1], with the
// bounding box of its four control points
__device__ __forceinline__ void curve_segment_item(const double *ctrl, int nc, double *seg,
                                                   double *box, int s) {
  for (int o = 0; o < 2; o++) {
    double Q0 = ctrl[2 * (((s - 3) % nc + nc) % nc) + o];
    double Q1 = ctrl[2 * (((s - 2) % nc + nc) % nc) + o];
    double Q2 = ctrl[2 * (((s - 1) % nc + nc) % nc) + o];
    double Q3 = ctrl[2 * s + o];
    seg[8 * s + 4 * o + 0] = (Q0 + 4.0 * Q1 + Q2) / 6.0;
    seg[8 * s + 4 * o + 1] = (Q2 - Q0) / 2.0;
    seg[8 * s + 4 * o + 2] = (Q0 - 2.0 * Q1 + Q2) / 2.0;
    seg[8 * s + 4 * o + 3] = (-Q0 + 3.0 * Q1 - 3.0 * Q2 + Q3) / 6.0;
    box[4 * s + 2 * o] = fmin(fmin(Q0, Q1), fmin(Q2, Q3));
    box[4 * s + 2 * o + 1] = fmax(fmax(Q0, Q1), fmax(Q2, Q3));
  }
}

// the spline trimming curves whose segments a k_dir_tables launch forms
// (curve k takes blocks blk[k] .. blk[k+1]-1 of that part)
struct SegJobs {
  int n;
  int blk[TW_MAXCURVES + 1];
  int nc[TW_MAXCURVES];
  const double *ctrl[TW_MAXCURVES];
  double *seg[TW_MAXCURVES], *box[TW_MAXCURVES];
};

// blocks [0, b0): (element, point) pairs (WQ points); [b0, b0 + b1): test functions (WQ
// ranges); [b0 + b1, b0 + b1 + b2): element Gauss points (Gauss tables); the
// rest (direction 0 only): the spline curves' segments
__global__ void __launch_bounds__(32) k_dir_tables(Dir D0, Dir D1, int b0, int b1, int b2,
                                                   SegJobs S) {
  const Dir &D = blockIdx.y ? D1 : D0;
  const int b = blockIdx.x;
  if (b < b0) {
    const int t = b * 32 + threadIdx.x, e = t / (D.p + 1);
    if (e < D.nel) wq_point_item(D, e, t - e * (D.p + 1));
  } else if (b < b0 + b1) {
    const int i = (b - b0) * 32 + threadIdx.x;
    if (i < D.n) wq_ranges_item(D, i);
  } else if (b < b0 + b1 + b2) {
    const int id = (b - b0 - b1) * 32 + threadIdx.x;
    if (id < D.nel * (D.p + 1)) gauss_tables_item(D, id);
  } else if (blockIdx.y == 0) {
    const int j = b - b0 - b1 - b2;
    for (int k = 0; k < S.n; k++)
      if (j >= S.blk[k] && j < S.blk[k + 1]) {
        const int sg = (j - S.blk[k]) * 32 + threadIdx.x;
        if (sg < S.nc[k]) curve_segment_item(S.ctrl[k], S.nc[k], S.seg[k], S.box[k], sg);
      }
  }
}

// B_j(x_k) from the WQ basis table (zero off the span)
__device__ __forceinline__ double Bjk(const Dir &D, int j, int k) {
  int a = j - D.qel[k];
  return (a >= 0 && a <= D.p) ? D.Bq[k * (D.p + 1) + a] : 0.0;
}

// Eq. 5 for test function i: min-norm weights, then V = W * B_j (R2, R3).
// Groups of TW_WQ_G lanes own one test function each (group_minnorm: the
// lanes of a group own the points c = gl + G u of its system), so a warp
// solves 32 / TW_WQ_G systems at once; the systems' matrices sit in dynamic
// shared memory with row stride lda = max qmax + 1.
#define TW_WQ_WARPS 2
#define TW_WQ_G 8
#define TW_WQ_SYS (TW_WQ_WARPS * 32 / TW_WQ_G)  // systems per block
#define TW_WQ_CPL ((TW_QMAX + TW_WQ_G - 1) / TW_WQ_G)
__global__ void __launch_bounds__(32 * TW_WQ_WARPS) k_wq_weights(Dir D0, Dir D1, int lda,
                                                                int *flag) {
  const Dir &D = blockIdx.y ? D1 : D0;
  extern __shared__ double wq_dyn[];  // TW_WQ_SYS x TW_WIN x lda
  __shared__ double sb[TW_WQ_SYS][TW_WIN], sd[TW_WQ_SYS][TW_WIN], sbeta[TW_WQ_SYS][TW_WIN];
  __shared__ int sing[TW_WQ_SYS];
  constexpr int G = TW_WQ_G, CPL = TW_WQ_CPL;
  const int lane = threadIdx.x & 31, gl = lane & (G - 1);
  const int sys = threadIdx.x / G;  // the block's system of this lane's group
  const int i = blockIdx.x * TW_WQ_SYS + sys;
  const int p = D.p, p1 = p + 1, W2 = 2 * p + 1;
  // Eq. 5's equations: the trial functions whose support overlaps supp B_i
  // with positive measure, a contiguous run of i-p .. i+p (with a repeated
  // knot some of them only touch supp B_i at that knot)
  int m = 0, N = 0, jlo = 0, q0 = 0;
  if (i < D.n) {
    jlo = max(0, i - p);
    int jhi = min(D.n - 1, i + p);
    if (D.mixed) {  // simple knots: the whole run overlaps
      while (jlo < i && !(D.U[jlo + p + 1] > D.U[i])) jlo++;
      while (jhi > i && !(D.U[jhi] < D.U[i + p + 1])) jhi--;
    }
    m = jhi - jlo + 1;
    q0 = D.qbeg[i];
    N = D.qcnt[i];
    if (N > TW_QMAX || N >= lda) {
      if (gl == 0) atomicOr(flag, TWF_QMAX);
      m = N = 0;
    }
  }
  double *A = wq_dyn + (size_t)sys * TW_WIN * lda;
  const int elo = max(0, i - p), ehi = min(D.nel - 1, i);
  for (int c = gl; c < N; c += G)
    for (int r = 0; r < m; r++) A[r * lda + c] = Bjk(D, jlo + r, q0 + c);
  for (int r = gl; r < m; r += G) {
    int j = jlo + r;
    double s = 0.0;
    int ea = max(elo, max(0, j - p)), eb = min(ehi, min(D.nel - 1, j));
    for (int e = ea; e <= eb; e++)  // the Gauss products w_g h B_i B_j, tabulated per element
      for (int g = 0; g < p1; g++) s += D.GW[((size_t)(e * p1 + g) * p1 + (i - e)) * p1 + (j - e)];
    sb[sys][r] = s;
  }
  if (gl == 0) sing[sys] = 0;
  __syncwarp();
  double w[CPL];
  group_minnorm<G, CPL>(m, N, A, lda, sb[sys], sd[sys], sbeta[sys], gl, &sing[sys], w);
  __syncwarp();
  if (i >= D.n) return;  // the group only (no collective below)
  if (gl == 0 && sing[sys]) atomicOr(flag, TWF_SINGULAR);
#pragma unroll
  for (int u = 0; u < CPL; u++) {
    const int c = gl + G * u;
    if (c >= D.qmax) break;
    const double wc = c < N ? w[u] : 0.0;
    D.W[(size_t)i * D.qmax + c] = wc;
    for (int r = 0; r < W2; r++) {
      int j = i - p + r;
      double v = 0.0;
      if (c < N && j >= 0 && j < D.n) v = wc * Bjk(D, j, q0 + c);
      D.V[((size_t)i * D.qmax + c) * W2 + r] = v;
    }
  }
  for (int r = gl; r < W2; r += G) {
    int j = i - p + r;
    int lo = 0, hi = 0;
    if (j >= 0 && j < D.n) {
      int ea = max(elo, max(0, j - p)), eb = min(ehi, min(D.nel - 1, j));
      lo = wq_off(D, ea) - q0;
      hi = wq_off(D, eb + 1) - q0;
    }
    D.crange[i * W2 + r] = lo | (hi << 16);
  }
}

// ---------------------------------------------------------------------------
// trimming curve: its first point, the knot lines' crossings, its features


__device__ void curve_point0(const Curve &C, double *xy) {
  if (C.kind == TW_TRIM_CIRCLE) {
    xy[0] = C.prm[0] + C.prm[2];
    xy[1] = C.prm[1];
  } else if (C.kind == TW_TRIM_ELLIPSE) {
    xy[0] = C.prm[0] + C.prm[2] * cos(C.prm[4]);
    xy[1] = C.prm[1] + C.prm[2] * sin(C.prm[4]);
  } else if (C.kind == TW_TRIM_BSPLINE3) {
    xy[0] = C.seg[0];
    xy[1] = C.seg[4];
  } else {
    xy[0] = xy[1] = -1e300;
  }
}

// Crossings of the curve with whole lines, sorted: lines [0, nel1] are the
// vertical knot lines x = bp1[l], [nel1+1, nel1+nel2+1] the horizontal knot
// lines, and the last nel2 the horizontal lines through the element centres of
// each row (visibility by the parity of crossings to the right, reading R8).
__device__ __forceinline__ void line_hits_item(const CurveSet &C, const Dir &A, const Dir &B,
                                               int l, double *hits, int *nh, int *flag) {
  int o;
  double s;
  if (l <= A.nel) {
    o = 0;
    s = A.bp[l];
  } else if (l <= A.nel + B.nel + 1) {
    o = 1;
    s = B.bp[l - A.nel - 1];
  } else {
    int e2 = l - A.nel - B.nel - 2;
    o = 1;
    s = 0.5 * (B.bp[e2] + B.bp[e2 + 1]);
  }
  int n = set_line_hits(C, o, s, -1e300, 1e300, hits + (size_t)l * TW_HITCAP, TW_HITCAP);
  if (n < 0) {
    atomicOr(flag, TWF_HITCAP);
    n = 0;
  }
  nh[l] = n;
}

__device__ __forceinline__ int any_hit_in(const double *h, int n, double lo, double hi) {
  for (int k = 0; k < n; k++)
    if (h[k] > lo && h[k] < hi) return 1;
  return 0;
}

// R8: an element is cut iff the curve meets its open box: a crossing inside
// one of its four open edges (corner touches excluded), or the whole curve
// inside it; otherwise visible iff its centre is
__device__ __forceinline__ uint8_t classify_elem(const CurveSet &C, const Dir &A, const Dir &B,
                                                 const double *hits, const int *nh, int id) {
  int e1 = id % A.nel, e2 = id / A.nel;
  double a1 = A.bp[e1], b1 = A.bp[e1 + 1], a2 = B.bp[e2], b2 = B.bp[e2 + 1];
  if (!(b1 > a1) || !(b2 > a2)) {  // R8: an empty span has no measure
    return TW_ELEM_EMPTY;
  }
  if (C.n == 0) {
    return TW_ELEM_REGULAR;
  }
  double d1 = TW_CORNER * (b1 - a1), d2 = TW_CORNER * (b2 - a2);
  const int hv = A.nel + 1;  // first horizontal knot line
  const int hc = A.nel + B.nel + 2;  // first centre line
  int cut = any_hit_in(hits + (size_t)e1 * TW_HITCAP, nh[e1], a2 + d2, b2 - d2) ||
            any_hit_in(hits + (size_t)(e1 + 1) * TW_HITCAP, nh[e1 + 1], a2 + d2, b2 - d2) ||
            any_hit_in(hits + (size_t)(hv + e2) * TW_HITCAP, nh[hv + e2], a1 + d1, b1 - d1) ||
            any_hit_in(hits + (size_t)(hv + e2 + 1) * TW_HITCAP, nh[hv + e2 + 1], a1 + d1, b1 - d1);
  for (int k = 0; k < C.n && !cut; k++) {  // a whole curve inside the element
    double p0[2];
    curve_point0(C.c[k], p0);
    cut = p0[0] > a1 && p0[0] < b1 && p0[1] > a2 && p0[1] < b2;
  }
  uint8_t st;
  if (cut) {
    st = TW_ELEM_CUT;
  } else {
    double xc = 0.5 * (a1 + b1);
    int vis;
    if (C.n == 1) {
      const Curve &C0 = C.c[0];
      const double *h = hits + (size_t)(hc + e2) * TW_HITCAP;
      int right = 0;
      for (int k = 0; k < nh[hc + e2]; k++) right += h[k] > xc;
      // parity of the crossings to the right for a closed curve; the half-plane
      // of a line is tested directly
      int inside = C0.kind == TW_TRIM_LINE ? curve_inside(C0, xc, 0.5 * (a2 + b2)) : (right & 1);
      vis = C0.keep_inside ? inside : !inside;
    } else {  // several curves: the centre against every curve's kept side
      vis = set_visible(C, xc, 0.5 * (a2 + b2));
    }
    st = vis ? TW_ELEM_REGULAR : TW_ELEM_INVISIBLE;
  }
  return st;
}

// element states, with the flags of the cut elements (eflag) and, for the
// Gauss method, of every regular element (gflag; for the hybrid and DWQ
// methods the classification of the functions adds the regular elements
// next to a cut function)
__global__ void k_classify_elems(CurveSet C, Dir A, Dir B, const double *hits, const int *nh,
                                 int method, uint8_t *estate, int32_t *eflag, int32_t *gflag) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= A.nel * B.nel) return;
  const uint8_t st = classify_elem(C, A, B, hits, nh, id);
  estate[id] = st;
  eflag[id] = st == TW_ELEM_CUT;
  gflag[id] = method == TW_METHOD_GAUSS && st == TW_ELEM_REGULAR;
}

// function state from its support elements; active flag for the scan.  The
// same threads clear the disc flags of both directions (nel + 1 each) and set
// every DWQ choice to none (-1) for the stages after.
__global__ void k_classify_funcs(Dir A, Dir B, const uint8_t *estate, uint8_t *fstate,
                                 int32_t *aflag, int method, int32_t *cflag, int32_t *counters,
                                 int32_t *dflag0, int32_t *dflag1, int32_t *choice,
                                 int32_t *gflag) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g <= A.nel) dflag0[g] = 0;
  if (g <= B.nel) dflag1[g] = 0;
  if (g >= A.n * B.n) return;
  reinterpret_cast<int4 *>(choice)[g] = make_int4(-1, -1, -1, -1);
  int i1 = g % A.n, i2 = g / A.n;
  int tot = 0, nreg = 0, ninv = 0;
  for (int e2 = max(0, i2 - B.p); e2 <= min(B.nel - 1, i2); e2++)
    for (int e1 = max(0, i1 - A.p); e1 <= min(A.nel - 1, i1); e1++) {
      uint8_t s = estate[e2 * A.nel + e1];
      if (s == TW_ELEM_EMPTY) continue;  // R8: the states of the elements with measure
      tot++;
      nreg += s == TW_ELEM_REGULAR;
      ninv += s == TW_ELEM_INVISIBLE;
    }
  uint8_t st = ninv == tot ? TW_FUNC_EXTERIOR : (nreg == tot ? TW_FUNC_INTERIOR : TW_FUNC_CUT);
  fstate[g] = st;
  aflag[g] = st != TW_FUNC_EXTERIOR;
  int c = st != TW_FUNC_EXTERIOR && (method == TW_METHOD_GAUSS || st == TW_FUNC_CUT);
  cflag[g] = c;
  if (st == TW_FUNC_CUT) atomicAdd(&counters[0], 1);
  if (st == TW_FUNC_INTERIOR) atomicAdd(&counters[1], 1);
  // hybrid Gauss and DWQ: the regular elements of a cut function's support
  // are integrated by Gauss (the same 1 from every such function)
  if (st == TW_FUNC_CUT && (method == TW_METHOD_HYBRID || method == TW_METHOD_DWQ))
    for (int e2 = max(0, i2 - B.p); e2 <= min(B.nel - 1, i2); e2++)
      for (int e1 = max(0, i1 - A.p); e1 <= min(A.nel - 1, i1); e1++)
        if (estate[e2 * A.nel + e1] == TW_ELEM_REGULAR) gflag[e2 * A.nel + e1] = 1;
}

// compacted lists from flags (exclusive scans already in pos), up to four per
// launch (blockIdx.y picks the list): list[pos[g]] = g for the flagged g, and
// slot[g] = pos[g] or -1 when a slot map is asked for.  With slot == pos this
// also turns the scan of the active flags into the active numbering (-1 for
// the inactive) and list into its inverse.
struct CompactJob {
  const int32_t *flag, *pos;
  int32_t *list, *slot;
  int64_t n;
};
struct CompactJobs {
  CompactJob j[4];
};
__global__ void k_compact(CompactJobs J) {
  const CompactJob &C = J.j[blockIdx.y];
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= C.n) return;
  if (C.flag[g]) {
    const int32_t ps = C.pos[g];
    C.list[ps] = (int32_t)g;
    if (C.slot) C.slot[g] = ps;
  } else if (C.slot) {
    C.slot[g] = -1;
  }
}
static void launch_compact(const CompactJob *jobs, int nj, cudaStream_t st) {
  CompactJobs J;
  int64_t nmax = 0;
  for (int k = 0; k < 4; k++) J.j[k] = jobs[k < nj ? k : 0];
  for (int k = 0; k < nj; k++) nmax = std::max(nmax, jobs[k].n);
  if (nmax == 0) return;
  k_compact<<<dim3((unsigned)((nmax + 255) / 256), nj), 256, 0, st>>>(J);
  TW_LAUNCH();
}

// R11: active columns in the (2p+1)^2 window; cnt[n_rows] = 0 closes the
// array, so that its exclusive scan ends with the total
__global__ void k_row_counts(Dir A, Dir B, const int32_t *act, int64_t *cnt, int n_rows) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g == 0) cnt[n_rows] = 0;
  if (g >= A.n * B.n) return;
  int32_t r = act[g];
  if (r < 0) return;
  int i1 = g % A.n, i2 = g / A.n, p = A.p;
  int64_t c = 0;
  for (int j2 = max(0, i2 - p); j2 <= min(B.n - 1, i2 + p); j2++)
    for (int j1 = max(0, i1 - p); j1 <= min(A.n - 1, i1 + p); j1++) c += act[j2 * A.n + j1] >= 0;
  cnt[r] = c;
}

// sum-factorised det J on the WQ grid: stage A contracts direction 2
__device__ __forceinline__ void geo_stageA_item(const Geo &G, const Dir &A, const Dir &B,
                                                double *Gt, int id) {
  int k2 = id / A.n, i1 = id % A.n, p1 = B.p + 1;
  int e2 = B.qel[k2];
  double x = 0, y = 0, dx = 0, dy = 0;
  for (int b = 0; b < p1; b++) {
    const double *pt = G.ctrl + 2 * ((size_t)(e2 + b) * G.n1 + i1);
    double v = B.Bq[k2 * p1 + b], d = B.dBq[k2 * p1 + b];
    x += pt[0] * v;
    y += pt[1] * v;
    dx += pt[0] * d;
    dy += pt[1] * d;
  }
  double *o = Gt + 4 * (size_t)id;
  o[0] = x;
  o[1] = y;
  o[2] = dx;
  o[3] = dy;
}

__global__ void k_cgrid(Geo G, Dir A, Dir B, const double *Gt, double *Cg) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= A.nq * B.nq) return;
  int k1 = id % A.nq, k2 = id / A.nq;
  double c = 1.0;
  if (G.coef_kind != TW_COEF_ONE) {
    if (G.geom_kind == TW_GEOM_SPLINE) {
      int p1 = A.p + 1, e1 = A.qel[k1];
      double xa = 0, ya = 0, xb = 0, yb = 0;
      for (int a = 0; a < p1; a++) {
        const double *g = Gt + 4 * ((size_t)k2 * A.n + e1 + a);
        double v = A.Bq[k1 * p1 + a], d = A.dBq[k1 * p1 + a];
        xa += g[0] * d;
        ya += g[1] * d;
        xb += g[2] * v;
        yb += g[3] * v;
      }
      c = xa * yb - xb * ya;
    }
    if (G.coef_kind == TW_COEF_DENSITY) c *= density_at(G, A.xq[k1], B.xq[k2]);
  }
  Cg[id] = c;
}

// ---------------------------------------------------------------------------
// cut-element rule (Sect. 3.1, reading R6).  Pass 0 counts, pass 1 writes.

__device__ void sort_small(double *v, int n) {
  for (int i = 1; i < n; i++) {
    double x = v[i];
    int j = i - 1;
    while (j >= 0 && v[j] > x) {
      v[j + 1] = v[j];
      j--;
    }
    v[j + 1] = x;
  }
}

// Curve-wide features, once per patch: tangent points of both kinds (the
// curve's tangent parallel to an axis) and the spline's segment joints.
// feat[(kind * fcap + k) * 2 + {0,1}], nfeat[kind], kind 2 = joints.  One
// warp per kind; a spline's segments are spread over the lanes and their
// points placed in segment order by a warp scan of the counts.
__device__ __forceinline__ void curve_features_warp(const CurveSet &S, int kind, int lane,
                                                    double *feat, int *nfeat, int fcap,
                                                    int *flag) {
  double *out = feat + (size_t)kind * fcap * 2;
  int n = 0;  // warp-uniform
  bool over = false;
  for (int ci = 0; ci < S.n && !over; ci++) {
    const Curve &C = S.c[ci];
    if (kind < 2 && C.kind == TW_TRIM_BSPLINE3) {
      int add = 0;  // this curve's points so far
      for (int s0 = 0; s0 < C.nc; s0 += 32) {
        const int sg = s0 + lane;
        double f[4];
        const int m = sg < C.nc ? seg_folds(C, sg, kind, f) : 0;
        int incl = m;
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        if (n + add + tot > fcap) {
          over = true;
          break;
        }
        for (int k = 0; k < 2 * m; k++) out[2 * (n + add + incl - m) + k] = f[k];
        add += tot;
      }
      if (!over) n += add;
    } else if (kind < 2) {
      // a conic writes its two tangent points unchecked
      int m = -1;
      if (lane == 0) m = fcap - n >= 2 ? curve_folds(C, kind, out + 2 * n, fcap - n) : -1;
      m = __shfl_sync(0xffffffffu, m, 0);
      if (m < 0) over = true;
      else n += m;
    } else if (C.kind == TW_TRIM_BSPLINE3) {
      const int m = min(C.nc, fcap - n);
      for (int sg = lane; sg < m; sg += 32) {
        out[2 * (n + sg)] = C.seg[8 * sg];
        out[2 * (n + sg) + 1] = C.seg[8 * sg + 4];
      }
      n += m;
    }
  }
  if (lane == 0) {
    if (over) atomicOr(flag, TWF_HITCAP);
    nfeat[kind] = n;
  }
}

// the knot lines' crossings (one-warp blocks [0, nbl), a line per thread) and
// the curve-wide features (three more blocks, a kind per block) in one launch
__global__ void __launch_bounds__(32) k_curve_lines(CurveSet C, Dir A, Dir B, double *hits,
                                                    int *nh, int nbl, double *feat, int *nfeat,
                                                    int fcap, int *flag) {
  const int b = blockIdx.x;
  if (b < nbl) {
    const int l = b * 32 + threadIdx.x;
    if (l < (A.nel + 1) + (B.nel + 1) + B.nel) line_hits_item(C, A, B, l, hits, nh, flag);
  } else {
    curve_features_warp(C, b - nbl, threadIdx.x, feat, nfeat, fcap, flag);
  }
}

// One block of 64 threads per cut element.  Pass 0 (pts == NULL) counts the
// element's points into cnt[ci] and, given scr, also writes them to the
// element's slot of cap points there (elements with more points leave cnt >
// cap and are counted in *ovf); pass 1 writes them from off[ci] on.  Order:
// piece, Gauss line, interval, inner Gauss point.  The element's edge
// crossings come from the knot-line table (hits/nh of k_curve_lines), the
// tangent points and joints from the curve-wide feature list; only the Gauss
// lines are solved here.  The visibility of a line's first interval is that of
// its end on the element edge, i.e. the parity of the edge line's crossings
// beyond it (the same ray test as curve_inside, read from the table).
// Cut-element rules (reading R6) in three flat passes, so that every lane of
// the root finding has a Gauss line of its own (a block per element left
// three quarters of the lanes idle):
//  k_cut_breaks  thread per cut element: inner direction and the sorted
//                breakpoints of the outer interval; (pieces) x q lines
//  k_cut_lines   thread per Gauss line of every element: the curve's
//                crossings of the line (stored) and the line's point count
//  k_cut_write   thread per line: its points, after the scan of the counts
// The points are grouped by element, then by line, visible interval and
// Gauss point.

// per element: cut_o, the breakpoints (br[ci * TW_BRCAP ..]) and its line count
__global__ void k_cut_breaks(Dir A, Dir B, const int32_t *cut_list, int ncut, int q,
                             const double *hits, const int *nh, const double *feat,
                             const int *nfeat, int fcap, int32_t *cut_o, int32_t *nbr_out,
                             double *br_all, int64_t *nlines, int *flag) {
  const int ci = blockIdx.x * blockDim.x + threadIdx.x;
  if (ci == 0) nlines[ncut] = 0;  // closes the counts for their exclusive scan
  if (ci >= ncut) return;
  const int e = cut_list[ci];
  const int e1 = e % A.nel, e2 = e / A.nel;
  const double a[2] = {A.bp[e1], B.bp[e2]}, b[2] = {A.bp[e1 + 1], B.bp[e2 + 1]};
  const double dl[2] = {TW_CORNER * (b[0] - a[0]), TW_CORNER * (b[1] - a[1])};
  const int hv = A.nel + 1;  // first horizontal knot line in the table
  // knot lines of the four edges: [o][side] (o = 0: x = const, o = 1: y = const)
  const int eline[2][2] = {{e1, e1 + 1}, {hv + e2, hv + e2 + 1}};
  double *br = br_all + (size_t)ci * TW_BRCAP;
  int bad = 0;
  // 1. extent of the curve in the box: edge crossings and tangent points,
  //    each counted up to TW_CORNER beyond the element
  double lo0 = 1e300, lo1 = 1e300, hi0 = -1e300, hi1 = -1e300;
  for (int o = 0; o < 2; o++)
    for (int sd = 0; sd < 2; sd++) {
      int l = eline[o][sd];
      double sv = sd ? b[o] : a[o];
      const double *h = hits + (size_t)l * TW_HITCAP;
      for (int k = 0; k < nh[l]; k++) {
        double v = h[k];
        if (!(v > a[1 - o] - dl[1 - o] && v < b[1 - o] + dl[1 - o])) continue;
        double X = o == 0 ? sv : v, Y = o == 0 ? v : sv;
        lo0 = fmin(lo0, X); hi0 = fmax(hi0, X); lo1 = fmin(lo1, Y); hi1 = fmax(hi1, Y);
      }
    }
  for (int kind = 0; kind < 2; kind++)
    for (int k = 0; k < nfeat[kind]; k++) {
      double X = feat[((size_t)kind * fcap + k) * 2], Y = feat[((size_t)kind * fcap + k) * 2 + 1];
      if (X >= a[0] - dl[0] && X <= b[0] + dl[0] && Y >= a[1] - dl[1] && Y <= b[1] + dl[1]) {
        lo0 = fmin(lo0, X); hi0 = fmax(hi0, X); lo1 = fmin(lo1, Y); hi1 = fmax(hi1, Y);
      }
    }
  // equal extents within TW_TIE of the element size: o = 0
  const int o = (hi0 - lo0 >= hi1 - lo1 - TW_TIE * fmax(b[0] - a[0], b[1] - a[1])) ? 0 : 1;
  const int in = 1 - o;
  // 2. breakpoints along o: crossings of the two edges parallel to o, tangent
  //    points that fold the lines xi_o = const, the spline's segment joints
  int n = 0;
  br[n++] = a[o];
  br[n++] = b[o];
  for (int sd = 0; sd < 2 && !bad; sd++) {
    int l = eline[in][sd];
    const double *h = hits + (size_t)l * TW_HITCAP;
    for (int k = 0; k < nh[l]; k++)
      if (h[k] > a[o] && h[k] < b[o]) {
        if (n >= TW_BRCAP) { bad = 1; break; }
        br[n++] = h[k];
      }
  }
  const int kinds[2] = {o, 2};
  for (int kk = 0; kk < 2 && !bad; kk++) {
    int kind = kinds[kk];
    for (int k = 0; k < nfeat[kind]; k++) {
      const double *f = feat + ((size_t)kind * fcap + k) * 2;
      double xo = f[o], xi = f[in];
      if (xo > a[o] && xo < b[o] && xi >= a[in] && xi <= b[in]) {
        if (n >= TW_BRCAP) { bad = 1; break; }
        br[n++] = xo;
      }
    }
  }
  if (bad) {
    atomicOr(flag, TWF_BRCAP);
    n = 1;
  } else {
    sort_small(br, n);
  }
  cut_o[ci] = o;
  nbr_out[ci] = n;
  nlines[ci] = (int64_t)(n - 1) * q;
}

// the element of line li: the last ci with line_off[ci] <= li
__device__ __forceinline__ int cut_line_elem(const int64_t *line_off, int ncut, int64_t li) {
  int lo = 0, hi = ncut - 1;
  while (lo < hi) {
    const int m = (lo + hi + 1) >> 1;
    if (line_off[m] <= li) lo = m;
    else hi = m - 1;
  }
  return lo;
}

// one Gauss line: its coordinate s, weight ws and inner interval [lo, hi]
struct CutLine {
  int ci, o;
  double s, ws, lo, hi;
};

__device__ __forceinline__ CutLine cut_line(Dir A, Dir B, const int32_t *cut_list,
                                            const int32_t *cut_o, const double *br_all,
                                            const int64_t *line_off, int ncut, int q,
                                            const double *qgx, const double *qgw, int64_t li) {
  CutLine L;
  L.ci = cut_line_elem(line_off, ncut, li);
  const int e = cut_list[L.ci], e1 = e % A.nel, e2 = e / A.nel;
  L.o = cut_o[L.ci];
  const int in = 1 - L.o;
  const int64_t loc = li - line_off[L.ci];
  const int pc = (int)(loc / q), g = (int)(loc % q);
  const double *br = br_all + (size_t)L.ci * TW_BRCAP;
  const double s0 = br[pc], s1 = br[pc + 1];
  L.s = s0 + (s1 - s0) * 0.5 * (qgx[g] + 1.0);
  L.ws = qgw[g] * 0.5 * (s1 - s0);
  L.lo = in == 0 ? A.bp[e1] : B.bp[e2];
  L.hi = in == 0 ? A.bp[e1 + 1] : B.bp[e2 + 1];
  if (!(s1 > s0)) L.ws = -1.0;  // an empty piece: no points
  return L;
}

// crossings (lh[li * TW_HITCAP ..], ln[li] of them; -1 for an empty piece),
// the visibility of the first interval and the line's point count
__global__ void k_cut_lines(CurveSet C, Dir A, Dir B, const int32_t *cut_list, int ncut, int q,
                            const double *qgx, const double *qgw, const double *hits,
                            const int *nh, const int32_t *cut_o, const double *br_all,
                            const int64_t *line_off, const int64_t *nl_tot, double *lh,
                            int32_t *ln, uint64_t *lvis, int64_t *lcnt, int *flag) {
  const int64_t L = *nl_tot;
  if (blockIdx.x == 0 && threadIdx.x == 0) lcnt[L] = 0;  // closes the counts for their scan
  for (int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; li < L;
       li += (int64_t)gridDim.x * blockDim.x) {
    const CutLine cl = cut_line(A, B, cut_list, cut_o, br_all, line_off, ncut, q, qgx, qgw, li);
    int64_t count = 0;
    int n = -1;
    uint64_t vis = 0;  // bit k: interval k of the line is visible
    if (cl.ws >= 0.0) {
      double h[TW_HITCAP + 2];
      n = set_line_hits(C, cl.o, cl.s, cl.lo, cl.hi, h + 1, TW_HITCAP);
      if (n < 0) {
        atomicOr(flag, TWF_HITCAP);
        n = -1;
      } else {
        h[0] = cl.lo;
        h[n + 1] = cl.hi;
        if (C.n == 1) {
          // one closed curve: the first interval's visibility from the parity
          // of the edge line's crossings beyond the line's first end, then
          // alternation at each crossing
          const Curve &C0 = C.c[0];
          const int e = cut_list[cl.ci], e1 = e % A.nel, e2 = e / A.nel;
          const int lfirst = cl.o == 1 ? e1 : A.nel + 1 + e2;
          const double *eh = hits + (size_t)lfirst * TW_HITCAP;
          int right = 0;
          for (int k = 0; k < nh[lfirst]; k++) right += eh[k] > cl.s;
          int inside = right & 1;
          if (C0.kind == TW_TRIM_LINE) {  // a half-plane: test the first interval's midpoint
            const double um = 0.5 * (h[0] + h[1]);
            inside = cl.o == 0 ? curve_inside(C0, cl.s, um) : curve_inside(C0, um, cl.s);
          }
          const int vis0 = C0.keep_inside ? inside : !inside;
          for (int k = 0; k <= n; k++)
            if (vis0 ^ (k & 1)) vis |= 1ull << k;
        } else {
          // several curves: each interval's midpoint against every kept side
          for (int k = 0; k <= n; k++) {
            const double um = 0.5 * (h[k] + h[k + 1]);
            const int v = cl.o == 0 ? set_visible(C, cl.s, um) : set_visible(C, um, cl.s);
            if (v) vis |= 1ull << k;
          }
        }
        for (int k = 0; k <= n; k++)
          if (h[k + 1] > h[k] && ((vis >> k) & 1ull)) count += q;
        for (int k = 0; k < n; k++) lh[li * TW_HITCAP + k] = h[k + 1];
      }
    }
    ln[li] = n;
    lvis[li] = vis;
    lcnt[li] = count;
  }
}

// thread per Gauss line: its points; the thread of an element's first line
// also writes the element's first point index (cut_off[ci]; every element of
// a successful set-up has at least one line), line 0 the total (cut_off[ncut])
__global__ void k_cut_write(Dir A, Dir B, const int32_t *cut_list, int ncut, int q,
                            const double *qgx, const double *qgw, const int32_t *cut_o,
                            const double *br_all, const int64_t *line_off, const int64_t *nl_tot,
                            const double *lh, const int32_t *ln, const uint64_t *lvis,
                            const int64_t *lpos, const int64_t *npts, int64_t *cut_off,
                            double *pts) {
  const int64_t L = *nl_tot;
  for (int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; li < L;
       li += (int64_t)gridDim.x * blockDim.x) {
    const CutLine cl = cut_line(A, B, cut_list, cut_o, br_all, line_off, ncut, q, qgx, qgw, li);
    if (line_off[cl.ci] == li) cut_off[cl.ci] = lpos[li];
    if (li == 0) cut_off[ncut] = *npts;
    const int n = ln[li];
    if (n < 0) continue;
    const uint64_t vis = lvis[li];
    double *dst = pts + 3 * lpos[li];
    int64_t w0 = 0;
    for (int k = 0; k <= n; k++) {
      const double u0 = k == 0 ? cl.lo : lh[li * TW_HITCAP + k - 1];
      const double u1 = k == n ? cl.hi : lh[li * TW_HITCAP + k];
      if (!(u1 > u0) || !((vis >> k) & 1ull)) continue;
      for (int hh = 0; hh < q; hh++) {
        double u = u0 + (u1 - u0) * 0.5 * (qgx[hh] + 1.0);
        double w = cl.ws * qgw[hh] * 0.5 * (u1 - u0);
        double *o3 = dst + 3 * w0;
        o3[0] = cl.o == 0 ? cl.s : u;
        o3[1] = cl.o == 0 ? u : cl.s;
        o3[2] = w;
        w0++;
      }
    }
  }
}

// per element: offset of its first point (cut_off[ncut] = all points)
__global__ void k_cut_offsets(int ncut, const int64_t *line_off, const int64_t *lpos,
                              const int64_t *npts, int64_t *cut_off) {
  const int ci = blockIdx.x * blockDim.x + threadIdx.x;
  if (ci < ncut) cut_off[ci] = lpos[line_off[ci]];
  if (ci == ncut) cut_off[ci] = *npts;
}


// per cut point: basis values in both directions and w * c.  The points come
// in Gauss lines of constant outer coordinate (R6); for the spline geometry
// the outer direction's basis and the control-net sums over it are formed once
// per line, so det J costs 4(p+1) FMAs per point instead of 4(p+1)^2.  One
// warp per cut element walks its points in chunks of 32: a ballot marks the
// lines that open in the chunk, the opening lane forms its line's outer basis,
// the lanes then form the control-net sums per (line, j), and each lane
// finishes its point; the warp synchronises only with itself.
#define TW_CPT_WARPS 4
#define TW_CPT_THREADS (32 * TW_CPT_WARPS)
__global__ void __launch_bounds__(TW_CPT_THREADS)
    k_cut_point_tables(Geo G, Dir A, Dir B, const int32_t *cut_list, const int64_t *off,
                       const int32_t *cut_o, int ncut, const double *pts, double *Bt,
                       double *wc) {
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ci = blockIdx.x * TW_CPT_WARPS + wib;
  if (ci >= ncut) return;  // the whole warp
  const int e = cut_list[ci];
  const int e1 = e % A.nel, e2 = e / A.nel, p = A.p, p1 = p + 1;
  const int o = cut_o[ci], in = 1 - o;
  const int eo = o == 0 ? e1 : e2, ei = o == 0 ? e2 : e1;
  const double *Uo = o == 0 ? A.U : B.U, *Ui = o == 0 ? B.U : A.U;
  const bool geo = G.geom_kind == TW_GEOM_SPLINE && G.coef_kind != TW_COEF_ONE;
  // per warp: the lines of the current chunk (at most 32)
  __shared__ double OVs[TW_CPT_WARPS][32][TW_MAXP1], ODs[TW_CPT_WARPS][32][TW_MAXP1];
  __shared__ double LSs[TW_CPT_WARPS][32][4][TW_MAXP1];  // control-net sums over the outer index
  // reciprocal knot differences of the element's outer and inner spans
  __shared__ double rcos[TW_CPT_WARPS][TW_SPAN_RC], rdos[TW_CPT_WARPS][TW_MAXP1];
  __shared__ double rcis[TW_CPT_WARPS][TW_SPAN_RC], rdis[TW_CPT_WARPS][TW_MAXP1];
  // the element's (p+1) x (p+1) block of the geometry's control net, [b][a]
  __shared__ double CPs[TW_CPT_WARPS][TW_MAXP1 * TW_MAXP1][2];
  double(*OV)[TW_MAXP1] = OVs[wib];
  double(*OD)[TW_MAXP1] = ODs[wib];
  double(*LS)[4][TW_MAXP1] = LSs[wib];
  double *rco = rcos[wib], *rdo = rdos[wib], *rci = rcis[wib], *rdi = rdis[wib];
  {  // both spans' reciprocal tables, one entry per lane
    const int ne = p * (p + 1) / 2 + p + 1;
    for (int t = lane; t < 2 * ne; t += 32) {
      const bool ot = t < ne;
      span_recip_entry(ot ? Uo : Ui, (ot ? eo : ei) + p, p, ot ? t : t - ne, ot ? rco : rci,
                       ot ? rdo : rdi);
    }
  }
  double(*CP)[2] = CPs[wib];
  if (geo)
    for (int t = lane; t < p1 * p1; t += 32) {
      const double *pt = G.ctrl + 2 * ((size_t)(e2 + t / p1) * G.n1 + (e1 + t % p1));
      CP[t][0] = pt[0];
      CP[t][1] = pt[1];
    }
  __syncwarp();
  const int64_t k0 = off[ci], k1 = off[ci + 1];
  for (int64_t base = k0; base < k1; base += 32) {
    const int64_t k = base + lane;
    const bool live = k < k1;
    // a line opens at the chunk's first point and where the outer coordinate changes
    const double so = live ? pts[3 * k + o] : 0.0;
    const bool start = live && (lane == 0 || so != pts[3 * (k - 1) + o]);
    const unsigned m = __ballot_sync(0xffffffffu, start);
    const int nl = __popc(m);
    // line of this point = (line starts up to and including it) - 1
    const int l = __popc(m & ((2u << lane) - 1u)) - 1;
    if (start) {  // the line's outer basis, once
      double v[TW_MAXP1], d[TW_MAXP1];
      basis_ders_rc(Uo, eo + p, so, p, rco, rdo, v, d);
      for (int a = 0; a <= p; a++) {
        OV[l][a] = v[a];
        OD[l][a] = d[a];
      }
    }
    __syncwarp();
    // per line and inner index j: the control net summed over the outer index
    // (o = 0: over a for each b = j; o = 1: over b for each a = j)
    if (geo)
      for (int u = lane; u < nl * p1; u += 32) {
        const int L = u / p1, j = u % p1;
        double sxd = 0, syd = 0, sxv = 0, syv = 0;
        for (int a = 0; a <= p; a++) {
          const double *pt = CP[o == 0 ? j * p1 + a : a * p1 + j];  // control point (e1+., e2+.)
          sxd += pt[0] * OD[L][a];
          syd += pt[1] * OD[L][a];
          sxv += pt[0] * OV[L][a];
          syv += pt[1] * OV[L][a];
        }
        LS[L][0][j] = sxd;
        LS[L][1][j] = syd;
        LS[L][2][j] = sxv;
        LS[L][3][j] = syv;
      }
    __syncwarp();
    if (live) {
      const double x1 = pts[3 * k], x2 = pts[3 * k + 1];
      const double xi = o == 0 ? x2 : x1;
      double v[TW_MAXP1], d[TW_MAXP1];
      basis_ders_rc(Ui, ei + p, xi, p, rci, rdi, v, d);
      for (int a = 0; a < p1; a++) {
        Bt[(2 * k + o) * p1 + a] = OV[l][a];
        Bt[(2 * k + in) * p1 + a] = v[a];
      }
      double c = 1.0;
      if (G.coef_kind != TW_COEF_ONE) {
        if (geo) {
          // derivative along the outer direction: outer-derivative sums times the
          // inner values; along the inner one: outer-value sums times the inner
          // derivatives
          double xo = 0, yo = 0, xn = 0, yn = 0;
          for (int j = 0; j <= p; j++) {
            xo += LS[l][0][j] * v[j];
            yo += LS[l][1][j] * v[j];
            xn += LS[l][2][j] * d[j];
            yn += LS[l][3][j] * d[j];
          }
          // det J = x_xi1 y_xi2 - x_xi2 y_xi1
          c = o == 0 ? xo * yn - xn * yo : xn * yo - xo * yn;
        }
        if (G.coef_kind == TW_COEF_DENSITY) c *= density_at(G, x1, x2);
      }
      wc[k] = pts[3 * k + 2] * c;
    }
    __syncwarp();  // the chunk's line data are rewritten by the next chunk
  }
}


// c at the Gauss points of the listed elements, one warp per element.  For the
// spline geometry the control net is contracted over direction 1 once per
// (g1, b) and then per point over b: the same sums, in the same order, as
// coef_from, with 4 (p+1)^3 instead of 4 (p+1)^4 products per element.
__device__ __forceinline__ void gauss_c_warp(const Geo &G, const Dir &A, const Dir &B,
                                             const int32_t *glist, double *gc, int sl, int lane,
                                             double (*T)[TW_MAXP1][4]) {
  const int p = A.p, p1 = p + 1;
  const int e = glist[sl], e1 = e % A.nel, e2 = e / A.nel;
  const bool spline = G.geom_kind == TW_GEOM_SPLINE && G.coef_kind != TW_COEF_ONE;
  if (spline) {
    for (int t = lane; t < p1 * p1; t += 32) {
      const int g1 = t / p1, bb = t % p1;
      const double *v1 = A.GB + (e1 * p1 + g1) * p1, *d1 = A.dGB + (e1 * p1 + g1) * p1;
      double sxa = 0, sya = 0, sxb = 0, syb = 0;
      for (int aa = 0; aa <= p; aa++) {
        const double *pt = G.ctrl + 2 * ((size_t)(e2 + bb) * G.n1 + (e1 + aa));
        sxa += pt[0] * d1[aa];
        sya += pt[1] * d1[aa];
        sxb += pt[0] * v1[aa];
        syb += pt[1] * v1[aa];
      }
      T[g1][bb][0] = sxa;
      T[g1][bb][1] = sya;
      T[g1][bb][2] = sxb;
      T[g1][bb][3] = syb;
    }
    __syncwarp();
  }
  for (int t = lane; t < p1 * p1; t += 32) {
    const int g1 = t % p1, g2 = t / p1;
    double c = 1.0;
    if (G.coef_kind != TW_COEF_ONE) {
      double dj = 1.0;
      if (G.geom_kind == TW_GEOM_SPLINE) {
        const double *v2 = B.GB + (e2 * p1 + g2) * p1, *d2 = B.dGB + (e2 * p1 + g2) * p1;
        double xa = 0, ya = 0, xb = 0, yb = 0;
        for (int bb = 0; bb <= p; bb++) {
          xa += T[g1][bb][0] * v2[bb];
          ya += T[g1][bb][1] * v2[bb];
          xb += T[g1][bb][2] * d2[bb];
          yb += T[g1][bb][3] * d2[bb];
        }
        dj = xa * yb - xb * ya;
      }
      if (G.coef_kind == TW_COEF_DENSITY) {
        const double x1 = A.bp[e1] + (A.bp[e1 + 1] - A.bp[e1]) * 0.5 * (A.gx[g1] + 1.0);
        const double x2 = B.bp[e2] + (B.bp[e2 + 1] - B.bp[e2]) * 0.5 * (B.gx[g2] + 1.0);
        dj *= density_at(G, x1, x2);
      }
      c = dj;
    }
    gc[(size_t)sl * p1 * p1 + g2 * p1 + g1] = c;
  }
}

// stage A of the grid's det J (blocks [0, nbA), a (k2, i1) per thread) and the
// element-Gauss c tables (the other blocks, an element per warp) in one launch
#define TW_GC_WARPS 8
__global__ void __launch_bounds__(32 * TW_GC_WARPS)
    k_geo_gauss_c(Geo G, Dir A, Dir B, double *Gt, int nbA, const int32_t *glist, int ng,
                  double *gc) {
  __shared__ double T[TW_GC_WARPS][TW_MAXP1][TW_MAXP1][4];
  if ((int)blockIdx.x < nbA) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id < B.nq * A.n) geo_stageA_item(G, A, B, Gt, id);
    return;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int sl = ((int)blockIdx.x - nbA) * TW_GC_WARPS + w;
  if (sl < ng) gauss_c_warp(G, A, B, glist, gc, sl, lane, T[w]);
}

// ---------------------------------------------------------------------------
// DWQ (Sect. 3.3)

// R7: region R = R1 x R2 of regular (or empty) elements with simple discs and
// the most elements.  One
// warp per cut function (from the compacted list of cut functions, count on
// the device): the support's elements are counted into a 2-D prefix table of
// non-regular elements, so each candidate's "all regular" test is four
// lookups; lanes take the candidates c = oa * nopt1 + ob (the order of the
// tie rules) and a warp max over the key (elements, fewer discs, earlier c)
// picks the first best candidate.
#define TW_CHOICE_WARPS 4
__global__ void __launch_bounds__(32 * TW_CHOICE_WARPS)
    k_dwq_choice(Dir A, Dir B, const uint8_t *estate, const int32_t *cutfn,
                 const int32_t *ncutfn, int32_t *choice, int32_t *dflag0, int32_t *dflag1,
                 int32_t *counter) {
  constexpr int PW = TW_MAXP1 + 1;  // prefix table width (support <= p+1 elements)
  __shared__ int pre[TW_CHOICE_WARPS][PW * PW];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int *T = pre[wib];
  const int nitems = *ncutfn;
  for (int item = blockIdx.x * TW_CHOICE_WARPS + wib; item < nitems;
       item += gridDim.x * TW_CHOICE_WARPS) {
    const int g = cutfn[item];
    const int i[2] = {g % A.n, g / A.n};
    const Dir *D[2] = {&A, &B};
    int lo[2], hi[2], nopt[2];
    for (int d = 0; d < 2; d++) {
      lo[d] = max(0, i[d] - D[d]->p);
      hi[d] = min(D[d]->nel - 1, i[d]);
      nopt[d] = 1 + 2 * (hi[d] - lo[d]);
    }
    const int w1 = hi[0] - lo[0] + 1, w2 = hi[1] - lo[1] + 1;
    // T[y][x] = non-regular elements in [lo0, lo0 + x) x [lo1, lo1 + y)
    for (int t = lane; t < PW * PW; t += 32) T[t] = 0;
    __syncwarp();
    for (int t = lane; t < w1 * w2; t += 32) {  // empty elements have no measure
      const int x = t % w1, y = t / w1;
      const uint8_t st = estate[(lo[1] + y) * A.nel + lo[0] + x];
      T[(y + 1) * PW + x + 1] = st != TW_ELEM_REGULAR && st != TW_ELEM_EMPTY;
    }
    __syncwarp();
    if (lane < w2)  // prefix along x, row by row
      for (int x = 1; x <= w1; x++) T[(lane + 1) * PW + x] += T[(lane + 1) * PW + x - 1];
    __syncwarp();
    if (lane <= w1)  // then along y, column by column
      for (int y = 1; y <= w2; y++) T[y * PW + lane] += T[(y - 1) * PW + lane];
    __syncwarp();
    int best = 0;
    for (int c = lane; c < nopt[0] * nopt[1]; c += 32) {
      const int oo[2] = {c / nopt[1], c % nopt[1]};
      int kind[2], r0[2], r1[2];
      for (int d = 0; d < 2; d++) {
        const int m = hi[d] - lo[d];
        if (oo[d] == 0) { kind[d] = 0; r0[d] = lo[d]; r1[d] = hi[d]; }
        else if (oo[d] <= m) { kind[d] = 1; r0[d] = lo[d]; r1[d] = lo[d] + oo[d] - 1; }
        else { kind[d] = 2; r0[d] = lo[d] + oo[d] - m; r1[d] = hi[d]; }
      }
      const int x0 = r0[0] - lo[0], x1 = r1[0] - lo[0] + 1;
      const int y0 = r0[1] - lo[1], y1 = r1[1] - lo[1] + 1;
      const int bad = T[y1 * PW + x1] - T[y0 * PW + x1] - T[y1 * PW + x0] + T[y0 * PW + x0];
      if (bad) continue;
      // a disc is a simple knot: t inserted p times reaches multiplicity p+1
      bool simple = true;
      for (int d = 0; d < 2; d++)
        if (kind[d] != 0) {
          const double *bp = D[d]->bp;
          const int sv = kind[d] == 1 ? r1[d] + 1 : r0[d];
          simple = simple && bp[sv - 1] < bp[sv] && bp[sv] < bp[sv + 1];
        }
      if (!simple) continue;
      const int nel = (x1 - x0) * (y1 - y0);
      const int disc = (kind[0] != 0) + (kind[1] != 0);
      const int key = (nel << 16) | ((3 - disc) << 10) | (1023 - c);
      best = max(best, key);
    }
    best = __reduce_max_sync(0xffffffffu, best);
    if (best > 0 && lane == 0) {
      const int c = 1023 - (best & 1023);
      const int oo[2] = {c / nopt[1], c % nopt[1]};
      int out[4];
      for (int d = 0; d < 2; d++) {
        const int m = hi[d] - lo[d];
        if (oo[d] == 0) { out[2 * d] = 0; out[2 * d + 1] = -1; }
        else if (oo[d] <= m) { out[2 * d] = 1; out[2 * d + 1] = lo[d] + oo[d]; }
        else { out[2 * d] = 2; out[2 * d + 1] = lo[d] + oo[d] - m; }
      }
      int32_t *o = choice + 4 * g;
      o[0] = out[0]; o[1] = out[1]; o[2] = out[2]; o[3] = out[3];
      if (out[0]) dflag0[out[1]] = 1;
      if (out[2]) dflag1[out[3]] = 1;
      atomicAdd(counter, 1);
    }
    __syncwarp();  // T is reused by the warp's next function
  }
}

// refined knot vector after inserting t = U[p+s] p more times
__device__ __forceinline__ double ref_knot(const Dir &D, int s, int k) {
  int p = D.p;
  if (k <= p + s) return D.U[k];
  if (k <= 2 * p + s) return D.U[p + s];
  return D.U[k - p];
}

// values of the p+1 refined functions on the element e of x: the triangular
// scheme with knots K[0..2p-1] = U'[span-p+1 .. span+p], its denominators
// K[p+r] - K[p-j+r] taken as the reciprocals rc[j(j-1)/2 + r] of that span
// (formed once per window element and shared by its points)
static __device__ __noinline__ void ref_basis_rc(const Dir &D, int s, int e, double x,
                                                 const double *rc, double *N) {
  int p = D.p;
  int span = e + p + (e >= s ? p : 0);
  double K[2 * TW_MAXP + 2];
  for (int k = 0; k < 2 * p; k++) K[k] = ref_knot(D, s, span - p + 1 + k);
  double left[TW_MAXP1], right[TW_MAXP1];
  N[0] = 1.0;
  for (int j = 1; j <= p; j++) {
    left[j] = x - K[p - j];
    right[j] = K[p - 1 + j] - x;
    double saved = 0.0;
    for (int r = 0; r < j; r++) {
      const double t = N[r] * rc[j * (j - 1) / 2 + r];
      N[r] = saved + right[r + 1] * t;
      saved = left[j - r] * t;
    }
    N[j] = saved;
  }
}


// The DWQ rules of both directions' disc knots, written per direction.
struct DwqOut {
  const int32_t *list;  // disc knots s (element index of t = bp[s])
  int n;
  double *x, *w, *B, *dB;
  int32_t *np, *k, *e, *r;
};

// One block per disc knot t = bp[s], the blocks of direction 0 first, then
// those of direction 1 (one launch for both): steps 1-4 of Sect. 3.3.  The
// refined basis is tabulated once per window point and per window Gauss point
// (shared memory); each refined system is then assembled by lookup and solved
// by its own warp.
#define TW_DWQ_THREADS 128  // 4 warps: three solve the 2p <= 12 refined systems (step 3)
#define TW_DWQ_G 8          // lanes per refined system in the solves
#define TW_DWQ_SMEM (sizeof(double) * 2 * TW_MAXP * TW_WIN * (TW_QMAX + 1))
__global__ void __launch_bounds__(TW_DWQ_THREADS)
    k_dwq_build(Dir A, Dir B, DwqOut o0, DwqOut o1, int *flag) {
  const bool d1 = (int)blockIdx.x >= o0.n;
  const int slot = d1 ? (int)blockIdx.x - o0.n : (int)blockIdx.x;
  const DwqOut &O = d1 ? o1 : o0;
  if (slot >= O.n) return;
  const Dir &D = d1 ? B : A;
  double *out_x = O.x, *out_w = O.w, *out_B = O.B, *out_dB = O.dB;
  int32_t *out_np = O.np, *out_k = O.k, *out_e = O.e, *out_r = O.r;
  int s = O.list[slot];
  int p = D.p, p1 = p + 1;
  double t = D.bp[s];
  __shared__ double xs[TW_LQMAX];
  __shared__ int xk[TW_LQMAX];                   // base point index, -1 for a nested point
  __shared__ double RB[TW_LQMAX][TW_MAXP1];      // refined functions on each point's span
  __shared__ int rsp[TW_LQMAX];                  // first refined function of that span
  __shared__ double RG[2 * TW_MAXP][TW_MAXP1][TW_MAXP1];  // [window element][g][a]
  __shared__ double GWt[2 * TW_MAXP][TW_MAXP1];  // Gauss weight x half the element length
  __shared__ int npts;
  __shared__ double Sc[TW_MAXP][TW_MAXP1];             // S[i + r][i], i = s + col
  __shared__ double Wt[2 * TW_MAXP][TW_LQMAX];         // refined weights of l = s + row
  int ewlo = max(0, s - p), ewhi = min(D.nel - 1, s + p - 1);
  int nwe = ewhi - ewlo + 1;
  // refined points: base points + nested points next to t (R5).  Lane e of the
  // first warp assembles and sorts window element e's points (at most p + 1),
  // a warp scan of the counts places them
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x, e = ewlo + lane;
    int m = 0, add = 0, k0 = 0;
    if (lane < nwe) {
      k0 = wq_off(D, e);
      m = wq_off(D, e + 1) - k0;
      if ((e == s - 1 || e == s) && m < p1) add = p1 - m;
    }
    const int cnt = m + add;
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int off = incl - cnt;
    if (lane < nwe && total <= TW_LQMAX) {
      double lx[TW_MAXP1 + 1];
      int lk[TW_MAXP1 + 1];
      int n = 0;
      for (int k = k0; k < k0 + m; k++) {
        lx[n] = D.xq[k];
        lk[n] = k;
        n++;
      }
      if (add > 0) {
        // gaps (a, x1), (x1, x2), (x2, b); fewest points first, ties: middle,
        // then the gap next to t, then the other
        double ed[4] = {D.bp[e], D.xq[k0], D.xq[k0 + 1], D.bp[e + 1]};
        int gc[3] = {0, 0, 0};
        int nearg = (e == s - 1) ? 2 : 0;
        int pref[3] = {1, nearg, 2 - nearg};
        for (int r = 0; r < add; r++) {
          int best = pref[0];
          for (int k = 1; k < 3; k++)
            if (gc[pref[k]] < gc[best]) best = pref[k];
          gc[best]++;
        }
        for (int gp = 0; gp < 3; gp++)
          for (int j = 0; j < gc[gp]; j++) {
            lx[n] = ed[gp] + (ed[gp + 1] - ed[gp]) * (double)(j + 1) / (double)(gc[gp] + 1);
            lk[n] = -1;
            n++;
          }
      }
      // insertion sort of the element's (x, k) pairs
      for (int a2 = 1; a2 < n; a2++) {
        double x = lx[a2];
        int kk = lk[a2], b2 = a2 - 1;
        while (b2 >= 0 && lx[b2] > x) {
          lx[b2 + 1] = lx[b2];
          lk[b2 + 1] = lk[b2];
          b2--;
        }
        lx[b2 + 1] = x;
        lk[b2 + 1] = kk;
      }
      for (int j = 0; j < n; j++) {
        xs[off + j] = lx[j];
        xk[off + j] = lk[j];
      }
    }
    if (lane == 0) {
      if (total > TW_LQMAX) atomicOr(flag, TWF_LQMAX);
      npts = total > TW_LQMAX ? 0 : total;
    }
  }
  // reciprocal knot differences of the window elements' refined spans and of
  // their coarse spans, in the third and fourth warps (an empty span's entries
  // are never read)
  __shared__ double rcw[2 * TW_MAXP][TW_SPAN_RC];
  __shared__ double rcc[2 * TW_MAXP][TW_SPAN_RC], rdc[2 * TW_MAXP][TW_MAXP1];
  if (threadIdx.x >= 64) {
    const int nrc = p * (p + 1) / 2, ne = nrc + p + 1;
    for (int id = (int)threadIdx.x - 64; id < nwe * (nrc + ne); id += (int)blockDim.x - 64) {
      if (id < nwe * nrc) {
        const int el = id / nrc, t0 = id - el * nrc, e = ewlo + el;
        int j = 1, r = t0;
        while (r >= j) {
          r -= j;
          j++;
        }
        const int span = e + p + (e >= s ? p : 0);
        rcw[el][t0] = 1.0 / (ref_knot(D, s, span + 1 + r) - ref_knot(D, s, span + 1 - j + r));
      } else {
        const int c = id - nwe * nrc, el = c / ne;
        span_recip_entry(D.U, ewlo + el + p, p, c - el * ne, rcc[el], rdc[el]);
      }
    }
  }
  // step 1: S columns by p local Boehm insertions (Eq. 10) on B_i's own knots,
  // in the second warp, concurrently with the first warp's point assembly
  const int sc_col = (int)threadIdx.x - 32;
  if (sc_col >= 0 && sc_col < p) {
    int i = s + sc_col;
    double tau[2 * TW_MAXP + 2], c[TW_MAXP1], cn[TW_MAXP1];
    int L = p + 2;
    for (int k = 0; k < L; k++) tau[k] = D.U[i + k];
    c[0] = 1.0;
    int nc = 1;
    for (int r = 0; r < p; r++) {
      int sp = 0;
      for (int k = 0; k < L - 1; k++)
        if (tau[k] <= t) sp = k;
      for (int k = 0; k <= nc; k++) {
        double al;
        if (k <= sp - p) al = 1.0;
        else if (k >= sp + 1) al = 0.0;
        else al = (t - tau[k]) / (tau[k + p] - tau[k]);
        double ck = k < nc ? c[k] : 0.0, ckm = k > 0 ? c[k - 1] : 0.0;
        cn[k] = al * ck + (1.0 - al) * ckm;
      }
      nc++;
      for (int k = 0; k < nc; k++) c[k] = cn[k];
      for (int k = L; k > sp + 1; k--) tau[k] = tau[k - 1];
      tau[sp + 1] = t;
      L++;
    }
    for (int r = 0; r <= p; r++) Sc[sc_col][r] = c[r];
  }
  __syncthreads();
  const int np_ = npts;
  // refined basis at the window points and at the window elements' Gauss points
  for (int id = threadIdx.x; id < np_ + nwe * p1; id += blockDim.x) {
    double N[TW_MAXP1];
    if (id < np_) {
      int e = elem_of(D.bp, D.nel, xs[id]);
      // (a window point lies inside a window element; the clamp only keeps
      // the table read in bounds)
      ref_basis_rc(D, s, e, xs[id], rcw[min(max(e - ewlo, 0), nwe - 1)], N);
      rsp[id] = e + (e >= s ? p : 0);
      for (int a2 = 0; a2 <= p; a2++) RB[id][a2] = N[a2];
    } else {
      int j = id - np_, el = j / p1, g = j % p1, e = ewlo + el;
      double x = D.bp[e] + (D.bp[e + 1] - D.bp[e]) * 0.5 * (D.gx[g] + 1.0);
      GWt[el][g] = D.gw[g] * 0.5 * (D.bp[e + 1] - D.bp[e]);
      if (D.bp[e + 1] > D.bp[e]) ref_basis_rc(D, s, e, x, rcw[el], N);
      else  // the zero-length span of a repeated knot
        for (int a2 = 0; a2 <= p; a2++) N[a2] = 0.0;
      for (int a2 = 0; a2 <= p; a2++) RG[el][g][a2] = N[a2];
    }
  }
  __syncthreads();
  // step 3: WQ weights of the refined functions l = s .. s+2p-1 (Eq. 5): a
  // group of TW_DWQ_G lanes per refined system (group_minnorm), eight systems
  // per warp, so the first ceil(2p / 8) warps solve them all; the systems'
  // matrices sit in dynamic shared memory (TW_DWQ_SMEM bytes)
  constexpr int G = TW_DWQ_G, CPL = (TW_QMAX + TW_DWQ_G - 1) / TW_DWQ_G;
  extern __shared__ double dwq_dyn[];
  double (*sA)[TW_WIN * (TW_QMAX + 1)] = (double (*)[TW_WIN * (TW_QMAX + 1)])dwq_dyn;
  __shared__ double sb[2 * TW_MAXP][TW_WIN], sd[2 * TW_MAXP][TW_WIN], sbeta[2 * TW_MAXP][TW_WIN];
  __shared__ int sing[2 * TW_MAXP];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31, gl = lane & (G - 1);
  const int lda = TW_QMAX + 1;
  if (wib * (32 / G) < 2 * p && np_ > 0) {  // warp-uniform
    const int li = wib * (32 / G) + lane / G;
    const bool live = li < 2 * p;
    int l = s + li;
    int nref = D.n + p;
    int rows[TW_WIN], m = 0, c0 = 0, N = 0;
    double ul = 0.0, uh = 0.0;
    if (live) {
      ul = ref_knot(D, s, l);
      uh = ref_knot(D, s, l + p + 1);
      for (int mm = max(0, l - p); mm <= min(nref - 1, l + p); mm++) {
        double lo = fmax(ul, ref_knot(D, s, mm)), hi = fmin(uh, ref_knot(D, s, mm + p + 1));
        if (hi > lo) rows[m++] = mm;
      }
      // points of supp B~_l: a contiguous run of the sorted window points
      while (c0 < np_ && !(xs[c0] > ul)) c0++;
      while (c0 + N < np_ && xs[c0 + N] < uh) N++;
      if (N > TW_QMAX) {
        if (gl == 0) atomicOr(flag, TWF_QMAX);
        N = 0;
      }
    }
    double *A = sA[live ? li : 0];
    for (int c = gl; c < N; c += G) {
      int k = c0 + c;
      for (int r = 0; r < m; r++) {
        int aa = rows[r] - rsp[k];
        A[r * lda + c] = (aa >= 0 && aa <= p) ? RB[k][aa] : 0.0;
      }
    }
    for (int r = gl; r < m && N > 0; r += G) {
      int mr = rows[r];
      double acc = 0.0;
      for (int el = 0; el < nwe; el++) {
        int e = ewlo + el;
        double ea = D.bp[e], eb = D.bp[e + 1];
        if (eb <= ul || ea >= uh || !(eb > ea)) continue;
        int f0 = e + (e >= s ? p : 0);
        int al = l - f0, am = mr - f0;
        if (al < 0 || al > p || am < 0 || am > p) continue;
        for (int g = 0; g < p1; g++) acc += GWt[el][g] * RG[el][g][al] * RG[el][g][am];
      }
      sb[li][r] = acc;
    }
    if (live && gl == 0) sing[li] = 0;
    __syncwarp();
    double w[CPL];
    const int ms = N > 0 ? m : 0;
    group_minnorm<G, CPL>(ms, N, A, lda, live ? sb[li] : sb[0], live ? sd[li] : sd[0],
                          live ? sbeta[li] : sbeta[0], gl, live ? &sing[li] : &sing[0], w);
    __syncwarp();
    if (live) {
      if (gl == 0 && sing[li]) atomicOr(flag, TWF_SINGULAR);
      for (int k = gl; k < np_; k += G) Wt[li][k] = 0.0;
    }
    __syncwarp();
    if (live) {
#pragma unroll
      for (int u = 0; u < CPL; u++) {
        const int c = gl + G * u;
        if (c < N) Wt[li][c0 + c] = w[u];
      }
    }
    __syncwarp();
  }
  __syncthreads();
  // step 4: w_i = sum over refined l on the side of S[l][i] w~_l  (reading R4)
  for (int id = threadIdx.x; id < p * 2 * TW_LQMAX; id += blockDim.x) {
    int col = id / (2 * TW_LQMAX), side = (id / TW_LQMAX) % 2, k = id % TW_LQMAX;
    double acc = 0.0;
    if (k < np_) {
      int i = s + col;
      for (int r = 0; r <= p; r++) {
        int l = i + r;
        int lside = (l <= p + s - 1) ? 0 : 1;
        if (lside != side) continue;
        acc += Sc[col][r] * Wt[l - s][k];
      }
    }
    out_w[(((size_t)slot * p + col) * 2 + side) * TW_LQMAX + k] = acc;
  }
  for (int k = threadIdx.x; k < TW_LQMAX; k += blockDim.x) {
    out_x[(size_t)slot * TW_LQMAX + k] = k < np_ ? xs[k] : 0.0;
    out_k[(size_t)slot * TW_LQMAX + k] = k < np_ ? xk[k] : -1;
    // coarse element, coarse basis values and derivatives of each window
    // point (the derivatives give the geometry map's Jacobian at nested points)
    int e = 0;
    double N[TW_MAXP1], dN[TW_MAXP1];
    if (k < np_) {
      e = elem_of(D.bp, D.nel, xs[k]);
      const int el = min(max(e - ewlo, 0), nwe - 1);
      basis_ders_rc(D.U, e + p, xs[k], p, rcc[el], rdc[el], N, dN);
    }
    out_e[(size_t)slot * TW_LQMAX + k] = e;
    for (int a2 = 0; a2 <= p; a2++) {
      out_B[((size_t)slot * TW_LQMAX + k) * p1 + a2] = k < np_ ? N[a2] : 0.0;
      out_dB[((size_t)slot * TW_LQMAX + k) * p1 + a2] = k < np_ ? dN[a2] : 0.0;
    }
  }
  // per coarse function i = s + col and side: the contiguous run of window
  // points inside supp B_i on that side of t
  for (int id = threadIdx.x; id < 2 * p; id += blockDim.x) {
    int col = id >> 1, side = id & 1, i = s + col;
    double lo = side == 0 ? D.U[i] : t, hi = side == 0 ? t : D.U[i + p + 1];
    int k0 = 0;
    while (k0 < np_ && !(xs[k0] > lo)) k0++;
    int k1 = k0;
    while (k1 < np_ && xs[k1] < hi) k1++;
    out_r[((size_t)slot * p + col) * 2 + side] = k0 | (k1 << 16);
  }
  if (threadIdx.x == 0) out_np[slot] = np_;
}

// Element matrices of the cut elements, M_e[a][b] = sum_q w_q c_q B_a B_b over the
// element's rule (Sect. 3.1), sum-factorised along the rule's Gauss lines: on a
// line xi_o = s the outer basis values are constant, so the inner sums
// I(ai,bi) = sum_h w_h c_h B_ai(u_h) B_bi(u_h) are formed first and then
// M[(ao,ai)][(bo,bi)] += B_ao(s) B_bo(s) I(ai,bi).  Both factors are symmetric
// in their index pair, so only the unordered pairs {ao,bo} x {ai,bi} are
// accumulated ((p+1)(p+2)/2 squared instead of (p+1)^4 products per line) and
// M, symmetric, is written out from them.  One warp per element, no block
// barrier: lane u < (p+1)(p+2)/2 forms the line's inner sum and outer product
// of pair u, then every lane adds them into its share of the accumulators.
// The lines and their points come from the rule's layout (line_off per
// element, lpos per line); sums run in point and line order (deterministic).
#define TW_CM_WARPS 4
template <int P>
__device__ __forceinline__ int sym_pair(int a, int b) {  // a <= b
  return a * (P + 1) - a * (a - 1) / 2 + (b - a);
}
template <int P>
__global__ void __launch_bounds__(32 * TW_CM_WARPS)
    k_cut_matrices(const int64_t *line_off, const int64_t *lpos, const int32_t *cut_o, int ncut,
                   const double *Bt, const double *wc, double *M) {
  constexpr int P1 = P + 1, NL = P1 * P1, U = P1 * (P1 + 1) / 2, NO = U * U;
  constexpr int NPL = (NO + 31) / 32;
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ci = blockIdx.x * TW_CM_WARPS + wib;
  if (ci >= ncut) return;  // the whole warp
  __shared__ double Fs[TW_CM_WARPS][U], Is[TW_CM_WARPS][U], As[TW_CM_WARPS][NO];
  double *F = Fs[wib], *I = Is[wib], *Acc = As[wib];
  const int o = cut_o[ci], in = 1 - o;
  // this lane's pair (lanes below U): u -> (pa, pb), pa <= pb
  int pa = 0, pb = 0;
  if (lane < U) {
    int r = lane;
    while (r >= P1 - pa) {
      r -= P1 - pa;
      pa++;
    }
    pb = pa + r;
  }
  double acc[NPL];
#pragma unroll
  for (int j = 0; j < NPL; j++) acc[j] = 0.0;
  // the element's Gauss lines (R6) and their points, from the rule's layout
  const int64_t L0 = line_off[ci], L1 = line_off[ci + 1];
  for (int64_t L = L0; L < L1; L++) {
    const int64_t k = lpos[L], ke = lpos[L + 1];
    if (ke == k) continue;  // a line with no visible interval (uniform)
    if (lane < U) {
      double sum = 0.0;
#pragma unroll 4
      for (int64_t h = k; h < ke; h++) {
        const double *bv = Bt + (2 * h + in) * P1;
        sum = fma(wc[h] * bv[pa], bv[pb], sum);
      }
      const double *bo_ = Bt + (2 * k + o) * P1;
      I[lane] = sum;
      F[lane] = bo_[pa] * bo_[pb];
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < NPL; j++) {
      const int m = lane + 32 * j;
      if (m < NO) acc[j] = fma(F[m / U], I[m % U], acc[j]);
    }
    __syncwarp();  // F, I rewritten by the next line
  }
#pragma unroll
  for (int j = 0; j < NPL; j++) {
    const int m = lane + 32 * j;
    if (m < NO) Acc[m] = acc[j];
  }
  __syncwarp();
  // M[(a2,a1)][(b2,b1)] from the pair accumulators, consecutive lanes on
  // consecutive entries
  double *Me = M + (size_t)ci * NL * NL;
  for (int t = lane; t < NL * NL; t += 32) {
    const int r = t / NL, c = t % NL;
    const int a1 = r % P1, a2 = r / P1, b1 = c % P1, b2 = c / P1;
    const int ao = o == 0 ? a1 : a2, ai = o == 0 ? a2 : a1;
    const int bo = o == 0 ? b1 : b2, bi = o == 0 ? b2 : b1;
    const int po = sym_pair<P>(min(ao, bo), max(ao, bo));
    const int pi = sym_pair<P>(min(ai, bi), max(ai, bi));
    Me[t] = Acc[po * U + pi];
  }
}

static void launch_cut_matrices(tw_patch *P, const int64_t *line_off, const int64_t *lpos,
                                cudaStream_t st) {
  const unsigned nb = (unsigned)((P->ncut + TW_CM_WARPS - 1) / TW_CM_WARPS);
  switch (P->p) {
#define TW_CM(PP) case PP: k_cut_matrices<PP><<<nb, 32 * TW_CM_WARPS, 0, st>>>(line_off, lpos, P->cut_o, P->ncut, P->cut_B, P->cut_wc, P->cut_M); break;
    TW_CM(1) TW_CM(2) TW_CM(3) TW_CM(4) TW_CM(5) TW_CM(6)
#undef TW_CM
  }
  TW_LAUNCH();
}

// Element matrices of the regular elements some row integrates by Gauss
// (Sect. 3.2), sum-factorised at element level:
//   T[a1][b1][g2] = sum_g1 w1 B_a1 B_b1 c(g1, g2),
//   M[(a1,a2)][(b1,b2)] = sum_g2 T[a1][b1][g2] w2 B_a2 B_b2.
template <int P>
__global__ void __launch_bounds__(256) k_gauss_matrices(Dir A, Dir B, const int32_t *glist, int ng,
                                                       const double *gc, const uint8_t *fstate,
                                                       int method, double *M) {
  constexpr int P1 = P + 1, NL = P1 * P1, P3 = P1 * P1 * P1;
  const int sl = blockIdx.x;
  if (sl >= ng) return;
  const int e = glist[sl], e1 = e % A.nel, e2 = e / A.nel;
  __shared__ double T[P3];
  // weighted products of the element's basis at its Gauss points,
  // W[g][a][b] = w_g h B_a(x_g) B_b(x_g), per direction
  __shared__ double W1[P3], W2[P3];
  // only the rows of test functions formed by the cut-row kernel are ever
  // read (cut functions; every active function for the Gauss method)
  __shared__ int flag[NL], need[NL];
  __shared__ int nneed;
  const double *c = gc + (size_t)sl * NL;  // [g2][g1]
  const double *GW1 = A.GW + (size_t)e1 * P3, *GW2 = B.GW + (size_t)e2 * P3;
  for (int id = threadIdx.x; id < P3; id += blockDim.x) {
    W1[id] = GW1[id];
    W2[id] = GW2[id];
  }
  for (int a = threadIdx.x; a < NL; a += blockDim.x) {
    const uint8_t st = fstate[(size_t)(e2 + a / P1) * A.n + (e1 + a % P1)];
    flag[a] = st != TW_FUNC_EXTERIOR && (method == TW_METHOD_GAUSS || st == TW_FUNC_CUT);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0;
    for (int a = 0; a < NL; a++)
      if (flag[a]) need[n++] = a;
    nneed = n;
  }
  for (int id = threadIdx.x; id < P3; id += blockDim.x) {
    const int a1 = id / NL, b1 = (id / P1) % P1, g2 = id % P1;
    double s = 0.0;
#pragma unroll
    for (int g1 = 0; g1 < P1; g1++) s = fma(W1[(g1 * P1 + a1) * P1 + b1], c[g2 * P1 + g1], s);
    T[id] = s;
  }
  __syncthreads();
  double *Me = M + (size_t)sl * NL * NL;
  for (int id = threadIdx.x; id < nneed * NL; id += blockDim.x) {
    const int a = need[id / NL], b = id % NL;
    const int a1 = a % P1, a2 = a / P1, b1 = b % P1, b2 = b / P1;
    double s = 0.0;
#pragma unroll
    for (int g2 = 0; g2 < P1; g2++)
      s = fma(T[(a1 * P1 + b1) * P1 + g2], W2[(g2 * P1 + a2) * P1 + b2], s);
    Me[a * NL + b] = s;
  }
}

static void launch_gauss_matrices_impl(tw_patch *P, const int32_t *glist, cudaStream_t st);
static void launch_gauss_matrices(tw_patch *P, const int32_t *glist, cudaStream_t st) {
  int ps = prof_start(st);
  launch_gauss_matrices_impl(P, glist, st);
  prof_stop(ps, TW_STAGE_GAUSSMAT, st);
}
static void launch_gauss_matrices_impl(tw_patch *P, const int32_t *glist, cudaStream_t st) {
  switch (P->p) {
#define TW_GM(PP) case PP: k_gauss_matrices<PP><<<P->ngslot, 256, 0, st>>>(P->d[0], P->d[1], glist, P->ngslot, P->gc, P->fstate, P->method, P->gmat); break;
    TW_GM(1) TW_GM(2) TW_GM(3) TW_GM(4) TW_GM(5) TW_GM(6)
#undef TW_GM
  }
  TW_LAUNCH();
}

// ---------------------------------------------------------------------------
// host orchestration

#define TW_GAUSS_DEVICES 64
static std::mutex g_gauss_mu;
static double *g_gauss[TW_GAUSS_DEVICES][65];

int gauss_rule(int q, cudaStream_t s, const double **out) {
  int dev = 0;
  if (check_cuda(cudaGetDevice(&dev), "gauss_rule")) return TW_ECUDA;
  if (q < 1 || q > 64 || dev < 0 || dev >= TW_GAUSS_DEVICES) {
    set_error("gauss_rule: order %d or device %d out of range", q, dev);
    return TW_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_gauss_mu);
  if (!g_gauss[dev][q]) {
    double *d = nullptr;
    if (check_cuda(cudaMalloc(&d, sizeof(double) * 2 * q), "gauss_rule: cudaMalloc")) return TW_ENOMEM;
    k_gauss_nodes<<<1, 64, 0, s>>>(q, d, d + q);
    TW_LAUNCH();
    // other streams read the rule later: complete it now
    if (check_cuda(cudaStreamSynchronize(s), "gauss_rule")) return TW_ECUDA;
    g_gauss[dev][q] = d;
  }
  *out = g_gauss[dev][q];
  return 0;
}

static int read_flag(tw_patch *P, const char *stage) {
  int f = 0;
  if (check_cuda(cudaMemcpyAsync(&f, P->flag, sizeof(int), cudaMemcpyDeviceToHost, P->stream),
                 stage))
    return TW_ECUDA;
  if (check_cuda(cudaStreamSynchronize(P->stream), stage)) return TW_ECUDA;
  if (f) {
    set_error("%s: device check failed (flags 0x%x: %s%s%s%s%s%s)", stage, f,
              (f & TWF_BRCAP) ? "too many breakpoints in a cut element; " : "",
              (f & TWF_HITCAP) ? "too many curve crossings in a cut element; " : "",
              (f & TWF_SINGULAR) ? "singular WQ system; " : "",
              (f & TWF_QMAX) ? "too many points in one support; " : "",
              (f & TWF_LQMAX) ? "too many refined points around a disc; " : "",
              (f & TWF_RULECAP) ? "region rule too long; " : "");
    return (f & TWF_SINGULAR) ? TW_ECUDA : TW_EUNSUPPORTED;
  }
  return 0;
}

#define G1(n) (unsigned)(((n) + 255) / 256), 256, 0, st
// one warp per block, for the short thread-per-item kernels whose items each
// run a long FP64 chain (basis evaluations, root finding): a 256-thread block
// would put eight such warps on one SM's FP64 pipe while other SMs idle
#define G32(n) (unsigned)(((n) + 31) / 32), 32, 0, st

int build_tables(tw_patch *P) {
  cudaStream_t st = P->stream;
  Dir &A = P->d[0];
  Dir &B = P->d[1];
  int p = P->p, p1 = p + 1;
  int rc;
  // counters[16] | tot32[8] (read back together after the classification) and
  // tot64[4]: zeroed by the patch's packed upload
  int32_t *counters = P->cnt32;
  int64_t *tot64 = P->cnt64;
  int32_t *tot32 = counters + 16;

  // Gauss rules (p+1 for elements, qc for cut pieces), cached per process
  const double *er = nullptr, *qr = nullptr;
  if ((rc = gauss_rule(p1, st, &er)) || (rc = gauss_rule(P->qc, st, &qr))) return rc;
  for (int d = 0; d < 2; d++) {
    P->d[d].gx = er;
    P->d[d].gw = er + p1;
  }
  P->qrule = qr;
  const double *qgx = qr, *qgw = qr + P->qc;

  // WQ layout, basis tables, weights (Eq. 5): both directions per launch
  {
    const int b0 = (std::max(A.nel, B.nel) * p1 + 31) / 32, b1 = (std::max(A.n, B.n) + 31) / 32;
    const int b2 = (std::max(A.nel, B.nel) * p1 + 31) / 32;
    SegJobs S;  // with the spline curves' segments
    S.n = 0;
    S.blk[0] = 0;
    for (int ci = 0; ci < P->curves.n; ci++) {
      const Curve &Cv = P->curves.c[ci];
      if (Cv.kind != TW_TRIM_BSPLINE3) continue;
      S.ctrl[S.n] = P->curve_ctrl[ci];
      S.nc[S.n] = Cv.nc;
      S.seg[S.n] = (double *)Cv.seg;
      S.box[S.n] = (double *)Cv.box;
      S.blk[S.n + 1] = S.blk[S.n] + (Cv.nc + 31) / 32;
      S.n++;
    }
    k_dir_tables<<<dim3(b0 + b1 + b2 + S.blk[S.n], 2), 32, 0, st>>>(A, B, b0, b1, b2, S);
    TW_LAUNCH();
    const int nw = std::max(A.n, B.n);
    const int lda = std::max(A.qmax, B.qmax) + 1;
    const size_t wsm = sizeof(double) * TW_WQ_SYS * TW_WIN * lda;
    const int pw = prof_start(st);
    k_wq_weights<<<dim3((nw + TW_WQ_SYS - 1) / TW_WQ_SYS, 2), 32 * TW_WQ_WARPS, wsm, st>>>(
        A, B, lda, P->flag);
    prof_stop(pw, TW_STAGE_WQW, st);
    TW_LAUNCH();
  }
  if ((rc = check_cuda(cudaGetLastError(), "wq tables"))) return rc;

  // classification (Sect. 2.2)
  int64_t ne = (int64_t)A.nel * B.nel, nf = (int64_t)A.n * B.n;
  int32_t *aflag = (int32_t *)dalloc(P, sizeof(int32_t) * nf);
  int32_t *cflag = (int32_t *)dalloc(P, sizeof(int32_t) * nf);
  int32_t *cpos = (int32_t *)dalloc(P, sizeof(int32_t) * nf);
  int32_t *eflag = (int32_t *)dalloc(P, sizeof(int32_t) * ne);
  int32_t *epos = (int32_t *)dalloc(P, sizeof(int32_t) * ne);
  int32_t *gflag = (int32_t *)dalloc(P, sizeof(int32_t) * ne);
  int32_t *gpos = (int32_t *)dalloc(P, sizeof(int32_t) * ne);
  if (!aflag || !cflag || !cpos || !eflag || !epos || !gflag || !gpos) return TW_ENOMEM;
  int32_t *dflag[2], *dpos[2];  // disc knots of the DWQ regions (R7), per direction
  for (int d = 0; d < 2; d++) {
    dflag[d] = (int32_t *)dalloc(P, sizeof(int32_t) * (P->d[d].nel + 1));
    dpos[d] = (int32_t *)dalloc(P, sizeof(int32_t) * (P->d[d].nel + 1));
    if (!dflag[d] || !dpos[d]) return TW_ENOMEM;
  }
  int fcap = 4;
  for (int ci = 0; ci < P->curves.n; ci++) fcap += 2 * P->curves.c[ci].nc + 4;
  double *lh, *feat;
  int *lnh, *nfeat;
  {
    int nl = (A.nel + 1) + (B.nel + 1) + B.nel;
    lh = (double *)dalloc(P, sizeof(double) * (size_t)nl * TW_HITCAP);
    lnh = (int *)dalloc(P, sizeof(int) * nl);
    feat = (double *)dalloc(P, sizeof(double) * 3 * 2 * (size_t)fcap);
    nfeat = (int *)dalloc(P, sizeof(int) * 4);
    if (!lh || !lnh || !feat || !nfeat) return TW_ENOMEM;
    if (P->curves.n > 0) {
      const int nbl = (nl + 31) / 32;
      k_curve_lines<<<nbl + 3, 32, 0, st>>>(P->curves, A, B, lh, lnh, nbl, feat, nfeat, fcap,
                                            P->flag);
      TW_LAUNCH();
    }
    k_classify_elems<<<G1(ne)>>>(P->curves, A, B, lh, lnh, P->method, P->estate, eflag, gflag);
    TW_LAUNCH();
  }
  k_classify_funcs<<<G1(nf)>>>(A, B, P->estate, P->fstate, aflag, P->method, cflag, counters,
                               dflag[0], dflag[1], P->choice, gflag);
  TW_LAUNCH();
  if ((rc = scan2_impl<int32_t>(aflag, P->act, nf, tot32 + 0, cflag, cpos, nf, tot32 + 1, st, P)))
    return rc;
  // cut elements and the regular elements integrated by Gauss (flagged above)
  if ((rc = scan2_impl<int32_t>(eflag, epos, ne, tot32 + 2, gflag, gpos, ne, tot32 + 3, st, P)))
    return rc;
  // DWQ choice (R7) and disc flags
  if (P->method == TW_METHOD_DWQ) {
    // the cut functions (cflag marks exactly those for DWQ) as a list, its
    // length read by the choice kernel from the scan's total
    int32_t *cfl = (int32_t *)dalloc(P, sizeof(int32_t) * nf);
    if (!cfl) return TW_ENOMEM;
    const CompactJob cj = {cflag, cpos, cfl, nullptr, nf};
    launch_compact(&cj, 1, st);
    const int nb = (int)std::min<int64_t>((nf + TW_CHOICE_WARPS - 1) / TW_CHOICE_WARPS, 152 * 8);
    k_dwq_choice<<<nb, 32 * TW_CHOICE_WARPS, 0, st>>>(A, B, P->estate, cfl, tot32 + 1, P->choice,
                                                       dflag[0], dflag[1], counters + 2);
    TW_LAUNCH();
  }
  if ((rc = scan2_impl<int32_t>(dflag[0], dpos[0], A.nel + 1, tot32 + 4, dflag[1], dpos[1],
                                B.nel + 1, tot32 + 5, st, P)))
    return rc;
  int32_t h24[24];
  cudaMemcpyAsync(h24, counters, sizeof(h24), cudaMemcpyDeviceToHost, st);
  const int32_t *hcount = h24, *hc = h24 + 16;
  if ((rc = read_flag(P, "classification"))) return rc;
  P->n_rows = hc[0];
  P->ncutrows = hc[1];
  P->ncut = hc[2];
  P->ngslot = hc[3];
  P->ndisc[0] = hc[4];
  P->ndisc[1] = hc[5];
  P->ncutfns = hcount[0];
  P->n_interior = hcount[1];
  P->ndwqrows = hcount[2];

  // active numbering and CSR pattern (R11)
  P->rowg = (int32_t *)dalloc(P, sizeof(int32_t) * (P->n_rows + 1));
  P->row_ptr = (int64_t *)dalloc(P, sizeof(int64_t) * (P->n_rows + 1));
  int64_t *cnt = (int64_t *)dalloc(P, sizeof(int64_t) * (P->n_rows + 1));
  P->cutrows = (int32_t *)dalloc(P, sizeof(int32_t) * (P->ncutrows + 1));
  P->cut_list = (int32_t *)dalloc(P, sizeof(int32_t) * (P->ncut + 1));
  P->cut_off = (int64_t *)dalloc(P, sizeof(int64_t) * (P->ncut + 1));
  int32_t *glist = (int32_t *)dalloc(P, sizeof(int32_t) * (P->ngslot + 1));
  P->gc = (double *)dalloc(P, sizeof(double) * ((size_t)P->ngslot * p1 * p1 + 1));
  if (!P->rowg || !P->row_ptr || !cnt || !P->cutrows || !P->cut_list || !P->cut_off ||
      !glist || !P->gc)
    return TW_ENOMEM;
  {  // active numbering (act, -1 off the active set) and its inverse rowg; the
     // cut-row, cut-element and Gauss-element lists with their slot maps
    const CompactJob cj[4] = {{aflag, P->act, P->rowg, P->act, nf},
                              {cflag, cpos, P->cutrows, nullptr, nf},
                              {eflag, epos, P->cut_list, P->cut_slot, ne},
                              {gflag, gpos, glist, P->gslot, ne}};
    launch_compact(cj, 4, st);
  }
  k_row_counts<<<G1(nf)>>>(A, B, P->act, cnt, P->n_rows);
  TW_LAUNCH();
  // n_rows + 1 entries, the last 0: row_ptr[n_rows] = nnz
  if ((rc = exclusive_scan_i64(cnt, P->row_ptr, P->n_rows + 1, tot64 + 0, st, P))) return rc;

  // c at the WQ grid (Eq. 6), sum-factorised for the spline geometry
  double *Gt = nullptr;
  if (P->geo.geom_kind == TW_GEOM_SPLINE && P->geo.coef_kind != TW_COEF_ONE) {
    Gt = (double *)dalloc(P, sizeof(double) * 4 * (size_t)B.nq * A.n);
    if (!Gt) return TW_ENOMEM;
  }
  {  // stage A of the grid (spline geometry) with the element Gauss c tables
    const int nbA = Gt ? (int)(((int64_t)B.nq * A.n + 255) / 256) : 0;
    const int nbG = (P->ngslot + TW_GC_WARPS - 1) / TW_GC_WARPS;
    if (nbA + nbG > 0) {
      k_geo_gauss_c<<<nbA + nbG, 32 * TW_GC_WARPS, 0, st>>>(P->geo, A, B, Gt, nbA, glist,
                                                           P->ngslot, P->gc);
      TW_LAUNCH();
    }
  }
  k_cgrid<<<G1((int64_t)A.nq * B.nq)>>>(P->geo, A, B, Gt, P->C);
  TW_LAUNCH();
  // element matrices (skipped above TW_GMAT_BUDGET bytes: the cut-row kernel
  // then integrates those elements row by row)
  if (P->ngslot > 0) {
    size_t nl = (size_t)p1 * p1;
    size_t bytes = (size_t)P->ngslot * nl * nl * sizeof(double);
    P->gmat = nullptr;
    if (bytes <= TW_GMAT_BUDGET) {
      P->gmat = (double *)dalloc(P, bytes);
      if (!P->gmat) return TW_ENOMEM;
      launch_gauss_matrices(P, glist, st);
    }
  }
  // cut-element rules: breakpoints per element, then one thread per Gauss line
  // (crossings and point count), a scan, and the points written per line
  P->cut_o = (int32_t *)dalloc(P, sizeof(int32_t) * (P->ncut + 1));
  if (!P->cut_o) return TW_ENOMEM;
  double *cbr = nullptr, *clh = nullptr;
  int64_t *line_off = nullptr, *lpos = nullptr;
  int32_t *cln = nullptr;
  uint64_t *clv = nullptr;
  int64_t nlines = 0;
  if (P->ncut > 0) {
    cbr = (double *)dalloc(P, sizeof(double) * (size_t)P->ncut * TW_BRCAP);
    int32_t *cnbr = (int32_t *)dalloc(P, sizeof(int32_t) * P->ncut);
    int64_t *cnl = (int64_t *)dalloc(P, sizeof(int64_t) * (P->ncut + 1));
    line_off = (int64_t *)dalloc(P, sizeof(int64_t) * (P->ncut + 1));
    if (!cbr || !cnbr || !cnl || !line_off) return TW_ENOMEM;
    k_cut_breaks<<<G32(P->ncut)>>>(A, B, P->cut_list, P->ncut, P->qc, lh, lnh, feat, nfeat, fcap,
                                  P->cut_o, cnbr, cbr, cnl, P->flag);
    TW_LAUNCH();
    if ((rc = exclusive_scan_i64(cnl, line_off, P->ncut + 1, tot64 + 2, st, P))) return rc;
    cudaMemcpyAsync(&nlines, tot64 + 2, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if ((rc = check_cuda(cudaStreamSynchronize(st), "cut rules"))) return rc;
    clh = (double *)dalloc(P, sizeof(double) * ((size_t)nlines * TW_HITCAP + 1));
    cln = (int32_t *)dalloc(P, sizeof(int32_t) * (nlines + 1));
    clv = (uint64_t *)dalloc(P, sizeof(uint64_t) * (nlines + 1));
    int64_t *clc = (int64_t *)dalloc(P, sizeof(int64_t) * (nlines + 1));
    lpos = (int64_t *)dalloc(P, sizeof(int64_t) * (nlines + 1));
    if (!clh || !cln || !clv || !clc || !lpos) return TW_ENOMEM;
    if (nlines == 0) cudaMemsetAsync(clc, 0, sizeof(int64_t), st);  // else closed by k_cut_lines
    if (nlines > 0) {
      // 64-thread blocks: a patch has only ~10^4 lines, and 256-thread
      // blocks would leave most SMs idle on this FP64-heavy kernel
      k_cut_lines<<<(unsigned)((nlines + 63) / 64), 64, 0, st>>>(
          P->curves, A, B, P->cut_list, P->ncut, P->qc, qgx, qgw, lh, lnh, P->cut_o, cbr, line_off,
          tot64 + 2, clh, cln, clv, clc, P->flag);
      TW_LAUNCH();
    }
    if ((rc = exclusive_scan_i64(clc, lpos, nlines + 1, tot64 + 1, st, P))) return rc;
    if (nlines == 0) {  // no Gauss lines (only after a breakpoint overflow): offsets here
      k_cut_offsets<<<G1(P->ncut + 1)>>>(P->ncut, line_off, lpos, tot64 + 1, P->cut_off);
      TW_LAUNCH();
    }
  }
  int64_t h64[2] = {0, 0};
  cudaMemcpyAsync(h64, tot64, sizeof(h64), cudaMemcpyDeviceToHost, st);
  if ((rc = read_flag(P, "cut rules"))) return rc;
  P->nnz = h64[0];
  P->ncutpts = P->ncut > 0 ? h64[1] : 0;
  P->cut_pts = (double *)dalloc(P, sizeof(double) * (3 * P->ncutpts + 1));
  P->cut_wc = (double *)dalloc(P, sizeof(double) * (P->ncutpts + 1));
  P->cut_B = (double *)dalloc(P, sizeof(double) * (2 * P->ncutpts * p1 + 1));
  P->cut_M = (double *)dalloc(P, sizeof(double) * ((size_t)P->ncut * p1 * p1 * p1 * p1 + 1));
  if (!P->cut_pts || !P->cut_wc || !P->cut_B || !P->cut_M) return TW_ENOMEM;
  if (P->ncut > 0) {
    if (nlines > 0) {
      k_cut_write<<<(unsigned)((nlines + 63) / 64), 64, 0, st>>>(
          A, B, P->cut_list, P->ncut, P->qc, qgx, qgw, P->cut_o, cbr, line_off, tot64 + 2, clh,
          cln, clv, lpos, tot64 + 1, P->cut_off, P->cut_pts);
      TW_LAUNCH();
    }
    k_cut_point_tables<<<(P->ncut + TW_CPT_WARPS - 1) / TW_CPT_WARPS, TW_CPT_THREADS, 0, st>>>(
        P->geo, A, B, P->cut_list, P->cut_off, P->cut_o, P->ncut, P->cut_pts, P->cut_B,
        P->cut_wc);
    TW_LAUNCH();
    launch_cut_matrices(P, line_off, lpos, st);
  }
  // DWQ rules per disc knot, both directions in one launch
  DwqOut dout[2];
  CompactJob dj[2];  // the disc knots of both directions as lists, one launch
  for (int d = 0; d < 2; d++) {
    Dir &D = P->d[d];
    int nd = P->ndisc[d];
    P->dwq_x[d] = (double *)dalloc(P, sizeof(double) * ((size_t)nd * TW_LQMAX + 1));
    P->dwq_np[d] = (int32_t *)dalloc(P, sizeof(int32_t) * (nd + 1));
    P->dwq_w[d] = (double *)dalloc(P, sizeof(double) * ((size_t)nd * p * 2 * TW_LQMAX + 1));
    P->dwq_k[d] = (int32_t *)dalloc(P, sizeof(int32_t) * ((size_t)nd * TW_LQMAX + 1));
    P->dwq_e[d] = (int32_t *)dalloc(P, sizeof(int32_t) * ((size_t)nd * TW_LQMAX + 1));
    P->dwq_B[d] = (double *)dalloc(P, sizeof(double) * ((size_t)nd * TW_LQMAX * p1 + 1));
    P->dwq_dB[d] = (double *)dalloc(P, sizeof(double) * ((size_t)nd * TW_LQMAX * p1 + 1));
    P->dwq_r[d] = (int32_t *)dalloc(P, sizeof(int32_t) * ((size_t)nd * p * 2 + 1));
    if (!P->dwq_k[d] || !P->dwq_e[d] || !P->dwq_B[d] || !P->dwq_dB[d] || !P->dwq_r[d])
      return TW_ENOMEM;
    int32_t *dlist = (int32_t *)dalloc(P, sizeof(int32_t) * (nd + 1));
    if (!P->dwq_x[d] || !P->dwq_np[d] || !P->dwq_w[d] || !dlist) return TW_ENOMEM;
    dj[d] = CompactJob{dflag[d], dpos[d], dlist, P->disc_slot[d], (int64_t)D.nel + 1};
    dout[d] = DwqOut{dlist,          nd,           P->dwq_x[d], P->dwq_w[d], P->dwq_B[d],
                     P->dwq_dB[d],   P->dwq_np[d], P->dwq_k[d], P->dwq_e[d], P->dwq_r[d]};
  }
  launch_compact(dj, 2, st);
  if (P->ndisc[0] + P->ndisc[1] > 0) {
    static std::once_flag dwq_attr[64];
    int dev = 0;
    cudaGetDevice(&dev);
    std::call_once(dwq_attr[dev & 63], [] {
      cudaFuncSetAttribute(k_dwq_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)TW_DWQ_SMEM);
    });
    const int pd = prof_start(st);
    k_dwq_build<<<P->ndisc[0] + P->ndisc[1], TW_DWQ_THREADS, TW_DWQ_SMEM, st>>>(
        A, B, dout[0], dout[1], P->flag);
    prof_stop(pd, TW_STAGE_DWQ, st);
    TW_LAUNCH();
  }
  if ((rc = check_cuda(cudaGetLastError(), "set-up kernels"))) return rc;
  return read_flag(P, "patch set-up");
}


}  // namespace tw
