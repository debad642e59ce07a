// tw_batch.cu -- forming many patches' mass matrices with one persistent launch.
//
// A batch owns, for a fixed list of patches and output CSR buffers:
//  * a device array of per-patch descriptors (the patch tables and outputs);
//  * a work list of items -- interior tiles (patch, i2, first i1) sized by a
//    tile chosen per (degree, precision) by the autotuner, cut rows (patch,
//    row) and row-pointer chunks -- ordered by estimated cost, largest first;
//  * a CUDA graph that resets the work counters and runs, for each degree
//    present, persistent launches of k_batch<PREC, P, ROLE> on their own
//    branches of the graph: every block takes the next item of its launch's
//    list with an atomicAdd on that launch's counter and runs its body, until
//    the list is exhausted (blocks never wait on one another).  The kernel is
//    compiled per degree and role so that its registers and shared memory are
//    those of its bodies (one kernel over all degrees spilled and carried the
//    largest tile's shared memory into every block); see ROLE_LIGHT.
// Items write disjoint parts of the outputs and every body sums in a fixed
// order, so the result equals the one-patch formation bit for bit.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "tw_bodies.cuh"

namespace tw {

int ensure_split_tables(tw_patch *P, cudaStream_t s);
Tables32 tables32(const tw_patch *P, bool split, const void *col, const void *val);

struct BatchPatch {
  RowArgs ra;
  Tables32 tb;  // FP32-pipe tables of the batch's precision
  const int32_t *cutrows;
  const int64_t *rp_in;
  int64_t nrp;
  int64_t *rp_out;
  int32_t *col;
  void *val;
  int p;
};

enum { IT_INTERIOR = 0, IT_CUTROW = 1, IT_ROWPTR = 2, IT_GATHER = 3 };
#define TW_GATHER_ROWS 8  // gather rows per item: one per warp of the block
#define TW_RP_CHUNK 4096

template <int PREC, int P>
__device__ __forceinline__ void run_interior(const BatchPatch &b, int i2, int i1a, int T,
                                             char *smem, uint64_t *bar, uint32_t *phase) {
  const RowArgs &a = b.ra;
  if constexpr (PREC == TW_PREC_FP64)
    interior_tile<P>(a.A, a.B, a.C, a.fstate, a.act, a.rp, b.col, (double *)b.val, i2, i1a, T,
                     smem, interior_kmax(P, T), a.A.mixed != 0);
  else
    interior_tile32<P, PREC == TW_PREC_FP32X2>(a.A, a.B, b.tb, a.fstate, a.act, a.rp, b.col,
                                               b.val, i2, i1a, T, smem, bar, phase, a.flag,
                                               a.A.mixed != 0);
}

template <int PREC, int P>
__device__ __forceinline__ void run_cutrow(const BatchPatch &b, int g, char *smem) {
  if constexpr (PREC == TW_PREC_FP32)
    cutrow_item<P, float>(b.ra, g, b.col, (float *)b.val, smem);
  else
    cutrow_item<P, double>(b.ra, g, b.col, (double *)b.val, smem);
}

template <int PREC, int P>
__device__ __forceinline__ void run_gather(const BatchPatch &b, int g, int lane,
                                           const double **tab) {
  if constexpr (PREC == TW_PREC_FP32)
    cutrow_gather_warp<P, float>(b.ra, g, lane, tab, b.col, (float *)b.val);
  else
    cutrow_gather_warp<P, double>(b.ra, g, lane, tab, b.col, (double *)b.val);
}

// Roles of a persistent launch.  Per degree the replayed graph runs a LIGHT
// launch and, where there are any, a HEAVY one, on separate branches.  LIGHT
// takes interior tiles (bound by the FP64 pipe) interleaved with the cut rows
// that only gather precomputed element matrices (bound by load latency), so
// that every SM works on both kinds at once, at the interior tile's ~48
// registers and as many resident blocks; run one after the other, the two
// phases took the sum of their times, and inside one launch with the
// block-per-row cut-row body (~96-128 registers) the gathers ran at a quarter
// of their occupancy.  HEAVY takes the block-per-row cut rows (DWQ regions,
// naive rows).
enum { ROLE_HEAVY = 0, ROLE_LIGHT = 2 };
__host__ __device__ constexpr int batch_min_blocks(int P, int ROLE) {
  return ROLE == ROLE_HEAVY ? (P <= 4 ? 3 : 2) : (P <= 5 ? 5 : 4);
}
#define TW_NQ (3 * TW_MAXP + 3)  // launches q = 3 p + role

// item = {kind | P << 4 | T << 8, patch, x, y}; a gather item is up to
// TW_GATHER_ROWS cut rows (x = first index into the patch's cut-row list,
// y = count), one per warp.  Every item of one launch has degree P and the
// launch's role.
template <int PREC, int P, int ROLE>
__global__ void __launch_bounds__(256, batch_min_blocks(P, ROLE))
    k_batch(const BatchPatch *__restrict__ bp, const int4 *__restrict__ items, int nitems,
            int *counter) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int cur;
  __shared__ uint64_t bar;  // bulk copies of the FP32-pipe tiles
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  uint32_t phase = 0;
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
    __syncthreads();
    const int it = cur;
    __syncthreads();
    if (it >= nitems) break;
    const int4 w = items[it];
    const int kind = w.x & 15, T = w.x >> 8;
    const BatchPatch &b = bp[w.y];
    if constexpr (ROLE == ROLE_HEAVY) {
      run_cutrow<PREC, P>(b, w.z, smem);
    } else if constexpr (ROLE == ROLE_LIGHT) {
      if (kind == IT_INTERIOR) {
        run_interior<PREC, P>(b, w.z, w.w, T, smem, &bar, &phase);
      } else if (kind == IT_GATHER) {
        const int wib = threadIdx.x >> 5;
        if (wib < w.w)
          run_gather<PREC, P>(b, b.cutrows[w.z + wib], threadIdx.x & 31,
                              (const double **)smem + wib * (TW_MAXP1 * TW_MAXP1));
      } else {
        const int64_t lo = (int64_t)w.z * TW_RP_CHUNK;
        const int64_t hi = min(b.nrp, lo + TW_RP_CHUNK);
        for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) b.rp_out[k] = b.rp_in[k];
      }
    }
    __syncthreads();
  }
}

// candidate interior tiles per degree: up to 64 rows at p <= 4, 32 above, so
// the tile's staged outputs keep the block's shared memory near 56 KB
static const int g_tiles[3] = {16, 32, 64};
static int tile_max(int p) { return p <= 4 ? 64 : 32; }

// dynamic shared memory of a launch: the cut-row body's, or the interior
// tile's for tile height t
template <int P>
static size_t batch_smem(int prec, int role, int t) {
  const size_t g = sizeof(double *) * TW_GATHER_ROWS * TW_MAXP1 * TW_MAXP1;
  const size_t i = prec == TW_PREC_FP64 ? interior_smem(P, t)
                                        : interior32_smem(P, t, prec == TW_PREC_FP32X2);
  const size_t s = role == ROLE_HEAVY ? sizeof(CutSmem<P>) : std::max(g, i);
  return (s + 15) / 16 * 16;
}

static std::mutex g_tune_mu;
static int g_tuned[64][3][TW_MAXP + 1];  // [device][precision][p] -> tile (0: not tuned)

}  // namespace tw

using namespace tw;

struct tw_batch {
  int n, precision, nitems;
  // per launch q = 2 p + role: grid, dynamic shared memory, slice of the item
  // list, work counter, graph branch
  int grid[TW_NQ];
  size_t smem[TW_NQ];
  int ioff[TW_NQ], icnt[TW_NQ];
  BatchPatch *dpatch;
  int4 *ditems;
  int *counter;
  cudaStream_t cap;
  cudaStream_t br[TW_NQ];
  cudaEvent_t fork, join[TW_NQ];
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  int tile[TW_MAXP + 1];
  double tune_ms[TW_MAXP + 1][3];
};

static void batch_free(tw_batch *B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  if (B->cap) cudaStreamDestroy(B->cap);
  for (int q = 0; q < TW_NQ; q++) {
    if (B->br[q]) cudaStreamDestroy(B->br[q]);
    if (B->join[q]) cudaEventDestroy(B->join[q]);
  }
  if (B->fork) cudaEventDestroy(B->fork);
  cudaFree(B->dpatch);
  cudaFree(B->ditems);
  cudaFree(B->counter);
  free(B);
}

template <int PREC, int P, int ROLE>
static void launch_q_t(tw_batch *B, const int4 *items, int nitems, int *counter, cudaStream_t s) {
  const int q = 3 * P + ROLE;
  k_batch<PREC, P, ROLE><<<B->grid[q], 256, B->smem[q], s>>>(B->dpatch, items, nitems, counter);
  TW_LAUNCH();
}

// sizes launch q for tile t: dynamic shared memory and grid (SMs x resident blocks)
template <int PREC, int P, int ROLE>
static cudaError_t size_q_t(tw_batch *B, int nsm, int t) {
  const int q = 3 * P + ROLE;
  B->smem[q] = batch_smem<P>(PREC, ROLE, t);
  cudaError_t e = cudaFuncSetAttribute(k_batch<PREC, P, ROLE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)B->smem[q]);
  int occ = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<PREC, P, ROLE>, 256,
                                                      B->smem[q]);
  if (e == cudaSuccess && occ <= 0) e = cudaErrorInvalidConfiguration;
  B->grid[q] = nsm * occ;
  return e;
}

// dispatch on (precision, degree, role) at run time; op 0 launches, op 1 sizes
template <int PREC, int P>
static cudaError_t q_op_r(tw_batch *B, int role, int op, const int4 *items, int nitems,
                          int *counter, cudaStream_t s, int nsm, int t) {
  if (role == ROLE_HEAVY) {
    if (op == 0) { launch_q_t<PREC, P, ROLE_HEAVY>(B, items, nitems, counter, s); return cudaSuccess; }
    return size_q_t<PREC, P, ROLE_HEAVY>(B, nsm, t);
  }
  if (op == 0) { launch_q_t<PREC, P, ROLE_LIGHT>(B, items, nitems, counter, s); return cudaSuccess; }
  return size_q_t<PREC, P, ROLE_LIGHT>(B, nsm, t);
}

template <int PREC>
static cudaError_t q_op_p(tw_batch *B, int q, int op, const int4 *items, int nitems, int *counter,
                          cudaStream_t s, int nsm, int t) {
  const int p = q / 3, role = q % 3;
  switch (p) {
    case 1: return q_op_r<PREC, 1>(B, role, op, items, nitems, counter, s, nsm, t);
    case 2: return q_op_r<PREC, 2>(B, role, op, items, nitems, counter, s, nsm, t);
    case 3: return q_op_r<PREC, 3>(B, role, op, items, nitems, counter, s, nsm, t);
    case 4: return q_op_r<PREC, 4>(B, role, op, items, nitems, counter, s, nsm, t);
    case 5: return q_op_r<PREC, 5>(B, role, op, items, nitems, counter, s, nsm, t);
    case 6: return q_op_r<PREC, 6>(B, role, op, items, nitems, counter, s, nsm, t);
  }
  return cudaErrorInvalidValue;
}

static cudaError_t q_op(tw_batch *B, int q, int op, const int4 *items, int nitems, int *counter,
                        cudaStream_t s, int nsm, int t) {
  if (B->precision == TW_PREC_FP64)
    return q_op_p<TW_PREC_FP64>(B, q, op, items, nitems, counter, s, nsm, t);
  if (B->precision == TW_PREC_FP32)
    return q_op_p<TW_PREC_FP32>(B, q, op, items, nitems, counter, s, nsm, t);
  return q_op_p<TW_PREC_FP32X2>(B, q, op, items, nitems, counter, s, nsm, t);
}

// the persistent launch q over items[0..nitems) (counter reset by the caller)
static void launch_q(tw_batch *B, int q, const int4 *items, int nitems, int *counter,
                     cudaStream_t s) {
  q_op(B, q, 0, items, nitems, counter, s, 0, 0);
}

static cudaError_t size_q(tw_batch *B, int q, int nsm, int t) {
  return q_op(B, q, 1, nullptr, 0, nullptr, nullptr, nsm, t);
}

static int item_code(int kind, int p, int T) { return kind | (p << 4) | (T << 8); }

// interior tiles of every patch of degree p with tile T
static void interior_items(const std::vector<tw_patch *> &pt, int p, int T, std::vector<int4> &out) {
  for (int k = 0; k < (int)pt.size(); k++) {
    tw_patch *P = pt[k];
    if (P->p != p || P->method == TW_METHOD_GAUSS || P->n_interior == 0) continue;
    for (int i2 = 0; i2 < P->d[1].n; i2++)
      for (int i1a = 0; i1a < P->d[0].n; i1a += T)
        out.push_back(make_int4(item_code(IT_INTERIOR, p, T), k, i2, i1a));
  }
}

extern "C" int tw_batch_create(tw_patch *const *patches, int n, int precision,
                               int64_t *const *row_ptr, int32_t *const *col, void *const *val,
                               void *stream, tw_batch **out) {
  if (!patches || n <= 0 || !row_ptr || !col || !val || !out) {
    set_error("tw_batch_create: NULL argument or empty batch");
    return TW_EINVAL;
  }
  if (precision < TW_PREC_FP64 || precision > TW_PREC_FP32X2) {
    set_error("tw_batch_create: unknown precision %d", precision);
    return TW_EINVAL;
  }
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<tw_patch *> pt(patches, patches + n);
  std::vector<BatchPatch> hp(n);
  for (int k = 0; k < n; k++) {
    tw_patch *P = pt[k];
    if (!P || !row_ptr[k] || (P->nnz > 0 && (!col[k] || !val[k]))) {
      set_error("tw_batch_create: patch %d or its outputs are NULL", k);
      return TW_EINVAL;
    }
    // the persistent kernel carves tiles of 16, 32 or 64 rows with the static
    // bound on their WQ points (simple knots always fit; a mixed-continuity
    // patch with many points next to repeated knots may not)
    for (int lt = 4; lt <= 6; lt++)
      if (P->ktile[lt] > interior_kmax(P->p, 1 << lt)) {
        set_error("tw_batch_create: patch %d has %d WQ points under a tile of %d rows, beyond "
                  "the batch's %d (form it with tw_form_mass)",
                  k, P->ktile[lt], 1 << lt, interior_kmax(P->p, 1 << lt));
        return TW_EUNSUPPORTED;
      }
    if (precision != TW_PREC_FP64) {
      if (P->d[0].qmax > 4 * P->p || P->d[1].qmax > 4 * P->p) {
        set_error("tw_batch_create: patch %d has more than 4p WQ points in one support", k);
        return TW_EUNSUPPORTED;
      }
      int rc = ensure_split_tables(P, s);
      if (rc) return rc;
    }
    BatchPatch &b = hp[k];
    memset(&b, 0, sizeof(b));
    RowArgs &ra = b.ra;
    ra.A = P->d[0];
    ra.B = P->d[1];
    ra.G = P->geo;
    ra.estate = P->estate;
    ra.fstate = P->fstate;
    ra.act = P->act;
    ra.rp = P->row_ptr;
    ra.C = P->C;
    ra.gslot = P->gslot;
    ra.gc = P->gc;
    ra.cut_slot = P->cut_slot;
    ra.cut_off = P->cut_off;
    ra.cut_B = P->cut_B;
    ra.cut_wc = P->cut_wc;
    ra.cut_pts = P->cut_pts;
    ra.cut_M = P->cut_M;
    ra.choice = P->choice;
    for (int d = 0; d < 2; d++) {
      ra.disc_slot[d] = P->disc_slot[d];
      ra.dwq_x[d] = P->dwq_x[d];
      ra.dwq_np[d] = P->dwq_np[d];
      ra.dwq_w[d] = P->dwq_w[d];
      ra.dwq_k[d] = P->dwq_k[d];
      ra.dwq_e[d] = P->dwq_e[d];
      ra.dwq_B[d] = P->dwq_B[d];
      ra.dwq_dB[d] = P->dwq_dB[d];
      ra.dwq_r[d] = P->dwq_r[d];
    }
    ra.gmat = P->gmat;
    ra.method = P->method;
    ra.flag = P->flag;
    if (precision != TW_PREC_FP64)
      b.tb = tables32(P, precision == TW_PREC_FP32X2, col[k], val[k]);
    b.cutrows = P->cutrows;
    b.rp_in = P->row_ptr;
    b.nrp = P->n_rows + 1;
    b.rp_out = row_ptr[k];
    b.col = col[k];
    b.val = val[k];
    b.p = P->p;
  }
  tw_batch *B = (tw_batch *)calloc(1, sizeof(tw_batch));
  B->n = n;
  B->precision = precision;
  int present[TW_MAXP + 1] = {0};
  for (auto *P : pt) present[P->p] = 1;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  for (int p = 1; p <= TW_MAXP; p++) {
    if (!present[p]) continue;
    // LIGHT is sized for each candidate tile while the tiles are tuned, and
    // for the chosen tile after
    cudaError_t e = size_q(B, 3 * p + ROLE_LIGHT, nsm, tile_max(p));
    if (e != cudaSuccess) {
      set_error("tw_batch_create: persistent kernel of degree %d does not fit (%s)", p,
                cudaGetErrorString(e));
      batch_free(B);
      return TW_ECUDA;
    }
  }
  if (cudaMalloc(&B->dpatch, sizeof(BatchPatch) * n) != cudaSuccess ||
      cudaMalloc(&B->counter, sizeof(int) * (TW_NQ)) != cudaSuccess) {
    set_error("tw_batch_create: out of device memory");
    batch_free(B);
    return TW_ENOMEM;
  }
  cudaMemcpyAsync(B->dpatch, hp.data(), sizeof(BatchPatch) * n, cudaMemcpyHostToDevice, s);

  // cut rows per degree: the ones that only gather precomputed element
  // matrices (cutrow_is_gather) in groups of TW_GATHER_ROWS, one warp each
  // (LIGHT), the others one item each (HEAVY)
  std::vector<int4> gath[TW_MAXP + 1], heavy[TW_MAXP + 1];
  for (int k = 0; k < n; k++) {
    tw_patch *P = pt[k];
    const int p = P->p;
    if (P->ncutrows == 0) continue;
    std::vector<int32_t> rows(P->ncutrows);
    cudaMemcpy(rows.data(), P->cutrows, sizeof(int32_t) * P->ncutrows, cudaMemcpyDeviceToHost);
    const bool gather = P->gmat && P->method != TW_METHOD_NAIVE;
    std::vector<int32_t> choice;
    if (gather && P->method == TW_METHOD_DWQ) {
      choice.resize((size_t)4 * P->d[0].n * P->d[1].n);
      cudaMemcpy(choice.data(), P->choice, sizeof(int32_t) * choice.size(), cudaMemcpyDeviceToHost);
    }
    int run0 = -1, runn = 0;
    for (int r = 0; r <= P->ncutrows; r++) {
      bool isg = false;
      if (r < P->ncutrows && gather) isg = choice.empty() || choice[(size_t)4 * rows[r]] < 0;
      if (isg && runn > 0 && run0 + runn == r && runn < TW_GATHER_ROWS) {
        runn++;
        continue;
      }
      if (runn > 0) gath[p].push_back(make_int4(item_code(IT_GATHER, p, 0), k, run0, runn));
      runn = 0;
      if (r == P->ncutrows) break;
      if (isg) {
        run0 = r;
        runn = 1;
      } else {
        heavy[p].push_back(make_int4(item_code(IT_CUTROW, p, 0), k, rows[r], 0));
      }
    }
  }
  // LIGHT's list for tile T: the gathers and the interior tiles interleaved by
  // the fraction of each list taken, so that the items in flight are a mix of
  // both kinds from the first to the last
  auto light_items = [&](int p, int T) {
    std::vector<int4> inner, out;
    interior_items(pt, p, T, inner);
    const std::vector<int4> &cut = gath[p];
    size_t a2 = 0, b2 = 0;
    while (a2 < cut.size() || b2 < inner.size()) {
      const bool take_cut =
          b2 >= inner.size() ||
          (a2 < cut.size() && (2 * a2 + 1) * inner.size() <= (2 * b2 + 1) * cut.size());
      out.push_back(take_cut ? cut[a2++] : inner[b2++]);
    }
    return out;
  };

  // autotuner: per degree present, time the LIGHT launch of that degree
  // (its interior tiles interleaved with its gathers) with each candidate tile
  // (best of 2) and keep the fastest; results are cached per device,
  // precision and degree
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int p = 1; p <= TW_MAXP; p++) {
    B->tile[p] = 32;
    if (!present[p]) continue;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      if (dev < 64 && g_tuned[dev][precision][p]) {
        B->tile[p] = g_tuned[dev][precision][p];
        continue;
      }
    }
    double best = 1e300;
    for (int c = 0; c < 3; c++) {
      B->tune_ms[p][c] = 0.0;
      if (g_tiles[c] > tile_max(p)) continue;
      std::vector<int4> it = light_items(p, g_tiles[c]);
      B->tune_ms[p][c] = 0.0;
      if (it.empty()) continue;
      const int q = 3 * p + ROLE_LIGHT;
      if (size_q(B, q, nsm, g_tiles[c]) != cudaSuccess) continue;
      int4 *dit = nullptr;
      if (cudaMalloc(&dit, sizeof(int4) * it.size()) != cudaSuccess) break;
      cudaMemcpyAsync(dit, it.data(), sizeof(int4) * it.size(), cudaMemcpyHostToDevice, s);
      float ms = 1e30f;
      for (int rep = 0; rep < 2; rep++) {
        cudaMemsetAsync(B->counter + q, 0, sizeof(int), s);
        cudaEventRecord(e0, s);
        launch_q(B, q, dit, (int)it.size(), B->counter + q, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms = std::min(ms, t);
      }
      cudaFree(dit);
      B->tune_ms[p][c] = ms;
      if (ms < best) {
        best = ms;
        B->tile[p] = g_tiles[c];
      }
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (dev < 64) g_tuned[dev][precision][p] = B->tile[p];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int p = 1; p <= TW_MAXP; p++) {
    if (!present[p]) continue;
    cudaError_t e = size_q(B, 3 * p + ROLE_LIGHT, nsm, B->tile[p]);
    if (e == cudaSuccess) e = size_q(B, 3 * p + ROLE_HEAVY, nsm, 0);
    if (e != cudaSuccess) {
      set_error("tw_batch_create: interior launch of degree %d does not fit (%s)", p,
                cudaGetErrorString(e));
      batch_free(B);
      return TW_ECUDA;
    }
  }

  // the work list, degree by degree: HEAVY's block-per-row cut rows, then
  // LIGHT's interleaved gathers and interior tiles, row-pointer copies last
  std::vector<int4> items;
  for (int p = TW_MAXP; p >= 1; p--) {
    const int qh = 3 * p + ROLE_HEAVY, ql = 3 * p + ROLE_LIGHT;
    B->ioff[qh] = (int)items.size();
    items.insert(items.end(), heavy[p].begin(), heavy[p].end());
    B->icnt[qh] = (int)heavy[p].size();
    B->ioff[ql] = (int)items.size();
    std::vector<int4> li = light_items(p, B->tile[p]);
    items.insert(items.end(), li.begin(), li.end());
    for (int k = 0; k < n; k++) {
      if (pt[k]->p != p) continue;
      int64_t nrp = pt[k]->n_rows + 1;
      for (int64_t c = 0; c * TW_RP_CHUNK < nrp; c++)
        items.push_back(make_int4(item_code(IT_ROWPTR, p, 0), k, (int)c, 0));
    }
    B->icnt[ql] = (int)items.size() - B->ioff[ql];
  }
  B->nitems = (int)items.size();
  if (cudaMalloc(&B->ditems, sizeof(int4) * std::max<size_t>(1, items.size())) != cudaSuccess) {
    set_error("tw_batch_create: out of device memory for %d items", B->nitems);
    batch_free(B);
    return TW_ENOMEM;
  }
  cudaMemcpyAsync(B->ditems, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, s);
  if (check_cuda(cudaStreamSynchronize(s), "tw_batch_create")) {
    batch_free(B);
    return TW_ECUDA;
  }
  // one graph: reset the counters, then one persistent launch per degree on
  // its own branch (fork / join through events), so the degrees' launches
  // run concurrently within one replay
  cudaError_t e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
  for (int q = 0; q < TW_NQ && e == cudaSuccess; q++) {
    if (!B->icnt[q]) continue;
    e = cudaStreamCreateWithFlags(&B->br[q], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->join[q], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(B->counter, 0, sizeof(int) * (TW_NQ), B->cap);
    cudaEventRecord(B->fork, B->cap);
    for (int role : {ROLE_HEAVY, ROLE_LIGHT})
      for (int p = TW_MAXP; p >= 1; p--) {
        const int q = 3 * p + role;
        if (!B->icnt[q]) continue;
        cudaStreamWaitEvent(B->br[q], B->fork, 0);
        launch_q(B, q, B->ditems + B->ioff[q], B->icnt[q], B->counter + q, B->br[q]);
        cudaEventRecord(B->join[q], B->br[q]);
        cudaStreamWaitEvent(B->cap, B->join[q], 0);
      }
    e = cudaStreamEndCapture(B->cap, &B->graph);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, B->graph, 0);
  if (e != cudaSuccess) {
    set_error("tw_batch_create: graph capture failed: %s", cudaGetErrorString(e));
    batch_free(B);
    return TW_ECUDA;
  }
  *out = B;
  return TW_OK;
}

extern "C" int tw_batch_run(tw_batch *B, void *stream) {
  if (!B) {
    set_error("tw_batch_run: NULL batch");
    return TW_EINVAL;
  }
  g_launches++;
  return check_cuda(cudaGraphLaunch(B->exec, (cudaStream_t)stream), "tw_batch_run");
}

extern "C" int tw_batch_info(const tw_batch *B, int64_t *info) {
  if (!B || !info) {
    set_error("tw_batch_info: NULL argument");
    return TW_EINVAL;
  }
  int64_t grid = 0, smem = 0;
  for (int q = 0; q < TW_NQ; q++)
    if (B->icnt[q]) {
      grid = std::max<int64_t>(grid, B->grid[q]);
      smem = std::max<int64_t>(smem, (int64_t)B->smem[q]);
    }
  info[0] = B->n;
  info[1] = B->nitems;
  info[2] = grid;
  info[3] = smem;
  for (int p = 1; p <= TW_MAXP; p++) info[3 + p] = B->tile[p];
  return TW_OK;
}

extern "C" int tw_batch_destroy(tw_batch *B) {
  batch_free(B);
  return TW_OK;
}
