// tw_batch.cu -- forming many patches' mass matrices with one persistent launch.
//
// A batch owns, for a fixed list of patches and output CSR buffers:
//  * a device array of per-patch descriptors (the patch tables and outputs);
//  * a work list of items -- interior tiles (patch, i2, first i1) sized by a
//    tile chosen per (degree, precision) by the autotuner, cut rows (patch,
//    row) and row-pointer chunks -- ordered by estimated cost, largest first;
//  * a CUDA graph of one memset of the work counter and one persistent launch
//    of k_batch: every block takes the next item with an atomicAdd on the
//    counter and runs its body, until the list is exhausted (blocks never wait
//    on one another).
// Items write disjoint parts of the outputs and every body sums in a fixed
// order, so the result equals the one-patch formation bit for bit.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "tw_bodies.cuh"

namespace tw {

int ensure_split_tables(tw_patch *P, cudaStream_t s);

struct BatchPatch {
  RowArgs ra;
  const float2 *Cf, *Vf0, *Vf1;
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

template <int PREC>
__device__ __forceinline__ void run_interior(const BatchPatch &b, int P, int i2, int i1a, int T,
                                             char *smem) {
  const RowArgs &a = b.ra;
  switch (P) {
#define TW_IT(PP)                                                                                \
  case PP:                                                                                       \
    if constexpr (PREC == TW_PREC_FP64)                                                          \
      interior_tile<PP>(a.A, a.B, a.C, a.fstate, a.act, a.rp, b.col, (double *)b.val, i2, i1a, T, \
                        smem);                                                                   \
    else                                                                                         \
      interior_tile32<PP, PREC == TW_PREC_FP32X2>(a.A, a.B, b.Cf, b.Vf0, b.Vf1, a.fstate, a.act,  \
                                                  a.rp, b.col, b.val, i2, i1a, T, smem);         \
    break;
    TW_IT(1) TW_IT(2) TW_IT(3) TW_IT(4) TW_IT(5) TW_IT(6)
#undef TW_IT
  }
}

template <int PREC>
__device__ __forceinline__ void run_cutrow(const BatchPatch &b, int P, int g, char *smem) {
  switch (P) {
#define TW_CR(PP)                                                          \
  case PP:                                                                 \
    if constexpr (PREC == TW_PREC_FP32)                                    \
      cutrow_item<PP, float>(b.ra, g, b.col, (float *)b.val, smem);        \
    else                                                                   \
      cutrow_item<PP, double>(b.ra, g, b.col, (double *)b.val, smem);      \
    break;
    TW_CR(1) TW_CR(2) TW_CR(3) TW_CR(4) TW_CR(5) TW_CR(6)
#undef TW_CR
  }
}

template <int PREC>
__device__ __forceinline__ void run_gather(const BatchPatch &b, int P, int g, int lane,
                                           const double **tab) {
  switch (P) {
#define TW_CG(PP)                                                                    \
  case PP:                                                                           \
    if constexpr (PREC == TW_PREC_FP32)                                              \
      cutrow_gather_warp<PP, float>(b.ra, g, lane, tab, b.col, (float *)b.val);      \
    else                                                                             \
      cutrow_gather_warp<PP, double>(b.ra, g, lane, tab, b.col, (double *)b.val);    \
    break;
    TW_CG(1) TW_CG(2) TW_CG(3) TW_CG(4) TW_CG(5) TW_CG(6)
#undef TW_CG
  }
}

// item = {kind | P << 4 | T << 8, patch, x, y}; a gather item is up to
// TW_GATHER_ROWS cut rows (x = first index into the patch's cut-row list,
// y = count), one per warp
template <int PREC>
__global__ void __launch_bounds__(256, 3) k_batch(const BatchPatch *__restrict__ bp,
                                               const int4 *__restrict__ items, int nitems,
                                               int *counter) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int cur;
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
    __syncthreads();
    const int it = cur;
    __syncthreads();
    if (it >= nitems) break;
    const int4 w = items[it];
    const int kind = w.x & 15, P = (w.x >> 4) & 15, T = w.x >> 8;
    const BatchPatch &b = bp[w.y];
    if (kind == IT_INTERIOR) {
      run_interior<PREC>(b, P, w.z, w.w, T, smem);
    } else if (kind == IT_CUTROW) {
      run_cutrow<PREC>(b, P, w.z, smem);
    } else if (kind == IT_GATHER) {
      const int wib = threadIdx.x >> 5;
      if (wib < w.w)
        run_gather<PREC>(b, P, b.cutrows[w.z + wib], threadIdx.x & 31,
                         (const double **)smem + wib * (TW_MAXP1 * TW_MAXP1));
    } else {
      const int64_t lo = (int64_t)w.z * TW_RP_CHUNK;
      const int64_t hi = min(b.nrp, lo + TW_RP_CHUNK);
      for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) b.rp_out[k] = b.rp_in[k];
    }
    __syncthreads();
  }
}

// candidate interior tiles per degree: up to 64 rows at p <= 4, 32 above, so
// the tile's staged outputs keep the block's shared memory near 56 KB
static const int g_tiles[3] = {16, 32, 64};
static int tile_max(int p) { return p <= 4 ? 64 : 32; }

static size_t batch_smem(int prec) {
  size_t s = std::max(sizeof(CutSmem<TW_MAXP>),
                      sizeof(double *) * TW_GATHER_ROWS * TW_MAXP1 * TW_MAXP1);
  for (int p = 1; p <= TW_MAXP; p++) {
    const int t = tile_max(p);
    size_t i = prec == TW_PREC_FP64 ? interior_smem(p, t)
                                    : interior32_smem(p, t, prec == TW_PREC_FP32X2);
    s = std::max(s, i);
  }
  return (s + 15) / 16 * 16;
}

static std::mutex g_tune_mu;
static int g_tuned[64][3][TW_MAXP + 1];  // [device][precision][p] -> tile (0: not tuned)

}  // namespace tw

using namespace tw;

struct tw_batch {
  int n, precision, grid, nitems;
  size_t smem;
  BatchPatch *dpatch;
  int4 *ditems;
  int *counter;
  cudaStream_t cap;
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
  cudaFree(B->dpatch);
  cudaFree(B->ditems);
  cudaFree(B->counter);
  free(B);
}

template <int PREC>
static void launch_batch(tw_batch *B, const int4 *items, int nitems, cudaStream_t s) {
  k_batch<PREC><<<B->grid, 256, B->smem, s>>>(B->dpatch, items, nitems, B->counter);
  TW_LAUNCH();
}

static void launch_any(tw_batch *B, const int4 *items, int nitems, cudaStream_t s) {
  if (B->precision == TW_PREC_FP64) launch_batch<TW_PREC_FP64>(B, items, nitems, s);
  else if (B->precision == TW_PREC_FP32) launch_batch<TW_PREC_FP32>(B, items, nitems, s);
  else launch_batch<TW_PREC_FP32X2>(B, items, nitems, s);
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
    if (precision != TW_PREC_FP64) {
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
      ra.dwq_r[d] = P->dwq_r[d];
    }
    ra.gmat = P->gmat;
    ra.method = P->method;
    ra.flag = P->flag;
    b.Cf = P->Cf;
    b.Vf0 = P->Vf[0];
    b.Vf1 = P->Vf[1];
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
  B->smem = batch_smem(precision);
  int dev = 0, nsm = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaSuccess;
  if (precision == TW_PREC_FP64) {
    e = cudaFuncSetAttribute(k_batch<TW_PREC_FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<TW_PREC_FP64>, 256, B->smem);
  } else if (precision == TW_PREC_FP32) {
    e = cudaFuncSetAttribute(k_batch<TW_PREC_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<TW_PREC_FP32>, 256, B->smem);
  } else {
    e = cudaFuncSetAttribute(k_batch<TW_PREC_FP32X2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<TW_PREC_FP32X2>, 256, B->smem);
  }
  if (e != cudaSuccess || occ <= 0) {
    set_error("tw_batch_create: persistent kernel does not fit (%s, occupancy %d)",
              cudaGetErrorString(e), occ);
    batch_free(B);
    return TW_ECUDA;
  }
  B->grid = nsm * occ;
  if (cudaMalloc(&B->dpatch, sizeof(BatchPatch) * n) != cudaSuccess ||
      cudaMalloc(&B->counter, sizeof(int)) != cudaSuccess) {
    set_error("tw_batch_create: out of device memory");
    batch_free(B);
    return TW_ENOMEM;
  }
  cudaMemcpyAsync(B->dpatch, hp.data(), sizeof(BatchPatch) * n, cudaMemcpyHostToDevice, s);

  // autotuner: per degree present, time the interior tiles of that degree's
  // patches with each candidate tile (persistent launch, best of 2) and keep
  // the fastest; results are cached per device, precision and degree
  int present[TW_MAXP + 1] = {0};
  for (auto *P : pt) present[P->p] = 1;
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
      std::vector<int4> it;
      interior_items(pt, p, g_tiles[c], it);
      B->tune_ms[p][c] = 0.0;
      if (it.empty()) continue;
      int4 *dit = nullptr;
      if (cudaMalloc(&dit, sizeof(int4) * it.size()) != cudaSuccess) break;
      cudaMemcpyAsync(dit, it.data(), sizeof(int4) * it.size(), cudaMemcpyHostToDevice, s);
      float ms = 1e30f;
      for (int rep = 0; rep < 2; rep++) {
        cudaMemsetAsync(B->counter, 0, sizeof(int), s);
        cudaEventRecord(e0, s);
        launch_any(B, dit, (int)it.size(), s);
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

  // the work list: cut rows (heaviest) by degree descending, interior tiles by
  // degree descending, row-pointer copies last
  // rows that only gather precomputed element matrices (cutrow_is_gather) go
  // in groups of TW_GATHER_ROWS, one warp each; the others are one item each
  std::vector<int4> items;
  for (int p = TW_MAXP; p >= 1; p--)
    for (int k = 0; k < n; k++) {
      tw_patch *P = pt[k];
      if (P->p != p || P->ncutrows == 0) continue;
      std::vector<int32_t> rows(P->ncutrows);
      cudaMemcpy(rows.data(), P->cutrows, sizeof(int32_t) * P->ncutrows, cudaMemcpyDeviceToHost);
      const bool gather = P->gmat && P->method != TW_METHOD_NAIVE;
      std::vector<int32_t> choice;
      if (gather && P->method == TW_METHOD_DWQ) {
        choice.resize((size_t)4 * P->d[0].n * P->d[1].n);
        cudaMemcpy(choice.data(), P->choice, sizeof(int32_t) * choice.size(),
                   cudaMemcpyDeviceToHost);
      }
      int run0 = -1, runn = 0;
      for (int r = 0; r <= P->ncutrows; r++) {
        bool isg = false;
        if (r < P->ncutrows && gather)
          isg = choice.empty() || choice[(size_t)4 * rows[r]] < 0;
        if (isg && runn > 0 && run0 + runn == r && runn < TW_GATHER_ROWS) {
          runn++;
          continue;
        }
        if (runn > 0) items.push_back(make_int4(item_code(IT_GATHER, p, 0), k, run0, runn));
        runn = 0;
        if (r == P->ncutrows) break;
        if (isg) {
          run0 = r;
          runn = 1;
        } else {
          items.push_back(make_int4(item_code(IT_CUTROW, p, 0), k, rows[r], 0));
        }
      }
    }
  for (int p = TW_MAXP; p >= 1; p--) interior_items(pt, p, B->tile[p], items);
  for (int k = 0; k < n; k++) {
    int64_t nrp = pt[k]->n_rows + 1;
    for (int64_t c = 0; c * TW_RP_CHUNK < nrp; c++)
      items.push_back(make_int4(item_code(IT_ROWPTR, 0, 0), k, (int)c, 0));
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
  // one graph: reset the counter, one persistent launch
  cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
  e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(B->counter, 0, sizeof(int), B->cap);
    launch_any(B, B->ditems, B->nitems, B->cap);
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
  info[0] = B->n;
  info[1] = B->nitems;
  info[2] = B->grid;
  info[3] = (int64_t)B->smem;
  for (int p = 1; p <= TW_MAXP; p++) info[3 + p] = B->tile[p];
  return TW_OK;
}

extern "C" int tw_batch_destroy(tw_batch *B) {
  batch_free(B);
  return TW_OK;
}
