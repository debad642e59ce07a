// tw_api.cu -- the C-ABI entry points of include/trimwq.h: descriptor
// validation, device allocation of the patch tables and dispatch to the
// set-up, formation and solver kernels.  Host code only orchestrates: every
// step of the method runs in a kernel.
#include <cmath>
#include <cstdarg>
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include <atomic>
#include <mutex>
#include <vector>

#include "tw_internal.cuh"

namespace tw {

std::atomic<int64_t> g_launches{0};
std::atomic<int64_t> g_pool_allocs{0};
static std::mutex g_prof_mu;

// ---- stage profiler: event pairs on the launching stream ----
struct ProfRec {
  int stage;
  cudaEvent_t a, b;
};
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof;

int prof_start(cudaStream_t s) {
  if (!g_prof_on) return -1;
  ProfRec r;
  r.stage = -1;
  cudaEventCreate(&r.a);
  cudaEventCreate(&r.b);
  cudaEventRecord(r.a, s);
  std::lock_guard<std::mutex> lock(g_prof_mu);
  g_prof.push_back(r);
  return (int)g_prof.size() - 1;
}

void prof_stop(int slot, int stage, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_prof_mu);
  if (slot < 0 || slot >= (int)g_prof.size()) return;
  g_prof[slot].stage = stage;
  cudaEventRecord(g_prof[slot].b, s);
}
static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int check_cuda(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return 0;
  set_error("%s: %s", what, cudaGetErrorString(e));
  return TW_ECUDA;
}

// The library's device memory comes from one stream-ordered pool per device
// that keeps freed memory for reuse (release threshold: unlimited), so a
// patch's tables are carved from memory the previous patches returned rather
// than mapped anew after every synchronisation.  The pool holds at most the
// peak of the library's live allocations until the process exits.
#define TW_POOL_MAX_DEVICES 64
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[TW_POOL_MAX_DEVICES];

static cudaMemPool_t library_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= TW_POOL_MAX_DEVICES) return nullptr;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pool[dev] = pool;
  }
  return g_pool[dev];
}

// During tw_patch_create the small tables are carved from TW_ARENA_SLAB-byte
// slabs (256-byte aligned), so creating a patch makes a handful of pool
// allocations instead of one per table; larger tables get their own.
#define TW_ARENA_SLAB ((size_t)2 << 20)

void *dalloc(tw_patch *P, size_t bytes) {
  size_t need = ((bytes ? bytes : 16) + 255) & ~(size_t)255;
  if (P->arena_on && need <= P->arena_left) {
    void *q = P->arena;
    P->arena += need;
    P->arena_left -= need;
    return q;
  }
  const bool slab = P->arena_on && need <= TW_ARENA_SLAB / 4;
  if (P->nallocs >= (int)(sizeof(P->allocs) / sizeof(P->allocs[0]))) {
    set_error("internal: too many device allocations for one patch");
    return nullptr;
  }
  void *p = nullptr;
  const size_t sz = slab ? TW_ARENA_SLAB : need;
  cudaMemPool_t pool = library_pool();
  cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, sz, pool, P->stream)
                       : cudaMallocAsync(&p, sz, P->stream);
  if (e != cudaSuccess) {
    set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return nullptr;
  }
  P->allocs[P->nallocs++] = p;
  g_pool_allocs++;
  if (slab) {
    P->arena = (char *)p + need;
    P->arena_left = TW_ARENA_SLAB - need;
  }
  return p;
}

void release_to(tw_patch *P, int mark) {
  while (P->nallocs > mark) cudaFreeAsync(P->allocs[--P->nallocs], P->stream);
}

// R1 point counts per knot span: none on the zero-length span of a repeated
// knot, p+1 on a span touching a knot of multiplicity >= 2 (the domain ends, a
// repeated interior knot), 2 elsewhere.  cnt[e] for e = 0..nel-1.
static void wq_counts(const double *U, int nk, int p, int nel, int *cnt) {
  auto mult = [&](int j) {  // multiplicity of the knot value U[j]
    int a = j, b = j;
    while (a > 0 && U[a - 1] == U[j]) a--;
    while (b + 1 < nk && U[b + 1] == U[j]) b++;
    return b - a + 1;
  };
  for (int e = 0; e < nel; e++) {
    const int j = p + e;
    if (!(U[j + 1] > U[j])) cnt[e] = 0;
    else cnt[e] = (mult(j) >= 2 || mult(j + 1) >= 2) ? p + 1 : 2;
  }
}

static int valid_open_knots(const double *U, int nk, int p, const char *what) {
  if (!U) {
    set_error("%s: knots pointer is NULL", what);
    return 0;
  }
  int nel = nk - 2 * p - 1;
  if (nel < 2) {
    set_error("%s: need at least 2 elements (nknots = %d, p = %d)", what, nk, p);
    return 0;
  }
  for (int k = 0; k < nk; k++)
    if (!std::isfinite(U[k])) {
      set_error("%s: knot %d is not finite", what, k);
      return 0;
    }
  for (int k = 1; k <= p; k++)
    if (U[k] != U[0] || U[nk - 1 - k] != U[nk - 1]) {
      set_error("%s: knot vector is not open (p+1 equal end knots)", what);
      return 0;
    }
  if (!(U[p + 1] > U[p]) || !(U[nk - 1 - p] > U[nk - 2 - p])) {
    set_error("%s: knot vector is not open (more than p+1 equal end knots)", what);
    return 0;
  }
  for (int k = p; k < nk - p - 1; k++)
    if (U[k + 1] < U[k]) {
      set_error("%s: knots must be non-decreasing", what);
      return 0;
    }
  // interior knots (positions p+1 .. nk-p-2) of multiplicity m <= p: C^{p-m}
  for (int k = p + 1; k + p <= nk - p - 2; k++)
    if (U[k + p] == U[k]) {
      set_error("%s: interior knot %g of multiplicity > p (C^-1)", what, U[k]);
      return 0;
    }
  return 1;
}

}  // namespace tw

using namespace tw;

// curve k of a descriptor: -1 the trim_* fields, else trim_extra[k]
static tw_trim_curve curve_of(const tw_patch_desc *d, int k) {
  if (k >= 0) return d->trim_extra[k];
  tw_trim_curve t;
  t.kind = d->trim_kind;
  t.keep_inside = d->trim_keep_inside;
  for (int m = 0; m < 6; m++) t.params[m] = d->trim_params[m];
  t.nctrl = d->trim_nctrl;
  t.ctrl = d->trim_ctrl;
  return t;
}

static bool valid_curve(const tw_trim_curve &t, int k) {
  const char *which = k < 0 ? "trim" : "trim_extra";
  if (t.kind < TW_TRIM_NONE || t.kind > TW_TRIM_LINE) {
    set_error("tw_patch_create: unknown %s kind %d", which, t.kind);
    return false;
  }
  if (t.kind == TW_TRIM_CIRCLE && !(t.params[2] > 0)) {
    set_error("tw_patch_create: circle radius must be > 0");
    return false;
  }
  if (t.kind == TW_TRIM_ELLIPSE && !(t.params[2] > 0 && t.params[3] > 0)) {
    set_error("tw_patch_create: ellipse semi-axes must be > 0");
    return false;
  }
  if (t.kind == TW_TRIM_LINE && !(t.params[0] != t.params[2] || t.params[1] != t.params[3])) {
    set_error("tw_patch_create: a trimming line needs two distinct points");
    return false;
  }
  if (t.kind == TW_TRIM_BSPLINE3 && (!t.ctrl || t.nctrl < 4 || t.nctrl > 4096)) {
    set_error("tw_patch_create: spline curve needs 4..4096 control points");
    return false;
  }
  return true;
}

extern "C" const char *tw_last_error(void) { return g_err; }
extern "C" int64_t tw_launch_count(void) { return g_launches.load(); }

extern "C" int tw_pool_info(int64_t *info3) {
  if (!info3) {
    tw::set_error("tw_pool_info: NULL argument");
    return TW_EINVAL;
  }
  info3[0] = tw::g_pool_allocs.load();
  info3[1] = info3[2] = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= TW_POOL_MAX_DEVICES) return TW_OK;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lock(tw::g_pool_mu);
    pool = tw::g_pool[dev];
  }
  if (!pool) return TW_OK;
  uint64_t v = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v) == cudaSuccess)
    info3[1] = (int64_t)v;
  v = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v) == cudaSuccess)
    info3[2] = (int64_t)v;
  return TW_OK;
}

extern "C" int tw_profile_enable(int on) {
  g_prof_on = on != 0;
  return TW_OK;
}

extern "C" int tw_profile_read(int stage, double *total_ms, int64_t *count) {
  if (stage < 0 || stage >= TW_NSTAGES) {
    set_error("tw_profile_read: unknown stage %d", stage);
    return TW_EINVAL;
  }
  double ms = 0.0;
  int64_t n = 0;
  std::lock_guard<std::mutex> lock(g_prof_mu);
  std::vector<ProfRec> keep;
  for (auto &r : g_prof) {
    if (r.stage != stage) {
      keep.push_back(r);
      continue;
    }
    float t = 0.f;
    cudaEventSynchronize(r.b);
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms += t;
    n++;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_prof.swap(keep);
  if (total_ms) *total_ms = ms;
  if (count) *count = n;
  return TW_OK;
}

// Stream-ordered: the frees run when the patch's stream reaches them, and no
// pending work of the patch reads its host structures (every call that copies
// into them synchronises before it returns), so they are released at once.
extern "C" int tw_patch_destroy(tw_patch *P) {
  if (!P) return TW_OK;
  for (int k = P->nallocs - 1; k >= 0; k--) cudaFreeAsync(P->allocs[k], P->stream);
  free(P->ext);
  free(P);
  return TW_OK;
}

extern "C" int tw_patch_create(const tw_patch_desc *desc, tw_patch **out) {
  if (!desc || !out) {
    set_error("tw_patch_create: NULL argument");
    return TW_EINVAL;
  }
  *out = nullptr;
  int p = desc->p[0];
  if (p < 1 || p > TW_MAXP || desc->p[1] != p) {
    set_error("tw_patch_create: degrees (%d, %d) unsupported (need p1 == p2 in 1..%d)",
              desc->p[0], desc->p[1], TW_MAXP);
    return TW_EUNSUPPORTED;
  }
  for (int d = 0; d < 2; d++)
    if (!valid_open_knots(desc->knots[d], desc->nknots[d], p, d ? "knots[1]" : "knots[0]"))
      return TW_EINVAL;
  if (desc->trim_nextra < 0 || desc->trim_nextra > TW_MAXCURVES - 1 ||
      (desc->trim_nextra > 0 && !desc->trim_extra)) {
    set_error("tw_patch_create: trim_nextra must be 0..%d with a curve array", TW_MAXCURVES - 1);
    return TW_EINVAL;
  }
  for (int k = -1; k < desc->trim_nextra; k++) {
    tw_trim_curve t = curve_of(desc, k);
    if (!valid_curve(t, k)) return TW_EINVAL;
  }
  if (desc->geom_kind != TW_GEOM_IDENTITY && desc->geom_kind != TW_GEOM_SPLINE) {
    set_error("tw_patch_create: unknown geom_kind %d", desc->geom_kind);
    return TW_EINVAL;
  }
  if (desc->geom_kind == TW_GEOM_SPLINE && !desc->geom_ctrl) {
    set_error("tw_patch_create: spline geometry without control net");
    return TW_EINVAL;
  }
  if (desc->coef_kind < TW_COEF_ONE || desc->coef_kind > TW_COEF_DENSITY) {
    set_error("tw_patch_create: unknown coef_kind %d", desc->coef_kind);
    return TW_EINVAL;
  }
  if (desc->coef_kind == TW_COEF_DENSITY) {
    for (int d = 0; d < 2; d++) {
      int q = desc->dens_p[d];
      if (q < 0 || q > TW_MAXP || !desc->dens_coef ||
          !valid_open_knots(desc->dens_knots[d], desc->dens_nknots[d], q, "density knots"))
        return TW_EINVAL;
    }
  }
  if (desc->method < TW_METHOD_GAUSS || desc->method > TW_METHOD_NAIVE) {
    set_error("tw_patch_create: unknown method %d", desc->method);
    return TW_EINVAL;
  }
  if (desc->cut_order < 0 || desc->cut_order > 64) {
    set_error("tw_patch_create: cut_order must be in 0..64");
    return TW_EINVAL;
  }
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
    set_error("tw_patch_create: no CUDA device");
    return TW_ECUDA;
  }

  tw_patch *P = (tw_patch *)calloc(1, sizeof(tw_patch));
  if (!P) {
    set_error("tw_patch_create: out of host memory");
    return TW_ENOMEM;
  }
  P->arena_on = 1;
  P->p = p;
  P->method = desc->method;
  P->qc = desc->cut_order > 0 ? desc->cut_order : p + 1;
  P->stream = (cudaStream_t)desc->stream;
  int rc = TW_ENOMEM;
  cudaStream_t st = P->stream;
  // host staging of the breakpoints, kept until the set-up's final
  // synchronisation (the copies may read them until then)
  double *hbp[2] = {nullptr, nullptr};
  int *hoff[2] = {nullptr, nullptr};
  uint8_t *htwo[2] = {nullptr, nullptr};
  // the small tables (knots, breakpoints, WQ offsets and flags, curve control
  // points, the zeroed error flags) go up in one copy from one packed staging
  // buffer, kept with the others: each entry is (address of the device
  // pointer to set, host source or NULL for zeros, bytes)
  struct Upload {
    void *dst;
    const void *src;
    size_t bytes;
  };
  Upload ups[11 + TW_MAXCURVES];
  int nup = 0;
  char *hpack = nullptr, *dpack = nullptr;
  size_t packed = 0;
#define ALLOC(ptr, T, n)                                   \
  do {                                                     \
    (ptr) = (T *)dalloc(P, sizeof(T) * (size_t)(n));       \
    if (!(ptr)) goto fail;                                 \
  } while (0)
  {
    for (int d = 0; d < 2; d++) {
      Dir &D = P->d[d];
      D.p = p;
      D.nk = desc->nknots[d];
      D.n = D.nk - p - 1;
      D.nel = D.n - p;
      // the WQ layout (R1) on the host: offsets per element, two-point rows
      hoff[d] = (int *)malloc(sizeof(int) * (D.nel + 1));
      htwo[d] = (uint8_t *)malloc((size_t)D.n);
      if (!hoff[d] || !htwo[d]) {
        set_error("tw_patch_create: out of host memory");
        goto fail;
      }
      wq_counts(desc->knots[d], D.nk, p, D.nel, hoff[d] + 1);
      hoff[d][0] = 0;
      for (int e = 0; e < D.nel; e++) {
        if (hoff[d][e + 1] == 0) P->mixed = 1;
        hoff[d][e + 1] += hoff[d][e];
      }
      D.nq = hoff[d][D.nel];
      D.qmax = 0;
      for (int i = 0; i < D.n; i++) {
        int lo = i - p < 0 ? 0 : i - p, hi = i < D.nel - 1 ? i : D.nel - 1;
        int c = hoff[d][hi + 1] - hoff[d][lo];
        if (c > D.qmax) D.qmax = c;
        // point-major rows: away from the end elements, two points in each
        // support element (every such row for simple knots)
        bool two = i >= p + 1 && i <= D.nel - 2;
        for (int e = lo; e <= hi && two; e++) two = hoff[d][e + 1] - hoff[d][e] == 2;
        htwo[d][i] = two ? 1 : 0;
      }
      if (d == 0)  // WQ points of the tiles of T consecutive test functions i1
        for (int lt = 0; lt < 7; lt++) {
          const int T = 1 << lt;
          int km = 0;
          for (int i1a = 0; i1a < D.n; i1a += T) {
            const int i1b = std::min(D.n, i1a + T);
            const int k = hoff[d][std::min(D.nel - 1, i1b - 1) + 1] - hoff[d][std::max(0, i1a - p)];
            km = std::max(km, k);
          }
          P->ktile[lt] = km;
        }
      if (D.qmax > TW_QMAX) {
        set_error("tw_patch_create: %d WQ points in one support exceed %d", D.qmax, TW_QMAX);
        rc = TW_EUNSUPPORTED;
        goto fail;
      }
      int W = 2 * p + 1;
      ALLOC(D.xq, double, D.nq);
      ALLOC(D.qel, int, D.nq);
      ALLOC(D.qbeg, int, D.n);
      ALLOC(D.qcnt, int, D.n);
      ALLOC(D.Bq, double, (size_t)D.nq * (p + 1));
      ALLOC(D.dBq, double, (size_t)D.nq * (p + 1));
      ALLOC(D.W, double, (size_t)D.n * D.qmax);
      ALLOC(D.V, double, (size_t)D.n * D.qmax * W);
      ALLOC(D.crange, int, (size_t)D.n * W);
      ALLOC(D.GB, double, (size_t)D.nel * (p + 1) * (p + 1));
      ALLOC(D.dGB, double, (size_t)D.nel * (p + 1) * (p + 1));
      ALLOC(D.GW, double, (size_t)D.nel * (p + 1) * (p + 1) * (p + 1));
      ups[nup++] = Upload{&D.qoff, hoff[d], sizeof(int) * (D.nel + 1)};
      ups[nup++] = Upload{&D.two, htwo[d], (size_t)D.n};
      hbp[d] = (double *)malloc(sizeof(double) * (D.nel + 1));
      if (!hbp[d]) {
        set_error("tw_patch_create: out of host memory");
        goto fail;
      }
      for (int e = 0; e <= D.nel; e++) hbp[d][e] = desc->knots[d][p + e];
      ups[nup++] = Upload{&D.U, desc->knots[d], sizeof(double) * D.nk};
      ups[nup++] = Upload{&D.bp, hbp[d], sizeof(double) * (D.nel + 1)};
    }
    Dir &A = P->d[0];
    Dir &B = P->d[1];
    A.mixed = B.mixed = P->mixed;
    // curves (the untrimmed kind left out)
    P->curves.n = 0;
    for (int k = -1; k < desc->trim_nextra; k++) {
      const tw_trim_curve t = curve_of(desc, k);
      if (t.kind == TW_TRIM_NONE) continue;
      const int ci = P->curves.n++;
      Curve &Cv = P->curves.c[ci];
      Cv.kind = t.kind;
      Cv.keep_inside = t.keep_inside;
      for (int m = 0; m < 6; m++) Cv.prm[m] = t.params[m];
      Cv.nc = t.kind == TW_TRIM_BSPLINE3 ? t.nctrl : 0;
      Cv.seg = Cv.box = nullptr;
      P->curve_ctrl[ci] = nullptr;
      if (Cv.nc > 0) {
        double *seg, *box;
        ALLOC(seg, double, 8 * Cv.nc);
        ALLOC(box, double, 4 * Cv.nc);
        Cv.seg = seg;
        Cv.box = box;
        ups[nup++] = Upload{&P->curve_ctrl[ci], t.ctrl, sizeof(double) * 2 * Cv.nc};
      }
    }
    // geometry and coefficient
    P->geo.geom_kind = desc->geom_kind;
    P->geo.coef_kind = desc->coef_kind;
    P->geo.n1 = A.n;
    if (desc->geom_kind == TW_GEOM_SPLINE) {
      double *g;
      ALLOC(g, double, 2 * (size_t)A.n * B.n);
      cudaMemcpyAsync(g, desc->geom_ctrl, sizeof(double) * 2 * (size_t)A.n * B.n,
                      cudaMemcpyHostToDevice, st);
      P->geo.ctrl = g;
    }
    if (desc->coef_kind == TW_COEF_DENSITY) {
      for (int d = 0; d < 2; d++) {
        double *u;
        P->geo.dp[d] = desc->dens_p[d];
        P->geo.dnk[d] = desc->dens_nknots[d];
        ALLOC(u, double, desc->dens_nknots[d]);
        cudaMemcpyAsync(u, desc->dens_knots[d], sizeof(double) * desc->dens_nknots[d],
                        cudaMemcpyHostToDevice, st);
        P->geo.dU[d] = u;
      }
      size_t m = (size_t)(desc->dens_nknots[0] - desc->dens_p[0] - 1) *
                 (desc->dens_nknots[1] - desc->dens_p[1] - 1);
      double *c;
      ALLOC(c, double, m);
      cudaMemcpyAsync(c, desc->dens_coef, sizeof(double) * m, cudaMemcpyHostToDevice, st);
      P->geo.dcoef = c;
    }
    int64_t ne = (int64_t)A.nel * B.nel, nf = (int64_t)A.n * B.n;
    ALLOC(P->estate, uint8_t, ne);
    ALLOC(P->fstate, uint8_t, nf);
    ALLOC(P->act, int32_t, nf);
    ALLOC(P->choice, int32_t, 4 * nf);
    ALLOC(P->cut_slot, int32_t, ne);
    ALLOC(P->gslot, int32_t, ne);
    ALLOC(P->disc_slot[0], int32_t, A.nel + 1);
    ALLOC(P->disc_slot[1], int32_t, B.nel + 1);
    ALLOC(P->C, double, (size_t)A.nq * B.nq);
    ups[nup++] = Upload{&P->flag, nullptr, 4 * sizeof(int32_t)};
    ups[nup++] = Upload{&P->cnt32, nullptr, 24 * sizeof(int32_t)};
    ups[nup++] = Upload{&P->cnt64, nullptr, 4 * sizeof(int64_t)};
    for (int k = 0; k < nup; k++) packed += (ups[k].bytes + 15) & ~(size_t)15;
    hpack = (char *)malloc(packed);
    if (!hpack) {
      set_error("tw_patch_create: out of host memory");
      goto fail;
    }
    ALLOC(dpack, char, packed);
    {
      size_t off = 0;
      for (int k = 0; k < nup; k++) {
        if (ups[k].src) memcpy(hpack + off, ups[k].src, ups[k].bytes);
        else memset(hpack + off, 0, ups[k].bytes);
        void *dv = dpack + off;
        memcpy(ups[k].dst, &dv, sizeof(void *));
        off += (ups[k].bytes + 15) & ~(size_t)15;
      }
    }
    cudaMemcpyAsync(dpack, hpack, packed, cudaMemcpyHostToDevice, st);
    {
      int ps = prof_start(st);
      rc = build_tables(P);
      prof_stop(ps, TW_STAGE_SETUP, st);
    }
    if (rc) goto fail;
  }
#undef ALLOC
  P->arena_on = 0;
  for (int d = 0; d < 2; d++) {  // build_tables ended with a synchronisation of the stream
    free(hbp[d]);
    free(hoff[d]);
    free(htwo[d]);
  }
  free(hpack);
  *out = P;
  return TW_OK;
fail:
  if (rc == TW_ENOMEM && !g_err[0]) set_error("tw_patch_create: out of device memory");
  if (P) cudaStreamSynchronize(P->stream);  // the copies from the staging are done
  tw_patch_destroy(P);
  for (int d = 0; d < 2; d++) {
    free(hbp[d]);
    free(hoff[d]);
    free(htwo[d]);
  }
  free(hpack);
  return rc;
}

extern "C" int tw_patch_info(const tw_patch *P, int64_t *info) {
  if (!P || !info) {
    set_error("tw_patch_info: NULL argument");
    return TW_EINVAL;
  }
  info[0] = P->d[0].n;
  info[1] = P->d[1].n;
  info[2] = P->d[0].nel;
  info[3] = P->d[1].nel;
  info[4] = P->d[0].nq;
  info[5] = P->d[1].nq;
  info[6] = P->n_rows;
  info[7] = P->nnz;
  info[8] = P->ncut;
  info[9] = P->ncutfns;
  info[10] = P->ncutpts;
  info[11] = P->ndwqrows;
  info[12] = P->ndisc[0] + P->ndisc[1];
  info[13] = P->n_interior;
  info[14] = P->p;
  info[15] = P->method;
  return TW_OK;
}

extern "C" int tw_form_mass(tw_patch *P, int precision, int64_t *row_ptr, int32_t *col, void *val,
                            void *stream) {
  if (!P || !row_ptr || (P->nnz > 0 && (!col || !val))) {
    set_error("tw_form_mass: NULL argument");
    return TW_EINVAL;
  }
  if (precision != TW_PREC_FP64 && precision != TW_PREC_FP32 && precision != TW_PREC_FP32X2) {
    set_error("tw_form_mass: unknown precision %d", precision);
    return TW_EINVAL;
  }
  return form_mass_launch(P, precision, row_ptr, col, val, (cudaStream_t)stream);
}

extern "C" int tw_form_mass_rowsf(tw_patch *P, int precision, int64_t *row_ptr, int32_t *col,
                                  void *val, void *stream) {
  if (!P || !row_ptr || (P->nnz > 0 && (!col || !val))) {
    set_error("tw_form_mass_rowsf: NULL argument");
    return TW_EINVAL;
  }
  if (precision != TW_PREC_FP64 && precision != TW_PREC_FP32 && precision != TW_PREC_FP32X2) {
    set_error("tw_form_mass_rowsf: unknown precision %d", precision);
    return TW_EINVAL;
  }
  return form_mass_launch(P, precision, row_ptr, col, val, (cudaStream_t)stream, true);
}

extern "C" int tw_states(const tw_patch *P, uint8_t *estate, uint8_t *fstate, int32_t *act,
                         void *stream) {
  if (!P) {
    set_error("tw_states: NULL patch");
    return TW_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int64_t ne = (int64_t)P->d[0].nel * P->d[1].nel, nf = (int64_t)P->d[0].n * P->d[1].n;
  if (estate) cudaMemcpyAsync(estate, P->estate, ne, cudaMemcpyDeviceToDevice, s);
  if (fstate) cudaMemcpyAsync(fstate, P->fstate, nf, cudaMemcpyDeviceToDevice, s);
  if (act) cudaMemcpyAsync(act, P->act, nf * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  return check_cuda(cudaGetLastError(), "tw_states");
}

extern "C" int tw_patch_table(const tw_patch *P, int which, void *dst, int64_t cap, int64_t *count,
                              void *stream) {
  if (!P) {
    set_error("tw_patch_table: NULL patch");
    return TW_EINVAL;
  }
  const void *src = nullptr;
  int64_t n = 0;
  size_t es = sizeof(double);
  int p1 = P->p + 1;
  switch (which) {
    case 0: case 1: src = P->d[which].xq; n = P->d[which].nq; break;
    case 2: case 3: src = P->d[which - 2].W; n = (int64_t)P->d[which - 2].n * P->d[which - 2].qmax; break;
    case 4: src = P->C; n = (int64_t)P->d[0].nq * P->d[1].nq; break;
    case 5: src = P->cut_pts; n = 3 * P->ncutpts; break;
    case 6: src = P->cut_off; n = P->ncut + 1; es = sizeof(int64_t); break;
    case 7: src = P->cut_list; n = P->ncut; es = sizeof(int32_t); break;
    case 8: src = P->choice; n = 4 * (int64_t)P->d[0].n * P->d[1].n; es = sizeof(int32_t); break;
    case 9: src = P->d[0].gx; n = p1; break;
    case 10: src = P->d[0].gw; n = p1; break;
    case 11: case 12: src = P->d[which - 11].Bq; n = (int64_t)P->d[which - 11].nq * p1; break;
    case 13: case 14: src = P->d[which - 13].GB; n = (int64_t)P->d[which - 13].nel * p1 * p1; break;
    case 15: case 16: src = P->d[which - 15].U; n = P->d[which - 15].nk; break;
    default:
      set_error("tw_patch_table: unknown table %d", which);
      return TW_EINVAL;
  }
  if (count) *count = n;
  if (!dst) return TW_OK;
  if (cap < n) {
    set_error("tw_patch_table: capacity %lld < %lld", (long long)cap, (long long)n);
    return TW_EINVAL;
  }
  if (n > 0)
    cudaMemcpyAsync(dst, src, es * n, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  return check_cuda(cudaGetLastError(), "tw_patch_table");
}

extern "C" int tw_rhs(tw_patch *P, const tw_func *f, double *b, void *stream) {
  if (!P || !f || !b) {
    set_error("tw_rhs: NULL argument");
    return TW_EINVAL;
  }
  return rhs_launch(P, f, b, (cudaStream_t)stream);
}

extern "C" int tw_rhs_points(tw_patch *P, int64_t *npts, double *xi, double *x, void *stream) {
  if (!P || !npts) {
    set_error("tw_rhs_points: NULL argument");
    return TW_EINVAL;
  }
  return rhs_points_run(P, npts, xi, x, (cudaStream_t)stream);
}

extern "C" int tw_rhs_values(tw_patch *P, const double *fvals, double *b, void *stream) {
  if (!P || !b || (!fvals && (int64_t)P->d[0].nq * P->d[1].nq > 0)) {
    set_error("tw_rhs_values: NULL argument");
    return TW_EINVAL;
  }
  return rhs_values_run(P, fvals, b, (cudaStream_t)stream);
}

extern "C" int tw_l2_project(tw_patch *P, const tw_func *f, const int64_t *row_ptr,
                             const int32_t *col, const double *val, double *u, double tol,
                             int maxit, int *iters, double *relres, void *stream) {
  if (!P || !f || !row_ptr || !col || !val || !u) {
    set_error("tw_l2_project: NULL argument");
    return TW_EINVAL;
  }
  if (!(tol > 0) || maxit < 0) {
    set_error("tw_l2_project: need tol > 0 and maxit >= 0");
    return TW_EINVAL;
  }
  return l2_project_run(P, f, row_ptr, col, val, u, tol, maxit, iters, relres,
                        (cudaStream_t)stream);
}

extern "C" int tw_loss(tw_patch *P, const tw_func *g, const double *u, double *loss,
                       double *dLdu, void *stream) {
  if (!P || !g || !u || !loss || (!dLdu && P->n_rows > 0)) {
    set_error("tw_loss: NULL argument");
    return TW_EINVAL;
  }
  return loss_run(P, g, u, loss, dLdu, (cudaStream_t)stream);
}

extern "C" int tw_l2_project_adjoint(tw_patch *P, const tw_func *f, const int64_t *row_ptr,
                                     const int32_t *col, const double *val, const double *dLdu,
                                     const double *u, double *lam, double *grad, double tol,
                                     int maxit, int *iters, double *relres, void *stream) {
  if (!P || !f || !row_ptr || !col || !val || !dLdu || !u || !lam || !grad) {
    set_error("tw_l2_project_adjoint: NULL argument");
    return TW_EINVAL;
  }
  if (P->geo.coef_kind != TW_COEF_DENSITY) {
    set_error("tw_l2_project_adjoint: the patch has no density spline (TW_COEF_DENSITY)");
    return TW_EINVAL;
  }
  if (!(tol > 0) || maxit < 0) {
    set_error("tw_l2_project_adjoint: need tol > 0 and maxit >= 0");
    return TW_EINVAL;
  }
  return adjoint_run(P, f, row_ptr, col, val, dLdu, u, lam, grad, tol, maxit, iters, relres,
                     (cudaStream_t)stream);
}
