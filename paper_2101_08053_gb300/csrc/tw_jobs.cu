// tw_jobs.cu -- many patches at once from native host threads (tw_run_jobs).
//
// Creating a patch is a chain of set-up kernels with a few host
// synchronisations (sizes read back between stages), so one host thread
// creating one patch leaves most of the GPU idle; patches are independent, and
// the GPU overlaps the chains of several patches on their own streams.  The
// jobs are taken by a persistent pool of host threads (grown on demand, kept
// until the process exits) so that a batch of patches costs no thread start-up
// and runs no interpreter code between its calls.  The calling thread works on
// jobs too.  The paper forms one patch at a time; this is scheduling only.
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <string>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "tw_internal.cuh"

namespace tw {

namespace {

#define TW_POOL_MAX_THREADS 64

// A batch is run by the calling thread and up to want - 1 helpers.  Helpers
// join a batch only under the lock and only while it accepts helpers; the
// batch stops accepting them before run() returns, and run() returns once every
// task has finished and no helper is inside the batch.
class JobPool {
 public:
  ~JobPool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto &t : threads_) t.join();
  }

  void run(int want, int n, const std::function<void(int)> &body) {
    std::lock_guard<std::mutex> serial(run_mu_);  // one batch at a time
    const int helpers = std::max(0, std::min(want, TW_POOL_MAX_THREADS) - 1);
    {
      std::lock_guard<std::mutex> lk(mu_);
      while ((int)threads_.size() < helpers) threads_.emplace_back([this] { loop(); });
      body_ = &body;
      n_ = n;
      next_.store(0);
      done_ = 0;
      open_ = helpers;
      gen_++;
    }
    cv_.notify_all();
    work();
    std::unique_lock<std::mutex> lk(mu_);
    open_ = 0;  // late helpers do not join this batch
    done_cv_.wait(lk, [this] { return done_ == n_ && inside_ == 0; });
    body_ = nullptr;
  }

 private:
  void loop() {
    int64_t seen = 0;
    std::unique_lock<std::mutex> lk(mu_);
    for (;;) {
      cv_.wait(lk, [&] { return stop_ || (gen_ != seen && open_ > 0); });
      if (stop_) return;
      seen = gen_;
      open_--;
      inside_++;
      lk.unlock();
      work();
      lk.lock();
      inside_--;
      if (done_ == n_ && inside_ == 0) done_cv_.notify_all();
    }
  }

  void work() {
    for (;;) {
      const int k = next_.fetch_add(1);
      if (k >= n_) break;
      (*body_)(k);
      std::lock_guard<std::mutex> lk(mu_);
      done_++;
      if (done_ == n_ && inside_ == 0) done_cv_.notify_all();
    }
  }

  std::mutex run_mu_, mu_;
  std::condition_variable cv_, done_cv_;
  std::vector<std::thread> threads_;
  const std::function<void(int)> *body_ = nullptr;
  std::atomic<int> next_{0};
  int n_ = 0, done_ = 0, open_ = 0, inside_ = 0;
  int64_t gen_ = 0;
  bool stop_ = false;
};

JobPool &pool() {
  static JobPool p;
  return p;
}

}  // namespace

}  // namespace tw

using namespace tw;

extern "C" int tw_run_jobs(tw_job *jobs, int n, int nthreads) {
  if (n < 0 || (n > 0 && !jobs)) {
    set_error("tw_run_jobs: bad job list");
    return TW_EINVAL;
  }
  if (n == 0) return TW_OK;
  for (int k = 0; k < n; k++) {
    jobs[k].patch = nullptr;
    jobs[k].status = TW_OK;
    if (!jobs[k].desc) {
      set_error("tw_run_jobs: job %d has no descriptor", k);
      return TW_EINVAL;
    }
  }
  int dev = 0;
  if (check_cuda(cudaGetDevice(&dev), "tw_run_jobs: cudaGetDevice")) return TW_ECUDA;
  int want = nthreads > 0 ? nthreads : (int)std::thread::hardware_concurrency();
  want = std::max(1, std::min(want, n));
  std::vector<std::string> msg(n);
  auto body = [&](int k) {
    tw_job &J = jobs[k];
    cudaSetDevice(dev);
    tw_patch *P = nullptr;
    int rc = tw_patch_create(J.desc, &P);
    if (rc == TW_OK && J.row_ptr) {
      if (P->n_rows > J.rows_capacity || P->nnz > J.nnz_capacity) {
        set_error("tw_run_jobs: CSR buffers hold %lld rows / %lld entries, the matrix has "
                  "%lld / %lld",
                  (long long)J.rows_capacity, (long long)J.nnz_capacity, (long long)P->n_rows,
                  (long long)P->nnz);
        rc = TW_EINVAL;
      } else {
        rc = tw_form_mass(P, J.precision, J.row_ptr, J.col, J.val, J.desc->stream);
      }
      // the result into host memory, ordered after the formation on the stream
      const size_t vb = J.precision == TW_PREC_FP32 ? sizeof(float) : sizeof(double);
      cudaStream_t st = (cudaStream_t)J.desc->stream;
      if (rc == TW_OK && J.h_row_ptr)
        rc = check_cuda(cudaMemcpyAsync(J.h_row_ptr, J.row_ptr, sizeof(int64_t) * (P->n_rows + 1),
                                        cudaMemcpyDeviceToHost, st),
                        "tw_run_jobs: row_ptr to host");
      if (rc == TW_OK && J.h_col && P->nnz > 0)
        rc = check_cuda(cudaMemcpyAsync(J.h_col, J.col, sizeof(int32_t) * P->nnz,
                                        cudaMemcpyDeviceToHost, st),
                        "tw_run_jobs: col to host");
      if (rc == TW_OK && J.h_val && P->nnz > 0)
        rc = check_cuda(cudaMemcpyAsync(J.h_val, J.val, vb * P->nnz, cudaMemcpyDeviceToHost, st),
                        "tw_run_jobs: val to host");
    }
    J.patch = P;
    J.status = rc;
    if (rc != TW_OK) msg[k] = tw_last_error();
  };
  pool().run(want, n, body);
  for (int k = 0; k < n; k++)
    if (jobs[k].status != TW_OK) {
      set_error("tw_run_jobs: job %d: %s", k, msg[k].c_str());
      return jobs[k].status;
    }
  return TW_OK;
}
