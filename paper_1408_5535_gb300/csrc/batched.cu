// Batched PHSVDS: many independent sparse matrices solved concurrently on one
// GPU (include/phsvds.h, phsvds_solve_batched).
//
// Each worker host thread owns a context (its own CUDA stream and pinned
// staging area) and takes matrices from a shared queue, largest first, so the
// long solves start early and the short ones fill the gaps.  Every solve is
// the full method of phsvds_solve, with its own SpMM plan picked by the
// autotuner for that matrix.  The solves of different workers overlap on the
// GPU: one solve's small kernels and its per-iteration host decisions leave
// most SMs idle, which the other solves' kernels use.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "kernels.h"
#include "phsvds.h"

extern "C" phsvds_status phsvds_solve_batched(phsvds_handle h, int count, const phsvds_csr* mats, int ptr_on_device,
                                              int k, phsvds_target target, double tol, phsvds_precond precond,
                                              const phsvds_opts* opts, int concurrency, phsvds_result* out) {
  if (!h || count < 0 || (count > 0 && (!mats || !out)) || concurrency < 0) return PHSVDS_ERR_INVALID;
  if (count == 0) return PHSVDS_OK;
  const int device = ph::handle_device(h);
  // device-resident inputs may still be written by work queued on h's stream
  if (cudaSetDevice(device) != cudaSuccess || cudaStreamSynchronize(ph::handle_stream(h)) != cudaSuccess)
    return PHSVDS_ERR_CUDA;
  for (int i = 0; i < count; ++i) {
    out[i].status = PHSVDS_ERR_INVALID;
    out[i].message[0] = '\0';
    std::memset(&out[i].stats, 0, sizeof(out[i].stats));
  }
  int workers = concurrency > 0 ? concurrency : std::min(count, 4);
  workers = std::max(1, std::min(workers, count));
  // largest work first: the stored entries are the cost of one product
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return mats[a].nnz > mats[b].nnz; });
  std::atomic<int> next{0};
  std::atomic<int> create_failed{0};
  auto work = [&]() {
    phsvds_handle wh = nullptr;
    const phsvds_status cs = phsvds_create(&wh, device, nullptr);
    if (cs != PHSVDS_OK) {
      create_failed.fetch_add(1);
      return;  // the remaining workers take this worker's share
    }
    int t;
    while ((t = next.fetch_add(1)) < count) {
      const int i = order[t];
      const phsvds_csr& a = mats[i];
      phsvds_result& r = out[i];
      r.status = phsvds_solve(wh, a.m, a.n, a.nnz, a.row_ptr, a.col_idx, a.val, ptr_on_device, k, target, tol,
                              precond, opts, r.sigma, r.U, r.V, r.resid, &r.stats);
      if (r.status != PHSVDS_OK) {
        std::strncpy(r.message, phsvds_last_error(wh), sizeof(r.message) - 1);
        r.message[sizeof(r.message) - 1] = '\0';
      }
    }
    phsvds_destroy(wh);
  };
  std::vector<std::thread> pool;
  pool.reserve(workers);
  for (int w = 0; w < workers; ++w) pool.emplace_back(work);
  for (auto& th : pool) th.join();
  if (create_failed.load() == workers) return PHSVDS_ERR_CUDA;
  phsvds_status first = PHSVDS_OK;
  for (int i = 0; i < count && first == PHSVDS_OK; ++i)
    if (out[i].status != PHSVDS_OK) first = out[i].status;
  return first;
}
