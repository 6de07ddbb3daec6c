// Batched solve: many independent (N, beta, P) instances on one GPU.
//
// Instances are independent, so the batch is a task queue drained by a pool of
// host worker threads, each driving its own context on its own non-blocking
// CUDA stream; the GPU runs the workers' launch sequences concurrently (the
// per-row panel chains of small instances overlap with the updates of large
// ones).  Instances are taken largest first (longest-processing-time order by
// N^3 L^2, the analogue of the paper's work-balancing column assignment).
// Each worker inherits the options of the parent context (update path,
// Karatsuba levels, CUDA-graph capture of each factorisation, autotuned update
// schedules).
#include "hk.h"
#include "hk_internal.h"

#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

extern "C" int hk_batch_solve_impl(hk_ctx *parent, int device, const long long *opts, int count, const int *N,
                                   const int *bnum, const int *bden, const int *P, const hk_mp *const *moments,
                                   int iters, int nthreads, hk_mp *lambda_out, int *status_out, int *iters_out) {
  if (count < 0 || !N || !bnum || !bden || !P || !moments || !lambda_out || !status_out) return HK_ERR_ARG;
  for (int k = 0; k < count; k++)
    if (N[k] < 1 || P[k] < 32 || P[k] % 32 || !moments[k] || !lambda_out[k].limbs) return HK_ERR_ARG;
  if (count == 0) return HK_OK;
  (void)parent;
  // every instance reports its own outcome; one that no worker reaches keeps
  // this code
  for (int k = 0; k < count; k++) {
    status_out[k] = HK_ERR_CUDA;
    if (iters_out) iters_out[k] = 0;
  }
  std::vector<int> order(count);
  for (int k = 0; k < count; k++) order[k] = k;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    const double ca = (double)N[a] * N[a] * N[a] * (double)P[a] * P[a];
    const double cb = (double)N[b] * N[b] * N[b] * (double)P[b] * P[b];
    return ca > cb;
  });
  const int nw = std::max(1, std::min(nthreads, count));
  std::atomic<int> next(0);
  std::atomic<int> started(0);
  auto worker = [&]() {
    if (cudaSetDevice(device) != cudaSuccess) return;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return;
    hk_ctx *w = nullptr;
    if (hk_create(&w, device, s) != HK_OK) {
      cudaStreamDestroy(s);
      return;
    }
    started.fetch_add(1);
    for (int o = 0; o < 6; o++) hk_set_option(w, o, opts[o]);
    for (;;) {
      const int q = next.fetch_add(1);
      if (q >= count) break;
      const int k = order[q];
      int rc = hk_load_moments(w, N[k], bnum[k], bden[k], P[k], moments[k]);
      int bad = -1;
      if (rc == HK_OK) rc = hk_factor(w, &bad);
      int used = 0;
      if (rc == HK_OK) rc = hk_smallest_eig(w, iters, &lambda_out[k], &used);
      status_out[k] = rc;
      if (iters_out) {
        int64_t st[6] = {0};
        if (rc == HK_OK && iters == 0) hk_get_stats(w, st, 6);
        iters_out[k] = (rc == HK_OK && iters == 0 && !st[5]) ? -used : used;
      }
    }
    hk_destroy(w);
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nw; t++) pool.emplace_back(worker);
  for (auto &th : pool) th.join();
  // HK_ERR_CUDA only when no worker could start (then no instance ran); a
  // worker that failed to start leaves its share to the others
  return started.load() > 0 ? HK_OK : HK_ERR_CUDA;
}
