// Batched lambda paths: many independent fits (each Alg. 1 over a warm-started lambda path,
// Sec. 6.4) on one GPU.  Each fit is driven by glam_fit_path on its own plan, whose private
// stream carries all of its kernels and captured CUDA graphs; a pool of host worker threads takes
// the fits in index order, so the kernels of different fits run side by side on the device and
// one fit's host-side steps (graph launches, reads of the device stop flag) overlap the others'
// device work.
#include <algorithm>
#include <atomic>
#include <exception>
#include <string>
#include <thread>
#include <unordered_set>
#include <vector>

#include "glam_internal.cuh"

using namespace glam;

int glam_fit_path_batched(int nitems, glam_plan* const* plans, glam_batch_item* items,
                          const glam_opts* opts, int max_threads) {
  if (nitems < 0) return thread_fail(GLAM_EINVAL, "glam_fit_path_batched: nitems < 0");
  if (nitems == 0) return GLAM_OK;
  if (plans == nullptr || items == nullptr)
    return thread_fail(GLAM_EINVAL, "glam_fit_path_batched: NULL plans or items");
  {
    std::unordered_set<const glam_plan*> seen;
    for (int i = 0; i < nitems; ++i) {
      if (plans[i] == nullptr) return thread_fail(GLAM_EINVAL, "glam_fit_path_batched: NULL plan");
      if (!seen.insert(plans[i]).second)
        return thread_fail(GLAM_EINVAL, "glam_fit_path_batched: a plan appears twice");
    }
    for (int i = 0; i < nitems; ++i)
      if (plan_components(plans[i]) != 1)  // an item holds the three designs of one component
        return thread_fail(GLAM_EINVAL, "glam_fit_path_batched: plans with c > 1 components are not batched");
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess)
    return thread_fail(GLAM_ECUDA, "glam_fit_path_batched: cudaGetDevice failed");
  int nt = max_threads;
  if (nt <= 0) {
    const unsigned hc = std::thread::hardware_concurrency();
    nt = (int)std::min<unsigned>(hc == 0 ? 4u : hc, (unsigned)nitems);
  }
  nt = std::max(1, std::min(nt, nitems));
  std::atomic<int> next{0};
  auto worker = [&]() {
    cudaSetDevice(dev);  // the worker's calls go to the caller's device
    while (true) {
      const int i = next.fetch_add(1);
      if (i >= nitems) break;
      glam_batch_item& it = items[i];
      int nfit = 0;
      it.status = glam_fit_path(plans[i], it.X, it.Y, it.W, it.pen_w, it.nlambda, it.lambda, opts,
                                it.Theta0, it.Theta_path, it.stats, &nfit);
      it.nfit = nfit;
    }
  };
  if (nt == 1) {
    worker();
  } else {
    std::vector<std::thread> pool;
    try {
      pool.reserve(nt);
      for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
    } catch (const std::exception&) {
      // the system gave fewer threads than asked for (no exception may leave this C entry
      // point): the caller's thread takes fits too
      worker();
    }
    for (auto& th : pool) th.join();
  }
  for (int i = 0; i < nitems; ++i)
    if (items[i].status != GLAM_OK) return items[i].status;
  return GLAM_OK;
}
