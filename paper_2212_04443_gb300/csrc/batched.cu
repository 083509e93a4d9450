// Many independent eigenproblems side by side: a pool of worker handles, each with its own
// stream, takes graphs largest-first and runs Algorithm 2 on each.  The GPU overlaps the
// workers' kernels; the per-iteration host decisions of one solve (locking, restarts) no
// longer leave the device idle, because another worker's kernels are queued meanwhile.
//
// Cooperative kernels of the workers are launched with one block: two multi-block
// cooperative grids from different streams could each end up partly resident, waiting on
// blocks that cannot start, whereas a one-block grid is either wholly resident or not
// started.  The batched problems are small (act_max <= a few tens), where one block suffices.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include <cstring>

#include "handle.cuh"

#define HCUDA(expr) BCHDAV_CUDA_OK(expr, h)

namespace {

bchdav_status make_worker(bchdav_handle parent, bchdav_handle* out) {
  *out = nullptr;
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaGetLastError();
    parent->set_error(BCHDAV_ERR_CUDA, std::string("worker stream: ") + cudaGetErrorString(e));
    return BCHDAV_ERR_CUDA;
  }
  bchdav_handle w = new bchdav_handle_s();
  w->stream = s;
  w->owns_stream = true;
  w->device = parent->device;
  w->sms = parent->sms;
  w->coop_grid_cap = 1;
  *out = w;
  return BCHDAV_OK;
}

}  // namespace

extern "C" {

bchdav_status bchdav_release_workspace(bchdav_handle h) {
  if (!h) return BCHDAV_ERR_ARG;
  HCUDA(cudaStreamSynchronize(h->stream));
  h->release_all();
  return BCHDAV_OK;
}

int64_t bchdav_launch_count(void) {
  return (int64_t)__atomic_load_n(&bchdav::g_launches, __ATOMIC_RELAXED);
}

bchdav_status bchdav_set_batch_workers(bchdav_handle h, int32_t n_workers) {
  if (!h || n_workers < 1 || n_workers > 64) return BCHDAV_ERR_ARG;
  h->batch_workers = n_workers;
  return BCHDAV_OK;
}

bchdav_status bchdav_solve_batched(bchdav_handle h, int32_t n_graphs, const bchdav_csr* As,
                                   const int32_t* k, const int32_t* b, const int32_t* m,
                                   const int32_t* act_max, double tol, const bchdav_opts* opts,
                                   double* const* evals, double* const* evecs,
                                   bchdav_info* infos, float* per_graph_ms) {
  if (!h) return BCHDAV_ERR_ARG;
  if (n_graphs < 0 || (n_graphs > 0 && (!As || !k || !b || !m || !evals || !evecs))) {
    h->set_error(BCHDAV_ERR_ARG, "solve_batched: missing per-graph arrays");
    return BCHDAV_ERR_ARG;
  }
  if (n_graphs == 0) return BCHDAV_OK;
  const int nw = std::min<int>(h->batch_workers, n_graphs);
  while ((int)h->workers.size() < nw) {
    bchdav_handle w = nullptr;
    BCHDAV_TRY(make_worker(h, &w));
    h->workers.push_back(w);
  }
  // inputs prepared on the caller's stream must be complete before other streams read them
  HCUDA(cudaStreamSynchronize(h->stream));

  // largest first (longest-processing-time order): work ~ nnz * b per filter step
  std::vector<int> order(n_graphs);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return (double)As[x].nnz * b[x] > (double)As[y].nnz * b[y];
  });
  bchdav_opts base;
  std::memset(&base, 0, sizeof(base));
  if (opts) base = *opts;
  base.v_init = nullptr;
  base.k_init = 0;
  base.ld_v_init = 0;

  std::atomic<int> next{0};
  std::vector<bchdav_status> st(n_graphs, BCHDAV_OK);
  std::mutex err_mu;
  std::string first_err;
  const int device = h->device;
  auto run = [&](bchdav_handle w) {
    cudaSetDevice(device);
    for (;;) {
      const int q = next.fetch_add(1);
      if (q >= n_graphs) break;
      const int i = order[q];
      bchdav_opts o = base;
      o.seed = base.seed + (uint64_t)i;
      bchdav_info inf;
      std::memset(&inf, 0, sizeof(inf));
      const auto t0 = std::chrono::steady_clock::now();
      bchdav_status s = bchdav_solve(w, &As[i], k[i], b[i], m[i], act_max ? act_max[i] : 0, tol,
                                     &o, evals[i], evecs[i], &inf);
      cudaError_t e = cudaStreamSynchronize(w->stream);
      const auto t1 = std::chrono::steady_clock::now();
      if (s == BCHDAV_OK && e != cudaSuccess) {
        s = BCHDAV_ERR_CUDA;
        w->set_error(s, std::string("batched solve: ") + cudaGetErrorString(e));
      }
      st[i] = s;
      inf.status = s;
      if (infos) infos[i] = inf;
      if (per_graph_ms)
        per_graph_ms[i] = (float)std::chrono::duration<double, std::milli>(t1 - t0).count();
      if (s < 0) {
        std::lock_guard<std::mutex> lk(err_mu);
        if (first_err.empty()) first_err = "graph " + std::to_string(i) + ": " + w->err;
      }
    }
  };
  std::vector<std::thread> threads;
  try {
    for (int t = 1; t < nw; ++t) threads.emplace_back(run, h->workers[t]);
  } catch (...) {
    // fewer threads than asked: the ones running (and this one) take all graphs
  }
  run(h->workers[0]);
  for (std::thread& t : threads) t.join();
  cudaSetDevice(device);

  bchdav_status worst = BCHDAV_OK;
  for (int i = 0; i < n_graphs; ++i) {
    if (st[i] < 0) {
      h->set_error(st[i], first_err);
      return st[i];
    }
    if (st[i] == BCHDAV_NOT_CONVERGED) worst = BCHDAV_NOT_CONVERGED;
  }
  return worst;
}

}  // extern "C"
