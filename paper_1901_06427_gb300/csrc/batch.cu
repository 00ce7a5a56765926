// Ensembles of independent confined suspensions (the equilibrium-ensemble
// runs of Sec. V: many independent trajectories).  Each system is a grid
// object with its own workspaces.  One SEM step of the whole ensemble is a
// work queue: a fixed number of worker threads, each with its own stream,
// take the next system from a shared counter, rebind its grid to their
// stream and run its step, so the small kernels of different systems overlap
// on the GPU.  The queue is ordered longest first by each system's duration
// in the previous batch step (by its unknown count before the first), which
// keeps the workers evenly loaded over systems of uneven size.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rbfib.h"
#include "common.cuh"

// Defined with the grid (rbfib.cu): rebinds a grid to another stream between
// calls.
void rbfib_grid_bind_stream(rbfib_grid* g, cudaStream_t s);

struct rbfib_batch {
  int n = 0;
  int workers = 1;
  int device = 0;
  std::vector<cudaStream_t> streams;
  std::vector<rbfib_grid*> grids;
  std::vector<double> cost;   // seconds of each system's last step (0 = not yet run)
  std::string err;
};

extern "C" {

int rbfib_create_batch(int32_t n_sys, const rbfib_grid_desc* descs, int32_t n_workers, rbfib_batch** out) {
  if (!out || n_sys < 1 || !descs || n_workers < 1) return RBFIB_EINVAL;
  *out = nullptr;
  rbfib_batch* b = new rbfib_batch();
  b->n = n_sys;
  b->workers = n_workers < n_sys ? n_workers : n_sys;
  if (cudaGetDevice(&b->device) != cudaSuccess) { delete b; return RBFIB_ECUDA; }
  for (int w = 0; w < b->workers; ++w) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t t : b->streams) cudaStreamDestroy(t);
      delete b;
      return RBFIB_ECUDA;
    }
    b->streams.push_back(s);
  }
  b->grids.assign(n_sys, nullptr);
  b->cost.assign(n_sys, 0.0);
  for (int i = 0; i < n_sys; ++i) {
    const int st = rbfib_create_grid(&descs[i], b->streams[i % b->workers], &b->grids[i]);
    if (st != RBFIB_OK) {
      for (rbfib_grid* g : b->grids) rbfib_destroy(g);
      for (cudaStream_t t : b->streams) cudaStreamDestroy(t);
      delete b;
      return st;
    }
  }
  *out = b;
  return RBFIB_OK;
}

void rbfib_destroy_batch(rbfib_batch* b) {
  if (!b) return;
  for (rbfib_grid* g : b->grids) rbfib_destroy(g);
  for (cudaStream_t s : b->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  delete b;
}

rbfib_grid* rbfib_batch_grid(rbfib_batch* b, int32_t sys) {
  if (!b || sys < 0 || sys >= b->n) return nullptr;
  return b->grids[sys];
}

int rbfib_batch_sem_step(rbfib_batch* b, const rbfib_sem_params* params, const uint64_t* seeds, uint64_t step,
                         const uint32_t* attempts, double* const* q, double* const* quat, rbfib_step_info* infos,
                         int32_t* status) {
  if (!b || !params || !seeds || !q || !quat || !status) return RBFIB_EINVAL;
  // queue order: longest first; systems not yet timed by their unknown count
  std::vector<double> key(b->n);
  bool timed = true;
  for (int i = 0; i < b->n; ++i) timed = timed && b->cost[i] > 0.0;
  for (int i = 0; i < b->n; ++i) {
    if (timed) { key[i] = b->cost[i]; continue; }
    int64_t off[7] = {0, 0, 0, 0, 0, 0, 0};
    rbfib_saddle_layout(b->grids[i], off);
    key[i] = (double)off[6];
  }
  std::vector<int> order(b->n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return key[a] > key[c]; });
  std::atomic<int> next{0};
  auto work = [&](int w) {
    cudaSetDevice(b->device);
    for (int t = next.fetch_add(1); t < b->n; t = next.fetch_add(1)) {
      const int i = order[t];
      rbfib_grid_bind_stream(b->grids[i], b->streams[w]);
      const auto t0 = std::chrono::steady_clock::now();
      status[i] = rbfib_sem_step(b->grids[i], &params[i], seeds[i], step, attempts ? attempts[i] : 0u, q[i], quat[i],
                                 infos ? &infos[i] : nullptr);
      b->cost[i] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
  };
  std::vector<std::thread> th;
  for (int w = 1; w < b->workers; ++w) th.emplace_back(work, w);
  work(0);
  for (auto& t : th) t.join();
  int first = RBFIB_OK;
  for (int i = 0; i < b->n; ++i)
    if (status[i] != RBFIB_OK && status[i] != RBFIB_EREJECT && first == RBFIB_OK) first = status[i];
  return first;
}

}  // extern "C"
