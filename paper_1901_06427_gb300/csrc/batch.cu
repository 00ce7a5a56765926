// Ensembles of independent confined suspensions (the equilibrium-ensemble
// runs of Sec. V: many independent trajectories).  Each system is a grid
// object with its own workspaces and its own device-driven SEM-step graph
// (the whole step, restart cycles and refinement sweeps included, runs on
// the device without host round trips).  One SEM step of the whole ensemble
// launches every system's graph: systems are sorted by unknown count and
// dealt round-robin to a fixed number of worker streams (so each stream gets
// an even share of large and small systems), the workers' host threads
// launch in parallel, and the small kernels of different systems overlap on
// the GPU.  Then every stream is synchronised once.
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
// calls; launches a grid's device-driven SEM step without waiting (false:
// not available, run rbfib_sem_step instead) and, once its stream has been
// synchronised, returns the step's status and information.
void rbfib_grid_bind_stream(rbfib_grid* g, cudaStream_t s);
bool rbfib_grid_step_launch(rbfib_grid* g, const rbfib_sem_params* p, uint64_t seed, uint64_t step,
                            uint32_t attempt, double* q, double* quat);
int rbfib_grid_step_finish(rbfib_grid* g, rbfib_step_info* info);

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
  // largest systems first, dealt round-robin to the worker streams
  std::vector<double> key(b->n);
  for (int i = 0; i < b->n; ++i) {
    int64_t off[7] = {0, 0, 0, 0, 0, 0, 0};
    rbfib_saddle_layout(b->grids[i], off);
    key[i] = (double)off[6];
  }
  std::vector<int> order(b->n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return key[a] > key[c]; });
  // Worker w launches the device-driven step graphs of systems w, w + W, ...
  // of that order on its stream without waiting (a system whose graph is not
  // available runs its host-orchestrated step there and then); then every
  // stream is synchronised and the launched steps report.  A system's first
  // step captures its graph, which the workers do in parallel.
  std::vector<char> launched(b->n, 0);
  auto work = [&](int w) {
    cudaSetDevice(b->device);
    for (int t = w; t < b->n; t += b->workers) {
      const int i = order[t];
      rbfib_grid_bind_stream(b->grids[i], b->streams[w]);
      const auto t0 = std::chrono::steady_clock::now();
      const uint32_t att = attempts ? attempts[i] : 0u;
      if (rbfib_grid_step_launch(b->grids[i], &params[i], seeds[i], step, att, q[i], quat[i])) {
        launched[i] = 1;
      } else {
        status[i] = rbfib_sem_step(b->grids[i], &params[i], seeds[i], step, att, q[i], quat[i],
                                   infos ? &infos[i] : nullptr);
      }
      b->cost[i] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
  };
  std::vector<std::thread> th;
  for (int w = 1; w < b->workers; ++w) th.emplace_back(work, w);
  work(0);
  for (auto& t : th) t.join();
  for (cudaStream_t s : b->streams)
    if (cudaStreamSynchronize(s) != cudaSuccess) return RBFIB_ECUDA;
  for (int i = 0; i < b->n; ++i)
    if (launched[i]) status[i] = rbfib_grid_step_finish(b->grids[i], infos ? &infos[i] : nullptr);
  int first = RBFIB_OK;
  for (int i = 0; i < b->n; ++i)
    if (status[i] != RBFIB_OK && status[i] != RBFIB_EREJECT && first == RBFIB_OK) first = status[i];
  return first;
}

}  // extern "C"
