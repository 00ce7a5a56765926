// Ensembles of independent confined suspensions (the equilibrium-ensemble
// runs of Sec. V: many independent trajectories).  Each system is a grid
// object with its own workspaces and its own device-driven SEM-step graph
// (the whole step, restart cycles and refinement sweeps included, runs on
// the device without host round trips).  One SEM step of the whole ensemble
// launches every system's graph: systems are sorted by unknown count and
// dealt round-robin to a fixed number of worker streams (so each stream gets
// an even share of large and small systems), the workers' host threads
// launch in parallel, and the small kernels of different systems overlap on
// the GPU.  Then every stream is synchronised once.  In the one-graph form
// (rbfib_batch_set_one_graph) every system's step is instead captured as a
// branch of a single graph, and a batch step is that graph's one launch and
// one synchronisation.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
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
// The one-graph form (rbfib.cu): whether a grid's step can be captured now,
// staging a step's counters, and capturing every system's step as parallel
// branches of one graph.
bool rbfib_grid_step_ready(rbfib_grid* g, const rbfib_sem_params* p, const double* q, const double* quat);
void rbfib_grid_stage_step(rbfib_grid* g, uint64_t seed, uint64_t step, uint32_t attempt);
bool rbfib_batch_graph_build(rbfib_grid* const* gs, int n, const rbfib_sem_params* params, double* const* q,
                             double* const* quat, cudaStream_t s, cudaGraphExec_t* out);

struct rbfib_batch {
  int n = 0;
  int workers = 1;
  int device = 0;
  std::vector<cudaStream_t> streams;
  std::vector<rbfib_grid*> grids;
  std::vector<double> cost;   // seconds of each system's last step (0 = not yet run)
  std::string err;
  // one-graph form: every system's step as a branch of one graph, launched
  // once per batch step on gstream; rebuilt when a system's parameters or
  // configuration buffers change
  int one_graph = 0;
  cudaStream_t gstream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<rbfib_sem_params> gparams;
  std::vector<double*> gq, gquat;
  bool gfailed = false;        // the capture failed for the current key: not retried until it changes
  long long graph_steps = 0;   // batch steps run as one graph launch
};

namespace {

bool same_params(const rbfib_sem_params& a, const rbfib_sem_params& c) {
  return std::memcmp(&a, &c, sizeof(rbfib_sem_params)) == 0;
}

// One batch step as one graph launch; false (nothing launched) when some
// system's step cannot be captured yet (its first step builds the body
// block on the host) or the capture failed.
bool batch_graph_step(rbfib_batch* b, const rbfib_sem_params* params, const uint64_t* seeds, uint64_t step,
                      const uint32_t* attempts, double* const* q, double* const* quat, rbfib_step_info* infos,
                      int32_t* status, int& first) {
  // every system must be able to run device-driven now (a step that left a
  // coupled body block invalid sends the next one to the host path)
  for (int i = 0; i < b->n; ++i)
    if (!rbfib_grid_step_ready(b->grids[i], &params[i], q[i], quat[i])) return false;
  bool same_key = (b->gexec != nullptr || b->gfailed) && (int)b->gparams.size() == b->n;
  for (int i = 0; same_key && i < b->n; ++i)
    same_key = same_params(b->gparams[i], params[i]) && b->gq[i] == q[i] && b->gquat[i] == quat[i];
  if (same_key && b->gfailed) return false;
  if (!same_key) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    if (!b->gstream && cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking) != cudaSuccess) {
      b->gstream = nullptr;
      return false;
    }
    for (cudaStream_t s : b->streams)
      if (cudaStreamSynchronize(s) != cudaSuccess) return false;
    b->gparams.assign(params, params + b->n);
    b->gq.assign(q, q + b->n);
    b->gquat.assign(quat, quat + b->n);
    b->gfailed = !rbfib_batch_graph_build(b->grids.data(), b->n, params, q, quat, b->gstream, &b->gexec);
    if (b->gfailed) return false;
  }
  // work queued on the grids' own streams comes first
  for (cudaStream_t s : b->streams)
    if (cudaStreamSynchronize(s) != cudaSuccess) return false;
  for (int i = 0; i < b->n; ++i) rbfib_grid_stage_step(b->grids[i], seeds[i], step, attempts ? attempts[i] : 0u);
  if (cudaGraphLaunch(b->gexec, b->gstream) != cudaSuccess || cudaStreamSynchronize(b->gstream) != cudaSuccess) {
    first = RBFIB_ECUDA;
    for (int i = 0; i < b->n; ++i) status[i] = RBFIB_ECUDA;
    return true;
  }
  ++b->graph_steps;
  for (int i = 0; i < b->n; ++i) status[i] = rbfib_grid_step_finish(b->grids[i], infos ? &infos[i] : nullptr);
  first = RBFIB_OK;
  for (int i = 0; i < b->n; ++i)
    if (status[i] != RBFIB_OK && status[i] != RBFIB_EREJECT && first == RBFIB_OK) first = status[i];
  return true;
}

}  // namespace

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
  if (b->gstream) cudaStreamSynchronize(b->gstream);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->gstream) cudaStreamDestroy(b->gstream);
  for (rbfib_grid* g : b->grids) rbfib_destroy(g);
  for (cudaStream_t s : b->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  delete b;
}

int rbfib_batch_set_one_graph(rbfib_batch* b, int32_t on) {
  if (!b || (on != 0 && on != 1)) return RBFIB_EINVAL;
  b->one_graph = on;
  return RBFIB_OK;
}

int64_t rbfib_batch_graph_steps(const rbfib_batch* b) { return b ? b->graph_steps : -1; }

rbfib_grid* rbfib_batch_grid(rbfib_batch* b, int32_t sys) {
  if (!b || sys < 0 || sys >= b->n) return nullptr;
  return b->grids[sys];
}

int rbfib_batch_sem_step(rbfib_batch* b, const rbfib_sem_params* params, const uint64_t* seeds, uint64_t step,
                         const uint32_t* attempts, double* const* q, double* const* quat, rbfib_step_info* infos,
                         int32_t* status) {
  if (!b || !params || !seeds || !q || !quat || !status) return RBFIB_EINVAL;
  if (b->one_graph) {
    int first = RBFIB_OK;
    if (batch_graph_step(b, params, seeds, step, attempts, q, quat, infos, status, first)) return first;
  }
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
