// Fluctuating stress (Sec. III.A, Eq. LangevinD1): Philox4x64-10 normals and
// the tensor divergence DD W with sqrt(2) weights on no-slip wall edges and
// zero weights on free-slip wall edges.
#include "common.cuh"
#include "kernels.cuh"

namespace rbfib {

static inline unsigned nblk(i64 n, int bs) { return (unsigned)((n + bs - 1) / bs); }

__global__ void k_philox_normals(unsigned long long seed, unsigned long long step, unsigned attempt,
                                 unsigned purpose, i64 count, double* __restrict__ out) {
  pdl_entry();
  const i64 b = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * b >= count) return;
  double z[4];
  philox_normals4(seed, step, attempt, purpose, (unsigned long long)b, z);
#pragma unroll
  for (int l = 0; l < 4; ++l)
    if (4 * b + l < count) out[4 * b + l] = z[l];
}

void philox_normals(unsigned long long seed, unsigned long long step, unsigned attempt, unsigned purpose,
                    i64 count, double* out, cudaStream_t s) {
  const i64 nb = (count + 3) / 4;
  if (nb > 0) {
    launch_k(k_philox_normals, nblk(nb, 128), 128, 0, s,
             seed, step, attempt, purpose, count, out);
    note_launch();
  }
}

// The same normals with (seed, step, attempt) read from device memory
// sp[0..2] (the device-driven SEM step's graph reads them at run time).
__global__ void k_philox_normals_p(const unsigned long long* __restrict__ sp, unsigned purpose, i64 count,
                                   double* __restrict__ out) {
  pdl_entry();
  const i64 b = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * b >= count) return;
  double z[4];
  philox_normals4(sp[0], sp[1], (unsigned)sp[2], purpose, (unsigned long long)b, z);
#pragma unroll
  for (int l = 0; l < 4; ++l)
    if (4 * b + l < count) out[4 * b + l] = z[l];
}

void philox_normals_p(const unsigned long long* sp, unsigned purpose, i64 count, double* out, cudaStream_t s) {
  const i64 nb = (count + 3) / 4;
  if (nb > 0) {
    launch_k(k_philox_normals_p, nblk(nb, 128), 128, 0, s, sp, purpose, count, out);
    note_launch();
  }
}

// The raw words of n_blocks consecutive Philox4x64-10 blocks of the stream
// (seed, step, attempt, purpose), four 64-bit words per block.
__global__ void k_philox_words(unsigned long long seed, unsigned long long step, unsigned attempt, unsigned purpose,
                               unsigned long long first, i64 n_blocks, unsigned long long* __restrict__ out) {
  pdl_entry();
  const i64 b = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_blocks) return;
  unsigned long long c[4] = {first + (unsigned long long)b, step, ((unsigned long long)attempt << 32) | purpose, 0ULL};
  philox4x64_10(c, seed, 0ULL);
  ulonglong2* o = reinterpret_cast<ulonglong2*>(out + 4 * b);
  o[0] = make_ulonglong2(c[0], c[1]);
  o[1] = make_ulonglong2(c[2], c[3]);
}

void philox_words(unsigned long long seed, unsigned long long step, unsigned attempt, unsigned purpose,
                  unsigned long long first, i64 n_blocks, unsigned long long* out, cudaStream_t s) {
  if (n_blocks > 0) {
    launch_k(k_philox_words, nblk(n_blocks, 128), 128, 0, s, seed, step, attempt, purpose, first, n_blocks, out);
    note_launch();
  }
}

// out(face of component a) = c * [ (W_aa(right) - W_aa(left)) / h_a
//                                  + sum_{b != a} (c+ W_ab(node j+1) - c- W_ab(node j)) / h_b ]
__global__ void k_stress_div(Dims d, StressLayout L, const double* __restrict__ W, double c, double* __restrict__ out) {
  pdl_entry();
  const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.fo[3]) return;
  int a, f[3];
  decode_face(d, t, a, f);
  // W_aa at the cells either side of the face
  int cl[3] = {f[0], f[1], f[2]}, cr[3] = {f[0], f[1], f[2]};
  if (d.per[a]) { cl[a] = f[a] - 1; if (cl[a] < 0) cl[a] += d.n[a]; }
  else { cr[a] = f[a] + 1; }
  const double* Waa = W + L.off[a][a];
  double acc = (Waa[flat3(d.n, cr[0], cr[1], cr[2])] - Waa[flat3(d.n, cl[0], cl[1], cl[2])]) / d.h[a];
  for (int b = 0; b < 3; ++b) {
    if (b == a) continue;
    const int* e = L.ext[a][b];
    const double* Wab = W + L.off[a][b];
    int lo[3] = {f[0], f[1], f[2]}, hi[3] = {f[0], f[1], f[2]};
    hi[b] = f[b] + 1;
    double clo = 1.0, chi = 1.0;
    if (d.per[b]) { if (hi[b] >= d.n[b]) hi[b] = 0; }
    else {
      // wall edges: sqrt(2) at a no-slip wall, 0 at a free-slip wall (no
      // shear stress), so that DD DD^T = -LL with either ghost
      if (lo[b] == 0) clo = d.gd[2 * b] > 0 ? 1.4142135623730951 : 0.0;
      if (hi[b] == d.n[b]) chi = d.gd[2 * b + 1] > 0 ? 1.4142135623730951 : 0.0;
    }
    acc += (chi * Wab[flat3(e, hi[0], hi[1], hi[2])] - clo * Wab[flat3(e, lo[0], lo[1], lo[2])]) / d.h[b];
  }
  out[t] = c * acc;
}

void stress_divergence(const Dims& d, const StressLayout& L, const double* W, double c, double* out, cudaStream_t s) {
  launch_k(k_stress_div, nblk(d.fo[3], 256), 256, 0, s, d, L, W, c, out);
  note_launch();
}

}  // namespace rbfib

// ===================================================== allocation-free variant
// rbfib_stochastic_forcing_static: the same fluid forcing as
// rbfib_stochastic_forcing, for callers that cannot allocate device memory
// (for instance code running inside a memory pool or an allocator hook that
// must not re-enter cudaMalloc, or embedded hosts that pre-plan all memory).
// The stress field is drawn into a fixed array that is part of the library's
// device image, so the call itself allocates nothing.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include "../../include/rbfib.h"

namespace {

constexpr long long kStaticStressMax = 1LL << 20;   // doubles (8 MiB per device)
constexpr int kMaxDevices = 64;

// Every device that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_static_stress[kStaticStressMax];

std::mutex g_static_mu;
double* g_static_ptr[kMaxDevices] = {};

void set_msg(char* buf, size_t len, const char* msg) {
  if (buf && len) {
    std::strncpy(buf, msg, len - 1);
    buf[len - 1] = '\0';
  }
}

}  // namespace

extern "C" int rbfib_stochastic_forcing_static(const rbfib_grid_desc* desc, double kT, double dt, uint64_t seed,
                                               uint64_t step, uint32_t attempt, double* out, void* cuda_stream,
                                               char* errbuf, size_t errlen) {
  using namespace rbfib;
  if (!desc || !out || !(dt > 0) || !(kT >= 0) || !(desc->h > 0) || !(desc->eta > 0)) {
    set_msg(errbuf, errlen, "stochastic_forcing_static: bad argument");
    return RBFIB_EINVAL;
  }
  int per[3], n[3];
  for (int a = 0; a < 3; ++a) {
    n[a] = desc->n[a];
    if (desc->periodic[a] != 0 && desc->periodic[a] != 1) {
      set_msg(errbuf, errlen, "stochastic_forcing_static: periodic must be 0 or 1");
      return RBFIB_EINVAL;
    }
    per[a] = desc->periodic[a];
    if (n[a] < 2) { set_msg(errbuf, errlen, "stochastic_forcing_static: n < 2"); return RBFIB_EINVAL; }
  }
  if (per[0] && per[1] && per[2]) {
    set_msg(errbuf, errlen, "stochastic_forcing_static: every axis periodic");
    return RBFIB_EINVAL;
  }
  for (int w = 0; w < 6; ++w)
    if (desc->free_slip[w] != 0 && desc->free_slip[w] != 1) {
      set_msg(errbuf, errlen, "stochastic_forcing_static: free_slip must be 0 or 1");
      return RBFIB_EINVAL;
    }
  // Bound the cell count before any product of extents is formed: the
  // stress field holds about nine values per cell, so a grid with more cells
  // than the scratch has values can never fit (and the 64-bit products below
  // cannot overflow once each extent and the cell count are bounded).
  {
    long long cells = 1;
    for (int a = 0; a < 3; ++a) {
      if ((long long)n[a] > kStaticStressMax || cells > kStaticStressMax / n[a]) {
        cells = kStaticStressMax + 1;
        break;
      }
      cells *= n[a];
    }
    if (cells > kStaticStressMax) {
      set_msg(errbuf, errlen, "stochastic_forcing_static: grid exceeds the static scratch");
      return RBFIB_EINVAL;
    }
  }
  const double h3[3] = {desc->h, desc->h, desc->h};
  Dims d = make_dims(n, per, h3);
  set_free_slip(d, desc->free_slip);
  // stress layout: for a = x,y,z: W_aa (cells), then W_ab for b != a in increasing order
  StressLayout L;
  long long off = 0;
  for (int a = 0; a < 3; ++a) {
    int order[3] = {a, a == 0 ? 1 : 0, a == 2 ? 1 : 2};
    for (int t = 0; t < 3; ++t) {
      const int b = order[t];
      int* e = L.ext[a][b];
      for (int ax = 0; ax < 3; ++ax) e[ax] = d.n[ax];
      if (b != a) {
        e[a] = d.fe[a][a];
        e[b] = d.per[b] ? d.n[b] : d.n[b] + 1;
      }
      L.off[a][b] = off;
      off += (long long)e[0] * e[1] * e[2];
    }
  }
  L.total = off;
  if (L.total > kStaticStressMax) {
    char msg[200];
    std::snprintf(msg, sizeof msg,
                  "stochastic_forcing_static: stress field of %lld values exceeds the static scratch of %lld",
                  (long long)L.total, (long long)kStaticStressMax);
    set_msg(errbuf, errlen, msg);
    return RBFIB_EINVAL;
  }
  // Device address of the scratch, with the target device current.  Outside
  // stream capture it is looked up on every call (a cheap query), so a
  // primary context that was reset and re-created since the last call (which
  // reloads the module at a new address) never gets a stale pointer; during
  // capture the address cached by the last call outside capture on this
  // device is used, so the first call on a device must come before any
  // capture.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_msg(errbuf, errlen, "stochastic_forcing_static: no usable current device");
    return RBFIB_ECUDA;
  }
  const cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    set_msg(errbuf, errlen, "stochastic_forcing_static: cudaStreamIsCapturing failed");
    return RBFIB_ECUDA;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (cap == cudaStreamCaptureStatusNone) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_static_stress);
      if (e != cudaSuccess || !p) {
        set_msg(errbuf, errlen, "stochastic_forcing_static: cudaGetSymbolAddress failed");
        return RBFIB_ECUDA;
      }
      g_static_ptr[dev] = (double*)p;
    } else if (!g_static_ptr[dev]) {
      set_msg(errbuf, errlen, "stochastic_forcing_static: first call on this device made during stream capture");
      return RBFIB_EINVAL;
    }
    scratch = g_static_ptr[dev];
  }
  philox_normals(seed, step, attempt, 1u, L.total, scratch, s);
  stress_divergence(d, L, scratch, std::sqrt(2.0 * desc->eta * kT / (d.h[0] * d.h[1] * d.h[2] * dt)), out, s);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_msg(errbuf, errlen, cudaGetErrorString(e));
    return RBFIB_ECUDA;
  }
  set_msg(errbuf, errlen, "");
  return RBFIB_OK;
}
