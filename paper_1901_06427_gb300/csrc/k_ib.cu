// Immersed-boundary and rigid-body kernels (Sec. III.B): body geometry,
// blob-to-cell binning, spreading S, interpolation J, the rigid maps K and
// K^T, the fused body rows of the saddle operator, the body-block
// preconditioner and the forces of Sec. V.
#include "common.cuh"
#include "kernels.cuh"

namespace rbfib {

static inline unsigned nblk(i64 n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ------------------------------------------------------------- geometry

__global__ void k_geometry(int nbl, const int* __restrict__ bob, const double* __restrict__ ref,
                           const double* __restrict__ q, const double* __restrict__ quat,
                           double* __restrict__ r, double* __restrict__ arm) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbl) return;
  const int p = bob[i];
  double R[9];
  quat_rot(quat + 4 * p, R);
  const double x = ref[3 * i], y = ref[3 * i + 1], z = ref[3 * i + 2];
  for (int a = 0; a < 3; ++a) {
    const double d = R[3 * a] * x + R[3 * a + 1] * y + R[3 * a + 2] * z;
    arm[3 * i + a] = d;
    r[3 * i + a] = q[3 * p + a] + d;
  }
}

void geometry(int nbl, const int* bob, const double* ref, const double* q, const double* quat,
              double* r, double* arm, cudaStream_t s) {
  if (nbl > 0) { launch_k(k_geometry, nblk(nbl, 128), 128, 0, s, nbl, bob, ref, q, quat, r, arm); note_launch(); }
}

// -------------------------------------------------------------- binning
__global__ void k_bin_keys(Dims d, int nbl, const double* __restrict__ r, int* __restrict__ key,
                           int* __restrict__ count) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbl) return;
  int c[3];
  for (int a = 0; a < 3; ++a) {
    int v = (int)floor(r[3 * i + a] / d.h[a]);
    if (d.per[a]) { v %= d.n[a]; if (v < 0) v += d.n[a]; }
    else { v = v < 0 ? 0 : (v > d.n[a] - 1 ? d.n[a] - 1 : v); }
    c[a] = v;
  }
  const int k = (int)flat3(d.n, c[0], c[1], c[2]);
  key[i] = k;
  atomicAdd(count + k, 1);
}

// exclusive scan, three phases
__global__ void k_scan_blocks(const int* __restrict__ in, int n, int* __restrict__ out, int* __restrict__ bsum) {
  pdl_entry();
  __shared__ int sh[1024];
  const int i = blockIdx.x * 1024 + threadIdx.x;
  int v = i < n ? in[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int t = (int)threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = sh[threadIdx.x] - v;
  if (threadIdx.x == 1023) bsum[blockIdx.x] = sh[1023];
}
__global__ void k_scan_sums(int* bsum, int nb) {
  pdl_entry();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int acc = 0;
    for (int b = 0; b < nb; ++b) { int v = bsum[b]; bsum[b] = acc; acc += v; }
  }
}
__global__ void k_scan_add(int* out, int n, const int* __restrict__ bsum) {
  pdl_entry();
  const int i = blockIdx.x * 1024 + threadIdx.x;
  if (i < n) out[i] += bsum[blockIdx.x];
}

__global__ void k_bin_scatter(int nbl, const int* __restrict__ key, const int* __restrict__ off,
                              int* __restrict__ fill, int* __restrict__ perm) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbl) return;
  const int k = key[i];
  perm[off[k] + atomicAdd(fill + k, 1)] = i;
}

// stable order inside each bin: insertion sort by blob id
__global__ void k_bin_sort(i64 nc, const int* __restrict__ off, int* __restrict__ perm) {
  pdl_entry();
  const i64 c = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int b = off[c], e = off[c + 1];
  for (int i = b + 1; i < e; ++i) {
    int v = perm[i], j = i - 1;
    while (j >= b && perm[j] > v) { perm[j + 1] = perm[j]; --j; }
    perm[j + 1] = v;
  }
}

// scratch: key (nbl), count (nc + 1), fill (nc), bsum (nc/1024 + 2)
void binning(const Dims& d, int nbl, const double* r, int* perm, int* off, int* key, int* count,
             int* fill, int* bsum, cudaStream_t s) {
  const i64 n1 = d.nc + 1;
  cudaMemsetAsync(count, 0, sizeof(int) * n1, s);
  cudaMemsetAsync(fill, 0, sizeof(int) * d.nc, s);
  if (nbl > 0) { launch_k(k_bin_keys, nblk(nbl, 128), 128, 0, s, d, nbl, r, key, count); note_launch(); }
  const int nb = (int)((n1 + 1023) / 1024);
  launch_k(k_scan_blocks, nb, 1024, 0, s, count, (int)n1, off, bsum);
  note_launch();
  launch_k(k_scan_sums, 1, 32, 0, s, bsum, nb);
  note_launch();
  launch_k(k_scan_add, nb, 1024, 0, s, off, (int)n1, bsum);
  note_launch();
  if (nbl > 0) {
    launch_k(k_bin_scatter, nblk(nbl, 128), 128, 0, s, nbl, key, off, fill, perm);
    note_launch();
    launch_k(k_bin_sort, nblk(d.nc, 256), 256, 0, s, d.nc, off, perm);
    note_launch();
  }
}

// ----------------------------------------------------- spread / interpolate
// Folded kw^3-point stencil of one blob and component.  For each point: flat
// face index (within component a), folded weight, and affine ghost weight
// (sum over folded tangential axes, in x,y,z order, of sign * 2 u_w).
struct Stencil27 {
  AxisStencil ax[3];
};

RBFIB_DEVFN void load_stencil(const Dims& d, int a, const double* x, Stencil27& S) {
  axis_stencil(d, a, 0, x[0], S.ax[0]);
  axis_stencil(d, a, 1, x[1], S.ax[1]);
  axis_stencil(d, a, 2, x[2], S.ax[2]);
}

template <typename T>
__global__ void k_spread(Dims d, int nbl, const int* __restrict__ perm, const double* __restrict__ r,
                         const T* __restrict__ lam, double scale, T* __restrict__ f) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * nbl) return;
  const int s = t / 3, a = t - 3 * s;
  const int i = perm ? perm[s] : s;
  const double val = (double)lam[3 * i + a] * scale;
  if (val == 0.0) return;
  Stencil27 S;
  load_stencil(d, a, r + 3 * i, S);
  T* fa = f + d.fo[a];
  const int kw = d.kw;
  for (int z = 0; z < kw; ++z) {
    if (!S.ax[2].keep[z]) continue;
    const double wz = S.ax[2].w[z] * S.ax[2].sgn[z];
    for (int y = 0; y < kw; ++y) {
      if (!S.ax[1].keep[y]) continue;
      const double wyz = wz * S.ax[1].w[y] * S.ax[1].sgn[y];
      for (int x = 0; x < kw; ++x) {
        if (!S.ax[0].keep[x]) continue;
        const double w = wyz * S.ax[0].w[x] * S.ax[0].sgn[x];
        atomicAdd(fa + flat3(d.fe[a], S.ax[0].idx[x], S.ax[1].idx[y], S.ax[2].idx[z]), (T)(w * val));
      }
    }
  }
}

// out[3i+a] = beta * out + alpha * (J v)_ia + gamma * (wall ghost part)_ia
template <typename T>
RBFIB_DEVFN void interp_one(const Dims& d, const Walls& wl, int a, const double* x, const T* __restrict__ v,
                            double& jv, double& aff) {
  Stencil27 S;
  load_stencil(d, a, x, S);
  const T* va = v + d.fo[a];
  jv = 0.0; aff = 0.0;
  const int kw = d.kw;
  for (int z = 0; z < kw; ++z) {
    if (!S.ax[2].keep[z]) continue;
    for (int y = 0; y < kw; ++y) {
      if (!S.ax[1].keep[y]) continue;
      for (int xx = 0; xx < kw; ++xx) {
        if (!S.ax[0].keep[xx]) continue;
        const int pt[3] = {xx, y, z};
        double w = 1.0, sg = 1.0, af = 0.0;
        for (int ax = 0; ax < 3; ++ax) {
          const AxisStencil& A = S.ax[ax];
          w *= A.w[pt[ax]];
          if (A.sgn[pt[ax]] < 0) {
            if (A.wall[pt[ax]] >= 0) af += sg * 2.0 * wl.v[A.wall[pt[ax]]][a];
            sg = -sg;
          }
        }
        if (v) jv += w * sg * (double)va[flat3(d.fe[a], S.ax[0].idx[xx], S.ax[1].idx[y], S.ax[2].idx[z])];
        aff += w * af;
      }
    }
  }
}

template <typename T>
__global__ void k_interp(Dims d, Walls wl, int nbl, const double* __restrict__ r, const T* __restrict__ v,
                         double alpha, double beta, double gamma, T* __restrict__ out) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * nbl) return;
  const int i = t / 3, a = t - 3 * i;
  double jv, aff;
  interp_one(d, wl, a, r + 3 * i, (alpha != 0.0) ? v : (const T*)nullptr, jv, aff);
  double o = alpha * jv + gamma * aff;
  if (beta != 0.0) o += beta * (double)out[t];
  out[t] = (T)o;
}

// -------------------------------------------- per-configuration stencil table
// Folded kernel weights of every blob and component, computed once per
// configuration (FP64 for the FP64 operators, FP32 for the preconditioner and
// the FP32 operators) so that every J / S application is a plain gather or
// scatter.
__global__ void k_stencil_build(Dims d, int nbl, const double* __restrict__ r, BlobStencil<double>* __restrict__ s64,
                                BlobStencil<float>* __restrict__ s32) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * nbl) return;
  const int i = t / 3, a = t - 3 * i;
  BlobStencil<double> S;
  BlobStencil<float> F;
  for (int ax = 0; ax < 3; ++ax) {
    AxisStencil A;
    axis_stencil(d, a, ax, r[3 * i + ax], A);
    for (int k = 0; k < kKMax; ++k) {
      const bool in = k < d.kw && A.keep[k];
      const double w = in ? A.w[k] * (double)A.sgn[k] : 0.0;
      S.idx[kKMax * ax + k] = in ? A.idx[k] : 0;
      S.w[kKMax * ax + k] = w;
      F.idx[kKMax * ax + k] = S.idx[kKMax * ax + k];
      F.w[kKMax * ax + k] = (float)w;
    }
  }
  s64[t] = S;
  s32[t] = F;
}

void stencil_build(const Dims& d, int nbl, const double* r, BlobStencil<double>* s64, BlobStencil<float>* s32,
                   cudaStream_t s) {
  if (nbl > 0) { launch_k(k_stencil_build, nblk(3 * (i64)nbl, 128), 128, 0, s, d, nbl, r, s64, s32); note_launch(); }
}

template <typename T> RBFIB_DEVFN const BlobStencil<T>* table_of(const BodyView& b);
template <> RBFIB_DEVFN const BlobStencil<double>* table_of<double>(const BodyView& b) { return b.st64; }
template <> RBFIB_DEVFN const BlobStencil<float>* table_of<float>(const BodyView& b) { return b.st32; }

// f_a += val * w at the kernel points, one atomic per point.
template <typename T>
RBFIB_DEVFN void warp_spread(const Dims& d, int a, const BlobStencil<T>* __restrict__ S, T val, T* __restrict__ f,
                             int lane) {
  if (val == T(0)) return;
  T* fa = f + d.fo[a];
  const int kw = d.kw, np = kw * kw * kw;
  for (int p = lane; p < np; p += 32) {
    const int x = p % kw, y = (p / kw) % kw, z = p / (kw * kw);
    const T w = S->w[x] * S->w[kKMax + y] * S->w[2 * kKMax + z];
    if (w != T(0)) atomicAdd(fa + flat3(d.fe[a], S->idx[x], S->idx[kKMax + y], S->idx[2 * kKMax + z]), w * val);
  }
}

// out = r_lam + J v  (body-block preconditioner input), warp per blob component
template <typename T>
__global__ void k_interp_res(Dims d, int nbl, const BlobStencil<T>* __restrict__ tab, const T* __restrict__ v,
                             const T* __restrict__ rl, T* __restrict__ out) {
  pdl_entry();
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (gw >= 3 * nbl) return;
  const T jv = warp_interp<T>(d, gw % 3, tab + gw, v, lane);
  if (lane == 0) out[gw] = rl[gw] + jv;
}

template <typename T>
void interp_res(const Dims& d, const BodyView& b, const T* v, const T* rl, T* out, cudaStream_t s) {
  if (b.nbl > 0) {
    const BlobStencil<T>* tab = nullptr;
    if constexpr (sizeof(T) == 8) tab = (const BlobStencil<T>*)b.st64; else tab = (const BlobStencil<T>*)b.st32;
    launch_k(k_interp_res<T>, nblk(32 * 3 * (i64)b.nbl, 128), 128, 0, s, d, b.nbl, tab, v, rl, out);
    note_launch();
  }
}

// out = alpha * J v + beta * out with the configuration's table
template <typename T>
__global__ void k_interp_tab(Dims d, int nbl, const BlobStencil<T>* __restrict__ tab, const T* __restrict__ v,
                             double alpha, double beta, T* __restrict__ out) {
  pdl_entry();
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (gw >= 3 * nbl) return;
  const T jv = warp_interp<T>(d, gw % 3, tab + gw, v, lane);
  if (lane == 0) {
    double o = alpha * (double)jv;
    if (beta != 0.0) o += beta * (double)out[gw];
    out[gw] = (T)o;
  }
}

void interp_tab(const Dims& d, const BodyView& b, const double* v, double alpha, double beta, double* out,
                cudaStream_t s) {
  if (b.nbl > 0) {
    launch_k(k_interp_tab<double>, nblk(32 * 3 * (i64)b.nbl, 128), 128, 0, s, d, b.nbl, b.st64, v, alpha, beta, out);
    note_launch();
  }
}

// f += scale * S-like scatter of lam with the configuration's table (no 1/dV)
__global__ void k_spread_tab(Dims d, int nbl, const int* __restrict__ perm, const BlobStencil<double>* __restrict__ tab,
                             const double* __restrict__ lam, double scale, double* __restrict__ f) {
  pdl_entry();
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (gw >= 3 * nbl) return;
  const int s = gw / 3, a = gw - 3 * s;
  const int i = perm ? perm[s] : s;
  warp_spread<double>(d, a, tab + 3 * i + a, lam[3 * i + a] * scale, f, lane);
}

void spread_tab(const Dims& d, const BodyView& b, const double* lam, double scale, double* f, cudaStream_t s) {
  if (b.nbl > 0) {
    launch_k(k_spread_tab, nblk(32 * 3 * (i64)b.nbl, 128), 128, 0, s, d, b.nbl, b.perm, b.st64, lam, scale, f);
    note_launch();
  }
}

// --------------------------------------------------- saddle body rows (fused)
// warps [0, 3 N_bl): y_lam = -J v + K U            (warp per blob component)
// warps [3 N_bl, 3 N_bl + N_b): y_U = K^T lam       (warp per body, FP64 sums)
// warps beyond: y_v -= S lam / dV                  (warp per blob component, bin order)
template <typename T>
__global__ void k_saddle_bodies(Dims d, BodyView b, const T* __restrict__ v, const T* __restrict__ lam,
                                const T* __restrict__ U, T* __restrict__ yv, T* __restrict__ ylam, T* __restrict__ yU,
                                double inv_dV) {
  pdl_entry();
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nA = 3 * b.nbl, nB = b.nb;
  const BlobStencil<T>* tab = table_of<T>(b);
  if (gw < nA) {
    const int i = gw / 3, a = gw - 3 * i;
    const T jv = warp_interp<T>(d, a, tab + gw, v, lane);
    if (lane == 0) {
      const int p = b.bob[i];
      const double* ar = b.arm + 3 * i;
      const double w0 = (double)U[6 * p + 3], w1 = (double)U[6 * p + 4], w2 = (double)U[6 * p + 5];
      double cr;
      if (a == 0) cr = w1 * ar[2] - w2 * ar[1];
      else if (a == 1) cr = w2 * ar[0] - w0 * ar[2];
      else cr = w0 * ar[1] - w1 * ar[0];
      ylam[gw] = (T)(-(double)jv + ((double)U[6 * p + a] + cr));
    }
  } else if (gw < nA + nB) {
    const int p = gw - nA;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int i = b.boff[p] + lane; i < b.boff[p + 1]; i += 32) {
      const double lx = (double)lam[3 * i], ly = (double)lam[3 * i + 1], lz = (double)lam[3 * i + 2];
      const double* ar = b.arm + 3 * i;
      acc[0] += lx; acc[1] += ly; acc[2] += lz;
      acc[3] += ar[1] * lz - ar[2] * ly;
      acc[4] += ar[2] * lx - ar[0] * lz;
      acc[5] += ar[0] * ly - ar[1] * lx;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c)
      for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    if (lane < 6) yU[6 * p + lane] = (T)acc[lane];
  } else if (gw < 2 * nA + nB) {
    const int s = gw - nA - nB;
    const int sb = s / 3, a = s - 3 * sb;
    const int i = b.perm ? b.perm[sb] : sb;
    warp_spread<T>(d, a, tab + 3 * i + a, (T)(-(double)lam[3 * i + a] * inv_dV), yv, lane);
  }
}

template <typename T>
void saddle_bodies(const Dims& d, const BodyView& b, const T* v, const T* lam, const T* U,
                   T* yv, T* ylam, T* yU, cudaStream_t s) {
  if (b.nbl == 0) return;
  const i64 warps = 2 * 3 * (i64)b.nbl + b.nb;
  const double inv_dV = 1.0 / (d.h[0] * d.h[1] * d.h[2]);
  launch_k(k_saddle_bodies<T>, nblk(32 * warps, 128), 128, 0, s, d, b, v, lam, U, yv, ylam, yU, inv_dV);
  note_launch();
}

template <typename T>
void spread(const Dims& d, int nbl, const int* perm, const double* r, const T* lam, double scale, T* f,
            cudaStream_t s) {
  if (nbl > 0) {
    launch_k(k_spread<T>, nblk(3 * (i64)nbl, 128), 128, 0, s,
             d, nbl, perm, r, lam, scale, f);
    note_launch();
  }
}

template <typename T>
void interp(const Dims& d, const Walls& wl, int nbl, const double* r, const T* v, double alpha,
            double beta, double gamma, T* out, cudaStream_t s) {
  if (nbl > 0) {
    launch_k(k_interp<T>, nblk(3 * (i64)nbl, 128), 128, 0, s,
             d, wl, nbl, r, v, alpha, beta, gamma, out);
    note_launch();
  }
}

// K^T lam per body (FP64): out = alpha * K^T lam + beta * out
template <typename T>
__global__ void k_kt(int nb, const int* __restrict__ boff, const double* __restrict__ arm,
                     const T* __restrict__ lam, double alpha, double beta, double* __restrict__ out) {
  pdl_entry();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nb) return;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int i = boff[warp] + lane; i < boff[warp + 1]; i += 32) {
    const double lx = (double)lam[3 * i], ly = (double)lam[3 * i + 1], lz = (double)lam[3 * i + 2];
    const double* ar = arm + 3 * i;
    acc[0] += lx; acc[1] += ly; acc[2] += lz;
    acc[3] += ar[1] * lz - ar[2] * ly;
    acc[4] += ar[2] * lx - ar[0] * lz;
    acc[5] += ar[0] * ly - ar[1] * lx;
  }
  for (int c = 0; c < 6; ++c)
    for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
  if (lane < 6) {
    double o = alpha * acc[lane];
    if (beta != 0.0) o += beta * out[6 * warp + lane];
    out[6 * warp + lane] = o;
  }
}

void kt_apply(int nb, const int* boff, const double* arm, const double* lam, double alpha, double beta,
              double* out, cudaStream_t s) {
  if (nb > 0) {
    launch_k(k_kt<double>, nblk(32 * (i64)nb, 128), 128, 0, s,
             nb, boff, arm, lam, alpha, beta, out);
    note_launch();
  }
}

// K U per blob: out = alpha * (u + w x arm) + beta * out
__global__ void k_k(int nbl, const int* __restrict__ bob, const double* __restrict__ arm,
                    const double* __restrict__ U, double alpha, double beta, double* __restrict__ out) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * nbl) return;
  const int i = t / 3, a = t - 3 * i;
  const int p = bob[i];
  const double* ar = arm + 3 * i;
  const double w0 = U[6 * p + 3], w1 = U[6 * p + 4], w2 = U[6 * p + 5];
  double cr;
  if (a == 0) cr = w1 * ar[2] - w2 * ar[1];
  else if (a == 1) cr = w2 * ar[0] - w0 * ar[2];
  else cr = w0 * ar[1] - w1 * ar[0];
  double o = alpha * (U[6 * p + a] + cr);
  if (beta != 0.0) o += beta * out[t];
  out[t] = o;
}

void k_apply(int nbl, const int* bob, const double* arm, const double* U, double alpha, double beta,
             double* out, cudaStream_t s) {
  if (nbl > 0) { launch_k(k_k, nblk(3 * (i64)nbl, 128), 128, 0, s, nbl, bob, arm, U, alpha, beta, out); note_launch(); }
}

// ------------------------------------------------ body-block preconditioner
// Per body p of shape s (body frame, rotated by R_p):
//   s'  = R^T (r_lam + J v~)                (input sres already holds r_lam + J v~)
//   U'  = N_s (R^T r_U + K_s^T M_s^-1 s')
//   lam' = M_s^-1 (K_s U' - s')
//   lam = R lam',  U = (R u', R w')
// M_s: free-space RPY blob mobility of the shape's reference blobs; N_s =
// (K_s^T M_s^-1 K_s)^-1; both precomputed on the host.
template <typename T>
__global__ void k_body_precond(int nb, const int* __restrict__ boff, const int* __restrict__ shape_of,
                               const i64* __restrict__ shape_minv_off, const T* __restrict__ minv,
                               const double* __restrict__ nmat, const int* __restrict__ shape_ref_blob,
                               const double* __restrict__ ref, const double* __restrict__ quat,
                               const T* __restrict__ sres, const T* __restrict__ rU,
                               T* __restrict__ zlam, T* __restrict__ zU, double* __restrict__ zlam64,
                               double* __restrict__ zU64) {
  pdl_entry();
  extern __shared__ unsigned char shraw[];
  T* sh = (T*)shraw;
  const int p = blockIdx.x;
  if (p >= nb) return;
  const int b0 = boff[p], nbp = boff[p + 1] - b0;
  const int n3 = 3 * nbp;
  const int s = shape_of[p];
  const T* Mi = minv + shape_minv_off[s];
  const double* Ns = nmat + 36 * s;
  const double* rf = ref + 3 * shape_ref_blob[s];
  T* sp = sh;            // n3: s'
  T* tp = sh + n3;       // n3: M^-1 s', later K U' - s'
  __shared__ double w6[6];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double R[9];
  quat_rot(quat + 4 * p, R);
  for (int i = threadIdx.x; i < nbp; i += blockDim.x) {
    const T* x = sres + 3 * (b0 + i);
    for (int a = 0; a < 3; ++a)
      sp[3 * i + a] = (T)(R[a] * (double)x[0] + R[3 + a] * (double)x[1] + R[6 + a] * (double)x[2]);
  }
  __syncthreads();
  // tp = M^-1 sp, one warp per row, lanes over columns (coalesced)
  for (int row = wid; row < n3; row += nw) {
    T acc = T(0);
    for (int c = lane; c < n3; c += 32) acc += Mi[(i64)row * n3 + c] * sp[c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) tp[row] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double f[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < nbp; ++i) {
      const double t0 = tp[3 * i], t1 = tp[3 * i + 1], t2 = tp[3 * i + 2];
      const double* a = rf + 3 * i;
      f[0] += t0; f[1] += t1; f[2] += t2;
      f[3] += a[1] * t2 - a[2] * t1;
      f[4] += a[2] * t0 - a[0] * t2;
      f[5] += a[0] * t1 - a[1] * t0;
    }
    double ru[6];
    for (int c = 0; c < 6; ++c) ru[c] = (double)rU[6 * p + c];
    for (int h = 0; h < 2; ++h)
      for (int a = 0; a < 3; ++a)
        f[3 * h + a] += R[a] * ru[3 * h] + R[3 + a] * ru[3 * h + 1] + R[6 + a] * ru[3 * h + 2];
    for (int r = 0; r < 6; ++r) {
      double acc = 0.0;
      for (int c = 0; c < 6; ++c) acc += Ns[6 * r + c] * f[c];
      w6[r] = acc;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nbp; i += blockDim.x) {
    const double* a = rf + 3 * i;
    const double kx = w6[0] + (w6[4] * a[2] - w6[5] * a[1]);
    const double ky = w6[1] + (w6[5] * a[0] - w6[3] * a[2]);
    const double kz = w6[2] + (w6[3] * a[1] - w6[4] * a[0]);
    tp[3 * i] = (T)kx - sp[3 * i];
    tp[3 * i + 1] = (T)ky - sp[3 * i + 1];
    tp[3 * i + 2] = (T)kz - sp[3 * i + 2];
  }
  __syncthreads();
  for (int row = wid; row < n3; row += nw) {
    T acc = T(0);
    for (int c = lane; c < n3; c += 32) acc += Mi[(i64)row * n3 + c] * tp[c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sp[row] = acc;   // lam' (s' no longer needed)
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nbp; i += blockDim.x) {
    const T* l = sp + 3 * i;
    for (int a = 0; a < 3; ++a) {
      const T x = (T)(R[3 * a] * (double)l[0] + R[3 * a + 1] * (double)l[1] + R[3 * a + 2] * (double)l[2]);
      zlam[3 * (b0 + i) + a] = x;
      if (zlam64) zlam64[3 * (b0 + i) + a] = (double)x;
    }
  }
  if (threadIdx.x < 6) {
    const int h = threadIdx.x / 3, a = threadIdx.x % 3;
    const T u = (T)(R[3 * a] * w6[3 * h] + R[3 * a + 1] * w6[3 * h + 1] + R[3 * a + 2] * w6[3 * h + 2]);
    zU[6 * p + threadIdx.x] = u;
    if (zU64) zU64[6 * p + threadIdx.x] = (double)u;
  }
}

template <typename T>
void body_precond(const BodyView& b, const PrecondView& pv, const T* sres, const T* rU, T* zlam, T* zU,
                  double* zlam64, double* zU64, cudaStream_t s) {
  if (b.nb == 0) return;
  const size_t shm = sizeof(T) * (2 * 3 * (size_t)pv.max_blobs + 8);
  const T* mi = nullptr;
  if constexpr (sizeof(T) == 8) mi = (const T*)pv.minv; else mi = (const T*)pv.minv32;
  launch_k(k_body_precond<T>, b.nb, 256, shm, s, b.nb, b.boff, pv.shape_of, pv.minv_off, mi, pv.nmat,
           pv.shape_ref_blob, b.ref, b.quat, sres, rU, zlam, zU, zlam64, zU64);
  note_launch();
}

// ------------------------------------------------------------------ forces
RBFIB_DEVFN double soft(double r, double phi0, double b, double dd) {
  return (phi0 / b) * (r < dd ? 1.0 : exp((dd - r) / b));
}

__global__ void k_forces(Dims d, Potentials P, int nb, const int* __restrict__ boff,
                         const double* __restrict__ q, const double* __restrict__ r,
                         const double* __restrict__ arm, const double* __restrict__ fext,
                         double* __restrict__ out) {
  pdl_entry();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nb) return;
  double F[6] = {0, 0, 0, 0, 0, 0};
  const double L[3] = {d.n[0] * d.h[0], d.n[1] * d.h[1], d.n[2] * d.h[2]};
  const double* qp = q + 3 * p;
  F[2] -= P.gravity;
  if (P.pair_phi0 != 0.0 || P.yuk_u0 != 0.0) {
    for (int o = 0; o < nb; ++o) {
      if (o == p) continue;
      double dv[3];
      for (int a = 0; a < 3; ++a) {
        double x = qp[a] - q[3 * o + a];
        if (d.per[a]) x -= L[a] * rint(x / L[a]);
        dv[a] = x;
      }
      const double rr = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
      double mag = 0.0;
      if (P.pair_phi0 != 0.0) mag += soft(rr, P.pair_phi0, P.pair_b, P.pair_d);
      if (P.yuk_u0 != 0.0)
        mag += P.yuk_u0 * P.yuk_dh * exp((P.yuk_dh - rr) / P.yuk_lambda) * (1.0 / (P.yuk_lambda * rr) + 1.0 / (rr * rr));
      for (int a = 0; a < 3; ++a) F[a] += mag * dv[a] / rr;
    }
  }
  if (P.wall_phi0 != 0.0) {
    for (int a = 0; a < 3; ++a) {
      if (d.per[a]) continue;
      F[a] += soft(qp[a], P.wall_phi0, P.wall_b, P.wall_d);
      F[a] -= soft(L[a] - qp[a], P.wall_phi0, P.wall_b, P.wall_d);
    }
  }
  if (P.bw_phi0 != 0.0 || P.blob_g != 0.0) {
    for (int i = boff[p]; i < boff[p + 1]; ++i) {
      double f[3] = {0, 0, -P.blob_g};
      if (P.bw_phi0 != 0.0)
        for (int a = 0; a < 3; ++a) {
          if (d.per[a]) continue;
          f[a] += soft(r[3 * i + a], P.bw_phi0, P.bw_b, P.bw_d);
          f[a] -= soft(L[a] - r[3 * i + a], P.bw_phi0, P.bw_b, P.bw_d);
        }
      const double* ar = arm + 3 * i;
      F[0] += f[0]; F[1] += f[1]; F[2] += f[2];
      F[3] += ar[1] * f[2] - ar[2] * f[1];
      F[4] += ar[2] * f[0] - ar[0] * f[2];
      F[5] += ar[0] * f[1] - ar[1] * f[0];
    }
  }
  if (P.sub_u0 != 0.0) {
    const double c = 4.0 * M_PI / (sqrt(3.0) * P.sub_s);
    const double k1[2] = {-c * sqrt(3.0) / 2.0, -0.5 * c}, k2[2] = {-c * sqrt(3.0) / 2.0, 0.5 * c};
    const double ks[3][2] = {{k1[0] - k2[0], k1[1] - k2[1]}, {k1[0], k1[1]}, {k2[0], k2[1]}};
    const double X[2] = {qp[0], qp[1] - L[1] / 2.0};
    double g[2] = {0, 0};
    for (int t = 0; t < 3; ++t) {
      const double sn = sin(X[0] * ks[t][0] + X[1] * ks[t][1]);
      g[0] += sn * ks[t][0];
      g[1] += sn * ks[t][1];
    }
    F[0] -= 0.5 * P.sub_u0 * g[0];
    F[1] -= 0.5 * P.sub_u0 * g[1];
  }
  for (int c = 0; c < 6; ++c) out[6 * p + c] = F[c] + (fext ? fext[6 * p + c] : 0.0);
}

void body_forces(const Dims& d, const Potentials& P, const BodyView& b, const double* fext, double* out,
                 cudaStream_t s) {
  if (b.nb > 0) {
    launch_k(k_forces, nblk(b.nb, 64), 64, 0, s,
             d, P, b.nb, b.boff, b.q, b.r, b.arm, fext, out);
    note_launch();
  }
}

// ----------------------------------------------------------- SEM helpers
RBFIB_DEVFN void quat_mul(const double* p, const double* q, double* o) {
  o[0] = p[0] * q[0] - p[1] * q[1] - p[2] * q[2] - p[3] * q[3];
  o[1] = p[0] * q[1] + p[1] * q[0] + p[2] * q[3] - p[3] * q[2];
  o[2] = p[0] * q[2] - p[1] * q[3] + p[2] * q[0] + p[3] * q[1];
  o[3] = p[0] * q[3] + p[1] * q[2] - p[2] * q[1] + p[3] * q[0];
}

// quat_out = normalise(q(phi) * quat), q(phi) = (cos |phi|/2, sin(|phi|/2) phi/|phi|)
RBFIB_DEVFN void rotate_quat(const double* quat, const double phi[3], double* out) {
  const double ang = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
  const double half = 0.5 * ang;
  const double s = ang > 0.0 ? sin(half) / ang : 0.5;
  const double dq[4] = {cos(half), s * phi[0], s * phi[1], s * phi[2]};
  double o[4];
  quat_mul(dq, quat, o);
  const double nrm = sqrt(o[0] * o[0] + o[1] * o[1] + o[2] * o[2] + o[3] * o[3]);
  for (int c = 0; c < 4; ++c) out[c] = o[c] / nrm;
}

// W^FT = kT [W^f / L_p ; W^tau]
__global__ void k_wft(int nb, const double* __restrict__ wn, const double* __restrict__ Lp, double kT,
                      double* __restrict__ wft) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 6 * nb) return;
  const int p = t / 6, c = t % 6;
  wft[t] = c < 3 ? kT * wn[t] / Lp[p] : kT * wn[t];
}

void wft(int nb, const double* wn, const double* Lp, double kT, double* out, cudaStream_t s) {
  if (nb > 0) { launch_k(k_wft, nblk(6 * (i64)nb, 128), 128, 0, s, nb, wn, Lp, kT, out); note_launch(); }
}

// q' = q + a * (scale_t L_p W^f)  or  q' = q + a * U_trans;  quat' = Rotate(quat, a * W^tau | a * w)
__global__ void k_move(int nb, const double* __restrict__ q, const double* __restrict__ quat,
                       const double* __restrict__ vec6, const double* __restrict__ Lp, double a,
                       double* __restrict__ qo, double* __restrict__ quato) {
  pdl_entry();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nb) return;
  const double lp = Lp ? Lp[p] : 1.0;
  for (int c = 0; c < 3; ++c) qo[3 * p + c] = q[3 * p + c] + (a * lp) * vec6[6 * p + c];
  const double phi[3] = {a * vec6[6 * p + 3], a * vec6[6 * p + 4], a * vec6[6 * p + 5]};
  rotate_quat(quat + 4 * p, phi, quato + 4 * p);
}

void move_bodies(int nb, const double* q, const double* quat, const double* vec6, const double* Lp, double a,
                 double* qo, double* quato, cudaStream_t s) {
  if (nb > 0) { launch_k(k_move, nblk(nb, 64), 64, 0, s, nb, q, quat, vec6, Lp, a, qo, quato); note_launch(); }
}

__global__ void k_outside(Dims d, int nbl, const double* __restrict__ r, int* __restrict__ flag) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbl) return;
  for (int a = 0; a < 3; ++a) {
    if (d.per[a]) continue;
    const double x = r[3 * i + a];
    if (!(x >= 0.0 && x <= d.n[a] * d.h[a])) atomicOr(flag, 1);
  }
}

// End of a device-driven SEM step: (q, quat) take the new configuration
// unless a blob left the domain (flag) or a status word is nonzero (a
// failed solve or body-block set-up); rejected[0] records the rejection.
__global__ void k_accept(int nb, const int* __restrict__ flag, const int* __restrict__ st, int nst, int st_stride,
                         const double* __restrict__ qn, const double* __restrict__ quatn, double* __restrict__ q,
                         double* __restrict__ quat, int* __restrict__ rejected) {
  pdl_entry();
  bool ok = flag[0] == 0;
  for (int i = 0; i < nst; ++i) ok = ok && st[i * st_stride] == 0;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) rejected[0] = flag[0] != 0 ? 1 : 0;
  if (!ok) return;
  for (int i = t; i < 3 * nb; i += gridDim.x * blockDim.x) q[i] = qn[i];
  for (int i = t; i < 4 * nb; i += gridDim.x * blockDim.x) quat[i] = quatn[i];
}
void accept_step(int nb, const int* flag, const int* st, int nst, int st_stride, const double* qn,
                 const double* quatn, double* q, double* quat, int* rejected, cudaStream_t s) {
  launch_k(k_accept, 1, 128, 0, s, nb, flag, st, nst, st_stride, qn, quatn, q, quat, rejected);
  note_launch();
}

void outside_check(const Dims& d, int nbl, const double* r, int* flag, cudaStream_t s) {
  if (nbl > 0) { launch_k(k_outside, nblk(nbl, 128), 128, 0, s, d, nbl, r, flag); note_launch(); }
}

#define INST(T)                                                                                          \
  template void saddle_bodies<T>(const Dims&, const BodyView&, const T*, const T*, const T*, T*, T*, T*, \
                                 cudaStream_t);                                                          \
  template void spread<T>(const Dims&, int, const int*, const double*, const T*, double, T*, cudaStream_t); \
  template void interp<T>(const Dims&, const Walls&, int, const double*, const T*, double, double, double, \
                          T*, cudaStream_t);                                                             \
  template void body_precond<T>(const BodyView&, const PrecondView&, const T*, const T*, T*, T*, double*, double*,        \
                                cudaStream_t);                                                          \
  template void interp_res<T>(const Dims&, const BodyView&, const T*, const T*, T*, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace rbfib

namespace rbfib {

// ------------------------------------------------------------------ adjoint
// arm_i = r_i - q_p for blob positions given as independent inputs
__global__ void k_arms_from_positions(int nbl, const int* __restrict__ bob, const double* __restrict__ r,
                                      const double* __restrict__ q, double* __restrict__ arm) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * nbl) return;
  arm[t] = r[t] - q[3 * bob[t / 3] + t % 3];
}

void arms_from_positions(int nbl, const int* bob, const double* r, const double* q, double* arm, cudaStream_t s) {
  if (nbl > 0) {
    launch_k(k_arms_from_positions, nblk(3 * (i64)nbl, 128), 128, 0, s,
             nbl, bob, r, q, arm);
    note_launch();
  }
}

// dL/dr_i = sum_a lam_ia D(zv)_ia + sum_a zl_ia D(v)_ia - zl_i x w_p - lam_i x tau_p,
// D(f)_ia,b = sum over the 27 folded kernel points of d w_a / d r_b * f_a.
// One warp per blob; lanes over kernel points; FP64; deterministic.
__global__ void k_adjoint_positions(Dims d, int nbl, const int* __restrict__ bob, const double* __restrict__ r,
                                    const double* __restrict__ v, const double* __restrict__ lam,
                                    const double* __restrict__ U, const double* __restrict__ zv,
                                    const double* __restrict__ zl, const double* __restrict__ zU,
                                    double* __restrict__ dr) {
  pdl_entry();
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= nbl) return;
  double g[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < 3; ++a) {
    AxisStencil S[3];
    axis_stencil(d, a, 0, r[3 * i], S[0]);
    axis_stencil(d, a, 1, r[3 * i + 1], S[1]);
    axis_stencil(d, a, 2, r[3 * i + 2], S[2]);
    double A[3] = {0.0, 0.0, 0.0}, Bv[3] = {0.0, 0.0, 0.0};
    const int kw = d.kw, np = kw * kw * kw;
    for (int q = lane; q < np; q += 32) {
      const int pt[3] = {q % kw, (q / kw) % kw, q / (kw * kw)};
      bool keep = true;
      double sg = 1.0;
      for (int ax = 0; ax < 3; ++ax) { keep = keep && S[ax].keep[pt[ax]]; sg *= (double)S[ax].sgn[pt[ax]]; }
      if (keep) {
        const i64 id = d.fo[a] + flat3(d.fe[a], S[0].idx[pt[0]], S[1].idx[pt[1]], S[2].idx[pt[2]]);
        const double fz = zv[id], fv = v[id];
        for (int b = 0; b < 3; ++b) {
          const int c1 = (b + 1) % 3, c2 = (b + 2) % 3;
          const double dw = S[b].dw[pt[b]] * S[c1].w[pt[c1]] * S[c2].w[pt[c2]] * sg;
          A[b] += dw * fz;
          Bv[b] += dw * fv;
        }
      }
    }
    for (int b = 0; b < 3; ++b)
      for (int o = 16; o > 0; o >>= 1) {
        A[b] += __shfl_xor_sync(0xffffffffu, A[b], o);
        Bv[b] += __shfl_xor_sync(0xffffffffu, Bv[b], o);
      }
    const double la = lam[3 * i + a], za = zl[3 * i + a];
    for (int b = 0; b < 3; ++b) g[b] += la * A[b] + za * Bv[b];
  }
  if (lane == 0) {
    const int p = bob[i];
    const double* w = U + 6 * p + 3;
    const double* tau = zU + 6 * p + 3;
    const double* z = zl + 3 * i;
    const double* l = lam + 3 * i;
    dr[3 * i + 0] = g[0] - (z[1] * w[2] - z[2] * w[1]) - (l[1] * tau[2] - l[2] * tau[1]);
    dr[3 * i + 1] = g[1] - (z[2] * w[0] - z[0] * w[2]) - (l[2] * tau[0] - l[0] * tau[2]);
    dr[3 * i + 2] = g[2] - (z[0] * w[1] - z[1] * w[0]) - (l[0] * tau[1] - l[1] * tau[0]);
  }
}

void adjoint_positions(const Dims& d, int nbl, const int* bob, const double* r, const double* v, const double* lam,
                       const double* U, const double* zv, const double* zl, const double* zU, double* dr,
                       cudaStream_t s) {
  if (nbl > 0) {
    launch_k(k_adjoint_positions, nblk(32 * (i64)nbl, 128), 128, 0, s, d, nbl, bob, r, v, lam, U, zv, zl, zU, dr);
    note_launch();
  }
}

}  // namespace rbfib
