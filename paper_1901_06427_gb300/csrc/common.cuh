// Shared device-side definitions: grid dimensions, index decoding, the
// three-point kernel and its wall folding.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

typedef long long i64;

// Dimensions of one (multigrid) level of the MAC grid.  Spacing may differ per
// axis on semi-coarsened levels.
struct Dims {
  int n[3];          // cells per axis
  int per[3];        // 1 = periodic axis
  double h[3];       // spacing per axis
  int fe[3][3];      // fe[a][ax]: extent of component a's unknown faces along ax
  i64 fo[4];         // offsets of the three face blocks; fo[3] = N_f
  i64 nc;            // N_c
  double ih[3], ih2[3];   // 1/h, 1/h^2 per axis (precomputed: no divisions in kernels)
  float ihf[3], ih2f[3];
  int kw;            // immersed-boundary kernel points per axis (3 or 6)
  // Walls -x, +x, -y, +y, -z, +z: change of the Laplacian's diagonal (in
  // units of 1/h^2) when a tangential velocity's neighbour lies beyond the
  // wall.  +1 at a no-slip wall (ghost = -self), -1 at a free-slip wall
  // (ghost = +self: zero tangential stress), 0 on periodic axes.
  int gd[6];
};

// Value of a tangential ghost beyond wall w in units of its mirror point:
// -1 (no-slip) or +1 (free-slip).
__host__ __device__ inline int ghost_sign(const Dims& d, int w) { return -d.gd[w]; }

template <typename T> __host__ __device__ inline T inv_h(const Dims& d, int ax);
template <> __host__ __device__ inline double inv_h<double>(const Dims& d, int ax) { return d.ih[ax]; }
template <> __host__ __device__ inline float inv_h<float>(const Dims& d, int ax) { return d.ihf[ax]; }
template <typename T> __host__ __device__ inline T inv_h2(const Dims& d, int ax);
template <> __host__ __device__ inline double inv_h2<double>(const Dims& d, int ax) { return d.ih2[ax]; }
template <> __host__ __device__ inline float inv_h2<float>(const Dims& d, int ax) { return d.ih2f[ax]; }

inline Dims make_dims(const int n[3], const int per[3], const double h[3]) {
  Dims d;
  for (int a = 0; a < 3; ++a) { d.n[a] = n[a]; d.per[a] = per[a]; d.h[a] = h[a]; }
  i64 off = 0;
  for (int a = 0; a < 3; ++a) {
    for (int ax = 0; ax < 3; ++ax) d.fe[a][ax] = n[ax];
    if (!per[a]) d.fe[a][a] = n[a] - 1;
    d.fo[a] = off;
    off += (i64)d.fe[a][0] * d.fe[a][1] * d.fe[a][2];
  }
  d.fo[3] = off;
  d.nc = (i64)n[0] * n[1] * n[2];
  d.kw = 3;
  for (int w = 0; w < 6; ++w) d.gd[w] = per[w / 2] ? 0 : 1;
  for (int a = 0; a < 3; ++a) {
    d.ih[a] = 1.0 / h[a];
    d.ih2[a] = 1.0 / (h[a] * h[a]);
    d.ihf[a] = (float)d.ih[a];
    d.ih2f[a] = (float)d.ih2[a];
  }
  return d;
}

// Marks free-slip walls (fs[w] != 0 for wall w on a bounded axis).
inline void set_free_slip(Dims& d, const int fs[6]) {
  for (int w = 0; w < 6; ++w)
    if (!d.per[w / 2]) d.gd[w] = fs[w] ? -1 : 1;
}

__host__ __device__ inline i64 flat3(const int e[3], int i, int j, int k) {
  return (i64)i + (i64)e[0] * ((i64)j + (i64)e[1] * k);
}

// Decode a global face index into (component, i, j, k).  Grids are limited
// to fewer than 2^31 unknowns, so the index arithmetic is 32-bit.
__device__ inline void decode_face(const Dims& d, i64 f, int& a, int c[3]) {
  a = (f >= d.fo[1]) + (f >= d.fo[2]);
  const unsigned l = (unsigned)(f - d.fo[a]);
  const unsigned e0 = d.fe[a][0], e1 = d.fe[a][1];
  const unsigned t = l / e0;
  c[0] = (int)(l - t * e0);
  c[2] = (int)(t / e1);
  c[1] = (int)(t - (unsigned)c[2] * e1);
}

__device__ inline void decode_cell(const Dims& d, i64 l64, int c[3]) {
  const unsigned l = (unsigned)l64;
  const unsigned e0 = d.n[0], e1 = d.n[1];
  const unsigned t = l / e0;
  c[0] = (int)(l - t * e0);
  c[2] = (int)(t / e1);
  c[1] = (int)(t - (unsigned)c[2] * e1);
}

// Points of one red-black colour ((i + j + k) % 2 == color) of the three face
// grids: thread t -> component, row (j, k) and i.  Returns false for the
// padding thread of an odd-length row.
struct ColorMap { unsigned cnt[3]; unsigned hx[3]; };

inline ColorMap make_color_map_faces(const Dims& d) {
  ColorMap m;
  for (int a = 0; a < 3; ++a) {
    m.hx[a] = (unsigned)(d.fe[a][0] + 1) / 2;
    m.cnt[a] = m.hx[a] * (unsigned)d.fe[a][1] * (unsigned)d.fe[a][2];
  }
  return m;
}
inline ColorMap make_color_map_cells(const Dims& d) {
  ColorMap m;
  m.hx[0] = (unsigned)(d.n[0] + 1) / 2;
  m.cnt[0] = m.hx[0] * (unsigned)d.n[1] * (unsigned)d.n[2];
  m.cnt[1] = m.cnt[2] = 0; m.hx[1] = m.hx[2] = 1;
  return m;
}

__device__ inline bool color_face(const Dims& d, const ColorMap& m, unsigned t, int color, int& a, int c[3]) {
  a = 0;
  if (t >= m.cnt[0]) { t -= m.cnt[0]; a = 1; if (t >= m.cnt[1]) { t -= m.cnt[1]; a = 2; } }
  if (t >= m.cnt[a]) return false;
  const unsigned hx = m.hx[a], e1 = d.fe[a][1];
  const unsigned row = t / hx;
  const unsigned mm = t - row * hx;
  c[2] = (int)(row / e1);
  c[1] = (int)(row - (unsigned)c[2] * e1);
  c[0] = (int)(2 * mm + ((c[1] + c[2] + color) & 1));
  return c[0] < d.fe[a][0];
}

__device__ inline bool color_cell(const Dims& d, const ColorMap& m, unsigned t, int color, int c[3]) {
  if (t >= m.cnt[0]) return false;
  const unsigned hx = m.hx[0], e1 = d.n[1];
  const unsigned row = t / hx;
  const unsigned mm = t - row * hx;
  c[2] = (int)(row / e1);
  c[1] = (int)(row - (unsigned)c[2] * e1);
  c[0] = (int)(2 * mm + ((c[1] + c[2] + color) & 1));
  return c[0] < d.n[0];
}

// Largest kernel width (points per axis).
constexpr int kKMax = 6;

// Per-configuration kernel stencil of one blob and velocity component:
// indices along x, y, z (kw each, at [kKMax * axis + t]) and the folded
// weights (sign included, zero for dropped points).
template <typename W>
struct BlobStencil {
  int idx[3 * kKMax];
  W w[3 * kKMax];
};

// Three-point Peskin kernel: the unique phi on |r| < 3/2 with partition of
// unity, zero first moment and sum of squares 1/2.
__device__ inline double phi3(double r) {
  r = fabs(r);
  if (r <= 0.5) return (1.0 + sqrt(1.0 - 3.0 * r * r)) / 3.0;
  if (r < 1.5) {
    double t = 1.0 - r;
    return (5.0 - 3.0 * r - sqrt(1.0 - 3.0 * t * t)) / 6.0;
  }
  return 0.0;
}

// phi'(r), odd in r.
__device__ inline double dphi3(double r) {
  double a = fabs(r), s = r < 0 ? -1.0 : 1.0;
  if (a <= 0.5) return s * (-a / sqrt(1.0 - 3.0 * a * a));
  if (a < 1.5) {
    double t = 1.0 - a;
    return s * ((-3.0 - 3.0 * t / sqrt(1.0 - 3.0 * t * t)) / 6.0);
  }
  return 0.0;
}

// Six-point kernel of three continuous derivatives (support |r| < 3): the
// six weights phi(r + 2 - t), t = 0..5, at a shift r in [0, 1), and their
// derivatives d/dr.  The weights are the solution of the kernel's defining
// conditions (even and odd sums 1/2, first and third moments 0, second
// moment K = 59/60 - sqrt(29)/20, sum of squares C = 5431/19200 +
// 51 sqrt(29)/6400): affine in the root t(r) = phi(r - 3) of
// 28 t^2 + beta(r) t + gamma(r) = 0 that vanishes at r = 0.
__device__ inline void six_weights(double r, double w[6], double dw[6]) {
  const double s29 = 5.385164807134504;   // sqrt(29)
  const double r2 = r * r, r3 = r2 * r;
  const double beta = -7.0 / 3.0 * r3 - 1.5 * r2 + (9.0 + 7.0 * s29) / 20.0 * r + (31.0 + 3.0 * s29) / 40.0;
  const double gq = 1.0 / 32.0 - s29 / 48.0;
  const double gamma = 5.0 / 72.0 * r3 * r3 + gq * r2 * r2;
  const double t = -2.0 * gamma / (beta + sqrt(beta * beta - 112.0 * gamma));
  const double dbeta = -7.0 * r2 - 3.0 * r + (9.0 + 7.0 * s29) / 20.0;
  const double dgamma = 5.0 / 12.0 * r2 * r3 + 4.0 * gq * r3;
  const double dt = -(dbeta * t + dgamma) / (56.0 * t + beta);
  const double c1 = (13.0 - s29) / 80.0, c2 = (7.0 + s29) / 40.0, c0 = 29.0 / 480.0 - s29 / 160.0;
  w[0] = -r3 / 12.0 + r2 / 8.0 - c1 * r + c0 + t;
  w[1] = r3 / 6.0 - c2 * r + 0.25 - 3.0 * t;
  w[2] = -r2 / 4.0 + 91.0 / 240.0 + s29 / 80.0 + 2.0 * t;
  w[3] = -r3 / 6.0 + c2 * r + 0.25 + 2.0 * t;
  w[4] = r3 / 12.0 + r2 / 8.0 + c1 * r + c0 - 3.0 * t;
  w[5] = t;
  dw[0] = -r2 / 4.0 + r / 4.0 - c1 + dt;
  dw[1] = r2 / 2.0 - c2 - 3.0 * dt;
  dw[2] = -r / 2.0 + 2.0 * dt;
  dw[3] = -r2 / 2.0 + c2 + 2.0 * dt;
  dw[4] = r2 / 4.0 + r / 4.0 + c1 - 3.0 * dt;
  dw[5] = dt;
}

// The kw kernel points of a blob coordinate x along axis ax for velocity
// component a, folded at walls:
//   - a point on a wall-normal boundary face is dropped (zero normal velocity);
//   - a point beyond a wall mirrors onto the reflected interior point with
//     sign -1, or +1 for a tangential component at a free-slip wall; a
//     tangential ghost of a no-slip wall also records which wall it came from
//     (its affine ghost value is 2 u_w);
//   - a point whose mirror is not an unknown is dropped.
struct AxisStencil {
  int idx[kKMax];      // compact index along the axis
  double w[kKMax];     // kernel weight phi(s - p)
  double dw[kKMax];    // dphi/dx (derivative with respect to the blob coordinate)
  signed char sgn[kKMax];
  signed char wall[kKMax];   // tangential ghost wall id (2 ax or 2 ax + 1) or -1
  bool keep[kKMax];
};

// Points p = p0 + t (t < kw) of a coordinate s in grid units: three points
// from p0 = floor(s + 1/2) - 1, six from p0 = floor(s) - 2.
__device__ inline void axis_stencil(const Dims& d, int a, int ax, double x, AxisStencil& S) {
  const double o = (ax == a) ? 0.0 : 0.5;
  const double s = x / d.h[ax] - o;
  const int kw = d.kw;
  const double fl = floor(s);
  const int i0 = kw == 6 ? (int)fl - 2 : (int)floor(s + 0.5) - 1;
  double w6[6], dw6[6];
  if (kw == 6) six_weights(s - fl, w6, dw6);
  const int n = d.n[ax];
  for (int t = 0; t < kw; ++t) {
    const int p = i0 + t;
    if (kw == 6) {
      S.w[t] = w6[t];
      S.dw[t] = dw6[t] / d.h[ax];
    } else {
      S.w[t] = phi3(s - (double)p);
      S.dw[t] = dphi3(s - (double)p) / d.h[ax];
    }
    S.sgn[t] = 1;
    S.wall[t] = -1;
    if (d.per[ax]) {
      int m = p % n; if (m < 0) m += n;
      S.idx[t] = m; S.keep[t] = true;
    } else if (ax == a) {          // normal component: physical faces 0..n
      if (p >= 1 && p <= n - 1) { S.idx[t] = p - 1; S.keep[t] = true; }
      else if (p < 0) { int m = -p; S.idx[t] = m - 1; S.sgn[t] = -1; S.keep[t] = (m >= 1 && m <= n - 1); }
      else if (p > n) { int m = 2 * n - p; S.idx[t] = m - 1; S.sgn[t] = -1; S.keep[t] = (m >= 1 && m <= n - 1); }
      else { S.idx[t] = 0; S.keep[t] = false; }
    } else {                       // tangential: cell centres 0..n-1
      if (p < 0) {
        const int m = -1 - p, gs = ghost_sign(d, 2 * ax);
        S.idx[t] = m; S.sgn[t] = (signed char)gs; S.wall[t] = gs < 0 ? 2 * ax : -1; S.keep[t] = (m <= n - 1);
      } else if (p > n - 1) {
        const int m = 2 * n - 1 - p, gs = ghost_sign(d, 2 * ax + 1);
        S.idx[t] = m; S.sgn[t] = (signed char)gs; S.wall[t] = gs < 0 ? 2 * ax + 1 : -1; S.keep[t] = (m >= 0);
      } else { S.idx[t] = p; S.keep[t] = true; }
    }
  }
}

// Philox4x64-10 (Salmon et al., SC11): multipliers, Weyl constants.
__device__ inline void philox4x64_10(unsigned long long c[4], unsigned long long k0, unsigned long long k1) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

__device__ inline double philox_uniform(unsigned long long w) {
  return (double)((w >> 12) * 2ULL + 1ULL) * 0x1.0p-53;
}

// Four standard normals of Philox block b of stream (seed, step, attempt, purpose).
__device__ inline void philox_normals4(unsigned long long seed, unsigned long long step,
                                       unsigned attempt, unsigned purpose,
                                       unsigned long long b, double out[4]) {
  unsigned long long c[4] = {b, step, ((unsigned long long)attempt << 32) | purpose, 0ULL};
  philox4x64_10(c, seed, 0ULL);
#pragma unroll
  for (int pr = 0; pr < 2; ++pr) {
    const double u0 = philox_uniform(c[2 * pr]), u1 = philox_uniform(c[2 * pr + 1]);
    const double rad = sqrt(-2.0 * log(u0));
    double sn, cs;
    sincospi(2.0 * u1, &sn, &cs);
    out[2 * pr] = rad * cs;
    out[2 * pr + 1] = rad * sn;
  }
}

#define RBFIB_DEVFN __device__ __forceinline__

// (J v)_ia by one warp.  Three-point kernel: lane l < 27 takes kernel point
// (l % 3, l / 3 % 3, l / 9).  Six-point kernel: the 216 points p = l, l + 32,
// ... are (p % 6, p / 6 % 6, p / 36).
template <typename T>
RBFIB_DEVFN T warp_interp(const Dims& d, int a, const BlobStencil<T>* __restrict__ S, const T* __restrict__ v,
                          int lane) {
  T val = T(0);
  const T* va = v + d.fo[a];
  if (d.kw == 3) {
    if (lane < 27) {
      const int x = lane % 3, y = (lane / 3) % 3, z = lane / 9;
      const T w = S->w[x] * S->w[kKMax + y] * S->w[2 * kKMax + z];
      if (w != T(0)) val = w * va[flat3(d.fe[a], S->idx[x], S->idx[kKMax + y], S->idx[2 * kKMax + z])];
    }
  } else {
    for (int p = lane; p < 216; p += 32) {
      const int x = p % 6, y = (p / 6) % 6, z = p / 36;
      const T w = S->w[x] * S->w[kKMax + y] * S->w[2 * kKMax + z];
      if (w != T(0)) val += w * va[flat3(d.fe[a], S->idx[x], S->idx[kKMax + y], S->idx[2 * kKMax + z])];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
  return val;
}


// Rotation matrix (row-major) of a unit quaternion (w, x, y, z).
RBFIB_DEVFN void quat_rot(const double* qt, double R[9]) {
  const double w = qt[0], x = qt[1], y = qt[2], z = qt[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

// Programmatic dependent launch.  Every kernel of the library begins with
// pdl_entry(), before it touches global memory: griddepcontrol.wait returns
// once the kernels this grid depends on have completed and their memory
// operations are visible (at once for a normal launch).  A kernel launched
// by launch_k carries the programmatic-serialization attribute, so it may be
// launched as soon as every block of its predecessor has exited, without
// waiting for the predecessor's completion to be processed; since its own
// first instruction is the wait, neither read-after-write nor
// write-after-read order between the two kernels changes.  No kernel
// releases its dependents early (griddepcontrol.launch_dependents): on
// GB300 that placed the blocks of the next short grid while the current one
// still occupied SMs, and the two-sphere SEM step ran 6% slower, against
// 1.8% faster with the release at block exit.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

namespace rbfib {
// false when RBFIB_NO_PDL is set in the environment (read once)
bool pdl_enabled();
}  // namespace rbfib

// Launches kernel k on stream s with programmatic stream serialization (a
// plain launch when it is disabled).  Launch errors are left to
// cudaGetLastError, as with the <<<>>> syntax.
template <typename... P, typename... A>
inline void launch_k(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = rbfib::pdl_enabled() ? 1 : 0;
  (void)cudaLaunchKernelEx(&cfg, k, static_cast<A&&>(args)...);
}

#include <atomic>
namespace rbfib {
// Count of kernel launches issued by the library (host side, all grids and
// threads).
extern std::atomic<unsigned long long> g_launches;
inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace rbfib
