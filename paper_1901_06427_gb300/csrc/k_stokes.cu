// MAC-grid Stokes kernels (Sec. III.A): the homogeneous Stokes operator and
// the geometric multigrid used by the projection preconditioner of the
// velocity-pressure block.  Templated on the storage/arithmetic type T
// (double for the FP64 path, float inside FP64 iterative refinement).
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace rbfib {

// ---------------------------------------------------------------- helpers
template <typename T>
RBFIB_DEVFN T face_at(const Dims& d, const T* __restrict__ v, int a, const int c[3]) {
  return v[d.fo[a] + flat3(d.fe[a], c[0], c[1], c[2])];
}

// Laplacian of component a at compact face c with the ghost-reflection
// boundary conditions: Dirichlet zero at wall-normal boundary faces along a,
// ghost = -self across no-slip and +self across free-slip walls along
// tangential axes (d.gd), wrap on periodic axes.
// Returns sum_nb u_nb / h^2 (neighbours) and the diagonal coefficient.
template <typename T>
RBFIB_DEVFN void lap_parts(const Dims& d, const T* __restrict__ v, int a, const int c[3], T& nbsum, T& diag) {
  nbsum = T(0);
  diag = T(0);
  const i64 base = d.fo[a];
  const int* e = d.fe[a];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const T ih2 = inv_h2<T>(d, ax);
    diag += T(2) * ih2;
    int lo[3] = {c[0], c[1], c[2]}, hi[3] = {c[0], c[1], c[2]};
    lo[ax] -= 1; hi[ax] += 1;
    if (d.per[ax]) {
      if (lo[ax] < 0) lo[ax] += e[ax];
      if (hi[ax] >= e[ax]) hi[ax] -= e[ax];
      nbsum += (v[base + flat3(e, lo[0], lo[1], lo[2])] + v[base + flat3(e, hi[0], hi[1], hi[2])]) * ih2;
    } else {
      if (lo[ax] >= 0) nbsum += v[base + flat3(e, lo[0], lo[1], lo[2])] * ih2;
      else if (ax != a) diag += T(d.gd[2 * ax]) * ih2;
      if (hi[ax] < e[ax]) nbsum += v[base + flat3(e, hi[0], hi[1], hi[2])] * ih2;
      else if (ax != a) diag += T(d.gd[2 * ax + 1]) * ih2;
    }
  }
}

// ------------------------------------------------------- Stokes operator
// Laplacian parts on a level with one spacing h on every axis: neighbour sum
// and diagonal in units of 1/h^2 (fewer multiplies in the FP64 operator).
template <typename T>
RBFIB_DEVFN void lap_parts_uniform(const Dims& d, const T* __restrict__ v, int a, const int c[3], T& nbsum, int& diag) {
  nbsum = T(0);
  diag = 6;
  const i64 base = d.fo[a];
  const int* e = d.fe[a];
  const i64 id = base + flat3(e, c[0], c[1], c[2]);
  const i64 str[3] = {1, (i64)e[0], (i64)e[0] * e[1]};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int lo = c[ax] - 1, hi = c[ax] + 1;
    if (d.per[ax]) {
      nbsum += v[lo < 0 ? id + (e[ax] - 1) * str[ax] : id - str[ax]];
      nbsum += v[hi >= e[ax] ? id - (e[ax] - 1) * str[ax] : id + str[ax]];
    } else {
      if (lo >= 0) nbsum += v[id - str[ax]]; else if (ax != a) diag += d.gd[2 * ax];
      if (hi < e[ax]) nbsum += v[id + str[ax]]; else if (ax != a) diag += d.gd[2 * ax + 1];
    }
  }
}

template <typename T>
__global__ void k_stokes_apply(Dims d, T eta, const T* __restrict__ v, const T* __restrict__ p,
                               T* __restrict__ yv, T* __restrict__ yp) {
  pdl_entry();
  const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  const i64 nf = d.fo[3];
  if (t < nf) {
    int a, c[3];
    decode_face(d, t, a, c);
    const T u = v[t];
    T visc;
    if (d.h[0] == d.h[1] && d.h[1] == d.h[2]) {
      T nb;
      int di;
      lap_parts_uniform(d, v, a, c, nb, di);
      visc = (eta * inv_h2<T>(d, 0)) * ((T)di * u - nb);
    } else {
      T nb, dg;
      lap_parts(d, v, a, c, nb, dg);
      visc = eta * (dg * u - nb);
    }
    // pressure gradient across the face
    int cl[3] = {c[0], c[1], c[2]}, cr[3] = {c[0], c[1], c[2]};
    if (d.per[a]) { cl[a] = c[a] - 1; if (cl[a] < 0) cl[a] += d.n[a]; }
    else { cr[a] = c[a] + 1; }
    const T gp = (p[flat3(d.n, cr[0], cr[1], cr[2])] - p[flat3(d.n, cl[0], cl[1], cl[2])]) * inv_h<T>(d, a);
    yv[t] = visc + gp;
  } else if (t < nf + d.nc) {
    const i64 l = t - nf;
    int c[3];
    decode_cell(d, l, c);
    T div = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T vr = T(0), vl = T(0);
      int f[3] = {c[0], c[1], c[2]};
      if (d.per[a]) {
        vl = face_at(d, v, a, f);
        f[a] = c[a] + 1; if (f[a] >= d.n[a]) f[a] = 0;
        vr = face_at(d, v, a, f);
      } else {
        if (c[a] <= d.n[a] - 2) vr = face_at(d, v, a, f);
        if (c[a] >= 1) { f[a] = c[a] - 1; vl = face_at(d, v, a, f); }
      }
      div += (vr - vl) * inv_h<T>(d, a);
    }
    yp[l] = -div;
  }
}

// Column-chunked Stokes operator for uniform spacing.  A thread owns one
// (x, y) point and one chunk of KC z-planes (kKChunk, or 2 on small grids) and computes, in turn, the
// three momentum rows (one per face grid) and the divergence row of that
// column chunk, so the pressure and velocity rows it touches are reused from
// L1/L2 by all four rows instead of being fetched once per grid.  Along z the
// neighbours stay in registers.  No index divisions; 32-bit offsets.
constexpr int kKChunk = 8;

template <int KC, typename T>
RBFIB_DEVFN void momentum_column(const Dims& d, int a, int i, int j, int k0, T eta, T ih, T ih2,
                                 const T* __restrict__ v, const T* __restrict__ p, T* __restrict__ yv) {
  const int e0 = d.fe[a][0], e1 = d.fe[a][1], e2 = d.fe[a][2];
  if (i >= e0 || j >= e1 || k0 >= e2) return;
  const int k1 = min(k0 + KC, e2);
  const int nx = d.n[0], ny = d.n[1];
  const unsigned base = (unsigned)d.fo[a];
  const unsigned sy = (unsigned)e0, sz = (unsigned)e0 * (unsigned)e1;
  const T* va = v + base;
  const bool perz = d.per[2];
  int dxy = 4;
  unsigned xm = 0, xp = 0, ym = 0, yq = 0;
  bool hxm = true, hxp = true, hym = true, hyp = true;
  if (d.per[0]) { xm = i > 0 ? (unsigned)(i - 1) : (unsigned)(e0 - 1); xp = i < e0 - 1 ? (unsigned)(i + 1) : 0u; }
  else {
    xm = (unsigned)(i - 1); xp = (unsigned)(i + 1);
    if (i == 0) { hxm = false; if (a != 0) dxy += d.gd[0]; }
    if (i == e0 - 1) { hxp = false; if (a != 0) dxy += d.gd[1]; }
  }
  if (d.per[1]) { ym = j > 0 ? (unsigned)(j - 1) : (unsigned)(e1 - 1); yq = j < e1 - 1 ? (unsigned)(j + 1) : 0u; }
  else {
    ym = (unsigned)(j - 1); yq = (unsigned)(j + 1);
    if (j == 0) { hym = false; if (a != 1) dxy += d.gd[2]; }
    if (j == e1 - 1) { hyp = false; if (a != 1) dxy += d.gd[3]; }
  }
  int cxl = i, cxr = i, cyl = j, cyr = j;
  if (a == 0) { if (d.per[0]) cxl = i > 0 ? i - 1 : nx - 1; else cxr = i + 1; }
  if (a == 1) { if (d.per[1]) cyl = j > 0 ? j - 1 : ny - 1; else cyr = j + 1; }
  const unsigned row = (unsigned)i + sy * (unsigned)j;
  const unsigned rxm = xm + sy * (unsigned)j, rxp = xp + sy * (unsigned)j;
  const unsigned rym = (unsigned)i + sy * ym, ryp = (unsigned)i + sy * yq;
  const unsigned pl0 = (unsigned)cxl + (unsigned)nx * (unsigned)cyl, pr0 = (unsigned)cxr + (unsigned)nx * (unsigned)cyr;
  const unsigned pz = (unsigned)nx * (unsigned)ny;
  T um = T(0), u0 = va[row + sz * (unsigned)k0];
  bool hzm = true;
  if (k0 > 0) um = va[row + sz * (unsigned)(k0 - 1)];
  else if (perz) um = va[row + sz * (unsigned)(e2 - 1)];
  else hzm = false;
  const T s = eta * ih2;
#pragma unroll
  for (int kk = 0; kk < KC; ++kk) {
    const int k = k0 + kk;
    if (k >= k1) break;
    T up = T(0);
    bool hzp = true;
    if (k < e2 - 1) up = va[row + sz * (unsigned)(k + 1)];
    else if (perz) up = va[row];
    else hzp = false;
    const unsigned zo = sz * (unsigned)k;
    T nb = um + up;
    int diag = dxy + 2;
    if (!perz && a != 2) diag += (hzm ? 0 : d.gd[4]) + (hzp ? 0 : d.gd[5]);
    if (hxm) nb += va[rxm + zo];
    if (hxp) nb += va[rxp + zo];
    if (hym) nb += va[rym + zo];
    if (hyp) nb += va[ryp + zo];
    int czl = k, czr = k;
    if (a == 2) { if (perz) czl = k > 0 ? k - 1 : d.n[2] - 1; else czr = k + 1; }
    const T gp = (p[pr0 + pz * (unsigned)czr] - p[pl0 + pz * (unsigned)czl]) * ih;
    yv[base + row + zo] = s * ((T)diag * u0 - nb) + gp;
    um = u0; u0 = up; hzm = true;
  }
}

template <int KC, typename T>
RBFIB_DEVFN void divergence_column(const Dims& d, int i, int j, int k0, T ih, const T* __restrict__ v,
                                   T* __restrict__ yp) {
  const int nx = d.n[0], ny = d.n[1], nz = d.n[2];
  if (i >= nx || j >= ny || k0 >= nz) return;
  const int k1 = min(k0 + KC, nz);
  // x faces: compact index along x of the right / left face of cell i
  const int ex0 = d.fe[0][0], ey1 = d.fe[1][1];
  const T* vx = v + (unsigned)d.fo[0];
  const T* vy = v + (unsigned)d.fo[1];
  const T* vz = v + (unsigned)d.fo[2];
  int xr, xl; bool hxr, hxl;
  if (d.per[0]) { xl = i; xr = i + 1 < nx ? i + 1 : 0; hxr = hxl = true; }
  else { xr = i; xl = i - 1; hxr = i <= nx - 2; hxl = i >= 1; }
  int yr, yl; bool hyr, hyl;
  if (d.per[1]) { yl = j; yr = j + 1 < ny ? j + 1 : 0; hyr = hyl = true; }
  else { yr = j; yl = j - 1; hyr = j <= ny - 2; hyl = j >= 1; }
  const unsigned sxy = (unsigned)ex0 * (unsigned)ny;            // x-face plane
  const unsigned syy = (unsigned)nx * (unsigned)ey1;            // y-face plane
  const unsigned szz = (unsigned)nx * (unsigned)ny;             // z-face plane
#pragma unroll
  for (int kk = 0; kk < KC; ++kk) {
    const int k = k0 + kk;
    if (k >= k1) break;
    T div = T(0);
    if (hxr) div += vx[(unsigned)xr + (unsigned)ex0 * (unsigned)j + sxy * (unsigned)k];
    if (hxl) div -= vx[(unsigned)xl + (unsigned)ex0 * (unsigned)j + sxy * (unsigned)k];
    if (hyr) div += vy[(unsigned)i + (unsigned)nx * (unsigned)yr + syy * (unsigned)k];
    if (hyl) div -= vy[(unsigned)i + (unsigned)nx * (unsigned)yl + syy * (unsigned)k];
    int zr, zl; bool hzr, hzl;
    if (d.per[2]) { zl = k; zr = k + 1 < nz ? k + 1 : 0; hzr = hzl = true; }
    else { zr = k; zl = k - 1; hzr = k <= nz - 2; hzl = k >= 1; }
    const unsigned cz = (unsigned)i + (unsigned)nx * (unsigned)j;
    if (hzr) div += vz[cz + szz * (unsigned)zr];
    if (hzl) div -= vz[cz + szz * (unsigned)zl];
    yp[(unsigned)i + (unsigned)nx * ((unsigned)j + (unsigned)ny * (unsigned)k)] = -div * ih;
  }
}

template <int KC, typename T>
RBFIB_DEVFN void stokes_cols_body(const Dims& d, T eta, const T* __restrict__ v, const T* __restrict__ p,
                                  T* __restrict__ yv, T* __restrict__ yp) {
  const int k0 = KC * (int)blockIdx.z;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const T ih = inv_h<T>(d, 0), ih2 = inv_h2<T>(d, 0);
  momentum_column<KC, T>(d, 0, i, j, k0, eta, ih, ih2, v, p, yv);
  momentum_column<KC, T>(d, 1, i, j, k0, eta, ih, ih2, v, p, yv);
  momentum_column<KC, T>(d, 2, i, j, k0, eta, ih, ih2, v, p, yv);
  divergence_column<KC, T>(d, i, j, k0, ih, v, yp);
}

// One thread per (i, j) column and KC z-planes, all four grids.
template <int KC>
__global__ void __launch_bounds__(128) k_stokes_cols_f32(Dims d, float eta, const float* __restrict__ v,
                                                             const float* __restrict__ p, float* __restrict__ yv,
                                                             float* __restrict__ yp) {
  pdl_entry();
  stokes_cols_body<KC, float>(d, eta, v, p, yv, yp);
}
template <int KC>
__global__ void __launch_bounds__(128) k_stokes_cols_f64(Dims d, double eta, const double* __restrict__ v,
                                                         const double* __restrict__ p, double* __restrict__ yv,
                                                         double* __restrict__ yp) {
  pdl_entry();
  stokes_cols_body<KC, double>(d, eta, v, p, yv, yp);
}
template <int KC>
inline void launch_cols(dim3 gr, cudaStream_t s, const Dims& d, float eta, const float* v, const float* p, float* yv,
                        float* yp) {
  launch_k(k_stokes_cols_f32<KC>, gr, dim3(d.n[0] >= 96 ? 128 : 32, d.n[0] >= 96 ? 1 : 4), 0, s, d, eta, v, p, yv, yp);
}
template <int KC>
inline void launch_cols(dim3 gr, cudaStream_t s, const Dims& d, double eta, const double* v, const double* p,
                        double* yv, double* yp) {
  launch_k(k_stokes_cols_f64<KC>, gr, dim3(d.n[0] >= 96 ? 128 : 32, d.n[0] >= 96 ? 1 : 4), 0, s, d, eta, v, p, yv, yp);
}

// Pipelined 2.5D Stokes operator for large grids (uniform spacing).  A 32 x 8
// block owns a 32 x 8 tile of all four grids and marches a chunk of kPZ
// z-planes.  Each plane of the tile, with a one-point halo in x and y, is
// copied into a ring of kPS shared-memory stages by cp.async, kPD planes ahead
// of the plane being computed, so every thread keeps several planes of loads
// in flight instead of waiting on each one.  All neighbours (x, y from the
// staged halo, z from the neighbouring stages) are read from shared memory;
// one barrier per plane.  Each staged value is fetched from global memory
// once per block (halo rows and planes are shared with neighbouring blocks
// through L2).
constexpr int kPX = 32, kPY = 8, kPZ = 32;
constexpr int kPW = kPX + 2, kPH = kPY + 2, kPSlots = kPW * kPH;   // staged plane of one grid
constexpr int kPLoads = (kPSlots + kPX * kPY - 1) / (kPX * kPY);    // slots per thread
// planes in flight ahead of the one computed, and ring stages (the planes
// k - 1, k, k + 1 being read plus the ones in flight): deeper for FP32, whose
// kernel is bound by bytes in flight; FP64 is bound by its arithmetic.
template <typename T> __host__ __device__ constexpr int pipe_depth() { return sizeof(T) == 4 ? 6 : 3; }
template <typename T> __host__ __device__ constexpr int pipe_stages() { return pipe_depth<T>() + 3; }
template <typename T>
__host__ __device__ constexpr int pipe_smem_bytes() { return pipe_stages<T>() * 4 * kPSlots * (int)sizeof(T); }

// Copies one element, or writes zero to the slot when nbytes == 0 (the source
// is then not read).
template <typename T>
RBFIB_DEVFN void cp_async_elem(unsigned dst, const T* src, unsigned nbytes) {
  if constexpr (sizeof(T) == 8) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(nbytes) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(nbytes) : "memory");
  }
}
template <typename T>
RBFIB_DEVFN void cp_async_elem(unsigned dst, const T* src) {
  if constexpr (sizeof(T) == 8) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
  }
}
RBFIB_DEVFN void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
RBFIB_DEVFN void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename T, bool PX, bool PY, bool PZ>
RBFIB_DEVFN void stokes_pipe_body(const Dims& d, T eta, const T* __restrict__ v, const T* __restrict__ p,
                                  T* __restrict__ yv, T* __restrict__ yp, T* sm) {
  constexpr int kPD = pipe_depth<T>(), kPS = pipe_stages<T>();
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + kPX * ty;
  const int x0 = blockIdx.x * kPX, y0 = blockIdx.y * kPY;
  const int k0 = blockIdx.z * kPZ;
  const int nx = d.n[0], ny = d.n[1], nz = d.n[2];
  const int k1 = min(k0 + kPZ, nz);
  // grid g = 0, 1, 2: face components; g = 3: pressure cells
  const T* src[4] = {v + d.fo[0], v + d.fo[1], v + d.fo[2], p};
  unsigned psz[4];
  int ezm[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const int* e = g < 3 ? d.fe[g] : d.n;
    ezm[g] = e[2] - 1;
    psz[g] = (unsigned)e[0] * (unsigned)e[1];
  }
  // Staging: thread tid fills slot tid and, for tid < kPSlots - 256, slot
  // tid + 256 of each grid's (kPH x kPW) plane tile.  Points beyond a wall
  // (and whole planes beyond a z wall) are staged as zero, so neighbours that
  // do not exist add nothing to the stencil sums; their source offsets are
  // clamped onto the grid and not read.
  unsigned off[kPLoads][4];
  unsigned okm = 0;
#pragma unroll
  for (int l = 0; l < kPLoads; ++l) {
    const int s = min(tid + kPX * kPY * l, kPSlots - 1);
    const int ly = s / kPW, lx = s - ly * kPW;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const int* e = g < 3 ? d.fe[g] : d.n;
      int gx = x0 + lx - 1, gy = y0 + ly - 1;
      bool ok = true;
      if (PX) gx = (gx + e[0]) % e[0];
      else { ok = ok && gx >= 0 && gx < e[0]; gx = min(max(gx, 0), e[0] - 1); }
      if (PY) gy = (gy + e[1]) % e[1];
      else { ok = ok && gy >= 0 && gy < e[1]; gy = min(max(gy, 0), e[1] - 1); }
      off[l][g] = (unsigned)gx + (unsigned)e[0] * (unsigned)gy;
      if (ok) okm |= 1u << (4 * l + g);
    }
  }
  const bool second = tid + kPX * kPY < kPSlots;
  constexpr unsigned kGridBytes = kPSlots * sizeof(T), kStageBytes = 4 * kGridBytes;
  const unsigned dst0 = (unsigned)__cvta_generic_to_shared(sm) + (unsigned)tid * (unsigned)sizeof(T);
  // a tile whose staged points all lie inside every grid on the x and y walls
  // (block-uniform), on a plane that exists for all four grids, copies
  // without per-slot tests
  const bool tile_in = (PX || (x0 >= 1 && x0 + kPX <= nx - 2)) && (PY || (y0 >= 1 && y0 + kPY <= ny - 2));
  int ist = 0;   // stage of the next plane to issue
  auto issue = [&](int kk) {
    if (kk <= k1) {
      const unsigned dst = dst0 + (unsigned)ist * kStageBytes;
      if (tile_in && (PZ || (kk >= 0 && kk <= nz - 2))) {
        const int zz = PZ ? (kk < 0 ? kk + nz : (kk >= nz ? kk - nz : kk)) : kk;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const T* base = src[g] + psz[g] * (unsigned)zz;
          cp_async_elem<T>(dst + g * kGridBytes, base + off[0][g]);
          if (second) cp_async_elem<T>(dst + g * kGridBytes + kPX * kPY * sizeof(T), base + off[1][g]);
        }
      } else {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          int zz;
          unsigned nb = (unsigned)sizeof(T);
          if (PZ) zz = kk < 0 ? kk + nz : (kk >= nz ? kk - nz : kk);
          else {
            if (kk < 0 || kk > ezm[g]) nb = 0u;
            zz = min(max(kk, 0), ezm[g]);
          }
          const T* base = src[g] + psz[g] * (unsigned)zz;
          cp_async_elem<T>(dst + g * kGridBytes, base + off[0][g], (okm >> g & 1u) ? nb : 0u);
          if (second)
            cp_async_elem<T>(dst + g * kGridBytes + kPX * kPY * sizeof(T), base + off[1][g],
                             (okm >> (4 + g) & 1u) ? nb : 0u);
        }
      }
      ist = ist + 1 < kPS ? ist + 1 : 0;
    }
    cp_async_commit();
  };
  // prologue: planes k0 - 1 .. k0 + kPD
#pragma unroll
  for (int q = 0; q < kPD + 2; ++q) issue(k0 - 1 + q);

  const int i = x0 + tx, j = y0 + ty;
  const T s = eta * inv_h2<T>(d, 0), ih = inv_h<T>(d, 0);
  const int c0 = (ty + 1) * kPW + tx + 1;   // this thread's centre slot
  constexpr bool pxw = !PX, pyw = !PY;
  // momentum rows: per component, in-plane validity, the diagonal times
  // eta/h^2 (a missing neighbour across a tangential wall is the ghost -u0
  // of a no-slip wall, which adds one to the diagonal, or +u0 of a free-slip
  // wall, which takes one off), output offset at plane 0
  bool in[3];
  T sdiag[3];
  unsigned obase[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int* e = d.fe[a];
    in[a] = i < e[0] && j < e[1];
    int dg = 6;
    if (a != 0 && pxw) dg += (i == 0 ? d.gd[0] : 0) + (i == e[0] - 1 ? d.gd[1] : 0);
    if (a != 1 && pyw) dg += (j == 0 ? d.gd[2] : 0) + (j == e[1] - 1 ? d.gd[3] : 0);
    sdiag[a] = s * (T)dg;
    obase[a] = (unsigned)d.fo[a] + (unsigned)i + (unsigned)e[0] * (unsigned)j;
  }
  const bool inc = i < nx && j < ny;
  const unsigned cbase = (unsigned)i + (unsigned)nx * (unsigned)j;
  int stm = 0;   // stage of plane k - 1
  // this thread's column values of the four grids on planes k - 1, k, k + 1
  // stay in registers; each plane brings one new value per grid
  T zm[4], zc[4], zp[4];
  for (int k = k0; k < k1; ++k) {
    cp_async_wait<kPD - 1>();
    __syncthreads();
    issue(k + kPD + 1);
    const int st0 = stm + 1 < kPS ? stm + 1 : 0;
    const int stp = st0 + 1 < kPS ? st0 + 1 : 0;
    const T* S0 = sm + st0 * 4 * kPSlots;
    const T* Sp = sm + stp * 4 * kPSlots;
    if (k == k0) {
      const T* Sm = sm + stm * 4 * kPSlots;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        zm[g] = Sm[g * kPSlots + c0];
        zc[g] = S0[g * kPSlots + c0];
      }
    }
#pragma unroll
    for (int g = 0; g < 4; ++g) zp[g] = Sp[g * kPSlots + c0];
    stm = st0;
    // ghosts across the z walls for the tangential components
    const T zadj = PZ ? T(0) : s * (T)((k == 0 ? d.gd[4] : 0) + (k == nz - 1 ? d.gd[5] : 0));
    const T pc = zc[3];
    T um[3], ux[3], uy[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T* U0 = S0 + a * kPSlots;
      um[a] = U0[c0 - 1];
      ux[a] = U0[c0 + 1];
      uy[a] = U0[c0 - kPW];
      const T yq = U0[c0 + kPW];
      const T nb = ((um[a] + ux[a]) + (uy[a] + yq)) + (zm[a] + zp[a]);
      const T sd = a != 2 ? sdiag[a] + zadj : sdiag[a];
      T dp;
      if (a == 0) dp = pxw ? S0[3 * kPSlots + c0 + 1] - pc : pc - S0[3 * kPSlots + c0 - 1];
      else if (a == 1) dp = pyw ? S0[3 * kPSlots + c0 + kPW] - pc : pc - S0[3 * kPSlots + c0 - kPW];
      else dp = PZ ? pc - zm[3] : zp[3] - pc;
      const T y = sd * zc[a] - s * nb + dp * ih;
      const bool store = in[a] && (a != 2 || PZ || k < nz - 1);
      if (store) yv[obase[a] + psz[a] * (unsigned)k] = y;
      if (a == 1) uy[1] = yq;   // divergence uses the +y neighbour of v_y when y is periodic
    }
    // divergence: faces beyond a wall were staged as zero
    T div = pxw ? zc[0] - um[0] : ux[0] - zc[0];
    div += pyw ? zc[1] - S0[kPSlots + c0 - kPW] : uy[1] - zc[1];
    div += PZ ? zp[2] - zc[2] : zc[2] - zm[2];
    if (inc) yp[cbase + psz[3] * (unsigned)k] = -div * ih;
#pragma unroll
    for (int g = 0; g < 4; ++g) { zm[g] = zc[g]; zc[g] = zp[g]; }
  }
  // drain the (empty or unused) groups still in flight before the block exits
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <typename T, bool PX, bool PY, bool PZ>
__global__ void __launch_bounds__(kPX * kPY, sizeof(T) == 4 ? 4 : 3)
    k_stokes_pipe(Dims d, T eta, const T* __restrict__ v, const T* __restrict__ p, T* __restrict__ yv,
                  T* __restrict__ yp) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char pipe_smem[];
  stokes_pipe_body<T, PX, PY, PZ>(d, eta, v, p, yv, yp, reinterpret_cast<T*>(pipe_smem));
}
template <typename T, bool PX, bool PY, bool PZ>
void launch_pipe_as(const Dims& d, cudaStream_t s, T eta, const T* v, const T* p, T* yv, T* yp) {
  static std::once_flag f;
  std::call_once(f, [] {
    cudaFuncSetAttribute(k_stokes_pipe<T, PX, PY, PZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         pipe_smem_bytes<T>());
  });
  dim3 gr((d.n[0] + kPX - 1) / kPX, (d.n[1] + kPY - 1) / kPY, (d.n[2] + kPZ - 1) / kPZ);
  launch_k(k_stokes_pipe<T, PX, PY, PZ>, gr, dim3(kPX, kPY), pipe_smem_bytes<T>(), s, d, eta, v, p, yv, yp);
}
template <typename T>
void launch_pipe(const Dims& d, cudaStream_t s, T eta, const T* v, const T* p, T* yv, T* yp) {
  switch ((d.per[0] ? 1 : 0) | (d.per[1] ? 2 : 0) | (d.per[2] ? 4 : 0)) {
    case 0: launch_pipe_as<T, false, false, false>(d, s, eta, v, p, yv, yp); break;
    case 1: launch_pipe_as<T, true, false, false>(d, s, eta, v, p, yv, yp); break;
    case 2: launch_pipe_as<T, false, true, false>(d, s, eta, v, p, yv, yp); break;
    case 3: launch_pipe_as<T, true, true, false>(d, s, eta, v, p, yv, yp); break;
    case 4: launch_pipe_as<T, false, false, true>(d, s, eta, v, p, yv, yp); break;
    case 5: launch_pipe_as<T, true, false, true>(d, s, eta, v, p, yv, yp); break;
    case 6: launch_pipe_as<T, false, true, true>(d, s, eta, v, p, yv, yp); break;
    default: launch_pipe_as<T, true, true, true>(d, s, eta, v, p, yv, yp); break;
  }
}
// The pipelined kernel serves grids with at least this many unknowns (the
// column kernel fills the GPU better on small grids).
constexpr i64 kPipeMinUnknowns = (i64)2 * 1024 * 1024;

// ------------------------------------------ velocity multigrid (A = -eta LL)
// Diagonal of -LL at a face (a ghost across a tangential no-slip wall adds
// 1/h^2, across a free-slip wall takes 1/h^2 off).
template <typename T>
RBFIB_DEVFN T lap_diag(const Dims& d, int a, const int c[3]) {
  T dg = T(0);
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const T ih2 = inv_h2<T>(d, ax);
    dg += T(2) * ih2;
    if (!d.per[ax] && ax != a) {
      if (c[ax] == 0) dg += T(d.gd[2 * ax]) * ih2;
      if (c[ax] == d.fe[a][ax] - 1) dg += T(d.gd[2 * ax + 1]) * ih2;
    }
  }
  return dg;
}

// One red-black Gauss-Seidel half sweep: threads map to the points of one colour.
template <typename T>
__global__ void k_vel_rbgs(Dims d, ColorMap m, T eta, int color, T* __restrict__ u, const T* __restrict__ rhs) {
  pdl_entry();
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  int a, c[3];
  if (!color_face(d, m, t, color, a, c)) return;
  T nb, dg;
  lap_parts(d, u, a, c, nb, dg);
  const i64 id = d.fo[a] + flat3(d.fe[a], c[0], c[1], c[2]);
  u[id] = (rhs[id] / eta + nb) / dg;
}

// Red-black half sweep for one spacing h on every axis: blockIdx.z -> (face
// component a, plane k), y -> row j, x -> half-row index, so the point is
// ((2 h' + parity), j, k) with no divisions.  The update is
// u = (rhs h^2 / eta + sum of neighbours) / count, where count = 6 plus one
// per tangential no-slip ghost and minus one per free-slip ghost; missing
// wall-normal neighbours are zero.
template <typename T>
RBFIB_DEVFN T smooth_div(T a, int c);
template <>
RBFIB_DEVFN float smooth_div<float>(float a, int c) { return __fdividef(a, (float)c); }
template <>
RBFIB_DEVFN double smooth_div<double>(double a, int c) { return a / (double)c; }

template <typename T>
__global__ void k_vel_rbgs_u(Dims d, T sh, int color, T* __restrict__ u, const T* __restrict__ rhs) {
  pdl_entry();
  const int nz = d.n[2];
  const int a = (int)blockIdx.z / nz, k = (int)blockIdx.z - a * nz;
  const int e0 = d.fe[a][0], e1 = d.fe[a][1], e2 = d.fe[a][2];
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int i = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x) + ((j + k + color) & 1);
  if (k >= e2 || j >= e1 || i >= e0) return;
  T* ua = u + (unsigned)d.fo[a];
  const unsigned sy = (unsigned)e0, sz = (unsigned)e0 * (unsigned)e1;
  const unsigned id = (unsigned)i + sy * (unsigned)j + sz * (unsigned)k;
  T nb = T(0);
  int cnt = 6;
  // x
  if (d.per[0]) nb += ua[i > 0 ? id - 1 : id + (e0 - 1)] + ua[i < e0 - 1 ? id + 1 : id - (e0 - 1)];
  else {
    if (i > 0) nb += ua[id - 1]; else if (a != 0) cnt += d.gd[0];
    if (i < e0 - 1) nb += ua[id + 1]; else if (a != 0) cnt += d.gd[1];
  }
  // y
  if (d.per[1]) nb += ua[j > 0 ? id - sy : id + sy * (e1 - 1)] + ua[j < e1 - 1 ? id + sy : id - sy * (e1 - 1)];
  else {
    if (j > 0) nb += ua[id - sy]; else if (a != 1) cnt += d.gd[2];
    if (j < e1 - 1) nb += ua[id + sy]; else if (a != 1) cnt += d.gd[3];
  }
  // z
  if (d.per[2]) nb += ua[k > 0 ? id - sz : id + sz * (e2 - 1)] + ua[k < e2 - 1 ? id + sz : id - sz * (e2 - 1)];
  else {
    if (k > 0) nb += ua[id - sz]; else if (a != 2) cnt += d.gd[4];
    if (k < e2 - 1) nb += ua[id + sz]; else if (a != 2) cnt += d.gd[5];
  }
  ua[id] = smooth_div<T>(rhs[(unsigned)d.fo[a] + id] * sh + nb, cnt);
}

// Same for the Neumann pressure operator -D G: count = number of existing
// neighbours (6 on periodic axes).
template <typename T>
__global__ void k_p_rbgs_u(Dims d, T sh, int color, T* __restrict__ u, const T* __restrict__ rhs) {
  pdl_entry();
  const int n0 = d.n[0], n1 = d.n[1], n2 = d.n[2];
  const int k = blockIdx.z;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int i = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x) + ((j + k + color) & 1);
  if (j >= n1 || i >= n0) return;
  const unsigned sy = (unsigned)n0, sz = (unsigned)n0 * (unsigned)n1;
  const unsigned id = (unsigned)i + sy * (unsigned)j + sz * (unsigned)k;
  T nb = T(0);
  int cnt = 0;
  if (d.per[0]) { nb += u[i > 0 ? id - 1 : id + (n0 - 1)] + u[i < n0 - 1 ? id + 1 : id - (n0 - 1)]; cnt += 2; }
  else {
    if (i > 0) { nb += u[id - 1]; ++cnt; }
    if (i < n0 - 1) { nb += u[id + 1]; ++cnt; }
  }
  if (d.per[1]) { nb += u[j > 0 ? id - sy : id + sy * (n1 - 1)] + u[j < n1 - 1 ? id + sy : id - sy * (n1 - 1)]; cnt += 2; }
  else {
    if (j > 0) { nb += u[id - sy]; ++cnt; }
    if (j < n1 - 1) { nb += u[id + sy]; ++cnt; }
  }
  if (d.per[2]) { nb += u[k > 0 ? id - sz : id + sz * (n2 - 1)] + u[k < n2 - 1 ? id + sz : id - sz * (n2 - 1)]; cnt += 2; }
  else {
    if (k > 0) { nb += u[id - sz]; ++cnt; }
    if (k < n2 - 1) { nb += u[id + sz]; ++cnt; }
  }
  u[id] = cnt > 0 ? smooth_div<T>(rhs[id] * sh + nb, cnt) : u[id];
}

// Diagonal count of face (a; i, j, k) of the uniform-spacing velocity
// operator: 6 plus one per tangential no-slip ghost, minus one per
// free-slip ghost.
RBFIB_DEVFN int face_count(const Dims& d, int a, int i, int j, int k, int e0, int e1, int e2) {
  int c = 6;
  if (a != 0 && !d.per[0]) c += (i == 0 ? d.gd[0] : 0) + (i == e0 - 1 ? d.gd[1] : 0);
  if (a != 1 && !d.per[1]) c += (j == 0 ? d.gd[2] : 0) + (j == e1 - 1 ? d.gd[3] : 0);
  if (a != 2 && !d.per[2]) c += (k == 0 ? d.gd[4] : 0) + (k == e2 - 1 ? d.gd[5] : 0);
  return c;
}

// The first two half sweeps of a V-cycle from a zero initial guess in one
// launch (uniform spacing): colour-0 faces get u = rhs h^2 / (eta count);
// a colour-1 face adds its colour-0 neighbours' values, formed on the fly
// from their right-hand sides, in the same order as k_vel_rbgs_u.
template <typename T>
__global__ void k_vel_first2_u(Dims d, T sh, T* __restrict__ u, const T* __restrict__ rhs) {
  pdl_entry();
  const int nz = d.n[2];
  const int a = (int)blockIdx.z / nz, k = (int)blockIdx.z - a * nz;
  const int e0 = d.fe[a][0], e1 = d.fe[a][1], e2 = d.fe[a][2];
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= e2 || j >= e1 || i >= e0) return;
  const T* ra = rhs + (unsigned)d.fo[a];
  const unsigned sy = (unsigned)e0, sz = (unsigned)e0 * (unsigned)e1;
  const unsigned id = (unsigned)i + sy * (unsigned)j + sz * (unsigned)k;
  const int cnt = face_count(d, a, i, j, k, e0, e1, e2);
  if (((i + j + k) & 1) == 0) {
    u[(unsigned)d.fo[a] + id] = smooth_div<T>(ra[id] * sh, cnt);
    return;
  }
  auto first = [&](int ii, int jj, int kk) {
    const unsigned nid = (unsigned)ii + sy * (unsigned)jj + sz * (unsigned)kk;
    return smooth_div<T>(ra[nid] * sh, face_count(d, a, ii, jj, kk, e0, e1, e2));
  };
  T nb = T(0);
  // x
  if (d.per[0]) nb += first(i > 0 ? i - 1 : e0 - 1, j, k) + first(i < e0 - 1 ? i + 1 : 0, j, k);
  else {
    if (i > 0) nb += first(i - 1, j, k);
    if (i < e0 - 1) nb += first(i + 1, j, k);
  }
  // y
  if (d.per[1]) nb += first(i, j > 0 ? j - 1 : e1 - 1, k) + first(i, j < e1 - 1 ? j + 1 : 0, k);
  else {
    if (j > 0) nb += first(i, j - 1, k);
    if (j < e1 - 1) nb += first(i, j + 1, k);
  }
  // z
  if (d.per[2]) nb += first(i, j, k > 0 ? k - 1 : e2 - 1) + first(i, j, k < e2 - 1 ? k + 1 : 0);
  else {
    if (k > 0) nb += first(i, j, k - 1);
    if (k < e2 - 1) nb += first(i, j, k + 1);
  }
  u[(unsigned)d.fo[a] + id] = smooth_div<T>(ra[id] * sh + nb, cnt);
}

// Neumann pressure analogue: count = number of existing neighbours.
RBFIB_DEVFN int cell_count(const Dims& d, int i, int j, int k) {
  int c = 0;
  c += d.per[0] ? 2 : (i > 0) + (i < d.n[0] - 1);
  c += d.per[1] ? 2 : (j > 0) + (j < d.n[1] - 1);
  c += d.per[2] ? 2 : (k > 0) + (k < d.n[2] - 1);
  return c;
}
template <typename T>
__global__ void k_p_first2_u(Dims d, T sh, T* __restrict__ u, const T* __restrict__ rhs) {
  pdl_entry();
  const int n0 = d.n[0], n1 = d.n[1], n2 = d.n[2];
  const int k = blockIdx.z;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n1 || i >= n0) return;
  const unsigned sy = (unsigned)n0, sz = (unsigned)n0 * (unsigned)n1;
  const unsigned id = (unsigned)i + sy * (unsigned)j + sz * (unsigned)k;
  const int cnt = cell_count(d, i, j, k);
  if (cnt == 0) { u[id] = T(0); return; }
  if (((i + j + k) & 1) == 0) {
    u[id] = smooth_div<T>(rhs[id] * sh, cnt);
    return;
  }
  auto first = [&](int ii, int jj, int kk) {
    const unsigned nid = (unsigned)ii + sy * (unsigned)jj + sz * (unsigned)kk;
    const int c = cell_count(d, ii, jj, kk);
    return c > 0 ? smooth_div<T>(rhs[nid] * sh, c) : T(0);
  };
  T nb = T(0);
  if (d.per[0]) nb += first(i > 0 ? i - 1 : n0 - 1, j, k) + first(i < n0 - 1 ? i + 1 : 0, j, k);
  else {
    if (i > 0) nb += first(i - 1, j, k);
    if (i < n0 - 1) nb += first(i + 1, j, k);
  }
  if (d.per[1]) nb += first(i, j > 0 ? j - 1 : n1 - 1, k) + first(i, j < n1 - 1 ? j + 1 : 0, k);
  else {
    if (j > 0) nb += first(i, j - 1, k);
    if (j < n1 - 1) nb += first(i, j + 1, k);
  }
  if (d.per[2]) nb += first(i, j, k > 0 ? k - 1 : n2 - 1) + first(i, j, k < n2 - 1 ? k + 1 : 0);
  else {
    if (k > 0) nb += first(i, j, k - 1);
    if (k < n2 - 1) nb += first(i, j, k + 1);
  }
  u[id] = smooth_div<T>(rhs[id] * sh + nb, cnt);
}

// First half sweep from a zero initial guess: colour 0 gets rhs / (eta diag),
// colour 1 is zeroed.
template <typename T>
__global__ void k_vel_first(Dims d, T eta, T* __restrict__ u, const T* __restrict__ rhs) {
  pdl_entry();
  const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.fo[3]) return;
  int a, c[3];
  decode_face(d, t, a, c);
  u[t] = (((c[0] + c[1] + c[2]) & 1) == 0) ? rhs[t] / (eta * lap_diag<T>(d, a, c)) : T(0);
}

// One-dimensional transfer stencils.  kind: 0 = not coarsened,
// 1 = face-centred on a periodic axis, 2 = face-centred on a wall axis,
// 3 = cell-centred.  gs_lo, gs_hi: value of a cell-centred ghost beyond the
// low / high wall in units of the adjacent interior value (-1 Dirichlet,
// +1 Neumann), or 2 on a periodic axis.
struct T1 { int cnt; int idx[3]; float w[3]; };   // weights exact in FP32

// Lanes that share one coarse point of the fused residual-restriction
// (a power of two dividing 32).
constexpr int kRestrictLanes = 4;

__device__ inline void restrict_1d(int kind, int ic, int nfext, T1& s) {
  if (kind == 0) { s.cnt = 1; s.idx[0] = ic; s.w[0] = 1.0f; return; }
  if (kind == 3) { s.cnt = 2; s.idx[0] = 2 * ic; s.idx[1] = 2 * ic + 1; s.w[0] = s.w[1] = 0.5f; return; }
  if (kind == 1) {   // periodic faces, compact == physical; fine extent nfext
    int P = 2 * ic;
    s.cnt = 3;
    s.idx[0] = (P - 1 + nfext) % nfext; s.w[0] = 0.25f;
    s.idx[1] = P; s.w[1] = 0.5f;
    s.idx[2] = (P + 1) % nfext; s.w[2] = 0.25f;
    return;
  }
  // wall faces: coarse compact ic <-> physical Q = ic + 1 <-> fine physical 2Q
  int P = 2 * (ic + 1);
  s.cnt = 3;
  s.idx[0] = P - 2; s.w[0] = 0.25f;    // fine compact of physical P-1
  s.idx[1] = P - 1; s.w[1] = 0.5f;
  s.idx[2] = P;     s.w[2] = 0.25f;    // physical P+1
}

__device__ inline void prolong_1d(int kind, int jf, int ncext, float gs_lo, float gs_hi, T1& s) {
  if (kind == 0) { s.cnt = 1; s.idx[0] = jf; s.w[0] = 1.0f; return; }
  if (kind == 1) {
    if ((jf & 1) == 0) { s.cnt = 1; s.idx[0] = jf / 2; s.w[0] = 1.0f; return; }
    s.cnt = 2; s.idx[0] = (jf - 1) / 2; s.idx[1] = ((jf + 1) / 2) % ncext; s.w[0] = s.w[1] = 0.5f; return;
  }
  if (kind == 2) {   // fine physical P = jf + 1; coarse physical Q; boundary Q carry zero
    int P = jf + 1;
    if ((P & 1) == 0) { s.cnt = 1; s.idx[0] = P / 2 - 1; s.w[0] = 1.0f; return; }
    s.cnt = 0;
    int q1 = (P - 1) / 2, q2 = (P + 1) / 2;
    int nq = ncext + 1;   // coarse physical faces 0..nq
    if (q1 >= 1 && q1 <= nq - 1) { s.idx[s.cnt] = q1 - 1; s.w[s.cnt] = 0.5f; ++s.cnt; }
    if (q2 >= 1 && q2 <= nq - 1) { s.idx[s.cnt] = q2 - 1; s.w[s.cnt] = 0.5f; ++s.cnt; }
    return;
  }
  // cell-centred linear interpolation
  int jc = jf >> 1;
  int nb = (jf & 1) ? jc + 1 : jc - 1;
  s.cnt = 2;
  s.idx[0] = jc; s.w[0] = 0.75f;
  if (nb < 0 || nb >= ncext) {
    const float ghost_sign = nb < 0 ? gs_lo : gs_hi;
    if (ghost_sign == 2.0f) { nb = (nb + ncext) % ncext; s.idx[1] = nb; s.w[1] = 0.25f; }   // periodic
    else { s.cnt = 1; s.w[0] = 0.75f + 0.25f * ghost_sign; }
  } else { s.idx[1] = nb; s.w[1] = 0.25f; }
}

// Restriction of the face residuals rhs - A u, computed on the fly at the fine
// points, to the coarse level: full weighting along a face-centred axis,
// averaging of the two children along cell-centred axes.
template <typename T>
__global__ void k_vel_restrict_res(Dims df, Dims dc, int3 cz, T eta, const T* __restrict__ uf,
                                   const T* __restrict__ rhsf, T* __restrict__ rc) {
  pdl_entry();
  // kRestrictLanes lanes per coarse point share its fine residuals
  const i64 gt = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  const i64 t = gt / kRestrictLanes;
  const int sub = (int)(gt % kRestrictLanes);
  float acc = 0.f;
  if (t < dc.fo[3]) {
    int a, c[3];
    decode_face(dc, t, a, c);
    const int cf[3] = {cz.x, cz.y, cz.z};
    T1 s[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      int kind = !cf[ax] ? 0 : (ax == a ? (df.per[ax] ? 1 : 2) : 3);
      restrict_1d(kind, c[ax], df.fe[a][ax], s[ax]);
    }
    const int nyz = s[1].cnt * s[2].cnt, tot = s[0].cnt * nyz;
    for (int q = sub; q < tot; q += kRestrictLanes) {
      const int x = q / nyz, y = (q - x * nyz) / s[2].cnt, z = q - x * nyz - y * s[2].cnt;
      const int fc[3] = {s[0].idx[x], s[1].idx[y], s[2].idx[z]};
      T nb, dg;
      lap_parts(df, uf, a, fc, nb, dg);
      const i64 id = df.fo[a] + flat3(df.fe[a], fc[0], fc[1], fc[2]);
      const T r = rhsf[id] - eta * (dg * uf[id] - nb);
      acc += (s[0].w[x] * s[1].w[y] * s[2].w[z]) * (float)r;
    }
  }
#pragma unroll
  for (int o = 1; o < kRestrictLanes; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (t < dc.fo[3] && sub == 0) rc[t] = (T)acc;
}

template <typename T>
__global__ void k_vel_prolong(Dims df, Dims dc, int3 cz, const T* __restrict__ uc, T* __restrict__ uf) {
  pdl_entry();
  const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= df.fo[3]) return;
  int a, c[3];
  decode_face(df, t, a, c);
  const int cf[3] = {cz.x, cz.y, cz.z};
  T1 s[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    int kind = !cf[ax] ? 0 : (ax == a ? (df.per[ax] ? 1 : 2) : 3);
    const float gs_lo = df.per[ax] ? 2.0f : (float)ghost_sign(df, 2 * ax);
    const float gs_hi = df.per[ax] ? 2.0f : (float)ghost_sign(df, 2 * ax + 1);
    prolong_1d(kind, c[ax], dc.fe[a][ax], gs_lo, gs_hi, s[ax]);
  }
  T acc = T(0);
  for (int x = 0; x < s[0].cnt; ++x)
    for (int y = 0; y < s[1].cnt; ++y)
      for (int z = 0; z < s[2].cnt; ++z)
        acc += (T)(s[0].w[x] * s[1].w[y] * s[2].w[z]) *
               uc[dc.fo[a] + flat3(dc.fe[a], s[0].idx[x], s[1].idx[y], s[2].idx[z])];
  uf[t] += (T)acc;
}

// ---------------------------------- pressure multigrid (-L_p = -D G, Neumann)
template <typename T>
RBFIB_DEVFN void plap_parts(const Dims& d, const T* __restrict__ p, const int c[3], T& nbsum, T& diag) {
  nbsum = T(0); diag = T(0);
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const T ih2 = inv_h2<T>(d, ax);
    int lo[3] = {c[0], c[1], c[2]}, hi[3] = {c[0], c[1], c[2]};
    lo[ax] -= 1; hi[ax] += 1;
    if (d.per[ax]) {
      if (lo[ax] < 0) lo[ax] += d.n[ax];
      if (hi[ax] >= d.n[ax]) hi[ax] -= d.n[ax];
      nbsum += (p[flat3(d.n, lo[0], lo[1], lo[2])] + p[flat3(d.n, hi[0], hi[1], hi[2])]) * ih2;
      diag += T(2) * ih2;
    } else {
      if (lo[ax] >= 0) { nbsum += p[flat3(d.n, lo[0], lo[1], lo[2])] * ih2; diag += ih2; }
      if (hi[ax] < d.n[ax]) { nbsum += p[flat3(d.n, hi[0], hi[1], hi[2])] * ih2; diag += ih2; }
    }
  }
}

template <typename T>
__global__ void k_p_rbgs(Dims d, ColorMap m, int color, T* __restrict__ u, const T* __restrict__ rhs) {
  pdl_entry();
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  int c[3];
  if (!color_cell(d, m, t, color, c)) return;
  T nb, dg;
  plap_parts(d, u, c, nb, dg);
  const i64 id = flat3(d.n, c[0], c[1], c[2]);
  u[id] = (rhs[id] + nb) / dg;
}

template <typename T>
RBFIB_DEVFN T plap_diag(const Dims& d, const int c[3]) {
  T dg = T(0);
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const T ih2 = inv_h2<T>(d, ax);
    if (d.per[ax]) dg += T(2) * ih2;
    else dg += ih2 * (T)((c[ax] > 0) + (c[ax] < d.n[ax] - 1));
  }
  return dg;
}

template <typename T>
__global__ void k_p_first(Dims d, T* __restrict__ u, const T* __restrict__ rhs) {
  pdl_entry();
  const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.nc) return;
  int c[3];
  decode_cell(d, t, c);
  u[t] = (((c[0] + c[1] + c[2]) & 1) == 0) ? rhs[t] / plap_diag<T>(d, c) : T(0);
}

template <typename T>
__global__ void k_p_restrict_res(Dims df, Dims dc, int3 cz, const T* __restrict__ uf, const T* __restrict__ rhsf,
                                 T* __restrict__ rc) {
  pdl_entry();
  const i64 gt = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  const i64 t = gt / kRestrictLanes;
  const int sub = (int)(gt % kRestrictLanes);
  float acc = 0.f;
  if (t < dc.nc) {
    int c[3];
    decode_cell(dc, t, c);
    const int cf[3] = {cz.x, cz.y, cz.z};
    T1 s[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) restrict_1d(cf[ax] ? 3 : 0, c[ax], df.n[ax], s[ax]);
    const int nyz = s[1].cnt * s[2].cnt, tot = s[0].cnt * nyz;
    for (int q = sub; q < tot; q += kRestrictLanes) {
      const int x = q / nyz, y = (q - x * nyz) / s[2].cnt, z = q - x * nyz - y * s[2].cnt;
      const int fc[3] = {s[0].idx[x], s[1].idx[y], s[2].idx[z]};
      T nb, dg;
      plap_parts(df, uf, fc, nb, dg);
      const i64 id = flat3(df.n, fc[0], fc[1], fc[2]);
      acc += (s[0].w[x] * s[1].w[y] * s[2].w[z]) * (float)(rhsf[id] - (dg * uf[id] - nb));
    }
  }
#pragma unroll
  for (int o = 1; o < kRestrictLanes; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (t < dc.nc && sub == 0) rc[t] = (T)acc;
}

template <typename T>
__global__ void k_p_prolong(Dims df, Dims dc, int3 cz, const T* __restrict__ uc, T* __restrict__ uf) {
  pdl_entry();
  const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= df.nc) return;
  int c[3];
  decode_cell(df, t, c);
  const int cf[3] = {cz.x, cz.y, cz.z};
  T1 s[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const float gs = df.per[ax] ? 2.0f : 1.0f;
    prolong_1d(cf[ax] ? 3 : 0, c[ax], dc.n[ax], gs, gs, s[ax]);
  }
  T acc = T(0);
  for (int x = 0; x < s[0].cnt; ++x)
    for (int y = 0; y < s[1].cnt; ++y)
      for (int z = 0; z < s[2].cnt; ++z)
        acc += (T)(s[0].w[x] * s[1].w[y] * s[2].w[z]) * uc[flat3(dc.n, s[0].idx[x], s[1].idx[y], s[2].idx[z])];
  uf[t] += (T)acc;
}

// Coarsest-level solves: one block, red-black sweeps with block barriers.
template <typename T>
__global__ void k_vel_coarse(Dims d, T eta, T* __restrict__ u, const T* __restrict__ rhs, int sweeps) {
  pdl_entry();
  const i64 n = d.fo[3];
  for (i64 t = threadIdx.x; t < n; t += blockDim.x) u[t] = T(0);
  __syncthreads();
  for (int s = 0; s < sweeps; ++s) {
    for (int color = 0; color < 2; ++color) {
      for (i64 t = threadIdx.x; t < n; t += blockDim.x) {
        int a, c[3];
        decode_face(d, t, a, c);
        if (((c[0] + c[1] + c[2]) & 1) != color) continue;
        T nb, dg;
        lap_parts(d, u, a, c, nb, dg);
        u[t] = (rhs[t] / eta + nb) / dg;
      }
      __syncthreads();
    }
  }
}

template <typename T>
__global__ void k_p_coarse(Dims d, T* __restrict__ u, T* __restrict__ rhs, int sweeps) {
  pdl_entry();
  __shared__ double red[1024];
  const i64 n = d.nc;
  double s = 0.0;
  for (i64 t = threadIdx.x; t < n; t += blockDim.x) s += (double)rhs[t];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const T mean = (T)(red[0] / (double)n);
  __syncthreads();
  for (i64 t = threadIdx.x; t < n; t += blockDim.x) { rhs[t] -= mean; u[t] = T(0); }
  __syncthreads();
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int color = 0; color < 2; ++color) {
      for (i64 t = threadIdx.x; t < n; t += blockDim.x) {
        int c[3];
        decode_cell(d, t, c);
        if (((c[0] + c[1] + c[2]) & 1) != color) continue;
        T nb, dg;
        plap_parts(d, u, c, nb, dg);
        u[t] = (rhs[t] + nb) / dg;
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------ projection preconditioner
// q = r_pi + D v~ ; pi = -eta q (and its FP64 copy pi64 unless null)
template <typename T>
__global__ void k_div_q(Dims d, T eta, const T* __restrict__ vt, const T* __restrict__ rpi,
                        T* __restrict__ q, T* __restrict__ pi, double* __restrict__ pi64) {
  pdl_entry();
  const i64 l = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= d.nc) return;
  int c[3];
  decode_cell(d, l, c);
  T div = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T vr = T(0), vl = T(0);
    int f[3] = {c[0], c[1], c[2]};
    if (d.per[a]) {
      vl = face_at(d, vt, a, f);
      f[a] = c[a] + 1; if (f[a] >= d.n[a]) f[a] = 0;
      vr = face_at(d, vt, a, f);
    } else {
      if (c[a] <= d.n[a] - 2) vr = face_at(d, vt, a, f);
      if (c[a] >= 1) { f[a] = c[a] - 1; vl = face_at(d, vt, a, f); }
    }
    div += (vr - vl) * inv_h<T>(d, a);
  }
  const T qq = rpi[l] + div;
  q[l] = qq;
  const T pv = -eta * qq;
  pi[l] = pv;
  if (pi64) pi64[l] = (double)pv;
}

// v += G phi (and its FP64 copy v64 unless null)
template <typename T>
__global__ void k_add_grad(Dims d, const T* __restrict__ phi, T* __restrict__ v, double* __restrict__ v64) {
  pdl_entry();
  const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.fo[3]) return;
  int a, c[3];
  decode_face(d, t, a, c);
  int cl[3] = {c[0], c[1], c[2]}, cr[3] = {c[0], c[1], c[2]};
  if (d.per[a]) { cl[a] = c[a] - 1; if (cl[a] < 0) cl[a] += d.n[a]; }
  else { cr[a] = c[a] + 1; }
  const T nv = v[t] + (phi[flat3(d.n, cr[0], cr[1], cr[2])] - phi[flat3(d.n, cl[0], cl[1], cl[2])]) * inv_h<T>(d, a);
  v[t] = nv;
  if (v64) v64[t] = (double)nv;
}

// ---------------------------------------------------------------- launchers
static inline unsigned nblk(i64 n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <typename T>
void stokes_apply(const Dims& d, T eta, const T* v, const T* p, T* yv, T* yp, cudaStream_t s, int bs) {
  const bool uniform = d.h[0] == d.h[1] && d.h[1] == d.h[2];
  if (uniform && d.fo[3] + d.nc < ((i64)1 << 31)) {
    if (d.fo[3] + d.nc >= kPipeMinUnknowns) {
      launch_pipe(d, s, eta, v, p, yv, yp);
    } else {
      // small grids: short z-chunks, for enough threads to fill the GPU
      const int bx = d.n[0] >= 96 ? 128 : 32, by = 128 / bx;
      if (d.fo[3] + d.nc >= kPipeMinUnknowns / 4) {
        dim3 grid((d.n[0] + bx - 1) / bx, (d.n[1] + by - 1) / by, (d.n[2] + kKChunk - 1) / kKChunk);
        launch_cols<kKChunk>(grid, s, d, eta, v, p, yv, yp);
      } else {
        dim3 grid((d.n[0] + bx - 1) / bx, (d.n[1] + by - 1) / by, (d.n[2] + 1) / 2);
        launch_cols<2>(grid, s, d, eta, v, p, yv, yp);
      }
    }
  } else {
    const i64 n = d.fo[3] + d.nc;
    launch_k(k_stokes_apply<T>, nblk(n, bs), bs, 0, s, d, eta, v, p, yv, yp);
  }
  note_launch();
}
template <typename T>
void vel_rbgs(const Dims& d, T eta, int color, T* u, const T* rhs, cudaStream_t s, int bs) {
  if (d.h[0] == d.h[1] && d.h[1] == d.h[2] && d.fo[3] < ((i64)1 << 31)) {
    // 32 half-row points x bs / 32 rows per block
    const int by = std::max(1, bs / 32);
    dim3 grid((d.n[0] / 2 + 1 + 31) / 32, (d.n[1] + by - 1) / by, 3 * d.n[2]);
    launch_k(k_vel_rbgs_u<T>, grid, dim3(32, by), 0, s, d, (T)(d.h[0] * d.h[0] / (double)eta), color, u, rhs);
  } else {
    const ColorMap m = make_color_map_faces(d);
    launch_k(k_vel_rbgs<T>, nblk((i64)m.cnt[0] + m.cnt[1] + m.cnt[2], bs), bs, 0, s, d, m, eta, color, u, rhs);
  }
  note_launch();
}
template <typename T>
void vel_first(const Dims& d, T eta, T* u, const T* rhs, cudaStream_t s) {
  launch_k(k_vel_first<T>, nblk(d.fo[3], 256), 256, 0, s, d, eta, u, rhs);
  note_launch();
}
// First two half sweeps from a zero guess in one launch on uniform spacing;
// false (nothing launched) otherwise.
template <typename T>
bool vel_first2(const Dims& d, T eta, T* u, const T* rhs, cudaStream_t s, int bs) {
  if (!(d.h[0] == d.h[1] && d.h[1] == d.h[2] && d.fo[3] < ((i64)1 << 31))) return false;
  const int by = std::max(1, bs / 32);
  dim3 grid((d.n[0] + 31) / 32, (d.n[1] + by - 1) / by, 3 * d.n[2]);
  launch_k(k_vel_first2_u<T>, grid, dim3(32, by), 0, s, d, (T)(d.h[0] * d.h[0] / (double)eta), u, rhs);
  note_launch();
  return true;
}
template <typename T>
bool p_first2(const Dims& d, T* u, const T* rhs, cudaStream_t s, int bs) {
  if (!(d.h[0] == d.h[1] && d.h[1] == d.h[2] && d.nc < ((i64)1 << 31))) return false;
  const int by = std::max(1, bs / 32);
  dim3 grid((d.n[0] + 31) / 32, (d.n[1] + by - 1) / by, d.n[2]);
  launch_k(k_p_first2_u<T>, grid, dim3(32, by), 0, s, d, (T)(d.h[0] * d.h[0]), u, rhs);
  note_launch();
  return true;
}
template <typename T>
void vel_restrict_res(const Dims& df, const Dims& dc, int3 cz, T eta, const T* uf, const T* rhsf, T* rc,
                      cudaStream_t s) {
  launch_k(k_vel_restrict_res<T>, nblk(kRestrictLanes * dc.fo[3], 256), 256, 0, s, df, dc, cz, eta, uf, rhsf, rc);
  note_launch();
}
template <typename T>
void vel_prolong(const Dims& df, const Dims& dc, int3 cz, const T* uc, T* uf, cudaStream_t s) {
  launch_k(k_vel_prolong<T>, nblk(df.fo[3], 256), 256, 0, s, df, dc, cz, uc, uf);
  note_launch();
}
template <typename T>
void vel_coarse(const Dims& d, T eta, T* u, const T* rhs, int sweeps, cudaStream_t s) {
  launch_k(k_vel_coarse<T>, 1, 1024, 0, s, d, eta, u, rhs, sweeps);
  note_launch();
}
template <typename T>
void p_rbgs(const Dims& d, int color, T* u, const T* rhs, cudaStream_t s, int bs) {
  if (d.h[0] == d.h[1] && d.h[1] == d.h[2] && d.nc < ((i64)1 << 31)) {
    const int by = std::max(1, bs / 32);
    dim3 grid((d.n[0] / 2 + 1 + 31) / 32, (d.n[1] + by - 1) / by, d.n[2]);
    launch_k(k_p_rbgs_u<T>, grid, dim3(32, by), 0, s, d, (T)(d.h[0] * d.h[0]), color, u, rhs);
  } else {
    const ColorMap m = make_color_map_cells(d);
    launch_k(k_p_rbgs<T>, nblk(m.cnt[0], bs), bs, 0, s, d, m, color, u, rhs);
  }
  note_launch();
}
template <typename T>
void p_first(const Dims& d, T* u, const T* rhs, cudaStream_t s) {
  launch_k(k_p_first<T>, nblk(d.nc, 256), 256, 0, s, d, u, rhs);
  note_launch();
}
template <typename T>
void p_restrict_res(const Dims& df, const Dims& dc, int3 cz, const T* uf, const T* rhsf, T* rc, cudaStream_t s) {
  launch_k(k_p_restrict_res<T>, nblk(kRestrictLanes * dc.nc, 256), 256, 0, s, df, dc, cz, uf, rhsf, rc);
  note_launch();
}
template <typename T>
void p_prolong(const Dims& df, const Dims& dc, int3 cz, const T* uc, T* uf, cudaStream_t s) {
  launch_k(k_p_prolong<T>, nblk(df.nc, 256), 256, 0, s, df, dc, cz, uc, uf);
  note_launch();
}
template <typename T>
void p_coarse(const Dims& d, T* u, T* rhs, int sweeps, cudaStream_t s) {
  launch_k(k_p_coarse<T>, 1, 1024, 0, s, d, u, rhs, sweeps);
  note_launch();
}
template <typename T>
void div_q(const Dims& d, T eta, const T* vt, const T* rpi, T* q, T* pi, double* pi64, cudaStream_t s) {
  launch_k(k_div_q<T>, nblk(d.nc, 256), 256, 0, s, d, eta, vt, rpi, q, pi, pi64);
  note_launch();
}
template <typename T>
void add_grad(const Dims& d, const T* phi, T* v, double* v64, cudaStream_t s) {
  launch_k(k_add_grad<T>, nblk(d.fo[3], 256), 256, 0, s, d, phi, v, v64);
  note_launch();
}

#define INST(T)                                                                                  \
  template void stokes_apply<T>(const Dims&, T, const T*, const T*, T*, T*, cudaStream_t, int);  \
  template void vel_rbgs<T>(const Dims&, T, int, T*, const T*, cudaStream_t, int);               \
  template void vel_first<T>(const Dims&, T, T*, const T*, cudaStream_t);                         \
  template bool vel_first2<T>(const Dims&, T, T*, const T*, cudaStream_t, int);                   \
  template bool p_first2<T>(const Dims&, T*, const T*, cudaStream_t, int);                        \
  template void vel_restrict_res<T>(const Dims&, const Dims&, int3, T, const T*, const T*, T*, cudaStream_t); \
  template void p_first<T>(const Dims&, T*, const T*, cudaStream_t);                              \
  template void p_restrict_res<T>(const Dims&, const Dims&, int3, const T*, const T*, T*, cudaStream_t); \
  template void vel_prolong<T>(const Dims&, const Dims&, int3, const T*, T*, cudaStream_t);      \
  template void vel_coarse<T>(const Dims&, T, T*, const T*, int, cudaStream_t);                  \
  template void p_rbgs<T>(const Dims&, int, T*, const T*, cudaStream_t, int);                    \
  template void p_prolong<T>(const Dims&, const Dims&, int3, const T*, T*, cudaStream_t);        \
  template void p_coarse<T>(const Dims&, T*, T*, int, cudaStream_t);                             \
  template void div_q<T>(const Dims&, T, const T*, const T*, T*, T*, double*, cudaStream_t);     \
  template void add_grad<T>(const Dims&, const T*, T*, double*, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace rbfib
