// Exact solve of a coarse multigrid level by fast diagonalisation.  On a
// uniform box level every grid of the projection preconditioner has a
// separable operator: a velocity component of -eta LL (Sec. III.A; the
// ghost-reflection rows at tangential walls, odd at a no-slip and even at a
// free-slip wall, and the Dirichlet rows at the wall-normal boundary faces)
// and the Neumann pressure operator -D G are
// Kronecker sums of 1D second differences, one per axis.  Their eigenvectors
// are sine / cosine / Fourier bases in closed form, so the level solve is
// three 1D transforms, a diagonal scaling and three transforms back, done in
// shared memory.  This is the coarsest solve of the
// V-cycles; the bases are built on the host once per grid and checked
// against the explicit 1D matrices.  Each grid is solved by one cluster of
// CTAs that split its z-planes (see k_fd_solve).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>

#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.cuh"

namespace rbfib {
namespace {

// kGhost: odd ghost at both ends (no-slip walls); kNeumann: even ghost at
// both ends (free-slip walls, and the pressure); kGhostNeumann /
// kNeumannGhost: odd at the low end and even at the high end, or the reverse.
enum AxisKind { kDirichlet, kGhost, kNeumann, kPeriodic, kGhostNeumann, kNeumannGhost };

// The 1D second-difference matrix (times h^2) of one kind: 2 on the
// diagonal, -1 off it; a missing neighbour adds +1 (ghost = -self),
// nothing (Dirichlet boundary value 0) or -1 (Neumann, ghost = self);
// periodic rows wrap.
void axis_matrix(AxisKind kind, int m, std::vector<double>& T) {
  T.assign((size_t)m * m, 0.0);
  for (int j = 0; j < m; ++j) {
    T[(size_t)j * m + j] += 2.0;
    for (int s = -1; s <= 1; s += 2) {
      int nb = j + s;
      if (kind == kPeriodic) { nb = (nb + m) % m; T[(size_t)j * m + nb] -= 1.0; continue; }
      if (nb >= 0 && nb < m) { T[(size_t)j * m + nb] -= 1.0; continue; }
      const bool odd = kind == kGhost || (kind == kGhostNeumann && s < 0) || (kind == kNeumannGhost && s > 0);
      const bool even = kind == kNeumann || (kind == kGhostNeumann && s > 0) || (kind == kNeumannGhost && s < 0);
      if (odd) T[(size_t)j * m + j] += 1.0;
      else if (even) T[(size_t)j * m + j] -= 1.0;
    }
  }
}

// Orthonormal eigenvectors Q[j * m + k] = q_k(j) and eigenvalues of the
// matrix above: DST-I (Dirichlet), DST-II (ghost), DCT-II (Neumann), DST-IV
// (odd low end, even high end), DCT-IV (the reverse), real Fourier
// (periodic).  lam_0 = 0 exactly for the Neumann and periodic kinds.
void axis_basis(AxisKind kind, int m, std::vector<double>& Q, std::vector<double>& lam) {
  const double pi = 3.14159265358979323846;
  Q.assign((size_t)m * m, 0.0);
  lam.assign(m, 0.0);
  for (int k = 0; k < m; ++k) {
    double th = 0.0, c = 0.0;
    for (int j = 0; j < m; ++j) {
      double v = 0.0;
      switch (kind) {
        case kDirichlet:
          th = pi * (k + 1) / (m + 1);
          c = std::sqrt(2.0 / (m + 1));
          v = c * std::sin(th * (j + 1));
          break;
        case kGhost:
          th = pi * (k + 1) / m;
          c = std::sqrt((k == m - 1 ? 1.0 : 2.0) / m);
          v = c * std::sin(th * (j + 0.5));
          break;
        case kNeumann:
          th = pi * k / m;
          c = std::sqrt((k == 0 ? 1.0 : 2.0) / m);
          v = c * std::cos(th * (j + 0.5));
          break;
        case kGhostNeumann:
          th = pi * (k + 0.5) / m;
          v = std::sqrt(2.0 / m) * std::sin(th * (j + 0.5));
          break;
        case kNeumannGhost:
          th = pi * (k + 0.5) / m;
          v = std::sqrt(2.0 / m) * std::cos(th * (j + 0.5));
          break;
        case kPeriodic: {
          // columns: constant; cos / sin pairs of frequency r; (-1)^j for even m
          const int r = (k + 1) / 2;
          th = 2.0 * pi * r / m;
          if (k == 0) v = std::sqrt(1.0 / m);
          else if (2 * r == m) v = std::sqrt(1.0 / m) * ((j & 1) ? -1.0 : 1.0);
          else if (k & 1) v = std::sqrt(2.0 / m) * std::cos(th * j);
          else v = std::sqrt(2.0 / m) * std::sin(th * j);
          break;
        }
      }
      Q[(size_t)j * m + k] = v;
    }
    lam[k] = (k == 0 && (kind == kNeumann || kind == kPeriodic)) ? 0.0 : 2.0 - 2.0 * std::cos(th);
  }
}

// max |T Q - Q diag(lam)| and max |Q^T Q - I|
bool basis_ok(AxisKind kind, int m, const std::vector<double>& Q, const std::vector<double>& lam) {
  std::vector<double> T;
  axis_matrix(kind, m, T);
  double e1 = 0.0, e2 = 0.0;
  for (int i = 0; i < m; ++i)
    for (int k = 0; k < m; ++k) {
      double r = -Q[(size_t)i * m + k] * lam[k], o = (i == k) ? -1.0 : 0.0;
      for (int j = 0; j < m; ++j) {
        r += T[(size_t)i * m + j] * Q[(size_t)j * m + k];
        o += Q[(size_t)j * m + i] * Q[(size_t)j * m + k];
      }
      e1 = std::fmax(e1, std::fabs(r));
      e2 = std::fmax(e2, std::fabs(o));
    }
  return e1 <= 1e-12 * 4.0 * m && e2 <= 1e-13 * m;
}

// Basis rows in the table are padded to a multiple of 8 floats (zeros), so
// that chunks of outputs read whole 16-byte words inside their row.
RBFIB_DEVFN int fd_pad(int e) { return (e + 7) & ~7; }

// One 1D transform along x (AX = 0) or y (AX = 1) of the planes [0, np) of a
// slab (e0 x e1 x np, x fastest): out[.., c, ..] = sum_t M[t * ep + c] in[.., t, ..].
// A thread takes kFDChunk consecutive outputs of one line (chunk-major order,
// so a warp shares the basis rows, read as broadcast 16-byte loads) and keeps
// them in registers while it walks the line's inputs once.
constexpr int kFDChunk = 16;
template <int AX>
__device__ __noinline__ void fd_pass_xy(const float* __restrict__ in, float* __restrict__ out,
                                        const float* __restrict__ M, int e0, int e1, int np) {
  const int e = AX == 0 ? e0 : e1;
  const int ep = fd_pad(e);
  const int st = AX == 0 ? 1 : e0;
  const int nlines = (AX == 0 ? e1 : e0) * np;
  const int nchunks = (e + kFDChunk - 1) / kFDChunk;
  for (int it = threadIdx.x; it < nlines * nchunks; it += blockDim.x) {
    const int ch = it / nlines, L = it - ch * nlines;
    const int base = AX == 0 ? L * e0 : (L % e0) + e0 * e1 * (L / e0);
    const int c0 = ch * kFDChunk;
    // 16-byte words of the chunk inside the padded row (ep = e rounded up to
    // 8); outputs past e come from the zero padding and are not stored
    const int nq = min(kFDChunk, ep - c0) / 4;
    float acc[kFDChunk];
#pragma unroll
    for (int c = 0; c < kFDChunk; ++c) acc[c] = 0.f;
    const float* row = M + c0;
    const float* src = in + base;
#pragma unroll 2
    for (int t = 0; t < e; ++t) {
      const float xt = src[t * st];
      const float4* r4 = reinterpret_cast<const float4*>(row + t * ep);
#pragma unroll
      for (int q = 0; q < kFDChunk / 4; ++q) {
        if (q < nq) {
          const float4 m = r4[q];
          acc[4 * q] = fmaf(m.x, xt, acc[4 * q]);
          acc[4 * q + 1] = fmaf(m.y, xt, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(m.z, xt, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(m.w, xt, acc[4 * q + 3]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < kFDChunk; ++c)
      if (c0 + c < e) out[base + (c0 + c) * st] = acc[c];
  }
  __syncthreads();
}

// The z-columns of one grid (e_z <= E, E a multiple of 8), spread over the
// threads of the cluster: each column is read from the CTAs owning its
// planes, transformed forward, scaled by the inverse eigenvalues, transformed
// back and written to the same places.
template <int E>
__device__ __noinline__ void fd_columns(cooperative_groups::cluster_group& cl, float* A, const float* Q2,
                                        const float* QT2, const float* L0, const float* L1, const float* L2,
                                        float scale, int e0, int e1, int e2, int pz, int rank) {
  const int pl = e0 * e1, p2 = fd_pad(e2);
  for (int col = rank * blockDim.x + threadIdx.x; col < pl; col += kFDCtas * blockDim.x) {
    const int i = col % e0, j = col / e0;
    float x[E], y[E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
      x[k] = 0.f;
      if (k < e2) {
        const int owner = k / pz;
        x[k] = cl.map_shared_rank(A, owner)[(k - owner * pz) * pl + col];
      }
    }
    const float sxy = L0[i] + L1[j];
#pragma unroll
    for (int c = 0; c < E; ++c) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < E; ++k) acc = fmaf(Q2[min(k, e2 - 1) * p2 + c], x[k], acc);   // x[k] = 0 past e2
      const float s = scale * (sxy + L2[c]);
      y[c] = (c < e2 && s > 0.f) ? acc / s : 0.f;   // the zero mode of a singular grid is dropped
    }
#pragma unroll
    for (int k = 0; k < E; ++k) {
      float acc = 0.f;
#pragma unroll
      for (int c = 0; c < E; ++c) acc = fmaf(QT2[min(c, e2 - 1) * p2 + k], y[c], acc);   // y[c] = 0 past e2
      if (k < e2) {
        const int owner = k / pz;
        cl.map_shared_rank(A, owner)[(k - owner * pz) * pl + col] = acc;
      }
    }
  }
}

// One cluster of kFDCtas CTAs per grid.  CTA r owns the z-planes
// [r pz, (r + 1) pz) of its grid in shared memory.  Forward x and y
// transforms on the own planes; cluster barrier; each thread then takes whole
// z-columns (read through distributed shared memory into registers), applies
// the forward z transform, the eigenvalue scaling and the backward z
// transform, and writes the column back; cluster barrier; backward y and x
// transforms on the own planes.
__global__ void __cluster_dims__(kFDCtas, 1, 1) __launch_bounds__(kFDThreads)
    k_fd_solve(FDParams P, float* __restrict__ u, const float* __restrict__ rhs) {
  pdl_entry();
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) float fsm[];
  const FDGrid& G = P.g[blockIdx.x / kFDCtas];
  const int rank = (int)cl.block_rank();
  const int e0 = G.e[0], e1 = G.e[1], e2 = G.e[2], pl = e0 * e1;
  const int pz = (e2 + kFDCtas - 1) / kFDCtas;
  const int z0 = min(e2, rank * pz), np = min(e2, z0 + pz) - z0;
  // table (16-byte aligned rows), then the two slab buffers
  float* M = fsm;
  float* A = M + ((G.tabn + 3) & ~3);
  float* B = A + ((pz * pl + 3) & ~3);
  // Staging by asynchronous copies, all issued before the one wait: the table
  // in 16-byte words (every grid's segment starts on a 16-byte boundary of
  // the table and is zero-padded to whole words; M and A are 16-byte aligned)
  // and the own planes of the right-hand side element by element.
  {
    const unsigned msm = (unsigned)__cvta_generic_to_shared(M);
    const float4* tab4 = reinterpret_cast<const float4*>(P.tab + G.tab0);
    const int nw = (G.tabn + 3) >> 2;
    for (int t = threadIdx.x; t < nw; t += blockDim.x)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(msm + 16u * (unsigned)t), "l"(tab4 + t)
                   : "memory");
    const unsigned asm0 = (unsigned)__cvta_generic_to_shared(A);
    const float* src = rhs + G.off + (long long)z0 * pl;
    for (int t = threadIdx.x; t < np * pl; t += blockDim.x)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(asm0 + 4u * (unsigned)t), "l"(src + t)
                   : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  }
  __syncthreads();
  // per axis: Q (forward uses M[t][c] = q_c(t)), Q^T (backward), both e x ep,
  // then the eigenvalues (padded to ep); ep = e rounded up to 8
  const int p0 = fd_pad(e0), p1 = fd_pad(e1), p2 = fd_pad(e2);
  const float* Q0 = M;
  const float* QT0 = Q0 + e0 * p0;
  const float* L0 = QT0 + e0 * p0;
  const float* Q1 = L0 + p0;
  const float* QT1 = Q1 + e1 * p1;
  const float* L1 = QT1 + e1 * p1;
  const float* Q2 = L1 + p1;
  const float* QT2 = Q2 + e2 * p2;
  const float* L2 = QT2 + e2 * p2;
  fd_pass_xy<0>(A, B, Q0, e0, e1, np);
  fd_pass_xy<1>(B, A, Q1, e0, e1, np);
  cl.sync();
  // z-columns: forward transform, scaling, backward transform, in registers
  const int rz = (e2 + 7) & ~7;
  if (rz == 8) fd_columns<8>(cl, A, Q2, QT2, L0, L1, L2, G.scale, e0, e1, e2, pz, rank);
  else if (rz == 16) fd_columns<16>(cl, A, Q2, QT2, L0, L1, L2, G.scale, e0, e1, e2, pz, rank);
  else if (rz == 24) fd_columns<24>(cl, A, Q2, QT2, L0, L1, L2, G.scale, e0, e1, e2, pz, rank);
  else if (rz == 32) fd_columns<32>(cl, A, Q2, QT2, L0, L1, L2, G.scale, e0, e1, e2, pz, rank);
  else if (rz == 40) fd_columns<40>(cl, A, Q2, QT2, L0, L1, L2, G.scale, e0, e1, e2, pz, rank);
  else fd_columns<48>(cl, A, Q2, QT2, L0, L1, L2, G.scale, e0, e1, e2, pz, rank);
  cl.sync();
  fd_pass_xy<1>(A, B, QT1, e0, e1, np);
  fd_pass_xy<0>(B, A, QT0, e0, e1, np);
  for (int t = threadIdx.x; t < np * pl; t += blockDim.x) u[G.off + (long long)z0 * pl + t] = A[t];
}

// ------------------------------------------------------------------------
// The same solve spread over the whole GPU, in three launches: the forward x
// and y transforms of every z-plane (one CTA per plane of every grid), the z
// transform, eigenvalue scaling and backward z transform of every column
// (one CTA per 32 adjacent columns), and the backward y and x transforms of
// every plane.  The level arrays stay in L2 between the launches.  On a fine
// level (up to kFDLine points per axis: the whole two-sphere grid) the
// cluster kernel above leaves most SMs idle; this form uses a CTA per plane.

// 16 x 16 threads per plane, each owning a 3 x 3 register tile of the (at
// most 48 x 48) plane.
constexpr int kFWT = 16;
constexpr int kFWR = kFDLine / kFWT;
static_assert(kFWT * kFWR == kFDLine, "register tile covers a line");

RBFIB_DEVFN int fd_planes(const FDGrid& G) { return G.e[2]; }
RBFIB_DEVFN int fd_col_tiles(const FDGrid& G) { return (G.e[0] * G.e[1] + 31) / 32; }

// Block index -> (grid gi, item k within the grid), items counted by f.
template <int (*F)(const FDGrid&)>
RBFIB_DEVFN void fd_item(const FDParams& P, int& k, int& gi) {
  gi = 0;
  while (gi < P.ng - 1 && k >= F(P.g[gi])) { k -= F(P.g[gi]); ++gi; }
}

// cp.async helpers: 16-byte and 4-byte global -> shared copies, one wait.
RBFIB_DEVFN void fdw_cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src) : "memory");
}
RBFIB_DEVFN void fdw_cp4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src) : "memory");
}
RBFIB_DEVFN void fdw_wait() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Stages the first e columns of the e rows of a basis table (rows padded to
// fd_pad(e) floats, 16-byte aligned) into M[kFDLine][kFDLine] by 16-byte
// copies (the words past e carry the table's zero padding, or a neighbouring
// column that is never read).
RBFIB_DEVFN void fdw_stage_basis(float (*M)[kFDLine], const float* tab, int e) {
  const int ep = fd_pad(e), wpr = (e + 3) >> 2;
  for (int t = threadIdx.x; t < e * wpr; t += blockDim.x) {
    const int r = t / wpr, w = t - r * wpr;
    fdw_cp16(&M[r][4 * w], tab + r * ep + 4 * w);
  }
}

// One plane, one chunk of kFWT output columns (blockIdx.y): out = A_y (in
// A_x), the 1D transforms along x then y, with the forward bases (dir 0) or
// their transposes (dir 1).  Both transforms keep the output column: column
// c of A_x acts on the rows of the plane, and the y transform mixes rows of
// the same column, so a plane's columns split over independent CTAs (three
// per plane of 48 points, which keeps more SMs busy than one CTA per plane).
// 16 x 16 threads: thread (tx, ty) owns column c0 + tx of rows ty + 16 a.
__global__ void __launch_bounds__(kFWT * kFWT) k_fdw_xy(FDParams P, const float* __restrict__ in,
                                                         float* __restrict__ out, int dir) {
  pdl_entry();
  __shared__ float X[kFDLine][kFDLine + 1];
  __shared__ float T[kFDLine][kFWT + 1];
  __shared__ __align__(16) float Mx[kFDLine][kFWT];
  __shared__ __align__(16) float My[kFDLine][kFDLine];
  int k = blockIdx.x, gi;
  fd_item<fd_planes>(P, k, gi);
  const FDGrid& G = P.g[gi];
  const int e0 = G.e[0], e1 = G.e[1], p0 = fd_pad(e0), p1 = fd_pad(e1);
  const int c0 = blockIdx.y * kFWT;
  if (c0 >= e0) return;
  const float* Q0 = P.tab + G.tab0;
  const float* QT0 = Q0 + e0 * p0;
  const float* Q1 = QT0 + e0 * p0 + p0;
  const float* QT1 = Q1 + e1 * p1;
  const float* ax = dir ? QT0 : Q0;
  const int tx = threadIdx.x % kFWT, ty = threadIdx.x / kFWT;
  // every copy issued before the one wait: the chunk's columns of A_x (rows
  // padded to 8 floats, so the 16 columns from c0 are four whole 16-byte
  // words inside the row), A_y and the plane
  for (int t = threadIdx.x; t < e0 * (kFWT / 4); t += blockDim.x) {
    const int r = t / (kFWT / 4), w = t - r * (kFWT / 4);
    if (c0 + 4 * w < p0) fdw_cp16(&Mx[r][4 * w], ax + r * p0 + c0 + 4 * w);
  }
  fdw_stage_basis(My, dir ? QT1 : Q1, e1);
  const float* src = in + G.off + (long long)k * e0 * e1;
  for (int r = ty; r < e1; r += kFWT)
    for (int c = tx; c < e0; c += kFWT) fdw_cp4(&X[r][c], src + r * e0 + c);
  fdw_wait();
  __syncthreads();
  // T[j][c] = sum_i X[j][i] A_x[i][c0 + c]  (rows j >= e1 are never read back)
  float acc[kFWR];
#pragma unroll
  for (int a = 0; a < kFWR; ++a) acc[a] = 0.f;
#pragma unroll 4
  for (int i = 0; i < e0; ++i) {
    const float m = Mx[i][tx];
#pragma unroll
    for (int a = 0; a < kFWR; ++a) acc[a] = fmaf(X[ty + kFWT * a][i], m, acc[a]);
  }
#pragma unroll
  for (int a = 0; a < kFWR; ++a) {
    T[ty + kFWT * a][tx] = acc[a];
    acc[a] = 0.f;
  }
  __syncthreads();
  // out[r][c] = sum_j A_y[j][r] T[j][c]
#pragma unroll 4
  for (int j = 0; j < e1; ++j) {
    const float t = T[j][tx];
#pragma unroll
    for (int a = 0; a < kFWR; ++a) acc[a] = fmaf(My[j][ty + kFWT * a], t, acc[a]);
  }
  float* dst = out + G.off + (long long)k * e0 * e1;
  const int c = c0 + tx;
#pragma unroll
  for (int a = 0; a < kFWR; ++a) {
    const int r = ty + kFWT * a;
    if (r < e1 && c < e0) dst[r * e0 + c] = acc[a];
  }
}

// 32 adjacent columns (fixed x, y; all z) of one grid, in place: forward z
// transform, division by s (l_x + l_y + l_z) (the zero mode of a singular
// grid dropped), backward z transform.  Thread (column ci, group gr) forms
// the coefficients gr, gr + 8, ... of its column.
__global__ void __launch_bounds__(256) k_fdw_z(FDParams P, float* __restrict__ data) {
  pdl_entry();
  __shared__ float Z[kFDLine][33];
  __shared__ __align__(16) float Mz[kFDLine][kFDLine];
  __shared__ __align__(16) float MzT[kFDLine][kFDLine];
  int tile = blockIdx.x, gi;
  fd_item<fd_col_tiles>(P, tile, gi);
  const FDGrid& G = P.g[gi];
  const int e0 = G.e[0], e1 = G.e[1], e2 = G.e[2], pl = e0 * e1;
  const int p0 = fd_pad(e0), p1 = fd_pad(e1), p2 = fd_pad(e2);
  const float* L0 = P.tab + G.tab0 + 2 * e0 * p0;
  const float* L1 = L0 + p0 + 2 * e1 * p1;
  const float* Q2 = L1 + p1;
  const float* QT2 = Q2 + e2 * p2;
  const float* L2 = QT2 + e2 * p2;
  fdw_stage_basis(Mz, Q2, e2);
  fdw_stage_basis(MzT, QT2, e2);
  const int col0 = tile * 32;
  float* base = data + G.off;
  {
    const int c = threadIdx.x & 31;
    if (col0 + c < pl)
      for (int kk = threadIdx.x >> 5; kk < e2; kk += 8) fdw_cp4(&Z[kk][c], base + (long long)kk * pl + col0 + c);
  }
  fdw_wait();
  __syncthreads();
  const int ci = threadIdx.x & 31, gr = threadIdx.x >> 5;
  const int col = col0 + ci;
  const bool live = col < pl;
  const float sxy = live ? L0[col % e0] + L1[col / e0] : 0.f;
  float y[kFDLine / 8];
#pragma unroll
  for (int q = 0; q < kFDLine / 8; ++q) {
    const int c = gr + 8 * q;
    float acc = 0.f;
    if (c < e2 && live) {
#pragma unroll 4
      for (int kk = 0; kk < e2; ++kk) acc = fmaf(Mz[kk][c], Z[kk][ci], acc);
      const float s = G.scale * (sxy + L2[c]);
      acc = s > 0.f ? acc / s : 0.f;
    }
    y[q] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kFDLine / 8; ++q) {
    const int c = gr + 8 * q;
    if (c < e2) Z[c][ci] = y[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kFDLine / 8; ++q) {
    const int kk = gr + 8 * q;
    if (kk < e2 && live) {
      float acc = 0.f;
#pragma unroll 4
      for (int c = 0; c < e2; ++c) acc = fmaf(MzT[c][kk], Z[c][ci], acc);
      base[(long long)kk * pl + col] = acc;
    }
  }
}

}  // namespace

// Whole-GPU form of fd_solve: tmp holds the level's transformed coefficients
// (as many floats as u).
void fd_solve_wide(const FDParams& P, float* u, const float* rhs, float* tmp, cudaStream_t s) {
  int planes = 0, tiles = 0;
  for (int g = 0; g < P.ng; ++g) {
    planes += P.g[g].e[2];
    tiles += (P.g[g].e[0] * P.g[g].e[1] + 31) / 32;
  }
  int chunks = 1;
  for (int g = 0; g < P.ng; ++g) chunks = std::max(chunks, (P.g[g].e[0] + kFWT - 1) / kFWT);
  launch_k(k_fdw_xy, dim3(planes, chunks), kFWT * kFWT, 0, s, P, rhs, tmp, 0);
  note_launch();
  launch_k(k_fdw_z, tiles, 256, 0, s, P, tmp);
  note_launch();
  launch_k(k_fdw_xy, dim3(planes, chunks), kFWT * kFWT, 0, s, P, (const float*)tmp, u, 1);
  note_launch();
}

// The whole-GPU form for levels whose largest grid has more than
// kFDWideMin points (the cluster kernel is faster on the small coarse levels,
// e.g. 17 against 19 us at 24 x 24 x 16); RBFIB_FD_WIDE_MIN overrides the
// threshold (read once).
constexpr long long kFDWideMin = 32768;
bool fd_use_wide(const FDParams& P) {
  static const long long lim = [] {
    const char* e = std::getenv("RBFIB_FD_WIDE_MIN");
    return e ? std::atoll(e) : kFDWideMin;
  }();
  long long m = 0;
  for (int g = 0; g < P.ng; ++g) m = std::max(m, (long long)P.g[g].e[0] * P.g[g].e[1] * P.g[g].e[2]);
  return m > lim;
}

// Longest line solved by fast diagonalisation: kFDLine, or a smaller value
// from RBFIB_FD_LINE (read once; for measurements of the multigrid levels
// above the exact solve).
int fd_line_limit() {
  static const int lim = [] {
    const char* e = std::getenv("RBFIB_FD_LINE");
    const int v = e ? std::atoi(e) : kFDLine;
    return (v >= 1 && v <= kFDLine) ? v : kFDLine;
  }();
  return lim;
}

bool fd_plan(const Dims& d, bool faces, double eta, std::vector<float>& tab, FDParams& P, std::string& why) {
  P = FDParams{};
  P.ng = faces ? 3 : 1;
  const size_t tab_start = tab.size();
  auto fail = [&](const char* w) { why = w; tab.resize(tab_start); return false; };
  int smem = 0;
  for (int g = 0; g < P.ng; ++g) {
    FDGrid& G = P.g[g];
    const int* e = faces ? d.fe[g] : d.n;
    long long n = 1;
    for (int ax = 0; ax < 3; ++ax) {
      G.e[ax] = e[ax];
      n *= e[ax];
      if (e[ax] < 1 || e[ax] > fd_line_limit()) return fail("extent");
    }
    if (n > kFDMaxPoints) return fail("points");
    G.off = faces ? d.fo[g] : 0;
    G.scale = faces ? (float)eta : 1.0f;
    G.tab0 = (int)tab.size();
    for (int ax = 0; ax < 3; ++ax) {
      AxisKind kind;
      if (d.per[ax]) kind = kPeriodic;
      else if (!faces) kind = kNeumann;
      else if (ax == g) kind = kDirichlet;
      else {
        const bool even_lo = ghost_sign(d, 2 * ax) > 0, even_hi = ghost_sign(d, 2 * ax + 1) > 0;
        kind = even_lo ? (even_hi ? kNeumann : kNeumannGhost) : (even_hi ? kGhostNeumann : kGhost);
      }
      std::vector<double> Q, lam;
      axis_basis(kind, e[ax], Q, lam);
      if (!basis_ok(kind, e[ax], Q, lam)) return fail("basis check");
      const int m = e[ax], mp = (m + 7) & ~7;
      const double ih2 = 1.0 / (d.h[ax] * d.h[ax]);
      for (int t = 0; t < m; ++t)
        for (int c = 0; c < mp; ++c) tab.push_back(c < m ? (float)Q[(size_t)t * m + c] : 0.f);
      for (int t = 0; t < m; ++t)
        for (int c = 0; c < mp; ++c) tab.push_back(c < m ? (float)Q[(size_t)c * m + t] : 0.f);
      for (int c = 0; c < mp; ++c) tab.push_back(c < m ? (float)(lam[c] * ih2) : 0.f);
    }
    G.tabn = (int)tab.size() - G.tab0;
    // every grid's segment starts on a 16-byte boundary of the table
    while (tab.size() % 4) tab.push_back(0.f);
    const long long slab = (long long)((e[2] + kFDCtas - 1) / kFDCtas) * e[0] * e[1];
    smem = std::max(smem, (int)((((G.tabn + 3) & ~3) + 2 * ((slab + 3) & ~3)) * sizeof(float)));
  }
  P.smem = smem;
  return true;
}

void fd_solve(const FDParams& P, float* u, const float* rhs, cudaStream_t s) {
  static std::once_flag f;
  std::call_once(f, [] {
    cudaFuncSetAttribute(k_fd_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, kFDMaxSmem);
  });
  launch_k(k_fd_solve, P.ng * kFDCtas, kFDThreads, P.smem, s, P, u, rhs);
  note_launch();
}

}  // namespace rbfib
