// Exact solve of a coarse multigrid level by fast diagonalisation.  On a
// uniform box level every grid of the projection preconditioner has a
// separable operator: a velocity component of -eta LL (Sec. III.A; the
// ghost-reflection rows at tangential walls and the Dirichlet rows at the
// wall-normal boundary faces) and the Neumann pressure operator -D G are
// Kronecker sums of 1D second differences, one per axis.  Their eigenvectors
// are sine / cosine / Fourier bases in closed form, so the level solve is
// three 1D transforms, a diagonal scaling and three transforms back, done in
// shared memory.  This is the coarsest solve of the
// V-cycles; the bases are built on the host once per grid and checked
// against the explicit 1D matrices.  Each grid is solved by one cluster of
// CTAs that split its z-planes (see k_fd_solve).
#include <cmath>
#include <mutex>

#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.cuh"

namespace rbfib {
namespace {

enum AxisKind { kDirichlet, kGhost, kNeumann, kPeriodic };

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
      if (nb >= 0 && nb < m) T[(size_t)j * m + nb] -= 1.0;
      else if (kind == kGhost) T[(size_t)j * m + j] += 1.0;
      else if (kind == kNeumann) T[(size_t)j * m + j] -= 1.0;
    }
  }
}

// Orthonormal eigenvectors Q[j * m + k] = q_k(j) and eigenvalues of the
// matrix above: DST-I (Dirichlet), DST-II (ghost), DCT-II (Neumann), real
// Fourier (periodic).  lam_0 = 0 exactly for the Neumann and periodic kinds.
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
  else fd_columns<32>(cl, A, Q2, QT2, L0, L1, L2, G.scale, e0, e1, e2, pz, rank);
  cl.sync();
  fd_pass_xy<1>(A, B, QT1, e0, e1, np);
  fd_pass_xy<0>(B, A, QT0, e0, e1, np);
  for (int t = threadIdx.x; t < np * pl; t += blockDim.x) u[G.off + (long long)z0 * pl + t] = A[t];
}

}  // namespace

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
      if (e[ax] < 1 || e[ax] > kFDLine) return fail("extent");
    }
    if (n > kFDMaxPoints) return fail("points");
    G.off = faces ? d.fo[g] : 0;
    G.scale = faces ? (float)eta : 1.0f;
    G.tab0 = (int)tab.size();
    for (int ax = 0; ax < 3; ++ax) {
      AxisKind kind;
      if (d.per[ax]) kind = kPeriodic;
      else if (!faces) kind = kNeumann;
      else kind = (ax == g) ? kDirichlet : kGhost;
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
  k_fd_solve<<<P.ng * kFDCtas, kFDThreads, P.smem, s>>>(P, u, rhs);
  note_launch();
}

}  // namespace rbfib
