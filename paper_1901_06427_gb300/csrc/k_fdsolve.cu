// Exact solve of a coarse multigrid level by fast diagonalisation.  On a
// uniform box level every grid of the projection preconditioner has a
// separable operator: a velocity component of -eta LL (Sec. III.A; the
// ghost-reflection rows at tangential walls and the Dirichlet rows at the
// wall-normal boundary faces) and the Neumann pressure operator -D G are
// Kronecker sums of 1D second differences, one per axis.  Their eigenvectors
// are sine / cosine / Fourier bases in closed form, so the level solve is
// three 1D transforms, a diagonal scaling and three transforms back, done by
// one CTA per grid in shared memory.  This is the coarsest solve of the
// V-cycles; the bases are built on the host once per grid and checked
// against the explicit 1D matrices.
#include <cmath>
#include <mutex>

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

// One 1D transform along axis AX: out[.., c, ..] = sum_t M[t * e + c] in[.., t, ..].
template <int AX>
RBFIB_DEVFN void fd_pass(const float* __restrict__ in, float* __restrict__ out, const float* __restrict__ M, int e0,
                         int e1, int e2) {
  const int n = e0 * e1 * e2;
  const int e = AX == 0 ? e0 : (AX == 1 ? e1 : e2);
  const int st = AX == 0 ? 1 : (AX == 1 ? e0 : e0 * e1);
  for (int o = threadIdx.x; o < n; o += blockDim.x) {
    int c;
    if (AX == 0) c = o % e0;
    else if (AX == 1) c = (o / e0) % e1;
    else c = o / (e0 * e1);
    const float* src = in + (o - c * st);
    float acc = 0.f;
    for (int t = 0; t < e; ++t) acc = fmaf(M[t * e + c], src[t * st], acc);
    out[o] = acc;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(1024) k_fd_solve(FDParams P, float* __restrict__ u, const float* __restrict__ rhs) {
  extern __shared__ float fsm[];
  const FDGrid& G = P.g[blockIdx.x];
  const int e0 = G.e[0], e1 = G.e[1], e2 = G.e[2], n = e0 * e1 * e2;
  float* A = fsm;
  float* B = A + n;
  float* M = B + n;
  for (int t = threadIdx.x; t < G.tabn; t += blockDim.x) M[t] = P.tab[G.tab0 + t];
  for (int t = threadIdx.x; t < n; t += blockDim.x) A[t] = rhs[G.off + t];
  __syncthreads();
  // per axis: Q (forward uses M[t][c] = q_c(t)), Q^T (backward), eigenvalues
  const float* Q0 = M;
  const float* QT0 = Q0 + e0 * e0;
  const float* L0 = QT0 + e0 * e0;
  const float* Q1 = L0 + e0;
  const float* QT1 = Q1 + e1 * e1;
  const float* L1 = QT1 + e1 * e1;
  const float* Q2 = L1 + e1;
  const float* QT2 = Q2 + e2 * e2;
  const float* L2 = QT2 + e2 * e2;
  fd_pass<0>(A, B, Q0, e0, e1, e2);
  fd_pass<1>(B, A, Q1, e0, e1, e2);
  fd_pass<2>(A, B, Q2, e0, e1, e2);
  for (int o = threadIdx.x; o < n; o += blockDim.x) {
    const int i = o % e0, j = (o / e0) % e1, k = o / (e0 * e1);
    const float s = G.scale * (L0[i] + L1[j] + L2[k]);
    B[o] = s > 0.f ? B[o] / s : 0.f;   // the zero mode of a singular grid is dropped
  }
  __syncthreads();
  fd_pass<2>(B, A, QT2, e0, e1, e2);
  fd_pass<1>(A, B, QT1, e0, e1, e2);
  fd_pass<0>(B, A, QT0, e0, e1, e2);
  for (int t = threadIdx.x; t < n; t += blockDim.x) u[G.off + t] = A[t];
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
      if (e[ax] < 1 || e[ax] > kFDMaxExtent) return fail("extent");
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
      const int m = e[ax];
      const double ih2 = 1.0 / (d.h[ax] * d.h[ax]);
      for (int t = 0; t < m; ++t)
        for (int c = 0; c < m; ++c) tab.push_back((float)Q[(size_t)t * m + c]);
      for (int t = 0; t < m; ++t)
        for (int c = 0; c < m; ++c) tab.push_back((float)Q[(size_t)c * m + t]);
      for (int k = 0; k < m; ++k) tab.push_back((float)(lam[k] * ih2));
    }
    G.tabn = (int)tab.size() - G.tab0;
    smem = std::max(smem, (int)((2 * n + G.tabn) * sizeof(float)));
  }
  P.smem = smem;
  return true;
}

void fd_solve(const FDParams& P, float* u, const float* rhs, cudaStream_t s) {
  static std::once_flag f;
  std::call_once(f, [] {
    cudaFuncSetAttribute(k_fd_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)((2 * kFDMaxPoints + 3 * (2 * kFDMaxExtent * kFDMaxExtent + kFDMaxExtent)) * sizeof(float)));
  });
  k_fd_solve<<<P.ng, 1024, P.smem, s>>>(P, u, rhs);
  note_launch();
}

}  // namespace rbfib
