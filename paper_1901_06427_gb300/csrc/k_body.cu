// Coupled body block of the preconditioner for suspensions with few blobs:
// the Schur complement [-M K; K^T 0] of the saddle operator with the blob
// mobility M replaced by the free-space Rotne-Prager-Yamakawa mobility of all
// blobs of all bodies (inter-body coupling included).  Built once per
// configuration: dense RPY matrix; its inverse (FP32) by in-place
// Gauss-Jordan (no pivoting: the RPY matrix is symmetric positive definite)
// or, when the previous configuration's inverse is close, by two
// Newton-Schulz steps from it; P = M^-1 K; N = (K^T M^-1 K)^-1 (FP64).
// Applied by one cluster of CTAs.
#include <algorithm>
#include <cmath>

#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.cuh"

namespace rbfib {

static inline unsigned nblk(i64 n, int bs) { return (unsigned)((n + bs - 1) / bs); }

__global__ void k_rpy_full(int nbl, const double* __restrict__ r, double a, double eta, float* __restrict__ M) {
  pdl_entry();
  const i64 n3 = 3 * (i64)nbl;
  const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n3 * n3) return;
  const int row = (int)(t / n3), col = (int)(t - (i64)row * n3);
  const int i = row / 3, p = row % 3, j = col / 3, q = col % 3;
  const double c0 = 1.0 / (6.0 * M_PI * eta * a);
  double v;
  if (i == j) {
    v = (p == q) ? c0 : 0.0;
  } else {
    const double d[3] = {r[3 * i] - r[3 * j], r[3 * i + 1] - r[3 * j + 1], r[3 * i + 2] - r[3 * j + 2]};
    const double rr2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double rr = sqrt(rr2);
    double fI, fR;
    if (rr >= 2.0 * a) {
      const double c = 1.0 / (8.0 * M_PI * eta * rr);
      fI = c * (1.0 + 2.0 * a * a / (3.0 * rr2));
      fR = c * (1.0 - 2.0 * a * a / rr2);
    } else {
      fI = c0 * (1.0 - 9.0 * rr / (32.0 * a));
      fR = c0 * (3.0 * rr / (32.0 * a));
    }
    v = (p == q ? fI : 0.0) + fR * d[p] * d[q] / rr2;
  }
  M[t] = (float)v;
}

// In-place Gauss-Jordan inverse of an n x n matrix by one block (no
// pivoting; the matrices are symmetric positive definite).  Per pivot k the
// pivot column and row are staged in shared memory, then each warp updates
// whole rows (lanes along the row).  status is set to 1 on a zero pivot.
template <typename R>
__global__ void k_gj_inverse(R* __restrict__ A, int n, int* __restrict__ status) {
  pdl_entry();
  extern __shared__ unsigned char shraw[];
  R* col = (R*)shraw;   // column k
  R* prow = col + n;    // row k
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < n; ++k) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      col[i] = A[(i64)i * n + k];
      prow[i] = A[(i64)k * n + i];
    }
    __syncthreads();
    const R p = prow[k];
    if (!(p > R(0) || p < R(0))) {
      if (threadIdx.x == 0) *status = 1;
      return;
    }
    const R ip = R(1) / p;
    for (int i = wid; i < n; i += nw) {
      R* Ai = A + (i64)i * n;
      if (i == k) {
        for (int j = lane; j < n; j += 32) Ai[j] = (j == k) ? ip : prow[j] * ip;
      } else {
        const R f = col[i] * ip;
        for (int j = lane; j < n; j += 32) Ai[j] = (j == k) ? -f : Ai[j] - f * prow[j];
      }
    }
    __syncthreads();
  }
}

// P = M^-1 K (n3 x 6 nb): column (p, c) of K is nonzero on the blobs of body p
// only: identity for c < 3, w x arm for c >= 3.
__global__ void k_mk(int nbl, int nb, const int* __restrict__ boff, const double* __restrict__ arm,
                     const float* __restrict__ Mi, float* __restrict__ P) {
  pdl_entry();
  const i64 n3 = 3 * (i64)nbl, m = 6 * (i64)nb;
  const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n3 * m) return;
  const int row = (int)(t / m), col = (int)(t - (i64)row * m);
  const int p = col / 6, c = col % 6;
  double acc = 0.0;
  for (int i = boff[p]; i < boff[p + 1]; ++i) {
    const float* Mr = Mi + (i64)row * n3 + 3 * i;
    if (c < 3) {
      acc += Mr[c];
    } else {
      // (w x arm) for w = e_{c-3}: e_x x d = (0, -dz, dy), e_y x d = (dz, 0, -dx), e_z x d = (-dy, dx, 0)
      const double* d = arm + 3 * i;
      double k0, k1, k2;
      if (c == 3) { k0 = 0; k1 = -d[2]; k2 = d[1]; }
      else if (c == 4) { k0 = d[2]; k1 = 0; k2 = -d[0]; }
      else { k0 = -d[1]; k1 = d[0]; k2 = 0; }
      acc += Mr[0] * k0 + Mr[1] * k1 + Mr[2] * k2;
    }
  }
  P[t] = (float)acc;
}

// A = K^T P (6 nb x 6 nb, FP64)
__global__ void k_ktp(int nbl, int nb, const int* __restrict__ boff, const double* __restrict__ arm,
                      const float* __restrict__ P, double* __restrict__ A) {
  pdl_entry();
  const int m = 6 * nb;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * m) return;
  const int row = t / m, col = t - row * m;
  const int p = row / 6, c = row % 6;
  double acc = 0.0;
  for (int i = boff[p]; i < boff[p + 1]; ++i) {
    const double x = P[(i64)(3 * i) * m + col], y = P[(i64)(3 * i + 1) * m + col], z = P[(i64)(3 * i + 2) * m + col];
    const double* d = arm + 3 * i;
    if (c == 0) acc += x;
    else if (c == 1) acc += y;
    else if (c == 2) acc += z;
    else if (c == 3) acc += d[1] * z - d[2] * y;
    else if (c == 4) acc += d[2] * x - d[0] * z;
    else acc += d[0] * y - d[1] * x;
  }
  A[t] = acc;
}

// Square FP32 products for the Newton-Schulz update of the inverse
// (n x n, row-major): MODE 0 forms C = I - A B and adds sum(C_ij^2) to
// *ss; MODE 1 forms C = D + A B.  16 x 16 output tiles on 64 threads (a
// 2 x 2 block of outputs each), so that even n = 252 spreads over 256 CTAs;
// the A rows and B columns of a tile are staged through shared memory in
// k-slices of up to kNSK (one slice for n <= kNSK, all of its loads in
// flight at once), A transposed so that a thread reads its two rows and its
// two columns of a k step as two 8-byte loads.  Entries past n are
// zero-filled.  n <= 1536: these products take microseconds, so they stay
// on the FP32 pipe.
constexpr int kNSTile = 16, kNSK = 256, kNSPad = kNSTile + 2;
template <int MODE>
__global__ void __launch_bounds__(64) k_ns_gemm(int n, const float* __restrict__ A, const float* __restrict__ B,
                                                const float* __restrict__ D, float* __restrict__ C,
                                                double* __restrict__ ss) {
  pdl_entry();
  __shared__ __align__(16) float As[kNSK][kNSPad];   // As[k][r] = A[r0 + r][k0 + k]
  __shared__ __align__(16) float Bs[kNSK][kNSTile];  // Bs[k][c] = B[k0 + k][c0 + c]
  __shared__ double red[2];
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  const int r0 = blockIdx.y * kNSTile, c0 = blockIdx.x * kNSTile;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k0 = 0; k0 < n; k0 += kNSK) {
    const int kc = min(kNSK, n - k0);
    // Thread tid stages elements tid + 64 q (q < 64) of each slice, in two
    // batches of 32 loads per matrix held in registers, so that the loads
    // of a batch are in flight together.  A: consecutive threads along k
    // (element (r, kk) = (q / 4, 64 (q % 4) + tid), coalesced rows of A);
    // B: consecutive threads along the tile's columns ((kk, c) =
    // (4 q + tid / 16, tid % 16)).
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float ra[32], rb[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int qq = 32 * h + q;
        const int r = qq >> 2, ka = 64 * (qq & 3) + tid;
        const int kb = 4 * qq + (tid >> 4), c = tid & 15;
        ra[q] = (ka < kc && r0 + r < n) ? A[(i64)(r0 + r) * n + k0 + ka] : 0.f;
        rb[q] = (kb < kc && c0 + c < n) ? B[(i64)(k0 + kb) * n + c0 + c] : 0.f;
      }
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int qq = 32 * h + q;
        As[64 * (qq & 3) + tid][qq >> 2] = ra[q];
        Bs[4 * qq + (tid >> 4)][tid & 15] = rb[q];
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kc; ++kk) {
      const float2 a = *reinterpret_cast<const float2*>(&As[kk][2 * ty]);
      const float2 b = *reinterpret_cast<const float2*>(&Bs[kk][2 * tx]);
      acc[0][0] = fmaf(a.x, b.x, acc[0][0]);
      acc[0][1] = fmaf(a.x, b.y, acc[0][1]);
      acc[1][0] = fmaf(a.y, b.x, acc[1][0]);
      acc[1][1] = fmaf(a.y, b.y, acc[1][1]);
    }
    __syncthreads();
  }
  double sq = 0.0;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int row = r0 + 2 * ty + u, col = c0 + 2 * tx + q;
      if (row >= n || col >= n) continue;
      const i64 o = (i64)row * n + col;
      float v;
      if (MODE == 0) {
        v = (row == col ? 1.f : 0.f) - acc[u][q];
        sq += (double)v * (double)v;
      } else {
        v = D[o] + acc[u][q];
      }
      C[o] = v;
    }
  if (MODE == 0) {
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((tid & 31) == 0) red[tid >> 5] = sq;
    __syncthreads();
    if (tid == 0) atomicAdd(ss, red[0] + red[1]);
  }
}

template <int MODE>
void ns_gemm(int n, const float* A, const float* B, const float* D, float* C, double* ss, cudaStream_t s) {
  const unsigned nt = (unsigned)((n + kNSTile - 1) / kNSTile);
  launch_k(k_ns_gemm<MODE>, dim3(nt, nt), 64, 0, s, n, A, B, D, C, ss);
  note_launch();
}

// Rotates the previous configuration's inverse with each body's rotation
// since then: X_ij <- D_b(i) X_ij D_b(j)^T for the 3 x 3 blocks (blobs i, j
// of bodies b(i), b(j)), D_p = R(quat_new_p) R(quat_old_p)^T.  The RPY tensor
// is rotation-covariant, so rotating each body rigidly about its centre turns
// the intra-body blocks of M into exactly these; for a single body the
// rotated inverse is exact.  With several bodies the start's error comes from
// the inter-body blocks of M, which the move also changes.  One thread per
// block, in place.
__global__ void k_rotate_inverse(int nbl, const int* __restrict__ bob, const double* __restrict__ qnew,
                                 const double* __restrict__ qold, float* __restrict__ X) {
  pdl_entry();
  const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (i64)nbl * nbl) return;
  const int i = (int)(t / nbl), j = (int)(t - (i64)i * nbl);
  double D[2][9];
  const int body[2] = {bob[i], bob[j]};
  for (int s = 0; s < 2; ++s) {
    double Rn[9], Ro[9];
    quat_rot(qnew + 4 * body[s], Rn);
    quat_rot(qold + 4 * body[s], Ro);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        D[s][3 * a + b] = Rn[3 * a] * Ro[3 * b] + Rn[3 * a + 1] * Ro[3 * b + 1] + Rn[3 * a + 2] * Ro[3 * b + 2];
  }
  const i64 n3 = 3 * (i64)nbl;
  float* Xb = X + (3 * (i64)i) * n3 + 3 * (i64)j;
  double x[9], y[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) x[3 * a + b] = (double)Xb[a * n3 + b];
  // y = D_i x D_j^T
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double acc = 0.0;
      for (int c = 0; c < 3; ++c)
        for (int e = 0; e < 3; ++e) acc += D[0][3 * a + c] * x[3 * c + e] * D[1][3 * b + e];
      y[3 * a + b] = acc;
    }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Xb[a * n3 + b] = (float)y[3 * a + b];
}

// Build the coupled body block for a new configuration: M^-1, P = M^-1 K and
// N = (K^T M^-1 K)^-1.
//  - warm: Minv holds the inverse of the previous configuration's M, built
//    at the body orientations qold (NULL: unknown).  The start X0 is that
//    inverse rotated with each body's rotation since (k_rotate_inverse).
//    The configuration moves little between SEM steps, so X0 is a close
//    start for the Newton-Schulz iteration X <- X + X (I - M X), which
//    converges quadratically while ||I - M X|| < 1 (the spectral norm, which
//    the Frobenius norm bounds).  With ||R0||_F = ||I - M X0||_F at most
//    kNSMaxStart, kNSIters iterations leave a residual of at most
//    kNSMaxStart^(2^kNSIters) (FP32 roundoff in practice); each iteration is
//    two n x n products on the whole GPU, against n sequential pivot steps on
//    one SM for Gauss-Jordan.
//  - otherwise, or when R0 is larger (a first configuration, a large move):
//    in-place Gauss-Jordan.
// Mw, Tw, Uw: n3 x n3 FP32 work matrices; ss: one device double; ss_host:
// pinned host double (the choice needs one read of ||R0||).  Returns true
// when the warm start was taken.
constexpr double kNSMaxStart = 0.95;
constexpr int kNSIters = 8;   // even: the result lands in Minv
// The pieces of the set-up, also used one by one by the device-driven SEM
// step (where the warm-start decision is an IF/ELSE graph node).
// Warm start: Mw = M of the new configuration, X0 = Minv rotated with each
// body's rotation since it was built (when qnew and qold are known), and
// Tw = R0 = I - M X0 with ss[0] = ||R0||_F^2.
void dense_body_warm_start(int nbl, const int* bob, const double* r, const double* qnew, const double* qold,
                           double a, double eta, float* Minv, float* Mw, float* Tw, double* ss, cudaStream_t s) {
  const i64 n3 = 3 * (i64)nbl;
  launch_k(k_rpy_full, nblk(n3 * n3, 256), 256, 0, s, nbl, r, a, eta, Mw);
  note_launch();
  if (qnew && qold) {
    launch_k(k_rotate_inverse, nblk((i64)nbl * nbl, 128), 128, 0, s, nbl, bob, qnew, qold, Minv);
    note_launch();
  }
  cudaMemsetAsync(ss, 0, sizeof(double), s);
  ns_gemm<0>((int)n3, Mw, Minv, nullptr, Tw, ss, s);
}
// kNSIters Newton-Schulz steps from X0 = Minv with R0 in Tw; the result
// lands in Minv (kNSIters is even).
void dense_body_ns(int nbl, float* Minv, const float* Mw, float* Tw, float* Uw, double* ss, cudaStream_t s) {
  const int n3 = 3 * nbl;
  float* X = Minv;
  float* Y = Uw;
  for (int it = 0; it < kNSIters; ++it) {
    if (it > 0) ns_gemm<0>(n3, Mw, X, nullptr, Tw, ss, s);   // R = I - M X
    ns_gemm<1>(n3, X, Tw, X, Y, nullptr, s);                 // X' = X + X R
    float* t = X; X = Y; Y = t;
  }
}
// Gauss-Jordan inverse of M into Minv (from Mw when it is not null, else
// Minv holds M); status = 1 on a zero pivot.
void dense_body_gj(int nbl, float* Minv, const float* Mw, int* status, cudaStream_t s) {
  const i64 n3 = 3 * (i64)nbl;
  if (Mw) cudaMemcpyAsync(Minv, Mw, sizeof(float) * n3 * n3, cudaMemcpyDeviceToDevice, s);
  launch_k(k_gj_inverse<float>, 1, 1024, 2 * sizeof(float) * n3, s, Minv, (int)n3, status);
  note_launch();
}
// P = M^-1 K and N = (K^T P)^-1 (FP64 Gauss-Jordan; status = 1 on a zero pivot).
void dense_body_finish(int nbl, int nb, const int* boff, const double* arm, const float* Minv, float* P, double* N,
                       int* status, cudaStream_t s) {
  const i64 n3 = 3 * (i64)nbl, m = 6 * (i64)nb;
  launch_k(k_mk, nblk(n3 * m, 256), 256, 0, s, nbl, nb, boff, arm, Minv, P);
  note_launch();
  launch_k(k_ktp, nblk(m * m, 256), 256, 0, s, nbl, nb, boff, arm, P, N);
  note_launch();
  launch_k(k_gj_inverse<double>, 1, 1024, 2 * sizeof(double) * m, s, N, (int)m, status);
  note_launch();
}

// IF/ELSE condition of the device-driven warm start: ||R0||_F <= kNSMaxStart;
// warm[0] counts the builds that take the Newton-Schulz branch.
__global__ void k_ns_decide(const double* ss, cudaGraphConditionalHandle h, long long* warm) {
  pdl_entry();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const bool ok = ss[0] <= kNSMaxStart * kNSMaxStart;
  if (ok) warm[0] += 1;
  cudaGraphSetConditional(h, ok ? 1u : 0u);
}
void ns_decide(const double* ss, cudaGraphConditionalHandle h, long long* warm, cudaStream_t s) {
  launch_k(k_ns_decide, 1, 32, 0, s, ss, h, warm);
  note_launch();
}

cudaError_t dense_body_build(int nbl, int nb, const int* boff, const int* bob, const double* r, const double* arm,
                             const double* qnew, const double* qold, double a, double eta, float* Minv, float* P,
                             double* N, int* status, float* Mw, float* Tw, float* Uw, double* ss, double* ss_host,
                             bool warm, cudaStream_t s, bool* used_out) {
  const i64 n3 = 3 * (i64)nbl;
  cudaError_t e;
#define RB_CK(call)                      \
  if ((e = (call)) != cudaSuccess) return e
  RB_CK(cudaMemsetAsync(status, 0, sizeof(int), s));
  bool used = false;
  *used_out = false;
  if (warm) {
    dense_body_warm_start(nbl, bob, r, qnew, qold, a, eta, Minv, Mw, Tw, ss, s);
    RB_CK(cudaMemcpyAsync(ss_host, ss, sizeof(double), cudaMemcpyDeviceToHost, s));
    RB_CK(cudaStreamSynchronize(s));
    const double r0 = std::sqrt(std::max(ss_host[0], 0.0));
    if (r0 <= kNSMaxStart) {
      dense_body_ns(nbl, Minv, Mw, Tw, Uw, ss, s);
      used = true;
    } else {
      dense_body_gj(nbl, Minv, Mw, status, s);
    }
  } else {
    launch_k(k_rpy_full, nblk(n3 * n3, 256), 256, 0, s, nbl, r, a, eta, Minv);
    note_launch();
    dense_body_gj(nbl, Minv, nullptr, status, s);
  }
  dense_body_finish(nbl, nb, boff, arm, Minv, P, N, status, s);
  *used_out = used;
  return cudaGetLastError();
#undef RB_CK
}

// Apply on one cluster of kBodyCtas CTAs: t = M^-1 s; f = r_U + K^T t;
// U = N f; lam = M^-1 (K U - s) = P U - t with P = M^-1 K from the set-up.
// The rows of t, U and lam are split over the CTAs; t and U are exchanged
// through distributed shared memory.  s, r_U in, lam, U out (type T;
// internal FP32 / FP64).  With tab set, the kernel first forms
// s = r_lam + J v itself (one warp per blob component over the cluster,
// written to sres, then a cluster barrier), which saves a launch.
constexpr int kBodyCtas = 8;

template <typename T>
__global__ void __cluster_dims__(kBodyCtas, 1, 1) __launch_bounds__(512)
    k_dense_body_apply(int nbl, int nb, const int* __restrict__ boff, const int* __restrict__ bob,
                       const double* __restrict__ arm, const float* __restrict__ Mi, const float* __restrict__ P,
                       const double* __restrict__ N, const T* __restrict__ sres, const T* __restrict__ rU,
                       T* __restrict__ zlam, T* __restrict__ zU, double* __restrict__ zlam64,
                       double* __restrict__ zU64, Dims d, const BlobStencil<T>* __restrict__ tab,
                       const T* __restrict__ v, const T* __restrict__ rl, T* __restrict__ sres_out) {
  pdl_entry();
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ unsigned char shraw[];
  const int n3 = 3 * nbl, m = 6 * nb;
  const int rank = (int)cl.block_rank();
  const int rpc = (n3 + kBodyCtas - 1) / kBodyCtas, upc = (m + kBodyCtas - 1) / kBodyCtas;
  const int r0 = rank * rpc, r1 = min(n3, r0 + rpc);
  const int u0 = rank * upc, u1 = min(m, u0 + upc);
  double* f = (double*)shraw;      // m
  double* Uall = f + m;            // m
  double* Uloc = Uall + m;         // upc (this CTA's rows of U)
  float* sv = (float*)(Uloc + upc);   // n3
  float* tloc = sv + n3;              // rpc (this CTA's rows of t)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (tab) {
    for (int c = rank * nw + wid; c < n3; c += kBodyCtas * nw) {
      const T jv = warp_interp<T>(d, c % 3, tab + c, v, lane);
      if (lane == 0) sres_out[c] = rl[c] + jv;
    }
    cl.sync();   // release / acquire at cluster scope: every CTA's rows of s are visible
    for (int i = threadIdx.x; i < n3; i += blockDim.x) sv[i] = (float)__ldcg(sres_out + i);
  } else {
    for (int i = threadIdx.x; i < n3; i += blockDim.x) sv[i] = (float)sres[i];
  }
  __syncthreads();
  // rows of t = M^-1 s, one warp per row
  for (int row = r0 + wid; row < r1; row += nw) {
    const float* Mr = Mi + (i64)row * n3;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int c = lane;
    for (; c + 96 < n3; c += 128) {
      a0 = fmaf(Mr[c], sv[c], a0);
      a1 = fmaf(Mr[c + 32], sv[c + 32], a1);
      a2 = fmaf(Mr[c + 64], sv[c + 64], a2);
      a3 = fmaf(Mr[c + 96], sv[c + 96], a3);
    }
    for (; c < n3; c += 32) a0 = fmaf(Mr[c], sv[c], a0);
    float acc = (a0 + a1) + (a2 + a3);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) tloc[row - r0] = acc;
  }
  cl.sync();
  // f = r_U + K^T t (every CTA, t read from its owners)
  for (int p = wid; p < nb; p += nw) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int i = boff[p] + lane; i < boff[p + 1]; i += 32) {
      double t3[3];
      for (int a = 0; a < 3; ++a) {
        const int row = 3 * i + a, owner = row / rpc;
        const float* tr = cl.map_shared_rank(tloc, owner);
        t3[a] = tr[row - owner * rpc];
      }
      const double x = t3[0], y = t3[1], z = t3[2];
      const double* d = arm + 3 * i;
      acc[0] += x; acc[1] += y; acc[2] += z;
      acc[3] += d[1] * z - d[2] * y;
      acc[4] += d[2] * x - d[0] * z;
      acc[5] += d[0] * y - d[1] * x;
    }
    for (int c = 0; c < 6; ++c)
      for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    if (lane < 6) f[6 * p + lane] = acc[lane] + (double)rU[6 * p + lane];
  }
  __syncthreads();
  // this CTA's rows of U = N f
  for (int r = u0 + (int)threadIdx.x; r < u1; r += blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < m; ++c) acc = fma(N[(i64)r * m + c], f[c], acc);
    Uloc[r - u0] = acc;
    zU[r] = (T)acc;
    if (zU64) zU64[r] = (double)(T)acc;
  }
  cl.sync();
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    const int owner = c / upc;
    Uall[c] = cl.map_shared_rank(Uloc, owner)[c - owner * upc];
  }
  __syncthreads();
  // this CTA's rows of lam = P U - t
  for (int row = r0 + (int)threadIdx.x; row < r1; row += blockDim.x) {
    const float* Pr = P + (i64)row * m;
    float acc = -tloc[row - r0];
    for (int c = 0; c < m; ++c) acc = fmaf(Pr[c], (float)Uall[c], acc);
    zlam[row] = (T)acc;
    if (zlam64) zlam64[row] = (double)(T)acc;
  }
  cl.sync();   // no CTA leaves while another may still read its shared memory
}

template <typename T>
void dense_body_apply(int nbl, int nb, const int* boff, const int* bob, const double* arm, const float* Minv,
                      const float* P, const double* N, const T* sres, const T* rU, T* zlam, T* zU, double* zlam64,
                      double* zU64, cudaStream_t s, const Dims* d, const BlobStencil<T>* tab, const T* v,
                      const T* rl, T* sres_out) {
  const int n3 = 3 * nbl, m = 6 * nb;
  const int rpc = (n3 + kBodyCtas - 1) / kBodyCtas, upc = (m + kBodyCtas - 1) / kBodyCtas;
  const size_t shm = sizeof(double) * (2 * (size_t)m + upc) + sizeof(float) * ((size_t)n3 + rpc);
  launch_k(k_dense_body_apply<T>, kBodyCtas, 512, shm, s, nbl, nb, boff, bob, arm, Minv, P, N, sres, rU, zlam, zU,
           zlam64, zU64, d ? *d : Dims{}, tab, v, rl, sres_out);
  note_launch();
}

template void dense_body_apply<float>(int, int, const int*, const int*, const double*, const float*, const float*,
                                      const double*, const float*, const float*, float*, float*, double*, double*,
                                      cudaStream_t, const Dims*, const BlobStencil<float>*, const float*, const float*,
                                      float*);
template void dense_body_apply<double>(int, int, const int*, const int*, const double*, const float*,
                                       const float*, const double*, const double*, const double*, double*, double*,
                                       double*, double*, cudaStream_t, const Dims*, const BlobStencil<double>*,
                                       const double*, const double*, double*);

}  // namespace rbfib
