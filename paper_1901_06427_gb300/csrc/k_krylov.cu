// Krylov building blocks for FGMRES (Sec. III.C; the paper solves the
// saddle system with a preconditioned flexible GMRES): multi-column inner
// products with FP64 accumulation (warp shuffles -> block -> fixed-order
// final sum, deterministic), fused multi-axpy with the norm of the result,
// Givens rotations and the small triangular solve on the device.
#include <cstdint>
#include <cstdlib>

#include "common.cuh"
#include "kernels.cuh"

namespace rbfib {

static inline unsigned nblk(i64 n, int bs) { return (unsigned)((n + bs - 1) / bs); }

RBFIB_DEVFN double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum (blockDim.x multiple of 32, <= 1024); result valid in thread 0
RBFIB_DEVFN double block_sum(double v) {
  __shared__ double sh[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0) v = warp_sum(v);
  return v;
}

// Whether a multi-column sweep can use 16-byte loads: both arrays 16-byte
// aligned and every column start too.
template <typename T>
inline int vec_ok(const T* a, const T* b, i64 ld, int ncols) {
  auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  return al(a) && al(b) && (ncols <= 1 || ((ld * (i64)sizeof(T)) & 15) == 0) ? 1 : 0;
}

// Block-level completion of a grid-wide reduction: thread 0 stores this
// block's value, then counts the block in; the last block (the one that
// brings the counter to gridDim.x) gets true, with the other blocks' values
// visible, and resets the counter for the next launch.  No block waits.
RBFIB_DEVFN bool finish_last(double* slots, double v, unsigned* counter) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    slots[blockIdx.x] = v;
    __threadfence();
    const unsigned done = atomicAdd(counter, 1u);
    last = done == gridDim.x - 1;
    if (last) *counter = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

template <typename T>
RBFIB_DEVFN T ldcg_t(const T* p) { return __ldcg(p); }

// In the last block of a first-pass multi-axpy (all threads): with
// nrm2w = ||w'||^2 and the projection coefficients coef[0..k), decide whether
// the second pass is needed and reset its coefficients (see ReorthCtl).
RBFIB_DEVFN void reorth_decide(const ReorthCtl& ctl, double nrm2w, const double* coef, int k) {
  double hh = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double c = coef[i];
    hh = fma(c, c, hh);
    ctl.h2[i] = 0.0;
  }
  hh = block_sum(hh);
  if (threadIdx.x == 0) {
    const int again = (nrm2w < ctl.tau2 * (nrm2w + hh)) ? 1 : 0;
    ctl.flag[0] = again;
    ctl.flag[1] += again;   // second passes taken (reset by the solver)
    if (ctl.use_handle) cudaGraphSetConditional(ctl.handle, (unsigned)again);
  }
}

// Per column: the blocks' shares of the unweighted sum w . V_col over [0, n)
// (16-byte loads when vec) go to part[col * gridDim.x + block]; the last
// block to finish a column (atomic counter, reset afterwards) adds them up
// and forms out[col] = wf * sum + (1 - wf) * sum_{nfl <= i < n} w_i V_col,i:
// the inner product with weight wf on the fluid entries and 1 on the body
// entries (re-read here, they are few).  FP32: FP32 products and per-thread
// FP32 sums, FP64 across threads and blocks (enough for the FP32 inner solve
// of the refinement).
template <typename T>
__global__ void k_dot_part(const T* __restrict__ w, const T* __restrict__ V, i64 ldv, i64 n, i64 nfl, double wf,
                           double* __restrict__ part, unsigned* __restrict__ cnt, double* __restrict__ out,
                           int vec, const int* __restrict__ gate) {
  pdl_entry();
  if (gate && *gate == 0) return;
  const int col = blockIdx.y;
  const T* v = V + (i64)col * ldv;
  const i64 stride = (i64)gridDim.x * blockDim.x, t0 = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  double acc;
  if constexpr (sizeof(T) == 8) {
    double a0 = 0.0, a1 = 0.0;
    if (vec) {
      const double2* w2 = reinterpret_cast<const double2*>(w);
      const double2* v2 = reinterpret_cast<const double2*>(v);
      for (i64 i = t0; i < (n >> 1); i += stride) {
        const double2 x = w2[i], y = v2[i];
        a0 = fma(x.x, y.x, a0);
        a1 = fma(x.y, y.y, a1);
      }
      if ((n & 1) && t0 == 0) a0 = fma(w[n - 1], v[n - 1], a0);
    } else {
      for (i64 i = t0; i < n; i += stride) a0 = fma(w[i], v[i], a0);
    }
    acc = a0 + a1;
  } else {
    float s0 = 0.f, s1 = 0.f;
    if (vec) {
      const float4* w4 = reinterpret_cast<const float4*>(w);
      const float4* v4 = reinterpret_cast<const float4*>(v);
      for (i64 i = t0; i < (n >> 2); i += stride) {
        const float4 x = w4[i], y = v4[i];
        s0 = fmaf(x.x, y.x, fmaf(x.y, y.y, s0));
        s1 = fmaf(x.z, y.z, fmaf(x.w, y.w, s1));
      }
      if (t0 < (n & 3)) s0 = fmaf((float)w[(n & ~(i64)3) + t0], (float)v[(n & ~(i64)3) + t0], s0);
    } else {
      for (i64 i = t0; i < n; i += stride) s0 = fmaf((float)w[i], (float)v[i], s0);
    }
    acc = (double)s0 + (double)s1;
  }
  acc = block_sum(acc);
  if (!finish_last(part + (i64)col * gridDim.x, acc, cnt + col)) return;
  double s = 0.0, body = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(part + (i64)col * gridDim.x + i);
  if (wf != 1.0)
    for (i64 i = nfl + threadIdx.x; i < n; i += blockDim.x) body = fma((double)w[i], (double)v[i], body);
  s = block_sum(wf * s + (1.0 - wf) * body);
  if (threadIdx.x == 0) out[col] = s;
}

// ---------------------------------------------------------------------------
// Register-blocked Gram-Schmidt sweeps (16-byte aligned vectors).
//
// A block covers chunks of 256 * R 16-byte vectors (R per thread, kept in
// registers) of the rows; blockIdx.y picks a group of kCG basis columns.  w
// is loaded once per chunk and column group (not once per column), so a
// thread issues R independent loads per column and kCG columns per group
// before it needs their products: enough loads in flight to keep the FP64
// pipe, the bound of these sweeps on GB300, busy.  The per-column sums of a
// block are reduced by a butterfly transpose within each warp (each lane
// ends with one column's warp total after kCG + 1 additions instead of
// 5 kCG) and across warps through shared memory.
constexpr int kCG = 8;

template <typename T> struct Vec16;
template <> struct Vec16<double> { typedef double2 t; static constexpr int w = 2; typedef double acc; };
template <> struct Vec16<float> { typedef float4 t; static constexpr int w = 4; typedef float acc; };

RBFIB_DEVFN double dot16(const double2& a, const double2& b, double c) { return fma(a.y, b.y, fma(a.x, b.x, c)); }
RBFIB_DEVFN float dot16(const float4& a, const float4& b, float c) {
  return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, c))));
}
RBFIB_DEVFN void axpy16(double f, const double2& v, double2& x) { x.x = fma(f, v.x, x.x); x.y = fma(f, v.y, x.y); }
RBFIB_DEVFN void axpy16(float f, const float4& v, float4& x) {
  x.x = fmaf(f, v.x, x.x); x.y = fmaf(f, v.y, x.y); x.z = fmaf(f, v.z, x.z); x.w = fmaf(f, v.w, x.w);
}
RBFIB_DEVFN double fma_a(double a, double b, double c) { return fma(a, b, c); }
RBFIB_DEVFN float fma_a(float a, float b, float c) { return fmaf(a, b, c); }
constexpr int kGivensMaxCols = 128;   // largest column count of one sweep
RBFIB_DEVFN void zero16(double2& a) { a = make_double2(0.0, 0.0); }
RBFIB_DEVFN void zero16(float4& a) { a = make_float4(0.f, 0.f, 0.f, 0.f); }

// v[0..8) per lane -> the warp total of column col = 4 b4 + 2 b3 + b2 (b =
// bits of the lane) in every lane; lanes with (lane & 3) == 0 hold the eight
// totals.  Works on A = float or double.
template <typename A>
RBFIB_DEVFN A warp_transpose_sum8(A v[kCG]) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const A send = b4 ? v[j] : v[j + 4];
    const A keep = b4 ? v[j + 4] : v[j];
    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const A send = b3 ? v[j] : v[j + 2];
    const A keep = b3 ? v[j + 2] : v[j];
    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  {
    const A send = b2 ? v[0] : v[1];
    const A keep = b2 ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  A t = v[0];
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  return t;
}

// Per block: sums over the block's threads of acc[0..kCG), in FP64; the
// result for column c is returned by thread c (c < kCG).
template <typename A>
RBFIB_DEVFN double block_transpose_sum8(A acc[kCG]) {
  __shared__ double sh[8][kCG];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const A t = warp_transpose_sum8<A>(acc);
  if ((lane & 3) == 0) sh[wid][lane >> 2] = (double)t;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < kCG) {
    const int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) s += sh[i][threadIdx.x];
  }
  __syncthreads();
  return s;
}

// out[c] = <w, V_c>_W for c < k (weight wf on the first nfl entries, 1 on the
// rest); nv = n / Vec16::w whole vectors, the n - nv Vec16::w trailing
// elements added by the first chunk.  Partials: part[c * gridDim.x + bx];
// the last block to finish (one counter for the launch) adds them up with
// the body-entry weight correction.
template <typename T, int R>
__global__ void __launch_bounds__(256) k_gs_dot(const T* __restrict__ w, const T* __restrict__ V, i64 ldv, int k,
                                                i64 n, i64 nfl, double wf, double* __restrict__ part,
                                                unsigned* __restrict__ cnt, double* __restrict__ out,
                                                const int* __restrict__ gate) {
  pdl_entry();
  if (gate && *gate == 0) return;
  typedef typename Vec16<T>::t VT;
  typedef typename Vec16<T>::acc A;
  constexpr int W = Vec16<T>::w;
  const i64 nv = n / W;
  const i64 chunk = 256 * (i64)R;
  const i64 nchunks = (nv + chunk - 1) / chunk;
  // columns split evenly over the groups (gridDim.y): at most kCG each
  const int cpg = (k + gridDim.y - 1) / gridDim.y;
  const int c0 = blockIdx.y * cpg, c1 = min(k, c0 + cpg);
  const VT* w4 = reinterpret_cast<const VT*>(w);
  A acc[kCG];
#pragma unroll
  for (int c = 0; c < kCG; ++c) acc[c] = (A)0;
  for (i64 ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const i64 base = ch * chunk + threadIdx.x;
    VT wr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const i64 i = base + (i64)r * 256;
      if (i < nv) wr[r] = w4[i]; else zero16(wr[r]);
    }
#pragma unroll
    for (int c = 0; c < kCG; ++c) {
      if (c0 + c < c1) {
        const VT* v4 = reinterpret_cast<const VT*>(V + (i64)(c0 + c) * ldv);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const i64 i = base + (i64)r * 256;
          if (i < nv) acc[c] = dot16(wr[r], v4[i], acc[c]);
        }
      }
    }
  }
  if (blockIdx.x == 0) {   // trailing elements that do not fill a 16-byte vector
    const i64 i = nv * W + threadIdx.x;
    if (i < n) {
      const A x = (A)w[i];
#pragma unroll
      for (int c = 0; c < kCG; ++c)
        if (c0 + c < c1) acc[c] += x * (A)V[(i64)(c0 + c) * ldv + i];
    }
  }
  const double s = block_transpose_sum8<A>(acc);
  __shared__ bool last;
  if (threadIdx.x < kCG && c0 + (int)threadIdx.x < c1) {
    part[(i64)(c0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(cnt, 1u);
    last = done == gridDim.x * gridDim.y - 1;
    if (last) *cnt = 0u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // one warp per column: partials of the blocks, then the body entries
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = wid; c < k; c += nw) {
    double t = 0.0, body = 0.0;
    for (int i = lane; i < (int)gridDim.x; i += 32) t += __ldcg(part + (i64)c * gridDim.x + i);
    if (wf != 1.0)
      for (i64 i = nfl + lane; i < n; i += 32) body = fma((double)w[i], (double)V[(i64)c * ldv + i], body);
    t = warp_sum(wf * t + (1.0 - wf) * body);
    if (lane == 0) out[c] = t;
  }
}

// w += sign * sum_{c < k} coef[c] V_c over 16-byte vectors (R per thread
// per chunk), then, when nrm2 is not null, nrm2[0] = ||w||_W^2 of the result
// (block sums, the last block adds them up with the body correction).
template <typename T, int R>
__global__ void __launch_bounds__(256) k_gs_axpy(T* __restrict__ w, const T* __restrict__ V, i64 ldv, int k,
                                                 const double* __restrict__ coef, double sign, i64 n, i64 nfl,
                                                 double wf, double* __restrict__ part, unsigned* __restrict__ cnt,
                                                 double* __restrict__ nrm2, ReorthCtl ctl,
                                                 const int* __restrict__ gate) {
  pdl_entry();
  if (gate && *gate == 0) return;
  typedef typename Vec16<T>::t VT;
  typedef typename Vec16<T>::acc A;
  constexpr int W = Vec16<T>::w;
  __shared__ A cf[kGivensMaxCols];
  for (int i = threadIdx.x; i < k; i += blockDim.x) cf[i] = (A)(sign * coef[i]);
  __syncthreads();
  const i64 nv = n / W;
  const i64 chunk = 256 * (i64)R;
  const i64 nchunks = (nv + chunk - 1) / chunk;
  VT* w4 = reinterpret_cast<VT*>(w);
  A nrm = (A)0;
  for (i64 ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const i64 base = ch * chunk + threadIdx.x;
    VT x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const i64 i = base + (i64)r * 256;
      if (i < nv) x[r] = w4[i]; else zero16(x[r]);
    }
    int c = 0;
    for (; c + 4 <= k; c += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const VT* v4 = reinterpret_cast<const VT*>(V + (i64)(c + u) * ldv);
        const A f = cf[c + u];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const i64 i = base + (i64)r * 256;
          if (i < nv) axpy16(f, v4[i], x[r]);
        }
      }
    }
    for (; c < k; ++c) {
      const VT* v4 = reinterpret_cast<const VT*>(V + (i64)c * ldv);
      const A f = cf[c];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const i64 i = base + (i64)r * 256;
        if (i < nv) axpy16(f, v4[i], x[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const i64 i = base + (i64)r * 256;
      if (i < nv) {
        w4[i] = x[r];
        nrm = dot16(x[r], x[r], nrm);
      }
    }
  }
  if (blockIdx.x == 0) {
    const i64 i = nv * W + threadIdx.x;
    if (i < n) {
      A x = (A)w[i];
      for (int c = 0; c < k; ++c) x = fma_a(cf[c], (A)V[(i64)c * ldv + i], x);
      w[i] = (T)x;
      nrm = fma_a(x, x, nrm);
    }
  }
  if (!nrm2) return;
  const double acc = block_sum((double)nrm);
  if (!finish_last(part, acc, cnt)) return;
  double t = 0.0, body = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(part + i);
  if (wf != 1.0)
    for (i64 i = nfl + threadIdx.x; i < n; i += blockDim.x) {
      const double x = (double)ldcg_t(w + i);
      body = fma(x, x, body);
    }
  t = block_sum(wf * t + (1.0 - wf) * body);
  if (threadIdx.x == 0) nrm2[0] = t;
  if (ctl.flag) {
    __shared__ double tt;
    if (threadIdx.x == 0) tt = t;
    __syncthreads();
    reorth_decide(ctl, tt, coef, k);
  }
}

// Row blocks of a register-blocked sweep: one per chunk of 256 R vectors, so
// that no block carries a second chunk while others idle (a block that does
// finishes last and sets the launch's duration), capped by the partial
// buffer's nparts slots per column on large grids.
inline int gs_blocks(i64 nv, int R, int nparts) {
  const i64 chunks = (nv + 256 * (i64)R - 1) / (256 * (i64)R);
  return (int)std::max<i64>(1, std::min<i64>(chunks, nparts));
}

// plain sum of nparts partials
__global__ void k_sum_finish(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  pdl_entry();
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[0] = acc;
}

// About 32 elements per thread: few blocks, each with long independent
// FP64 FMA chains (FP64 throughput is the bound).
inline int dot_blocks(i64 n, int nparts) {
  const i64 b = (n + 256 * 32 - 1) / (256 * 32);
  return (int)std::max<i64>(1, std::min<i64>(b, nparts));
}

template <typename T>
void multi_dot(const T* w, const T* V, i64 ldv, int ncols, i64 n, i64 nfl, double wf, double* part, int nparts,
               double* out, cudaStream_t s, const int* gate) {
  if (vec_ok(w, V, ldv, ncols) && ncols <= kGivensMaxCols) {
    constexpr int R = 4;
    const int groups = (ncols + kCG - 1) / kCG;
    const int nb = gs_blocks(n / Vec16<T>::w, R, nparts);
    launch_k(k_gs_dot<T, R>, dim3(nb, groups), 256, 0, s, w, V, ldv, ncols, n, nfl, wf, part,
             part_counters(part, nparts) + kDotCounter, out, gate);
    note_launch();
    return;
  }
  const int nb = dot_blocks(n, nparts);
  dim3 grid(nb, ncols);
  launch_k(k_dot_part<T>, grid, 256, 0, s, w, V, ldv, n, nfl, wf, part, part_counters(part, nparts), out,
           vec_ok(w, V, ldv, ncols), gate);
  note_launch();
}

// w += sign * sum_c coef[c] V_c (16-byte loads when vec, two rows per thread
// step in FP64, four in FP32); part[blockIdx.x] = partial unweighted ||w||^2
template <typename T>
__global__ void k_multi_axpy(T* __restrict__ w, const T* __restrict__ V, i64 ldv, int ncols,
                             const double* __restrict__ coef, double sign, i64 n, i64 nfl, double wf,
                             double* __restrict__ part, unsigned* __restrict__ cnt, double* __restrict__ nrm2,
                             int vec, ReorthCtl ctl, const int* __restrict__ gate) {
  pdl_entry();
  if (gate && *gate == 0) return;
  __shared__ double c[128];
  for (int i = threadIdx.x; i < ncols; i += blockDim.x) c[i] = sign * coef[i];
  __syncthreads();
  const i64 stride = (i64)gridDim.x * blockDim.x, t0 = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  double nrm = 0.0;
  if constexpr (sizeof(T) == 8) {
    if (vec) {
      double2* w2 = reinterpret_cast<double2*>(w);
      for (i64 i = t0; i < (n >> 1); i += stride) {
        double2 x = w2[i];
        for (int k = 0; k < ncols; ++k) {
          const double2 y = reinterpret_cast<const double2*>(V + (i64)k * ldv)[i];
          x.x = fma(c[k], y.x, x.x);
          x.y = fma(c[k], y.y, x.y);
        }
        w2[i] = x;
        nrm = fma(x.x, x.x, fma(x.y, x.y, nrm));
      }
      if ((n & 1) && t0 == 0) {
        double x = w[n - 1];
        for (int k = 0; k < ncols; ++k) x = fma(c[k], V[(i64)k * ldv + n - 1], x);
        w[n - 1] = x;
        nrm = fma(x, x, nrm);
      }
    } else {
      for (i64 i = t0; i < n; i += stride) {
        double x = w[i];
        for (int k = 0; k < ncols; ++k) x = fma(c[k], V[(i64)k * ldv + i], x);
        w[i] = x;
        nrm = fma(x, x, nrm);
      }
    }
  } else {
    __shared__ float c32[128];
    for (int i = threadIdx.x; i < ncols; i += blockDim.x) c32[i] = (float)c[i];
    __syncthreads();
    float s0 = 0.f;
    if (vec) {
      float4* w4 = reinterpret_cast<float4*>(w);
      for (i64 i = t0; i < (n >> 2); i += stride) {
        float4 x = w4[i];
        for (int k = 0; k < ncols; ++k) {
          const float4 y = reinterpret_cast<const float4*>(V + (i64)k * ldv)[i];
          x.x = fmaf(c32[k], y.x, x.x);
          x.y = fmaf(c32[k], y.y, x.y);
          x.z = fmaf(c32[k], y.z, x.z);
          x.w = fmaf(c32[k], y.w, x.w);
        }
        w4[i] = x;
        s0 = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, s0))));
      }
      if (t0 < (n & 3)) {
        const i64 i = (n & ~(i64)3) + t0;
        float x = (float)w[i];
        for (int k = 0; k < ncols; ++k) x = fmaf(c32[k], (float)V[(i64)k * ldv + i], x);
        w[i] = (T)x;
        s0 = fmaf(x, x, s0);
      }
    } else {
      for (i64 i = t0; i < n; i += stride) {
        float x = (float)w[i];
        for (int k = 0; k < ncols; ++k) x = fmaf(c32[k], (float)V[(i64)k * ldv + i], x);
        w[i] = (T)x;
        s0 = fmaf(x, x, s0);
      }
    }
    nrm = s0;
  }
  if (!nrm2) return;
  // weighted norm of the result: the last block adds up the blocks' sums and
  // the body-block correction (1 - wf) sum_{i >= nfl} w_i^2
  const double acc = block_sum(nrm);
  if (!finish_last(part, acc, cnt)) return;
  double s = 0.0, body = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(part + i);
  if (wf != 1.0)
    for (i64 i = nfl + threadIdx.x; i < n; i += blockDim.x) {
      const double x = (double)ldcg_t(w + i);
      body = fma(x, x, body);
    }
  s = block_sum(wf * s + (1.0 - wf) * body);
  if (threadIdx.x == 0) nrm2[0] = s;
  if (ctl.flag) {
    __shared__ double tt;
    if (threadIdx.x == 0) tt = s;
    __syncthreads();
    reorth_decide(ctl, tt, coef, ncols);
  }
}

template <typename T>
void multi_axpy(T* w, const T* V, i64 ldv, int ncols, const double* coef, double sign, i64 n, i64 nfl, double wf,
                double* part, int nparts, double* nrm2, cudaStream_t s, const ReorthCtl* ctl, const int* gate) {
  const ReorthCtl c = (ctl && nrm2) ? *ctl : ReorthCtl{nullptr, nullptr, 0.0, 0, 0};
  if (vec_ok(w, V, ldv, ncols) && ncols <= kGivensMaxCols) {
    constexpr int R = 2;
    const int nb = gs_blocks(n / Vec16<T>::w, R, nparts);
    launch_k(k_gs_axpy<T, R>, nb, 256, 0, s, w, V, ldv, ncols, coef, sign, n, nfl, wf, part,
             part_counters(part, nparts) + kAxpyCounter, nrm2, c, gate);
    note_launch();
    return;
  }
  launch_k(k_multi_axpy<T>, nparts, 256, 0, s, w, V, ldv, ncols, coef, sign, n, nfl, wf, part,
           part_counters(part, nparts) + kAxpyCounter, nrm2, vec_ok(w, V, ldv, ncols), c, gate);
  note_launch();
}

// mode 0: out = in * d[0]; mode 1: out = in / d[0]; mode 2: out = in / sqrt(d[0])
// (a zero divisor gives zeros)
template <typename T>
__global__ void k_scale(T* __restrict__ out, const T* __restrict__ in, const double* __restrict__ denom, int invert,
                        i64 n, float* __restrict__ out32) {
  pdl_entry();
  // one thread per block forms the factor (FP64 square root and division
  // are long instruction sequences)
  __shared__ double fs;
  if (threadIdx.x == 0) {
    const double dv = invert == 2 ? sqrt(fmax(denom[0], 0.0)) : denom[0];
    fs = invert ? (dv != 0.0 ? 1.0 / dv : 0.0) : dv;
  }
  __syncthreads();
  const double f = fs;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    const T v = (T)((double)in[i] * f);
    out[i] = v;
    if (out32) out32[i] = (float)v;
  }
}

// Occupies the stream for a fixed number of SM clock cycles (one thread;
// ends by itself).  Used by the kernel timer so that the host has queued a
// timed launch and its closing event before the stream reaches them.
__global__ void k_delay(long long cycles) {
  pdl_entry();
  const long long t0 = clock64();
  while (clock64() - t0 < cycles) {
  }
}
void gpu_delay(long long cycles, cudaStream_t s) {
  k_delay<<<1, 1, 0, s>>>(cycles);
  note_launch();
}

// An empty kernel: calibrates the kernel timer's per-launch event overhead.
__global__ void k_empty() { pdl_entry(); }
void gpu_empty(cudaStream_t s) {
  k_empty<<<1, 32, 0, s>>>();
  note_launch();
}

template <typename T>
void scale_by(T* out, const T* in, const double* denom, int invert, i64 n, cudaStream_t s, float* out32) {
  const unsigned nb = (unsigned)std::min<i64>(nblk(n, 256), 152 * 8);
  launch_k(k_scale<T>, nb, 256, 0, s, out, in, denom, invert, n, out32);
  note_launch();
}

// Hessenberg column j: H[0..j] = hcol (CGS sum), H[j+1] = sqrt(hnext2); apply
// the previous rotations, form rotation j, update g; res_out = |g[j+1]|.
// Givens update of Hessenberg column j (64 threads or more): the column (CGS
// sums hcol + hcol2, then ||w||), the previous rotations and g are staged in
// shared memory by all threads.  Applying rotations 0..j-1 carries one entry
// down the column: with x_0 = h_0, rotation i outputs h_i = c_i x_i +
// s_i h_{i+1} and passes on x_{i+1} = -s_i x_i + c_i h_{i+1}, a first-order
// linear recurrence.  FP64 latency is long on this GPU, so from j =
// kGivensScanMin on (below, one thread runs the j dependent steps; measured
// on GB300: 5.3 us at j = 0 and 0.17 us more per rotation, against a flat
// 7.2 us for the scan) the first warp evaluates it as a scan of affine maps
// x -> a x + b (a_i = -s_i, b_i = c_i h_{i+1}; composing f_b after f_a
// gives (a_b a_a, a_b b_a + b_b)): each lane composes the maps of its
// segment of E = ceil(j / 32) consecutive rotations, a five-step shuffle
// scan composes the segments, and each lane then runs its segment from the
// carry entering it.  |a_i| <= 1, so no partial product grows.  One thread
// then forms rotation j and updates g; all threads write the column back.
// Returns |g[j+1]|; r_out = the new diagonal entry (every thread).
constexpr int kGivensMax = 128;
constexpr int kGivensSeg = kGivensMax / 32;   // rotations per lane at most
constexpr int kGivensScanMin = 16;            // j from which the scan is faster (GB300)
RBFIB_DEVFN double givens_core(double* H, int ldh, double* cs, double* sn, double* g, int j, const double* hcol,
                               const double* hcol2, const double* hnext2, double& r_out) {
  __shared__ double h[kGivensMax + 2], c[kGivensMax], s[kGivensMax];
  __shared__ double res, rdiag, carry_out;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) h[i] = hcol[i] + (hcol2 ? hcol2[i] : 0.0);
  for (int i = threadIdx.x; i < j; i += blockDim.x) { c[i] = cs[i]; s[i] = sn[i]; }
  __syncthreads();
  if (j < kGivensScanMin) {
    // few rotations: one thread runs the recurrence (the scan's fixed cost
    // of about a microsecond is larger than the chain here)
    if (threadIdx.x == 0) {
      double x = h[0];
      for (int i = 0; i < j; ++i) {
        const double hi1 = h[i + 1];
        h[i] = c[i] * x + s[i] * hi1;
        x = -s[i] * x + c[i] * hi1;
      }
      carry_out = x;
    }
  } else if (threadIdx.x < 32) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x;
    const int E = (j + 31) >> 5;
    const int i0 = min(lane * E, j), i1 = min(i0 + E, j);
    // this lane's rotations and the entries below them, in registers (the
    // entries are overwritten below)
    double cr[kGivensSeg], sr[kGivensSeg], hn[kGivensSeg];
    double A = 1.0, B = 0.0;   // composition of the segment's maps
#pragma unroll
    for (int e = 0; e < kGivensSeg; ++e) {
      const int i = i0 + e;
      cr[e] = 1.0; sr[e] = 0.0; hn[e] = 0.0;
      if (i < i1) {
        cr[e] = c[i]; sr[e] = s[i]; hn[e] = h[i + 1];
        const double a = -sr[e], b = cr[e] * hn[e];
        B = fma(a, B, b);
        A = a * A;
      }
    }
    const double h0 = h[0];
    __syncwarp();
    // inclusive scan over the lanes' segments (later segment after earlier)
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const double Ap = __shfl_up_sync(full, A, d), Bp = __shfl_up_sync(full, B, d);
      if (lane >= d) { B = fma(A, Bp, B); A = A * Ap; }
    }
    // the carried entry entering this lane's segment
    double Ae = __shfl_up_sync(full, A, 1), Be = __shfl_up_sync(full, B, 1);
    if (lane == 0) { Ae = 1.0; Be = 0.0; }
    double x = fma(Ae, h0, Be);
#pragma unroll
    for (int e = 0; e < kGivensSeg; ++e) {
      const int i = i0 + e;
      if (i < i1) {
        h[i] = fma(cr[e], x, sr[e] * hn[e]);
        x = fma(-sr[e], x, cr[e] * hn[e]);
      }
    }
    if (j == 0 ? lane == 0 : (i0 < i1 && i1 == j)) carry_out = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double a = carry_out, b = sqrt(fmax(hnext2[0], 0.0));
    const double r = hypot(a, b);
    const double cj = r > 0 ? a / r : 1.0, sj = r > 0 ? b / r : 0.0;
    cs[j] = cj; sn[j] = sj;
    h[j] = r;
    h[j + 1] = 0.0;
    rdiag = r;
    const double gj = g[j];
    g[j + 1] = -sj * gj;
    g[j] = cj * gj;
    res = fabs(sj * gj);
  }
  __syncthreads();
  double* hc = H + (i64)j * ldh;
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) hc[i] = h[i];
  r_out = rdiag;
  return res;
}

__global__ void k_givens(double* H, int ldh, double* cs, double* sn, double* g, int j, const double* hcol,
                         const double* hcol2, const double* hnext2, double* res_out) {
  pdl_entry();
  double r;
  const double res = givens_core(H, ldh, cs, sn, g, j, hcol, hcol2, hnext2, r);
  if (threadIdx.x == 0) res_out[0] = res;
}

void givens_step(double* H, int ldh, double* cs, double* sn, double* g, int j, const double* hcol,
                 const double* hcol2, const double* hnext2, double* res_out, cudaStream_t s) {
  launch_k(k_givens, 1, 64, 0, s, H, ldh, cs, sn, g, j, hcol, hcol2, hnext2, res_out);
  note_launch();
}

// y = H[0:k,0:k]^{-1} g (upper triangular, column-major with leading dim
// ldh; k <= kTriMax, the longest restart cycle), by one block of kTriMax
// threads.  The triangle is staged in shared memory and the diagonal's
// reciprocals formed in parallel; back substitution then goes column by
// column: thread i forms y_i = r_i / H_ii from its own running entry r_i,
// and after one barrier every thread t < i takes H_ti y_i off its r_t.  So
// the dependent chain per column is one product, one barrier and one FMA
// (the FP64 latency of this GPU made the one-thread row-by-row form, with
// its entries read back from memory, take about 54 us at k = 33).
constexpr int kTriMax = 64;
RBFIB_DEVFN void tri_core(const double* H, int ldh, const double* g, int k, double* y) {
  __shared__ double Hs[kTriMax][kTriMax];   // Hs[c][t] = H(t, c), t <= c
  __shared__ double dinv[kTriMax], ys[kTriMax];
  const int t = threadIdx.x;
  for (int c = 0; c < k; ++c)
    for (int i = t; i <= c; i += blockDim.x) Hs[c][i] = H[(i64)c * ldh + i];
  double r = 0.0;
  if (t < k) {
    r = g[t];
    dinv[t] = 1.0 / H[(i64)t * ldh + t];
  }
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    if (t == i) ys[i] = r * dinv[i];
    __syncthreads();
    if (t < i) r = fma(-Hs[i][t], ys[i], r);
  }
  if (t < k) y[t] = ys[t];
}

__global__ void __launch_bounds__(kTriMax) k_tri(const double* H, int ldh, const double* g, int k, double* y) {
  pdl_entry();
  tri_core(H, ldh, g, k, y);
}

void tri_solve(const double* H, int ldh, const double* g, int k, double* y, cudaStream_t s) {
  launch_k(k_tri, 1, kTriMax, 0, s, H, ldh, g, k, y);
  note_launch();
}

template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ in, B* __restrict__ out, i64 n) {
  pdl_entry();
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    out[i] = (B)in[i];
}
template <typename A, typename B>
void convert(const A* in, B* out, i64 n, cudaStream_t s) {
  const unsigned nb = (unsigned)std::min<i64>(nblk(n, 256), 152 * 8);
  if (n > 0) { launch_k(k_convert<A, B>, nb, 256, 0, s, in, out, n); note_launch(); }
}

// y = a x + b y
template <typename T>
__global__ void k_axpby(T* __restrict__ y, const T* __restrict__ x, double a, double b, i64 n) {
  pdl_entry();
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    double v = a * (double)x[i];
    if (b != 0.0) v += b * (double)y[i];
    y[i] = (T)v;
  }
}
template <typename T>
void axpby(T* y, const T* x, double a, double b, i64 n, cudaStream_t s) {
  const unsigned nb = (unsigned)std::min<i64>(nblk(n, 256), 152 * 8);
  if (n > 0) { launch_k(k_axpby<T>, nb, 256, 0, s, y, x, a, b, n); note_launch(); }
}

// x -= mean(x)  (two passes, deterministic)
__global__ void k_sub(double* x, i64 n, const double* mean_sum) {
  pdl_entry();
  const double m = mean_sum[0] / (double)n;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) x[i] -= m;
}
__global__ void k_sum_part(const double* __restrict__ x, i64 n, double* part) {
  pdl_entry();
  double acc = 0.0;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) acc += x[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}
void project_mean(double* x, i64 n, double* part, int nparts, cudaStream_t s) {
  if (n == 0) return;
  launch_k(k_sum_part, nparts, 256, 0, s, x, n, part);
  note_launch();
  launch_k(k_sum_finish, 1, 256, 0, s, part, nparts, part + nparts);
  note_launch();
  launch_k(k_sub, nparts, 256, 0, s, x, n, part + nparts);
  note_launch();
}

// bv += eta * 2 u_w / h^2 on faces adjacent (along a tangential axis) to a moving wall
template <typename T>
__global__ void k_wall_rhs(Dims d, Walls wl, double eta, T* __restrict__ bv) {
  pdl_entry();
  const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.fo[3]) return;
  int a, c[3];
  decode_face(d, t, a, c);
  double add = 0.0;
  for (int b = 0; b < 3; ++b) {
    if (b == a || d.per[b]) continue;
    const double ih2 = 1.0 / (d.h[b] * d.h[b]);
    if (c[b] == 0) add += eta * 2.0 * wl.v[2 * b][a] * ih2;
    if (c[b] == d.n[b] - 1) add += eta * 2.0 * wl.v[2 * b + 1][a] * ih2;
  }
  if (add != 0.0) bv[t] = (T)((double)bv[t] + add);
}
template <typename T>
void wall_rhs(const Dims& d, const Walls& wl, double eta, T* bv, cudaStream_t s) {
  launch_k(k_wall_rhs<T>, nblk(d.fo[3], 256), 256, 0, s, d, wl, eta, bv);
  note_launch();
}

#define INST(T)                                                                                              \
  template void multi_dot<T>(const T*, const T*, i64, int, i64, i64, double, double*, int, double*, cudaStream_t, \
                             const int*);                                                                        \
  template void multi_axpy<T>(T*, const T*, i64, int, const double*, double, i64, i64, double, double*, int,    \
                              double*, cudaStream_t, const ReorthCtl*, const int*);                              \
  template void scale_by<T>(T*, const T*, const double*, int, i64, cudaStream_t, float*);                       \
  template void axpby<T>(T*, const T*, double, double, i64, cudaStream_t);                                      \
  template void wall_rhs<T>(const Dims&, const Walls&, double, T*, cudaStream_t);
INST(double)
INST(float)
#undef INST
template void convert<double, float>(const double*, float*, i64, cudaStream_t);
template void convert<float, double>(const float*, double*, i64, cudaStream_t);

}  // namespace rbfib

// =================================================================
// Device-side state of one restart cycle of FGMRES run as a CUDA graph.
// ist: [0] columns done in this cycle k, [1] total iterations, [2] continue
// flag; dpar: [0] absolute tolerance, [1] max iterations, [2] ||w||^2 of the
// current residual w (written by the cycle's last reduction).
namespace rbfib {

template <typename T>
__global__ void k_fg_start(T* __restrict__ V0, const T* __restrict__ w, i64 n, double* __restrict__ gvec, int m,
                           int* __restrict__ ist, const double* __restrict__ dpar, float* __restrict__ V0_32,
                           IterConds conds) {
  pdl_entry();
  __shared__ double bs, fs;   // one thread per block forms beta and 1 / beta
  if (threadIdx.x == 0) {
    bs = sqrt(fmax(dpar[2], 0.0));
    fs = bs > 0.0 ? 1.0 / bs : 0.0;
  }
  __syncthreads();
  const double beta = bs, f = fs;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    const T v = (T)((double)w[i] * f);
    V0[i] = v;
    if (V0_32) V0_32[i] = (float)v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    gvec[0] = beta;
    for (int i = 1; i <= m; ++i) gvec[i] = 0.0;
    ist[0] = 0;
    ist[2] = 1;
  }
  if (blockIdx.x == 0 && (int)threadIdx.x < conds.n)
    cudaGraphSetConditional(conds.h[threadIdx.x], threadIdx.x == 0 ? 1u : 0u);
}

template <typename T>
void fg_start(T* V0, const T* w, i64 n, double* gvec, int m, int* ist, const double* dpar, cudaStream_t s,
              float* V0_32, const IterConds* conds) {
  const unsigned nb = (unsigned)std::min<i64>(nblk(n, 256), 152 * 8);
  IterConds c{};
  if (conds) c = *conds;
  launch_k(k_fg_start<T>, nb, 256, 0, s, V0, w, n, gvec, m, ist, dpar, V0_32, c);
  note_launch();
}

// Givens update of column j (as k_givens) plus the continue decision.
RBFIB_DEVFN void givens_flag_body(double* H, int ldh, double* cs, double* sn, double* g, int j, const double* hcol,
                                  const double* hcol2, const double* hnext2, double* res_out, int* ist,
                                  const double* dpar) {
  double r;
  const double res = givens_core(H, ldh, cs, sn, g, j, hcol, hcol2, hnext2, r);
  if (threadIdx.x != 0) return;
  res_out[0] = res;
  ist[0] = j + 1;
  ist[1] += 1;
  const bool cont = (res > dpar[0]) && ((double)ist[1] < dpar[1]) && isfinite(res) && (r > 0.0);
  ist[2] = cont ? 1 : 0;
}

// The last two steps of a captured Arnoldi iteration in one launch, since
// neither needs the other: blocks [0, gridDim.x - 1) normalise the new basis
// vector, v = w / sqrt(nrm2) (and its FP32 copy when out32 is not null);
// the last block applies the Givens update of column j and sets the continue
// flag, and with use_next also the condition of the next iteration's IF node
// (so no launch of its own sets it).  The update's FP64 recurrence then runs
// beside the scaling instead of in a launch of its own.
template <typename T>
__global__ void k_scale_givens(T* __restrict__ out, const T* __restrict__ in, i64 n, float* __restrict__ out32,
                               double* H, int ldh, double* cs, double* sn, double* g, int j, const double* hcol,
                               const double* hcol2, const double* nrm2, double* res_out, int* ist,
                               const double* dpar, cudaGraphConditionalHandle next, int use_next) {
  pdl_entry();
  if (blockIdx.x == gridDim.x - 1) {
    givens_flag_body(H, ldh, cs, sn, g, j, hcol, hcol2, nrm2, res_out, ist, dpar);
    if (use_next && threadIdx.x == 0) cudaGraphSetConditional(next, ist[2] ? 1u : 0u);
    return;
  }
  __shared__ double fs;
  if (threadIdx.x == 0) {
    const double dv = sqrt(fmax(nrm2[0], 0.0));
    fs = dv != 0.0 ? 1.0 / dv : 0.0;
  }
  __syncthreads();
  const double f = fs;
  const i64 stride = (i64)(gridDim.x - 1) * blockDim.x;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const T v = (T)((double)in[i] * f);
    out[i] = v;
    if (out32) out32[i] = (float)v;
  }
}

template <typename T>
void scale_givens(T* out, const T* in, i64 n, float* out32, double* H, int ldh, double* cs, double* sn, double* g,
                  int j, const double* hcol, const double* hcol2, const double* nrm2, double* res_out, int* ist,
                  const double* dpar, cudaStream_t s, const cudaGraphConditionalHandle* next) {
  const unsigned nb = (unsigned)std::min<i64>(nblk(n, 256), 152 * 8);
  launch_k(k_scale_givens<T>, nb + 1, 256, 0, s, out, in, n, out32, H, ldh, cs, sn, g, j, hcol, hcol2, nrm2,
           res_out, ist, dpar, next ? *next : cudaGraphConditionalHandle{}, next ? 1 : 0);
  note_launch();
}
template void scale_givens<double>(double*, const double*, i64, float*, double*, int, double*, double*, double*,
                                   int, const double*, const double*, const double*, double*, int*, const double*,
                                   cudaStream_t, const cudaGraphConditionalHandle*);
template void scale_givens<float>(float*, const float*, i64, float*, double*, int, double*, double*, double*, int,
                                  const double*, const double*, const double*, double*, int*, const double*,
                                  cudaStream_t, const cudaGraphConditionalHandle*);

__global__ void __launch_bounds__(kTriMax) k_tri_dev(const double* H, int ldh, const double* g, const int* ist,
                                                     double* y) {
  pdl_entry();
  tri_core(H, ldh, g, min(ist[0], kTriMax), y);
}

void tri_solve_dev(const double* H, int ldh, const double* g, const int* ist, double* y, cudaStream_t s) {
  launch_k(k_tri_dev, 1, kTriMax, 0, s, H, ldh, g, ist, y);
  note_launch();
}

// w += sign * sum_{c < ist[0]} coef[c] V_c  (column count read on the device)
template <typename T>
__global__ void k_multi_axpy_dev(T* __restrict__ w, const T* __restrict__ V, i64 ldv, const int* __restrict__ ist,
                                 const double* __restrict__ coef, double sign, i64 n) {
  pdl_entry();
  __shared__ double c[128];
  const int ncols = ist[0];
  for (int i = threadIdx.x; i < ncols; i += blockDim.x) c[i] = sign * coef[i];
  __syncthreads();
  if constexpr (sizeof(T) == 4) {
    __shared__ float c32[128];
    for (int i = threadIdx.x; i < ncols; i += blockDim.x) c32[i] = (float)c[i];
    __syncthreads();
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
      float x = (float)w[i];
      for (int k = 0; k < ncols; ++k) x = fmaf(c32[k], (float)V[(i64)k * ldv + i], x);
      w[i] = (T)x;
    }
  } else {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
      double x = (double)w[i];
      for (int k = 0; k < ncols; ++k) x = fma(c[k], (double)V[(i64)k * ldv + i], x);
      w[i] = (T)x;
    }
  }
}

template <typename T>
void multi_axpy_dev(T* w, const T* V, i64 ldv, const int* ist, const double* coef, double sign, i64 n, int nparts,
                    cudaStream_t s) {
  launch_k(k_multi_axpy_dev<T>, nparts, 256, 0, s, w, V, ldv, ist, coef, sign, n);
  note_launch();
}

template void fg_start<double>(double*, const double*, i64, double*, int, int*, const double*, cudaStream_t,
                               float*, const IterConds*);
template void fg_start<float>(float*, const float*, i64, double*, int, int*, const double*, cudaStream_t, float*,
                              const IterConds*);
template void multi_axpy_dev<double>(double*, const double*, i64, const int*, const double*, double, i64, int,
                                     cudaStream_t);
template void multi_axpy_dev<float>(float*, const float*, i64, const int*, const double*, double, i64, int,
                                    cudaStream_t);

}  // namespace rbfib

// =================================================================
// Control of device-driven solves (a whole SEM step captured as one graph:
// the restart cycles of a solve inside a WHILE node, the refinement sweeps
// inside another).  One thread each; dpar and ist as for the cycle graphs,
// plus dpar[3] = ||b||^2 of the solve.  info: [0] iterations, [1] status
// (RBFIB_OK, RBFIB_ENOCONV, RBFIB_ENAN), [2] restart cycles run, [3] second
// Gram-Schmidt passes taken; rel: the true relative residual.
namespace rbfib {

constexpr int kStOk = 0, kStNoConv = -2, kStNaN = -3;

// Start of a solve: tolerance, budget and residual of x = 0; the WHILE
// condition is whether any cycle is needed.  rtol_p / maxit_p (may be null)
// override the constants (the refinement's inner solves set them per sweep).
__global__ void k_solve_init(double* dpar, int* ist, double rtol, int maxit, const double* rtol_p,
                             const int* maxit_p, cudaGraphConditionalHandle h, int* info, double* rel) {
  pdl_entry();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double bn2 = dpar[3];
  const double rt = rtol_p ? rtol_p[0] : rtol;
  const int mi = maxit_p ? maxit_p[0] : maxit;
  dpar[0] = rt * sqrt(fmax(bn2, 0.0));
  dpar[1] = (double)mi;
  dpar[2] = bn2;
  dpar[4] = rt;
  for (int i = 0; i < 8; ++i) ist[i] = 0;
  const bool go = bn2 > 0.0 && isfinite(bn2) && mi > 0;
  info[0] = 0;
  info[1] = isfinite(bn2) ? (go || bn2 == 0.0 ? kStOk : kStNoConv) : kStNaN;
  info[2] = 0;
  info[3] = 0;
  rel[0] = 0.0;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

// After a restart cycle: the true relative residual decides whether another
// cycle runs (no convergence yet, budget left, the cycle made progress).
__global__ void k_solve_check(const double* dpar, const int* ist, cudaGraphConditionalHandle h, int* info,
                              double* rel) {
  pdl_entry();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double r = sqrt(fmax(dpar[2], 0.0) / dpar[3]);
  const bool nan = !isfinite(r);
  const bool conv = !nan && r <= dpar[4];
  const int k = ist[0], it = ist[1];
  const bool more = !nan && !conv && (double)it < dpar[1] && k > 0;
  info[0] = it;
  info[1] = conv ? kStOk : (nan ? kStNaN : kStNoConv);
  info[2] += 1;
  info[3] = ist[5];
  rel[0] = r;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

void solve_init(double* dpar, int* ist, double rtol, int maxit, const double* rtol_p, const int* maxit_p,
                cudaGraphConditionalHandle h, int* info, double* rel, cudaStream_t s) {
  launch_k(k_solve_init, 1, 32, 0, s, dpar, ist, rtol, maxit, rtol_p, maxit_p, h, info, rel);
  note_launch();
}
void solve_check(const double* dpar, const int* ist, cudaGraphConditionalHandle h, int* info, double* rel,
                 cudaStream_t s) {
  launch_k(k_solve_check, 1, 32, 0, s, dpar, ist, h, info, rel);
  note_launch();
}

// Refinement state rst: [0] ||b||^2, [1] relative residual, [2] inner
// tolerance of the next sweep; rsi: [0] inner iterations so far, [1] sweeps,
// [2] status, [3] inner iteration cap of the next sweep.
__global__ void k_refine_init(double* rst, int* rsi, cudaGraphConditionalHandle h, int* info, double* rel) {
  pdl_entry();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double bn2 = rst[0];
  const bool go = bn2 > 0.0 && isfinite(bn2);
  rst[1] = go ? 1.0 : 0.0;
  rsi[0] = 0;
  rsi[1] = 0;
  rsi[2] = isfinite(bn2) ? kStOk : kStNaN;
  info[0] = 0;
  info[1] = rsi[2];
  info[2] = 0;
  info[3] = 0;
  rel[0] = 0.0;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

// Before a sweep: its inner tolerance max(inner_tol, rtol / (2 rel)) and
// iteration cap min(budget left, m).
__global__ void k_refine_sweep(double* rst, int* rsi, double rtol, double inner_tol, int maxit, int m) {
  pdl_entry();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  rst[2] = fmax(inner_tol, 0.5 * rtol / rst[1]);
  rsi[3] = min(maxit - rsi[0], m);
}

// After a sweep: rn2 = ||b - A x||^2 (FP64); inner = the inner solve's info.
__global__ void k_refine_check(const double* rn2, double* rst, int* rsi, const int* inner, double rtol, int maxit,
                               cudaGraphConditionalHandle h, int* info, double* rel) {
  pdl_entry();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double r = sqrt(fmax(rn2[0], 0.0) / rst[0]);
  rst[1] = r;
  rsi[0] += inner[0];
  rsi[1] += 1;
  const bool nan = !isfinite(r) || inner[1] == kStNaN;
  const bool conv = !nan && r <= rtol;
  const bool more = !nan && !conv && rsi[0] < maxit && rsi[1] < 50;
  rsi[2] = conv ? kStOk : (nan ? kStNaN : kStNoConv);
  info[0] = rsi[0];
  info[1] = rsi[2];
  info[2] = rsi[1];
  info[3] += inner[3];
  rel[0] = r;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

void refine_init(double* rst, int* rsi, cudaGraphConditionalHandle h, int* info, double* rel, cudaStream_t s) {
  launch_k(k_refine_init, 1, 32, 0, s, rst, rsi, h, info, rel);
  note_launch();
}
void refine_sweep(double* rst, int* rsi, double rtol, double inner_tol, int maxit, int m, cudaStream_t s) {
  launch_k(k_refine_sweep, 1, 32, 0, s, rst, rsi, rtol, inner_tol, maxit, m);
  note_launch();
}
void refine_check(const double* rn2, double* rst, int* rsi, const int* inner, double rtol, int maxit,
                  cudaGraphConditionalHandle h, int* info, double* rel, cudaStream_t s) {
  launch_k(k_refine_check, 1, 32, 0, s, rn2, rst, rsi, inner, rtol, maxit, h, info, rel);
  note_launch();
}

// Condition of an IF node from a device int (nonzero -> 1).
__global__ void k_cond_from(const int* flag, cudaGraphConditionalHandle h) {
  pdl_entry();
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h, flag[0] ? 1u : 0u);
}
void cond_from(const int* flag, cudaGraphConditionalHandle h, cudaStream_t s) {
  launch_k(k_cond_from, 1, 32, 0, s, flag, h);
  note_launch();
}

}  // namespace rbfib
