// Fluctuating stress (Sec. III.A, Eq. LangevinD1): Philox4x64-10 normals and
// the tensor divergence DD W with sqrt(2) weights on wall edges.
#include "common.cuh"
#include "kernels.cuh"

namespace rbfib {

static inline unsigned nblk(i64 n, int bs) { return (unsigned)((n + bs - 1) / bs); }

__global__ void k_philox_normals(unsigned long long seed, unsigned long long step, unsigned attempt,
                                 unsigned purpose, i64 count, double* __restrict__ out) {
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
  if (nb > 0) { k_philox_normals<<<nblk(nb, 128), 128, 0, s>>>(seed, step, attempt, purpose, count, out); note_launch(); }
}

// out(face of component a) = c * [ (W_aa(right) - W_aa(left)) / h_a
//                                  + sum_{b != a} (c+ W_ab(node j+1) - c- W_ab(node j)) / h_b ]
__global__ void k_stress_div(Dims d, StressLayout L, const double* __restrict__ W, double c, double* __restrict__ out) {
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
      if (lo[b] == 0) clo = 1.4142135623730951;
      if (hi[b] == d.n[b]) chi = 1.4142135623730951;
    }
    acc += (chi * Wab[flat3(e, hi[0], hi[1], hi[2])] - clo * Wab[flat3(e, lo[0], lo[1], lo[2])]) / d.h[b];
  }
  out[t] = c * acc;
}

void stress_divergence(const Dims& d, const StressLayout& L, const double* W, double c, double* out, cudaStream_t s) {
  k_stress_div<<<nblk(d.fo[3], 256), 256, 0, s>>>(d, L, W, c, out);
  note_launch();
}

}  // namespace rbfib
