// Launchers of the device kernels, grouped by file.  All launches are
// asynchronous on the given stream.
#pragma once
#include <string>
#include <vector>

#include "common.cuh"

namespace rbfib {

struct Walls { double v[6][3]; };   // wall velocities, walls -x,+x,-y,+y,-z,+z

// Device views of the bodies of one configuration.
struct BodyView {
  int nb = 0, nbl = 0;
  const int* boff = nullptr;     // nb + 1
  const int* bob = nullptr;      // body of blob, nbl
  const int* perm = nullptr;     // blob order sorted by cell (may be null)
  const double* ref = nullptr;   // nbl x 3 (body frame)
  const double* q = nullptr;     // nb x 3
  const double* quat = nullptr;  // nb x 4
  const double* r = nullptr;     // nbl x 3 blob positions
  const double* arm = nullptr;   // nbl x 3 r - q
  const BlobStencil<double>* st64 = nullptr;   // 3 nbl folded kernel stencils
  const BlobStencil<float>* st32 = nullptr;
};

struct PrecondView {
  int max_blobs = 0;
  const int* shape_of = nullptr;
  const i64* minv_off = nullptr;
  const double* minv = nullptr;
  const float* minv32 = nullptr;
  const double* nmat = nullptr;
  const int* shape_ref_blob = nullptr;
};

struct Potentials {
  double gravity;
  double blob_g;     // force -blob_g z on every blob
  double pair_phi0, pair_b, pair_d;
  double wall_phi0, wall_b, wall_d;
  double bw_phi0, bw_b, bw_d;
  double yuk_u0, yuk_dh, yuk_lambda;
  double sub_u0, sub_s;
};

// Offsets and extents of the nine stress blocks (global order: for a = x,y,z:
// W_aa then W_ab for the other two axes b in increasing order).
struct StressLayout {
  i64 off[3][3];
  int ext[3][3][3];
  i64 total;
};

// k_stokes.cu
template <typename T> void stokes_apply(const Dims&, T eta, const T* v, const T* p, T* yv, T* yp, cudaStream_t,
                                        int block = 256);
template <typename T> void vel_rbgs(const Dims&, T eta, int color, T* u, const T* rhs, cudaStream_t, int block = 256);
// The first two half sweeps (colours 0 then 1) from a zero guess in one
// launch; false, with nothing launched, when the spacing is not uniform.
template <typename T> bool vel_first2(const Dims&, T eta, T* u, const T* rhs, cudaStream_t, int bs);
template <typename T> bool p_first2(const Dims&, T* u, const T* rhs, cudaStream_t, int bs);
template <typename T> void vel_first(const Dims&, T eta, T* u, const T* rhs, cudaStream_t);
template <typename T> void vel_restrict_res(const Dims&, const Dims&, int3, T eta, const T* uf, const T* rhsf,
                                            T* rc, cudaStream_t);
template <typename T> void p_first(const Dims&, T* u, const T* rhs, cudaStream_t);
template <typename T> void p_restrict_res(const Dims&, const Dims&, int3, const T* uf, const T* rhsf, T* rc,
                                          cudaStream_t);
template <typename T> void vel_prolong(const Dims&, const Dims&, int3, const T*, T*, cudaStream_t);
template <typename T> void vel_coarse(const Dims&, T eta, T* u, const T* rhs, int sweeps, cudaStream_t);
template <typename T> void p_rbgs(const Dims&, int color, T* u, const T* rhs, cudaStream_t, int block = 256);
template <typename T> void p_prolong(const Dims&, const Dims&, int3, const T*, T*, cudaStream_t);
template <typename T> void p_coarse(const Dims&, T* u, T* rhs, int sweeps, cudaStream_t);
// pi64 / v64: FP64 copies of the outputs (null: none)
template <typename T> void div_q(const Dims&, T eta, const T* vt, const T* rpi, T* q, T* pi, double* pi64,
                                 cudaStream_t);
template <typename T> void add_grad(const Dims&, const T* phi, T* v, double* v64, cudaStream_t);

// Exact solve on a coarse multigrid level by fast diagonalisation (k_fdsolve.cu).
// The level operator of each grid (a velocity component of -eta LL, or the
// pressure operator -D G) is a Kronecker sum of 1D second differences; with
// orthonormal 1D eigenbases Q_x, Q_y, Q_z and eigenvalues l_x, l_y, l_z,
// A^-1 = (Q_x (x) Q_y (x) Q_z) diag(1 / (s (l_x + l_y + l_z))) (Q_x (x) Q_y (x) Q_z)^T,
// the zero mode of a singular operator dropped (pseudo-inverse).
constexpr int kFDMaxPoints = 48 * 48 * 48;  // points of one grid
constexpr int kFDLine = 48;                 // points along one axis
constexpr int kFDCtas = 8;           // CTAs (one cluster) per grid
constexpr int kFDThreads = 256;
// shared memory bound per CTA: table (3 axes, two padded e x e bases and e
// eigenvalues each) and two slab buffers of ceil(e_z / kFDCtas) planes
constexpr int kFDMaxSmem = (int)sizeof(float) * (3 * (2 * kFDLine * kFDLine + kFDLine) + 4 +
                                                 2 * (((kFDLine + kFDCtas - 1) / kFDCtas) * kFDLine * kFDLine + 4));
struct FDGrid {
  int e[3];        // extents
  long long off;   // offset of the grid in the level's solution / rhs arrays
  int tab0, tabn;  // segment of the basis table: per axis Q (e x e), Q^T (e x e), eigenvalues (e)
  float scale;     // operator scale (eta for velocity, 1 for pressure)
};
struct FDParams {
  int ng;          // grids (3 face components or 1 pressure grid), one CTA each
  FDGrid g[3];
  const float* tab;
  int smem;        // dynamic shared memory bytes of the largest grid
};
// Bases of every grid of a level; false if some grid exceeds the limits.
bool fd_plan(const Dims& d, bool faces, double eta, std::vector<float>& tab, FDParams& P, std::string& why);
void fd_solve(const FDParams& P, float* u, const float* rhs, cudaStream_t s);
void fd_solve_wide(const FDParams& P, float* u, const float* rhs, float* tmp, cudaStream_t s);
bool fd_use_wide(const FDParams& P);

// k_ib.cu
void geometry(int nbl, const int* bob, const double* ref, const double* q, const double* quat,
              double* r, double* arm, cudaStream_t);
void binning(const Dims&, int nbl, const double* r, int* perm, int* off, int* key, int* count, int* fill,
             int* bsum, cudaStream_t);
template <typename T> void saddle_bodies(const Dims&, const BodyView&, const T* v, const T* lam, const T* U,
                                         T* yv, T* ylam, T* yU, cudaStream_t);
template <typename T> void spread(const Dims&, int nbl, const int* perm, const double* r, const T* lam,
                                  double scale, T* f, cudaStream_t);
template <typename T> void interp(const Dims&, const Walls&, int nbl, const double* r, const T* v, double alpha,
                                  double beta, double gamma, T* out, cudaStream_t);
template <typename T> void interp_res(const Dims&, const BodyView&, const T* v, const T* rl, T* out, cudaStream_t);
// zlam64 / zU64: FP64 copies of the outputs (null: none)
template <typename T> void body_precond(const BodyView&, const PrecondView&, const T* sres, const T* rU,
                                        T* zlam, T* zU, double* zlam64, double* zU64, cudaStream_t);
void stencil_build(const Dims&, int nbl, const double* r, BlobStencil<double>* s64, BlobStencil<float>* s32,
                   cudaStream_t);
void interp_tab(const Dims&, const BodyView&, const double* v, double alpha, double beta, double* out, cudaStream_t);
void spread_tab(const Dims&, const BodyView&, const double* lam, double scale, double* f, cudaStream_t);
void kt_apply(int nb, const int* boff, const double* arm, const double* lam, double alpha, double beta,
              double* out, cudaStream_t);
void k_apply(int nbl, const int* bob, const double* arm, const double* U, double alpha, double beta,
             double* out, cudaStream_t);
void body_forces(const Dims&, const Potentials&, const BodyView&, const double* fext, double* out, cudaStream_t);
void wft(int nb, const double* wn, const double* Lp, double kT, double* out, cudaStream_t);
void move_bodies(int nb, const double* q, const double* quat, const double* vec6, const double* Lp, double a,
                 double* qo, double* quato, cudaStream_t);
void outside_check(const Dims&, int nbl, const double* r, int* flag, cudaStream_t);
void accept_step(int nb, const int* flag, const int* st, int nst, int st_stride, const double* qn,
                 const double* quatn, double* q, double* quat, int* rejected, cudaStream_t);
void arms_from_positions(int nbl, const int* bob, const double* r, const double* q, double* arm, cudaStream_t);
void adjoint_positions(const Dims&, int nbl, const int* bob, const double* r, const double* v, const double* lam,
                       const double* U, const double* zv, const double* zl, const double* zU, double* dr,
                       cudaStream_t);

// k_body.cu
cudaError_t dense_body_build(int nbl, int nb, const int* boff, const int* bob, const double* r, const double* arm,
                             const double* qnew, const double* qold, double a, double eta, float* Minv, float* P,
                             double* N, int* status, float* Mw, float* Tw, float* Uw, double* ss, double* ss_host,
                             bool warm, cudaStream_t, bool* used);
void dense_body_warm_start(int nbl, const int* bob, const double* r, const double* qnew, const double* qold,
                           double a, double eta, float* Minv, float* Mw, float* Tw, double* ss, cudaStream_t);
void dense_body_ns(int nbl, float* Minv, const float* Mw, float* Tw, float* Uw, double* ss, cudaStream_t);
void dense_body_gj(int nbl, float* Minv, const float* Mw, int* status, cudaStream_t);
void dense_body_finish(int nbl, int nb, const int* boff, const double* arm, const float* Minv, float* P, double* N,
                       int* status, cudaStream_t);
void ns_decide(const double* ss, cudaGraphConditionalHandle h, long long* warm, cudaStream_t);
// With tab (the configuration's stencil table of type T), the kernel forms
// its input s = rl + J v itself and stores it in sres_out; sres is unused.
template <typename T> void dense_body_apply(int nbl, int nb, const int* boff, const int* bob, const double* arm,
                                            const float* Minv, const float* P, const double* N, const T* sres,
                                            const T* rU, T* zlam, T* zU, double* zlam64, double* zU64,
                                            cudaStream_t, const Dims* d = nullptr,
                                            const BlobStencil<T>* tab = nullptr, const T* v = nullptr,
                                            const T* rl = nullptr, T* sres_out = nullptr);

// k_krylov.cu
// A grid's partial-sum buffer: nparts x kPartCols doubles, 8 spare doubles,
// then kPartCounters counters (unsigned) of the last-block reductions:
// [0, kPartCols) one per inner-product column, kAxpyCounter for the norm of
// a multi-axpy, kDotCounter for the register-blocked inner products.  The counters start at zero and every reduction resets its own.
constexpr int kPartCols = 130;
constexpr int kPartCounters = 160;
constexpr int kAxpyCounter = 140;
constexpr int kDotCounter = 141;     // the register-blocked multi-column inner product
inline size_t part_buffer_doubles(int nparts) { return (size_t)nparts * kPartCols + 8 + kPartCounters / 2; }
inline unsigned* part_counters(double* part, int nparts) {
  return reinterpret_cast<unsigned*>(part + (size_t)nparts * kPartCols + 8);
}
// Weighted inner products <x, y>_W with weight wf on the first nfl entries
// and 1 on the rest.
// Selective re-orthogonalisation in the Gram-Schmidt of FGMRES.  A first
// projection w' = w - V h (h = V^T w) whose result keeps at least a fraction
// tau of w (||w'||^2 >= tau2 (||w'||^2 + ||h||^2), Pythagoras for an
// orthonormal V) lost at most about eps / tau of orthogonality, and its
// second projection is skipped: the multi-axpy that forms w' writes
// *flag = 1 when the second pass is needed (else 0) and zeroes its
// coefficients h2[0..k), which the second pass overwrites when it runs.
struct ReorthCtl {
  int* flag;        // [0] the decision, [1] count of second passes taken
  double* h2;
  double tau2;
  // inside a captured graph: the handle of the IF node around the second
  // pass, set to the decision as well (use_handle = 1)
  cudaGraphConditionalHandle handle;
  int use_handle;
};
// gate (may be null): device flag; the launch does nothing when it is 0.
template <typename T> void multi_dot(const T* w, const T* V, i64 ldv, int ncols, i64 n, i64 nfl, double wf,
                                     double* part, int nparts, double* out, cudaStream_t,
                                     const int* gate = nullptr);
template <typename T> void multi_axpy(T* w, const T* V, i64 ldv, int ncols, const double* coef, double sign,
                                      i64 n, i64 nfl, double wf, double* part, int nparts, double* nrm2,
                                      cudaStream_t, const ReorthCtl* ctl = nullptr, const int* gate = nullptr);
void gpu_delay(long long cycles, cudaStream_t);
void gpu_empty(cudaStream_t);
// out = in * f with f = denom (invert 0), 1 / denom (1) or 1 / sqrt(denom) (2);
// out32, if not null, receives the same values rounded to FP32.
template <typename T> void scale_by(T* out, const T* in, const double* denom, int invert, i64 n, cudaStream_t,
                                    float* out32 = nullptr);
void givens_step(double* H, int ldh, double* cs, double* sn, double* g, int j, const double* hcol,
                 const double* hcol2, const double* hnext2, double* res_out, cudaStream_t);
void tri_solve(const double* H, int ldh, const double* g, int k, double* y, cudaStream_t);
template <typename A, typename B> void convert(const A* in, B* out, i64 n, cudaStream_t);
template <typename T> void axpby(T* y, const T* x, double a, double b, i64 n, cudaStream_t);
template <typename T> void wall_rhs(const Dims&, const Walls&, double eta, T* bv, cudaStream_t);
void project_mean(double* x, i64 n, double* part, int nparts, cudaStream_t);

// FGMRES restart cycle as a graph (k_krylov.cu).  The IF conditions of a
// cycle's iterations: iteration j's Givens update sets the condition of
// iteration j + 1; the cycle start resets them all (condition 0 to 1, the
// rest to 0), since a cycle that runs again inside a WHILE body keeps the
// values of its previous pass.
constexpr int kMaxRestart = 64;
struct IterConds {
  cudaGraphConditionalHandle h[kMaxRestart];
  int n;
};
template <typename T> void fg_start(T* V0, const T* w, i64 n, double* gvec, int m, int* ist, const double* dpar,
                                    cudaStream_t, float* V0_32 = nullptr, const IterConds* conds = nullptr);
template <typename T>
void scale_givens(T* out, const T* in, i64 n, float* out32, double* H, int ldh, double* cs, double* sn, double* g,
                  int j, const double* hcol, const double* hcol2, const double* nrm2, double* res_out, int* ist,
                  const double* dpar, cudaStream_t s, const cudaGraphConditionalHandle* next = nullptr);
void tri_solve_dev(const double* H, int ldh, const double* g, const int* ist, double* y, cudaStream_t);
// control of device-driven solves (k_krylov.cu)
void solve_init(double* dpar, int* ist, double rtol, int maxit, const double* rtol_p, const int* maxit_p,
                cudaGraphConditionalHandle h, int* info, double* rel, cudaStream_t);
void solve_check(const double* dpar, const int* ist, cudaGraphConditionalHandle h, int* info, double* rel,
                 cudaStream_t);
void refine_init(double* rst, int* rsi, cudaGraphConditionalHandle h, int* info, double* rel, cudaStream_t);
void refine_sweep(double* rst, int* rsi, double rtol, double inner_tol, int maxit, int m, cudaStream_t);
void refine_check(const double* rn2, double* rst, int* rsi, const int* inner, double rtol, int maxit,
                  cudaGraphConditionalHandle h, int* info, double* rel, cudaStream_t);
void cond_from(const int* flag, cudaGraphConditionalHandle h, cudaStream_t);
template <typename T> void multi_axpy_dev(T* w, const T* V, i64 ldv, const int* ist, const double* coef,
                                          double sign, i64 n, int nparts, cudaStream_t);

// k_noise.cu
void philox_normals(unsigned long long seed, unsigned long long step, unsigned attempt, unsigned purpose,
                    i64 count, double* out, cudaStream_t);
void philox_normals_p(const unsigned long long* sp, unsigned purpose, i64 count, double* out, cudaStream_t);
void philox_words(unsigned long long seed, unsigned long long step, unsigned attempt, unsigned purpose,
                  unsigned long long first, i64 n_blocks, unsigned long long* out, cudaStream_t);
void stress_divergence(const Dims&, const StressLayout&, const double* W, double c, double* out, cudaStream_t);

}  // namespace rbfib
