/* rbfib.h - C ABI of the GB300 RB-FIB mobility-solve library (librbfib.so).
 *
 * The library solves the constrained saddle-point system of the Rigid-Body
 * Fluctuating Immersed Boundary method (Sprinkle, Donev, Bhalla, Patankar,
 * "Brownian dynamics of fully confined suspensions of rigid particles without
 * Green's functions", Sec. III.C, Eqs. LangevinD1-D4) and advances rigid
 * bodies with the Split-Euler-Maruyama scheme (Sec. IV.B, Algorithm 1).
 *
 * Conventions shared by every entry point
 *  - Units: h, eta, kT and dt are inputs; all lengths are in the same units.
 *  - Pointers marked "device" are CUDA device memory owned by the caller; they
 *    are read/written only during the call, in stream order on the grid's
 *    stream.  Pointers marked "host" are host memory.  The library owns its own
 *    workspaces (allocated in rbfib_create_grid / rbfib_set_bodies).
 *  - Every call is asynchronous on the grid's stream unless it says otherwise;
 *    calls that return solver information synchronise the stream.
 *  - Return value: RBFIB_OK (0) or a negative RBFIB_E* status; no call exits,
 *    traps or throws.  rbfib_last_error() gives a one-line message.
 *  - Grid layout: velocity component a lives on a-faces.  Along its own axis a
 *    the unknown faces are physical faces p = 1..n_a-1 (wall axis; the two
 *    boundary faces carry zero normal velocity) or p = 0..n_a-1 (periodic),
 *    compact index p-1 or p; along the other axes faces sit at cell centres.
 *    Arrays are x-fastest over each component's extents.  Cells (i,j,k) are
 *    x-fastest.  Blob arrays are (N_bl, 3) row-major, body arrays (N_b, 6) =
 *    (u_x, u_y, u_z, w_x, w_y, w_z) or (f, tau).
 *  - Saddle vector x = [v_x | v_y | v_z | pi | lambda (N_bl x 3) | U (N_b x 6)]
 *    (offsets from rbfib_saddle_layout).
 */
#ifndef RBFIB_H
#define RBFIB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  RBFIB_OK = 0,
  RBFIB_EINVAL = -1,     /* bad argument or unsupported configuration        */
  RBFIB_ENOCONV = -2,    /* Krylov solve hit max_iter above the tolerance    */
  RBFIB_ENAN = -3,       /* non-finite residual                              */
  RBFIB_EREJECT = -4,    /* SEM step produced an unphysical configuration    */
  RBFIB_ETIMEOUT = -5,   /* reserved: no call of this library returns it (no */
                         /* kernel waits on a flag or a peer)                */
  RBFIB_ECUDA = -6,      /* a CUDA runtime call failed                       */
  RBFIB_EINTERNAL = -7   /* internal inconsistency (device error word set)   */
};

enum { RBFIB_FP64 = 0, RBFIB_FP32_REFINED = 1 };   /* rbfib_grid_desc.precision */
enum { RBFIB_DTYPE_F64 = 0, RBFIB_DTYPE_F32 = 1 };  /* element type of a vector  */

typedef struct rbfib_grid rbfib_grid;   /* opaque; owns all device workspaces */

/* Grid and solver description (Sec. III.A).  A domain with every axis periodic
 * is rejected (EINVAL). */
typedef struct {
  int32_t n[3];              /* cells per axis                                  */
  double  h;                 /* grid spacing; cell volume dV = h^3              */
  double  eta;               /* viscosity                                       */
  int32_t periodic[3];       /* 1: periodic axis, 0: walls on both ends         */
  double  wall_vel[6][3];    /* walls -x,+x,-y,+y,-z,+z; tangential components  */
                             /* only (a normal component gives EINVAL)          */
  int32_t free_slip[6];      /* walls -x,+x,-y,+y,-z,+z: 0 = no-slip, 1 =       */
                             /* free-slip (zero normal velocity and zero        */
                             /* tangential stress; Introduction).  Ignored on   */
                             /* periodic axes.  EINVAL: a value other than 0/1, */
                             /* a moving free-slip wall, or a velocity          */
                             /* component that no no-slip wall acts on (a       */
                             /* periodic axis a whose other axes are all        */
                             /* periodic or free-slip at both ends)             */
  int32_t kernel;            /* immersed-boundary kernel (Sec. III.B): 3 = the  */
                             /* three-point Peskin kernel, 6 = the six-point    */
                             /* kernel with three continuous derivatives        */
  int32_t precision;         /* RBFIB_FP64 or RBFIB_FP32_REFINED                */
  int32_t restart;           /* FGMRES restart length m (1..64)                 */
  int32_t max_iter;          /* total Krylov iterations allowed per solve       */
  double  rtol;              /* relative residual ||b - A x||_W / ||b||_W       */
} rbfib_grid_desc;

typedef struct {
  int32_t iterations;        /* Krylov iterations (all restarts, inner solves)  */
  int32_t refinements;       /* outer FP64 refinement sweeps (FP32 mode)        */
  double  rel_residual;      /* true relative residual of the returned x        */
} rbfib_solve_info;

/* Parameters of one Split-Euler-Maruyama step (Algorithm 1) and of the
 * potentials of Sec. V (a zero strength switches a potential off).  The force
 * law of each potential: Usoft Eq. (Usoft), Yukawa Eq. (YukawaPot),
 * substrate Sec. V.B.1. */
typedef struct {
  double dt, kT;
  double delta;              /* RFD step; <= 0 selects eps^(1/3), eps = 2^-52    */
  double gravity;            /* force -gravity * z on every body                */
  double blob_gravity;       /* force -blob_gravity * z on every blob (the      */
                             /* buoyant weight of App. A's boomerang blobs),   */
                             /* with its torque about the tracking point       */
  double pair_phi0, pair_b, pair_d;      /* Usoft between body centres          */
  double wall_phi0, wall_b, wall_d;      /* Usoft between centres and walls     */
  double blob_wall_phi0, blob_wall_b, blob_wall_d;   /* Usoft blob-wall         */
  double yukawa_u0, yukawa_dh, yukawa_lambda;        /* Yukawa pair             */
  double substrate_u0, substrate_s;                  /* substrate potential     */
  const double* force_ext;   /* device (N_b, 6) extra force/torque or NULL      */
  const double* slip;        /* device (N_bl, 3) active slip or NULL            */
  int32_t no_rfd;            /* 0: Algorithm 1.  1: steps 1-5 skipped and the   */
                             /* drift terms of step 6 set to zero (the naive   */
                             /* Euler-Maruyama scheme whose biased equilibrium */
                             /* App. A shows)                                  */
  int32_t reserved;          /* must be 0                                       */
} rbfib_sem_params;

typedef struct {
  rbfib_solve_info solve_rfd;       /* Algorithm 1 step 2                        */
  rbfib_solve_info solve_stokes;    /* Algorithm 1 step 4                        */
  rbfib_solve_info solve_main;      /* Algorithm 1 step 6                        */
  int32_t rejected;                 /* 1 if the new configuration was rejected   */
} rbfib_step_info;

/* Create a grid object bound to a CUDA stream (cudaStream_t, NULL = default).
 * Allocates the fluid workspaces and the multigrid hierarchy. */
int rbfib_create_grid(const rbfib_grid_desc* desc, void* cuda_stream, rbfib_grid** out);
void rbfib_destroy(rbfib_grid* g);
const char* rbfib_last_error(const rbfib_grid* g);   /* g may be NULL */

/* Bodies as rigid agglomerates of blobs (Sec. III.B).  blob_offsets (host,
 * n_bodies+1) delimit each body's blobs; ref_blobs (device, N_bl x 3) are the
 * blob offsets in the body frame; q (device, N_b x 3) tracking points; quat
 * (device, N_b x 4) unit quaternions (w,x,y,z).  Blob positions are
 * r_i = q_p + R(quat_p) ref_i.  Builds the blob-to-cell binning and the
 * body-block preconditioner.  Synchronises the stream.  EINVAL: a body with
 * no blob, or whose blobs lie on one line (its rotation about that line
 * would be undetermined: fewer than three non-collinear blobs). */
int rbfib_set_bodies(rbfib_grid* g, int32_t n_bodies, const int32_t* blob_offsets,
                     const double* ref_blobs, const double* q, const double* quat);

/* offsets[7] = start of v_x, v_y, v_z, pi, lambda, U and the total length. */
int rbfib_saddle_layout(const rbfib_grid* g, int64_t offsets[7]);

/* y = A x for the homogeneous saddle operator (Sec. III.C; sign convention:
 *   [-eta LL  G  -S  0; -D 0 0 0; -J 0 0 K; 0 0 K^T 0],
 * self-adjoint in the inner product weighted by dV on v and pi).  x and y are
 * device vectors of the saddle layout with element type dtype.  K^T sums are
 * accumulated in FP64 for either dtype. */
int rbfib_apply_saddle(rbfib_grid* g, const void* x, void* y, int32_t dtype);

/* z = P^{-1} r: the block preconditioner used inside the Krylov solves (the
 * paper defers its preconditioner to the cited rigid-multiblob work; this one
 * is ours): a projection-method multigrid V-cycle pair for the Stokes block
 * and, for the bodies, the Schur complement with the blob mobility replaced
 * by free-space Rotne-Prager-Yamakawa blocks.  r, z: device FP64 saddle
 * vectors; computed in FP32 internally. */
int rbfib_apply_preconditioner(rbfib_grid* g, const double* r, double* z);

/* Solve the constrained system (Eqs. LangevinD1-D4) with forces/torques FT
 * (device N_b x 6), optional active slip (device N_bl x 3), optional fluid
 * forcing (device, N_f face values added to the momentum right-hand side) and
 * the moving-wall terms of the grid.  Writes U (device N_b x 6) and, if
 * x_full != NULL, the whole solution (device, saddle layout, FP64, mean(pi)=0).
 * Uses right-preconditioned FGMRES to desc.rtol.  Synchronises. */
int rbfib_mobility_solve(rbfib_grid* g, const double* FT, const double* slip,
                         const double* fluid_rhs, double* U, double* x_full,
                         rbfib_solve_info* info);

/* Replace the current blob positions (device, N_bl x 3) by independent values:
 * arms become r_i - q_p; binning, kernel stencils and the body-block
 * preconditioner are rebuilt.  For mobility problems and their adjoint
 * (blob positions as inputs); rbfib_sem_step recomputes positions from q, quat. */
int rbfib_set_blob_positions(rbfib_grid* g, const double* r);

/* Adjoint of rbfib_mobility_solve (an extension; the paper defines the forward
 * map, Eqs. LangevinD1-D4): for a loss L(U) with gradient dL_dU (device N_b x 6)
 * at the forward solution x_fwd (device, saddle layout FP64, as returned in
 * x_full; this is the checkpointed forward state), writes dL/dr (device N_bl x 3,
 * blob positions as independent inputs) and dL/dslip (device N_bl x 3); either
 * may be NULL.  Because W A is symmetric (W = diag(dV, dV, 1, 1)), the adjoint
 * system A^T y = dL/dx is the forward system A z = [0, 0, 0, dL/dU], y = W z;
 * then dL/dslip = -z_lambda and
 *   dL/dr_i = sum_a lam_ia D(z_v)_ia + sum_a z_lam,ia D(v)_ia
 *             - z_lam,i x w_p - lam_i x tau_p,
 * with D(f)_ia = d(J f)_ia / d r_i from the kernel derivative phi' and tau_p
 * the rotational part of z_U.  Grids with moving walls give EINVAL.
 * Synchronises. */
int rbfib_mobility_solve_adjoint(rbfib_grid* g, const double* dL_dU, const double* x_fwd, double* dL_dr,
                                 double* dL_dslip, rbfib_solve_info* info);

/* Unconstrained Stokes solve (Algorithm 1 step 4): -eta LL v + G pi = f,
 * -D v = 0 with homogeneous boundary conditions; f and v are device face
 * arrays (N_f, FP64); pi (device N_c, FP64, mean zero) may be NULL. */
int rbfib_stokes_solve(rbfib_grid* g, const double* f, double* v, double* pi,
                       rbfib_solve_info* info);

/* One Split-Euler-Maruyama step (Algorithm 1, steps 1-7) from the
 * configuration (q, quat) (device, in/out).  The whole step runs as one
 * device-driven CUDA graph (restart cycles and refinement sweeps in WHILE
 * nodes, the rejection test on the device) captured at the first call and
 * again whenever p's contents or the q / quat pointers change; the call
 * synchronises once at the end.  With RBFIB_NO_GRAPHS=1 or
 * RBFIB_NO_STEP_GRAPH=1 in the environment (read when the grid is created),
 * or while a kernel timer is active, the host orchestrates the step.  Random numbers come from
 * Philox4x64-10 with key (seed, 0) and counter (block, step,
 * (attempt << 32) | purpose, 0).  On an unphysical new configuration (a blob
 * outside the domain along a wall axis) q and quat are left unchanged and the
 * call returns RBFIB_EREJECT; retry with attempt + 1 (Sec. V). */
int rbfib_sem_step(rbfib_grid* g, const rbfib_sem_params* p, uint64_t seed, uint64_t step,
                   uint32_t attempt, double* q, double* quat, rbfib_step_info* info);

/* ---- ensembles of independent systems ------------------------------------ */

/* An ensemble of independent suspensions (the many independent trajectories
 * of Sec. V), e.g. cuboids of different sizes.  System i gets a grid created
 * from descs[i] (host array of n_sys descriptors); the batch owns the grids
 * and n_workers streams.  Set each system's bodies with
 * rbfib_set_bodies(rbfib_batch_grid(b, i), ...).  The CUDA runtime maps
 * streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware queues (8 unless that
 * variable is set before the context is created); more workers than queues
 * share queues and serialise. */
typedef struct rbfib_batch rbfib_batch;
int rbfib_create_batch(int32_t n_sys, const rbfib_grid_desc* descs, int32_t n_workers, rbfib_batch** out);
void rbfib_destroy_batch(rbfib_batch* b);
rbfib_grid* rbfib_batch_grid(rbfib_batch* b, int32_t sys);   /* NULL if out of range */

/* One Split-Euler-Maruyama step of every system (Algorithm 1): system i uses
 * params[i], seeds[i], attempts[i] (NULL = 0) and its device configuration
 * q[i], quat[i] (host arrays of device pointers).  Each system's step is one
 * launch of its device-driven step graph (see rbfib_sem_step), captured at
 * its first step and again whenever its params or q / quat pointers change.
 * Systems, largest first, are dealt round-robin to the worker streams; the
 * workers' host threads launch in parallel without waiting, then every
 * stream is synchronised once.  A system's grid stays bound to the stream of
 * its worker, so a call made on a batch grid between batch steps runs on one
 * of the batch's streams.  status[i] receives each system's rbfib_sem_step
 * status (RBFIB_EREJECT leaves that system unchanged); infos may be NULL.
 * Returns the first status other than OK / EREJECT, else OK.  Synchronises
 * every worker stream. */
int rbfib_batch_sem_step(rbfib_batch* b, const rbfib_sem_params* params, const uint64_t* seeds, uint64_t step,
                         const uint32_t* attempts, double* const* q, double* const* quat, rbfib_step_info* infos,
                         int32_t* status);

/* One-graph form of rbfib_batch_sem_step (on = 1; 0, the default, restores
 * the worker streams above).  Once every system's step can run device-driven
 * (from its second step on: a coupled body block is first built on the
 * host), all systems' steps are captured as parallel branches of one CUDA
 * graph, each branch copying its system's seed / step / attempt from pinned
 * host memory, running the step and copying its report back; a batch step is
 * then one launch of that graph on a stream of the batch and one
 * synchronisation.  The graph is captured again when any system's params or
 * q / quat pointers change.  Steps that cannot use it (a system not ready,
 * a failed capture) run on the worker streams as before.  Returns
 * RBFIB_EINVAL for a NULL batch or on values other than 0 and 1.
 * rbfib_batch_graph_steps counts the batch steps run as one graph launch
 * (-1 for a NULL batch). */
int rbfib_batch_set_one_graph(rbfib_batch* b, int32_t on);
int64_t rbfib_batch_graph_steps(const rbfib_batch* b);

/* Body block of the preconditioner: dense = 1 when it is the coupled
 * all-blob RPY block (at least two bodies, 3 N_bl <= 1536, 6 N_b <= 384),
 * else 0 (per-shape blocks).  The coupled block's inverse RPY matrix is
 * rebuilt for every new configuration (rbfib_set_bodies,
 * rbfib_set_blob_positions, each SEM step): by Gauss-Jordan after
 * rbfib_set_bodies; otherwise by eight Newton-Schulz steps from the previous
 * inverse, rotated with each body's rotation since it was built (when the
 * orientations are known: not after rbfib_set_blob_positions), if that
 * start's residual ||I - M X||_F is at most 0.95, else by Gauss-Jordan.
 * warm_starts counts the builds that took the Newton-Schulz path.  Either
 * pointer may be NULL. */
int rbfib_body_block_info(const rbfib_grid* g, int32_t* dense, int64_t* warm_starts);

/* *device_driven = 1 if the grid's last SEM step ran as the device-driven
 * step graph (see rbfib_sem_step), 0 if the host orchestrated it. */
int rbfib_step_mode(const rbfib_grid* g, int32_t* device_driven);

/* Gram-Schmidt statistics of the grid's Krylov solves since it was created:
 * Arnoldi iterations and how many of them took the second (re-
 * orthogonalising) pass of classical Gram-Schmidt.  The second pass runs only
 * when the first leaves less than a fraction tau of the new vector's norm
 * (tau = 1e-3 for FP64 bases, 1e-2 for the FP32 bases of the refinement's inner solves); otherwise the
 * orthogonality lost is at most about eps / tau.  Either pointer may be
 * NULL. */
int rbfib_krylov_stats(const rbfib_grid* g, int64_t* iterations, int64_t* second_passes);

/* Threads per block the autotuner picked for this grid's finest-level
 * kernels: out[0] FP64 Stokes operator, out[1] FP32 Stokes operator (0 on
 * uniform spacing, whose Stokes kernels have fixed tile shapes), out[2]
 * velocity smoothing sweep, out[3] pressure smoothing sweep (as 32 x n/32
 * blocks on uniform spacing). */
int rbfib_tuned_blocks(const rbfib_grid* g, int32_t out[4]);

/* ---- building blocks of the hot path, exposed for parity checks ---------- */

/* Blob-to-cell counting sort of the current bodies: perm (device int32 N_bl)
 * and cell_offsets (device int32 N_c + 1); the blobs of cell c are
 * perm[cell_offsets[c] .. cell_offsets[c+1]) in increasing blob id.  Cell
 * index: floor(x/h) per axis, clamped on wall axes, wrapped on periodic ones. */
int rbfib_binning(rbfib_grid* g, int32_t* perm, int32_t* cell_offsets);

/* Current blob positions r (device, N_bl x 3, FP64). */
int rbfib_blob_positions(rbfib_grid* g, double* r);

/* Raw random words of the counter-based generator behind every random draw
 * of the method (the noise of Sec. IV.B and Eq. LangevinD1 is drawn from it):
 * Philox4x64-10 (Salmon et al., SC11) with key (seed, 0) and counter
 * (block, step, (attempt << 32) | purpose, 0), for the n_blocks blocks
 * first_block, first_block + 1, ...; out (device, 16-byte aligned,
 * 4 n_blocks uint64) receives each block's four words in order.  A null or
 * misaligned out with n_blocks > 0 gives RBFIB_EINVAL. */
int rbfib_philox_words(rbfib_grid* g, uint64_t seed, uint64_t step, uint32_t attempt, uint32_t purpose,
                       uint64_t first_block, int64_t n_blocks, uint64_t* out);

/* count standard normals of the Philox stream (seed, step, attempt, purpose)
 * into out (device FP64): normal g is lane g%4 of block g/4 (Box-Muller on the
 * block's uniforms u = (2 (word >> 12) + 1) 2^-53, lanes (0,1) and (2,3)). */
int rbfib_philox_normals(rbfib_grid* g, uint64_t seed, uint64_t step, uint32_t attempt,
                         uint32_t purpose, int64_t count, double* out);

/* Fluid forcing sqrt(2 eta kT / (dV dt)) DD W of Eq. LangevinD1 for the
 * stress drawn from purpose 1 of the Philox stream (device out, N_f FP64). */
int rbfib_stochastic_forcing(rbfib_grid* g, double kT, double dt, uint64_t seed,
                             uint64_t step, uint32_t attempt, double* out);

/* Spreading f = S lambda (device lambda N_bl x 3 -> device f N_f, FP64) and
 * interpolation u = J v (device v N_f -> device u N_bl x 3, FP64; with_walls
 * adds the ghost values of moving walls) at the current blob positions. */
int rbfib_spread(rbfib_grid* g, const double* lambda, double* f);
int rbfib_interpolate(rbfib_grid* g, const double* v, double* u, int32_t with_walls);

/* Body forces and torques of the potentials in p at the current configuration
 * (device out N_b x 6). */
int rbfib_body_forces(rbfib_grid* g, const rbfib_sem_params* p, double* out);

/* Allocation-free variant of rbfib_stochastic_forcing, for callers that cannot
 * allocate device memory: code running inside a custom allocator or memory
 * pool (where a nested cudaMalloc would re-enter it), or applications that
 * plan all of their device memory up front.  It needs no grid object: desc
 * gives the grid (n, h, periodic, eta; other fields ignored).  It writes the
 * same forcing as rbfib_stochastic_forcing (device out, N_f FP64) on the given
 * stream and calls no cudaMalloc, cudaFree or allocating library routine.
 *  - The stress field is drawn into a fixed device array of 2^20 doubles
 *    (8 MiB) that is part of the library image; every device that loads the
 *    library holds it until the process exits.  Grids whose stress field has
 *    more values (about 9 per cell) are rejected with RBFIB_EINVAL.
 *  - Each call made outside stream capture looks up the array's device
 *    address on the current device (so a context that was reset and
 *    re-created is handled); a call made while the stream is capturing uses
 *    the address found by the last call outside capture on that device, so
 *    make the first call on each device before any stream capture (a first
 *    call during capture returns RBFIB_EINVAL).
 *  - desc->periodic values other than 0 and 1 give RBFIB_EINVAL, as in
 *    rbfib_create_grid.
 *  - Every call shares the array and overwrites all of it that it uses; calls
 *    that overlap on the GPU (other streams, other threads) race.
 *  - errbuf (optional, errlen bytes) receives a one-line message.
 * The paper has no counterpart to this entry point. */
int rbfib_stochastic_forcing_static(const rbfib_grid_desc* desc, double kT, double dt, uint64_t seed,
                                    uint64_t step, uint32_t attempt, double* out, void* cuda_stream,
                                    char* errbuf, size_t errlen);

/* ---- instrumentation --------------------------------------------------- */

/* Number of kernel launches the library has issued so far (all grids). */
uint64_t rbfib_launch_count(void);

/* Kernel timer for roofline reports.  which: 0 off, 1 saddle matvec (Stokes
 * stencil + body rows), 2 finest-level velocity smoothing half sweep, 3
 * Krylov multi-column inner product, 4 Krylov multi-axpy, 5 exact solve of
 * the coarse multigrid level by fast diagonalisation (one 8-CTA cluster per
 * grid).  While a class is selected, the stream first idles for about 25 us
 * before each of its launches (so that the host has queued the launch and its
 * closing event), CUDA events are recorded on the grid's stream around each
 * launch, and the algorithmic bytes and floating-point operations of each
 * launch are added up:
 *   matvec: 2 n s + 24 N_bl + 56 N_b bytes; 10 N_f + 6 N_c + 400 N_bl operations
 *   smoothing half sweep: 2 N_f s bytes; 4.5 N_f operations
 *   inner product over k columns: (k + 1) n s bytes; 2 k n operations
 *   multi-axpy over k columns: (k + 2) n s bytes; 2 (k + 1) n operations
 *   coarse solve: per grid of P points and basis table of t floats,
 *     4 (2 P + t) bytes; 4 P (e_x + e_y + e_z) + P operations
 * (s = element size, n = vector length).  Selecting resets the counters.
 * _read synchronises the stream and returns the summed event time (ms), the
 * launch count, the bytes and the operations (each pointer may be NULL). */
int rbfib_kernel_timer(rbfib_grid* g, int32_t which);
int rbfib_kernel_timer_read(rbfib_grid* g, double* total_ms, int64_t* launches, double* alg_bytes,
                            double* alg_flops);

/* Per-launch overhead of the timer's event bracket: the median (us, over reps
 * in [1, 10000]) of the event time that the same bracket (idle wait, opening
 * event, one launch, closing event) records around an empty kernel on the
 * grid's stream.  Each timed launch's event time exceeds the kernel's own
 * duration by about this much; subtracting it gives a lower bound on that
 * duration (the empty kernel's own run time is subtracted too).
 * Synchronises the stream. */
int rbfib_kernel_timer_overhead(rbfib_grid* g, int32_t reps, double* median_us);

#ifdef __cplusplus
}
#endif
#endif /* RBFIB_H */
