"""ctypes binding of librbfib (include/rbfib.h).

Argument marshalling only: tensors are checked (CUDA device, dtype,
contiguity, length) and their device pointers handed to the C entry points,
which run on torch's current CUDA stream.  Names follow the C ABI without the
``rbfib_`` prefix.
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librbfib.so")

OK, EINVAL, ENOCONV, ENAN, EREJECT, ETIMEOUT, ECUDA, EINTERNAL = 0, -1, -2, -3, -4, -5, -6, -7
FP64, FP32_REFINED = 0, 1
DTYPE_F64, DTYPE_F32 = 0, 1
PURPOSE_FLUID, PURPOSE_BODY = 1, 2


class GridDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("h", ctypes.c_double), ("eta", ctypes.c_double),
                ("periodic", ctypes.c_int32 * 3), ("wall_vel", (ctypes.c_double * 3) * 6),
                ("free_slip", ctypes.c_int32 * 6), ("kernel", ctypes.c_int32), ("precision", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("rtol", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("rel_residual", ctypes.c_double)]

    def as_dict(self):
        return {"iterations": self.iterations, "refinements": self.refinements,
                "rel_residual": self.rel_residual}


class SemParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "dt", "kT", "delta", "gravity", "blob_gravity", "pair_phi0", "pair_b", "pair_d", "wall_phi0", "wall_b", "wall_d",
        "blob_wall_phi0", "blob_wall_b", "blob_wall_d", "yukawa_u0", "yukawa_dh", "yukawa_lambda",
        "substrate_u0", "substrate_s")] + [("force_ext", ctypes.c_void_p), ("slip", ctypes.c_void_p),
                                           ("no_rfd", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class StepInfo(ctypes.Structure):
    _fields_ = [("solve_rfd", SolveInfo), ("solve_stokes", SolveInfo), ("solve_main", SolveInfo),
                ("rejected", ctypes.c_int32)]

    def as_dict(self):
        return {"solve_rfd": self.solve_rfd.as_dict(), "solve_stokes": self.solve_stokes.as_dict(),
                "solve_main": self.solve_main.as_dict(), "rejected": self.rejected}


_lib = None


def lib():
    """Load librbfib.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"librbfib.so not found at {LIB_PATH}; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, D, I32, I64, U32, U64 = (ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_int64,
                                    ctypes.c_uint32, ctypes.c_uint64)
        sig = {
            "rbfib_create_grid": ([ctypes.POINTER(GridDesc), P, ctypes.POINTER(P)], I32),
            "rbfib_destroy": ([P], None),
            "rbfib_last_error": ([P], ctypes.c_char_p),
            "rbfib_set_bodies": ([P, I32, ctypes.POINTER(ctypes.c_int32), P, P, P], I32),
            "rbfib_saddle_layout": ([P, ctypes.POINTER(ctypes.c_int64)], I32),
            "rbfib_apply_saddle": ([P, P, P, I32], I32),
            "rbfib_apply_preconditioner": ([P, P, P], I32),
            "rbfib_mobility_solve": ([P, P, P, P, P, P, ctypes.POINTER(SolveInfo)], I32),
            "rbfib_stokes_solve": ([P, P, P, P, ctypes.POINTER(SolveInfo)], I32),
            "rbfib_set_blob_positions": ([P, P], I32),
            "rbfib_mobility_solve_adjoint": ([P, P, P, P, P, ctypes.POINTER(SolveInfo)], I32),
            "rbfib_sem_step": ([P, ctypes.POINTER(SemParams), U64, U64, U32, P, P, ctypes.POINTER(StepInfo)], I32),
            "rbfib_binning": ([P, P, P], I32),
            "rbfib_blob_positions": ([P, P], I32),
            "rbfib_philox_words": ([P, U64, U64, U32, U32, U64, I64, P], I32),
            "rbfib_philox_normals": ([P, U64, U64, U32, U32, I64, P], I32),
            "rbfib_stochastic_forcing": ([P, D, D, U64, U64, U32, P], I32),
            "rbfib_spread": ([P, P, P], I32),
            "rbfib_interpolate": ([P, P, P, I32], I32),
            "rbfib_body_forces": ([P, ctypes.POINTER(SemParams), P], I32),
            "rbfib_stochastic_forcing_static": ([ctypes.POINTER(GridDesc), D, D, U64, U64, U32, P, P,
                                                 ctypes.c_char_p, ctypes.c_size_t], I32),
            "rbfib_launch_count": ([], U64),
            "rbfib_tuned_blocks": ([P, ctypes.POINTER(ctypes.c_int32)], I32),
            "rbfib_krylov_stats": ([P, ctypes.POINTER(I64), ctypes.POINTER(I64)], I32),
            "rbfib_step_mode": ([P, ctypes.POINTER(I32)], I32),
            "rbfib_create_batch": ([I32, ctypes.POINTER(GridDesc), I32, ctypes.POINTER(P)], I32),
            "rbfib_destroy_batch": ([P], None),
            "rbfib_batch_grid": ([P, I32], P),
            "rbfib_batch_set_one_graph": ([P, I32], I32),
            "rbfib_batch_graph_steps": ([P], I64),
            "rbfib_batch_sem_step": ([P, ctypes.POINTER(SemParams), ctypes.POINTER(U64), U64, ctypes.POINTER(U32),
                                      ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(StepInfo),
                                      ctypes.POINTER(ctypes.c_int32)], I32),
            "rbfib_kernel_timer": ([P, I32], I32),
            "rbfib_kernel_timer_read": ([P, ctypes.POINTER(D), ctypes.POINTER(I64), ctypes.POINTER(D), ctypes.POINTER(D)], I32),
            "rbfib_kernel_timer_overhead": ([P, I32, ctypes.POINTER(D)], I32),
            "rbfib_body_block_info": ([P, ctypes.POINTER(I32), ctypes.POINTER(I64)], I32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


TIMER_OFF, TIMER_MATVEC, TIMER_SMOOTH, TIMER_DOT, TIMER_AXPY = 0, 1, 2, 3, 4


def launch_count():
    return int(lib().rbfib_launch_count())


def exported_symbols():
    return [n for n in dir(lib()) if n.startswith("rbfib_")]


class RbfibError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rbfib status {code}: {msg}")
        self.code = code


def _ptr(t, dtype=torch.float64, numel=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t.data_ptr()


def sem_params(workload_potentials=None, dt=0.05, kT=1.0, delta=0.0, force_ext=None, slip=None, rfd=True):
    """SemParams from a potentials dict of the seeded workloads; rfd=False
    runs the step without its drift terms (naive Euler-Maruyama)."""
    p = SemParams()
    p.dt, p.kT, p.delta = dt, kT, delta
    pot = workload_potentials or {}
    p.gravity = pot.get("gravity", 0.0)
    p.blob_gravity = pot.get("blob_gravity", 0.0)
    p.no_rfd = 0 if rfd else 1
    if "pair_soft" in pot:
        p.pair_phi0, p.pair_b, p.pair_d = (pot["pair_soft"][k] for k in ("phi0", "b", "d"))
    if "wall_soft" in pot:
        p.wall_phi0, p.wall_b, p.wall_d = (pot["wall_soft"][k] for k in ("phi0", "b", "d"))
    if "blob_wall_soft" in pot:
        p.blob_wall_phi0, p.blob_wall_b, p.blob_wall_d = (pot["blob_wall_soft"][k] for k in ("phi0", "b", "d"))
    if "yukawa" in pot:
        p.yukawa_u0, p.yukawa_dh, p.yukawa_lambda = (pot["yukawa"][k] for k in ("u0", "d_h", "lambda_d"))
    if "substrate" in pot:
        p.substrate_u0, p.substrate_s = pot["substrate"]["u0"], pot["substrate"]["s_lattice"]
    p.force_ext = _ptr(force_ext, name="force_ext")
    p.slip = _ptr(slip, name="slip")
    return p


class Grid:
    """A MAC grid with its solver workspaces, bound to torch's current stream."""

    def __init__(self, n, h=1.0, eta=1.0, periodic=(False, False, False), wall_vel=None,
                 precision=FP64, restart=30, max_iter=2000, rtol=1e-8, kernel=3, free_slip=None):
        d = _desc(n, h, eta, periodic, wall_vel, precision, restart, max_iter, rtol, kernel, free_slip)
        self.desc = d
        self.n = tuple(int(v) for v in n)
        self.stream = torch.cuda.current_stream()
        handle = ctypes.c_void_p()
        st = lib().rbfib_create_grid(ctypes.byref(d), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(handle))
        if st != OK:
            raise RbfibError(st, "create_grid failed")
        self._h = handle
        self.n_bodies = 0
        self.n_blobs = 0

    def close(self):
        if getattr(self, "_h", None):
            lib().rbfib_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            raise RbfibError(st, lib().rbfib_last_error(self._h).decode())

    # ------------------------------------------------------------ bodies
    def set_bodies(self, blob_offsets, ref_blobs, q, quat):
        off = np.ascontiguousarray(np.asarray(blob_offsets, dtype=np.int32))
        nb = off.size - 1
        nbl = int(off[-1]) if nb > 0 else 0
        dev = torch.device("cuda")
        ref = torch.as_tensor(np.asarray(ref_blobs), dtype=torch.float64, device=dev).contiguous()
        q = torch.as_tensor(np.asarray(q) if not isinstance(q, torch.Tensor) else q, dtype=torch.float64, device=dev).contiguous()
        quat = torch.as_tensor(np.asarray(quat) if not isinstance(quat, torch.Tensor) else quat, dtype=torch.float64, device=dev).contiguous()
        torch.cuda.current_stream().synchronize()   # the library may copy on another stream
        self._check(lib().rbfib_set_bodies(
            self._h, nb, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            _ptr(ref, numel=3 * nbl, name="ref_blobs") if nbl else None,
            _ptr(q, numel=3 * nb, name="q") if nb else None,
            _ptr(quat, numel=4 * nb, name="quat") if nb else None))
        self.n_bodies, self.n_blobs = nb, nbl

    def layout(self):
        off = (ctypes.c_int64 * 7)()
        self._check(lib().rbfib_saddle_layout(self._h, off))
        return [int(v) for v in off]

    @property
    def n_total(self):
        return self.layout()[6]

    # ----------------------------------------------------------- operators
    def apply_saddle(self, x, y=None):
        dtype = {torch.float64: DTYPE_F64, torch.float32: DTYPE_F32}[x.dtype]
        n = self.n_total
        if y is None:
            y = torch.empty_like(x)
        self._check(lib().rbfib_apply_saddle(self._h, _ptr(x, x.dtype, n, "x"), _ptr(y, x.dtype, n, "y"), dtype))
        return y

    def apply_preconditioner(self, r, z=None):
        n = self.n_total
        if z is None:
            z = torch.empty_like(r)
        self._check(lib().rbfib_apply_preconditioner(self._h, _ptr(r, numel=n, name="r"), _ptr(z, numel=n, name="z")))
        return z

    def mobility_solve(self, FT, slip=None, fluid_rhs=None, return_x=False):
        U = torch.empty(6 * self.n_bodies, dtype=torch.float64, device="cuda")
        x = torch.empty(self.n_total, dtype=torch.float64, device="cuda") if return_x else None
        info = SolveInfo()
        lay = self.layout()
        self._check(lib().rbfib_mobility_solve(
            self._h, _ptr(FT, numel=6 * self.n_bodies, name="FT"), _ptr(slip, numel=3 * self.n_blobs, name="slip"),
            _ptr(fluid_rhs, numel=lay[3], name="fluid_rhs"), _ptr(U), _ptr(x), ctypes.byref(info)))
        return (U, info.as_dict(), x) if return_x else (U, info.as_dict())

    def set_blob_positions(self, r):
        self._check(lib().rbfib_set_blob_positions(self._h, _ptr(r, numel=3 * self.n_blobs, name="r")))

    def mobility_solve_adjoint(self, dL_dU, x_fwd):
        dr = torch.empty(3 * max(self.n_blobs, 1), dtype=torch.float64, device="cuda")
        ds = torch.empty(3 * max(self.n_blobs, 1), dtype=torch.float64, device="cuda")
        info = SolveInfo()
        self._check(lib().rbfib_mobility_solve_adjoint(
            self._h, _ptr(dL_dU, numel=6 * self.n_bodies, name="dL_dU"), _ptr(x_fwd, numel=self.n_total, name="x_fwd"),
            _ptr(dr), _ptr(ds), ctypes.byref(info)))
        return dr[:3 * self.n_blobs], ds[:3 * self.n_blobs], info.as_dict()

    def stokes_solve(self, f):
        lay = self.layout()
        v = torch.empty(lay[3], dtype=torch.float64, device="cuda")
        pi = torch.empty(lay[4] - lay[3], dtype=torch.float64, device="cuda")
        info = SolveInfo()
        self._check(lib().rbfib_stokes_solve(self._h, _ptr(f, numel=lay[3], name="f"), _ptr(v), _ptr(pi),
                                             ctypes.byref(info)))
        return v, pi, info.as_dict()

    def sem_step(self, params, seed, step, attempt, q, quat, raise_on_reject=False):
        info = StepInfo()
        st = lib().rbfib_sem_step(self._h, ctypes.byref(params), int(seed), int(step), int(attempt),
                                  _ptr(q, numel=3 * self.n_bodies, name="q"),
                                  _ptr(quat, numel=4 * self.n_bodies, name="quat"), ctypes.byref(info))
        if st == EREJECT and not raise_on_reject:
            return st, info.as_dict()
        self._check(st)
        return st, info.as_dict()

    # ------------------------------------------------------ building blocks
    def binning(self):
        lay = self.layout()
        nc = lay[4] - lay[3]
        perm = torch.empty(max(self.n_blobs, 1), dtype=torch.int32, device="cuda")
        off = torch.empty(nc + 1, dtype=torch.int32, device="cuda")
        self._check(lib().rbfib_binning(self._h, _ptr(perm, torch.int32), _ptr(off, torch.int32)))
        return perm[:self.n_blobs], off

    def blob_positions(self):
        r = torch.empty(3 * max(self.n_blobs, 1), dtype=torch.float64, device="cuda")
        self._check(lib().rbfib_blob_positions(self._h, _ptr(r)))
        return r[:3 * self.n_blobs]

    def philox_words(self, seed, step, attempt, purpose, n_blocks, first_block=0):
        """(n_blocks, 4) int64 tensor holding the raw uint64 words bit for bit."""
        out = torch.empty((max(n_blocks, 1), 4), dtype=torch.int64, device="cuda")
        self._check(lib().rbfib_philox_words(self._h, seed, step, attempt, purpose, first_block, n_blocks,
                                             _ptr(out, torch.int64)))
        return out[:n_blocks]

    def philox_normals(self, seed, step, attempt, purpose, count):
        out = torch.empty(max(count, 1), dtype=torch.float64, device="cuda")
        self._check(lib().rbfib_philox_normals(self._h, seed, step, attempt, purpose, count, _ptr(out)))
        return out[:count]

    def stochastic_forcing(self, kT, dt, seed, step, attempt=0):
        out = torch.empty(self.layout()[3], dtype=torch.float64, device="cuda")
        self._check(lib().rbfib_stochastic_forcing(self._h, kT, dt, seed, step, attempt, _ptr(out)))
        return out

    def spread(self, lam):
        out = torch.empty(self.layout()[3], dtype=torch.float64, device="cuda")
        self._check(lib().rbfib_spread(self._h, _ptr(lam, numel=3 * self.n_blobs, name="lambda"), _ptr(out)))
        return out

    def interpolate(self, v, with_walls=False):
        out = torch.empty(3 * max(self.n_blobs, 1), dtype=torch.float64, device="cuda")
        self._check(lib().rbfib_interpolate(self._h, _ptr(v, numel=self.layout()[3], name="v"), _ptr(out),
                                            int(bool(with_walls))))
        return out[:3 * self.n_blobs]

    def kernel_timer(self, which):
        self._check(lib().rbfib_kernel_timer(self._h, int(which)))

    def kernel_timer_read(self):
        """(total ms, launches, algorithmic bytes, algorithmic operations)"""
        ms, n, b, f = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        self._check(lib().rbfib_kernel_timer_read(self._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b),
                                                  ctypes.byref(f)))
        return ms.value, n.value, b.value, f.value

    def body_block_info(self):
        """(coupled all-blob body block in use, Newton-Schulz warm starts taken)"""
        dense, warm = ctypes.c_int32(), ctypes.c_int64()
        self._check(lib().rbfib_body_block_info(self._h, ctypes.byref(dense), ctypes.byref(warm)))
        return bool(dense.value), int(warm.value)

    def kernel_timer_overhead(self, reps=200):
        """Median event-bracket time (us) of an empty kernel timed the way the
        kernel timer times each launch."""
        us = ctypes.c_double()
        self._check(lib().rbfib_kernel_timer_overhead(self._h, int(reps), ctypes.byref(us)))
        return us.value

    def tuned_blocks(self):
        out = (ctypes.c_int32 * 4)()
        self._check(lib().rbfib_tuned_blocks(self._h, out))
        return list(out)

    def step_mode(self):
        """1 if the last SEM step ran as the device-driven step graph, else 0."""
        v = ctypes.c_int32()
        self._check(lib().rbfib_step_mode(self._h, ctypes.byref(v)))
        return v.value

    def krylov_stats(self):
        """(Arnoldi iterations, second Gram-Schmidt passes taken) since creation."""
        it, sp = ctypes.c_int64(), ctypes.c_int64()
        self._check(lib().rbfib_krylov_stats(self._h, ctypes.byref(it), ctypes.byref(sp)))
        return it.value, sp.value

    def body_forces(self, params):
        out = torch.empty(6 * max(self.n_bodies, 1), dtype=torch.float64, device="cuda")
        self._check(lib().rbfib_body_forces(self._h, ctypes.byref(params), _ptr(out)))
        return out[:6 * self.n_bodies]


class _BatchMember(Grid):
    """A grid owned by a Batch (not created or destroyed here)."""

    def __init__(self, handle, desc, n):
        self._h = handle
        self.desc = desc
        self.n = tuple(n)
        self.n_bodies = 0
        self.n_blobs = 0

    def close(self):
        self._h = None


def _desc(n, h=1.0, eta=1.0, periodic=(False, False, False), wall_vel=None, precision=FP64, restart=30,
          max_iter=2000, rtol=1e-8, kernel=3, free_slip=None):
    """The C descriptor; free_slip: six flags for the walls -x, +x, -y, +y,
    -z, +z (True = free-slip)."""
    d = GridDesc()
    for a in range(3):
        d.n[a] = int(n[a])
        d.periodic[a] = int(bool(periodic[a]))
    d.h, d.eta = float(h), float(eta)
    wv = np.zeros((6, 3)) if wall_vel is None else np.asarray(wall_vel, dtype=np.float64).reshape(6, 3)
    for w in range(6):
        for c in range(3):
            d.wall_vel[w][c] = float(wv[w, c])
    fs = [False] * 6 if free_slip is None else list(free_slip)
    if len(fs) != 6:
        raise ValueError("free_slip needs one flag per wall")
    for w in range(6):
        d.free_slip[w] = int(bool(fs[w]))
    d.kernel, d.precision, d.restart, d.max_iter, d.rtol = (int(kernel), int(precision), int(restart),
                                                            int(max_iter), float(rtol))
    return d


class Batch:
    """An ensemble of independent systems advanced together (C ABI
    rbfib_create_batch / rbfib_batch_sem_step).

    The workers' streams overlap on the GPU only as far as the CUDA runtime
    gives them separate hardware queues: CUDA_DEVICE_MAX_CONNECTIONS (8 unless
    set in the environment before the CUDA context is created; at most 32).
    one_graph: every system's step as a branch of one graph, launched once per
    batch step (rbfib_batch_set_one_graph)."""

    def __init__(self, workloads_, precision=None, workers=16, restart=30, max_iter=4000, one_graph=False):
        n = len(workloads_)
        descs = (GridDesc * n)()
        for i, w in enumerate(workloads_):
            prec = precision if precision is not None else (FP32_REFINED if w.precision == "f32-refined" else FP64)
            descs[i] = _desc(w.n, w.h, w.eta, w.periodic, w.wall_vel, prec, restart, max_iter, w.rtol,
                             getattr(w, "kernel", 3), getattr(w, "free_slip", None))
        h = ctypes.c_void_p()
        st = lib().rbfib_create_batch(n, descs, int(workers), ctypes.byref(h))
        if st != OK:
            raise RbfibError(st, "create_batch failed")
        self._h = h
        if one_graph:
            st = lib().rbfib_batch_set_one_graph(self._h, 1)
            if st != OK:
                raise RbfibError(st, "batch_set_one_graph failed")
        self.systems = []
        for i, w in enumerate(workloads_):
            m = _BatchMember(lib().rbfib_batch_grid(self._h, i), descs[i], w.n)
            m.set_bodies(w.blob_offsets, w.ref_blobs, w.q, w.quat)
            self.systems.append(m)
        self.n = n

    def sem_step(self, params, seeds, step, q, quat, attempts=None):
        n = self.n
        P = (SemParams * n)(*params)
        S = (ctypes.c_uint64 * n)(*[int(s) for s in seeds])
        A = (ctypes.c_uint32 * n)(*([0] * n if attempts is None else [int(a) for a in attempts]))
        Q = (ctypes.c_void_p * n)(*[_ptr(t, numel=3 * m.n_bodies, name="q") for t, m in zip(q, self.systems)])
        QT = (ctypes.c_void_p * n)(*[_ptr(t, numel=4 * m.n_bodies, name="quat") for t, m in zip(quat, self.systems)])
        infos = (StepInfo * n)()
        status = (ctypes.c_int32 * n)()
        torch.cuda.current_stream().synchronize()   # inputs are read on the worker streams
        st = lib().rbfib_batch_sem_step(self._h, P, S, int(step), A, Q, QT, infos, status)
        if st != OK:
            raise RbfibError(st, "batch_sem_step failed")
        return list(status), [i.as_dict() for i in infos]

    def graph_steps(self):
        """Batch steps run as one graph launch (the one-graph form)."""
        return int(lib().rbfib_batch_graph_steps(self._h))

    def close(self):
        if getattr(self, "_h", None):
            for m in self.systems:
                m._h = None
            lib().rbfib_destroy_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def grid_for(workload, precision=None, restart=48, max_iter=4000, rtol=None):
    """A Grid with the workload's bodies set."""
    prec = precision if precision is not None else (FP32_REFINED if workload.precision == "f32-refined" else FP64)
    g = Grid(workload.n, h=workload.h, eta=workload.eta, periodic=workload.periodic, wall_vel=workload.wall_vel,
             precision=prec, restart=restart, max_iter=max_iter, rtol=workload.rtol if rtol is None else rtol,
             kernel=getattr(workload, "kernel", 3), free_slip=getattr(workload, "free_slip", None))
    g.set_bodies(workload.blob_offsets, workload.ref_blobs, workload.q, workload.quat)
    return g
