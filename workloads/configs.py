"""The benchmark workloads as seeded synthetic inputs.

Each workload mirrors a physical setup of the paper (Sec. V.A two spheres in a
cavity, Sec. V.B driven monolayer, App. A geometry) at the sizes used by the
benchmark.  All lengths are in units of the grid spacing h = 1; kT = 1 and
eta = 1 where the workload says so.  Positions, orientations and slip
coefficients come from numpy's Philox generator seeded with
WORKLOAD_SEED_BASE + workload index.
"""
from dataclasses import dataclass, field
import numpy as np

from .shells import icosahedral_shell

WORKLOAD_SEED_BASE = 0x1901064270000


@dataclass
class Body:
    ref_blobs: np.ndarray          # (n_blobs, 3) offsets in the body frame
    q: np.ndarray                  # (3,) tracking point
    quat: np.ndarray               # (4,) unit quaternion (w, x, y, z)


@dataclass
class Workload:
    name: str
    n: tuple                       # cells per axis
    h: float = 1.0
    periodic: tuple = (False, False, False)
    wall_vel: np.ndarray = field(default_factory=lambda: np.zeros((6, 3)))
    eta: float = 1.0
    kT: float = 1.0
    dt: float = 0.05
    steps: int = 1
    rtol: float = 1e-8
    precision: str = "f64"
    bodies: list = field(default_factory=list)
    force_torque: np.ndarray = None    # (N_b, 6) fixed external force/torque
    slip: np.ndarray = None            # (N_bl, 3) active slip
    potentials: dict = field(default_factory=dict)
    seed: int = 0
    kernel: int = 3                    # immersed-boundary kernel width (3 or 6 points per axis)
    free_slip: tuple = (False,) * 6    # walls -x, +x, -y, +y, -z, +z: True = free-slip

    # flat views used by both implementations -------------------------
    @property
    def n_bodies(self):
        return len(self.bodies)

    @property
    def blob_offsets(self):
        off = [0]
        for b in self.bodies:
            off.append(off[-1] + b.ref_blobs.shape[0])
        return np.array(off, dtype=np.int32)

    @property
    def ref_blobs(self):
        if not self.bodies:
            return np.zeros((0, 3))
        return np.ascontiguousarray(np.vstack([b.ref_blobs for b in self.bodies]))

    @property
    def q(self):
        if not self.bodies:
            return np.zeros((0, 3))
        return np.ascontiguousarray(np.array([b.q for b in self.bodies], dtype=np.float64))

    @property
    def quat(self):
        if not self.bodies:
            return np.zeros((0, 4))
        return np.ascontiguousarray(np.array([b.quat for b in self.bodies], dtype=np.float64))

    @property
    def n_blobs(self):
        return int(self.blob_offsets[-1])


def _rng(index):
    return np.random.Generator(np.random.Philox(WORKLOAD_SEED_BASE + index))


def random_unit_quaternions(rng, count):
    v = rng.standard_normal((count, 4))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    v[v[:, 0] < 0] *= -1.0
    return v


def single_sphere_box():
    """Deterministic mobility problem: one 42-blob shell of radius 2.5h at the
    centre of a 32^3 box with no-slip walls on all faces; unit force along x
    and unit torque along z; relative residual 1e-10."""
    shell = icosahedral_shell(42, 2.5)
    w = Workload(name="single-sphere-32c", n=(32, 32, 32), rtol=1e-10, seed=WORKLOAD_SEED_BASE)
    w.bodies = [Body(shell, np.array([16.0, 16.0, 16.0]), np.array([1.0, 0.0, 0.0, 0.0]))]
    w.force_torque = np.array([[1.0, 0.0, 0.0, 0.0, 0.0, 1.0]])
    return w


def two_sphere_cavity(steps=2000, kernel=3, free_slip=None):
    """Two 42-blob spheres (R = 2.5h) 6h apart along x in a 48x48x32 no-slip
    cuboid; kT = 1, eta = 1, dt = 0.05; gravity plus soft wall and pair
    repulsion of the form of Eq. (Usoft); orientations seeded.  kernel = 6:
    the same setup with the paper's six-point kernel; free_slip: the same box
    with the flagged walls (-x, +x, -y, +y, -z, +z) free-slip."""
    rng = _rng(1)
    shell = icosahedral_shell(42, 2.5)
    quats = random_unit_quaternions(rng, 2)
    fs = (False,) * 6 if free_slip is None else tuple(bool(v) for v in free_slip)
    name = "two-sphere-48x48x32" + ("" if kernel == 3 else "-6pt")
    if any(fs):
        name += "-free-slip-" + "".join(wn for wn, f in zip(("-x", "+x", "-y", "+y", "-z", "+z"), fs) if f)
    w = Workload(name=name, n=(48, 48, 32), dt=0.05,
                 steps=steps, rtol=1e-8, seed=WORKLOAD_SEED_BASE + 1, kernel=kernel, free_slip=fs)
    w.bodies = [Body(shell, np.array([21.0, 24.0, 16.0]), quats[0]),
                Body(shell, np.array([27.0, 24.0, 16.0]), quats[1])]
    R = 2.5
    w.potentials = {
        "gravity": 1.0,                                       # body force -g z (kT/h)
        "pair_soft": {"phi0": 4.0, "b": 0.1 * R, "d": 2.0 * R},
        "wall_soft": {"phi0": 4.0, "b": 0.1 * R, "d": R},
    }
    return w


def driven_monolayer(wall_speed=0.5, steps=500, cols=64, rows=16, nz=12, z=6.0):
    """1024 12-blob spheres (R = 1h) on a jittered lattice (64 columns x 16
    rows, spacing 6h, odd rows shifted 3h, z = 6h) in a 384x96x12 channel
    periodic in x; no-slip side and bottom walls, top wall moving at
    (wall_speed, 0, 0); Yukawa pair repulsion, per-blob soft wall repulsion and
    a commensurate substrate potential of amplitude 4kT; dt = 0.02.  Smaller
    monolayers of the same shape: cols x rows spheres in a
    (6 cols) x (6 rows) x nz channel at height z."""
    rng = _rng(2)
    shell = icosahedral_shell(12, 1.0)
    full = (cols, rows, nz) == (64, 16, 12)
    name = "monolayer-384x96x12" if full else f"monolayer-{6 * cols}x{6 * rows}x{nz}"
    w = Workload(name=name, n=(6 * cols, 6 * rows, nz), periodic=(True, False, False),
                 dt=0.02, steps=steps, rtol=1e-8, precision="f32-refined",
                 seed=WORKLOAD_SEED_BASE + 2)
    w.wall_vel = np.zeros((6, 3))
    w.wall_vel[5, 0] = wall_speed          # +z wall moves along x
    quats = random_unit_quaternions(rng, cols * rows)
    bodies = []
    for r in range(rows):
        for c in range(cols):
            x = 6.0 * c + (3.0 if r % 2 else 0.0) + 1.5
            y = 6.0 * r + 3.0
            jit = rng.uniform(-0.1, 0.1, size=3)
            bodies.append(Body(shell, np.array([x, y, z]) + jit, quats[len(bodies)]))
    w.bodies = bodies
    s_lat = 6.0
    w.potentials = {
        "yukawa": {"u0": 20.0, "d_h": 2.0, "lambda_d": (0.16 / 5.7) * s_lat},
        "blob_wall_soft": {"phi0": 4.0, "b": 0.1, "d": 1.0},
        "substrate": {"u0": 4.0, "s_lattice": s_lat},
    }
    return w


def _place_spheres(rng, n_sys, count, R, min_gap, wall_gap, max_tries=20000):
    L = np.asarray(n_sys, dtype=np.float64)
    centres = []
    tries = 0
    while len(centres) < count and tries < max_tries:
        tries += 1
        c = rng.uniform(wall_gap, L - wall_gap)
        if all(np.linalg.norm(c - o) >= min_gap for o in centres):
            centres.append(c)
    return np.array(centres).reshape(-1, 3)


def batched_ensemble(n_systems=256):
    """Independent cuboids with cubic grids n ~ U{16, 20, ..., 48} and 1..16
    12-blob spheres each (R = 1h), centre distance >= 2R + 2h and wall
    distance >= R + 1.5h; kT = 1, dt = 0.02."""
    rng = _rng(3)
    shell = icosahedral_shell(12, 1.0)
    systems = []
    for s in range(n_systems):
        n = int(rng.choice(np.arange(16, 49, 4)))
        count = int(rng.integers(1, 17))
        centres = _place_spheres(rng, (n, n, n), count, 1.0, 4.0, 2.5)
        quats = random_unit_quaternions(rng, centres.shape[0])
        w = Workload(name=f"ensemble-{s}", n=(n, n, n), dt=0.02, rtol=1e-8,
                     precision="f32-refined", seed=WORKLOAD_SEED_BASE + 3)
        w.bodies = [Body(shell, centres[i], quats[i]) for i in range(centres.shape[0])]
        w.potentials = {"wall_soft": {"phi0": 4.0, "b": 0.1, "d": 1.0},
                        "pair_soft": {"phi0": 4.0, "b": 0.1, "d": 2.0}}
        systems.append(w)
    return systems


def adjoint_suspension():
    """64 42-blob spheres (R = 2.5h) at seeded non-overlapping positions in a
    128x128x64 no-slip box with seeded active slip (per-blob N(0, 0.1^2),
    per-body mean removed so the slip integrates to zero)."""
    rng = _rng(4)
    shell = icosahedral_shell(42, 2.5)
    centres = _place_spheres(rng, (128, 128, 64), 64, 2.5, 7.0, 4.0)
    quats = random_unit_quaternions(rng, centres.shape[0])
    w = Workload(name="adjoint-128x128x64", n=(128, 128, 64), rtol=1e-8,
                 precision="f32-refined", seed=WORKLOAD_SEED_BASE + 4)
    w.bodies = [Body(shell, centres[i], quats[i]) for i in range(centres.shape[0])]
    slip = rng.normal(0.0, 0.1, size=(w.n_blobs, 3))
    off = w.blob_offsets
    for p in range(w.n_bodies):
        slip[off[p]:off[p + 1]] -= slip[off[p]:off[p + 1]].mean(axis=0)
    w.slip = slip
    w.force_torque = np.zeros((w.n_bodies, 6))
    return w


def small_case(n=(12, 10, 8), periodic=(False, False, False), n_bodies=2, blobs=12,
               radius=1.0, seed=7, wall_speed=0.0, near_wall=False, kernel=3, free_slip=None):
    """A small seeded problem for parity tests: a few shells placed at random
    (optionally hugging a wall) in a box of the given size; free_slip marks
    free-slip walls (which do not move)."""
    rng = np.random.Generator(np.random.Philox(WORKLOAD_SEED_BASE + 100 + seed))
    shell = icosahedral_shell(blobs, radius)
    L = np.asarray(n, dtype=np.float64)
    centres = []
    for _ in range(n_bodies):
        for _try in range(1000):
            lo = np.where(periodic, 0.0, radius + (0.3 if near_wall else 1.5))
            hi = np.where(periodic, L, L - radius - (0.3 if near_wall else 1.5))
            c = rng.uniform(lo, hi)
            if all(np.linalg.norm(c - o) >= 2 * radius + 1.0 for o in centres):
                centres.append(c)
                break
    quats = random_unit_quaternions(rng, len(centres))
    w = Workload(name=f"small-{n[0]}x{n[1]}x{n[2]}", n=tuple(n), periodic=tuple(periodic),
                 seed=WORKLOAD_SEED_BASE + 100 + seed, rtol=1e-10, kernel=kernel,
                 free_slip=tuple(bool(v) for v in free_slip) if free_slip is not None else (False,) * 6)
    w.bodies = [Body(shell, centres[i], quats[i]) for i in range(len(centres))]
    if wall_speed:
        w.wall_vel = np.zeros((6, 3))
        for ax in range(3):
            if not periodic[ax]:
                t = (ax + 1) % 3
                if not w.free_slip[2 * ax + 1]:
                    w.wall_vel[2 * ax + 1, t] = wall_speed
                if not w.free_slip[2 * ax]:
                    w.wall_vel[2 * ax, (ax + 2) % 3] = -0.5 * wall_speed
    w.force_torque = rng.standard_normal((len(centres), 6))
    w.slip = 0.1 * rng.standard_normal((w.n_blobs, 3))
    w.potentials = {"gravity": 1.0,
                    "pair_soft": {"phi0": 4.0, "b": 0.1 * radius, "d": 2.0 * radius},
                    "wall_soft": {"phi0": 4.0, "b": 0.1 * radius, "d": radius}}
    return w


def matvec_box(n=256, n_bodies=64):
    """A large no-slip box (n^3 cells, vectors well beyond the 129 MB L2) with
    42-blob spheres (R = 2.5h) at seeded non-overlapping positions: the
    saddle matvec at HBM-bound size."""
    rng = _rng(5)
    shell = icosahedral_shell(42, 2.5)
    centres = _place_spheres(rng, (n, n, n), n_bodies, 2.5, 7.0, 4.0)
    quats = random_unit_quaternions(rng, centres.shape[0])
    w = Workload(name=f"matvec-box-{n}c", n=(n, n, n), rtol=1e-8, seed=WORKLOAD_SEED_BASE + 5)
    w.bodies = [Body(shell, centres[i], quats[i]) for i in range(centres.shape[0])]
    return w


# The six-point kernel's blob hydrodynamic radius in grid units (Sec. V.A).
BLOB_RADIUS_6PT = 1.47


def two_sphere_msd(blobs=12):
    """The tight cavity of Sec. V.A: two neutrally buoyant spheres of
    hydrodynamic radius R_h = 0.656 um in a 3.478 x 1.739 x 1.739 um no-slip
    box, discretised with the six-point kernel at h = 0.0543 (4, 2, 1) um for
    12-, 42- and 162-blob spheres: 16 x 8 x 8, 32 x 16 x 16 or 64 x 32 x 32
    cells, R_h = 3.02h, 6.04h or 12.08h.  The geometric radius is R_h - a, a = 1.47h the blob radius (our
    reading; the paper takes it from a table of the cited multiblob work).
    Soft pair (d = 2 R_h) and wall (d = R_h) repulsion of Eq. (Usoft) with
    b = 0.1 R_h, Phi0 = 4 kT; kT = eta = 1; dt from the dimensionless step
    dtau = kT dt / (6 pi eta R_h^3) = 0.0044.  The spheres start side by side
    along x at mid-height (equilibrium starts come from Gibbs-Boltzmann
    samples)."""
    scale = {12: 1, 42: 2, 162: 4}[blobs]
    n = (16 * scale, 8 * scale, 8 * scale)
    Rh = 0.656 / (0.0543 * 4 / scale)
    Rg = Rh - BLOB_RADIUS_6PT
    shell = icosahedral_shell(blobs, Rg)
    w = Workload(name=f"two-sphere-msd-{blobs}blob-{n[0]}x{n[1]}x{n[2]}", n=n, kernel=6, rtol=1e-8,
                 seed=WORKLOAD_SEED_BASE + 20 + blobs)
    w.dt = 0.0044 * 6.0 * np.pi * Rh ** 3
    L = np.asarray(n, dtype=np.float64)
    w.bodies = [Body(shell, np.array([L[0] / 4, L[1] / 2, L[2] / 2]), np.array([1.0, 0, 0, 0])),
                Body(shell, np.array([3 * L[0] / 4, L[1] / 2, L[2] / 2]), np.array([1.0, 0, 0, 0]))]
    w.potentials = {"pair_soft": {"phi0": 4.0, "b": 0.1 * Rh, "d": 2.0 * Rh},
                    "wall_soft": {"phi0": 4.0, "b": 0.1 * Rh, "d": Rh}}
    w.hydrodynamic_radius = Rh
    return w


def boomerang_slit(dtau=0.14, n=(64, 64, 16)):
    """The confined boomerang of App. A: an L of 15 blobs (the cross point
    and two arms of 7 blobs, spacing s = 0.3 um = 0.925 a, so the six-point
    kernel's a = 1.47h gives h = 0.2208 um and s = 1.359h) in a 64h x 64h x 16h
    slit (n: a smaller slit for parity tests), periodic in x and y, no-slip
    walls in z; blob-wall repulsion of
    Eq. (Usoft) with d = a, b = 0.1 a, Phi0 = 4 kT; the buoyant weight
    m_e g = 1.57e-11 mg x 9.81 m/s^2 of every blob, 0.00819 kT/h at 300 K;
    kT = eta = 1 and dt from dtau = kT dt / (6 pi eta a^3).  The tracking
    point is the cross point; the body starts flat at mid-height."""
    a = BLOB_RADIUS_6PT
    s = 0.925 * a
    arm = [np.array([k * s, 0.0, 0.0]) for k in range(1, 8)] + [np.array([0.0, k * s, 0.0]) for k in range(1, 8)]
    ref = np.vstack([np.zeros((1, 3))] + [x[None, :] for x in arm])
    w = Workload(name=f"boomerang-slit-{n[0]}x{n[1]}x{n[2]}-dtau{dtau:g}", n=tuple(n), periodic=(True, True, False),
                 kernel=6, rtol=1e-8, seed=WORKLOAD_SEED_BASE + 30)
    w.dt = dtau * 6.0 * np.pi * a ** 3
    w.bodies = [Body(ref, np.array([n[0] / 2 - 2.0, n[1] / 2 - 2.0, n[2] / 2]), np.array([1.0, 0, 0, 0]))]
    kT_300K = 1.380649e-23 * 300.0
    weight = 1.57e-17 * 9.81 * 0.2208e-6 / kT_300K          # kT per h, per blob
    w.potentials = {"blob_wall_soft": {"phi0": 4.0, "b": 0.1 * a, "d": a}, "blob_gravity": weight}
    return w
