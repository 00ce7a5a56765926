"""Staggered MAC grid of Sec. III.A (velocities on faces, pressure at cell
centres, cell volume dV = h^3).

Layout (also the layout of the CUDA library's saddle vector):
  * cells (i, j, k), 0 <= i < n_x, flat index i + n_x (j + n_y k);
  * velocity component a lives on a-faces.  Along its own axis a the unknown
    faces are the physical faces p = 1 .. n_a - 1 on a wall axis (the two
    boundary faces carry the prescribed normal velocity, zero for tangentially
    moving walls) and p = 0 .. n_a - 1 on a periodic axis; the compact index is
    p - 1 (wall) or p (periodic).  Along the other two axes the face sits at a
    cell centre.  Flat index is x-fastest over the component's own extents.
  * the stochastic stress has nine independent components: W_aa at cell
    centres and, for b != a, W_ab on the edges at the a-face positions (along a),
    the nodes 0..n_b (wall) or 0..n_b-1 (periodic) along b, and cell centres
    along the third axis.

Walls (Introduction: any combination of periodic, no-slip and free-slip
boundaries along the axes).  Each wall of a bounded axis is no-slip (the
velocity equals the wall's, which may move tangentially) or free-slip (zero
normal velocity and zero tangential stress; it cannot drive the fluid, so its
velocity must be zero).
"""
import numpy as np


class Grid:
    def __init__(self, n, h=1.0, periodic=(False, False, False), wall_vel=None, kernel=3, free_slip=None):
        """kernel: points per axis of the immersed-boundary kernel (3: the
        three-point Peskin kernel; 6: the six-point kernel of Sec. III.B).
        free_slip: six flags for the walls -x, +x, -y, +y, -z, +z (True =
        free-slip, False = no-slip; ignored on periodic axes)."""
        self.n = tuple(int(v) for v in n)
        if kernel not in (3, 6):
            raise ValueError("kernel must be 3 or 6")
        self.kernel = int(kernel)
        self.h = float(h)
        self.periodic = tuple(bool(p) for p in periodic)
        if all(self.periodic):
            raise ValueError("at least one axis must be bounded by walls")
        wv = np.zeros((6, 3)) if wall_vel is None else np.array(wall_vel, dtype=np.float64).reshape(6, 3)
        for ax in range(3):
            if wv[2 * ax, ax] != 0.0 or wv[2 * ax + 1, ax] != 0.0:
                raise ValueError("walls move tangentially only")
        self.wall_vel = wv
        fs = [False] * 6 if free_slip is None else [bool(v) for v in free_slip]
        if len(fs) != 6:
            raise ValueError("free_slip needs one flag per wall")
        self.free_slip = tuple(fs[w] and not self.periodic[w // 2] for w in range(6))
        for w in range(6):
            if self.free_slip[w] and np.any(wv[w] != 0.0):
                raise ValueError("a free-slip wall cannot move")
        for a in range(3):
            if self.velocity_null_mode(a):
                raise ValueError(f"velocity component {a} has a constant null mode (no no-slip wall acts on it)")

    def velocity_null_mode(self, a):
        """True when a constant v_a satisfies every boundary condition, i.e.
        axis a is periodic and every other axis is periodic or free-slip at
        both walls; the viscous operator of v_a is then singular."""
        if not self.periodic[a]:
            return False
        return all(self.periodic[b] or (self.free_slip[2 * b] and self.free_slip[2 * b + 1])
                   for b in range(3) if b != a)

    # sizes -------------------------------------------------------------
    @property
    def dV(self):
        return self.h ** 3

    @property
    def N_c(self):
        return self.n[0] * self.n[1] * self.n[2]

    def face_ext(self, a):
        e = list(self.n)
        if not self.periodic[a]:
            e[a] = self.n[a] - 1
        return tuple(e)

    def n_face(self, a):
        e = self.face_ext(a)
        return e[0] * e[1] * e[2]

    @property
    def N_f(self):
        return sum(self.n_face(a) for a in range(3))

    def face_offset(self, a):
        return sum(self.n_face(b) for b in range(a))

    def node_count(self, b):
        return self.n[b] if self.periodic[b] else self.n[b] + 1

    def stress_ext(self, a, b):
        """Extents (x, y, z) of the stress block W_ab."""
        if a == b:
            return tuple(self.n)
        e = list(self.n)
        e[a] = self.face_ext(a)[a]
        e[b] = self.node_count(b)
        return tuple(e)

    def stress_blocks(self):
        """Global order of the nine stress blocks: for a = x, y, z: W_aa, then
        W_ab for the other two axes b in increasing order."""
        out = []
        for a in range(3):
            out.append((a, a))
            for b in range(3):
                if b != a:
                    out.append((a, b))
        return out

    @property
    def N_w(self):
        return sum(int(np.prod(self.stress_ext(a, b))) for a, b in self.stress_blocks())

    # index helpers (vectorised) ------------------------------------------
    @staticmethod
    def flat(ext, i, j, k):
        return i + ext[0] * (j + ext[1] * k)

    @staticmethod
    def grid_indices(ext):
        """Integer arrays (i, j, k) enumerating ext x-fastest."""
        k, j, i = np.meshgrid(np.arange(ext[2]), np.arange(ext[1]), np.arange(ext[0]), indexing="ij")
        return i.ravel(), j.ravel(), k.ravel()

    def face_phys(self, a, compact):
        """Physical face index along axis a of a compact a-face index."""
        return compact if self.periodic[a] else compact + 1

    def face_coords(self, a):
        ext = self.face_ext(a)
        idx = list(self.grid_indices(ext))
        x = []
        for ax in range(3):
            if ax == a:
                x.append(self.face_phys(a, idx[ax]) * self.h)
            else:
                x.append((idx[ax] + 0.5) * self.h)
        return np.stack(x, axis=1)

    def cell_coords(self):
        i, j, k = self.grid_indices(self.n)
        return np.stack([(i + 0.5) * self.h, (j + 0.5) * self.h, (k + 0.5) * self.h], axis=1)

    def length(self):
        return np.array(self.n, dtype=np.float64) * self.h
