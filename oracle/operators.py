"""Discrete fluid operators of Sec. III.A, assembled as sparse matrices.

  D   : faces -> cells, (Dv)_c = sum_a (v_a(right face) - v_a(left face)) / h
  G   : cells -> faces, defined as G = -D^T (the adjoint relation of Sec. III.A)
  DD  : stress -> faces, the tensor divergence with the boundary conditions
        built in: across a no-slip wall edge the stress enters with weight
        sqrt(2), across a free-slip wall edge with weight 0 (no shear stress)
  LL  : faces -> faces, the vector Laplacian LL = DD GG with GG = -DD^T
        (Sec. III.A), so LL = -DD DD^T

With sqrt(2) wall-edge weights, LL is the ghost-reflection Laplacian: a face
next to a wall along a tangential axis has the row (u_1 - 3 u_0 + 2 u_w)/h^2,
whose affine part 2 u_w / h^2 is returned by ``wall_velocity_rhs``; next to
a free-slip wall the row is (u_1 - u_0)/h^2 (ghost u_{-1} = u_0, zero normal
derivative of the tangential velocity).
"""
import numpy as np
import scipy.sparse as sp

from .grid import Grid

SQRT2 = np.sqrt(2.0)


def divergence(g: Grid):
    """D as a (N_c, N_f) CSR matrix."""
    ci, cj, ck = g.grid_indices(g.n)
    rows, cols, vals = [], [], []
    cell = g.flat(g.n, ci, cj, ck)
    for a in range(3):
        ext = g.face_ext(a)
        idx = [ci, cj, ck]
        for p_off, sgn in ((1, 1.0), (0, -1.0)):          # right face p = c_a + 1, left p = c_a
            p = idx[a] + p_off
            if g.periodic[a]:
                comp = np.mod(p, g.n[a])
                ok = np.ones_like(p, dtype=bool)
            else:
                ok = (p >= 1) & (p <= g.n[a] - 1)        # boundary faces carry zero normal velocity
                comp = p - 1
            fi = [ci, cj, ck]
            fi = [comp if ax == a else fi[ax] for ax in range(3)]
            fidx = g.face_offset(a) + g.flat(ext, *fi)
            rows.append(cell[ok]); cols.append(fidx[ok]); vals.append(np.full(ok.sum(), sgn / g.h))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(g.N_c, g.N_f))


def gradient(g: Grid):
    """G = -D^T, (N_f, N_c)."""
    return (-divergence(g).T).tocsr()


def stress_offsets(g: Grid):
    offs, o = {}, 0
    for a, b in g.stress_blocks():
        offs[(a, b)] = o
        o += int(np.prod(g.stress_ext(a, b)))
    return offs


def tensor_divergence(g: Grid):
    """DD as a (N_f, N_w) CSR matrix acting on the nine independent stress
    components (global block order of Grid.stress_blocks)."""
    offs = stress_offsets(g)
    rows, cols, vals = [], [], []
    for a in range(3):
        ext = g.face_ext(a)
        fi, fj, fk = g.grid_indices(ext)
        fidx = g.face_offset(a) + g.flat(ext, fi, fj, fk)
        comp = [fi, fj, fk]
        # d/dx_a of W_aa: cells either side of the face
        p = g.face_phys(a, comp[a])
        for cidx_a, sgn in ((p, 1.0), (p - 1, -1.0)):
            cc = np.mod(cidx_a, g.n[a]) if g.periodic[a] else cidx_a
            ci = [cc if ax == a else comp[ax] for ax in range(3)]
            rows.append(fidx); cols.append(offs[(a, a)] + g.flat(g.n, *ci))
            vals.append(np.full(fidx.size, sgn / g.h))
        # d/dx_b of W_ab on the edges below (node j) and above (node j+1)
        for b in range(3):
            if b == a:
                continue
            sext = g.stress_ext(a, b)
            j = comp[b]
            for node, sgn in ((j + 1, 1.0), (j, -1.0)):
                if g.periodic[b]:
                    nd = np.mod(node, g.n[b])
                    c = np.ones(node.size)
                else:
                    nd = node
                    c_lo = 0.0 if g.free_slip[2 * b] else SQRT2
                    c_hi = 0.0 if g.free_slip[2 * b + 1] else SQRT2
                    c = np.where(node == 0, c_lo, np.where(node == g.n[b], c_hi, 1.0))
                si = [nd if ax == b else comp[ax] for ax in range(3)]
                rows.append(fidx); cols.append(offs[(a, b)] + g.flat(sext, *si))
                vals.append(sgn * c / g.h)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(g.N_f, g.N_w))


def vector_laplacian(g: Grid):
    """LL = DD GG = -DD DD^T (Sec. III.A)."""
    DD = tensor_divergence(g)
    return (-(DD @ DD.T)).tocsr()


def wall_velocity_rhs(g: Grid, eta):
    """Affine part of -eta LL v for moving walls, moved to the right-hand side:
    +eta * 2 u_w / h^2 on every face adjacent (along a tangential axis b) to a
    wall moving with velocity u_w (component a of the wall velocity)."""
    out = np.zeros(g.N_f)
    for a in range(3):
        ext = g.face_ext(a)
        fi, fj, fk = g.grid_indices(ext)
        comp = [fi, fj, fk]
        base = g.face_offset(a) + g.flat(ext, fi, fj, fk)
        for b in range(3):
            if b == a or g.periodic[b]:
                continue
            lo = comp[b] == 0
            hi = comp[b] == g.n[b] - 1
            out[base[lo]] += eta * 2.0 * g.wall_vel[2 * b, a] / g.h ** 2
            out[base[hi]] += eta * 2.0 * g.wall_vel[2 * b + 1, a] / g.h ** 2
    return out
