"""Blob shells for spherical rigid bodies (Sec. V.A: spheres of 12, 42 or 162
approximately equally spaced blobs).

The 12-blob shell is the regular icosahedron; the 42-blob shell adds the 30
normalised edge midpoints; the 162-blob shell splits every triangle of the
42-blob geodesic shell once more.  With vertices (0, +-1, +-g) and their cyclic
permutations (g the golden ratio) the shell has the pyritohedral symmetry
group T_h, which maps the cube onto itself.
"""
import numpy as np


def _icosahedron_vertices():
    g = (1.0 + np.sqrt(5.0)) / 2.0
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v.append((0.0, s1, s2 * g))
            v.append((s1, s2 * g, 0.0))
            v.append((s2 * g, 0.0, s1))
    v = np.array(v, dtype=np.float64)
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def icosahedral_shell(n_blobs, radius):
    """Return an (n_blobs, 3) float64 array of blob offsets from the centre."""
    verts = _icosahedron_vertices()
    if n_blobs == 12:
        pts = verts
    elif n_blobs == 42:
        # edges of the icosahedron join vertices at the minimal distance
        d = np.linalg.norm(verts[:, None, :] - verts[None, :, :], axis=2)
        emin = np.min(d[d > 1e-12])
        mids = []
        for i in range(12):
            for j in range(i + 1, 12):
                if abs(d[i, j] - emin) < 1e-9:
                    m = verts[i] + verts[j]
                    mids.append(m / np.linalg.norm(m))
        assert len(mids) == 30
        pts = np.vstack([verts, np.array(mids)])
    elif n_blobs == 162:
        pts = _geodesic(verts, 2)
    else:
        raise ValueError("only 12-, 42- and 162-blob shells are provided")
    return np.ascontiguousarray(pts * float(radius))


def _icosahedron_faces(verts):
    """The 20 triangles of the icosahedron: vertex triples at the minimal
    pairwise distance."""
    d = np.linalg.norm(verts[:, None, :] - verts[None, :, :], axis=2)
    emin = np.min(d[d > 1e-12])
    adj = np.abs(d - emin) < 1e-9
    faces = [(i, j, k) for i in range(12) for j in range(i + 1, 12) for k in range(j + 1, 12)
             if adj[i, j] and adj[j, k] and adj[i, k]]
    assert len(faces) == 20
    return faces


def _geodesic(verts, levels):
    """Vertices of the icosahedron with each triangle split into four
    (edge midpoints pushed to the unit sphere) ``levels`` times: 12, 42, 162."""
    pts = [tuple(v) for v in verts]
    index = {p: i for i, p in enumerate(pts)}
    faces = _icosahedron_faces(verts)

    def mid(a, b):
        m = np.array(pts[a]) + np.array(pts[b])
        m = tuple(m / np.linalg.norm(m))
        key = tuple(np.round(m, 12))
        if key not in index:
            index[key] = len(pts)
            pts.append(m)
        return index[key]
    for _ in range(levels):
        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(pts)


def shell_12(radius=1.0):
    return icosahedral_shell(12, radius)


def shell_42(radius=2.5):
    return icosahedral_shell(42, radius)
