"""Blob-to-cell binning: the cell key of a blob and a stable counting sort
(no counterpart in the paper; the CUDA library uses it to order spreading).

Cell index along axis a: floor(x_a / h) with IEEE division, clamped to
[0, n_a - 1] on wall axes and taken modulo n_a on periodic axes; the key is the
flat cell index (x fastest).  The sort is stable in blob id.
"""
import numpy as np


def cell_keys(g, r):
    r = np.asarray(r, dtype=np.float64).reshape(-1, 3)
    idx = []
    for a in range(3):
        c = np.floor(r[:, a] / g.h).astype(np.int64)
        c = np.mod(c, g.n[a]) if g.periodic[a] else np.clip(c, 0, g.n[a] - 1)
        idx.append(c)
    return idx[0] + g.n[0] * (idx[1] + g.n[1] * idx[2])


def counting_sort(g, r):
    """(perm, offsets): blobs of cell c are perm[offsets[c]:offsets[c+1]] in
    increasing blob id."""
    keys = cell_keys(g, r)
    counts = np.zeros(g.N_c + 1, dtype=np.int64)
    for k in keys:
        counts[k + 1] += 1
    offsets = np.cumsum(counts)
    fill = offsets[:-1].copy()
    perm = np.zeros(keys.size, dtype=np.int64)
    for i, k in enumerate(keys):
        perm[fill[k]] = i
        fill[k] += 1
    return perm, offsets
