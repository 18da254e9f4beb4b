"""Combining block columns into shared submatrices (Section IV-C, "Generating
Submatrices From Multiple Block Columns").

A group G of block columns can share one submatrix over the union of their
neighbourhoods, N(G) = U_{j in G} N(j); its dimension is n_G = sum of the
block sizes in N(G), and it yields the block columns of every j in G.  The
paper's heuristic assumes the cost of a submatrix grows like n^3 and scores a
grouping by the estimated additional speedup (Eq. estimatedspeedup)

    S = sum_j n_j^3 / sum_G n_G^3

(single block columns in the numerator), and proposes to find groups by
k-means on the real-space positions of the block columns.  Here k-means runs
on the periodic box with minimum-image distances (the paper's runs ignored the
periodicity).  ``estimated_speedup`` also accepts a per-dimension cost
function, so the score can use measured times per n^3 instead of n^3 alone
(the tensor cores run small submatrices at a lower fraction of their peak).

Host-side planning on the pattern and coordinates only (NumPy / SciPy); it
computes nothing of the matrix function.
"""
from __future__ import annotations

import numpy as np


def neighbourhoods(row_ptr, col_idx):
    """N(j) for every block column j: the block rows of the stored blocks of
    column j (the pattern is symmetric, so row j's columns)."""
    row_ptr = np.asarray(row_ptr)
    col_idx = np.asarray(col_idx)
    return [col_idx[row_ptr[j]:row_ptr[j + 1]] for j in range(len(row_ptr) - 1)]


def group_dims(block_sizes, row_ptr, col_idx, labels):
    """n_G for every group: the dimension of the submatrix over the union of
    the group's neighbourhoods.  ``labels[j]`` is the group of block column j.
    Returns (dims, groups) with groups[g] the block columns of group g."""
    bs = np.asarray(block_sizes, dtype=np.int64)
    labels = np.asarray(labels)
    nbh = neighbourhoods(row_ptr, col_idx)
    groups = [np.flatnonzero(labels == g) for g in range(int(labels.max()) + 1)]
    groups = [g for g in groups if len(g)]
    dims = np.array([int(bs[np.unique(np.concatenate([nbh[j] for j in g]))].sum()) for g in groups],
                    dtype=np.int64)
    return dims, groups


def estimated_speedup(single_dims, group_dims_, cost=None):
    """Eq. estimatedspeedup: sum_j cost(n_j) / sum_G cost(n_G), with
    cost(n) = n^3 by default."""
    f = (lambda n: np.asarray(n, dtype=np.float64) ** 3) if cost is None else cost
    return float(np.sum(f(single_dims)) / np.sum(f(group_dims_)))


def periodic_kmeans(coords, box, k, seed=0, iters=30):
    """Lloyd's k-means on the periodic box: points go to the nearest centre
    by minimum-image distance; a centre moves to the circular mean of its
    points (per axis, the angle of the mean of exp(2 pi i x / L)).  Starts from
    k distinct points drawn with the seeded generator.  Returns labels in
    0..k-1 (every label used)."""
    from scipy.spatial import cKDTree
    coords = np.mod(np.asarray(coords, dtype=np.float64), box)
    box = np.asarray(box, dtype=np.float64)
    rng = np.random.default_rng(seed)
    centres = coords[rng.choice(len(coords), size=k, replace=False)].copy()
    labels = np.zeros(len(coords), dtype=np.int64)
    for it in range(iters):
        tree = cKDTree(np.mod(centres, box), boxsize=box)
        _d, new = tree.query(coords)
        if it > 0 and np.array_equal(new, labels):
            break
        labels = new
        ang = 2.0 * np.pi * coords / box
        for d in range(3):
            cs = np.bincount(labels, weights=np.cos(ang[:, d]), minlength=k)
            sn = np.bincount(labels, weights=np.sin(ang[:, d]), minlength=k)
            used = (cs != 0) | (sn != 0)
            centres[used, d] = np.mod(np.arctan2(sn[used], cs[used]) * box[d] / (2.0 * np.pi), box[d])
    # drop empty clusters, relabel 0..k'-1
    _u, labels = np.unique(labels, return_inverse=True)
    return labels


def consecutive_groups(nblk, size):
    """Groups of `size` consecutive block columns (the grouping the plan's
    column order already makes spatially compact)."""
    return np.arange(nblk) // size
