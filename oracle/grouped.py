"""Submatrices shared by groups of block columns (Section IV-C, "Generating
Submatrices From Multiple Block Columns").

Test infrastructure only, like the rest of ``oracle/``.  A group G of block
columns shares one submatrix over the union of their row sets,
N(G) = U_{j in G} N(j) (ascending, Section IV-A1 order): a_G = K[N(G), N(G)]
- mu I, S_G = sign(a_G) by the symmetric eigendecomposition (Eq.
eigendecompsym, signum(0) = 0), and for every member j the columns of block j
of (I - S_G) / 2 go into block column j of D, on K's pattern (rows N(j) only).
A group of one column is Section III-A's submatrix; one group holding every
column evaluates the dense sign of the whole K on the pattern.
"""
from __future__ import annotations

import numpy as np

from .submatrix import _block_lookup, column_structure, sign_by_eigh


def group_rows(m, members, structure=None):
    """N(G): the sorted union of the members' row sets."""
    if structure is None:
        structure = column_structure(m)
    return np.unique(np.concatenate([structure[int(j)] for j in members]))


def density_matrix_grouped(m, mu, groups, only=None):
    """D in K's block pattern with one submatrix per group; ``groups[j]`` is
    the group of block column j.  ``only`` restricts the evaluation to some
    groups (the block columns of the others are NaN)."""
    groups = np.asarray(groups)
    structure = column_structure(m)
    lookup = _block_lookup(m)
    bs = m.block_sizes
    out = np.full(m.vals.shape, np.nan)
    for g in (np.unique(groups) if only is None else np.asarray(only)):
        members = np.flatnonzero(groups == g)
        rows = group_rows(m, members, structure)
        loc = np.zeros(len(rows) + 1, dtype=np.int64)
        np.cumsum(bs[rows], out=loc[1:])
        n = int(loc[-1])
        a = np.zeros((n, n))
        for u, r in enumerate(rows):
            for v, c in enumerate(rows):
                hit = lookup.get((int(r), int(c)))
                if hit is None:
                    continue
                off, nr, nc, _p = hit
                a[loc[u]:loc[u + 1], loc[v]:loc[v + 1]] = m.vals[off:off + nr * nc].reshape(nr, nc)
        a -= mu * np.eye(n)
        s, _lam, _q = sign_by_eigh(a)
        half = 0.5 * (np.eye(n) - s)
        pos = {int(r): u for u, r in enumerate(rows)}
        for j in members:
            k = pos[int(j)]
            for i in structure[int(j)]:
                u = pos[int(i)]
                off, nr, nc, _p = lookup[(int(i), int(j))]
                out[off:off + nr * nc] = half[loc[u]:loc[u + 1], loc[k]:loc[k + 1]].reshape(-1)
    return out
