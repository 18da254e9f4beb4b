"""Water-like synthetic block-sparse matrices (seeded, deterministic per seed).

A system of ``N`` molecules sits in a periodic box.  Each molecule owns one
block of ``b`` basis functions, so the matrix has ``N x N`` blocks of size
``b x b``.  The recipe follows the shapes of the paper's workloads (liquid
water in an SZV basis, Section V), which are not available here:

* positions: a simple-cubic lattice of ``ceil(N^(1/3))`` sites per axis that
  fills the box at the liquid density of water (0.03343 molecules per cubic
  Angstrom, i.e. 1 g/cm^3), ``N`` sites taken by a seeded permutation, each
  jittered by U[-0.2, 0.2] lattice spacings per axis;
* pattern: block (i, j), i != j, is stored iff the minimum-image distance
  between the molecule centres is below the cutoff ``r_c`` (a distance cutoff
  stands in for the paper's epsilon_filter truncation, Section II-A);
* values: each stored off-diagonal block has entries N(0, 1) * 0.05 *
  exp(-r / 2 Angstrom) and its mirror block is the transpose, so the matrix
  is symmetric; each diagonal block is Q diag(occupied, virtual) Q^T with a
  Haar-random orthogonal Q and eigenvalues drawn uniformly from the occupied
  (negative) and virtual (positive) intervals.

Molecules are numbered in lattice order, so neighbouring indices are close
in space and the pattern is banded, as Section IV-B2 recommends.

Nothing here evaluates the matrix sign function or assembles submatrices.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

#: Liquid water at 1 g/cm^3, molecules per cubic Angstrom.
RHO_WATER = 0.03343


@dataclass
class BSRMatrix:
    """Symmetric block-sparse matrix in block-CSR form.

    Block ``p`` (CSR order) sits at block row ``r`` (``row_ptr[r] <= p <
    row_ptr[r+1]``), block column ``col_idx[p]``; its ``bs[r] * bs[col]``
    values are stored row-major at ``vals[val_ptr[p]:val_ptr[p+1]]``.
    Column indices are strictly increasing inside a row and every diagonal
    block is stored.
    """

    block_sizes: np.ndarray  # int32 [nblk]
    row_ptr: np.ndarray  # int64 [nblk + 1]
    col_idx: np.ndarray  # int32 [nnzb]
    vals: np.ndarray  # float64 [sum of block areas]
    coords: np.ndarray | None = None  # float64 [nblk, 3], Angstrom
    box: np.ndarray | None = None  # float64 [3], Angstrom
    mu: float = 0.0
    n_el: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def nblk(self) -> int:
        return int(self.block_sizes.shape[0])

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def n(self) -> int:
        return int(self.block_sizes.sum())

    @property
    def val_ptr(self) -> np.ndarray:
        rows = np.repeat(np.arange(self.nblk), np.diff(self.row_ptr))
        area = self.block_sizes[rows].astype(np.int64) * self.block_sizes[self.col_idx]
        out = np.zeros(self.nnzb + 1, dtype=np.int64)
        np.cumsum(area, out=out[1:])
        return out

    def with_vals(self, vals: np.ndarray) -> "BSRMatrix":
        """Same pattern and metadata, other values (e.g. a result D)."""
        return BSRMatrix(self.block_sizes, self.row_ptr, self.col_idx,
                         np.ascontiguousarray(vals, dtype=np.float64),
                         self.coords, self.box, self.mu, self.n_el, dict(self.meta))


def _lattice_positions(rng, n, lengths, jitter=0.2):
    """``n`` jittered sites of a simple lattice filling a box (origin 0).

    Sites are returned in lattice (x-major, then y, then z) order.
    """
    lengths = np.asarray(lengths, dtype=np.float64)
    vol_per = float(np.prod(lengths)) / n
    h = vol_per ** (1.0 / 3.0)
    m = np.maximum(1, np.ceil(lengths / h - 1e-9)).astype(np.int64)
    while int(np.prod(m)) < n:  # guard rounding: enlarge the shortest count
        m[np.argmin(m * h / lengths)] += 1
    spacing = lengths / m
    total = int(np.prod(m))
    chosen = np.sort(rng.permutation(total)[:n])
    ix = chosen // (m[1] * m[2])
    iy = (chosen // m[2]) % m[1]
    iz = chosen % m[2]
    base = (np.stack([ix, iy, iz], axis=1) + 0.5) * spacing
    jit = rng.uniform(-jitter, jitter, size=(n, 3)) * spacing
    return np.mod(base + jit, lengths)


def _pairs_within(coords, box, r_c):
    """All (i < j) with minimum-image distance < r_c, sorted; and distances."""
    n = coords.shape[0]
    ii, jj, rr = [], [], []
    chunk = max(1, int(4_000_000 // max(n, 1)))
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        d = coords[None, :, :] - coords[s:e, None, :]
        d -= box * np.round(d / box)
        r = np.sqrt(np.einsum("abk,abk->ab", d, d))
        a, bb = np.nonzero(r < r_c)
        a = a + s
        keep = bb > a
        ii.append(a[keep])
        jj.append(bb[keep])
        rr.append(r[a[keep] - s, bb[keep]])
    i = np.concatenate(ii).astype(np.int64)
    j = np.concatenate(jj).astype(np.int64)
    r = np.concatenate(rr)
    order = np.lexsort((j, i))
    return i[order], j[order], r[order]


def _haar_orthogonal(rng, count, b):
    g = rng.standard_normal((count, b, b))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diagonal(r, axis1=1, axis2=2))
    d[d == 0] = 1.0
    return q * d[:, None, :]


def assemble_bsr(coords, box, block, r_c, occ, virt, rng, coupling=0.05,
                 decay=2.0):
    """Draw the pattern and values for molecules at ``coords``.

    ``occ`` / ``virt`` are ``(count, lo, hi)``: how many eigenvalues of each
    diagonal block are drawn from U[lo, hi]; ``count_occ + count_virt`` must
    equal the block size ``block``.
    """
    n = coords.shape[0]
    n_occ, o_lo, o_hi = occ
    n_vir, v_lo, v_hi = virt
    if n_occ + n_vir != block:
        raise ValueError("occupied + virtual counts must equal the block size")
    # diagonal blocks
    q = _haar_orthogonal(rng, n, block)
    ev = np.concatenate([rng.uniform(o_lo, o_hi, size=(n, n_occ)),
                         rng.uniform(v_lo, v_hi, size=(n, n_vir))], axis=1)
    diag = np.einsum("nik,nk,njk->nij", q, ev, q)
    diag = 0.5 * (diag + np.transpose(diag, (0, 2, 1)))
    # off-diagonal blocks
    pi, pj, pr = _pairs_within(coords, box, r_c)
    off = rng.standard_normal((pi.shape[0], block, block))
    off *= (coupling * np.exp(-pr / decay))[:, None, None]
    # CSR over both triangles plus the diagonal
    rows = np.concatenate([np.arange(n), pi, pj])
    cols = np.concatenate([np.arange(n), pj, pi])
    src = np.concatenate([np.arange(n), n + np.arange(pi.shape[0]),
                          n + pi.shape[0] + np.arange(pi.shape[0])])
    order = np.lexsort((cols, rows))
    rows, cols, src = rows[order], cols[order], src[order]
    allblocks = np.concatenate([diag, off, np.transpose(off, (0, 2, 1))], axis=0)
    vals = np.ascontiguousarray(allblocks[src]).reshape(-1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    return BSRMatrix(
        block_sizes=np.full(n, block, dtype=np.int32),
        row_ptr=row_ptr,
        col_idx=cols.astype(np.int32),
        vals=vals,
        coords=coords,
        box=np.asarray(box, dtype=np.float64),
        n_el=float(n_occ * n),
        meta={"r_c": float(r_c), "block": int(block), "occ": occ, "virt": virt,
              "n_pairs": int(pi.shape[0])},
    )


def make_water(n_mol, block, r_c, occ, virt, seed, density=RHO_WATER, mu=0.0):
    """A periodic cube of ``n_mol`` molecules at ``density`` (molecules/A^3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    length = (n_mol / density) ** (1.0 / 3.0)
    box = np.array([length] * 3)
    coords = _lattice_positions(rng, n_mol, box)
    m = assemble_bsr(coords, box, block, r_c, occ, virt, rng)
    m.mu = float(mu)
    m.meta.update({"geometry": "cube", "seed": int(seed), "density": density})
    return m


def make_slab(seed, block=6, n_liquid=3840, n_vapour=256, lxy=40.0,
              vapour_density=0.2 * RHO_WATER, layer_density=1.0, r_c=None,
              occ=(3, -1.0, -0.3), virt=(3, 0.3, 1.0), mu=0.0):
    """Liquid layer plus vapour in a periodic box (a slab geometry).

    The liquid holds ``n_liquid`` molecules at ``layer_density`` times the
    density of water; the vapour region above it holds ``n_vapour`` at
    ``vapour_density``.  ``r_c`` defaults to a draw from U[7, 10] Angstrom.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if r_c is None:
        r_c = float(rng.uniform(7.0, 10.0))
    rho_l = RHO_WATER * layer_density
    t_liq = n_liquid / rho_l / (lxy * lxy)
    t_vap = n_vapour / vapour_density / (lxy * lxy)
    box = np.array([lxy, lxy, t_liq + t_vap])
    liq = _lattice_positions(rng, n_liquid, np.array([lxy, lxy, t_liq]))
    vap = _lattice_positions(rng, n_vapour, np.array([lxy, lxy, t_vap]))
    vap[:, 2] += t_liq
    coords = np.concatenate([liq, vap], axis=0)
    m = assemble_bsr(coords, box, block, r_c, occ, virt, rng)
    m.mu = float(mu)
    m.meta.update({"geometry": "slab", "seed": int(seed), "t_liquid": t_liq,
                   "t_vapour": t_vap, "layer_density": layer_density})
    return m


#: The five workloads: (description, builder keyword arguments).
CONFIGS = {
    0: dict(kind="cube", n_mol=32, block=6, r_c=6.0, occ=(3, -1.0, -0.3),
            virt=(3, 0.3, 1.0)),
    1: dict(kind="cube", n_mol=1024, block=23, r_c=8.0, occ=(4, -1.0, -0.3),
            virt=(19, 0.3, 1.5)),
    2: dict(kind="slab", block=6),
    3: dict(kind="cube", n_mol=2048, block=23, r_c=8.0, occ=(4, -1.0, -0.3),
            virt=(19, 0.3, 1.5)),
    4: dict(kind="cube", n_mol=20736, block=6, r_c=9.0, occ=(3, -1.0, -0.15),
            virt=(3, 0.15, 1.0)),
}


def make_config(i: int, seed: int | None = None, run: int | None = None,
                **overrides) -> BSRMatrix:
    """Workload ``i`` (0..4).  Seed defaults to ``1000 + i``; the slab
    workload (2) takes ``run`` instead, seeded ``2000 + run``."""
    spec = dict(CONFIGS[i])
    spec.update(overrides)
    kind = spec.pop("kind")
    if seed is None:
        seed = 2000 + run if (i == 2 and run is not None) else 1000 + i
    if kind == "slab":
        m = make_slab(seed, **spec)
    else:
        m = make_water(spec.pop("n_mol"), spec.pop("block"), spec.pop("r_c"),
                       spec.pop("occ"), spec.pop("virt"), seed, **spec)
    m.meta["config"] = i
    return m


def small_case(n_mol=24, block=4, r_c=5.0, seed=7, occ=None, virt=None,
               density=RHO_WATER, mu=0.0):
    """A small cube for unit tests (defaults: 24 molecules of 4 functions)."""
    if occ is None:
        occ = (block // 2, -1.0, -0.3)
    if virt is None:
        virt = (block - occ[0], 0.3, 1.0)
    return make_water(n_mol, block, r_c, occ, virt, seed, density=density, mu=mu)


def random_symmetric_bsr(block_sizes, density, seed, scale=1.0):
    """Random symmetric BSR with uneven block sizes (pattern tests only).

    Each off-diagonal block pair is stored with probability ``density``;
    values are N(0, scale^2) with the mirror block transposed.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    bs = np.asarray(block_sizes, dtype=np.int32)
    n = bs.shape[0]
    iu, ju = np.triu_indices(n, 1)
    keep = rng.uniform(size=iu.shape[0]) < density
    iu, ju = iu[keep], ju[keep]
    entries = {}
    for i in range(n):
        a = rng.standard_normal((bs[i], bs[i])) * scale
        entries[(i, i)] = 0.5 * (a + a.T)
    for i, j in zip(iu.tolist(), ju.tolist()):
        a = rng.standard_normal((bs[i], bs[j])) * scale
        entries[(i, j)] = a
        entries[(j, i)] = a.T.copy()
    keys = sorted(entries)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    for (r, _c) in keys:
        row_ptr[r + 1] += 1
    np.cumsum(row_ptr, out=row_ptr)
    col_idx = np.array([c for (_r, c) in keys], dtype=np.int32)
    vals = np.concatenate([entries[k].reshape(-1) for k in keys])
    return BSRMatrix(bs, row_ptr, col_idx, vals,
                     meta={"kind": "random", "seed": int(seed)})


def bsr_to_dense(m: BSRMatrix) -> np.ndarray:
    """Dense copy of a BSR matrix (for small test cases)."""
    off = np.zeros(m.nblk + 1, dtype=np.int64)
    np.cumsum(m.block_sizes, out=off[1:])
    out = np.zeros((m.n, m.n))
    vp = m.val_ptr
    for r in range(m.nblk):
        for p in range(m.row_ptr[r], m.row_ptr[r + 1]):
            c = m.col_idx[p]
            blk = m.vals[vp[p]:vp[p + 1]].reshape(m.block_sizes[r], m.block_sizes[c])
            out[off[r]:off[r + 1], off[c]:off[c + 1]] = blk
    return out


def summary(m: BSRMatrix) -> dict:
    """Pattern statistics (neighbour counts are the submatrix block counts)."""
    deg = np.diff(m.row_ptr)
    return {
        "nblk": m.nblk, "n": m.n, "nnzb": m.nnzb,
        "neighbours_min": int(deg.min()), "neighbours_mean": float(deg.mean()),
        "neighbours_max": int(deg.max()),
    }


__all__ = ["BSRMatrix", "CONFIGS", "make_config", "make_water", "make_slab",
           "small_case", "random_symmetric_bsr", "bsr_to_dense", "summary",
           "RHO_WATER"]


def _selfcheck():  # pragma: no cover - manual use
    for i in range(5):
        m = make_config(i)
        print(i, summary(m), math.fsum([0.0]))
