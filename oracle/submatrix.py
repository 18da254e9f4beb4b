"""Submatrix method for D = 1/2 (I - sign(K - mu I)), FP64 on host cores.

Test infrastructure only (see the package docstring).  Every function names
the passage of the paper it follows.  Readings of the paper used here:

* K is already orthogonalised, so S = I in Eq. DsignSym:
  D = 1/2 (I - sign(K - mu I)).
* The submatrix for block column j is built block-wise and structurally:
  block row i takes part iff block (i, j) is stored (Section IV-C, blocks of
  DBCSR), in ascending block order (Section IV-A1).
* signum(0) = 0 (Eq. signevext): an eigenvalue exactly at mu contributes 1/2.
* D keeps K's block pattern and is not symmetrised (Section III-A, step 3).
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np


# ---------------------------------------------------------------------------
# Pattern (Section III-A step 1; Section IV-A1)
# ---------------------------------------------------------------------------

def column_structure(m):
    """For every block column j: the block rows i whose block (i, j) is stored.

    Section III-A step 1 removes every row j with A_{j,i} = 0; applied per
    block column this keeps exactly the stored blocks of column j.  The scan
    goes over all block rows (the transpose of the CSR index), so it does not
    assume the pattern is symmetric.  Returns a list of ascending int arrays.
    """
    cols = [[] for _ in range(m.nblk)]
    for r in range(m.nblk):
        for p in range(int(m.row_ptr[r]), int(m.row_ptr[r + 1])):
            cols[int(m.col_idx[p])].append(r)
    return [np.array(sorted(c), dtype=np.int64) for c in cols]


def _block_lookup(m):
    """(row, col) -> (offset, rows, cols) of the stored block values."""
    vp = m.val_ptr
    table = {}
    for r in range(m.nblk):
        for p in range(int(m.row_ptr[r]), int(m.row_ptr[r + 1])):
            c = int(m.col_idx[p])
            table[(r, c)] = (int(vp[p]), int(m.block_sizes[r]), int(m.block_sizes[c]), p)
    return table


def assemble_submatrix(m, j, mu, rows=None, lookup=None):
    """Dense a_j = K[N(j), N(j)] - mu I (Section III-A step 1).

    Returns (a_j, rows, local offsets of each block in a_j, k) where ``k`` is
    the position of block j inside ``rows`` (step 3 names it).
    """
    if rows is None:
        rows = column_structure(m)[j]
    if lookup is None:
        lookup = _block_lookup(m)
    bs = m.block_sizes
    loc = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(bs[rows], out=loc[1:])
    n = int(loc[-1])
    a = np.zeros((n, n))
    for u, r in enumerate(rows):
        for v, c in enumerate(rows):
            hit = lookup.get((int(r), int(c)))
            if hit is None:
                continue  # absent block: structural zero
            off, nr, nc, _p = hit
            a[loc[u]:loc[u + 1], loc[v]:loc[v + 1]] = m.vals[off:off + nr * nc].reshape(nr, nc)
    a -= mu * np.eye(n)
    k = int(np.searchsorted(rows, j))
    assert rows[k] == j, "the diagonal block must be stored"
    return a, rows, loc, k


# ---------------------------------------------------------------------------
# Sign by symmetric eigendecomposition (Eq. eigendecompsym, Eq. signevext)
# ---------------------------------------------------------------------------

def signum(x):
    """signum with signum(0) = 0 (Eq. signevext); exact comparison with 0."""
    x = np.asarray(x, dtype=np.float64)
    return np.where(x > 0, 1.0, np.where(x < 0, -1.0, 0.0))


def sign_by_eigh(a):
    """sign(a) = Q signum(Lambda) Q^T for symmetric ``a`` (Eq. eigendecompsym).

    LAPACK's symmetric divide-and-conquer solver (``syevd``, as in Section
    IV-F) through ``numpy.linalg.eigh``.  Returns (sign, eigenvalues, Q).
    """
    lam, q = np.linalg.eigh(a)
    s = (q * signum(lam)[None, :]) @ q.T
    return s, lam, q


def submatrix_sign(m, j, mu, rows=None, lookup=None):
    """sign(a_j) for block column j, with the data needed to extract."""
    a, rows, loc, k = assemble_submatrix(m, j, mu, rows, lookup)
    s, lam, q = sign_by_eigh(a)
    return s, rows, loc, k, lam, q


def density_block_column(m, j, mu, rows=None, lookup=None):
    """Block column j of D (Section III-A step 3 with Eq. DsignSym, S = I).

    Column block k of 1/2 (I - sign(a_j)) is copied into block column j of D,
    one block per row of N(j).  Returns ``{(i, j): block values}``.
    """
    if lookup is None:
        lookup = _block_lookup(m)
    s, rows, loc, k, _lam, _q = submatrix_sign(m, j, mu, rows, lookup)
    n = s.shape[0]
    half = 0.5 * (np.eye(n) - s)
    c0, c1 = loc[k], loc[k + 1]
    out = {}
    for u, r in enumerate(rows):
        out[(int(r), int(j))] = half[loc[u]:loc[u + 1], c0:c1].copy()
    return out


def _worker_columns(args):
    m, mu, js = args
    structure = column_structure(m)
    lookup = _block_lookup(m)
    res = {}
    for j in js:
        res.update(density_block_column(m, int(j), mu, structure[int(j)], lookup))
    return res


def _pool(workers):
    """Process pool started with 'spawn', one BLAS thread per worker
    (the paper runs one thread per MPI rank, Section V)."""
    import multiprocessing as mp
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")
    return ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))


def density_matrix(m, mu=None, columns=None, workers=1):
    """D in K's block pattern (values array laid out like ``m.vals``).

    ``columns`` restricts the evaluation to some block columns (the other
    entries are NaN); ``workers > 1`` spreads block columns over a process
    pool.
    """
    if mu is None:
        mu = m.mu
    js = np.arange(m.nblk) if columns is None else np.asarray(columns)
    if workers > 1 and len(js) > 1:
        chunks = [js[w::workers] for w in range(workers)]
        res = {}
        with _pool(workers) as ex:
            for part in ex.map(_worker_columns, [(m, mu, c) for c in chunks if len(c)]):
                res.update(part)
    else:
        res = _worker_columns((m, mu, js))
    lookup = _block_lookup(m)
    out = np.full(m.vals.shape, np.nan)
    for (r, c), blk in res.items():
        off, nr, nc, _p = lookup[(r, c)]
        out[off:off + nr * nc] = blk.reshape(-1)
    return out


def trace_bsr(m, vals):
    """Tr of a BSR matrix in K's pattern: sum of diagonal-block diagonals in
    ascending (block, entry) order, FP64 with exact summation (math.fsum)."""
    lookup = _block_lookup(m)
    terms = []
    for j in range(m.nblk):
        off, nr, nc, _p = lookup[(j, j)]
        blk = np.asarray(vals[off:off + nr * nc]).reshape(nr, nc)
        terms.extend(np.diagonal(blk).tolist())
    return math.fsum(terms)


def dense_sign(a):
    """sign of a dense symmetric matrix by eigendecomposition (full-cover
    checks compare the method with this)."""
    return sign_by_eigh(a)[0]


# ---------------------------------------------------------------------------
# Canonical adaptation: Algorithm 1 (Section IV-G)
# ---------------------------------------------------------------------------

def decompose_all(m, mu=None):
    """Per submatrix: eigenvalues of a_j and the rows of Q that belong to
    block j (the only rows Algorithm 1 needs, Section IV-G last paragraph)."""
    if mu is None:
        mu = m.mu
    structure = column_structure(m)
    lookup = _block_lookup(m)
    out = []
    for j in range(m.nblk):
        a, rows, loc, k = assemble_submatrix(m, j, mu, structure[j], lookup)
        lam, q = np.linalg.eigh(a)
        out.append((lam, q[loc[k]:loc[k + 1], :].copy()))
    return out


def n_elec_alg1(decomps, mu_corr):
    """n_elec for a shift mu_corr of the chemical potential (Algorithm 1):
    sum over submatrices and over the columns k of block j of
    1/2 - 1/2 sum_l Q_kl^2 signum(lambda_l - mu_corr)."""
    total = []
    for lam, qrows in decomps:
        sl = signum(lam - mu_corr)
        w = (qrows * qrows) @ sl
        total.extend((0.5 - 0.5 * w).tolist())
    return math.fsum(total)


def mu_search_alg1(decomps, n_el, lo, hi, tol=1e-12, max_steps=200):
    """Bisection on mu_corr (Algorithm 1's update rule is left open by the
    paper; bisection is the rule Section IV-G names).  n_elec is a
    non-decreasing staircase in mu_corr.

    Returns (mu_corr, n_elec at mu_corr, steps, bracket).
    """
    n_lo = n_elec_alg1(decomps, lo)
    n_hi = n_elec_alg1(decomps, hi)
    if not (n_lo <= n_el <= n_hi):
        raise ValueError("bracket does not contain the electron count")
    steps = 0
    while hi - lo > tol and steps < max_steps:
        mid = 0.5 * (lo + hi)
        n_mid = n_elec_alg1(decomps, mid)
        steps += 1
        if n_mid == n_el:
            return mid, n_mid, steps, (lo, hi)
        if n_mid < n_el:
            lo = mid
        else:
            hi = mid
    mid = 0.5 * (lo + hi)
    return mid, n_elec_alg1(decomps, mid), steps, (lo, hi)


# ---------------------------------------------------------------------------
# Derivatives: band energy E = Tr(D K) (Eq. bandenergy)
# ---------------------------------------------------------------------------

def frechet_sign(lam, q, e):
    """Frechet derivative of sign at a = Q diag(lam) Q^T in direction e,
    in the eigenbasis (Daleckii-Krein): Q (Phi o (Q^T e Q)) Q^T with
    Phi_lm = (s_l - s_m) / (lam_l - lam_m) for lam_l != lam_m, else 0
    (signum is flat away from 0)."""
    s = signum(lam)
    dl = lam[:, None] - lam[None, :]
    ds = s[:, None] - s[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        phi = np.where(dl != 0, ds / dl, 0.0)
    return q @ (phi * (q.T @ e @ q)) @ q.T


def band_energy(m, d_vals):
    """E = Tr(D K) over K's block pattern (Eq. bandenergy, band part)."""
    lookup = _block_lookup(m)
    terms = []
    for (r, c), (off, nr, nc, _p) in lookup.items():
        d = np.asarray(d_vals[off:off + nr * nc]).reshape(nr, nc)
        koff, knr, knc, _ = lookup[(c, r)]
        k = m.vals[koff:koff + knr * knc].reshape(knr, knc)
        terms.append(float(np.sum(d * k.T)))
    return math.fsum(terms)


def sign_backward(m, dbar_vals, mu=None, columns=None):
    """Vector-Jacobian product of the submatrix density map K -> D.

    For upstream gradient Dbar (K's pattern), block column j contributes
    abar_j = -1/2 L_sign(a_j, G_j), where G_j is zero except its column block
    k, which holds Dbar's block column j; abar_j is then added into every
    stored block of K that a_j was assembled from.  Returns (Kbar values,
    dN/dmu) with dN/dmu = 1/2 sum_j sum_{c in block j} L_sign(a_j, I)_cc.
    """
    if mu is None:
        mu = m.mu
    structure = column_structure(m)
    lookup = _block_lookup(m)
    kbar = np.zeros(m.vals.shape)
    dndmu = []
    js = range(m.nblk) if columns is None else columns
    for j in js:
        a, rows, loc, k = assemble_submatrix(m, j, mu, structure[j], lookup)
        lam, q = np.linalg.eigh(a)
        n = a.shape[0]
        g = np.zeros((n, n))
        for u, r in enumerate(rows):
            off, nr, nc, _p = lookup[(int(r), int(j))]
            g[loc[u]:loc[u + 1], loc[k]:loc[k + 1]] = dbar_vals[off:off + nr * nc].reshape(nr, nc)
        abar = -0.5 * frechet_sign(lam, q, g)
        for u, r in enumerate(rows):
            for v, c in enumerate(rows):
                hit = lookup.get((int(r), int(c)))
                if hit is None:
                    continue
                off, nr, nc, _p = hit
                kbar[off:off + nr * nc] += abar[loc[u]:loc[u + 1], loc[v]:loc[v + 1]].reshape(-1)
        li = frechet_sign(lam, q, np.eye(n))
        dndmu.extend((0.5 * np.diagonal(li)[loc[k]:loc[k + 1]]).tolist())
    return kbar, math.fsum(dndmu)


def band_energy_grad(m, mu=None):
    """dE/dK for E = Tr(D K) with D from the submatrix method.

    Explicit part: dE/dK_(r,c) = D_(c,r)^T on the pattern; implicit part:
    ``sign_backward`` with Dbar_(r,c) = K_(c,r)^T (K symmetric, so K_(r,c)).
    Entries of a symmetric K are treated as independent: a finite difference
    that moves K_pq and K_qp together compares with Kbar_pq + Kbar_qp.
    """
    if mu is None:
        mu = m.mu
    d = density_matrix(m, mu)
    lookup = _block_lookup(m)
    explicit = np.zeros(m.vals.shape)
    dbar = np.zeros(m.vals.shape)
    for (r, c), (off, nr, nc, _p) in lookup.items():
        toff, tnr, tnc, _ = lookup[(c, r)]
        explicit[off:off + nr * nc] = d[toff:toff + tnr * tnc].reshape(tnr, tnc).T.reshape(-1)
        dbar[off:off + nr * nc] = m.vals[toff:toff + tnr * tnc].reshape(tnr, tnc).T.reshape(-1)
    implicit, _ = sign_backward(m, dbar, mu)
    return explicit + implicit
