"""Finite temperature: the Fermi function in place of signum.

Test infrastructure only, like the rest of ``oracle/``.  Section IV-F (its last
paragraph) notes that the eigendecomposition route to the submatrix result
extends to finite electronic temperature by replacing signum with the Fermi
function, and the Conclusion names finite temperature as the method's
generalisation.  With K already orthogonalised (S = I in Eq. DsignSym) the
density matrix becomes

    D = f(K - mu I),   f(x) = 1 / (1 + exp(x / kT)),

applied to every submatrix exactly as signum is in Section III-A: assemble
a_j = K[N(j), N(j)] - mu I, take f(a_j) = Q diag(f(lambda)) Q^T from the
symmetric eigendecomposition (Eq. eigendecompsym), and copy the columns of
block j into block column j of D.  As kT -> 0, f(x) -> (1 - signum(x)) / 2
with f(0) = 1/2, the zero-temperature D of ``oracle.submatrix``.

Readings (the paper gives no formula beyond "replace signum"):
* kT is in the units of K's eigenvalues; the Fermi function is the
  occupation 1 / (1 + exp((lambda - mu) / kT)).
* The electron count N(mu) = Tr D is Algorithm 1's count with signum replaced:
  sum over the columns c of block j of sum_l Q_cl^2 f(lambda_l - mu_corr).
* dN/dmu = sum_c sum_l Q_cl^2 f (1 - f) / kT > 0, so a Newton step on mu is
  well posed (at T = 0 it is zero almost everywhere); the search is a
  bracketed Newton iteration that falls back to bisection (Section IV-G names
  bisection for Algorithm 1's update).
* The gradient of the map K -> D is the Daleckii-Krein form with the Fermi
  function's divided differences; on the diagonal they are f'(lambda).
"""
from __future__ import annotations

import math

import numpy as np

from .submatrix import _block_lookup, _pool, assemble_submatrix, column_structure


def fermi(x, kT):
    """f(x) = 1 / (1 + exp(x / kT)), evaluated without overflow; kT > 0."""
    x = np.asarray(x, dtype=np.float64)
    t = x / kT
    e = np.exp(-np.abs(t))
    return np.where(t > 0, e / (1.0 + e), 1.0 / (1.0 + e))


def fermi_deriv(x, kT):
    """f'(x) = -f(x) (1 - f(x)) / kT."""
    f = fermi(x, kT)
    return -f * (1.0 - f) / kT


def fermi_by_eigh(a, kT):
    """f(a) = Q diag(f(lambda)) Q^T for symmetric ``a`` (Eq. eigendecompsym
    with signum replaced).  Returns (f(a), eigenvalues, Q)."""
    lam, q = np.linalg.eigh(a)
    return (q * fermi(lam, kT)[None, :]) @ q.T, lam, q


def density_block_column_T(m, j, mu, kT, rows=None, lookup=None):
    """Block column j of D = f(K - mu I) (Section III-A step 3)."""
    if lookup is None:
        lookup = _block_lookup(m)
    a, rows, loc, k = assemble_submatrix(m, j, mu, rows, lookup)
    fa, _lam, _q = fermi_by_eigh(a, kT)
    c0, c1 = loc[k], loc[k + 1]
    out = {}
    for u, r in enumerate(rows):
        out[(int(r), int(j))] = fa[loc[u]:loc[u + 1], c0:c1].copy()
    return out


def _worker_columns_T(args):
    m, mu, kT, js = args
    structure = column_structure(m)
    lookup = _block_lookup(m)
    res = {}
    for j in js:
        res.update(density_block_column_T(m, int(j), mu, kT, structure[int(j)], lookup))
    return res


def density_matrix_T(m, mu=None, kT=0.01, columns=None, workers=1):
    """D = f(K - mu I) by the submatrix method, in K's block pattern
    (entries of columns not evaluated are NaN)."""
    if mu is None:
        mu = m.mu
    js = np.arange(m.nblk) if columns is None else np.asarray(columns)
    if workers > 1 and len(js) > 1:
        chunks = [js[w::workers] for w in range(workers)]
        res = {}
        with _pool(workers) as ex:
            for part in ex.map(_worker_columns_T, [(m, mu, kT, c) for c in chunks if len(c)]):
                res.update(part)
    else:
        res = _worker_columns_T((m, mu, kT, js))
    lookup = _block_lookup(m)
    out = np.full(m.vals.shape, np.nan)
    for (r, c), blk in res.items():
        off, nr, nc, _p = lookup[(r, c)]
        out[off:off + nr * nc] = blk.reshape(-1)
    return out


# ---------------------------------------------------------------------------
# Electron count and its derivative (Algorithm 1 with signum replaced)
# ---------------------------------------------------------------------------

def n_elec_T(decomps, mu_corr, kT):
    """N for a shift mu_corr: sum over submatrices and the columns c of block
    j of sum_l Q_cl^2 f(lambda_l - mu_corr).  ``decomps`` as returned by
    ``oracle.decompose_all`` (eigenvalues of a_j, rows of Q of block j)."""
    total = []
    for lam, qrows in decomps:
        total.extend(((qrows * qrows) @ fermi(lam - mu_corr, kT)).tolist())
    return math.fsum(total)


def dn_dmu_T(decomps, mu_corr, kT):
    """dN/dmu_corr = sum_c sum_l Q_cl^2 f (1 - f) / kT (the chain rule on
    f(lambda - mu))."""
    total = []
    for lam, qrows in decomps:
        total.extend(((qrows * qrows) @ (-fermi_deriv(lam - mu_corr, kT))).tolist())
    return math.fsum(total)


def mu_search_newton_T(decomps, n_el, kT, lo, hi, tol=1e-12, max_steps=200):
    """mu_corr with N(mu_corr) = n_el: Newton steps on the smooth, strictly
    increasing N, kept inside a bracket [lo, hi] with N(lo) <= n_el <= N(hi);
    a step that leaves the bracket is replaced by bisection.
    Returns (mu_corr, N(mu_corr), steps)."""
    n_lo = n_elec_T(decomps, lo, kT)
    n_hi = n_elec_T(decomps, hi, kT)
    if not (n_lo <= n_el <= n_hi):
        raise ValueError("bracket does not contain the electron count")
    mu = 0.5 * (lo + hi)
    for steps in range(1, max_steps + 1):
        n = n_elec_T(decomps, mu, kT)
        if abs(n - n_el) <= tol * abs(n_el):
            return mu, n, steps
        if n < n_el:
            lo = mu
        else:
            hi = mu
        d = dn_dmu_T(decomps, mu, kT)
        nxt = mu - (n - n_el) / d if d > 0 else 0.5 * (lo + hi)
        if not (lo < nxt < hi):
            nxt = 0.5 * (lo + hi)
        mu = nxt
    return mu, n_elec_T(decomps, mu, kT), max_steps


# ---------------------------------------------------------------------------
# Gradient: Daleckii-Krein with the Fermi function
# ---------------------------------------------------------------------------

def frechet_fermi(lam, q, e, kT):
    """Frechet derivative of f at a = Q diag(lam) Q^T in direction e:
    Q (Phi o (Q^T e Q)) Q^T with Phi_lm = (f_l - f_m) / (lam_l - lam_m) for
    lam_l != lam_m and Phi = f'(lam_l) where they coincide."""
    f = fermi(lam, kT)
    fp = fermi_deriv(lam, kT)
    dl = lam[:, None] - lam[None, :]
    df = f[:, None] - f[None, :]
    same = dl == 0
    with np.errstate(divide="ignore", invalid="ignore"):
        phi = np.where(same, 0.5 * (fp[:, None] + fp[None, :]), df / np.where(same, 1.0, dl))
    return q @ (phi * (q.T @ e @ q)) @ q.T


def fermi_backward(m, dbar_vals, mu=None, kT=0.01, columns=None):
    """Vector-Jacobian product of K -> D = f(K - mu I) by the submatrix method.

    Block column j contributes abar_j = L_f(a_j, G_j), G_j holding Dbar's
    block column j in its columns of block j (zero elsewhere), added into
    every stored block of K that a_j was assembled from.  Returns (Kbar
    values, dN/dmu) with dN/dmu = -sum_j sum_{c in block j} L_f(a_j, I)_cc
    = sum_j sum_c (f (1 - f) / kT)(a_j)_cc."""
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
        abar = frechet_fermi(lam, q, g, kT)
        for u, r in enumerate(rows):
            for v, c in enumerate(rows):
                hit = lookup.get((int(r), int(c)))
                if hit is None:
                    continue
                off, nr, nc, _p = hit
                kbar[off:off + nr * nc] += abar[loc[u]:loc[u + 1], loc[v]:loc[v + 1]].reshape(-1)
        li = frechet_fermi(lam, q, np.eye(n), kT)
        dndmu.extend((-np.diagonal(li)[loc[k]:loc[k + 1]]).tolist())
    return kbar, math.fsum(dndmu)
