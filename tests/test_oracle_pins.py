"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test checks the oracle against the mathematics the paper states (the
sign function's definition, Eq. sign; its spectral form, Eqs. signev and
signevext; the three steps of Section III-A; Algorithm 1) through a route
the oracle does not use: a cyclic Jacobi eigensolver, the Schur-based
matrix square root, Sylvester inertia from an LDL^T factorisation, closed
forms and brute force on tiny inputs.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from oracle import submatrix as osub
from synth import bsr_to_dense, make_config, random_symmetric_bsr, small_case
from synth.water import make_water


# ---------------------------------------------------------------------------
# independent helpers (no oracle code)
# ---------------------------------------------------------------------------

def jacobi_eigh(a, sweeps=60):
    """Cyclic Jacobi rotations (brute force for n <= ~48)."""
    a = np.array(a, dtype=np.float64)
    n = a.shape[0]
    v = np.eye(n)
    for _ in range(sweeps):
        off = np.sqrt(np.sum(np.tril(a, -1) ** 2))
        if off < 1e-15 * max(1.0, np.linalg.norm(a)):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if abs(a[p, q]) < 1e-300:
                    continue
                theta = (a[q, q] - a[p, p]) / (2.0 * a[p, q])
                t = math.copysign(1.0, theta) / (abs(theta) + math.sqrt(theta * theta + 1.0))
                c = 1.0 / math.sqrt(t * t + 1.0)
                s = t * c
                rot = np.eye(n)
                rot[p, p] = c
                rot[q, q] = c
                rot[p, q] = s
                rot[q, p] = -s
                a = rot.T @ a @ rot
                v = v @ rot
    return np.diag(a).copy(), v


def sign_via_sqrtm(a):
    """sign(A) = A (A^2)^(-1/2) (Eq. sign) with the Schur square root."""
    root = sla.sqrtm(a @ a)
    root = np.real(root)
    return np.linalg.solve(root, a)


def count_negative_eigenvalues(a):
    """Sylvester inertia: number of negative eigenvalues from LDL^T."""
    _lu, d, _perm = sla.ldl(a)
    ev = []
    i = 0
    n = d.shape[0]
    while i < n:
        if i + 1 < n and d[i + 1, i] != 0.0:
            ev.extend(np.linalg.eigvalsh(d[i:i + 2, i:i + 2]).tolist())
            i += 2
        else:
            ev.append(d[i, i])
            i += 1
    return int(np.sum(np.array(ev) < 0))


def brute_force_submatrix_method(dense, block_sizes, mu):
    """Section III-A on a dense matrix, written out independently: for every
    block column find the block rows with any nonzero entry, take the
    principal submatrix, apply sign (sqrtm route) and copy the columns."""
    off = np.concatenate([[0], np.cumsum(block_sizes)])
    nb = len(block_sizes)
    out = np.zeros_like(dense)
    for j in range(nb):
        rows = [i for i in range(nb)
                if np.any(dense[off[i]:off[i + 1], off[j]:off[j + 1]] != 0) or i == j]
        idx = np.concatenate([np.arange(off[i], off[i + 1]) for i in rows])
        a = dense[np.ix_(idx, idx)] - mu * np.eye(len(idx))
        s = sign_via_sqrtm(a)
        half = 0.5 * (np.eye(len(idx)) - s)
        cols = np.arange(off[j], off[j + 1])
        cpos = [np.where(idx == c)[0][0] for c in cols]
        for u, gi in enumerate(idx):
            out[gi, cols] = half[u, cpos]
    return out


def dense_from_vals(m, vals):
    return bsr_to_dense(m.with_vals(vals))


# ---------------------------------------------------------------------------
# sign of one matrix (Eqs. sign, signev, signevext, eigendecompsym)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,seed", [(6, 0), (17, 1), (40, 2)])
def test_sign_matches_jacobi(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n))
    a = a + a.T
    s, _lam, _q = osub.sign_by_eigh(a)
    lam_j, v = jacobi_eigh(a)
    s_j = (v * np.sign(lam_j)) @ v.T
    assert np.max(np.abs(s - s_j)) < 1e-10


@pytest.mark.parametrize("n,seed", [(12, 3), (64, 4)])
def test_sign_matches_schur_sqrt(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n))
    a = a + a.T
    s = osub.sign_by_eigh(a)[0]
    assert np.max(np.abs(s - sign_via_sqrtm(a))) < 1e-9


def test_sign_closed_form_square_is_scalar():
    """A = Q diag(+-s) Q^T has A^2 = s^2 I, so sign(A) = A / s."""
    rng = np.random.default_rng(5)
    q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    s = 0.7
    d = np.where(rng.uniform(size=30) < 0.4, -s, s)
    a = (q * d) @ q.T
    sa = osub.sign_by_eigh(a)[0]
    assert np.max(np.abs(sa - a / s)) < 1e-13


def test_sign_of_diagonal_is_signum_with_zero():
    """Diagonal input: scalar signum per entry, and signum(0) = 0
    (Eq. signevext)."""
    d = np.array([-2.0, -0.5, 0.0, 0.25, 3.0, 0.0])
    s = osub.sign_by_eigh(np.diag(d))[0]
    assert np.array_equal(np.round(s, 15), np.diag([-1.0, -1.0, 0.0, 1.0, 1.0, 0.0]))


@pytest.mark.parametrize("seed", [0, 1])
def test_sign_invariants_on_submatrices(seed):
    """sign^2 = I and [sign(a), a] = 0 for every submatrix of a small case."""
    m = small_case(n_mol=20, block=4, r_c=5.5, seed=seed)
    struct = osub.column_structure(m)
    for j in range(m.nblk):
        s, _rows, _loc, _k, _lam, _q = osub.submatrix_sign(m, j, m.mu, struct[j])
        a = osub.assemble_submatrix(m, j, m.mu, struct[j])[0]
        assert np.max(np.abs(s @ s - np.eye(s.shape[0]))) < 1e-12
        assert np.max(np.abs(s @ a - a @ s)) < 1e-12


# ---------------------------------------------------------------------------
# the submatrix method (Section III-A)
# ---------------------------------------------------------------------------

def test_column_structure_is_block_rows_with_stored_blocks():
    m = random_symmetric_bsr([3, 1, 4, 2, 5, 2], density=0.4, seed=11)
    dense = bsr_to_dense(m)
    off = np.concatenate([[0], np.cumsum(m.block_sizes)])
    struct = osub.column_structure(m)
    for j in range(m.nblk):
        expect = [i for i in range(m.nblk)
                  if np.any(dense[off[i]:off[i + 1], off[j]:off[j + 1]] != 0)]
        assert struct[j].tolist() == expect


def test_assemble_matches_dense_indexing():
    m = random_symmetric_bsr([2, 3, 1, 4, 2, 3, 1], density=0.5, seed=12)
    dense = bsr_to_dense(m)
    off = np.concatenate([[0], np.cumsum(m.block_sizes)])
    for j in range(m.nblk):
        a, rows, loc, k = osub.assemble_submatrix(m, j, 0.3)
        idx = np.concatenate([np.arange(off[i], off[i + 1]) for i in rows])
        assert np.array_equal(a, dense[np.ix_(idx, idx)] - 0.3 * np.eye(len(idx)))
        assert rows[k] == j and loc[k] == sum(m.block_sizes[r] for r in rows[:k])


@pytest.mark.parametrize("sizes,density,seed,mu", [
    ([2, 3, 1, 4, 2, 3], 0.45, 21, 0.0),
    ([3, 3, 3, 3, 3, 3, 3, 3], 0.3, 22, 0.4),
    ([1, 5, 2, 2, 4, 1, 3], 0.6, 23, -0.2),
])
def test_density_matches_brute_force(sizes, density, seed, mu):
    m = random_symmetric_bsr(sizes, density=density, seed=seed)
    d = oracle.density_matrix(m, mu)
    got = dense_from_vals(m, d)
    want = brute_force_submatrix_method(bsr_to_dense(m), m.block_sizes, mu)
    pattern = dense_from_vals(m, np.ones_like(m.vals)) != 0
    assert np.max(np.abs(got - want)[pattern]) < 1e-9
    assert np.all(got[~pattern] == 0)


def test_uncoupled_blocks_are_exact_projectors():
    """Block-diagonal K (cutoff below the closest pair): every submatrix is a
    single diagonal block, so D_jj is the projector onto its occupied space:
    idempotent, commuting with K_jj, trace = number of occupied levels, and
    equal to (I - K (K^2)^(-1/2)) / 2."""
    m = make_water(12, 6, 0.5, (3, -1.0, -0.3), (3, 0.3, 1.0), seed=31)
    assert m.nnzb == m.nblk
    d = oracle.density_matrix(m, 0.0)
    for j in range(m.nblk):
        kb = m.vals[j * 36:(j + 1) * 36].reshape(6, 6)
        db = d[j * 36:(j + 1) * 36].reshape(6, 6)
        assert np.max(np.abs(db @ db - db)) < 1e-13
        assert np.max(np.abs(db @ kb - kb @ db)) < 1e-13
        assert abs(np.trace(db) - 3.0) < 1e-13
        ref = 0.5 * (np.eye(6) - sign_via_sqrtm(kb))
        assert np.max(np.abs(db - ref)) < 1e-10


def test_full_cover_equals_dense_sign():
    """Cutoff beyond half the box diagonal: every submatrix is all of K, so
    D is exactly 1/2 (I - sign(K - mu I)) of the whole matrix (Eq. DsignSym
    with S = I): idempotent, and Tr D is the integer count of eigenvalues
    below mu (Sylvester inertia)."""
    m = make_water(10, 4, 100.0, (2, -1.0, -0.3), (2, 0.3, 1.0), seed=41)
    assert m.nnzb == m.nblk * m.nblk
    for mu in (0.0, 0.35):
        d = dense_from_vals(m, oracle.density_matrix(m, mu))
        k = bsr_to_dense(m)
        ref = 0.5 * (np.eye(m.n) - sign_via_sqrtm(k - mu * np.eye(m.n)))
        assert np.max(np.abs(d - ref)) < 1e-9
        assert np.max(np.abs(d @ d - d)) < 1e-12
        count = count_negative_eigenvalues(k - mu * np.eye(m.n))
        assert abs(oracle.trace_bsr(m, oracle.density_matrix(m, mu)) - count) < 1e-10


def test_tie_at_mu_gives_one_half():
    """An eigenvalue exactly at mu (Eq. signevext): exactly representable
    diagonal blocks, uncoupled, mu equal to one of the diagonal entries."""
    bs = np.array([2, 2], dtype=np.int32)
    from synth.water import BSRMatrix
    vals = np.array([-0.5, 0.0, 0.0, 0.25,   # block (0,0)
                     -1.0, 0.0, 0.0, 0.75])  # block (1,1)
    m = BSRMatrix(bs, np.array([0, 1, 2]), np.array([0, 1], dtype=np.int32), vals)
    d = oracle.density_matrix(m, 0.25)
    assert d.tolist() == [1.0, 0.0, 0.0, 0.5, 1.0, 0.0, 0.0, 0.0]
    assert oracle.trace_bsr(m, d) == 2.5


def test_label_permutation_permutes_d():
    m = random_symmetric_bsr([2, 3, 1, 4, 2, 3, 2], density=0.45, seed=51)
    perm = np.array([4, 0, 6, 2, 5, 1, 3])  # new label of old block i is perm[i]
    dense = bsr_to_dense(m)
    off = np.concatenate([[0], np.cumsum(m.block_sizes)])
    inv = np.argsort(perm)
    new_sizes = m.block_sizes[inv]
    blocks = {}
    vp = m.val_ptr
    for r in range(m.nblk):
        for p in range(m.row_ptr[r], m.row_ptr[r + 1]):
            c = m.col_idx[p]
            blocks[(perm[r], perm[c])] = m.vals[vp[p]:vp[p + 1]]
    keys = sorted(blocks)
    from synth.water import BSRMatrix
    row_ptr = np.zeros(m.nblk + 1, dtype=np.int64)
    for (r, _c) in keys:
        row_ptr[r + 1] += 1
    np.cumsum(row_ptr, out=row_ptr)
    m2 = BSRMatrix(new_sizes.astype(np.int32), row_ptr,
                   np.array([c for _r, c in keys], dtype=np.int32),
                   np.concatenate([blocks[k] for k in keys]))
    d1 = dense_from_vals(m, oracle.density_matrix(m, 0.1))
    d2 = dense_from_vals(m2, oracle.density_matrix(m2, 0.1))
    off2 = np.concatenate([[0], np.cumsum(new_sizes)])
    for i in range(m.nblk):
        for j in range(m.nblk):
            a = d1[off[i]:off[i + 1], off[j]:off[j + 1]]
            b = d2[off2[perm[i]]:off2[perm[i] + 1], off2[perm[j]]:off2[perm[j] + 1]]
            assert np.max(np.abs(a - b)) < 1e-12
    assert dense.shape == d1.shape


def test_workers_agree_with_serial():
    m = small_case(n_mol=16, block=3, r_c=5.0, seed=3)
    d1 = oracle.density_matrix(m, 0.0)
    d2 = oracle.density_matrix(m, 0.0, workers=2)
    assert np.array_equal(d1, d2)


def test_config0_shapes_and_plateau():
    """The 32-molecule workload: every submatrix has a gap around mu = 0 and
    the trace is close to N_el = 96."""
    m = make_config(0)
    d = oracle.density_matrix(m, 0.0)
    assert np.all(np.isfinite(d))
    tr = oracle.trace_bsr(m, d)
    assert abs(tr - m.n_el) < 0.05 * m.n_el


# ---------------------------------------------------------------------------
# Algorithm 1 (Section IV-G)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mu_corr", [0.0, 0.2, -0.35])
def test_alg1_count_equals_trace_of_d(mu_corr):
    m = small_case(n_mol=18, block=4, r_c=5.5, seed=61)
    dec = oracle.decompose_all(m, 0.0)
    n_alg = oracle.n_elec_alg1(dec, mu_corr)
    tr = oracle.trace_bsr(m, oracle.density_matrix(m, mu_corr))
    assert abs(n_alg - tr) < 1e-11


def test_alg1_bisection_reaches_count():
    m = small_case(n_mol=18, block=4, r_c=5.5, seed=62)
    dec = oracle.decompose_all(m, 0.0)
    target = oracle.n_elec_alg1(dec, 0.0) + 3.0
    mu, n, _steps, (lo, hi) = oracle.mu_search_alg1(dec, target, -2.0, 2.0)
    # either exact hit on a plateau or a bracket across which N jumps over it
    assert abs(n - target) < 1e-9 or (oracle.n_elec_alg1(dec, lo) < target < oracle.n_elec_alg1(dec, hi))
    assert oracle.n_elec_alg1(dec, -2.0) < target < oracle.n_elec_alg1(dec, 2.0)


# ---------------------------------------------------------------------------
# derivatives (Daleckii-Krein) against finite differences and identities
# ---------------------------------------------------------------------------

def _frechet_by_fd(a, e, h=1e-6):
    return (sign_via_sqrtm(a + h * e) - sign_via_sqrtm(a - h * e)) / (2 * h)


def test_frechet_matches_fd_and_identities():
    rng = np.random.default_rng(71)
    n = 14
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([-rng.uniform(0.3, 1.0, 6), rng.uniform(0.3, 1.2, 8)])
    a = (q * lam) @ q.T
    lam_o, q_o = np.linalg.eigh(a)
    e = rng.standard_normal((n, n))
    e = e + e.T
    l_e = osub.frechet_sign(lam_o, q_o, e)
    assert np.max(np.abs(l_e - _frechet_by_fd(a, e))) < 1e-6
    s = osub.sign_by_eigh(a)[0]
    assert np.max(np.abs(osub.frechet_sign(lam_o, q_o, a))) < 1e-12       # L(A, A) = 0
    assert np.max(np.abs(osub.frechet_sign(lam_o, q_o, np.eye(n)))) < 1e-12  # L(A, I) = 0
    w = rng.standard_normal((n, n))
    comm = osub.frechet_sign(lam_o, q_o, w @ a - a @ w)
    assert np.max(np.abs(comm - (w @ s - s @ w))) < 1e-11   # L(A,[W,A]) = [W, sign A]


def test_band_energy_gradient_matches_fd():
    """dE/dK with K kept symmetric: moving K_pq and K_qp together compares
    with Kbar_pq + Kbar_qp (both triangles stored)."""
    m = small_case(n_mol=10, block=3, r_c=5.5, seed=81)
    g = oracle.band_energy_grad(m, 0.0)
    rng = np.random.default_rng(82)
    vp = m.val_ptr
    lookup = osub._block_lookup(m)
    rows_of = np.repeat(np.arange(m.nblk), np.diff(m.row_ptr))
    h = 1e-6
    for _ in range(8):
        p = int(rng.integers(m.nnzb))
        r, c = int(rows_of[p]), int(m.col_idx[p])
        nr, nc = int(m.block_sizes[r]), int(m.block_sizes[c])
        u, v = int(rng.integers(nr)), int(rng.integers(nc))
        i1 = vp[p] + u * nc + v
        toff = lookup[(c, r)][0]
        i2 = toff + v * nr + u

        def energy(delta):
            vals = m.vals.copy()
            vals[i1] += delta
            if i2 != i1:
                vals[i2] += delta
            mm = m.with_vals(vals)
            return oracle.band_energy(mm, oracle.density_matrix(mm, 0.0))
        fd = (energy(h) - energy(-h)) / (2 * h)
        an = g[i1] + (g[i2] if i2 != i1 else 0.0)
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (p, u, v, fd, an)


def test_dn_dmu_is_zero_at_zero_temperature():
    """L_sign(a, I) = 0 for nonsingular a, so the T = 0 electron count is a
    staircase in mu."""
    m = small_case(n_mol=8, block=3, r_c=5.5, seed=91)
    _kbar, dn = oracle.sign_backward(m, np.zeros_like(m.vals), 0.0)
    assert abs(dn) < 1e-12


# ---------------------------------------------------------------------------
# the pins catch planted mistakes (planted in the oracle, on the CPU)
# ---------------------------------------------------------------------------

def test_planted_signum_tie_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(osub, "signum", lambda x: np.where(np.asarray(x) >= 0, 1.0, -1.0))
    with pytest.raises(AssertionError):
        test_tie_at_mu_gives_one_half()


def test_planted_transpose_mistake_is_caught(monkeypatch):
    def wrong(a):
        lam, q = np.linalg.eigh(a)
        return (q.T * osub.signum(lam)[None, :]) @ q, lam, q
    monkeypatch.setattr(osub, "sign_by_eigh", wrong)
    with pytest.raises(AssertionError):
        test_sign_matches_jacobi(17, 1)


def test_planted_wrong_column_is_caught(monkeypatch):
    orig = osub.assemble_submatrix

    def shifted(m, j, mu, rows=None, lookup=None):
        a, rows, loc, k = orig(m, j, mu, rows, lookup)
        return a, rows, loc, (k + 1) % len(rows)
    monkeypatch.setattr(osub, "assemble_submatrix", shifted)
    with pytest.raises(AssertionError):
        test_density_matches_brute_force([3, 3, 3, 3, 3, 3, 3, 3], 0.3, 22, 0.4)
