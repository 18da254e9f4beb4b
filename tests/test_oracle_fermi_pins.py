"""Pins of the finite-temperature oracle (``oracle.fermi``: the Fermi function
in place of signum, Section IV-F's last paragraph) against routes it does not
use: the matrix exponential (scipy's scaling and squaring, no eigensolver),
closed forms, the zero-temperature oracle in the limit kT -> 0, central
differences, and a library root finder for the mu search.  Planted mistakes
in the oracle must fail them."""
import importlib

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.optimize as sopt

import oracle
from synth import bsr_to_dense, small_case
from synth.water import BSRMatrix, make_water

# the module (the package re-exports its function of the same name)
ofermi = importlib.import_module("oracle.fermi")


def fermi_by_expm(a, kT):
    """(I + exp(a / kT))^{-1}, the Fermi function of a matrix, through the
    matrix exponential (no eigendecomposition), written as
    exp(-B) (exp(B) + exp(-B))^{-1} with B = a / (2 kT): the matrix inverted
    is 2 cosh(B), whose eigenvalues are >= 2, so the solve is well conditioned."""
    b = a / (2.0 * kT)
    em = sla.expm(-b)
    return np.linalg.solve((sla.expm(b) + em).T, em.T).T


def dense_case(n, seed, lo=-1.0, hi=1.2):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = rng.uniform(lo, hi, n)
    a = (q * lam) @ q.T
    return 0.5 * (a + a.T)


def test_fermi_function_values():
    x = np.array([-3.0, -0.2, 0.0, 0.2, 3.0, 1e4, -1e4])
    kT = 0.1
    f = oracle.fermi(x, kT)
    direct = [1.0 / (1.0 + np.exp(v / kT)) if abs(v / kT) < 700 else (0.0 if v > 0 else 1.0) for v in x]
    assert np.allclose(f, direct, rtol=1e-15, atol=1e-300)
    assert f[2] == 0.5
    assert np.all(np.isfinite(f))
    assert np.allclose(oracle.fermi(x, kT) + oracle.fermi(-x, kT), 1.0, atol=1e-15)
    assert np.all(np.diff(oracle.fermi(np.linspace(-1, 1, 101), kT)) < 0)


@pytest.mark.parametrize("n,seed,kT", [(12, 1, 0.3), (30, 2, 0.1), (40, 3, 0.05)])
def test_fermi_of_matrix_matches_expm(n, seed, kT):
    a = dense_case(n, seed)
    want = fermi_by_expm(a, kT)
    got, _lam, _q = oracle.fermi_by_eigh(a, kT)
    assert np.max(np.abs(got - want)) < 1e-9


def test_square_scalar_closed_form():
    """A^2 = alpha I: A has eigenvalues +-sqrt(alpha), so
    f(A) = (I - tanh(sqrt(alpha) / (2 kT)) A / sqrt(alpha)) / 2."""
    rng = np.random.default_rng(7)
    n, alpha, kT = 10, 0.49, 0.2
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    a = (q * np.sqrt(alpha) * np.array([1, -1] * (n // 2))) @ q.T
    want = 0.5 * (np.eye(n) - np.tanh(np.sqrt(alpha) / (2 * kT)) * a / np.sqrt(alpha))
    got, _lam, _q = oracle.fermi_by_eigh(a, kT)
    assert np.max(np.abs(got - want)) < 1e-13


def test_uncoupled_diagonal_blocks_give_elementwise_fermi():
    """No off-diagonal blocks and diagonal diagonal blocks: every submatrix is
    one diagonal block, D = diag(f(d - mu)) exactly."""
    rng = np.random.default_rng(3)
    bs = np.array([3, 2, 4], dtype=np.int32)
    vals = []
    for b in bs:
        vals.append(np.diag(rng.uniform(-1, 1, b)).reshape(-1))
    m = BSRMatrix(bs, np.array([0, 1, 2, 3], np.int64), np.array([0, 1, 2], np.int32), np.concatenate(vals))
    mu, kT = 0.1, 0.07
    got = oracle.density_matrix_T(m, mu, kT)
    want = []
    for v, b in zip(vals, bs):
        d = np.diag(v.reshape(b, b))
        want.append(np.diag(1.0 / (1.0 + np.exp((d - mu) / kT))).reshape(-1))
    assert np.max(np.abs(got - np.concatenate(want))) < 1e-15


def test_full_cover_matches_dense_expm():
    """A cutoff that covers the box: every submatrix is the whole K, so each
    block column of D is that of f(K - mu I), through the exponential."""
    m = make_water(10, 4, 100.0, (2, -1.0, -0.3), (2, 0.3, 1.0), seed=41)
    mu, kT = 0.05, 0.08
    dense = bsr_to_dense(m)
    want_dense = fermi_by_expm(dense - mu * np.eye(dense.shape[0]), kT)
    got = oracle.density_matrix_T(m, mu, kT)
    off = np.concatenate([[0], np.cumsum(m.block_sizes)])
    vp = m.val_ptr
    for r in range(m.nblk):
        for p in range(int(m.row_ptr[r]), int(m.row_ptr[r + 1])):
            c = int(m.col_idx[p])
            blk = got[vp[p]:vp[p + 1]].reshape(m.block_sizes[r], m.block_sizes[c])
            assert np.max(np.abs(blk - want_dense[off[r]:off[r + 1], off[c]:off[c + 1]])) < 1e-10


def test_zero_temperature_limit():
    """kT far below every |eigenvalue - mu|: the Fermi function is the step
    (1 - signum) / 2 to within exp(-1/kT'), so D equals the T = 0 oracle."""
    m = small_case(n_mol=16, block=3, r_c=5.5, seed=102)
    dec = oracle.decompose_all(m, 0.0)
    gap = min(np.min(np.abs(lam)) for lam, _q in dec)
    assert gap > 1e-3
    d0 = oracle.density_matrix(m, 0.0)
    dT = oracle.density_matrix_T(m, 0.0, gap / 200.0)
    assert np.max(np.abs(dT - d0)) < 1e-12


def test_count_equals_trace_and_derivative_matches_fd():
    """N(mu) of the stored decompositions equals Tr D, and dN/dmu equals
    central differences of N."""
    m = small_case(n_mol=12, block=3, r_c=5.5, seed=9)
    kT = 0.05
    dec = oracle.decompose_all(m, 0.0)
    for mu_corr in (-0.2, 0.0, 0.15):
        d = oracle.density_matrix_T(m, mu_corr, kT)
        assert abs(oracle.trace_bsr(m, d) - oracle.n_elec_T(dec, mu_corr, kT)) < 1e-11
        h = 1e-5
        fd = (oracle.n_elec_T(dec, mu_corr + h, kT) - oracle.n_elec_T(dec, mu_corr - h, kT)) / (2 * h)
        dn = oracle.dn_dmu_T(dec, mu_corr, kT)
        assert dn > 0
        assert abs(dn - fd) < 1e-6 * max(1.0, abs(dn))


def test_frechet_fermi_matches_fd_of_expm():
    n, kT = 16, 0.1
    a = dense_case(n, 5)
    rng = np.random.default_rng(6)
    e = rng.standard_normal((n, n))
    lam, q = np.linalg.eigh(a)
    got = oracle.frechet_fermi(lam, q, e, kT)
    h = 1e-5
    fd = (fermi_by_expm(a + h * e, kT) - fermi_by_expm(a - h * e, kT)) / (2 * h)
    assert np.max(np.abs(got - fd)) < 1e-6 * np.max(np.abs(fd))
    # in the direction I: f'(a), i.e. -f (1 - f) / kT as a matrix function
    fa = fermi_by_expm(a, kT)
    assert np.max(np.abs(oracle.frechet_fermi(lam, q, np.eye(n), kT) + (fa - fa @ fa) / kT)) < 1e-9


def test_fermi_backward_matches_fd():
    """<Kbar, E> = d/dh <Dbar, D(K + h E)> for a symmetric direction E on the
    pattern; and the returned dN/dmu equals the count's derivative."""
    m = small_case(n_mol=8, block=3, r_c=5.5, seed=11)
    mu, kT = 0.02, 0.1
    rng = np.random.default_rng(2)
    dbar = rng.standard_normal(m.vals.shape)
    kbar, dn = oracle.fermi_backward(m, dbar, mu, kT)
    # a symmetric perturbation: E and its mirror blocks
    vp = m.val_ptr
    rows = np.repeat(np.arange(m.nblk), np.diff(m.row_ptr))
    pos = {(int(rows[p]), int(m.col_idx[p])): p for p in range(m.nnzb)}
    e = np.zeros(m.vals.shape)
    for (r, c), p in pos.items():
        if r <= c:
            blk = rng.standard_normal((m.block_sizes[r], m.block_sizes[c]))
            if r == c:
                blk = 0.5 * (blk + blk.T)
            e[vp[p]:vp[p + 1]] = blk.reshape(-1)
            q = pos[(c, r)]
            e[vp[q]:vp[q + 1]] = blk.T.reshape(-1)
    h = 1e-5
    mp = BSRMatrix(m.block_sizes, m.row_ptr, m.col_idx, m.vals + h * e)
    mm = BSRMatrix(m.block_sizes, m.row_ptr, m.col_idx, m.vals - h * e)
    fd = (np.dot(dbar, oracle.density_matrix_T(mp, mu, kT)) - np.dot(dbar, oracle.density_matrix_T(mm, mu, kT))) / (2 * h)
    assert abs(np.dot(kbar, e) - fd) < 1e-6 * max(1.0, abs(fd))
    dec = oracle.decompose_all(m, mu)
    assert abs(dn - oracle.dn_dmu_T(dec, 0.0, kT)) < 1e-9 * dn


def test_newton_search_matches_brentq():
    m = small_case(n_mol=12, block=3, r_c=5.5, seed=9)
    kT = 0.05
    dec = oracle.decompose_all(m, 0.0)
    n_el = 0.5 * (oracle.n_elec_T(dec, -0.4, kT) + oracle.n_elec_T(dec, 0.4, kT))
    mu, n, steps = oracle.mu_search_newton_T(dec, n_el, kT, -3.0, 3.0, tol=1e-13)
    root = sopt.brentq(lambda x: oracle.n_elec_T(dec, x, kT) - n_el, -3.0, 3.0, xtol=1e-15, rtol=1e-15)
    assert abs(mu - root) < 1e-9
    assert abs(n - n_el) <= 1e-13 * n_el
    assert steps < 60


def test_planted_fermi_sign_mistake_is_caught(monkeypatch):
    """f(x) = 1 / (1 + exp(-x / kT)) (occupying the wrong side) must fail the
    exponential route."""
    good = ofermi.fermi
    monkeypatch.setattr(ofermi, "fermi", lambda x, kT: good(-np.asarray(x), kT))
    a = dense_case(12, 1)
    got, _lam, _q = ofermi.fermi_by_eigh(a, 0.3)
    assert np.max(np.abs(got - fermi_by_expm(a, 0.3))) > 1e-3


def test_planted_missing_kT_in_derivative_is_caught(monkeypatch):
    """dN/dmu without the 1/kT factor must fail the central differences."""
    monkeypatch.setattr(ofermi, "fermi_deriv", lambda x, kT: -ofermi.fermi(x, kT) * (1 - ofermi.fermi(x, kT)))
    m = small_case(n_mol=12, block=3, r_c=5.5, seed=9)
    kT = 0.05
    dec = oracle.decompose_all(m, 0.0)
    h = 1e-5
    fd = (oracle.n_elec_T(dec, h, kT) - oracle.n_elec_T(dec, -h, kT)) / (2 * h)
    assert abs(ofermi.dn_dmu_T(dec, 0.0, kT) - fd) > 1e-3 * fd
