"""Pins of the grouped oracle (``oracle.grouped``: one submatrix per group of
block columns over the union of their row sets, Section IV-C) against routes
it does not use: a dense brute force with the Schur-root sign on tiny cases,
the dense sign of the whole K when one group holds every column or the
pattern covers the box, and the single-column method for groups of one."""
import importlib

import numpy as np
import scipy.linalg as sla

import oracle
from synth import bsr_to_dense, random_symmetric_bsr, small_case
from synth.water import make_water

ogrp = importlib.import_module("oracle.grouped")


def sign_via_sqrtm(a):
    """sign(A) = A (A^2)^(-1/2) (Eq. sign), Schur square root."""
    return np.linalg.solve(np.real(sla.sqrtm(a @ a)), a)


def brute_force_grouped(m, mu, groups):
    """Section IV-C on the dense matrix, written out independently: for every
    group the block rows with a nonzero block in any member column, the
    principal submatrix over them, its sign, and the member columns copied
    onto K's pattern."""
    dense = bsr_to_dense(m)
    off = np.concatenate([[0], np.cumsum(m.block_sizes)])
    nblk = m.nblk
    nz = np.zeros((nblk, nblk), dtype=bool)
    for i in range(nblk):
        for j in range(nblk):
            nz[i, j] = np.any(dense[off[i]:off[i + 1], off[j]:off[j + 1]] != 0)
    stored = np.zeros((nblk, nblk), dtype=bool)
    rows_of = np.repeat(np.arange(nblk), np.diff(m.row_ptr))
    stored[rows_of, m.col_idx] = True
    full = np.zeros_like(dense)
    for g in np.unique(groups):
        members = np.flatnonzero(groups == g)
        blocks = [i for i in range(nblk) if any(stored[i, j] for j in members)]
        idx = np.concatenate([np.arange(off[i], off[i + 1]) for i in blocks])
        a = dense[np.ix_(idx, idx)] - mu * np.eye(len(idx))
        d = 0.5 * (np.eye(len(idx)) - sign_via_sqrtm(a))
        for j in members:
            cols = np.arange(off[j], off[j + 1])
            cpos = [int(np.flatnonzero(idx == c)[0]) for c in cols]
            for i in blocks:
                if stored[i, j]:
                    rpos = [int(np.flatnonzero(idx == r)[0]) for r in range(off[i], off[i + 1])]
                    full[off[i]:off[i + 1], off[j]:off[j + 1]] = d[np.ix_(rpos, cpos)]
    out = np.zeros(m.vals.shape)
    vp = m.val_ptr
    for p in range(m.nnzb):
        r, c = rows_of[p], m.col_idx[p]
        out[vp[p]:vp[p + 1]] = full[off[r]:off[r + 1], off[c]:off[c + 1]].reshape(-1)
    return out


def test_groups_match_dense_brute_force():
    for seed in (3, 4, 5):
        m = random_symmetric_bsr([3, 2, 4, 3, 2, 3, 1, 4], density=0.35, seed=seed, scale=0.5)
        rng = np.random.default_rng(seed)
        groups = rng.integers(0, 3, m.nblk)
        groups = np.unique(groups, return_inverse=True)[1]
        got = ogrp.density_matrix_grouped(m, 0.1, groups)
        want = brute_force_grouped(m, 0.1, groups)
        assert np.max(np.abs(got - want)) < 1e-10


def test_singleton_groups_are_the_single_column_method():
    m = small_case(n_mol=14, block=3, r_c=5.5, seed=7)
    got = ogrp.density_matrix_grouped(m, 0.0, np.arange(m.nblk))
    assert np.max(np.abs(got - oracle.density_matrix(m, 0.0))) < 1e-12


def test_one_group_is_the_dense_sign_on_the_pattern():
    m = small_case(n_mol=10, block=3, r_c=5.0, seed=8)
    got = ogrp.density_matrix_grouped(m, 0.05, np.zeros(m.nblk, dtype=int))
    dense = bsr_to_dense(m)
    d = 0.5 * (np.eye(dense.shape[0]) - sign_via_sqrtm(dense - 0.05 * np.eye(dense.shape[0])))
    off = np.concatenate([[0], np.cumsum(m.block_sizes)])
    rows_of = np.repeat(np.arange(m.nblk), np.diff(m.row_ptr))
    vp = m.val_ptr
    for p in range(m.nnzb):
        r, c = rows_of[p], m.col_idx[p]
        assert np.max(np.abs(got[vp[p]:vp[p + 1]] - d[off[r]:off[r + 1], off[c]:off[c + 1]].reshape(-1))) < 1e-10


def test_full_cover_is_exact_for_any_grouping():
    m = make_water(10, 4, 100.0, (2, -1.0, -0.3), (2, 0.3, 1.0), seed=41)
    want = oracle.density_matrix(m, 0.0)
    for groups in (np.arange(m.nblk) // 3, np.array([0, 1] * 5)):
        assert np.max(np.abs(ogrp.density_matrix_grouped(m, 0.0, groups) - want)) < 1e-10


def test_planted_mistakes_are_caught(monkeypatch):
    """A submatrix over N(first member) only (fails to extract or disagrees)
    and a lost mu shift must both fail the brute force."""
    m = random_symmetric_bsr([3, 2, 4, 3, 2, 3, 1, 4], density=0.35, seed=3, scale=0.5)
    groups = np.array([0, 0, 1, 1, 2, 2, 3, 3])
    want = brute_force_grouped(m, 0.1, groups)
    good_rows, good_sign = ogrp.group_rows, ogrp.sign_by_eigh
    with monkeypatch.context() as mp:
        mp.setattr(ogrp, "group_rows", lambda m_, members, structure=None: good_rows(m_, members[:1], structure))
        try:
            got = ogrp.density_matrix_grouped(m, 0.1, groups)
            assert np.max(np.abs(got - want)) > 1e-6
        except KeyError:
            pass  # a member row outside the submatrix cannot be extracted
    with monkeypatch.context() as mp:
        mp.setattr(ogrp, "sign_by_eigh", lambda a: good_sign(a + 0.1 * np.eye(a.shape[0])))
        assert np.max(np.abs(ogrp.density_matrix_grouped(m, 0.1, groups) - want)) > 1e-6
