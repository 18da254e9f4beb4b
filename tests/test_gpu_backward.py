"""Adjoint of K -> D (submat_sign_backward, the coupled Newton-Schulz
iteration) against the oracle's Daleckii-Krein gradient, central finite
differences of the GPU forward map, and the identities of L_sign."""
import numpy as np
import pytest

import oracle
from oracle import submatrix as osub
from synth import small_case
from synth.water import make_water

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2004_10811_gb300 as p
    return p


def transpose_index(m):
    """perm such that vals[perm] lays out K_(c,r)^T in block (r, c)'s slots."""
    vp = m.val_ptr
    rows = np.repeat(np.arange(m.nblk), np.diff(m.row_ptr))
    pos = {(int(rows[p]), int(m.col_idx[p])): p for p in range(m.nnzb)}
    perm = np.empty(m.vals.shape[0], dtype=np.int64)
    for (r, c), p in pos.items():
        q = pos[(c, r)]
        br, bc = m.block_sizes[r], m.block_sizes[c]
        idx = np.arange(br * bc)
        u, v = idx // bc, idx % bc
        perm[vp[p] + idx] = vp[q] + v * br + u
    return perm


# adjoint_mode 1: the coupled iteration on the tensor cores (BF16x3 split
# products, about 16 bits), hence the wider bounds
@pytest.mark.parametrize("prec,mode,tol,dn_tol", [("fp64", 0, 1e-9, 1e-6), ("mixed", 0, 2e-5, 1e-6),
                                                  ("mixed", 1, 2e-4, 1e-3)])
def test_vjp_matches_daleckii_krein(pkg, prec, mode, tol, dn_tol):
    import torch
    m = small_case(n_mol=20, block=4, r_c=5.5, seed=101)
    rng = np.random.default_rng(1)
    dbar = rng.standard_normal(m.vals.shape)
    want, dn_want = oracle.sign_backward(m, dbar, 0.05)
    with pkg.Plan.from_bsr(m, prec=prec, adjoint_mode=mode) as plan:
        kbar, dn = plan.sign_backward(torch.from_numpy(m.vals).cuda(), 0.05,
                                      torch.from_numpy(dbar).cuda(), want_dn_dmu=True)
    got = kbar.cpu().numpy()
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
    assert abs(dn) < dn_tol and abs(dn_want) < 1e-9   # L_sign(a, I) = 0 at T = 0


def test_band_energy_gradient_through_autograd(pkg):
    """E = Tr(D K) = sum over blocks of D_(r,c) . K_(c,r)^T; torch autograd
    supplies the explicit term, the library the implicit one."""
    import torch
    m = small_case(n_mol=16, block=3, r_c=5.5, seed=102)
    perm = torch.from_numpy(transpose_index(m)).cuda()
    K = torch.from_numpy(m.vals.copy()).cuda().requires_grad_(True)
    with pkg.Plan.from_bsr(m, prec="fp64") as plan:
        sign_fn = pkg.make_autograd_sign(plan)
        D = sign_fn(K, 0.0)
        E = (D * K[perm]).sum()
        E.backward()
        got = K.grad.cpu().numpy()
    want = oracle.band_energy_grad(m, 0.0)
    assert abs(E.item() - oracle.band_energy(m, oracle.density_matrix(m, 0.0))) < 1e-10
    assert np.max(np.abs(got - want)) <= 1e-9 * np.max(np.abs(want))


def test_finite_differences_of_the_gpu_forward(pkg):
    """Central differences (h = 1e-6) of E = Tr(D K) evaluated by the FP64 GPU
    path, moving K_pq and K_qp together, against Kbar_pq + Kbar_qp."""
    import torch
    m = make_water(24, 4, 6.0, (2, -1.0, -0.3), (2, 0.3, 1.0), seed=103)
    perm_np = transpose_index(m)
    perm = torch.from_numpy(perm_np).cuda()
    rng = np.random.default_rng(2)
    h = 1e-6
    with pkg.Plan.from_bsr(m, prec="fp64") as plan:
        K0 = torch.from_numpy(m.vals.copy()).cuda()

        def energy(Kt):
            D = plan.sign(Kt, 0.0)
            return float((D * Kt[perm]).sum().item())

        D0 = plan.sign(K0, 0.0)
        kbar = plan.sign_backward(K0, 0.0, K0[perm].contiguous()).cpu().numpy()
        grad = D0[perm].cpu().numpy() + kbar
        for _ in range(64):
            i1 = int(rng.integers(m.vals.shape[0]))
            i2 = int(perm_np[i1])
            e = torch.zeros_like(K0)
            e[i1] += h
            if i2 != i1:
                e[i2] += h
            fd = (energy(K0 + e) - energy(K0 - e)) / (2 * h)
            an = grad[i1] + (grad[i2] if i2 != i1 else 0.0)
            assert abs(fd - an) <= 2e-6 * max(1.0, abs(an)), (i1, fd, an)


@pytest.mark.parametrize("prec,mode,tol", [("fp64", 0, 1e-9), ("fp32", 0, 2e-5), ("mixed", 1, 2e-4)])
def test_vjp_matches_daleckii_krein_at_128_molecules(pkg, prec, mode, tol):
    """The 2048x23 workload's recipe (block 23, cutoff 8 A, submatrices of
    1288-1840) at 128 molecules: the adjoint of block columns [0, 16) against
    the oracle's Daleckii-Krein gradient of the same columns."""
    import torch
    m = make_water(128, 23, 8.0, (4, -1.0, -0.3), (19, 0.3, 1.5), seed=104)
    cols = (0, 16)
    rng = np.random.default_rng(3)
    dbar = rng.standard_normal(m.vals.shape)
    want, _dn = oracle.sign_backward(m, dbar, 0.0, columns=range(*cols))
    with pkg.Plan.from_bsr(m, prec=prec, columns=cols, adjoint_mode=mode) as plan:
        kbar = plan.sign_backward(torch.from_numpy(m.vals).cuda(), 0.0, torch.from_numpy(dbar).cuda())
    got = kbar.cpu().numpy()
    assert np.max(np.abs(want)) > 0
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


def test_central_differences_on_the_2048x23_workload(pkg):
    """The 2048x23 workload itself (submatrices of 1472-1932): central
    differences (h = 1e-6) of E = Tr(D K) by the FP64 path against
    Kbar_pq + Kbar_qp plus the explicit term, on 8 entries.  Only the block
    columns whose submatrices contain both block rows of an entry (and the
    two columns of the explicit term) change E, so E and the adjoint are
    evaluated on those columns alone, with column-range plans (reading c11)."""
    import torch
    from synth import make_config
    m = make_config(3)
    rp, ci, vp = m.row_ptr, m.col_idx, m.val_ptr
    rows = np.repeat(np.arange(m.nblk), np.diff(rp))
    nbh = [set(ci[rp[j]:rp[j + 1]].tolist()) for j in range(m.nblk)]
    perm_np = transpose_index(m)
    rng = np.random.default_rng(11)
    entries, colsets = [], []
    while len(entries) < 8:  # entries whose affected column set is small
        p = int(rng.integers(m.nnzb))
        P, Q = int(rows[p]), int(ci[p])
        C = sorted({j for j in nbh[P] & nbh[Q] if P in nbh[j] and Q in nbh[j]} | {P, Q})
        if len(C) <= 26:
            entries.append(int(vp[p] + rng.integers(vp[p + 1] - vp[p])))
            colsets.append(C)

    def runs(cols):
        cols = sorted(set(cols))
        out, a = [], cols[0]
        for x, y in zip(cols, cols[1:] + [None]):
            if y != x + 1:
                out.append((a, x + 1))
                a = y
        return out

    plans = {}

    def plan(run):
        if run not in plans:
            plans[run] = pkg.Plan.from_bsr(m, prec="fp64", columns=run)
        return plans[run]

    K0 = torch.from_numpy(m.vals.copy()).cuda()
    Kt = K0[torch.from_numpy(perm_np).cuda()].contiguous()
    allc = sorted(set(j for C in colsets for j in C))
    D0 = torch.zeros_like(K0)
    kbar = torch.zeros_like(K0)
    for run in runs(allc):
        plan(run).sign(K0, 0.0, out=D0)
        kbar += plan(run).sign_backward(K0, 0.0, Kt)
    grad = D0.cpu().numpy()[perm_np] + kbar.cpu().numpy()
    h = 1e-6
    for i1, C in zip(entries, colsets):
        i2 = int(perm_np[i1])
        blocks = np.flatnonzero(np.isin(ci, C))
        pos = np.concatenate([np.arange(vp[b], vp[b + 1]) for b in blocks])
        es = []
        for sgn in (1.0, -1.0):
            v = m.vals.copy()
            v[i1] += sgn * h
            if i2 != i1:
                v[i2] += sgn * h
            Kd = torch.from_numpy(v).cuda()
            D = torch.zeros_like(Kd)
            for run in runs(C):
                plan(run).sign(Kd, 0.0, out=D)
            d = D.cpu().numpy()
            es.append(float(np.dot(d[pos], v[perm_np[pos]])))
        fd = (es[0] - es[1]) / (2 * h)
        an = grad[i1] + (grad[i2] if i2 != i1 else 0.0)
        assert abs(fd - an) <= 2e-6 * max(1.0, abs(an)), (i1, fd, an)
    for p in plans.values():
        p.close()
