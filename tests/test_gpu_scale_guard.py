"""The scale of X_0 against an adversarial spectrum (Section II-B: the
Newton-Schulz iteration keeps the sign of an eigenvalue only inside
(-sqrt 3, sqrt 3)).

The default scale tightens the rigorous bound beta = min(max row abs-sum,
||a||_F) by a 10-step power estimate of rho(a) from a fixed positive start
vector.  Here the dominant eigenvector of a is orthogonal to that start vector
and its eigenvalue is twice the next one, so the estimate finds only the rest
of the spectrum: 1 / (1.05 r) puts the dominant eigenvalue of X_0 near 1.9,
where an unguarded iteration converges to the wrong sign (and still to an
involution that commutes with a).  The certificate from the first squaring
must catch this on every path, forward and adjoint, and the results must
match the oracle element by element at each path's usual bound.
"""
import numpy as np
import pytest

import oracle
from synth.water import BSRMatrix

N = 200


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2004_10811_gb300 as p
    return p


def power_start_vector(n):
    """The power iteration's start vector: 0.5 + (h mod 2^16) / 2^16 with
    h = (2654435761 i + 12345) mod 2^32, h ^= h >> 15 (a fixed hash of i)."""
    i = np.arange(n, dtype=np.uint64)
    h = (i * np.uint64(2654435761) + np.uint64(12345)) & np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(15)
    return 0.5 + (h & np.uint64(0xFFFF)).astype(np.float64) / 65536.0


def adversarial(n=N, top=2.0, seed=0):
    """One dense symmetric n x n block: eigenvalue `top` on a unit vector u
    orthogonal to the start vector, the rest in [-1, -0.3] and [0.3, 1]."""
    rng = np.random.default_rng(seed)
    v = power_start_vector(n)
    u = rng.standard_normal(n)
    u -= v * (v @ u) / (v @ v)
    u /= np.linalg.norm(u)
    q, _ = np.linalg.qr(np.column_stack([u, rng.standard_normal((n, n - 1))]))
    q[:, 0] = u
    k = n // 3
    lam = np.concatenate([[top], rng.uniform(-1.0, -0.3, k), rng.uniform(0.3, 1.0, n - 1 - k)])
    a = (q * lam) @ q.T
    a = 0.5 * (a + a.T)
    m = BSRMatrix(np.array([n], np.int32), np.array([0, 1], np.int64), np.array([0], np.int32),
                  np.ascontiguousarray(a.reshape(-1)))
    return m, a, u


def test_the_start_vector_misses_the_dominant_eigenvector():
    """The construction itself (on the CPU): u is orthogonal to the start
    vector, and a bare power estimate from it leaves X_0's dominant
    eigenvalue beyond sqrt(3)."""
    m, a, u = adversarial()
    v = power_start_vector(N)
    assert abs(v @ u) < 1e-12 * np.linalg.norm(v)
    beta = min(np.max(np.sum(np.abs(a), axis=1)), np.linalg.norm(a))
    x = a / beta
    w = v.copy()
    for _ in range(10):
        y = x @ w
        est = np.linalg.norm(y) / np.linalg.norm(w)
        w = y / np.linalg.norm(y)
    assert (1.0 / (1.05 * est)) * (2.0 / beta) > np.sqrt(3.0)


@pytest.mark.gpu
@pytest.mark.parametrize("prec,kw,tol", [
    ("fp64", {}, 1e-10),
    ("fp32", {}, 1e-4),
    ("mixed", {}, 1e-7),
    ("mixed", {"iteration": 1}, 1e-7),
])
def test_forward_paths_keep_the_dominant_sign(pkg, prec, kw, tol):
    import torch
    m, a, _u = adversarial()
    want = oracle.density_matrix(m, 0.0)
    with pkg.Plan.from_bsr(m, prec=prec, **kw) as plan:
        D = plan.sign(torch.from_numpy(m.vals).cuda(), 0.0)
        st = plan.stats()
    got = D.cpu().numpy()
    err = float(np.max(np.abs(got - want)))
    assert err <= tol, (prec, kw, err)
    assert st["scale_reduced"] == 1
    # the trace counts the negative eigenvalues of a (the dominant one is positive)
    assert abs(np.trace(got.reshape(N, N)) - np.sum(np.linalg.eigvalsh(a) < 0)) < 1e-3


@pytest.mark.gpu
def test_bound_scale_needs_no_reduction(pkg):
    """beta_mode 1 (the rigorous bound alone) is safe by construction."""
    import torch
    m, _a, _u = adversarial()
    want = oracle.density_matrix(m, 0.0)
    with pkg.Plan.from_bsr(m, prec="fp64", beta_mode=1) as plan:
        D = plan.sign(torch.from_numpy(m.vals).cuda(), 0.0)
        st = plan.stats()
    assert float(np.max(np.abs(D.cpu().numpy() - want))) <= 1e-10
    assert st["scale_reduced"] == 0


@pytest.mark.gpu
@pytest.mark.parametrize("prec,mode,tol", [("fp64", 0, 1e-9), ("mixed", 0, 2e-5), ("mixed", 1, 2e-4)])
def test_adjoint_keeps_the_dominant_sign(pkg, prec, mode, tol):
    """The adjoint's coupled iteration scales E_0 with X_0, so the rescale
    must reach E_0 (and its transpose on the tensor cores) as well."""
    import torch
    m, _a, _u = adversarial()
    rng = np.random.default_rng(3)
    dbar = rng.standard_normal(m.vals.shape)
    want, _ = oracle.sign_backward(m, dbar, 0.0)
    with pkg.Plan.from_bsr(m, prec=prec, adjoint_mode=mode) as plan:
        kbar = plan.sign_backward(torch.from_numpy(m.vals).cuda(), 0.0, torch.from_numpy(dbar).cuda())
        st = plan.stats()
    got = kbar.cpu().numpy()
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
    assert st["scale_reduced"] == 1
