"""The entry point that allocates no memory (submat_dense_sign_noalloc).

Some callers cannot allocate: codes that reserve the whole GPU for their own
memory pool, allocators that forbid foreign allocations, and time steps where
an allocation's implicit device synchronisation is not acceptable.  For them
the dense one-matrix evaluation keeps all its scratch in a fixed device array
inside the library.  This checks it against the oracle's dense sign and
against the regular entry point (a plan with one dense block, FP64 path) on
two calls in a row, with the FP64 tolerance of the other parity tests, and
that oversize input is refused.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


@pytest.fixture(scope="module")
def sm():
    import __graft_entry__ as g
    g.build()
    from paper_2004_10811_gb300 import submat
    return submat


def dense_case(n, seed):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    k = n // 3
    lam = np.concatenate([rng.uniform(-1.2, -0.25, k), rng.uniform(0.25, 1.4, n - k)])
    a = (q * lam) @ q.T
    return 0.5 * (a + a.T)


def reference_dense(sm, a, mu):
    import torch
    n = a.shape[0]
    with sm.Plan(np.array([n], np.int32), np.array([0, 1], np.int64), np.array([0], np.int32),
                 prec="fp64") as plan:
        K = torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()
        return plan.sign(K, mu).cpu().numpy().reshape(n, n)


def test_noalloc_matches_plan_path_on_two_calls(sm):
    import torch
    cases = [(dense_case(512, 1), 0.05), (dense_case(191, 2), -0.1)]
    for a, mu in cases:
        n = a.shape[0]
        K = torch.from_numpy(a).cuda()
        d, iters = sm.dense_sign_noalloc(K, mu)
        torch.cuda.synchronize()
        got = d.cpu().numpy()
        want = reference_dense(sm, a, mu)
        err = np.max(np.abs(got - want))
        assert err <= TOL_FP64, (n, err)
        # the oracle: D = (I - sign(a - mu I)) / 2 by eigendecomposition
        import oracle
        d_or = 0.5 * (np.eye(n) - oracle.dense_sign(a - mu * np.eye(n)))
        assert np.max(np.abs(got - d_or)) <= TOL_FP64, n
        assert 5 < iters < 60


def test_noalloc_allocates_no_device_memory(sm):
    """After a first call (which loads the library's device code and with it
    the fixed scratch array), further calls on other sizes leave the device's
    free memory and torch's allocator untouched."""
    import torch
    a1, a2 = dense_case(300, 3), dense_case(97, 4)
    K1 = torch.from_numpy(a1).cuda()
    K2 = torch.from_numpy(a2).cuda()
    D1 = torch.empty_like(K1)
    D2 = torch.empty_like(K2)
    sm.dense_sign_noalloc(K1, 0.0, out=D1)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(2):
        sm.dense_sign_noalloc(K2, 0.1, out=D2)
        sm.dense_sign_noalloc(K1, -0.1, out=D1)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_rejects_oversize(sm):
    import torch
    K = torch.zeros(513, 513, dtype=torch.float64, device="cuda")
    with pytest.raises(sm.SubmatError) as ei:
        sm.dense_sign_noalloc(K, 0.0)
    assert ei.value.name == "INVALID_ARG"
