"""Parity of the CUDA path (through the C ABI) with the CPU oracle: FP64
Newton-Schulz, gather/scatter, trace, waves and the error statuses."""
import numpy as np
import pytest

import oracle
from synth import make_config, random_symmetric_bsr, small_case
from synth.water import BSRMatrix, make_water

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10   # max |D_gpu - D_oracle| for the FP64 path


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2004_10811_gb300 as p
    return p


def run(pkg, m, mu, **kw):
    import torch
    K = torch.from_numpy(m.vals).cuda()
    with pkg.Plan.from_bsr(m, **kw) as plan:
        D = plan.sign(K, mu)
        tr = plan.trace(D)
        stats = plan.stats()
        sub = plan.sub_stats()
    return D.cpu().numpy(), tr, stats, sub


@pytest.mark.parametrize("sizes,density,seed,mu", [
    ([2, 3, 1, 4, 2, 3], 0.45, 21, 0.0),
    ([5, 7, 3, 9, 2, 8, 6, 4, 7, 5, 3, 6], 0.35, 24, 0.15),
    ([1] * 70, 0.2, 25, -0.1),        # 1x1 blocks: element-wise method, ragged dims
])
def test_random_uneven_blocks(pkg, sizes, density, seed, mu):
    m = random_symmetric_bsr(sizes, density=density, seed=seed, scale=0.5)
    want = oracle.density_matrix(m, mu)
    got, tr, _st, _sub = run(pkg, m, mu)
    assert np.max(np.abs(got - want)) <= TOL_FP64
    assert abs(tr - oracle.trace_bsr(m, want)) <= 1e-12 * max(1.0, abs(tr))


def test_config0_fp64(pkg):
    m = make_config(0)
    want = oracle.density_matrix(m, 0.0)
    got, tr, st, sub = run(pkg, m, 0.0)
    err = np.max(np.abs(got - want))
    assert err <= TOL_FP64, err
    assert abs(tr - oracle.trace_bsr(m, want)) / m.n_el <= 1e-12
    assert st["not_converged"] == 0 and st["iters_max"] < 40
    assert np.all(sub["dims"] == np.diff(m.row_ptr) * 6)


def test_small_water_several_tiles(pkg):
    """Submatrices of 100-300 dims: several 64-wide tiles and ragged tails."""
    m = make_water(96, 5, 6.5, (2, -1.0, -0.3), (3, 0.3, 1.2), seed=77)
    want = oracle.density_matrix(m, 0.05, workers=4)
    got, tr, st, _sub = run(pkg, m, 0.05)
    assert st["n_max"] > 128
    assert np.max(np.abs(got - want)) <= TOL_FP64


def test_waves_match_single_wave(pkg):
    m = small_case(n_mol=40, block=4, r_c=5.5, seed=5)
    one, _t1, s1, _ = run(pkg, m, 0.0)
    many, _t2, s2, _ = run(pkg, m, 0.0, workspace_cap_bytes=1_200_000)
    assert s1["waves"] == 1 and s2["waves"] > 3
    assert np.array_equal(one, many)


def test_symmetrize_option(pkg):
    m = small_case(n_mol=24, block=3, r_c=5.0, seed=8)
    d, _t, _s, _ = run(pkg, m, 0.0)
    ds, _t, _s, _ = run(pkg, m, 0.0, symmetrize=True)
    vp = m.val_ptr
    rows = np.repeat(np.arange(m.nblk), np.diff(m.row_ptr))
    pos = {(int(rows[p]), int(m.col_idx[p])): p for p in range(m.nnzb)}
    for (r, c), p in pos.items():
        q = pos[(c, r)]
        a = d[vp[p]:vp[p + 1]].reshape(3, 3)
        b = d[vp[q]:vp[q + 1]].reshape(3, 3)
        assert np.allclose(ds[vp[p]:vp[p + 1]].reshape(3, 3), 0.5 * (a + b.T), atol=1e-15)


def test_uncoupled_and_full_cover(pkg):
    for m in (make_water(12, 6, 0.5, (3, -1.0, -0.3), (3, 0.3, 1.0), seed=31),
              make_water(10, 4, 100.0, (2, -1.0, -0.3), (2, 0.3, 1.0), seed=41)):
        want = oracle.density_matrix(m, 0.0)
        got, tr, _s, _ = run(pkg, m, 0.0)
        assert np.max(np.abs(got - want)) <= TOL_FP64
        assert abs(tr - m.n_el) < 1e-9


def test_nonfinite_input_is_reported(pkg):
    import torch
    m = small_case(n_mol=12, block=3, r_c=5.0, seed=9)
    vals = m.vals.copy()
    vals[17] = np.nan
    K = torch.from_numpy(vals).cuda()
    with pkg.Plan.from_bsr(m) as plan:
        with pytest.raises(pkg.SubmatError) as ei:
            plan.sign(K, 0.0)
        assert ei.value.name == "NONFINITE"


def test_tie_at_mu_and_singular_status(pkg):
    """Eigenvalue exactly at mu: the iteration keeps it at 0, D gets 1/2
    (Eq. signevext); the submatrix never becomes an involution, so the call
    reports NOT_CONVERGED with D written."""
    import torch
    bs = np.array([2, 2], dtype=np.int32)
    vals = np.array([-0.5, 0.0, 0.0, 0.25, -1.0, 0.0, 0.0, 0.75])
    m = BSRMatrix(bs, np.array([0, 1, 2]), np.array([0, 1], dtype=np.int32), vals)
    K = torch.from_numpy(vals).cuda()
    with pkg.Plan.from_bsr(m, max_iter=30) as plan:
        with pytest.raises(pkg.SubmatError) as ei:
            plan.sign(K, 0.25)
        assert ei.value.name == "NOT_CONVERGED"
        D = plan.sign(K, 0.25, allow_not_converged=True).cpu().numpy()
    assert D.tolist() == [1.0, 0.0, 0.0, 0.5, 1.0, 0.0, 0.0, 0.0]


def test_host_buffer_entry_point(pkg):
    import torch
    m = small_case(n_mol=20, block=4, r_c=5.5, seed=10)
    with pkg.Plan.from_bsr(m) as plan:
        d_dev = plan.sign(torch.from_numpy(m.vals).cuda(), 0.1).cpu().numpy()
        d_host = plan.sign_host(m.vals, 0.1)
    assert np.array_equal(d_dev, d_host)


def test_fp32_path_error_is_reported_not_bounded_by_mixed_tolerance(pkg):
    m = make_config(0)
    want = oracle.density_matrix(m, 0.0)
    got, _tr, st, _ = run(pkg, m, 0.0, prec="fp32")
    err = np.max(np.abs(got - want))
    assert err < 1e-4, err
