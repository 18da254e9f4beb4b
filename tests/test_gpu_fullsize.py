"""The GPU path at the full sizes of the five workloads, in the configuration
bench.py uses, on sampled block columns the oracle computes one by one."""
import numpy as np
import pytest

import oracle
from synth import make_config

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-7}


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2004_10811_gb300 as p
    return p


def sampled(m, count):
    step = max(1, m.nblk // count)
    return list(range(0, m.nblk, step))[:count] + [m.nblk - 1]


def check(pkg, m, prec, count, **kw):
    import torch
    cols = sampled(m, count)
    want = oracle.density_matrix(m, m.mu, columns=cols, workers=8)
    mask = ~np.isnan(want)
    K = torch.from_numpy(m.vals).cuda()
    with pkg.Plan.from_bsr(m, prec=prec, **kw) as plan:
        D = plan.sign(K, m.mu)
        st = plan.stats()
    got = D.cpu().numpy()
    err = float(np.max(np.abs(got[mask] - want[mask])))
    assert err <= TOL[prec], (err, st)
    # trace over the sampled diagonal blocks
    vp = m.val_ptr
    rows = np.repeat(np.arange(m.nblk), np.diff(m.row_ptr))
    dpos = {int(r): p for p, r in enumerate(rows) if m.col_idx[p] == r}
    tr_g = sum(np.trace(got[vp[dpos[j]]:vp[dpos[j] + 1]].reshape(m.block_sizes[j], -1)) for j in cols)
    tr_o = sum(np.trace(want[vp[dpos[j]]:vp[dpos[j] + 1]].reshape(m.block_sizes[j], -1)) for j in cols)
    assert abs(tr_g - tr_o) / m.n_el <= 1e-9
    return st


def test_water1024_b23_mixed(pkg):
    st = check(pkg, make_config(1), "mixed", 24)
    assert st["n_max"] > 1800


def test_slab4096_b6_mixed(pkg):
    st = check(pkg, make_config(2), "mixed", 32)
    assert st["n_min"] < 120 and st["n_max"] > 400   # uneven sizes in one batch


def test_water2048_b23_mixed(pkg):
    check(pkg, make_config(3), "mixed", 16)


def test_water20736_b6_mixed(pkg):
    """n = 124,416 with the gap shrunk to +-0.15; the batch is split into waves."""
    st = check(pkg, make_config(4), "mixed", 32)
    assert st["nsub"] == 20736


def test_water32_b6_fp64_and_slab_fp64_sample(pkg):
    check(pkg, make_config(0), "fp64", 32)
    # the FP64 path on a contiguous chunk of the slab (column-range plan)
    import torch
    m = make_config(2)
    cols = list(range(0, 64))
    want = oracle.density_matrix(m, m.mu, columns=cols, workers=8)
    mask = ~np.isnan(want)
    with pkg.Plan.from_bsr(m, prec="fp64", columns=(0, 64)) as plan:
        D = plan.sign(torch.from_numpy(m.vals).cuda(), m.mu, out=torch.zeros(m.vals.shape, dtype=torch.float64, device="cuda"))
    assert float(np.max(np.abs(D.cpu().numpy()[mask] - want[mask]))) <= 1e-10


def check_ranges(pkg, m, prec, ranges, tol):
    """Column-range plans on the full matrix: each evaluates a few contiguous
    block columns; the oracle computes the same columns one by one."""
    import torch
    cols = [j for a, b in ranges for j in range(a, b)]
    want = oracle.density_matrix(m, m.mu, columns=cols, workers=8)
    K = torch.from_numpy(m.vals).cuda()
    D = torch.zeros_like(K)
    worst = 0.0
    for a, b in ranges:
        with pkg.Plan.from_bsr(m, prec=prec, columns=(a, b)) as plan:
            plan.sign(K, m.mu, out=D)
            st = plan.stats()
        assert st["not_converged"] == 0
    got = D.cpu().numpy()
    mask = ~np.isnan(want)
    worst = float(np.max(np.abs(got[mask] - want[mask])))
    assert worst <= tol, worst
    return worst


@pytest.mark.parametrize("cfg", [1, 3, 4])
def test_fp64_path_at_full_size_on_column_ranges(pkg, cfg):
    """The plain FP64 path's 1e-10 bound on the workloads' own submatrices:
    1311-1909 dims (1024x23), 1472-1932 (2048x23), 504-672 (20736x6), on
    three column ranges spread over the system."""
    m = make_config(cfg)
    q = m.nblk
    ranges = [(0, 2), (q // 2, q // 2 + 2), (q - 2, q)]
    check_ranges(pkg, m, "fp64", ranges, TOL["fp64"])


def test_fp32_path_on_water1024_b23(pkg):
    """The FP32 path (Newton-Schulz in FP32, no refinement) on the 1024x23
    workload, every column evaluated: its error plateaus near 1e-6, so it is
    reported and held only to a loose bound, not to the mixed path's 1e-7."""
    import torch
    m = make_config(1)
    cols = sampled(m, 16)
    want = oracle.density_matrix(m, m.mu, columns=cols, workers=8)
    mask = ~np.isnan(want)
    with pkg.Plan.from_bsr(m, prec="fp32") as plan:
        D = plan.sign(torch.from_numpy(m.vals).cuda(), m.mu)
        st = plan.stats()
    err = float(np.max(np.abs(D.cpu().numpy()[mask] - want[mask])))
    print(f"fp32 path, 1024x23: max|dD| = {err:.3e} on {len(cols)} block columns, "
          f"iterations {st['iters_min']}-{st['iters_max']}")
    assert st["not_converged"] == 0
    assert err < 1e-4
