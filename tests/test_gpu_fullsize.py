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
