"""Parity of the mixed path (FP16x3 tensor-core Newton-Schulz + FP64-anchored
correction) with the CPU oracle: max|dD| <= 1e-7 and the trace."""
import numpy as np
import pytest

import oracle
from synth import make_config, random_symmetric_bsr
from synth.water import make_water

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-7


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2004_10811_gb300 as p
    return p


def run(pkg, m, mu, **kw):
    import torch
    K = torch.from_numpy(m.vals).cuda()
    with pkg.Plan.from_bsr(m, prec="mixed", **kw) as plan:
        D = plan.sign(K, mu)
        tr = plan.trace(D)
        st = plan.stats()
    return D.cpu().numpy(), tr, st


@pytest.mark.parametrize("hp_mode", [0, 1])
def test_config0_mixed(pkg, hp_mode):
    m = make_config(0)
    want = oracle.density_matrix(m, 0.0)
    got, tr, st = run(pkg, m, 0.0, hp_mode=hp_mode)
    err = np.max(np.abs(got - want))
    assert err <= TOL_MIXED, (err, st)
    assert abs(tr - oracle.trace_bsr(m, want)) / m.n_el <= 1e-9
    assert st["refine_rounds"] >= 1 and st["iters_max"] < 40


@pytest.mark.parametrize("hp_mode", [0, 1])
@pytest.mark.parametrize("n_mol,block,r_c,seed,mu", [
    (96, 5, 6.5, 77, 0.05),     # dims ~100-300: several 128-tiles, ragged tails
    (40, 23, 6.0, 78, 0.0),     # block 23 as in the large workloads
])
def test_water_mixed(pkg, n_mol, block, r_c, seed, mu, hp_mode):
    occ = max(1, block // 5)
    m = make_water(n_mol, block, r_c, (occ, -1.0, -0.3), (block - occ, 0.3, 1.2), seed=seed)
    want = oracle.density_matrix(m, mu, workers=4)
    got, tr, st = run(pkg, m, mu, hp_mode=hp_mode)
    err = np.max(np.abs(got - want))
    assert err <= TOL_MIXED, (err, st)
    assert abs(tr - oracle.trace_bsr(m, want)) / max(1.0, m.n_el) <= 1e-9


def test_uneven_blocks_mixed(pkg):
    m = random_symmetric_bsr([5, 7, 3, 9, 2, 8, 6, 4, 7, 5, 3, 6] * 3, density=0.3, seed=26, scale=0.3)
    want = oracle.density_matrix(m, 0.1)
    got, _tr, st = run(pkg, m, 0.1)
    assert np.max(np.abs(got - want)) <= TOL_MIXED, st


def test_one_round_is_enough_from_split_iterate(pkg):
    m = make_config(0)
    want = oracle.density_matrix(m, 0.0)
    got, _tr, _st = run(pkg, m, 0.0, refine_rounds=1)
    assert np.max(np.abs(got - want)) <= TOL_MIXED


def test_sliced_and_fp64_residual_products_agree(pkg):
    """The two ways of forming I - S^2 and S a (tensor-core slices, FP64 SIMT)
    give the same D to well below the mixed tolerance, with one round."""
    m = make_water(64, 23, 6.0, (4, -1.0, -0.3), (19, 0.3, 1.5), seed=5)
    d0, _t0, s0 = run(pkg, m, 0.0, hp_mode=0, refine_rounds=1)
    d1, _t1, s1 = run(pkg, m, 0.0, hp_mode=1, refine_rounds=1)
    assert s0["refine_fallback"] == 0 and s1["refine_fallback"] == 0
    assert np.max(np.abs(d0 - d1)) < 2e-8


@pytest.mark.parametrize("hp_mode", [0, 1])
def test_two_rounds(pkg, hp_mode):
    """A second correction round (36-bit grid for the sign iterate, level-cut
    slice products) lands well inside the FP64 path's 1e-10 bound."""
    m = make_water(40, 23, 6.0, (4, -1.0, -0.3), (19, 0.3, 1.5), seed=79)
    want = oracle.density_matrix(m, 0.0, workers=4)
    got, tr, st = run(pkg, m, 0.0, hp_mode=hp_mode, refine_rounds=2)
    assert st["refine_rounds"] == 2 and st["refine_fallback"] == 0, st
    assert np.max(np.abs(got - want)) <= 1e-10
    assert abs(tr - oracle.trace_bsr(m, want)) / m.n_el <= 1e-10


def test_autotune_picks_widths_and_keeps_parity(pkg):
    """submat_autotune times 128- and 256-wide tiles per tensor-core phase and
    keeps a valid choice; D from the tuning run and after it meet the bound."""
    import torch
    m = make_water(40, 23, 6.0, (4, -1.0, -0.3), (19, 0.3, 1.5), seed=80)
    want = oracle.density_matrix(m, 0.0, workers=4)
    K = torch.from_numpy(m.vals).cuda()
    with pkg.Plan.from_bsr(m, prec="mixed") as plan:
        D0 = torch.empty_like(K)
        w = plan.autotune(K, 0.0, out=D0)
        assert set(w) == {"ns", "correction", "sliced"} and all(v in (128, 256) for v in w.values()), w
        assert plan.options.tile_n_ns == w["ns"] and plan.options.tile_n_hp == w["sliced"]
        D1 = plan.sign(K, 0.0)
    for D in (D0, D1):
        assert np.max(np.abs(D.cpu().numpy() - want)) <= TOL_MIXED


def test_submatrices_above_2048_one_slice_product_per_accumulator(pkg):
    """Dims 2139-2645 (ld > 2048): each exact FP32 accumulator takes one slice
    product (63^2 x ld stays below 2^24 only for one), the planner still pairs
    accumulators of adjacent levels; block columns [0, 8) against the oracle."""
    import torch
    m = make_water(256, 23, 9.0, (4, -1.0, -0.3), (19, 0.3, 1.5), seed=106)
    cols = (0, 8)
    want = oracle.density_matrix(m, 0.0, columns=range(*cols))
    K = torch.from_numpy(m.vals).cuda()
    with pkg.Plan.from_bsr(m, prec="mixed", columns=cols) as plan:
        D = plan.sign(K, 0.0).cpu().numpy()
        st = plan.stats()
    assert st["n_max"] > 2048 and st["refine_fallback"] == 0, st
    vp = m.val_ptr
    mine = [p for p in range(m.nnzb) if cols[0] <= m.col_idx[p] < cols[1]]
    idx = np.concatenate([np.arange(vp[p], vp[p + 1]) for p in mine])
    assert np.max(np.abs(D[idx] - want[idx])) <= TOL_MIXED


def test_third_order_iteration(pkg):
    """iteration = 1: the paper's GPU iteration X (15I - 10X^2 + 3X^4) / 8,
    three symmetric products per step, fewer steps than Newton-Schulz, the
    same D within the mixed bound."""
    m = make_water(40, 23, 6.0, (4, -1.0, -0.3), (19, 0.3, 1.5), seed=81)
    want = oracle.density_matrix(m, 0.0, workers=4)
    got3, tr3, st3 = run(pkg, m, 0.0, iteration=1)
    got2, _tr2, st2 = run(pkg, m, 0.0)
    assert st3["refine_fallback"] == 0
    assert st3["iters_max"] < st2["iters_max"], (st3["iters_max"], st2["iters_max"])
    assert np.max(np.abs(got3 - want)) <= TOL_MIXED
    assert abs(tr3 - oracle.trace_bsr(m, want)) / m.n_el <= 1e-9
