"""Submatrices shared by groups of block columns (Section IV-C) on the GPU
against the grouped oracle, element by element."""
import numpy as np
import pytest

import oracle
from synth import make_config, random_symmetric_bsr, small_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2004_10811_gb300 as p
    return p


def run(pkg, m, mu, groups, **kw):
    import torch
    K = torch.from_numpy(m.vals).cuda()
    with pkg.Plan.from_bsr(m, groups=groups, **kw) as plan:
        D = plan.sign(K, mu)
        tr = plan.trace(D)
        st = plan.stats()
    return D.cpu().numpy(), tr, st


@pytest.mark.parametrize("seed", [3, 4])
def test_random_groups_uneven_blocks(pkg, seed):
    m = random_symmetric_bsr([3, 2, 4, 3, 2, 3, 1, 4, 5, 2, 3, 6], density=0.35, seed=seed, scale=0.5)
    groups = np.unique(np.random.default_rng(seed).integers(0, 4, m.nblk), return_inverse=True)[1]
    want = oracle.density_matrix_grouped(m, 0.1, groups)
    got, tr, st = run(pkg, m, 0.1, groups, prec="fp64")
    assert float(np.max(np.abs(got - want))) <= 1e-10
    assert st["nsub"] == groups.max() + 1


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-7)])
def test_kmeans_groups_on_water(pkg, prec, tol):
    from paper_2004_10811_gb300 import grouping
    m = small_case(n_mol=40, block=4, r_c=5.5, seed=5)
    groups = grouping.periodic_kmeans(m.coords, m.box, m.nblk // 2, seed=1)
    want = oracle.density_matrix_grouped(m, 0.0, groups)
    got, tr, st = run(pkg, m, 0.0, groups, prec=prec)
    assert float(np.max(np.abs(got - want))) <= tol
    assert abs(tr - oracle.trace_bsr(m, want)) <= 1e-9 * m.n_el


def test_singleton_groups_equal_the_plain_plan(pkg):
    """One column per group is the plain method; the member-wise scatter reads
    S from the other triangle, and X Y of two commuting symmetric matrices is
    symmetric only up to rounding on diagonal tiles."""
    import torch
    m = small_case(n_mol=24, block=3, r_c=5.5, seed=8)
    K = torch.from_numpy(m.vals).cuda()
    with pkg.Plan.from_bsr(m, prec="fp64") as plan:
        d0 = plan.sign(K, 0.0).cpu().numpy()
    d1, _tr, _st = run(pkg, m, 0.0, np.arange(m.nblk), prec="fp64")
    assert float(np.max(np.abs(d0 - d1))) <= 1e-14


def test_grouped_finite_temperature_matches_singletons_limit(pkg):
    """Finite temperature through the member-wise scatter: singleton groups
    against the plain finite-temperature oracle."""
    m = small_case(n_mol=20, block=4, r_c=5.5, seed=9)
    got, _tr, st = run(pkg, m, 0.0, np.arange(m.nblk), prec="fp64", kT=0.1)
    assert float(np.max(np.abs(got - oracle.density_matrix_T(m, 0.0, 0.1)))) <= 1e-10


def test_water20736_kmeans_pairs_sampled(pkg):
    """The 20736x6 workload with k-means groups of about two columns, mixed
    path, every group evaluated; the oracle computes 24 sampled groups."""
    from paper_2004_10811_gb300 import grouping
    m = make_config(4)
    groups = grouping.periodic_kmeans(m.coords, m.box, m.nblk // 2, seed=1)
    sample = np.linspace(0, groups.max(), 24).astype(int)
    want = oracle.density_matrix_grouped(m, m.mu, groups, only=sample)
    mask = ~np.isnan(want)
    got, _tr, st = run(pkg, m, m.mu, groups, prec="mixed")
    assert float(np.max(np.abs(got[mask] - want[mask]))) <= 1e-7
    assert st["refine_fallback"] == 0


def test_grouped_refusals(pkg):
    import torch
    m = small_case(n_mol=12, block=3, r_c=5.5, seed=9)
    groups = np.arange(m.nblk) // 2
    K = torch.from_numpy(m.vals).cuda()
    with pkg.Plan.from_bsr(m, prec="fp64", groups=groups) as plan:
        with pytest.raises(pkg.SubmatError) as ei:
            plan.sign_backward(K, 0.0, torch.ones_like(K))
        assert ei.value.name == "UNSUPPORTED"
    with pytest.raises(pkg.SubmatError) as ei:
        pkg.Plan.from_bsr(m, prec="fp64", groups=groups, columns=(0, 4))
    assert ei.value.name == "UNSUPPORTED"
