"""The multi-GPU data plane on one GPU: column-range plans fed only their halo
reassemble the single-plan result, and a world-size-1 NCCL process group
drives the same device-resident functions (halo exchange, trace and
electron-count allreduces, mu search, column allgather, Kbar reduction)
that N ranks use."""
import os
import socket

import numpy as np
import pytest

from paper_2004_10811_gb300.shard import (ShardedPattern, gather_columns, gpu_solver, sharded_backward,
                                          sharded_density, sharded_mu_search)
from synth.water import make_water

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2004_10811_gb300 as p
    return p


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed", 1e-10)])
def test_chunks_with_halo_only_reassemble_the_full_result(pkg, prec, tol):
    import torch
    m = make_water(96, 5, 6.5, (2, -1.0, -0.3), (3, 0.3, 1.2), seed=77)
    with pkg.Plan.from_bsr(m, prec=prec) as plan:
        full = plan.sign(torch.from_numpy(m.vals).cuda(), 0.0).cpu().numpy()
    world = 3
    got = np.zeros_like(full)
    for rank in range(world):
        sp = ShardedPattern(m.block_sizes, m.row_ptr, m.col_idx, rank, world)
        halo_only = np.zeros_like(m.vals)
        sp.scatter_values(halo_only, sp.halo, sp.gather_values(m.vals, sp.halo))
        d, _tr = gpu_solver(sp, prec=prec)(torch.from_numpy(halo_only).cuda(), 0.0, sp.chunk)
        sp.scatter_values(got, sp.mine, sp.gather_values(d.cpu().numpy(), sp.mine))
    assert np.max(np.abs(got - full)) <= tol


@pytest.fixture(scope="module")
def nccl():
    import torch.distributed as dist
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    yield dist
    dist.destroy_process_group()


def test_world_one_nccl_data_plane(pkg, nccl):
    import torch
    import oracle
    dist = nccl
    m = make_water(48, 6, 6.0, (3, -1.0, -0.3), (3, 0.3, 1.0), seed=12)
    sp = ShardedPattern(m.block_sizes, m.row_ptr, m.col_idx, 0, 1)
    K = torch.from_numpy(m.vals).cuda()
    solve = gpu_solver(sp, prec="fp64")
    d, tr = sharded_density(sp, K.clone(), 0.0, solve, dist)
    want = oracle.density_matrix(m, 0.0)
    assert d.is_cuda
    assert float(np.max(np.abs(gather_columns(sp, d, dist).cpu().numpy() - want))) <= 1e-10
    assert abs(tr - oracle.trace_bsr(m, want)) <= 1e-9 * m.n_el
    # finite temperature: Newton steps on the allreduced count
    kT = 0.05
    solveT = gpu_solver(sp, prec="fp64", kT=kT)
    plan = solveT.plan_for(sp.chunk)
    mu, dT, n, steps = sharded_mu_search(sp, K.clone(), m.n_el, 0.4, solveT, dist, tol=1e-11, max_steps=40,
                                         bound=4.0, kT=kT, dn_dmu=lambda: plan.stats()["dn_dmu"])
    assert abs(n - m.n_el) <= 1e-11 * m.n_el and steps < 20
    dec = oracle.decompose_all(m, 0.0)
    assert abs(oracle.n_elec_T(dec, mu, kT) - m.n_el) <= 1e-9 * m.n_el
    # Kbar reduced over the (one) rank
    dbar = torch.from_numpy(np.random.default_rng(4).standard_normal(m.vals.shape)).cuda()
    bplan = pkg.Plan.from_bsr(m, prec="fp64", columns=sp.chunk)
    kbar = sharded_backward(sp, K.clone(), 0.0, dbar,
                            lambda Kl, mu_, Db, chunk: bplan.sign_backward(Kl, mu_, Db), dist)
    kw, _ = oracle.sign_backward(m, dbar.cpu().numpy(), 0.0)
    assert float(np.max(np.abs(kbar.cpu().numpy() - kw))) <= 1e-9 * float(np.max(np.abs(kw)))
    bplan.close()
