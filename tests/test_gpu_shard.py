"""The column-range plans behind each rank's chunk (the multi-GPU partition)
reassemble the single-plan result, each fed only its halo blocks."""
import numpy as np
import pytest

from paper_2004_10811_gb300.shard import ShardedPattern, gpu_solver
from synth.water import make_water

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed", 1e-10)])
def test_chunks_with_halo_only_reassemble_the_full_result(prec, tol):
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2004_10811_gb300 as pkg
    m = make_water(96, 5, 6.5, (2, -1.0, -0.3), (3, 0.3, 1.2), seed=77)
    with pkg.Plan.from_bsr(m, prec=prec) as plan:
        full = plan.sign(torch.from_numpy(m.vals).cuda(), 0.0).cpu().numpy()
    world = 3
    got = np.zeros_like(full)
    for rank in range(world):
        sp = ShardedPattern(m.block_sizes, m.row_ptr, m.col_idx, rank, world)
        halo_only = np.zeros_like(m.vals)
        sp.scatter_values(halo_only, sp.halo, sp.gather_values(m.vals, sp.halo))
        d = gpu_solver(sp, prec=prec)(halo_only, 0.0, sp.chunk)
        mine = np.nonzero((sp.col_idx >= sp.chunk[0]) & (sp.col_idx < sp.chunk[1]))[0]
        sp.scatter_values(got, mine, sp.gather_values(d, mine))
    assert np.max(np.abs(got - full)) <= tol
