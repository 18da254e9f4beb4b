"""Multi-rank path on CPU: world-size-2 gloo ranks run the partition, the halo
exchange, the per-rank evaluation and the trace allreduce.  The per-rank
solver here is the CPU oracle (test infrastructure standing in for the GPU
plan), so the gathered D must equal the single-process oracle D exactly."""
import os
import socket

import numpy as np
import pytest

from paper_2004_10811_gb300.shard import (ShardedPattern, gather_columns, halo_blocks,
                                          partition_columns, sharded_density, submatrix_dims)
from synth import make_config, random_symmetric_bsr, small_case


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_partition_is_contiguous_balanced_and_complete():
    m = make_config(1)
    d = submatrix_dims(m.block_sizes, m.row_ptr, m.col_idx)
    for n in (1, 2, 3, 8, 64):
        ch = partition_columns(d, n)
        assert ch[0][0] == 0 and ch[-1][1] == m.nblk and len(ch) == n
        assert all(a < b for a, b in ch) and all(ch[i][1] == ch[i + 1][0] for i in range(n - 1))
        loads = [float((d[a:b].astype(float) ** 3).sum()) for a, b in ch]
        assert max(loads) <= 1.1 * sum(loads) / n + max(d.astype(float)) ** 3


def test_partition_edge_cases():
    assert partition_columns([5], 1) == [(0, 1)]
    ch = partition_columns([1, 1, 100, 1, 1], 5)
    assert ch == [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5)]
    with pytest.raises(ValueError):
        partition_columns([1, 2], 3)


def test_halo_is_exactly_what_the_submatrices_read():
    import oracle.submatrix as osub
    m = random_symmetric_bsr([2, 3, 1, 4, 2, 3, 2, 2], density=0.4, seed=5)
    struct = osub.column_structure(m)
    lookup = osub._block_lookup(m)
    for chunk in ((0, 3), (3, 8), (2, 5)):
        need = set()
        for j in range(*chunk):
            for r in struct[j]:
                for c in struct[j]:
                    if (int(r), int(c)) in lookup:
                        need.add(lookup[(int(r), int(c))][3])
        assert set(halo_blocks(m.row_ptr, m.col_idx, chunk).tolist()) == need


def _worker(rank, world, port, case, out):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = case()
    sp = ShardedPattern(m.block_sizes, m.row_ptr, m.col_idx, rank, world)
    # each rank starts with only the blocks of its own block rows
    owned = np.zeros_like(m.vals)
    rows = np.repeat(np.arange(m.nblk), np.diff(m.row_ptr))
    vp = sp.vp
    for p in np.nonzero(sp.owner == rank)[0]:
        owned[vp[p]:vp[p + 1]] = m.vals[vp[p]:vp[p + 1]]

    def solve(local_vals, mu, chunk):
        mm = m.with_vals(local_vals)
        d = oracle.density_matrix(mm, mu, columns=list(range(*chunk)))
        return np.nan_to_num(d, nan=0.0)

    d_local, tr = sharded_density(sp, owned, m.mu, solve, dist)
    d_all = gather_columns(sp, d_local, dist)
    if rank == 0:
        np.save(out, d_all)
        with open(out + ".tr", "w") as f:
            f.write(repr(tr))
    dist.barrier()
    dist.destroy_process_group()
    del rows


@pytest.mark.parametrize("world", [2, 3])
def test_two_and_three_gloo_ranks_reproduce_the_single_process_result(tmp_path, world):
    import multiprocessing as mp
    import oracle
    case = small_case
    out = str(tmp_path / "d.npy")
    ctx = mp.get_context("spawn")
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    m = case()
    want = oracle.density_matrix(m, m.mu)
    got = np.load(out)
    assert np.array_equal(got, want)
    tr = float(open(out + ".tr").read())
    assert abs(tr - oracle.trace_bsr(m, want)) < 1e-12
