"""Multi-rank path on CPU: gloo ranks (world size 2 and 3) run the partition,
the halo exchange, the per-rank evaluation, the trace and electron-count
allreduces, the finite-temperature mu search and the Kbar reduction, through
the same functions the GPU ranks use (CPU tensors here).  The per-rank solver
is the CPU oracle (test infrastructure standing in for the GPU plan), so the
results must equal the single-process oracle's."""
import os
import socket

import numpy as np
import pytest

from paper_2004_10811_gb300.shard import (ShardedPattern, exchange_halo, gather_columns, halo_blocks,
                                          partition_columns, sharded_backward, sharded_density,
                                          sharded_mu_search, submatrix_dims)
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


def _worker(rank, world, port, case, out, mode="density"):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = case()
    sp = ShardedPattern(m.block_sizes, m.row_ptr, m.col_idx, rank, world)
    # each rank starts with only the blocks of its own block rows
    owned = np.zeros_like(m.vals)
    vp = sp.vp
    for p in np.nonzero(sp.owner == rank)[0]:
        owned[vp[p]:vp[p + 1]] = m.vals[vp[p]:vp[p + 1]]
    K_local = torch.from_numpy(owned)
    kT = 0.05
    chunk_cols = list(range(*sp.chunk))

    def chunk_trace(d):
        tr = 0.0
        for j in chunk_cols:
            p = int(np.searchsorted(m.col_idx[m.row_ptr[j]:m.row_ptr[j + 1]], j)) + int(m.row_ptr[j])
            b = int(m.block_sizes[j])
            tr += float(np.trace(d[vp[p]:vp[p + 1]].reshape(b, b)))
        return tr

    last = {}

    def solve(K, mu, chunk):
        # the oracle on the values this rank holds (owned + exchanged halo)
        mm = m.with_vals(K.numpy())
        if mode == "mu_T":
            d = oracle.density_matrix_T(mm, mu, kT, columns=chunk_cols)
        else:
            d = oracle.density_matrix(mm, mu, columns=chunk_cols)
        d = np.nan_to_num(d, nan=0.0)
        last["d"] = d
        return torch.from_numpy(d), chunk_trace(d)

    def dn_dmu():
        # sum over the chunk's columns c of (F_cc - sum_k F_kc^2) / kT
        d = last["d"]
        sq = sum(float(np.sum(d[vp[p]:vp[p + 1]] ** 2)) for p in sp.mine)
        return (chunk_trace(d) - sq) / kT

    if mode == "density":
        d_local, tr = sharded_density(sp, K_local, m.mu, solve, dist)
        d_all = gather_columns(sp, d_local, dist)
        result = (d_all.numpy(), tr)
    elif mode == "mu_T":
        mu, d_local, n, steps = sharded_mu_search(sp, K_local, m.n_el, 0.4, solve, dist, tol=1e-12,
                                                  max_steps=60, bound=4.0, kT=kT, dn_dmu=dn_dmu)
        result = (gather_columns(sp, d_local, dist).numpy(), (mu, n, steps))
    else:  # backward
        exchange_halo(sp, K_local, dist)
        dbar = np.random.default_rng(3).standard_normal(m.vals.shape)

        def backward(K, mu, Dbar, chunk):
            kb, _ = oracle.sign_backward(m.with_vals(K.numpy()), Dbar.numpy(), mu, columns=chunk_cols)
            return torch.from_numpy(kb)

        kbar = sharded_backward(sp, K_local, m.mu, torch.from_numpy(dbar), backward, dist)
        result = (kbar.numpy(), None)
    if rank == 0:
        np.save(out, result[0])
        with open(out + ".tr", "w") as f:
            f.write(repr(result[1]))
    dist.barrier()
    dist.destroy_process_group()


def _run(world, case, out, mode):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, out, mode)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0


@pytest.mark.parametrize("world", [2, 3])
def test_two_and_three_gloo_ranks_reproduce_the_single_process_result(tmp_path, world):
    import oracle
    case = small_case
    out = str(tmp_path / "d.npy")
    _run(world, case, out, "density")
    m = case()
    want = oracle.density_matrix(m, m.mu)
    got = np.load(out)
    assert np.array_equal(got, want)
    tr = float(open(out + ".tr").read())
    assert abs(tr - oracle.trace_bsr(m, want)) < 1e-12


def test_finite_temperature_mu_search_over_two_gloo_ranks(tmp_path):
    """The electron count and dN/dmu allreduced over ranks: every rank takes
    the same Newton steps, and the search lands on the single-process
    oracle's root."""
    import oracle
    out = str(tmp_path / "d.npy")
    _run(2, small_case, out, "mu_T")
    m = small_case()
    mu, n, steps = eval(open(out + ".tr").read())
    dec = oracle.decompose_all(m, 0.0)
    mu_o, _n, _s = oracle.mu_search_newton_T(dec, m.n_el, 0.05, -4.0, 4.0, tol=1e-14)
    assert abs(n - m.n_el) <= 1e-12 * m.n_el
    assert abs(mu - mu_o) < 1e-9
    assert steps < 30
    assert np.max(np.abs(np.load(out) - oracle.density_matrix_T(m, mu, 0.05))) < 1e-12


def test_kbar_sum_reduced_over_three_gloo_ranks(tmp_path):
    import oracle
    out = str(tmp_path / "kbar.npy")
    _run(3, small_case, out, "backward")
    m = small_case()
    dbar = np.random.default_rng(3).standard_normal(m.vals.shape)
    want, _ = oracle.sign_backward(m, dbar, m.mu)
    assert np.max(np.abs(np.load(out) - want)) < 1e-12
