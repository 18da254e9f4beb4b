"""Sharding the submatrix method over ranks (one process per GPU).

Submatrices are independent (Section III-A), so ranks split the block columns
into contiguous chunks, balanced on the O(n_j^3) cost of their submatrices
(the greedy of Section IV-E: fill a rank until its load reaches
total / nranks, every rank gets at least one column).  Contiguous chunks keep
neighbouring columns -- which share most blocks -- on one rank (Section IV-B2).

Data movement, once per pattern and per K (Section IV-B1: every block goes
once to each rank that needs it):
  * a rank owns the K blocks of the block rows of its chunk;
  * it needs the blocks of every submatrix it evaluates: the halo;
  * one all-to-all moves the halo blocks; assembly is then local.
D's block columns are disjoint across ranks (no reduction).  The trace and
the electron count of the mu search are a sum-allreduce of one double; the
adjoint's Kbar contributions overlap and are sum-reduced.

The local evaluation is a ``Plan`` with ``columns=(lo, hi)``; tests may pass
any callable with the same contract.
"""
from __future__ import annotations

import numpy as np


def partition_columns(dims, nranks):
    """Contiguous chunks [lo, hi) of block columns, balanced on sum n_j^3."""
    dims = np.asarray(dims, dtype=np.float64)
    nblk = len(dims)
    if nranks < 1 or nranks > nblk:
        raise ValueError("need 1 <= nranks <= number of block columns")
    cost = dims ** 3
    target = cost.sum() / nranks
    bounds = [0]
    load = 0.0
    for j in range(nblk):
        left_cols = nblk - j
        left_ranks = nranks - len(bounds)
        # close the current chunk when it reached its share, or when every
        # remaining rank still needs one column
        if len(bounds) < nranks and j > bounds[-1] and (load >= target or left_cols <= left_ranks):
            bounds.append(j)
            load = 0.0
        load += cost[j]
    bounds.append(nblk)
    return [(bounds[r], bounds[r + 1]) for r in range(nranks)]


def submatrix_dims(block_sizes, row_ptr, col_idx):
    bs = np.asarray(block_sizes, dtype=np.int64)
    return np.array([bs[col_idx[row_ptr[j]:row_ptr[j + 1]]].sum() for j in range(len(bs))])


def owned_blocks(row_ptr, chunk):
    """CSR positions of the blocks in the block rows of the chunk."""
    lo, hi = chunk
    return np.arange(row_ptr[lo], row_ptr[hi], dtype=np.int64)


def halo_blocks(row_ptr, col_idx, chunk):
    """CSR positions of every stored block inside N(j) x N(j) for j in the chunk
    (what the chunk's submatrices are assembled from), sorted."""
    lo, hi = chunk
    need = set()
    for j in range(lo, hi):
        nbr = col_idx[row_ptr[j]:row_ptr[j + 1]]
        nset = set(int(x) for x in nbr)
        for i in nbr:
            for p in range(int(row_ptr[i]), int(row_ptr[i + 1])):
                if int(col_idx[p]) in nset:
                    need.add(p)
    return np.array(sorted(need), dtype=np.int64)


def block_value_ranges(block_sizes, row_ptr, col_idx):
    """value offset of each CSR block (length nnzb + 1)."""
    bs = np.asarray(block_sizes, dtype=np.int64)
    rows = np.repeat(np.arange(len(bs)), np.diff(row_ptr))
    area = bs[rows] * bs[np.asarray(col_idx)]
    vp = np.zeros(len(area) + 1, dtype=np.int64)
    np.cumsum(area, out=vp[1:])
    return vp


class ShardedPattern:
    """Per-rank view of one pattern: chunk, owned blocks, halo, exchange lists."""

    def __init__(self, block_sizes, row_ptr, col_idx, rank, nranks):
        self.block_sizes = np.asarray(block_sizes, dtype=np.int32)
        self.row_ptr = np.asarray(row_ptr, dtype=np.int64)
        self.col_idx = np.asarray(col_idx, dtype=np.int32)
        self.rank, self.nranks = rank, nranks
        dims = submatrix_dims(self.block_sizes, self.row_ptr, self.col_idx)
        self.chunks = partition_columns(dims, nranks)
        self.chunk = self.chunks[rank]
        self.vp = block_value_ranges(self.block_sizes, self.row_ptr, self.col_idx)
        # owner of every block = the rank whose chunk holds its block row
        rows = np.repeat(np.arange(len(self.block_sizes)), np.diff(self.row_ptr))
        bounds = np.array([c[0] for c in self.chunks] + [len(self.block_sizes)])
        self.owner = np.searchsorted(bounds, rows, side="right") - 1
        self.halo = halo_blocks(self.row_ptr, self.col_idx, self.chunk)
        # what this rank receives from each peer, and sends to each peer
        self.recv = [self.halo[self.owner[self.halo] == r] for r in range(nranks)]
        self.send = None  # filled by exchange_lists()

    def exchange_lists(self, dist):
        """Tell every owner which of its blocks this rank needs (one object
        all-gather of index lists, once per pattern)."""
        want = [self.recv[r].tolist() for r in range(self.nranks)]
        every = [None] * self.nranks
        dist.all_gather_object(every, want)
        # every[q][r]: blocks rank q needs from rank r; we send every[q][self.rank]
        self.send = [np.asarray(every[q][self.rank], dtype=np.int64) for q in range(self.nranks)]
        return self.send

    def gather_values(self, vals, blocks):
        if len(blocks) == 0:
            return np.zeros(0)
        return np.concatenate([vals[self.vp[p]:self.vp[p + 1]] for p in blocks])

    def scatter_values(self, out, blocks, flat):
        o = 0
        for p in blocks:
            a, b = self.vp[p], self.vp[p + 1]
            out[a:b] = flat[o:o + (b - a)]
            o += b - a


def exchange_halo(sp, owned_vals, dist):
    """All-to-all of halo blocks.  ``owned_vals`` is a full-length value array
    holding this rank's owned blocks (other entries ignored).  Returns a
    full-length array holding every block this rank needs."""
    import torch
    if sp.send is None:
        sp.exchange_lists(dist)
    send = [torch.from_numpy(sp.gather_values(owned_vals, sp.send[q])) for q in range(sp.nranks)]
    sizes = [int(sum(sp.vp[p + 1] - sp.vp[p] for p in sp.recv[q])) for q in range(sp.nranks)]
    recv = [torch.empty(sizes[q], dtype=torch.float64) for q in range(sp.nranks)]
    # point-to-point pairs (works on gloo and NCCL alike)
    reqs = []
    for q in range(sp.nranks):
        if q == sp.rank:
            recv[q].copy_(send[q])
            continue
        reqs.append(dist.isend(send[q].contiguous(), q))
        reqs.append(dist.irecv(recv[q], q))
    for rq in reqs:
        rq.wait()
    local = np.zeros_like(owned_vals)
    for q in range(sp.nranks):
        sp.scatter_values(local, sp.recv[q], recv[q].numpy())
    return local


def sharded_density(sp, owned_vals, mu, solve, dist):
    """This rank's block columns of D and the global trace.

    ``solve(local_vals, mu, chunk) -> D values`` evaluates the chunk's block
    columns (a column-range Plan on the GPU).  Returns (D values holding this
    rank's block columns, Tr D summed over ranks)."""
    import torch
    local = exchange_halo(sp, owned_vals, dist)
    d = solve(local, mu, sp.chunk)
    tr = 0.0
    for j in range(*sp.chunk):
        p = int(np.searchsorted(sp.col_idx[sp.row_ptr[j]:sp.row_ptr[j + 1]], j)) + int(sp.row_ptr[j])
        b = int(sp.block_sizes[j])
        tr += float(np.trace(d[sp.vp[p]:sp.vp[p + 1]].reshape(b, b)))
    t = torch.tensor([tr], dtype=torch.float64)
    dist.all_reduce(t)
    return d, float(t.item())


def gather_columns(sp, d_local, dist):
    """Allgather of the block columns of D (optional: D replicated).  The
    blocks of block column j are the CSR positions whose column index is j."""
    import torch
    mine = np.nonzero((sp.col_idx >= sp.chunk[0]) & (sp.col_idx < sp.chunk[1]))[0]
    flat = torch.from_numpy(sp.gather_values(d_local, mine))
    sizes = [None] * sp.nranks
    dist.all_gather_object(sizes, int(flat.numel()))
    bufs = [torch.empty(s, dtype=torch.float64) for s in sizes]
    _all_gather_uneven(bufs, flat, dist)
    out = np.zeros_like(d_local)
    for q in range(sp.nranks):
        lo, hi = sp.chunks[q]
        blocks = np.nonzero((sp.col_idx >= lo) & (sp.col_idx < hi))[0]
        sp.scatter_values(out, blocks, bufs[q].numpy())
    return out


def _all_gather_uneven(bufs, flat, dist):
    import torch
    n = max(b.numel() for b in bufs)
    pad = torch.zeros(n, dtype=flat.dtype)
    pad[:flat.numel()] = flat
    tmp = [torch.empty(n, dtype=flat.dtype) for _ in bufs]
    dist.all_gather(tmp, pad)
    for b, t in zip(bufs, tmp):
        b.copy_(t[:b.numel()])


def gpu_solver(pattern, device=None, **plan_kwargs):
    """A ``solve`` for ``sharded_density``: a column-range Plan on this rank's
    GPU (created on first use, reused for later calls with the same chunk)."""
    import torch
    from .submat import Plan
    cache = {}

    def solve(local_vals, mu, chunk):
        if chunk not in cache:
            cache[chunk] = Plan(pattern.block_sizes, pattern.row_ptr, pattern.col_idx,
                                columns=chunk, **plan_kwargs)
        K = torch.from_numpy(np.ascontiguousarray(local_vals)).to(device or "cuda")
        D = torch.zeros_like(K)
        cache[chunk].sign(K, mu, out=D)
        return D.cpu().numpy()

    return solve
