"""Sharding the submatrix method over ranks (one process per GPU).

Submatrices are independent (Section III-A), so ranks split the block columns
into contiguous chunks, balanced on the O(n_j^3) cost of their submatrices
(the greedy of Section IV-E: fill a rank until its load reaches
total / nranks, every rank gets at least one column).  Contiguous chunks keep
neighbouring columns -- which share most blocks -- on one rank (Section IV-B2).

Data movement (Section IV-B1: every block goes once to each rank that needs it):
  * a rank owns the K blocks of the block rows of its chunk;
  * it needs the blocks of every submatrix it evaluates: the halo;
  * one exchange of point-to-point messages moves the halo blocks, once per
    K; assembly is then local.
Everything lives in device memory on the rank's GPU: the value index lists
are built once per pattern, halo values are packed and unpacked on the
device, and the messages are device tensors (NCCL; gloo ranks use the same
code with CPU tensors).  D's block columns are disjoint across ranks (no
reduction); Tr D and the mu search's electron count (and dN/dmu at finite
temperature) are sum-allreduces of scalars; the adjoint's Kbar contributions
overlap and are sum-reduced in place.

The local evaluation is a ``Plan`` with ``columns=(lo, hi)``
(``gpu_solver``); tests may pass any callable with the same contract.
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


def value_index(vp, blocks):
    """Flat value positions of the given CSR blocks, in block order."""
    if len(blocks) == 0:
        return np.zeros(0, dtype=np.int64)
    return np.concatenate([np.arange(vp[p], vp[p + 1], dtype=np.int64) for p in blocks])


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
        self.nvals = int(self.vp[-1])
        # owner of every block = the rank whose chunk holds its block row
        rows = np.repeat(np.arange(len(self.block_sizes)), np.diff(self.row_ptr))
        bounds = np.array([c[0] for c in self.chunks] + [len(self.block_sizes)])
        self.owner = np.searchsorted(bounds, rows, side="right") - 1
        self.halo = halo_blocks(self.row_ptr, self.col_idx, self.chunk)
        # what this rank receives from each peer, and sends to each peer
        self.recv = [self.halo[self.owner[self.halo] == r] for r in range(nranks)]
        self.send = None  # filled by exchange_lists()
        # this rank's block columns of D (flat value positions)
        self.mine = np.nonzero((self.col_idx >= self.chunk[0]) & (self.col_idx < self.chunk[1]))[0]
        self._dev = {}

    def exchange_lists(self, dist):
        """Tell every owner which of its blocks this rank needs (one object
        all-gather of index lists, once per pattern)."""
        want = [self.recv[r].tolist() for r in range(self.nranks)]
        every = [None] * self.nranks
        dist.all_gather_object(every, want)
        # every[q][r]: blocks rank q needs from rank r; we send every[q][self.rank]
        self.send = [np.asarray(every[q][self.rank], dtype=np.int64) for q in range(self.nranks)]
        return self.send

    def device_index(self, device, dist=None):
        """Flat value positions, as int64 tensors on `device`, of what goes to
        and comes from every peer (built once per pattern and device)."""
        import torch
        key = str(device)
        if key not in self._dev:
            if self.send is None:
                self.exchange_lists(dist)
            t = lambda a: torch.from_numpy(a).to(device)
            self._dev[key] = {
                "send": [t(value_index(self.vp, self.send[q])) for q in range(self.nranks)],
                "recv": [t(value_index(self.vp, self.recv[q])) for q in range(self.nranks)],
                "mine": t(value_index(self.vp, self.mine)),
            }
        return self._dev[key]

    # host helpers (tests, and callers that hold NumPy arrays)
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


def exchange_halo(sp, K_local, dist):
    """Moves the halo blocks between ranks, in place: ``K_local`` (a
    full-length float64 tensor on this rank's device: its owned blocks filled,
    the rest anything) receives every block this rank's submatrices need.
    Packing and unpacking run on the device; the messages are batched
    point-to-point sends and receives (NCCL with CUDA tensors, gloo with CPU
    tensors).  Returns K_local."""
    import torch
    idx = sp.device_index(K_local.device, dist)
    sends = [K_local.index_select(0, idx["send"][q]) for q in range(sp.nranks)]
    recvs = [torch.empty(idx["recv"][q].numel(), dtype=K_local.dtype, device=K_local.device)
             for q in range(sp.nranks)]
    ops = []
    for q in range(sp.nranks):
        if q == sp.rank:
            recvs[q].copy_(sends[q])
            continue
        if sends[q].numel():
            ops.append(dist.P2POp(dist.isend, sends[q], q))
        if recvs[q].numel():
            ops.append(dist.P2POp(dist.irecv, recvs[q], q))
    if ops:
        for rq in dist.batch_isend_irecv(ops):
            rq.wait()
    for q in range(sp.nranks):
        if recvs[q].numel():
            K_local.index_copy_(0, idx["recv"][q], recvs[q])
    return K_local


def allreduce_sum(values, device, dist):
    """Sum of a few doubles over ranks, as one device allreduce."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t)
    return t.tolist()


def sharded_density(sp, K_local, mu, solve, dist, exchange=True):
    """This rank's block columns of D and the global trace.

    ``solve(K_local, mu, chunk) -> (D, tr)`` evaluates the chunk's block
    columns on this rank's device (D a full-length tensor, zero outside the
    chunk; tr the trace over the chunk).  Returns (D, Tr D summed over
    ranks)."""
    if exchange:
        exchange_halo(sp, K_local, dist)
    d, tr = solve(K_local, mu, sp.chunk)
    (total,) = allreduce_sum([tr], K_local.device, dist)
    return d, total


def sharded_mu_search(sp, K_local, n_el, mu0, solve, dist, tol=1e-9, max_steps=60, bound=None, kT=0.0,
                      dn_dmu=None):
    """mu with Tr D(mu) = n_el over all ranks (Section IV-G): every trial mu is
    evaluated on every rank's chunk and the electron count (and dN/dmu at
    finite temperature) is sum-allreduced, so all ranks take the same steps.
    Zero temperature: bisection on [mu0 - s, mu0 + s] on the side of n_el
    (s = 1.01 bound + 1e-12); finite temperature: Newton steps kept inside
    that bracket, bisection otherwise.  ``bound``: a spectral bound of the
    submatrices at mu0 (max over ranks is taken); ``dn_dmu()``: this rank's
    dN/dmu of the last evaluation.  Returns (mu, D, N, steps)."""
    exchange_halo(sp, K_local, dist)
    dev = K_local.device
    steps = 0

    def evaluate(mu):
        nonlocal steps
        d, tr = solve(K_local, mu, sp.chunk)
        vals = [tr, dn_dmu() if (kT > 0 and dn_dmu) else 0.0]
        n, dn = allreduce_sum(vals, dev, dist)
        steps += 1
        return d, n, dn

    d, n, dn = evaluate(mu0)
    mu = mu0
    if abs(n - n_el) <= tol * abs(n_el):
        return mu, d, n, steps
    (b,) = allreduce_sum([bound or 0.0], dev, dist)
    span = 1.01 * b + 1e-12 + (40.0 * kT if kT > 0 else 0.0)
    lo, hi = (mu0, mu0 + span) if n < n_el else (mu0 - span, mu0)
    while steps < max_steps and hi - lo > 1e-10 * max(b, 1e-300):
        nxt = 0.5 * (lo + hi)
        if kT > 0 and dn > 0:
            newton = mu - (n - n_el) / dn
            if lo < newton < hi:
                nxt = newton
        mu = nxt
        d, n, dn = evaluate(mu)
        if abs(n - n_el) <= tol * abs(n_el):
            break
        if n < n_el:
            lo = mu
        else:
            hi = mu
    return mu, d, n, steps


def sharded_backward(sp, K_local, mu, Dbar_local, backward, dist):
    """Kbar over all ranks: each rank adds the contributions of its chunk's
    submatrices (``backward(K_local, mu, Dbar, chunk) -> Kbar`` on the
    device), then one in-place sum-allreduce of the full-length Kbar (the
    contributions overlap on shared blocks).  ``Dbar_local`` must hold this
    rank's block columns of Dbar."""
    kbar = backward(K_local, mu, Dbar_local, sp.chunk)
    dist.all_reduce(kbar)
    return kbar


def gather_columns(sp, d_local, dist):
    """Allgather of the block columns of D on the device (optional: D
    replicated).  The blocks of block column j are the CSR positions whose
    column index is j."""
    import torch
    idx = sp.device_index(d_local.device, dist)
    flat = d_local.index_select(0, idx["mine"])
    sizes = [int(x) for x in allreduce_sizes(sp, flat.numel(), d_local.device, dist)]
    n = max(sizes)
    pad = torch.zeros(n, dtype=flat.dtype, device=flat.device)
    pad[:flat.numel()] = flat
    tmp = [torch.empty(n, dtype=flat.dtype, device=flat.device) for _ in range(sp.nranks)]
    dist.all_gather(tmp, pad)
    out = d_local.clone()
    for q in range(sp.nranks):
        lo, hi = sp.chunks[q]
        blocks = np.nonzero((sp.col_idx >= lo) & (sp.col_idx < hi))[0]
        pos = torch.from_numpy(value_index(sp.vp, blocks)).to(d_local.device)
        out.index_copy_(0, pos, tmp[q][:sizes[q]])
    return out


def allreduce_sizes(sp, mine, device, dist):
    """Every rank's element count, as one device allreduce of a one-hot vector."""
    import torch
    t = torch.zeros(sp.nranks, dtype=torch.float64, device=device)
    t[sp.rank] = float(mine)
    dist.all_reduce(t)
    return t.tolist()


def gpu_solver(pattern, device=None, **plan_kwargs):
    """A ``solve`` for ``sharded_density``: a column-range Plan on this rank's
    GPU (created on first use, reused for later calls with the same chunk).
    Takes and returns device tensors; D is a full-length tensor zero outside
    the chunk, and the trace is the chunk's."""
    import torch
    from .submat import Plan
    cache = {}

    def plan_for(chunk):
        if chunk not in cache:
            cache[chunk] = Plan(pattern.block_sizes, pattern.row_ptr, pattern.col_idx, columns=chunk,
                                **plan_kwargs)
        return cache[chunk]

    def solve(K_local, mu, chunk):
        plan = plan_for(chunk)
        D = torch.zeros_like(K_local)
        plan.sign(K_local, mu, out=D)
        return D, plan.trace(D)

    solve.plan_for = plan_for
    return solve
