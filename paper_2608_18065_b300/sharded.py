"""One minSR step (Algorithm 1) with the Ns samples split over the ranks of a
torch.distributed process group.

Samples are independent (exact autoregressive sampling, Sec. II.A), so rank r
of G draws its own range s0 .. s0 + n - 1 of the step's samples with their
own Philox counters, and evaluates their local energies (Sec. II.C) and
log-derivatives O (Sec. II.D) alone.  The steps that couple samples then
need three exchanges:

  1. an allreduce (sum) of the partial sums: the column sums of O per block
     (Np or 2 Np) and sum E_loc, sum |E_loc|^2 (3 doubles) -- the centring
     of O and eps-bar' (Eq. real-valued) and E, Var (Eq. energy);
  2. an allgather of the centred rows O' and of eps-bar' (rank order); every
     rank forms T = O'O'^T, lambda, x = (T + lambda I)^{-1} eps-bar' and eta
     (Eq. minsrR, App. F) from them (the solve is small and replicated);
  3. an allgather of delta theta = eta O'^T x by parameter ranges (rank r
     forms entries p0 .. p1 - 1), after which every rank applies the
     momentum and the update (App. B).

Rows gathered in rank order are a permutation of the single-rank rows, so
T, x and eps-bar' permute alike and delta theta is the single-rank step's up
to rounding.

The arithmetic runs in a backend with the methods forward, center, solve and
apply; ShardBackend drives libnqs (nqs_shard_* of a Context, every stage in
the library's kernels), and the collectives are torch.distributed's on the
backend's tensors (NCCL for device tensors).  Without an initialised process
group the step runs with G = 1.
"""
from dataclasses import dataclass

import torch
import torch.distributed as dist


def partition(total: int, world: int, rank: int):
    """(start, count) of rank's share of `total` items, the first
    total % world ranks one item more."""
    q, r = divmod(int(total), int(world))
    n = q + (1 if rank < r else 0)
    return rank * q + min(rank, r), n


class ShardBackend:
    """The libnqs stages of a sharded step on one context (its device)."""

    def __init__(self, ctx):
        self.ctx = ctx
        self.blocks = ctx.rows_per_sample
        self.np = ctx.np

    def new_stats(self):
        return self.ctx.new_stats()

    def forward(self, theta, hp, t, s0, n):
        return self.ctx.shard_forward(theta, hp, t, s0, n)

    def center(self, sums, ns, n, stats):
        return self.ctx.shard_center(sums, ns, n, stats)

    def solve(self, rows, eps, hp, t, p0, p1, stats):
        return self.ctx.shard_solve(rows, eps, hp, t, p0, p1, stats)

    def apply(self, theta, mom, dtheta, hp, t, stats):
        self.ctx.shard_apply(theta, mom, dtheta, hp, t, stats)


@dataclass
class Group:
    """Rank, size and process group of the step (G = 1 without one)."""
    rank: int = 0
    world: int = 1
    pg: object = None

    @staticmethod
    def current(pg=None):
        if dist.is_available() and dist.is_initialized():
            return Group(dist.get_rank(pg), dist.get_world_size(pg), pg)
        return Group()


def _allgather_rows(g: Group, x, counts, per_row):
    """Concatenation in rank order of every rank's x, whose leading
    dimension is counts[r] * per_row (padded to the largest for the
    collective, which wants equal sizes)."""
    if g.world == 1:
        return x
    rmax = max(counts) * per_row
    pad = torch.zeros((rmax,) + tuple(x.shape[1:]), dtype=x.dtype, device=x.device)
    pad[:x.shape[0]] = x
    outs = [torch.empty_like(pad) for _ in range(g.world)]
    dist.all_gather(outs, pad, group=g.pg)
    return outs


def sharded_step(backend, theta, mom, hp, step_index, stats=None, group: Group = None):
    """One step on this rank's share; theta and mom (every rank's copy)
    updated in place.  Returns the rank's step statistics (identical on
    every rank but for rounding in the solve's status flags)."""
    g = group or Group.current()
    ns = int(hp.ns)
    if stats is None:
        stats = backend.new_stats()
    counts = [partition(ns, g.world, r)[1] for r in range(g.world)]
    s0, n = partition(ns, g.world, g.rank)
    if n < 1:
        raise ValueError("more ranks than samples")
    # 1. local samples, E_loc, O; partial sums; allreduce
    sums = backend.forward(theta, hp, step_index, s0, n)
    if g.world > 1:
        dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=g.pg)
    # 2. centred rows and eps-bar'; allgather in rank order, block by block
    rows, eps = backend.center(sums, ns, n, stats)
    nb = backend.blocks
    if g.world > 1:
        rows_all = _allgather_rows(g, rows, counts, nb)
        eps_all = _allgather_rows(g, eps, counts, nb)
        rows = torch.cat([r[:counts[i] * nb] for i, r in enumerate(rows_all)], 0)
        eps = torch.cat([e[:counts[i] * nb] for i, e in enumerate(eps_all)], 0)
    # 3. T, lambda, x, eta; delta theta by parameter ranges; allgather
    p0, npar = partition(backend.np, g.world, g.rank)
    dth = backend.solve(rows, eps, hp, step_index, p0, p0 + npar, stats)
    if g.world > 1:
        pcounts = [partition(backend.np, g.world, r)[1] for r in range(g.world)]
        parts = _allgather_rows(g, dth, pcounts, 1)
        dth = torch.cat([q[:pcounts[i]] for i, q in enumerate(parts)], 0)
    backend.apply(theta, mom, dth, hp, step_index, stats)
    return stats
