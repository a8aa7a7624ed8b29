"""Particles split across the ranks of a torch.distributed group.

The paper parallelises its methods at the level of individual samples (Sec.
3): each particle's misfit gradient (Sec. 4.2, Eq. 26) depends on that
particle alone, so every rank computes the gradients of its own particles
with no communication. The update of Eq. 17 (SVGD) or Eq. 22-25 (sSVGD)
couples all particles through the kernel matrix, so an iteration has one
exchange: the particles and their gradients are all-gathered, every rank
applies the update to the whole ensemble on its own GPU (through the C ABI)
and keeps its rows. The update costs far less than the gradients (about
1/3000 of an iteration on the 120 x 300 workload), so repeating it on every
rank costs nothing measurable and keeps the ranks' ensembles identical
without a second exchange; the sSVGD noise, drawn from Philox keyed by
(seed, iteration, row, column), is the same on every rank.

Backends: NCCL gathers the CUDA tensors in place; gloo gathers host copies
(the multi-process tests run on CPU with gloo).
"""
import torch
import torch.distributed as dist


def rank_rows(n_local, group=None):
    """Row counts of every rank and this rank's first row in the gathered
    ensemble (rank order)."""
    world = dist.get_world_size(group)
    n = torch.tensor([int(n_local)], dtype=torch.int64)
    if dist.get_backend(group) == "nccl":
        n = n.cuda()
    counts = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts, n, group=group)
    counts = [int(c.item()) for c in counts]
    rank = dist.get_rank(group)
    return counts, sum(counts[:rank])


def gather_rows(t, counts, group=None):
    """All ranks' row blocks of t [n_local, ...] stacked in rank order; blocks
    of different sizes are padded to the largest for the collective."""
    world = len(counts)
    nmax = max(counts)
    nccl = dist.get_backend(group) == "nccl"
    src = t if nccl else t.detach().cpu()
    if src.shape[0] < nmax:
        pad = src.new_zeros((nmax - src.shape[0],) + tuple(src.shape[1:]))
        src = torch.cat([src, pad])
    bufs = [torch.empty_like(src) for _ in range(world)]
    dist.all_gather(bufs, src.contiguous(), group=group)
    full = torch.cat([b[:c] for b, c in zip(bufs, counts)])
    return full.to(t.device)


def sharded_update(X_local, G_local, update, group=None):
    """One coupled update of particles split across ranks.

    X_local [n_local, d] this rank's particles (updated in place), G_local
    [n_local, d] their gradients, update(X, G) a function that updates the
    whole ensemble X [n, d] in place, e.g.
        lambda X, G: svgd_step(X, G, eps, lo=lo, hi=hi, gscale=-1.0).
    Returns the gathered ensemble after the update (every rank holds the same
    one)."""
    counts, first = rank_rows(X_local.shape[0], group)
    X = gather_rows(X_local, counts, group)
    G = gather_rows(G_local, counts, group)
    update(X, G)
    X_local.copy_(X[first:first + X_local.shape[0]])
    return X
