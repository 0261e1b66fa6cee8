"""Distributed search over partitioned indexes (§3.4 of the paper).

Each node (one process per GPU) holds one partition of the points and builds
its own index over it, with no exchange during the build.  A query batch goes
to every node; each answers it on its own partition, and one exchange step
gathers the nodes' k-NN lists so that every query keeps the k nearest over all
partitions (the merge runs in the library's kernel, ``mask_merge_topk``).

Only collective plumbing lives here (torch.distributed: NCCL between GPUs,
gloo on CPU); the search and the merge are library calls.
"""

from __future__ import annotations

from . import mask as M


def partition_range(n: int, world: int, rank: int):
    """Contiguous partition [start, stop) of n items for `rank` of `world`:
    sizes differ by at most one, the first n % world ranks one larger."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def gather_results(ids, dists, group=None):
    """All-gather each rank's [nq x k] (ids, dists) into [world x nq x k]
    tensors on every rank (in rank order)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    all_ids = [torch.empty_like(ids) for _ in range(world)]
    all_d = [torch.empty_like(dists) for _ in range(world)]
    dist.all_gather(all_ids, ids.contiguous(), group=group)
    dist.all_gather(all_d, dists.contiguous(), group=group)
    return torch.stack(all_ids), torch.stack(all_d)


def gather_offsets(id_offset: int, device, group=None):
    """Every rank's first global id, in rank order ([world] int64 tensor)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    mine = torch.tensor([int(id_offset)], dtype=torch.int64, device=device)
    allo = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(allo, mine, group=group)
    return torch.cat(allo)


def query_partitioned(index, queries, k: int, probes, id_offset: int,
                      precision: int = M.MASK_FP32, group=None):
    """k-NN of `queries` (the same batch on every rank) over the union of all
    ranks' partitions: the local search, one all-gather of the [nq x k]
    lists, the merge.  `id_offset` is this rank's first global point id.
    Returns global (ids, dists) [nq x k] on every rank."""
    ids, dists = M.mask_query(index, queries, k, probes, precision)
    all_ids, all_d = gather_results(ids, dists, group)
    offs = gather_offsets(id_offset, all_ids.device, group)
    return M.mask_merge_topk(all_ids, all_d, offs)
