"""The multi-GPU paths are covered on CPU with two gloo ranks: the timing
aggregation bench.py uses under torchrun, and the distributed search of §3.4
(a contiguous partition per rank, an index per partition, one all-gather of
the ranks' k-NN lists; the merge kernel itself is checked on a GPU in
test_gpu_merge.py)."""

import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r answered its queries in (10 + 5r) ms and its steps took (100 + r) ms
    value, q_sum, tot = bench.weak_scaling_value(world, 3, 1000, 10.0 + 5.0 * rank,
                                                 100.0 + rank, "cpu")
    q.put((rank, value, q_sum, tot))
    dist.destroy_process_group()


def test_weak_scaling_aggregation_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, q_sum, tot in out:
        assert q_sum == 15.0 and tot == 101.0          # the slowest rank decides
        assert value == pytest.approx(2 * 3 * 1000 / 0.015)


# ----------------------------------------- the distributed search (§3.4)

def _search_rank(rank, world, port, q):
    """One rank: its contiguous partition of the points, an index over it
    (the oracle stands in for the GPU search on CPU ranks) probed everywhere,
    then the exchange step of dist.py (all-gather of the [nq x k] lists and
    of the ranks' first global ids)."""
    import sys
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle as O
    from paper_2208_02734_gb300 import dist as D
    from paper_2208_02734_gb300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mix = synth.IsotropicMixture(d=8, n_blobs=5, seed=0)
    X = mix.sample(1203, seed=0)
    Q = mix.sample(40, seed=1)                      # the same batch on every rank
    start, stop = D.partition_range(len(X), world, rank)
    idx = O.build(X[start:stop], [30, 4], 5, seed=rank)
    ids, dists, _ = idx.query(Q, 7, idx.k_per_level)   # every probe: exact within the partition
    all_ids, all_d = D.gather_results(torch.from_numpy(ids), torch.from_numpy(dists))
    offs = D.gather_offsets(start, "cpu")
    q.put((rank, all_ids.numpy(), all_d.numpy(), offs.numpy(), start, stop))
    dist.destroy_process_group()


def test_partitioned_search_gathers_what_the_exact_union_needs():
    import numpy as np
    import oracle as O
    from paper_2208_02734_gb300 import dist as D
    from paper_2208_02734_gb300 import synth
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_search_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    out = sorted((q.get(timeout=10) for _ in range(world)), key=lambda t: t[0])
    mix = synth.IsotropicMixture(d=8, n_blobs=5, seed=0)
    X = mix.sample(1203, seed=0)
    Q = mix.sample(40, seed=1)
    # partitions tile the points
    assert [(o[4], o[5]) for o in out] == [D.partition_range(1203, 2, r) for r in range(2)]
    assert out[0][5] == out[1][4] and out[1][5] == 1203
    for rank, all_ids, all_d, offs, _, _ in out:
        assert all_ids.shape == (world, 40, 7)
        assert offs.tolist() == [0, out[1][4]]
        assert np.array_equal(all_ids, out[0][1]) and np.array_equal(all_d, out[0][2])
    # the k smallest (distance, global id) of the gathered lists are the
    # exact k-NN over the union (what mask_merge_topk computes on a GPU)
    all_ids, all_d, offs = out[0][1], out[0][2], out[0][3]
    gid = np.where(all_ids >= 0, all_ids + offs[:, None, None], -1)
    gt_ids, gt_d = O.bruteforce_knn(X, Q, 7)
    for qi in range(40):
        cand_i, cand_d = gid[:, qi, :].reshape(-1), all_d[:, qi, :].reshape(-1)
        order = np.lexsort((cand_i, cand_d))[:7]
        assert cand_i[order].tolist() == gt_ids[qi].tolist()
        assert np.allclose(cand_d[order], gt_d[qi])


def test_partition_ranges():
    from paper_2208_02734_gb300 import dist as D
    for n, world in [(10, 3), (1203, 2), (7, 7), (5, 8)]:
        ranges = [D.partition_range(n, world, r) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
        sizes = [b - a for a, b in ranges]
        assert max(sizes) - min(sizes) <= 1
