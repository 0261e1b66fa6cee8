"""The serving loop (continuous batching over a resident index).

The central property: a request's answer is the same alone (mask_query on its
queries) and in any mix of concurrent requests, bit for bit, in every
precision -- each query's result depends only on the query.  Also: memory-
based admission keeps the estimated bytes in flight within the budget,
oversize requests are split, errors are reported per request, and close()
finishes queued work.
"""

import threading

import numpy as np
import pytest

from paper_2208_02734_gb300 import mask as M
from paper_2208_02734_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def c1_index():
    mix = synth.IsotropicMixture(d=16, n_blobs=10, sigma=1.0, box=10.0, seed=0)
    X = mix.sample(20_000, seed=0)
    Q = mix.sample(6_000, seed=1)
    idx = M.mask_build(torch.from_numpy(X).cuda(), [200, 20], 20, seed=0)
    yield X, Q, idx
    idx.free()


def mixed_requests(Q, n_req, seed, precisions=(M.MASK_FP32, M.MASK_BF16, M.MASK_FP8E4M3), P=3):
    """Requests shaped like the serving workload: batch ~ U[1, 512], k in
    {1, 10, 100}, probes ~ U{P..P+2} x U{3..5}, mixed precision (k <= 16 for
    the low-precision modes)."""
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(n_req):
        nq = int(rng.integers(1, 513))
        q0 = int(rng.integers(0, len(Q) - nq))
        prec = int(rng.choice(precisions))
        k = int(rng.choice([1, 10, 100] if prec == M.MASK_FP32 else [1, 10, 16]))
        probes = [int(rng.integers(P, P + 3)), int(rng.integers(3, 6))]
        reqs.append((Q[q0:q0 + nq], k, probes, prec))
    return reqs


def alone(idx, req):
    Qr, k, probes, prec = req
    ids, d = M.mask_query(idx, torch.from_numpy(np.ascontiguousarray(Qr)).cuda(), k, probes,
                          precision=prec)
    return ids.cpu().numpy(), d.cpu().numpy()


@pytest.mark.parametrize("P", [3, 12, 40])
def test_results_are_the_same_alone_and_in_the_mix(c1_index, P):
    # P >= 12: some queries keep fewer leaf clusters than probed (absent slots)
    X, Q, idx = c1_index
    reqs = mixed_requests(Q, 120, seed=P, P=P)
    want = [alone(idx, r) for r in reqs]
    with M.Server(idx, mem_budget=256 << 20, max_slots=4, max_batch=1024) as srv:
        tickets = [None] * len(reqs)

        def client(c):
            for i in range(c, len(reqs), 4):
                Qr, k, probes, prec = reqs[i]
                tickets[i] = srv.submit(Qr, k, probes, prec)

        th = [threading.Thread(target=client, args=(c,)) for c in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for i, t in enumerate(tickets):
            ids, d = t.result(timeout_ms=60_000)
            assert np.array_equal(ids, want[i][0]), i
            assert np.array_equal(d, want[i][1]), i
        st = srv.stats()
    assert st["requests_done"] == len(reqs) and st["requests_failed"] == 0
    assert st["queries_done"] == sum(len(r[0]) for r in reqs)
    assert st["batches"] < len(reqs)              # concurrent requests were merged
    assert st["graph_captures"] >= 1 and st["autotuned_shapes"] >= 1
    assert 0 < st["latency_p50_ms"] <= st["latency_p99_ms"] <= st["latency_max_ms"]
    assert st["peak_inflight_bytes"] <= 256 << 20


def test_memory_budget_bounds_the_work_in_flight(c1_index):
    X, Q, idx = c1_index
    budget = 3 << 20                               # a few small batches at a time
    reqs = mixed_requests(Q, 40, seed=1, precisions=(M.MASK_FP32,))
    reqs.append((Q[:3000], 10, [3, 3], M.MASK_FP32))   # larger than one batch: split
    want = [alone(idx, r) for r in reqs]
    with M.Server(idx, mem_budget=budget, max_slots=8, max_batch=4096) as srv:
        tickets = [srv.submit(*r) for r in reqs]
        for i, t in enumerate(tickets):
            ids, d = t.result(timeout_ms=60_000)
            assert np.array_equal(ids, want[i][0]) and np.array_equal(d, want[i][1]), i
        st = srv.stats()
    assert 0 < st["peak_inflight_bytes"] <= budget
    assert st["batches"] >= 2


def test_request_too_large_for_the_budget_fails_alone(c1_index):
    X, Q, idx = c1_index
    with M.Server(idx, mem_budget=64 << 10, max_slots=2, max_batch=64) as srv:
        t = srv.submit(Q[:10], 10, [3, 3])
        with pytest.raises(M.MaskError, match="MASK_ENOMEM"):
            t.result(timeout_ms=30_000)
        assert srv.stats()["requests_failed"] == 1


def test_submit_rejects_bad_requests(c1_index):
    X, Q, idx = c1_index
    with M.Server(idx, mem_budget=64 << 20) as srv:
        with pytest.raises(M.MaskError, match="MASK_EUNSUPPORTED"):
            srv.submit(Q[:4], 100, [3, 3], M.MASK_BF16)      # shortlist of 400 > 64
        with pytest.raises(M.MaskError, match="MASK_EINVAL"):
            srv.submit(Q[:4], 0, [3, 3])
        with pytest.raises(M.MaskError, match="MASK_EINVAL"):
            srv.submit(Q[:4], 5, [0, 3])
        t = srv.submit(Q[:0], 5, [3, 3])                     # empty request: done at once
        ids, _ = t.result(timeout_ms=1000)
        assert ids.shape == (0, 5)


def test_close_finishes_queued_requests(c1_index):
    X, Q, idx = c1_index
    reqs = mixed_requests(Q, 30, seed=2, precisions=(M.MASK_FP32,))
    want = [alone(idx, r) for r in reqs]
    srv = M.Server(idx, mem_budget=64 << 20, max_slots=2, max_batch=256)
    tickets = [srv.submit(*r) for r in reqs]
    srv.close()                                              # drains the queue
    for i, t in enumerate(tickets):
        assert np.array_equal(t.ids, want[i][0]) and np.array_equal(t.dists, want[i][1]), i


def test_server_refuses_a_sparse_index():
    A = synth.sparse_tfidf_like(500, 100, nnz_mean=5.0, seed=0)
    idx = M.mask_build_csr(A.row_ptr, A.col, A.val, 100, [8], 2, seed=0)
    with pytest.raises(M.MaskError, match="dense"):
        M.Server(idx, mem_budget=1 << 20)
    idx.free()
