"""The tensor-core cluster-major leaf scan (query_cm_tc.cu, rows of 32 or 64
floats) against the per-query scan, the mma.sync cluster-major scan and the
oracle.

Both cluster-major scans keep every row the exact per-query scan would keep
(their expanded-form filters carry proven rounding bounds) and key it with
the same arithmetic, so all three return the same ids and distances bit for
bit; the oracle's descent over the same index agrees up to near-ties.  The cases cover one and several 128-row
chunks per cluster with ragged tails, clusters kept by more than 16 queries
(several work items), items of 32 queries (K <= 16) and of 16 (K up to 32),
fewer queries per item, empty leaf clusters, absent leaf slots, candidate
lists that overflow (those queries are scanned in full), K from 1 to 32, and
rows of 32 and 64 floats (d = 60 padded).
"""

import numpy as np
import pytest

import oracle as O
from paper_2208_02734_gb300 import mask as M
from paper_2208_02734_gb300 import synth

from parity_util import arr, check_knn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(monkeypatch, idx, Q, k, probes, leaf, kernel=None):
    monkeypatch.setenv("MASK_LEAF_SCAN", leaf)
    if kernel is None:
        monkeypatch.delenv("MASK_CM_KERNEL", raising=False)
    else:
        monkeypatch.setenv("MASK_CM_KERNEL", kernel)
    return M.mask_query(idx, Q, k, probes)


@pytest.fixture(scope="module", params=[(64, 40_000, [300, 12]), (32, 30_000, [100, 8]),
                                        (60, 20_000, [40, 6])],
                ids=["d64", "d32", "d60"])
def built(request):
    d, n, kpl = request.param
    mix = synth.AnisotropicMixture(d=d, n_blobs=12, seed=3)
    X = mix.sample(n, seed=4)
    Q = mix.sample(2_000, seed=5)
    idx = M.mask_build(cuda(X), kpl, 5, seed=2)
    yield d, X, Q, idx
    idx.free()


@pytest.mark.parametrize("k,probes", [(10, [12, 4]), (1, [3, 2]), (16, [20, 6]), (17, [20, 6]),
                                     (32, [20, 6]), (10, [60, 1])])
def test_tc_scan_equals_the_other_scans(monkeypatch, built, k, probes):
    d, X, Q, idx = built
    Qd = cuda(Q)
    ref = run(monkeypatch, idx, Qd, k, probes, "query")
    tc = run(monkeypatch, idx, Qd, k, probes, "cluster")
    simt = run(monkeypatch, idx, Qd, k, probes, "cluster", kernel="simt")
    assert torch.equal(ref[0], tc[0]) and torch.equal(ref[1], tc[1])
    assert torch.equal(ref[0], simt[0]) and torch.equal(ref[1], simt[1])


@pytest.mark.parametrize("tile", [":32:0", ":20:0", ":16:0", ":8:0", ":3:0", ":1:0"])
def test_tc_scan_with_fewer_queries_per_item(monkeypatch, built, tile):
    d, X, Q, idx = built
    Qd = cuda(Q[:700])
    ref = run(monkeypatch, idx, Qd, 10, [12, 4], "query")
    tc = run(monkeypatch, idx, Qd, 10, [12, 4], "cluster" + tile)
    assert torch.equal(ref[0], tc[0]) and torch.equal(ref[1], tc[1])


def test_tc_scan_matches_the_oracle_descent(monkeypatch, built):
    d, X, Q, idx = built
    L = idx.info.n_levels
    levels = [M.mask_index_export_level(idx, lv) for lv in range(L)]
    oref = O.Index(X, [arr(e["centroids"]).astype(np.float64) for e in levels],
                   [arr(e["labels"]) for e in levels])
    sub = Q[:150]
    ids, dd = run(monkeypatch, idx, cuda(sub), 10, [12, 4], "cluster")
    ids_o, d_o, clear = oref.query(sub, 10, [12, 4])
    loose = check_knn(X, sub, arr(ids), arr(dd), ids_o, d_o, clear)
    assert loose <= 0.02 * len(sub)


def test_tc_scan_with_empty_leaf_clusters(monkeypatch):
    # every 5th leaf cluster hands its members to the next one
    d = 64
    mix = synth.IsotropicMixture(d=d, n_blobs=8, seed=6)
    X = mix.sample(12_000, seed=7)
    Q = mix.sample(900, seed=8)
    base = M.mask_build(cuda(X), [120, 10], 4, seed=1)
    levels = [M.mask_index_export_level(base, lv) for lv in range(2)]
    base.free()
    lab0 = arr(levels[0]["labels"]).astype(np.int64)
    remap = np.arange(120)
    empty = np.arange(0, 120, 5)
    remap[empty] = (empty + 1) % 120
    lab0 = remap[lab0].astype(np.int32)
    idx = M.mask_index_load(cuda(X), [cuda(levels[0]["centroids"]), cuda(levels[1]["centroids"])],
                            [cuda(lab0), cuda(levels[1]["labels"])])
    try:
        Qd = cuda(Q)
        ref = run(monkeypatch, idx, Qd, 10, [15, 5], "query")
        tc = run(monkeypatch, idx, Qd, 10, [15, 5], "cluster")
        assert torch.equal(ref[0], tc[0]) and torch.equal(ref[1], tc[1])
    finally:
        idx.free()


@pytest.mark.parametrize("cap", ["1", "7", "40"])
def test_tc_scan_candidate_overflow(monkeypatch, built, cap):
    # queries with more filter passes than their candidate list holds are
    # answered from every row of their kept clusters: same answers
    d, X, Q, idx = built
    Qd = cuda(Q[:600])
    ref = run(monkeypatch, idx, Qd, 10, [12, 4], "query")
    monkeypatch.setenv("MASK_CM_CAND_CAP", cap)
    tc = run(monkeypatch, idx, Qd, 10, [12, 4], "cluster")
    monkeypatch.delenv("MASK_CM_CAND_CAP")
    assert torch.equal(ref[0], tc[0]) and torch.equal(ref[1], tc[1])


def test_tc_scan_batch_independence(monkeypatch, built):
    d, X, Q, idx = built
    whole = run(monkeypatch, idx, cuda(Q[:1200]), 10, [12, 4], "cluster")
    part = run(monkeypatch, idx, cuda(Q[400:800]), 10, [12, 4], "cluster")
    assert torch.equal(whole[0][400:800], part[0]) and torch.equal(whole[1][400:800], part[1])
