"""Parity of the CSR (sparse-point) path with the FP64 oracle.

The oracle runs on the same rows densified (it has no sparse code: a CSR row
is the dense row with zeros elsewhere).  Inputs come from
synth.sparse_tfidf_like (L2-normalised rows, log-normal lengths, Zipf column
ids) at sizes the oracle finishes in seconds; each k-means step is
teacher-forced through the CSR entry points, the build is compared end to end,
and queries are compared with the oracle's descent over the very index the GPU
built (its exported centroids and labels).
"""

import numpy as np
import pytest

import oracle as O
from paper_2208_02734_gb300 import mask as M
from paper_2208_02734_gb300 import synth

from parity_util import RTOL, arr, check_close, check_knn, check_labels, check_rows_close, f64

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def dcsr(A):
    return cuda(A.row_ptr), cuda(A.col), cuda(A.val)


def workload(n=4000, d=600, nnz=25.0, seed=0):
    return synth.sparse_tfidf_like(n, d, nnz_mean=nnz, seed=seed)


# ------------------------------------------------------------------ assign

@pytest.mark.parametrize("n,d,nnz,k", [(3000, 600, 25.0, 64), (2000, 300, 12.0, 700),
                                        (500, 2000, 60.0, 1), (1500, 64, 8.0, 513)])
def test_csr_assign_matches_oracle(n, d, nnz, k):
    A = workload(n, d, nnz)
    X = A.to_dense()
    rng = np.random.default_rng(3)
    Cc = X[rng.choice(n, k, replace=False)].astype(np.float32)
    Cc += rng.normal(scale=0.01, size=Cc.shape).astype(np.float32)
    lab_o, dist_o = O.assign(X, Cc.astype(np.float64))
    lab_g, dist_g = M.mask_kmeans_assign_csr(*dcsr(A), d, cuda(Cc))
    check_labels(X, Cc, lab_g, lab_o)
    # the reported distance is that of the GPU's label
    d_of_g = np.array([O.sqdist_rows(Cc, [l], X[i])[0] for i, l in enumerate(arr(lab_g))])
    check_close(dist_g, d_of_g, rtol=RTOL, atol=1e-6, what="label distances")


def test_csr_assign_exact_ties_go_to_smallest_index():
    A = workload(1000, 200, 10.0)
    X = A.to_dense()
    Cc = X[[5, 9, 300, 77]].astype(np.float32)
    Cc = np.concatenate([Cc, Cc[::-1]])      # every centroid twice: j and 7 - j
    lab_g, _ = M.mask_kmeans_assign_csr(*dcsr(A), 200, cuda(Cc))
    lab_o, _ = O.assign(X, Cc.astype(np.float64))
    assert np.all(arr(lab_g) < 4)
    check_labels(X, Cc, lab_g, lab_o)


def test_csr_assign_empty_rows_and_host_buffers():
    A = workload(800, 100, 6.0)
    # make rows 0, 10 and the last empty
    lens = np.diff(A.row_ptr)
    keep = np.ones(A.nnz, bool)
    for r in [0, 10, A.n_rows - 1]:
        keep[A.row_ptr[r]:A.row_ptr[r + 1]] = False
        lens[r] = 0
    rp = np.zeros(A.n_rows + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    B = synth.CSR(rp, A.col[keep], A.val[keep], 100)
    X = B.to_dense()
    Cc = np.random.default_rng(0).normal(scale=0.1, size=(40, 100)).astype(np.float32)
    lab_o, _ = O.assign(X, Cc.astype(np.float64))
    lab_h, d_h = M.mask_kmeans_assign_csr(B.row_ptr, B.col, B.val, 100, Cc)
    lab_d, d_d = M.mask_kmeans_assign_csr(*dcsr(B), 100, cuda(Cc))
    assert np.array_equal(lab_h, arr(lab_d)) and np.array_equal(d_h, arr(d_d))
    check_labels(X, Cc, lab_h, lab_o)
    assert lab_h[0] == int(np.argmin((Cc.astype(np.float64) ** 2).sum(1)))


# ------------------------------------------------------------------ update

@pytest.mark.parametrize("n,d,nnz,k", [(3000, 600, 25.0, 64), (2000, 300, 12.0, 700)])
def test_csr_update_matches_oracle(n, d, nnz, k):
    A = workload(n, d, nnz)
    X = A.to_dense()
    rng = np.random.default_rng(1)
    lab = rng.integers(0, k, size=n).astype(np.int32)
    lab[lab == 3] = 4                                 # cluster 3 empty: keeps its centroid
    C_prev = rng.normal(size=(k, d)).astype(np.float32)
    C_o, _ = O.update(X, lab, C_prev.astype(np.float64))
    C_g, cnt = M.mask_kmeans_update_csr(*dcsr(A), d, cuda(lab), cuda(C_prev))
    check_rows_close(C_g, C_o, what="centroids")
    assert np.array_equal(arr(C_g)[3], C_prev[3])
    assert np.array_equal(arr(cnt), np.bincount(lab, minlength=k))


def test_csr_update_rejects_out_of_range_labels():
    A = workload(100, 50, 5.0)
    with pytest.raises(M.MaskError, match="labels out of range"):
        M.mask_kmeans_update_csr(*dcsr(A), 50, cuda(np.full(100, 7, np.int32)),
                                 cuda(np.zeros((3, 50), np.float32)))


# ------------------------------------------------------------ k-means++

@pytest.mark.parametrize("n,d,nnz,k,seed,level", [(3000, 600, 25.0, 64, 0, 0),
                                                   (5000, 2000, 40.0, 300, 4, 1),
                                                   (400, 50, 3.0, 400, 2, 0)])
def test_csr_kmeanspp_matches_oracle(n, d, nnz, k, seed, level):
    A = workload(n, d, nnz, seed=seed)
    X = A.to_dense()
    ch_o, C_o = O.seed_level(X, k, seed=seed, level=level)
    C_g, ch_g = M.mask_kmeanspp_csr(*dcsr(A), d, k, seed=seed, level=level)
    assert ch_g.tolist() == ch_o.tolist()
    assert np.array_equal(arr(C_g), X[ch_o].astype(np.float32))


def test_wide_dense_kmeanspp_matches_oracle():
    # dense rows wider than 256: one warp per row, no pruning
    rng = np.random.default_rng(7)
    X = (rng.normal(size=(3000, 700)) * rng.uniform(0.5, 2, size=(3000, 1))).astype(np.float32)
    ch_o, _ = O.seed_level(X, 90, seed=1, level=0)
    _, ch_g = M.mask_kmeanspp(cuda(X), 90, seed=1, level=0)
    assert ch_g.tolist() == ch_o.tolist()


# ------------------------------------------------------------ build

KPL, ITERS = [64, 8], 8


@pytest.fixture(scope="module")
def sparse_c():
    A = workload()
    Qa = synth.sparse_tfidf_like(300, 600, nnz_mean=25.0, seed=1)
    X = A.to_dense()
    idx_o = O.build(X, KPL, iters=ITERS, seed=0)
    idx = M.mask_build_csr(*dcsr(A), 600, KPL, ITERS, seed=0)
    yield A, Qa, X, idx_o, idx
    idx.free()


def test_csr_build_end_to_end_matches_oracle(sparse_c):
    A, _, X, idx_o, idx = sparse_c
    info = idx.info
    assert info.sparse == 1 and info.n == A.n_rows and info.d == 600
    X_in = X
    for lv in range(len(KPL)):
        e = M.mask_index_export_level(idx, lv)
        assert e["chosen"].tolist() == idx_o.chosen[lv].tolist(), f"seeding level {lv}"
        flips = check_labels(X_in, idx_o.centroids[lv], e["labels"], idx_o.labels[lv])
        assert flips == 0, f"{flips} tolerated label flips at level {lv}"
        check_rows_close(e["centroids"], idx_o.centroids[lv], what=f"centroids level {lv}")
        _, _, J = O.lloyd(X_in, f64(X_in)[idx_o.chosen[lv]], ITERS)
        check_close(e["objective"], J[0::2], rtol=1e-4, what="objective trace")
        assert np.all(np.diff(e["objective"]) <= 1e-5 * e["objective"][0])
        X_in = idx_o.centroids[lv]


def test_csr_build_host_input_equals_device_input(sparse_c):
    A, _, _, _, idx = sparse_c
    with M.mask_build_csr(A.row_ptr, A.col, A.val, 600, KPL, ITERS, seed=0) as idx_h:
        for lv in range(len(KPL)):
            eh = M.mask_index_export_level(idx_h, lv)
            ed = M.mask_index_export_level(idx, lv)
            assert np.array_equal(eh["labels"], ed["labels"])
            assert np.array_equal(eh["centroids"], ed["centroids"])


# ------------------------------------------------------------------ query

def oracle_of(idx, X):
    """The oracle's descent over the GPU-built index (FP32 centroids)."""
    es = [M.mask_index_export_level(idx, lv) for lv in range(idx.info.n_levels)]
    return O.Index(X, [e["centroids"].astype(np.float64) for e in es], [e["labels"] for e in es])


@pytest.mark.parametrize("leaf", ["query", "cluster"])
@pytest.mark.parametrize("k,probes", [(10, [16, 4]), (1, [1, 1]), (10, [3, 2]), (50, [64, 8]),
                                      (100, [2, 1])])
def test_csr_query_matches_oracle(monkeypatch, sparse_c, leaf, k, probes):
    # per-query leaf scan, or cluster-major (k <= 64; k = 100 falls back)
    monkeypatch.setenv("MASK_LEAF_SCAN", leaf)
    A, Qa, X, _, idx = sparse_c
    Q = Qa.to_dense()
    ref = oracle_of(idx, X)
    ids_o, d_o, clear = ref.query(Q, k, probes)
    ids_g, d_g = M.mask_query_csr(idx, *dcsr(Qa), k, probes)
    loose = check_knn(X, Q, ids_g, d_g, ids_o, d_o, clear)
    assert loose <= 0.01 * len(Q)


@pytest.mark.parametrize("k,probes", [(10, [16, 4]), (1, [3, 2]), (64, [32, 8]), (10, [60, 1])])
def test_csr_leaf_scans_agree_bitwise(monkeypatch, sparse_c, k, probes):
    # the cluster-major scan accumulates every (query, row) pair exactly like
    # the per-query scan; [60, 1] leaves absent leaf slots
    _, Qa, _, _, idx = sparse_c
    out = {}
    for leaf in ["query", "cluster"]:
        monkeypatch.setenv("MASK_LEAF_SCAN", leaf)
        out[leaf] = M.mask_query_csr(idx, *dcsr(Qa), k, probes)
    assert torch.equal(out["query"][0], out["cluster"][0])
    assert torch.equal(out["query"][1], out["cluster"][1])


def test_csr_long_queries_in_a_cluster_major_batch():
    # queries with more nonzeros than a cluster-major pass holds are served by
    # the per-query scan inside the same batch: both modes agree bit for bit
    A = synth.sparse_tfidf_like(3000, 3000, nnz_mean=30.0, seed=4)
    Qa = synth.sparse_tfidf_like(120, 3000, nnz_mean=700.0, nnz_sigma=0.5, seed=5)
    assert np.diff(Qa.row_ptr).max() > 1024
    with M.mask_build_csr(*dcsr(A), 3000, [40, 5], 4, seed=0) as idx:
        out = {}
        for leaf in ["query", "cluster"]:
            import os
            os.environ["MASK_LEAF_SCAN"] = leaf
            try:
                out[leaf] = M.mask_query_csr(idx, *dcsr(Qa), 10, [12, 3])
            finally:
                del os.environ["MASK_LEAF_SCAN"]
        assert torch.equal(out["query"][0], out["cluster"][0])
        assert torch.equal(out["query"][1], out["cluster"][1])
        X, Q = A.to_dense(), Qa.to_dense()
        ref = oracle_of(idx, X)
        ids_o, d_o, clear = ref.query(Q, 10, [12, 3])
        check_knn(X, Q, out["cluster"][0], out["cluster"][1], ids_o, d_o, clear)


def test_csr_probing_everything_is_exact_knn(sparse_c):
    A, Qa, X, _, idx = sparse_c
    Q = Qa.to_dense()[:100]
    ids_b, d_b = O.bruteforce_knn(X, Q, 10)
    ids_g, d_g = M.mask_query_csr(idx, *dcsr(Qa.rows(np.arange(100))), 10, KPL)
    check_knn(X, Q, ids_g, d_g, ids_b, d_b, np.ones(100, bool))


def test_csr_query_of_a_data_row_finds_it_at_zero(sparse_c):
    A, _, X, _, idx = sparse_c
    rows = np.arange(0, 4000, 97)
    ids, d = M.mask_query_csr(idx, *dcsr(A.rows(rows)), 3, KPL)
    assert np.array_equal(arr(ids)[:, 0], rows)
    assert np.all(arr(d)[:, 0] == 0.0)


def test_csr_query_results_do_not_depend_on_the_batch(sparse_c):
    _, Qa, _, _, idx = sparse_c
    ids_all, d_all = M.mask_query_csr(idx, *dcsr(Qa), 10, [16, 4])
    pos = 0
    for size in [1, 7, 92, 200]:
        sub = Qa.rows(np.arange(pos, pos + size))
        ids_p, d_p = M.mask_query_csr(idx, *dcsr(sub), 10, [16, 4])
        assert torch.equal(ids_p, ids_all[pos:pos + size])
        assert torch.equal(d_p, d_all[pos:pos + size])
        pos += size
    assert pos == Qa.n_rows


def test_csr_query_host_buffers_and_empty_batch(sparse_c):
    _, Qa, _, _, idx = sparse_c
    sub = Qa.rows(np.arange(40))
    ids_h, d_h = M.mask_query_csr(idx, sub.row_ptr, sub.col, sub.val, 10, [16, 4])
    ids_d, d_d = M.mask_query_csr(idx, *dcsr(sub), 10, [16, 4])
    assert np.array_equal(ids_h, arr(ids_d)) and np.array_equal(d_h, arr(d_d))
    empty = Qa.rows(np.arange(0))
    ids, _ = M.mask_query_csr(idx, *dcsr(empty), 10, [16, 4])
    assert ids.shape == (0, 10)


# --------------------------------------------------------- errors

def test_csr_rejects_malformed_inputs(sparse_c):
    A, Qa, _, _, idx = sparse_c
    rp, col, val = A.row_ptr.copy(), A.col.copy(), A.val.copy()
    bad_col = col.copy()
    bad_col[rp[1] - 1] = 600      # the last (largest) column of row 0: still increasing
    with pytest.raises(M.MaskError, match="outside"):
        M.mask_build_csr(rp, bad_col, val, 600, [8], 1, seed=0)
    unsorted = col.copy()
    b = rp[3]
    unsorted[b], unsorted[b + 1] = unsorted[b + 1], unsorted[b]
    with pytest.raises(M.MaskError, match="malformed"):
        M.mask_build_csr(rp, unsorted, val, 600, [8], 1, seed=0)
    shifted = rp + 1
    with pytest.raises(M.MaskError, match=r"row_ptr\[0\]"):
        M.mask_build_csr(shifted, col, val, 600, [8], 1, seed=0)
    with pytest.raises(M.MaskError, match="MASK_EUNSUPPORTED"):
        M.mask_build_csr(rp, col, val, 50_000, [8], 1, seed=0)
    with pytest.raises(M.MaskError, match="mask_query_csr"):
        M.mask_query(idx, cuda(np.zeros((2, 600), np.float32)), 5, [4, 2])
    with pytest.raises(M.MaskError, match="MASK_EUNSUPPORTED"):
        M.mask_query_csr(idx, *dcsr(Qa.rows(np.arange(4))), 5, [4, 2], precision=M.MASK_BF16)
    dense = M.mask_build(cuda(np.random.default_rng(0).normal(size=(300, 8)).astype(np.float32)),
                         [10], 2, seed=0)
    with pytest.raises(M.MaskError, match="mask_query"):
        M.mask_query_csr(dense, *dcsr(Qa.rows(np.arange(4))), 5, [4])
    dense.free()


def test_csr_update_of_a_cluster_beyond_2_20_members_sums_in_fp64():
    # 2^20 + 1 rows in cluster 0 (FP64 sums), the rest in cluster 1; every
    # row has the same few columns, values near 100, so FP32 running sums
    # would lose digits and only FP64 sums stay within one FP32 ulp of the
    # oracle's mean rounded to FP32
    m0, m1, d, per = (1 << 20) + 1, 5000, 40, 4
    n = m0 + m1
    rng = np.random.default_rng(12)
    cols = np.sort(rng.choice(d, per, replace=False)).astype(np.int32)
    rp = np.arange(0, (n + 1) * per, per, dtype=np.int64)
    col = np.tile(cols, n)
    val = (100.0 + rng.random(n * per)).astype(np.float32)
    A = synth.CSR(rp, col, val, d)
    lab = np.zeros(n, np.int32)
    lab[rng.choice(n, m1, replace=False)] = 1
    C_prev = np.zeros((2, d), np.float32)
    # oracle on the densified columns only (the others are exact zeros)
    Xc = val.reshape(n, per).astype(np.float64)
    C_o_c, cnt_o = O.update(Xc, lab, np.zeros((2, per)))
    C_g, cnt_g = M.mask_kmeans_update_csr(*dcsr(A), d, cuda(lab), cuda(C_prev))
    C_g = arr(C_g)
    assert arr(cnt_g).tolist() == cnt_o.tolist() == [m0, m1]
    other = np.setdiff1d(np.arange(d), cols)
    assert np.all(C_g[:, other] == 0.0)
    check_rows_close(C_g[:, cols], C_o_c, what="centroids")
    ref = C_o_c[0].astype(np.float32)
    ulps = np.abs(C_g[0, cols].astype(np.float64) - ref) / np.spacing(np.abs(ref))
    assert ulps.max() <= 1.0, (C_g[0, cols], C_o_c[0])
