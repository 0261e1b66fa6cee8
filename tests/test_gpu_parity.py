"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Inputs are seeded synthetic data (paper_2208_02734_gb300.synth).  Each k-means
step is teacher-forced with the oracle's state (same centroids / labels in);
the build is also compared end to end on the small dense workload (20,000 x 16,
10 blobs, 200/20 centroids, 20 Lloyd iterations); the query is compared on an
index assembled from the oracle's build (mask_index_load).
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


# ------------------------------------------------------------------ assign

ASSIGN_SHAPES = [(1000, 1, 7), (3000, 3, 200), (5000, 16, 257), (2000, 17, 64),
                 (4000, 64, 130), (700, 130, 33), (300, 8, 1), (129, 24, 128)]


@pytest.mark.parametrize("n,d,k", ASSIGN_SHAPES)
def test_assign_matches_oracle(n, d, k):
    rng = np.random.default_rng(n * 7 + d * 3 + k)
    X = (rng.normal(size=(n, d)) * 3 + rng.uniform(-10, 10, size=(1, d))).astype(np.float32)
    Cc = (X[rng.choice(n, k, replace=False)] + 0.05 * rng.normal(size=(k, d))).astype(np.float32)
    lab_o, dist_o = O.assign(X, Cc)
    lab_g, dist_g = M.mask_kmeans_assign(cuda(X), cuda(Cc))
    check_labels(X, Cc, lab_g, lab_o)
    eq = arr(lab_g) == lab_o
    check_close(arr(dist_g)[eq], dist_o[eq], atol=1e-30, what="assign dist")


@pytest.mark.parametrize("kernel", ["simt", "auto"])
@pytest.mark.parametrize("n,d,k", [(20_000, 16, 200), (30_000, 64, 1000), (5000, 40, 129),
                                   (4000, 64, 3), (3000, 8, 2)])
def test_assign_kernels_match_oracle(monkeypatch, kernel, n, d, k):
    # "auto" takes the tcgen05 (3xTF32) kernel for these dimensions (<= 64)
    monkeypatch.setenv("MASK_ASSIGN_KERNEL", kernel)
    mix = synth.AnisotropicMixture(d=d, n_blobs=20, seed=d)
    X = mix.sample(n, seed=1)
    Cc = X[np.random.default_rng(2).choice(n, k, replace=False)]
    lab_o, dist_o = O.assign(X, Cc)
    lab_g, dist_g = M.mask_kmeans_assign(cuda(X), cuda(Cc))
    check_labels(X, Cc, lab_g, lab_o)
    eq = arr(lab_g) == lab_o
    assert eq.mean() > 0.999
    check_close(arr(dist_g)[eq], dist_o[eq], atol=1e-30, what="assign dist")


def test_assign_exact_ties_go_to_smallest_index():
    rng = np.random.default_rng(3)
    base = rng.normal(size=(40, 16)).astype(np.float32)
    Cc = np.concatenate([base, base, base])          # every centroid three times
    X = np.concatenate([base, base + 0.25]).astype(np.float32)
    lab_g, _ = M.mask_kmeans_assign(cuda(X), cuda(Cc))
    lab_o, _ = O.assign(X, Cc)
    assert np.array_equal(arr(lab_g), lab_o)
    assert arr(lab_g).max() < 40


def test_assign_host_buffers_equal_device_buffers():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(3000, 16)).astype(np.float32)
    Cc = rng.normal(size=(50, 16)).astype(np.float32)
    lh, dh = M.mask_kmeans_assign(X, Cc)
    ld, dd = M.mask_kmeans_assign(cuda(X), cuda(Cc))
    assert isinstance(lh, np.ndarray)
    assert np.array_equal(lh, arr(ld)) and np.array_equal(dh, arr(dd))


# ------------------------------------------------------------------ update

@pytest.mark.parametrize("n,d,k", [(5000, 16, 200), (3000, 17, 64), (2000, 64, 33),
                                   (1000, 130, 7), (800, 3, 300)])
def test_update_matches_oracle(n, d, k):
    rng = np.random.default_rng(n + d)
    X = (rng.normal(size=(n, d)) * 2).astype(np.float32)
    Cprev = (rng.normal(size=(k, d)) * 2).astype(np.float32)
    Cprev[: k // 10] += 1000.0                        # far away: empty clusters
    lab, _ = O.assign(X, Cprev)
    C_o, cnt_o = O.update(X, lab, Cprev)
    C_g, cnt_g = M.mask_kmeans_update(cuda(X), cuda(lab), cuda(Cprev))
    assert np.array_equal(arr(cnt_g), cnt_o)
    assert (cnt_o == 0).sum() >= k // 10
    check_rows_close(C_g, C_o, what="centroids")
    empty = cnt_o == 0
    assert np.array_equal(arr(C_g)[empty], Cprev[empty])


def test_builds_are_bit_reproducible_with_large_clusters():
    # four clusters of ~5,000 points: membership lists longer than the
    # shared-memory sort, whose sums must still run in item order
    X = synth.IsotropicMixture(d=8, n_blobs=4, seed=3).sample(20_000, seed=3)
    out = []
    for _ in range(2):
        with M.mask_build(cuda(X), [4, 2], iters=4, seed=0) as idx:
            out.append([M.mask_index_export_level(idx, lv) for lv in range(2)])
    for a, b in zip(*out):
        assert np.array_equal(arr(a["centroids"]), arr(b["centroids"]))
        assert np.array_equal(arr(a["labels"]), arr(b["labels"]))
        assert np.array_equal(a["objective"], b["objective"])
    counts = np.bincount(arr(out[0][0]["labels"]), minlength=4)
    assert counts.max() > 4096


def test_update_of_a_large_cluster_matches_oracle():
    rng = np.random.default_rng(5)
    X = rng.normal(size=(13_000, 16)).astype(np.float32)
    lab = np.where(rng.random(13_000) < 0.8, 0, rng.integers(1, 6, 13_000)).astype(np.int32)
    C_prev = rng.normal(size=(6, 16)).astype(np.float32)
    C_o, _ = O.update(X, lab, C_prev.astype(np.float64))
    C_g, _ = M.mask_kmeans_update(cuda(X), cuda(lab), cuda(C_prev))
    check_rows_close(C_g, C_o, what="centroids")
    C_g2, _ = M.mask_kmeans_update(cuda(X), cuda(lab), cuda(C_prev))
    assert torch.equal(C_g, C_g2)


def _fp32_ulps(a_g, a_o):
    """|a_g - fl32(a_o)| in units of the FP32 spacing at fl32(a_o)."""
    ref = np.asarray(a_o, np.float64).astype(np.float32)
    spacing = np.spacing(np.abs(ref)).astype(np.float64)
    return np.abs(np.asarray(a_g, np.float64) - ref.astype(np.float64)) / spacing


def test_update_of_clusters_beyond_2_20_members_sums_in_fp64():
    # cluster 0 has 2^20 + 1 members (FP64 sums), cluster 1 exactly 2^20
    # (FP32 sums), cluster 2 a handful.  Coordinates near 1000 make FP32
    # running sums lose digits, so only FP64 sums land within one FP32 ulp of
    # the oracle's mean rounded to FP32.
    m0, m1, m2, d = (1 << 20) + 1, 1 << 20, 7, 8
    n = m0 + m1 + m2
    rng = np.random.default_rng(11)
    X = (1000.0 + rng.random((n, d)) * np.linspace(0.5, 4.0, d)).astype(np.float32)
    lab = np.concatenate([np.zeros(m0), np.ones(m1), np.full(m2, 2)]).astype(np.int32)
    lab = lab[rng.permutation(n)]
    C_prev = np.zeros((3, d), np.float32)
    C_o, cnt_o = O.update(X, lab, C_prev)
    C_g, cnt_g = M.mask_kmeans_update(cuda(X), cuda(lab), cuda(C_prev))
    assert arr(cnt_g).tolist() == [m0, m1, m2] == cnt_o.tolist()
    check_rows_close(C_g, C_o, what="centroids")
    assert _fp32_ulps(arr(C_g)[0], C_o[0]).max() <= 1.0, arr(C_g)[0] - C_o[0]


def test_update_rejects_out_of_range_labels():
    X = np.zeros((10, 4), np.float32)
    with pytest.raises(M.MaskError):
        M.mask_kmeans_update(cuda(X), cuda(np.full(10, 5, np.int32)), cuda(np.zeros((3, 4), np.float32)))


# ------------------------------------------------------------ k-means++

@pytest.mark.parametrize("n,d,k,seed,level", [(5000, 16, 60, 0, 0), (20000, 16, 200, 0, 0),
                                               (3000, 3, 300, 9, 2), (400, 33, 400, 5, 1)])
def test_kmeanspp_matches_oracle(n, d, k, seed, level):
    mix = synth.IsotropicMixture(d=d, n_blobs=10, seed=seed)
    X = mix.sample(n, seed=seed + 1)
    ch_o, C_o = O.seed_level(X, k, seed=seed, level=level)
    C_g, ch_g = M.mask_kmeanspp(cuda(X), k, seed=seed, level=level)
    assert ch_g.tolist() == ch_o.tolist()
    assert np.array_equal(arr(C_g), X[ch_o])


def test_kmeanspp_duplicates_exhaust_distinct_points():
    X = np.repeat(np.arange(5, dtype=np.float32)[:, None], 4, axis=0)  # 5 values x 4 copies
    ch_o, _ = O.seed_level(X, 12, seed=3, level=0)
    _, ch_g = M.mask_kmeanspp(cuda(X), 12, seed=3, level=0)
    assert ch_g.tolist() == ch_o.tolist()


@pytest.mark.slow
def test_kmeanspp_subsample_path_matches_oracle():
    n, k = 4_200_000, 1024                 # n*k > 2^32: seeding on 8k sampled points
    rng = np.random.default_rng(0)
    X = rng.normal(size=(n, 2)).astype(np.float32)
    ch_o, _ = O.seed_level(X, k, seed=5, level=0)
    _, ch_g = M.mask_kmeanspp(cuda(X), k, seed=5, level=0)
    assert ch_g.tolist() == ch_o.tolist()


# ------------------------------------------------------------ build (c1)

def small_dense_workload():
    mix = synth.IsotropicMixture(d=16, n_blobs=10, sigma=1.0, box=10.0, seed=0)
    return mix.sample(20_000, seed=0), mix.sample(1_000, seed=1)


@pytest.fixture(scope="module")
def c1():
    X, Q = small_dense_workload()
    idx_o = O.build(X, [200, 20], iters=20, seed=0)
    return X, Q, idx_o


def test_build_end_to_end_matches_oracle(c1):
    X, Q, idx_o = c1
    with M.mask_build(cuda(X), [200, 20], iters=20, seed=0) as idx:
        X_in = X
        for lv in range(2):
            e = M.mask_index_export_level(idx, lv)
            assert e["chosen"].tolist() == idx_o.chosen[lv].tolist(), f"seeding level {lv}"
            flips = check_labels(X_in, idx_o.centroids[lv], e["labels"], idx_o.labels[lv])
            assert flips == 0, f"{flips} tolerated label flips at level {lv}"
            check_rows_close(e["centroids"], idx_o.centroids[lv], what=f"centroids level {lv}")
            # objective after each assignment, against the oracle's own trace
            _, _, J = O.lloyd(X_in, f64(X_in)[idx_o.chosen[lv]], 20)
            check_close(e["objective"], J[0::2], rtol=1e-4, what="objective trace")
            assert np.all(np.diff(e["objective"]) <= 1e-5 * e["objective"][0])
            X_in = idx_o.centroids[lv]       # the oracle's input of the next level


def test_build_info_and_host_input(c1):
    X, _, _ = c1
    with M.mask_build(X, [200, 20], iters=2, seed=0) as idx:
        info = idx.info
        assert info.n == 20_000 and info.d == 16 and info.n_levels == 2
        assert list(info.k_per_level[:2]) == [200, 20]
        assert info.device_bytes >= 20_000 * 16 * 4


# ------------------------------------------------------------------ query

def oracle_index_fp32(idx_o):
    """The oracle's index with centroids rounded to FP32 (what the GPU holds)."""
    cs = [c.astype(np.float32) for c in idx_o.centroids]
    return O.Index(idx_o.X, [c.astype(np.float64) for c in cs], idx_o.labels), cs


@pytest.fixture(scope="module")
def loaded(c1):
    X, Q, idx_o = c1
    ref, cs = oracle_index_fp32(idx_o)
    idx = M.mask_index_load(cuda(X), [cuda(c) for c in cs], [cuda(lb) for lb in idx_o.labels])
    yield X, Q, ref, idx
    idx.free()


@pytest.mark.parametrize("leaf", ["query", "cluster"])
@pytest.mark.parametrize("k,probes", [(10, [3, 3]), (1, [1, 1]), (10, [1, 1]), (100, [5, 4]),
                                      (17, [2, 20]), (32, [40, 10])])
def test_query_matches_oracle(monkeypatch, loaded, leaf, k, probes):
    # leaf scan query by query, or cluster-major (k <= 32; larger k falls back)
    monkeypatch.setenv("MASK_LEAF_SCAN", leaf)
    X, Q, ref, idx = loaded
    ids_o, d_o, clear = ref.query(Q, k, probes)
    ids_g, d_g = M.mask_query(idx, cuda(Q), k, probes)
    loose = check_knn(X, Q, ids_g, d_g, ids_o, d_o, clear)
    assert loose <= 0.01 * len(Q)


@pytest.mark.parametrize("leaf", ["query", "cluster"])
def test_probes_beyond_the_children_kept(monkeypatch, loaded, leaf):
    # one top centroid kept (about 10 children) but 60 leaf probes: most of a
    # query's leaf slots are absent (-1) and must contribute nothing
    monkeypatch.setenv("MASK_LEAF_SCAN", leaf)
    X, Q, ref, idx = loaded
    ids_o, d_o, clear = ref.query(Q, 10, [60, 1])
    ids_g, d_g = M.mask_query(idx, cuda(Q), 10, [60, 1])
    loose = check_knn(X, Q, ids_g, d_g, ids_o, d_o, clear)
    assert loose <= 0.01 * len(Q)


@pytest.mark.parametrize("prec", [M.MASK_BF16, M.MASK_FP8E4M3])
def test_low_precision_probes_beyond_the_children_kept(loaded, prec):
    X, Q, ref, idx = loaded
    ids_f, _ = M.mask_query(idx, cuda(Q), 10, [60, 1])
    ids_l, d_l = M.mask_query(idx, cuda(Q), 10, [60, 1], precision=prec)
    ids_f, ids_l, d_l = arr(ids_f), arr(ids_l), arr(d_l)
    assert ids_l.min() >= -1 and ids_l.max() < len(X)
    for q in range(0, len(Q), 25):
        ok = ids_l[q] >= 0
        check_close(d_l[q][ok], O.sqdist_rows(X, ids_l[q][ok], Q[q]), rtol=RTOL, atol=1e-30,
                    what=f"re-ranked distances q={q}")
    overlap = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(ids_f, ids_l)])
    assert overlap >= 0.9, overlap


@pytest.mark.parametrize("tile", ["", ":16:1", ":8:0", ":8:1", ":3:2", ":1:0"])
def test_leaf_scan_paths_agree_bitwise(monkeypatch, loaded, tile):
    # both leaf scans evaluate sum_t (x_t - q_t)^2 in the same order, at every
    # cluster-major tile the serving autotuner may pick (queries per work
    # item, blocks per SM)
    X, Q, ref, idx = loaded
    out = {}
    for leaf in ["query", "cluster" + tile]:
        monkeypatch.setenv("MASK_LEAF_SCAN", leaf)
        out[leaf] = M.mask_query(idx, cuda(Q), 10, [12, 6])
    assert torch.equal(out["query"][0], out["cluster" + tile][0])
    assert torch.equal(out["query"][1], out["cluster" + tile][1])


def test_empty_leaf_clusters(monkeypatch, c1):
    # every 7th leaf cluster hands its members to the next one: queries still
    # keep the empty clusters' centroids, whose work items scan no rows
    X, Q, idx_o = c1
    _, cs = oracle_index_fp32(idx_o)
    k0 = len(cs[0])
    remap = np.arange(k0)
    empty = np.arange(0, k0, 7)
    remap[empty] = (empty + 1) % k0
    lab0 = remap[idx_o.labels[0]].astype(np.int32)
    labels = [lab0, idx_o.labels[1]]
    ref = O.Index(idx_o.X, [c.astype(np.float64) for c in cs], labels)
    idx = M.mask_index_load(cuda(X), [cuda(c) for c in cs], [cuda(lb) for lb in labels])
    try:
        out = {}
        for leaf in ["query", "cluster"]:
            monkeypatch.setenv("MASK_LEAF_SCAN", leaf)
            out[leaf] = M.mask_query(idx, cuda(Q), 10, [12, 6])
        assert torch.equal(out["query"][0], out["cluster"][0])
        assert torch.equal(out["query"][1], out["cluster"][1])
        ids_o, d_o, clear = ref.query(Q, 10, [12, 6])
        loose = check_knn(X, Q, out["cluster"][0], out["cluster"][1], ids_o, d_o, clear)
        assert loose <= 0.01 * len(Q)
        for prec in (M.MASK_BF16, M.MASK_FP8E4M3):
            ids_l, d_l = M.mask_query(idx, cuda(Q), 10, [12, 6], precision=prec)
            ids_l, d_l = arr(ids_l), arr(d_l)
            assert ids_l.min() >= -1 and ids_l.max() < len(X)
            for q in range(0, len(Q), 25):
                ok = ids_l[q] >= 0
                check_close(d_l[q][ok], O.sqdist_rows(X, ids_l[q][ok], Q[q]), rtol=RTOL,
                            atol=1e-30, what=f"re-ranked distances q={q}")
    finally:
        idx.free()


def test_probing_everything_is_exact_knn(loaded):
    X, Q, ref, idx = loaded
    ids_b, d_b = O.bruteforce_knn(X, Q[:200], 10)
    ids_g, d_g = M.mask_query(idx, cuda(Q[:200]), 10, [200, 20])
    check_knn(X, Q[:200], ids_g, d_g, ids_b, d_b, np.ones(200, bool))


def test_query_results_do_not_depend_on_the_batch(loaded):
    X, Q, ref, idx = loaded
    ids_all, d_all = M.mask_query(idx, cuda(Q), 10, [3, 3])
    pos = 0
    for size in [1, 7, 512, 200, 280]:
        ids_p, d_p = M.mask_query(idx, cuda(Q[pos:pos + size]), 10, [3, 3])
        assert torch.equal(ids_p, ids_all[pos:pos + size])
        assert torch.equal(d_p, d_all[pos:pos + size])
        pos += size
    assert pos == len(Q)


def test_query_host_buffers(loaded):
    X, Q, ref, idx = loaded
    ids_h, d_h = M.mask_query(idx, Q[:50], 10, [3, 3])
    ids_d, d_d = M.mask_query(idx, cuda(Q[:50]), 10, [3, 3])
    assert np.array_equal(ids_h, arr(ids_d)) and np.array_equal(d_h, arr(d_d))


def test_query_pads_when_fewer_candidates_than_k():
    X = np.array([[0, 0], [1, 0], [10, 0], [11, 0], [30, 0]], np.float32)
    C1 = np.array([[0.5, 0], [10.5, 0], [30, 0]], np.float32)
    C2 = np.array([[5, 0], [30, 0]], np.float32)
    idx = M.mask_index_load(cuda(X), [cuda(C1), cuda(C2)],
                            [cuda(np.array([0, 0, 1, 1, 2], np.int32)), cuda(np.array([0, 0, 1], np.int32))])
    ids, d = M.mask_query(idx, cuda(np.array([[0.2, 0]], np.float32)), 4, [1, 1])
    assert arr(ids)[0].tolist() == [0, 1, -1, -1]
    assert np.isinf(arr(d)[0][2:]).all()
    ids, _ = M.mask_query(idx, cuda(np.array([[0.2, 0]], np.float32)), 5, [9, 9])
    assert arr(ids)[0].tolist() == [0, 1, 2, 3, 4]
    idx.free()


def test_query_empty_batch(loaded):
    X, Q, ref, idx = loaded
    ids, d = M.mask_query(idx, cuda(Q[:0]), 10, [3, 3])
    assert ids.shape == (0, 10)


def test_descent_hand_worked_on_gpu():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "descent_2d.json")))
    f = lambda a: cuda(np.array(a, np.float32))  # noqa: E731
    idx = M.mask_index_load(f(g["points"]), [f(g["level1_centroids"]), f(g["level2_centroids"])],
                            [cuda(np.array(g["level1_labels"], np.int32)),
                             cuda(np.array(g["level2_labels"], np.int32))])
    for c in g["queries"]:
        ids, d = M.mask_query(idx, f([c["q"]]), c["k"], c["probes"])
        assert arr(ids)[0].tolist() == c["ids"]
        assert arr(d)[0].tolist() == [float("inf") if x == "inf" else x for x in c["dists"]]
    idx.free()


def test_export_and_reload_gives_the_same_answers(c1):
    X, Q, _ = c1
    with M.mask_build(cuda(X), [200, 20], iters=5, seed=1) as idx:
        e = [M.mask_index_export_level(idx, lv) for lv in range(2)]
        ids1, d1 = M.mask_query(idx, cuda(Q), 10, [3, 3])
    idx2 = M.mask_index_load(cuda(X), [cuda(x["centroids"]) for x in e],
                             [cuda(x["labels"]) for x in e])
    ids2, d2 = M.mask_query(idx2, cuda(Q), 10, [3, 3])
    idx2.free()
    assert torch.equal(ids1, ids2) and torch.equal(d1, d2)


# ------------------------------------------------- BF16 / FP8 + FP32 re-rank

@pytest.mark.parametrize("prec,min_overlap", [(M.MASK_BF16, 0.995), (M.MASK_FP8E4M3, 0.95)])
@pytest.mark.parametrize("leafk", [1, 10, 16])
def test_low_precision_query_reranks_exactly(loaded, prec, min_overlap, leafk):
    # the shortlist is ranked in low precision; what is returned is re-ranked
    # with exact FP32 distances, so every returned distance is exact
    X, Q, ref, idx = loaded
    probes = [3, 3]
    ids_o, d_o, _ = ref.query(Q, leafk, probes)
    ids_g, d_g = M.mask_query(idx, cuda(Q), leafk, probes, precision=prec)
    ids_g, d_g = arr(ids_g), arr(d_g)
    overlap = total = 0
    for q in range(len(Q)):
        ok = ids_g[q] >= 0
        assert len(set(ids_g[q][ok].tolist())) == ok.sum()
        assert np.all(np.diff(d_g[q][ok]) >= 0)
        check_close(d_g[q][ok], O.sqdist_rows(X, ids_g[q][ok], Q[q]), atol=1e-30,
                    what=f"re-ranked distances q={q}")
        want = set(ids_o[q][ids_o[q] >= 0].tolist())
        overlap += len(set(ids_g[q][ok].tolist()) & want)
        total += len(want)
    assert overlap / total >= min_overlap, overlap / total


def test_low_precision_rejects_long_shortlists(loaded):
    X, Q, ref, idx = loaded
    with pytest.raises(M.MaskError) as e:
        M.mask_query(idx, cuda(Q[:4]), 17, [3, 3], precision=M.MASK_BF16)
    assert e.value.status == M.MASK_EUNSUPPORTED


def test_mixed_precision_workload_recall_and_error(c1):
    # the small dense data and index, 10,000 queries: recall@10 of each mode
    # against the FP64 oracle's descent and against exact k-NN, and the
    # largest relative error of returned distances
    X, _, idx_o = c1
    mix = synth.IsotropicMixture(d=16, n_blobs=10, sigma=1.0, box=10.0, seed=0)
    Q = mix.sample(10_000, seed=2)
    ref, cs = oracle_index_fp32(idx_o)
    idx = M.mask_index_load(cuda(X), [cuda(c) for c in cs], [cuda(lb) for lb in idx_o.labels])
    ids_d, d_d, _ = ref.query(Q, 10, [3, 3])
    ids_b, d_b = O.bruteforce_knn(X, Q, 10)
    report = {}
    for name, prec in [("fp32", M.MASK_FP32), ("bf16", M.MASK_BF16), ("fp8", M.MASK_FP8E4M3)]:
        ids_g, d_g = M.mask_query(idx, cuda(Q), 10, [3, 3], precision=prec)
        ids_g, d_g = arr(ids_g), arr(d_g)
        hit_desc = hit_exact = 0
        err = 0.0
        for q in range(len(Q)):
            ok = ids_g[q] >= 0
            ex = O.sqdist_rows(X, ids_g[q][ok], Q[q])
            err = max(err, float(np.max(np.abs(d_g[q][ok] - ex) / np.maximum(ex, 1e-30))))
            hit_desc += len(set(ids_g[q][ok].tolist()) & set(ids_d[q].tolist()))
            hit_exact += int(np.sum(ex <= d_b[q, -1] * (1 + RTOL)))
        report[name] = (hit_desc / (10 * len(Q)), hit_exact / (10 * len(Q)), err)
    idx.free()
    print("mixed-precision report (recall vs descent, recall vs exact, max rel err):", report)
    assert report["fp32"][0] >= 0.999 and report["fp32"][2] <= RTOL
    assert report["bf16"][0] >= 0.995 and report["bf16"][2] <= RTOL
    assert report["fp8"][0] >= 0.95 and report["fp8"][2] <= RTOL
    for name in report:
        assert abs(report[name][1] - report["fp32"][1]) <= 0.05
