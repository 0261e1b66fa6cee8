"""Parity of the grouped build (§3.1, Algorithm 1 as printed), the descent to
the leaf clusters, the relocation pass (§4.1) and the exhaustive point query
of §4.2 with the FP64 oracle.  Inputs: 8 Gaussian clouds in R^2 (the paper's
synthetic setting; centres on a circle, spread set by the separation) and a
few higher-dimensional mixtures."""

import numpy as np
import pytest

import oracle as O
from paper_2208_02734_gb300 import mask as M
from paper_2208_02734_gb300 import synth

from parity_util import RTOL, arr, check_labels, check_rows_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def clouds(npc, sep, sigma, seed):
    return synth.gaussian_clouds_2d(npc, sep, sigma, seed=seed)


@pytest.mark.parametrize("n,lg,nc", [(80, 10, 5), (1600, 16, 8), (80_000, 30, 15), (15, 16, 8)])
def test_level_sizes_match_oracle(n, lg, nc):
    assert M.mask_grouped_levels(n, lg, nc) == O.grouped_sizes(n, lg, nc)


@pytest.mark.parametrize("npc,d,lg,nc,iters", [(200, 2, 16, 8, 10), (60, 16, 10, 5, 6),
                                               (40, 64, 20, 4, 4)])
def test_grouped_build_matches_oracle_level_by_level(npc, d, lg, nc, iters):
    if d == 2:
        X = clouds(npc, 10.0, 1.0, seed=0)
    else:
        X = synth.IsotropicMixture(d=d, n_blobs=8, seed=1).sample(8 * npc, seed=2)
    seed = 11
    idx = M.mask_build_grouped(cuda(X), lg, nc, iters, seed)
    sizes = O.grouped_sizes(len(X), lg, nc)
    assert list(idx.info.k_per_level[:idx.info.n_levels]) == sizes
    # teacher-forced per level: the oracle clusters the GPU's items of the
    # level with the same split and seeding streams
    items = X.astype(np.float64)
    flips = 0
    for lv in range(len(sizes)):
        e = M.mask_index_export_level(idx, lv)
        Cg, lab = arr(e["centroids"]), arr(e["labels"])
        m = len(items)
        G = m // lg
        groups = O.split_groups(m, G, O.level_state(seed, lv))
        Co = np.empty((G * nc, d))
        lo = np.empty(m, np.int32)
        for g in range(G):
            mem = np.flatnonzero(groups == g)
            _, C0 = O.kmeanspp(items[mem], nc, O.group_state(seed, lv, g))
            Cg_o, lg_o, _ = O.lloyd(items[mem], C0, iters)
            Co[g * nc:(g + 1) * nc] = Cg_o
            lo[mem] = g * nc + lg_o
        assert np.array_equal(lab // nc, lo // nc)           # every item in its group
        flips += check_labels(items, Cg, lab, lo)
        check_rows_close(Cg, Co, what=f"level {lv} centroids")
        items = Cg.astype(np.float64)
    assert flips <= 2, flips
    idx.free()


def test_descend_matches_oracle_on_the_oracle_index():
    X = clouds(100, 8.0, 1.5, seed=3)
    ref = O.build_grouped(X, 16, 8, 6, 5)
    Q = clouds(20, 8.0, 1.5, seed=4)
    L = len(ref.centroids)
    loaded = M.mask_index_load(cuda(X.astype(np.float32)),
                               [cuda(c.astype(np.float32)) for c in ref.centroids],
                               [cuda(lb) for lb in ref.labels])
    oref = O.Index(X.astype(np.float32), [c.astype(np.float32) for c in ref.centroids], ref.labels)
    for probes in ([1] * L, [4] + [2] * (L - 1)):
        got = arr(M.mask_descend(loaded, cuda(Q.astype(np.float32)), probes))
        want = O.descend(oref, Q.astype(np.float32), probes)
        _, _, clear = oref.query(Q.astype(np.float32), 1, probes)
        assert clear.mean() > 0.8
        assert np.array_equal(got[clear], want[clear])
    loaded.free()


def test_point_query_error_and_relocation_match_oracle():
    # §4.2: exhaustive point query of every indexed point (greedy descent);
    # §4.1: relocate the missed points, rebuild, query again
    X = clouds(200, 6.0, 1.5, seed=5).astype(np.float32)
    lg, nc, iters, seed = 16, 8, 6, 0
    idx = M.mask_build_grouped(cuda(X), lg, nc, iters, seed)
    L = idx.info.n_levels
    levels = [M.mask_index_export_level(idx, lv) for lv in range(L)]
    oref = O.Index(X, [arr(e["centroids"]).astype(np.float64) for e in levels],
                   [arr(e["labels"]) for e in levels])
    g0 = arr(levels[0]["labels"]) // nc
    missed, moved, g1 = M.mask_relocate(idx, cuda(X), nc, g0)
    o_missed, o_g1, o_moved = O.relocate(oref, nc, g0)
    # descents decided by a near-tie may go either way
    _, _, clear = oref.query(X, 1, [1] * L)
    assert abs(missed - o_missed) <= int((~clear).sum())
    if clear.all():
        assert missed == o_missed and moved == o_moved and np.array_equal(g1, o_g1)
    assert np.bincount(g1).min() >= nc
    # the greedy point query through the public query (k = 1) sees the same misses
    ids, _ = M.mask_query(idx, cuda(X), 1, [1] * L)
    self_found = arr(ids)[:, 0] == np.arange(len(X))
    assert int((~self_found).sum()) == missed
    idx.free()
    idx2 = M.mask_build_grouped(cuda(X), lg, nc, iters, seed, group0=g1)
    assert np.array_equal(arr(M.mask_index_export_level(idx2, 0)["labels"]) // nc, g1)
    idx2.free()


def test_grouped_build_rejects_bad_parameters():
    X = cuda(np.zeros((10, 2), np.float32))
    for lg, nc in [(16, 8), (4, 5), (0, 1)]:
        with pytest.raises(M.MaskError):
            M.mask_build_grouped(X, lg, nc, 3, 0)
    with pytest.raises(M.MaskError):   # group0 outside [0, n / lengthGroup)
        M.mask_build_grouped(X, 5, 2, 3, 0, group0=np.full(10, 2, np.int32))


# ------------------------------------------------------ range search (A3)

def _radius_clear_of_ties(index_o, Q, r):
    """Nudge r so that no centroid of any level and no point lies within a
    relative 2e-6 of the ball's boundary for any query (well beyond the FP32
    rounding of a 2-D squared distance, so FP32 and FP64 decide every
    membership alike)."""
    rows = [index_o.X] + list(index_o.centroids)
    for _ in range(50):
        r2, ok = r * r, True
        for R in rows:
            d = ((R[None, :, :] - Q[:, None, :]) ** 2).sum(-1)
            if np.any(np.abs(d - r2) <= 2e-6 * r2):
                ok = False
                break
        if ok:
            return r
        r *= 1.0137
    raise AssertionError("no tie-free radius found")


@pytest.mark.parametrize("build", ["global", "grouped"])
def test_range_query_matches_oracle(build):
    X = clouds(150, 6.0, 1.2, seed=7).astype(np.float32)
    Q = clouds(6, 6.0, 1.2, seed=8).astype(np.float32)
    if build == "global":
        ref = O.build(X, [120, 12], 6, 0)
    else:
        ref = O.build_grouped(X, 16, 8, 6, 1)
    cs = [c.astype(np.float32) for c in ref.centroids]
    oref = O.Index(X, [c.astype(np.float64) for c in cs], ref.labels)
    loaded = M.mask_index_load(cuda(X), [cuda(c) for c in cs], [cuda(lb) for lb in ref.labels])
    for r in (0.7, 2.0, 5.0, 40.0):
        r = _radius_clear_of_ties(oref, Q.astype(np.float64), r)
        got = M.mask_range_query(loaded, cuda(Q), r)
        want = O.range_query(oref, Q, r)
        for q in range(len(Q)):
            gi, gd = arr(got[q][0]), arr(got[q][1])
            wi, wd = want[q]
            # the same points (the radius is clear of ties); the order is by
            # (distance, id) on each side, so it may differ only where FP32
            # and FP64 distances of two points nearly tie
            assert sorted(gi.tolist()) == sorted(wi.tolist()), (r, q)
            assert np.all(np.diff(gd) >= 0)
            exact = O.sqdist_rows(X, gi, Q[q])
            assert np.allclose(gd, exact, rtol=RTOL, atol=1e-6)
            for a in np.flatnonzero(gi != wi):
                da, db = O.sqdist_rows(X, [gi[a], wi[a]], Q[q])
                assert abs(da - db) <= RTOL * max(da, db) + 1e-12, (r, q, a)
    # host buffers, an empty batch and a too-small buffer
    got_h = M.mask_range_query(loaded, Q, 40.0)
    assert sum(len(i) for i, _ in got_h) == sum(len(i) for i, _ in O.range_query(oref, Q, 40.0))
    assert M.mask_range_query(loaded, Q[:0], 1.0) == []
    counts = np.zeros(len(Q), np.int64)
    st = M.load().mask_range_query(loaded.handle, Q.ctypes.data, len(Q), 40.0, counts.ctypes.data,
                                   1, np.zeros(1, np.int64).ctypes.data, None, None)
    assert st == M.MASK_EINVAL and counts.sum() > 1
    loaded.free()


# ---------------------------------------------------------- insertion

def test_insertion_joins_the_reached_leaf_and_queries_see_it():
    X = clouds(150, 6.0, 1.2, seed=9).astype(np.float32)
    n0 = 1000
    idx = M.mask_build(cuda(X[:n0]), [100, 10], 6, seed=0)
    levels = [M.mask_index_export_level(idx, lv) for lv in range(2)]
    cs = [arr(e["centroids"]).astype(np.float64) for e in levels]
    labs = [arr(e["labels"]) for e in levels]
    leaf = arr(M.mask_insert(idx, cuda(X[n0:])))
    assert idx.info.n == len(X)
    oref0 = O.Index(X[:n0], cs, labs)
    want = O.descend(oref0, X[n0:], [1, 1])[:, 0]
    _, _, clear = oref0.query(X[n0:], 1, [1, 1])
    assert np.array_equal(leaf[clear], want[clear])
    # the updated index is the oracle's index with the new labels appended
    lab0 = arr(M.mask_index_export_level(idx, 0)["labels"])
    assert np.array_equal(lab0[:n0], labs[0]) and np.array_equal(lab0[n0:], leaf)
    oref = O.Index(X, cs, [lab0, labs[1]])
    Q = clouds(10, 6.0, 1.2, seed=10).astype(np.float32)
    ids, d = M.mask_query(idx, cuda(Q), 5, [4, 3])
    ids_o, d_o, clear = oref.query(Q, 5, [4, 3])
    from parity_util import check_knn
    check_knn(X, Q, arr(ids), arr(d), ids_o, d_o, clear)
    # each new point finds itself (it sits in the leaf it joined)
    ids_s, d_s = M.mask_query(idx, cuda(X[n0:]), 1, [1, 1])
    assert np.all(arr(d_s)[:, 0] == 0.0)
    idx.free()


# ---------------------------------------- one-launch greedy descent

@pytest.mark.parametrize("d", [2, 16, 64, 130])
def test_greedy_point_query_equals_the_general_descent(d):
    if d == 2:
        X = clouds(500, 6.0, 1.5, seed=11).astype(np.float32)
        idx = M.mask_build_grouped(cuda(X), 16, 8, 5, 3)
    else:
        X = synth.IsotropicMixture(d=d, n_blobs=6, seed=2).sample(6000, seed=3)
        idx = M.mask_build(cuda(X), [300, 30, 4], 5, seed=1)
    L = idx.info.n_levels
    Q = cuda(np.concatenate([X[:300], X[:300] + 0.01]))
    ids1, d1 = M.mask_query(idx, Q, 1, [1] * L)           # one launch
    ids2, d2 = M.mask_query(idx, Q, 2, [1] * L)           # the level-by-level scans
    assert torch.equal(ids1[:, 0], ids2[:, 0]) and torch.equal(d1[:, 0], d2[:, 0])
    leaf1 = M.mask_descend(idx, Q, [1] * L)
    leaf2 = M.mask_descend(idx, Q, [2] + [1] * (L - 1))
    assert torch.equal(leaf1[:, 0], leaf2[:, 0])
    idx.free()
