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
        check_rows_close(Cg, Co, rtol=1e-4, what=f"level {lv} centroids")
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
