"""Pins of the oracle's grouped build (§3.1, Algorithm 1 as printed), its
descent to the leaf clusters, the range search (§3.3, Algorithm 3) and the
relocation pass (§4.1), against what the paper prints and what holds by
construction.  CPU only."""

import itertools

import numpy as np
import pytest

import oracle as O


# ------------------------------------------------------- level sizes (P7)

def test_depths_of_tables_5_and_6():
    # §4.2.2, Tables 5-6: N = 80,000 points, lengthGroup / nCentroids
    # 10/5 ... 110/55 give depths 13, 12, 11, 11, 10, 10
    cfg = [(10, 5), (30, 15), (50, 25), (70, 35), (90, 45), (110, 55)]
    assert [len(O.grouped_sizes(80_000, lg, nc)) for lg, nc in cfg] == [13, 12, 11, 11, 10, 10]


def test_worked_example_of_section_3_1():
    # 80 points, lengthGroup 10, nCentroids 5: 8 groups give 40 centroids,
    # then 4 groups give 20, and so on
    assert O.grouped_sizes(80, 10, 5) == [40, 20, 10, 5]


def test_first_experiment_of_section_4_2():
    # 1,600 points in 100 groups of 16, 8 centroids each: 800 at the first
    # level; the top level has fewer than lengthGroup centroids; with the data
    # layer the index is 8 layers deep
    sizes = O.grouped_sizes(1600, 16, 8)
    assert sizes[0] == 800 and sizes[-1] < 16
    assert len(sizes) + 1 == 8
    assert sizes == [800, 400, 200, 96, 48, 24, 8]


def test_fewer_points_than_a_group_build_nothing():
    assert O.grouped_sizes(15, 16, 8) == []


# ---------------------------------------------------------- split (R16)

def test_split_sizes_differ_by_at_most_one():
    for m, G in [(17, 3), (1600, 100), (200, 12), (35, 7)]:
        g = O.split_groups(m, G, O.level_state(5, 1))
        sizes = np.bincount(g, minlength=G)
        base, extra = divmod(m, G)
        assert sizes.tolist() == [base + 1] * extra + [base] * (G - extra)


def test_split_is_uniform_over_partitions():
    # 4 items into 2 groups of 2: each of the 3 unordered pairings (6 ordered
    # assignments) is equally likely over many seeds
    counts = {}
    for seed in range(6000):
        g = tuple(O.split_groups(4, 2, O.level_state(seed, 0)))
        counts[g] = counts.get(g, 0) + 1
    assert len(counts) == 6
    freq = np.array(list(counts.values())) / 6000
    assert np.all(np.abs(freq - 1 / 6) < 0.025), counts


# ------------------------------------------------ grouped build (R16-R18)

def _clouds(npc, sep, sigma, seed):
    r = np.random.default_rng(seed)
    ang = np.arange(8) * 2 * np.pi / 8
    centres = np.stack([np.cos(ang), np.sin(ang)], 1) * sep
    return np.concatenate([c + sigma * r.normal(size=(npc, 2)) for c in centres])


def test_each_group_is_its_own_kmeans():
    X = _clouds(25, 10.0, 1.0, 0)
    lg, nc, iters, seed = 10, 5, 6, 3
    idx = O.build_grouped(X, lg, nc, iters, seed)
    items = X
    for lv, C in enumerate(idx.centroids):
        m = len(items)
        G = m // lg
        groups = O.split_groups(m, G, O.level_state(seed, lv))
        for g in range(G):
            members = np.flatnonzero(groups == g)            # ascending item index
            st = O.group_state(seed, lv, g)
            _, C0 = O.kmeanspp(items[members], nc, st)
            Cg, lab, _ = O.lloyd(items[members], C0, iters)
            assert np.array_equal(C[g * nc:(g + 1) * nc], Cg), (lv, g)
            assert np.array_equal(idx.labels[lv][members], g * nc + lab), (lv, g)
        items = C


def test_grouped_levels_chain_and_labels_stay_in_their_group():
    X = _clouds(50, 5.0, 1.0, 1)
    idx = O.build_grouped(X, 16, 8, 5, 0, )
    assert [c.shape[0] for c in idx.centroids] == O.grouped_sizes(400, 16, 8)
    n_in = 400
    for lv, lab in enumerate(idx.labels):
        assert len(lab) == n_in
        assert lab.min() >= 0 and lab.max() < idx.centroids[lv].shape[0]
        n_in = idx.centroids[lv].shape[0]


def test_given_level0_groups_replace_the_split():
    X = _clouds(20, 8.0, 1.0, 2)
    n, lg, nc = len(X), 10, 4
    g0 = np.arange(n, dtype=np.int32) % (n // lg)
    idx = O.build_grouped(X, lg, nc, 4, 7, group0=g0)
    # every point's leaf centroid lies in the point's given group
    assert np.array_equal(idx.labels[0] // nc, g0)


# -------------------------------------------------------------- descent

def test_descend_reaches_the_leaf_the_query_scans():
    X = _clouds(30, 6.0, 1.5, 3)
    idx = O.build_grouped(X, 12, 6, 5, 1)
    Q = _clouds(5, 6.0, 1.5, 4)
    L = len(idx.centroids)
    for probes in ([1] * L, [3] + [2] * (L - 1)):
        leaf = O.descend(idx, Q, probes)
        ids, _, _ = idx.query(Q, 5, probes)
        for q in range(len(Q)):
            members = np.flatnonzero(np.isin(idx.labels[0], leaf[q][leaf[q] >= 0]))
            got = ids[q][ids[q] >= 0]
            assert set(got.tolist()) <= set(members.tolist())
            # and they are the nearest of those members
            d = ((X[members] - Q[q]) ** 2).sum(1)
            best = members[np.lexsort((members, d))][:len(got)]
            assert got.tolist() == best.tolist()


def test_descend_with_every_probe_keeps_every_leaf():
    X = _clouds(10, 4.0, 1.0, 5)
    idx = O.build_grouped(X, 8, 4, 3, 2)
    k = idx.k_per_level
    leaf = O.descend(idx, X[:7], k)
    for q in range(7):
        d = ((idx.centroids[0] - X[q]) ** 2).sum(1)
        order = np.lexsort((np.arange(len(d)), d))
        assert leaf[q].tolist() == order.tolist()


# ------------------------------------------------------- range (A3, R19)

def test_range_covering_everything_is_the_exact_range_set():
    X = _clouds(15, 5.0, 1.0, 6)
    idx = O.build_grouped(X, 10, 5, 4, 3)
    Q = X[:6] + 0.1
    r = 1e3   # every centroid and point is inside the ball
    res = O.range_query(idx, Q, r)
    for q, (ids, d) in enumerate(res):
        e = ((X - Q[q]) ** 2).sum(1)
        order = np.lexsort((np.arange(len(X)), e))
        assert ids.tolist() == order.tolist()
        assert np.allclose(d, e[order])


def test_range_results_are_inside_the_ball_and_sorted():
    X = _clouds(40, 6.0, 1.2, 7)
    idx = O.build(X, [64, 8], 6, 0)
    Q = _clouds(4, 6.0, 1.2, 8)
    for r in (0.5, 1.5, 3.0):
        for q, (ids, d) in enumerate(O.range_query(idx, Q, r)):
            exact = ((X[ids] - Q[q]) ** 2).sum(1)
            assert np.allclose(d, exact)
            assert np.all(d <= r * r)
            assert np.all(np.diff(d) >= 0)
            # found points are a subset of the exact ball
            ball = np.flatnonzero(((X - Q[q]) ** 2).sum(1) <= r * r)
            assert set(ids.tolist()) <= set(ball.tolist())


def test_range_hand_worked_two_levels():
    # points on a line: two top centroids at 0.5 and 10.5 after one cluster
    # per pair; a query at 0.2 with radius 1 keeps only the left branch
    X = np.array([[0.0], [1.0], [10.0], [11.0]])
    C0 = np.array([[0.5], [10.5]])
    C1 = np.array([[5.5]])
    idx = O.Index(X, [C0, C1], [np.array([0, 0, 1, 1], np.int32), np.array([0, 0], np.int32)])
    # radius 1 around 0.2: the top centroid (5.5) is outside the ball -> nothing
    assert O.range_query(idx, [[0.2]], 1.0)[0][0].tolist() == []
    # radius 6: top kept; children 0.5 (in) and 10.5 (out); points 0 and 1 in
    ids, d = O.range_query(idx, [[0.2]], 6.0)[0]
    assert ids.tolist() == [0, 1] and np.allclose(d, [0.04, 0.64])


# --------------------------------------------------- relocation (§4.1, R20)

def test_relocation_moves_only_missed_points_and_keeps_groups_large_enough():
    X = _clouds(40, 4.0, 2.0, 9)
    n, lg, nc = len(X), 16, 8
    idx = O.build_grouped(X, lg, nc, 5, 0)
    g0 = idx.labels[0] // nc
    leaf = O.descend(idx, X, [1] * len(idx.centroids))[:, 0]
    missed, g1, moved = O.relocate(idx, nc, g0)
    assert missed == int(np.sum(leaf != idx.labels[0]))
    changed = np.flatnonzero(g1 != g0)
    assert len(changed) == moved <= missed
    assert np.all(leaf[changed] // nc == g1[changed])        # moved to the reached group
    assert np.all(leaf[changed] != idx.labels[0][changed])   # only missed points move
    assert np.bincount(g1).min() >= nc
    # the rebuilt index honours the new groups
    idx2 = O.build_grouped(X, lg, nc, 5, 0, group0=g1)
    assert np.array_equal(idx2.labels[0] // nc, g1)
