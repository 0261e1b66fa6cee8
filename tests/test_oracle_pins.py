"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: they use hand-worked examples
(tests/golden/), published generator outputs, closed-form probabilities,
invariants (Lloyd's monotone objective, probe-everything == exact search) and
brute force on tiny inputs, each chosen so that a dropped term, a wrong index
or a flipped comparison in the oracle fails at least one of them.
"""

import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2208_02734_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ------------------------------------------------------------------ R1: RNG

def test_splitmix64_reference_vectors():
    g = _golden("splitmix64.json")
    for v in g["vectors"]:
        r = O.SplitMix64(v["state"])
        assert [r.next() for _ in v["outputs"]] == [int(x) for x in v["outputs"]]


def test_uniform_draws_lie_in_unit_interval_and_are_uniform():
    r = O.SplitMix64(O.level_state(3, 1))
    u = np.array([r.uniform() for _ in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    hist = np.histogram(u, bins=10, range=(0, 1))[0]
    assert np.all(np.abs(hist - 2000) < 5 * math.sqrt(2000))


# ------------------------------------------------------------ R2: k-means++

def test_kmeanspp_hand_worked_1d():
    # draws of state 7: 0.38983, 0.016788, 0.90076, 0.58293
    # first = floor(0.38983 * 4) = 1 (x=1); D2 = [1,0,4,36], S=41,
    # target 0.688 -> prefix 1 at i=0 exceeds it -> pick 0;
    # D2 = [0,0,4,36], S=40, target 36.03 -> prefix reaches 40 at i=3 -> pick 3;
    # D2 = [0,0,4,0], S=4, target 2.33 -> pick 2.
    X = np.array([[0.0], [1.0], [3.0], [7.0]])
    chosen, C = O.kmeanspp(X, 4, state=7)
    assert chosen.tolist() == [1, 0, 3, 2]
    assert C[:, 0].tolist() == [1.0, 0.0, 7.0, 3.0]


def test_kmeanspp_never_picks_a_zero_probability_point():
    # SplitMix64's mixer maps 0 to 0, so from state -2*gamma the second draw
    # is exactly 0.0 and the target u*S is 0.  Draws: 0.20076, 0.0, 0.88331.
    # first = floor(0.2008 * 4) = 0; D2 = [0,0,16,81]; target 0: the first
    # prefix that EXCEEDS 0 is at i=2 (i=0,1 have probability 0);
    # D2 = [0,0,0,25], target 22.08 -> pick 3.
    gamma = 0x9E3779B97F4A7C15
    state = (-2 * gamma) & 0xFFFFFFFFFFFFFFFF
    r = O.SplitMix64(state)
    assert r.uniform() == pytest.approx(0.20076011277725214) and r.uniform() == 0.0
    X = np.array([[0.0], [0.0], [4.0], [9.0]])
    chosen, _ = O.kmeanspp(X, 3, state=state)
    assert chosen.tolist() == [0, 2, 3]


def test_kmeanspp_k_equals_n_selects_every_point():
    rng = np.random.default_rng(5)
    X = rng.normal(size=(17, 3))
    for s in range(5):
        chosen, C = O.kmeanspp(X, 17, state=s)
        assert sorted(chosen.tolist()) == list(range(17))
        np.testing.assert_array_equal(C, X[chosen])


def test_kmeanspp_second_pick_is_proportional_to_squared_distance():
    # points 0, 1, 3 on a line: given the first centre, the second is drawn
    # with probability D^2 / sum D^2 (closed form below)
    X = np.array([[0.0], [1.0], [3.0]])
    expect = {0: {1: 1 / 10, 2: 9 / 10}, 1: {0: 1 / 5, 2: 4 / 5}, 2: {0: 9 / 13, 1: 4 / 13}}
    counts = {f: {} for f in expect}
    firsts = np.zeros(3)
    trials = 12000
    for s in range(trials):
        chosen, _ = O.kmeanspp(X, 2, state=1000 + 7919 * s)
        f, g = int(chosen[0]), int(chosen[1])
        firsts[f] += 1
        counts[f][g] = counts[f].get(g, 0) + 1
    assert np.all(np.abs(firsts / trials - 1 / 3) < 0.02)
    for f, probs in expect.items():
        tot = sum(counts[f].values())
        for g, p in probs.items():
            assert abs(counts[f].get(g, 0) / tot - p) < 0.03, (f, g)


def test_kmeanspp_duplicates_fall_back_to_lowest_unchosen():
    X = np.array([[0.0], [0.0], [0.0], [5.0]])
    for s in range(20):
        chosen, C = O.kmeanspp(X, 4, state=s)
        assert sorted(chosen.tolist()) == [0, 1, 2, 3]
        # once the value 5 and one zero are centres, S = 0: lowest unchosen next
        rest = chosen[2:].tolist()
        assert rest == sorted(rest)


# -------------------------------------------------- R3: seeding subsample

def test_fisher_yates_partial_is_uniform_over_ordered_pairs():
    counts = {}
    trials = 20000
    for s in range(trials):
        a, b = O.subsample(5, 2, state=31 * s + 11).tolist()
        assert a != b and 0 <= a < 5 and 0 <= b < 5
        counts[(a, b)] = counts.get((a, b), 0) + 1
    assert len(counts) == 20
    for c in counts.values():
        assert abs(c / trials - 1 / 20) < 0.008


def test_fisher_yates_full_is_a_permutation():
    out = O.subsample(50, 50, state=9)
    assert sorted(out.tolist()) == list(range(50))


def test_seed_sample_size_reading():
    assert O.seed_sample_size(10_000_000, 32768) == 262144   # 3.3e11 > 2^32
    assert O.seed_sample_size(20_000, 200) == 20_000
    assert O.seed_sample_size(1_000_000, 4096) == 1_000_000  # 4.1e9 < 2^32
    assert O.seed_sample_size(32768, 1024) == 32768


@pytest.mark.slow
def test_seed_level_subsample_path_matches_its_definition():
    n, k = 4_200_000, 1024          # n*k = 4.3e9 > 2^32, 8k < n
    X = np.arange(n, dtype=np.float64)[:, None] * 1e-3
    chosen, C = O.seed_level(X, k, seed=5, level=0)
    state = O.level_state(5, 0)
    m = 8 * k
    sample = O.subsample(n, m, state)
    r = O.SplitMix64(state)
    for _ in range(m):
        r.next()
    ch_sub, C_sub = O.kmeanspp(X[sample], k, state=r.state.value)
    assert chosen.tolist() == sample[ch_sub].tolist()
    np.testing.assert_array_equal(C, C_sub)


# ------------------------------------------------------------- R4: Lloyd

@pytest.mark.parametrize("case", _golden("lloyd_2d.json")["cases"], ids=lambda c: c["name"])
def test_lloyd_hand_worked(case):
    X = np.array(case["points"], float)
    C, labels, J = O.lloyd(X, np.array(case["init"], float), case["iters"])
    np.testing.assert_array_equal(C, np.array(case["centroids"], float))
    assert labels.tolist() == case["labels"]
    np.testing.assert_array_equal(J, np.array(case["objective_trace"]))


def test_lloyd_objective_never_increases():
    mix = synth.IsotropicMixture(d=5, n_blobs=6, sigma=2.0, seed=2)
    X = mix.sample(3000, seed=3)
    for s in range(3):
        _, C0 = O.kmeanspp(X, 40, state=s)
        _, _, J = O.lloyd(X, C0, 12)
        assert np.all(np.diff(J) <= 1e-9 * J[0]), J


def test_lloyd_converged_state_is_a_fixed_point():
    rng = np.random.default_rng(1)
    X = np.concatenate([rng.normal(c, 0.3, size=(200, 2)) for c in ((0, 0), (5, 0), (0, 5))])
    _, C0 = O.kmeanspp(X, 3, state=4)
    C, labels, _ = O.lloyd(X, C0, 30)
    for j in range(3):
        np.testing.assert_allclose(C[j], X[labels == j].mean(axis=0), rtol=1e-12, atol=1e-12)
    D = ((X[:, None, :] - C[None, :, :]) ** 2).sum(-1)
    assert np.array_equal(labels, D.argmin(1))


# ------------------------------------------------- multilevel build (A1)

def test_build_levels_feed_each_other():
    mix = synth.IsotropicMixture(d=4, n_blobs=5, seed=0)
    X = mix.sample(2000, seed=1).astype(np.float64)
    idx = O.build(X, [60, 8], iters=5, seed=11)
    assert [c.shape for c in idx.centroids] == [(60, 4), (8, 4)]
    assert [len(lb) for lb in idx.labels] == [2000, 60]
    # level 1 (0-based) is seeded from level 0's centroids with its own stream
    chosen, C1 = O.seed_level(idx.centroids[0], 8, seed=11, level=1)
    assert chosen.tolist() == idx.chosen[1].tolist()
    C, lab, _ = O.lloyd(idx.centroids[0], C1, 5)
    np.testing.assert_array_equal(C, idx.centroids[1])
    np.testing.assert_array_equal(lab, idx.labels[1])


def test_one_to_one_ratio_makes_every_point_a_centroid():
    # 1:1 ratio (Sec. 5): with k_1 = N every point is its own cluster
    rng = np.random.default_rng(8)
    X = rng.normal(size=(120, 3))
    idx = O.build(X, [120, 10], iters=3, seed=2)
    assert sorted(map(tuple, idx.centroids[0])) == sorted(map(tuple, X))
    assert len(set(idx.labels[0].tolist())) == 120
    Q = rng.normal(size=(30, 3))
    ids, d, _ = idx.query(Q, 5, probes=[5, 10])
    bids, bd = O.bruteforce_knn(X, Q, 5)
    assert np.array_equal(ids, bids) and np.array_equal(d, bd)


# --------------------------------------------------- R5: top-down k-NN

def test_descent_hand_worked():
    g = _golden("descent_2d.json")
    idx = O.Index(g["points"], [g["level1_centroids"], g["level2_centroids"]],
                  [g["level1_labels"], g["level2_labels"]])
    for c in g["queries"]:
        ids, d, clear = idx.query(np.array([c["q"]], float), c["k"], c["probes"])
        assert ids[0].tolist() == c["ids"], c
        assert d[0].tolist() == [math.inf if x == "inf" else x for x in c["dists"]], c
        assert bool(clear[0]) == c["sel_clear"], c


def test_probe_everything_is_exact_knn():
    mix = synth.IsotropicMixture(d=6, n_blobs=4, seed=5)
    X = mix.sample(1500, seed=6)
    Q = mix.sample(60, seed=7)
    idx = O.build(X, [50, 7], iters=4, seed=1)
    ids, d, _ = idx.query(Q, 10, probes=[50, 7])
    bids, bd = O.bruteforce_knn(X, Q, 10)
    assert np.array_equal(ids, bids)
    assert np.array_equal(d, bd)


def test_bruteforce_matches_full_sort():
    rng = np.random.default_rng(0)
    X = rng.integers(0, 4, size=(150, 2)).astype(float)   # many exact ties
    Q = rng.integers(0, 4, size=(12, 2)).astype(float)
    ids, d = O.bruteforce_knn(X, Q, 9)
    for qi in range(len(Q)):
        dd = np.array([sum((X[i, t] - Q[qi, t]) ** 2 for t in range(2)) for i in range(len(X))])
        order = np.lexsort((np.arange(len(X)), dd))[:9]
        assert ids[qi].tolist() == order.tolist()
        assert d[qi].tolist() == dd[order].tolist()


def test_fewer_candidates_than_k_pads():
    X = np.array([[0.0, 0.0], [1.0, 0.0], [10.0, 0.0]])
    idx = O.Index(X, [[[0.5, 0.0], [10.0, 0.0]], [[5.0, 0.0]]], [[0, 0, 1], [0, 0]])
    ids, d, _ = idx.query(np.array([[0.0, 0.0]]), 4, probes=[1, 1])
    assert ids[0].tolist() == [0, 1, -1, -1]
    assert d[0].tolist() == [0.0, 1.0, math.inf, math.inf]


def test_probes_larger_than_level_are_clamped():
    X = np.array([[0.0], [1.0], [2.0], [3.0]])
    idx = O.Index(X, [[[0.5], [2.5]], [[1.5]]], [[0, 0, 1, 1], [0, 0]])
    ids, _, _ = idx.query(np.array([[2.9]]), 4, probes=[9, 9])
    assert ids[0].tolist() == [3, 2, 1, 0]


def test_results_do_not_depend_on_thread_count():
    mix = synth.IsotropicMixture(d=8, n_blobs=5, seed=1)
    X = mix.sample(3000, seed=2)
    Q = mix.sample(100, seed=3)
    try:
        O.set_threads(1)
        idx1 = O.build(X, [40, 6], iters=4, seed=3)
        r1 = idx1.query(Q, 10, [3, 2])
        O.set_threads(max(2, os.cpu_count() or 2))
        idx2 = O.build(X, [40, 6], iters=4, seed=3)
        r2 = idx2.query(Q, 10, [3, 2])
    finally:
        O.set_threads(os.cpu_count() or 1)
    for a, b in zip(idx1.centroids, idx2.centroids):
        assert np.array_equal(a, b)
    assert all(np.array_equal(a, b) for a, b in zip(r1, r2))


def test_point_query_error_is_small_on_separated_clouds():
    # Sec. 4.2: point search finds nearly every point of well-separated
    # Gaussian clouds (Table 3: at most 0.11 % missed).  A sanity band, not
    # an exact pin: the clouds and the index shape here are our own.
    rng = np.random.default_rng(0)
    centres = rng.uniform(-50, 50, size=(8, 2))
    X = np.concatenate([rng.normal(c, 1.0, size=(200, 2)) for c in centres])
    idx = O.build(X, [400, 25], iters=10, seed=0)
    ids, _, _ = idx.query(X, 1, probes=[1, 1])
    err1 = np.mean(ids[:, 0] != np.arange(len(X)))
    ids, _, _ = idx.query(X, 1, probes=[3, 3])
    err3 = np.mean(ids[:, 0] != np.arange(len(X)))
    assert err1 < 0.10 and err3 <= err1
