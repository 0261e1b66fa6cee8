"""Full-size checks: the 10,000,000 x 64 workload (1,000 anisotropic blobs,
Zipf 1.1 weights), index 32,768 / 1,024 / 32 with 15 Lloyd iterations, built
and queried through the same calls bench.py times.

At this size the oracle cannot rebuild the index, so the checks are on sampled
outputs the oracle computes one by one, and on properties that hold at any
size:
  - the first k-means++ picks of level 0 equal the oracle's on the same
    seeded subsample (8k of the 10^7 points, partial Fisher-Yates);
  - each level's objective after every assignment never increases;
  - sampled labels are the oracle's argmin over the built centroids (up to
    near-ties);
  - one update step of all 10^7 points under the built labels gives the
    oracle's mean for sampled clusters (teacher-forced);
  - returned distances of sampled queries equal the oracle's exact distances
    of the returned ids, results are ascending, the ids are those of the
    oracle's descent over the GPU-built index (up to near-tie swaps), and
    recall@10 against the oracle's exact k-NN meets the operating point's
    level;
  - both leaf scans give bit-identical results at this size.
"""

import numpy as np
import pytest

import oracle as O
from paper_2208_02734_gb300 import mask as M
from paper_2208_02734_gb300 import synth

from parity_util import RTOL, arr, check_close, check_knn, check_labels, check_rows_close

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

N, D, KPL, ITERS = 10_000_000, 64, [32768, 1024, 32], 15
PROBES = [96, 16, 4]   # the bench's operating point for recall@10 >= 0.95


@pytest.fixture(scope="module")
def built():
    mix = synth.AnisotropicMixture(d=D, n_blobs=1000, seed=0)
    X = mix.sample(N, seed=0)
    Q = mix.sample(10_000, seed=1)
    Xd = torch.from_numpy(X).cuda()
    Qd = torch.from_numpy(Q).cuda()
    idx = M.mask_build(Xd, KPL, ITERS, seed=0)
    yield X, Q, Xd, Qd, idx
    idx.free()


def test_first_kmeanspp_picks_match_oracle(built):
    X, _, _, _, idx = built
    e = M.mask_index_export_level(idx, 0)
    k = KPL[0]
    m = O.seed_sample_size(N, k)
    assert m == 8 * k
    state = O.level_state(0, 0)
    sample = O.subsample(N, m, state)
    r = O.SplitMix64(state)
    for _ in range(m):
        r.next()
    ch_sub, _ = O.kmeanspp(X[sample], 200, state=r.state.value)
    assert e["chosen"][:200].tolist() == sample[ch_sub].tolist()


def test_objective_never_increases(built):
    _, _, _, _, idx = built
    for lv in range(len(KPL)):
        J = M.mask_index_export_level(idx, lv)["objective"]
        assert len(J) == ITERS + 1
        assert np.all(np.diff(J) <= 1e-5 * J[0]), (lv, J)


def test_sampled_labels_are_the_oracle_argmin(built):
    X, _, _, _, idx = built
    e = M.mask_index_export_level(idx, 0)
    C = arr(e["centroids"])
    lab = arr(e["labels"])
    rows = np.random.default_rng(0).choice(N, 2000, replace=False)
    lab_o, _ = O.assign(X[rows], C.astype(np.float64))
    check_labels(X[rows], C, lab[rows], lab_o)


def test_full_size_update_step_on_sampled_clusters(built):
    # teacher-forced: the update of all 10^7 points under the built index's
    # final labels, checked cluster by cluster against the oracle's mean
    X, _, Xd, _, idx = built
    e = M.mask_index_export_level(idx, 0, device="cuda")
    C_new, cnt = M.mask_kmeans_update(Xd, e["labels"], e["centroids"])
    C_new, cnt, lab = arr(C_new), arr(cnt), arr(e["labels"])
    assert cnt.sum() == N and np.array_equal(cnt, np.bincount(lab, minlength=KPL[0]))
    order = np.argsort(lab, kind="stable")
    start = np.concatenate([[0], np.cumsum(cnt)])
    rng = np.random.default_rng(1)
    sample = np.concatenate([rng.choice(KPL[0], 60, replace=False),
                             np.argsort(cnt)[-4:]])   # and the largest clusters
    for j in sample:
        members = order[start[j]:start[j + 1]]
        C_o, _ = O.update(X[members], np.zeros(len(members), np.int32),
                          arr(e["centroids"])[j:j + 1].astype(np.float64))
        check_rows_close(C_new[j:j + 1], C_o, what=f"cluster {j} ({len(members)} members)")


def test_sampled_queries_against_oracle(built):
    X32, Q, _, Qd, idx = built
    X = X32.astype(np.float64)   # once: the oracle helpers take FP64 rows
    ids, dists = M.mask_query(idx, Qd, 10, PROBES)
    ids, dists = arr(ids), arr(dists)
    sel = np.arange(0, len(Q), len(Q) // 40)[:40]
    for q in sel:
        assert np.all(np.diff(dists[q]) >= 0)
        ok = ids[q] >= 0
        exact = O.sqdist_rows(X, ids[q][ok], Q[q])
        check_close(dists[q][ok], exact, rtol=RTOL, atol=1e-30, what=f"query {q}")
    # the oracle's descent (Algorithm 2, p_l kept per level) over the very
    # index the GPU built: same ids except near-tie swaps
    levels = [M.mask_index_export_level(idx, lv) for lv in range(len(KPL))]
    oidx = O.Index(X, [arr(lv["centroids"]).astype(np.float64) for lv in levels],
                   [arr(lv["labels"]) for lv in levels])
    ids_o, d_o, clear = oidx.query(Q[sel], 10, PROBES)
    loose = check_knn(X, Q[sel], ids[sel], dists[sel], ids_o, d_o, clear)
    assert loose <= len(sel) // 4, loose
    gt_ids, gt_d = O.bruteforce_knn(X, Q[sel], 10)
    hits = 0
    for i, q in enumerate(sel):
        exact = O.sqdist_rows(X, np.maximum(ids[q], 0), Q[q])
        hits += int(np.sum((ids[q] >= 0) & (exact <= gt_d[i, -1] * (1 + RTOL))))
    recall = hits / (10 * len(sel))
    assert recall >= 0.90, recall   # the 200-query estimate of the bench is 0.957


def test_leaf_scans_agree_at_full_size(built, monkeypatch):
    _, _, _, Qd, idx = built
    out = {}
    for leaf in ["query", "cluster"]:
        monkeypatch.setenv("MASK_LEAF_SCAN", leaf)
        out[leaf] = M.mask_query(idx, Qd[:500], 10, PROBES)
    assert torch.equal(out["query"][0], out["cluster"][0])
    assert torch.equal(out["query"][1], out["cluster"][1])
