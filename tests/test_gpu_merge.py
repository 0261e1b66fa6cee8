"""The exchange step of the distributed design (§3.4) on one GPU: G
partitions emulated by G indexes over disjoint slices of the points, each
queried on its own, merged by mask_merge_topk into the k-NN over the union."""

import numpy as np
import pytest

import oracle as O
from paper_2208_02734_gb300 import dist as D
from paper_2208_02734_gb300 import mask as M
from paper_2208_02734_gb300 import synth

from parity_util import RTOL, arr, check_knn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("G,k", [(2, 10), (3, 7), (8, 100)])
def test_partitioned_indexes_merge_to_the_exact_union(G, k):
    mix = synth.IsotropicMixture(d=16, n_blobs=6, seed=0)
    X = mix.sample(8000, seed=0)
    Q = mix.sample(64, seed=1)
    Qd = cuda(Q)
    ids, dists, offs = [], [], []
    for r in range(G):
        a, b = D.partition_range(len(X), G, r)
        with M.mask_build(cuda(X[a:b]), [40, 5], 5, seed=r) as idx:
            i, d = M.mask_query(idx, Qd, k, [40, 5])        # every probe: exact per partition
        ids.append(i)
        dists.append(d)
        offs.append(a)
    got_i, got_d = M.mask_merge_topk(torch.stack(ids), torch.stack(dists), cuda(np.array(offs)))
    gt_i, gt_d = O.bruteforce_knn(X, Q, k)
    check_knn(X, Q, got_i, got_d, gt_i, gt_d, np.ones(len(Q), bool))


def test_merge_kernel_against_a_sort():
    rng = np.random.default_rng(4)
    G, nq, k = 5, 33, 13
    d = np.sort(rng.random((G, nq, k)).astype(np.float32), axis=2)
    i = rng.integers(0, 1000, size=(G, nq, k)).astype(np.int64)
    d[1, :, 9:] = np.inf                     # padded tails
    i[1, :, 9:] = -1
    d[2, 3] = d[0, 3]                        # equal distances: ids decide
    offs = np.arange(G, dtype=np.int64) * 1000
    got_i, got_d = M.mask_merge_topk(cuda(i), cuda(d), cuda(offs))
    host_i, host_d = M.mask_merge_topk(i, d, offs)          # host buffers
    assert np.array_equal(arr(got_i), host_i) and np.array_equal(arr(got_d), host_d)
    for q in range(nq):
        gi = np.where(i[:, q] >= 0, i[:, q] + offs[:, None], -1).reshape(-1)
        gd = d[:, q].reshape(-1)
        valid = gi >= 0
        order = np.lexsort((gi[valid], gd[valid]))[:k]
        assert arr(got_i)[q].tolist() == gi[valid][order].tolist()
        assert np.array_equal(arr(got_d)[q], gd[valid][order])


def test_merge_pads_when_the_partitions_hold_fewer_than_k():
    i = np.full((2, 1, 4), -1, np.int64)
    d = np.full((2, 1, 4), np.inf, np.float32)
    i[0, 0, 0], d[0, 0, 0] = 3, 0.5
    got_i, got_d = M.mask_merge_topk(i, d, np.array([0, 10]))
    assert got_i.tolist() == [[3, -1, -1, -1]]
    assert got_d[0, 0] == np.float32(0.5) and np.all(np.isinf(got_d[0, 1:]))
    with pytest.raises(M.MaskError):
        M.mask_merge_topk(np.zeros((2, 1, 9000), np.int64), np.zeros((2, 1, 9000), np.float32))
