"""The seeded input generators (shared by the oracle-side and GPU-side tests).

The sparse generator's contract: log-normal row lengths with the stated
arithmetic mean, Zipf-distributed column ids drawn without replacement within
a row (successive sampling), sorted unique columns, unit-norm rows.
"""

import itertools

import numpy as np

from paper_2208_02734_gb300 import synth


def test_sparse_rows_are_well_formed():
    A = synth.sparse_tfidf_like(5000, 700, nnz_mean=30.0, seed=3)
    assert A.row_ptr[0] == 0 and np.all(np.diff(A.row_ptr) >= 1)
    for i in range(0, A.n_rows, 7):
        c = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0) and c.min() >= 0 and c.max() < 700
    sq = np.add.reduceat(A.val.astype(np.float64) ** 2, A.row_ptr[:-1])
    assert np.allclose(sq, 1.0, atol=1e-6)
    assert np.all(A.val > 0)


def test_sparse_row_lengths_are_lognormal_with_the_stated_mean():
    A = synth.sparse_tfidf_like(40_000, 20_000, nnz_mean=60.0, nnz_sigma=0.8, seed=0,
                                chunk=1 << 14)
    m = np.diff(A.row_ptr)
    assert abs(m.mean() - 60.0) < 1.0
    assert abs(np.log(m).std() - 0.8) < 0.03


def test_sparse_columns_follow_successive_zipf_sampling():
    # every row has exactly 2 columns out of 5 (sigma ~ 0): the probability of
    # the unordered pair {a, b} is p_a p_b / (1 - p_a) + p_b p_a / (1 - p_b)
    d, n = 5, 40_000
    A = synth.sparse_tfidf_like(n, d, nnz_mean=2.0, nnz_sigma=1e-9, zipf_s=1.0, seed=11)
    assert np.all(np.diff(A.row_ptr) == 2)
    vocab = np.random.default_rng([0, 0x70CA]).permutation(d)
    w = 1.0 / np.arange(1, d + 1)
    p = w / w.sum()
    pairs = A.col.reshape(-1, 2)
    for a, b in itertools.combinations(range(d), 2):
        ca, cb = sorted((vocab[a], vocab[b]))
        got = np.mean((pairs[:, 0] == ca) & (pairs[:, 1] == cb))
        want = p[a] * p[b] / (1 - p[a]) + p[b] * p[a] / (1 - p[b])
        assert abs(got - want) < 5 * np.sqrt(want * (1 - want) / n) + 1e-4, (a, b, got, want)


def test_sparse_generator_is_seeded_and_chunking_does_not_matter_for_shape():
    A = synth.sparse_tfidf_like(3000, 400, nnz_mean=20.0, seed=5)
    B = synth.sparse_tfidf_like(3000, 400, nnz_mean=20.0, seed=5)
    assert np.array_equal(A.row_ptr, B.row_ptr) and np.array_equal(A.col, B.col)
    assert np.array_equal(A.val, B.val)
    C = synth.sparse_tfidf_like(3000, 400, nnz_mean=20.0, seed=6)
    assert not np.array_equal(A.col[:100], C.col[:100])


def test_csr_rows_and_densify():
    A = synth.sparse_tfidf_like(50, 30, nnz_mean=5.0, seed=0)
    D = A.to_dense()
    sub = A.rows([3, 0, 49])
    assert np.array_equal(sub.to_dense(), D[[3, 0, 49]])
