"""Comparison rules between the CUDA path and the FP64 oracle.

Tolerance (FP32 mode): a GPU label or neighbour id must equal the oracle's,
except where the oracle's own distances show a near-tie (relative gap below
RTOL = 1e-5); distances and centroids must agree within RTOL relative.
"""

import numpy as np

import oracle as O

RTOL = 1e-5


def f64(a):
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.asarray(a, dtype=np.float64)


def arr(a):
    if hasattr(a, "detach"):
        return a.detach().cpu().numpy()
    return np.asarray(a)


def check_labels(X, Cc, lab_g, lab_o, rtol=RTOL):
    """GPU labels equal the oracle's except on oracle-side near-ties.
    Returns the number of (tolerated) differences."""
    X, Cc = f64(X), f64(Cc)
    lab_g, lab_o = arr(lab_g).astype(np.int64), arr(lab_o).astype(np.int64)
    assert lab_g.shape == lab_o.shape
    assert lab_g.min() >= 0 and lab_g.max() < len(Cc)
    diff = np.flatnonzero(lab_g != lab_o)
    for i in diff:
        dg, do = O.sqdist_rows(Cc, [lab_g[i], lab_o[i]], X[i])
        assert dg <= do * (1 + rtol) + 1e-30, (i, lab_g[i], lab_o[i], dg, do)
    return len(diff)


def check_rows_close(A_g, A_o, rtol=RTOL, what="rows"):
    """Row-wise relative error: max_t |a_g - a_o| <= rtol * max_t |a_o| (+ tiny)."""
    A_g, A_o = f64(A_g), f64(A_o)
    assert A_g.shape == A_o.shape
    scale = np.abs(A_o).max(axis=1, keepdims=True)
    err = np.abs(A_g - A_o)
    bad = err > rtol * scale + 1e-30
    assert not bad.any(), (what, np.argwhere(bad)[:5], err[bad][:5])


def check_close(a_g, a_o, rtol=RTOL, atol=0.0, what="values"):
    a_g, a_o = f64(a_g), f64(a_o)
    fin = np.isfinite(a_o)
    assert np.array_equal(fin, np.isfinite(a_g)), what
    err = np.abs(a_g[fin] - a_o[fin])
    bad = err > rtol * np.abs(a_o[fin]) + atol
    assert not bad.any(), (what, err[bad][:5], a_o[fin][bad][:5])


def check_knn(X, Q, ids_g, d_g, ids_o, d_o, clear, rtol=RTOL):
    """Compare GPU k-NN results with the oracle's (same index, same queries).

    Queries whose kept sets were decided without near-ties (clear) must return
    the oracle's ids except for near-tie swaps, with distances within rtol.
    Others (a near-tie picked a different centroid) must return valid results:
    distinct ids, correct distances, ascending order.  Returns the number of
    queries checked for validity only."""
    X, Q = f64(X), f64(Q)
    ids_g, d_g = arr(ids_g).astype(np.int64), f64(d_g)
    ids_o, d_o = arr(ids_o).astype(np.int64), f64(d_o)
    loose = 0
    for q in range(len(Q)):
        ok = ids_g[q] >= 0
        gi = ids_g[q][ok]
        assert len(set(gi.tolist())) == len(gi), ("duplicate ids", q)
        assert np.all(np.diff(d_g[q][ok]) >= 0), ("not ascending", q)
        exact = O.sqdist_rows(X, gi, Q[q]) if len(gi) else np.zeros(0)
        check_close(d_g[q][ok], exact, rtol=rtol, atol=1e-30, what=f"dist of returned ids q={q}")
        if clear[q]:
            assert np.array_equal(ok, ids_o[q] >= 0), ("padding differs", q)
            check_close(d_g[q], d_o[q], rtol=rtol, atol=1e-30, what=f"dists q={q}")
            for r in np.flatnonzero(ids_g[q] != ids_o[q]):
                dg, do = O.sqdist_rows(X, [ids_g[q][r], ids_o[q][r]], Q[q])
                assert abs(dg - do) <= rtol * max(dg, do) + 1e-30, ("id swap", q, r, dg, do)
        else:
            loose += 1
    return loose
