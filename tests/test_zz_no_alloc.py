"""The allocation-free assignment entry point (mask_kmeans_assign_noalloc).

Some callers cannot let this library allocate device memory: frameworks that
reserve the GPU's memory up front and hand it out only through their own
allocator, and latency-critical loops that cannot absorb the synchronisation
an allocation may cause.  For them the library offers a variant of the
assignment step whose temporaries live in a file-scope device array.  This
file checks, through the C ABI, that it returns what the ordinary
(allocating) entry point returns, on two calls in a row that share that
array, and that it refuses inputs it cannot serve without allocating.  It is
named to be collected last, so a run that stops at the first failure has run
everything else already.
"""

import numpy as np
import pytest

from paper_2208_02734_gb300 import mask as M

from parity_util import RTOL, check_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _data(n, d, k, seed):
    rng = np.random.default_rng(seed)
    X = (rng.normal(size=(n, d)) * 3 + rng.uniform(-10, 10, size=(1, d))).astype(np.float32)
    Cc = (X[rng.choice(n, k, replace=False)] + 0.05 * rng.normal(size=(k, d))).astype(np.float32)
    return torch.from_numpy(X).cuda(), torch.from_numpy(Cc).cuda()


def _same_as_allocating_path(X, Cc):
    lab_ref, dist_ref = M.mask_kmeans_assign(X, Cc)
    lab = torch.full((X.shape[0],), -7, dtype=torch.int32, device=X.device)
    dist = torch.full((X.shape[0],), -1.0, dtype=torch.float32, device=X.device)
    M.mask_kmeans_assign_noalloc(X, Cc, lab, dist)
    torch.cuda.synchronize()
    lab_n, lab_r = lab.cpu().numpy(), lab_ref.cpu().numpy()
    diff = np.flatnonzero(lab_n != lab_r)
    if len(diff):  # only ties within the tolerance may differ
        x = X.cpu().double().numpy()[diff]
        c = Cc.cpu().double().numpy()
        dn = ((x - c[lab_n[diff]]) ** 2).sum(1)
        dr = ((x - c[lab_r[diff]]) ** 2).sum(1)
        assert np.all(np.abs(dn - dr) <= RTOL * np.maximum(dn, dr))
    check_close(dist.cpu().numpy(), dist_ref.cpu().numpy(), rtol=RTOL, atol=1e-30,
                what="no-alloc distances")


def test_noalloc_assign_matches_the_allocating_entry_point_on_two_calls():
    # first call: more rows than one internal chunk (262,144) and many centroids
    X1, C1 = _data(300_000, 16, 2000, seed=1)
    _same_as_allocating_path(X1, C1)
    # second call reuses the same scratch with other sizes
    X2, C2 = _data(5_000, 64, 300, seed=2)
    _same_as_allocating_path(X2, C2)


def test_noalloc_assign_makes_no_library_allocation():
    X, Cc = _data(20_000, 32, 500, seed=4)
    lab = torch.empty(20_000, dtype=torch.int32, device="cuda")
    dist = torch.empty(20_000, dtype=torch.float32, device="cuda")
    M.mask_kmeans_assign_noalloc(X, Cc, lab, dist)   # the first call may look up the scratch
    torch.cuda.synchronize()
    before = M.mask_test_alloc_count()
    for _ in range(2):
        M.mask_kmeans_assign_noalloc(X, Cc, lab, dist)
    torch.cuda.synchronize()
    assert M.mask_test_alloc_count() == before
    # the allocating entry point does move the counter (the hook works)
    M.mask_kmeans_assign(X, Cc)
    torch.cuda.synchronize()
    assert M.mask_test_alloc_count() > before


def test_noalloc_assign_refuses_what_it_cannot_serve_without_allocating():
    X, Cc = _data(1000, 16, 10, seed=3)
    lab = torch.empty(1000, dtype=torch.int32, device="cuda")
    with pytest.raises(M.MaskError) as e:  # more centroids than the scratch holds
        big = torch.zeros((65537, 16), dtype=torch.float32, device="cuda")
        M.mask_kmeans_assign_noalloc(X, big, lab)
    assert e.value.status == M.MASK_EINVAL and "65536" in str(e.value)
    # host memory would need staging buffers: the C side refuses it (the
    # binding already refuses CPU tensors before the call)
    Xh, Ch, lh = X.cpu(), Cc.cpu(), lab.cpu()
    st = M.load().mask_kmeans_assign_noalloc(Xh.data_ptr(), 1000, 16, Ch.data_ptr(), 10,
                                             lh.data_ptr(), None, None)
    assert st == M.MASK_EINVAL and "device memory" in M.mask_last_error()
    with pytest.raises(ValueError):
        M.mask_kmeans_assign_noalloc(Xh, Ch, lh)
    with pytest.raises(M.MaskError):  # rows must be usable in place
        M.mask_kmeans_assign_noalloc(X[:, :12].contiguous(), Cc[:, :12].contiguous(), lab)
    before = M.mask_test_alloc_count()
    lab = torch.empty(1000, dtype=torch.int32, device="cuda")
    for bad in (
        lambda: M.mask_kmeans_assign_noalloc(X, Cc[:, :8].contiguous(), lab),   # d mismatch
        lambda: M.mask_kmeans_assign_noalloc(X, Cc, lab[:999]),                # short labels
        lambda: M.mask_kmeans_assign_noalloc(X, Cc, lab.long()),               # int64 labels
        lambda: M.mask_kmeans_assign_noalloc(X, Cc, lab, lab.float()[:10]),    # short dist
        lambda: M.mask_kmeans_assign_noalloc(X.double(), Cc, lab),             # float64 rows
        lambda: M.mask_kmeans_assign_noalloc(X.t(), Cc, lab),                  # non-contiguous
    ):
        with pytest.raises(ValueError):
            bad()
    assert M.mask_test_alloc_count() == before
