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


def test_noalloc_assign_refuses_what_it_cannot_serve_without_allocating():
    X, Cc = _data(1000, 16, 10, seed=3)
    lab = torch.empty(1000, dtype=torch.int32, device="cuda")
    with pytest.raises(M.MaskError) as e:  # more centroids than the scratch holds
        big = torch.zeros((65537, 16), dtype=torch.float32, device="cuda")
        M.mask_kmeans_assign_noalloc(X, big, lab)
    assert e.value.status == M.MASK_EINVAL and "65536" in str(e.value)
    with pytest.raises(M.MaskError):  # host memory would need staging buffers
        M.mask_kmeans_assign_noalloc(X.cpu(), Cc.cpu(), lab.cpu())
    with pytest.raises(M.MaskError):  # rows must be usable in place
        M.mask_kmeans_assign_noalloc(X[:, :12].contiguous(), Cc[:, :12].contiguous(), lab)
