"""Failure detection on the GPU without a fault: the library's device-side
waits are bounded and report instead of hanging.  A wait on a flag that
nothing sets runs out, returns MASK_ETIMEOUT, and leaves the context usable;
the same wait on a flag set before the launch returns MASK_OK."""

import numpy as np
import pytest

from paper_2208_02734_gb300 import mask as M

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_a_wait_that_runs_out_reports_and_the_context_stays_usable():
    assert M.mask_test_bounded_wait(True, 200_000) == "MASK_OK"
    assert M.mask_test_bounded_wait(False, 20_000) == "MASK_ETIMEOUT"
    # the context still works after the timed-out wait
    rng = np.random.default_rng(0)
    X = torch.from_numpy(rng.standard_normal((1000, 8)).astype(np.float32)).cuda()
    labels, _ = M.mask_kmeans_assign(X, X[:10].clone(), with_dist=False)
    assert np.array_equal(labels[:10].cpu().numpy(), np.arange(10))
    assert M.mask_test_bounded_wait(True, 200_000) == "MASK_OK"


def test_bounded_wait_rejects_a_bad_limit():
    with pytest.raises(M.MaskError, match="MASK_EINVAL"):
        M.mask_test_bounded_wait(False, -1)
