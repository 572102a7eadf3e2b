"""GPU: failure detection without a fault. A kernel's bounded mbarrier wait that can never complete gives up after its
limit, raises the context's device error flag and exits; the host reports ERR_TIMEOUT, clears the flag, and the
context keeps scoring correctly afterwards (the tensor-core kernels' own bounded waits no longer see a raised flag)."""
import time

import numpy as np
import pytest

from helpers import device_pyramid
from paper_1707_03268_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def test_bounded_wait_expiry_is_reported_and_the_context_recovers(torch):
    from paper_1707_03268_gb300 import tdpm as T
    ctx = T.tdpm_create(0)
    wl = synth.config_c2()
    mid = T.tdpm_load_model(ctx, wl.model)
    dp = device_pyramid(wl.pyramids[0], torch)

    def scores(prec):
        sid = T.tdpm_build_pyramid_scores(ctx, mid, dp, T.FORM_FULL, prec)
        out = [T.tdpm_get_maps(ctx, sid, T.MAP_FINAL_SCORE, c, j) for c in range(len(wl.model.components))
               for j in (10, 20, 30)]
        T.tdpm_release(ctx, sid)
        return out

    before = scores(T.PREC_BF16X3)
    t0 = time.monotonic()
    assert T.tdpm_selftest_bounded_wait(ctx) == T.ERR_TIMEOUT
    assert time.monotonic() - t0 < 10.0  # the wait's limit is about half a second
    after = scores(T.PREC_BF16X3)  # the tensor-core kernels' waits run normally again
    for a, b in zip(before, after):
        np.testing.assert_array_equal(a, b)
    # a second expiry is reported again (the flag was cleared, not left raised)
    assert T.tdpm_selftest_bounded_wait(ctx) == T.ERR_TIMEOUT
    T.tdpm_destroy(ctx)
