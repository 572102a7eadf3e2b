"""The allocation-free distance transform (tdpm_dt_noalloc) against the regular entry point (tdpm_dt).

tdpm_dt_noalloc serves callers that may not allocate device memory (applications whose memory belongs to another
allocator, latency-critical loops that cannot take cudaMalloc's synchronisation); it keeps its scratch in a fixed device
array inside the library. tdpm_dt runs the fused distance-transform kernel and tdpm_dt_noalloc the two-pass form
(x pass, intermediate in the fixed array, y pass). The two forms run the same per-line scans in the same order, so
their outputs must agree bit for bit; this test depends on that. Two calls in a row check that the shared scratch is
reused correctly. This file is collected last so that a failure here cannot hide another test's.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _regular(torch, T, S, d, sampling):
    xo, xs, nx, yo, ys, ny = sampling
    D = torch.empty((ny, nx), device="cuda")
    A = torch.empty((ny, nx), dtype=torch.int32, device="cuda")
    scratch = torch.empty(T.tdpm_dt_scratch_bytes(S.shape[0], nx), dtype=torch.uint8, device="cuda")
    T.tdpm_dt(S, d, xo, xs, nx, yo, ys, ny, D, A, scratch)
    torch.cuda.synchronize()
    return D.cpu().numpy(), A.cpu().numpy()


def _noalloc(torch, T, S, d, sampling):
    xo, xs, nx, yo, ys, ny = sampling
    D = torch.empty((ny, nx), device="cuda")
    A = torch.empty((ny, nx), dtype=torch.int32, device="cuda")
    T.tdpm_dt_noalloc(S, d, xo, xs, nx, yo, ys, ny, D, A)
    torch.cuda.synchronize()
    return D.cpu().numpy(), A.cpu().numpy()


def test_noalloc_matches_regular_entry_point_on_two_calls(torch):
    from paper_1707_03268_gb300 import tdpm as T
    rng = np.random.default_rng(77)
    cases = [((90, 160), [0.03, 0.01, -0.02, 0.02], (1, 2, 78, 0, 2, 45)),
             ((55, 75), [0.001, 0.05, 0.004, 0.1], (0, 1, 75, 3, 1, 52))]
    for (H, W), d, sampling in cases:
        S = torch.from_numpy(rng.normal(0, 1.0, size=(H, W)).astype(np.float32)).cuda()
        d = np.asarray(d, dtype=np.float32)
        D_ref, A_ref = _regular(torch, T, S, d, sampling)
        D_got, A_got = _noalloc(torch, T, S, d, sampling)
        np.testing.assert_array_equal(D_got, D_ref)
        np.testing.assert_array_equal(A_got, A_ref)


def test_noalloc_rejects_sizes_above_its_scratch(torch):
    from paper_1707_03268_gb300 import tdpm as T
    limit = T.tdpm_dt_noalloc_max_elements()
    H, W = 800, 800
    assert H * W > limit
    S = torch.zeros((H, W), device="cuda")
    D = torch.zeros((H, W), device="cuda")
    A = torch.zeros((H, W), dtype=torch.int32, device="cuda")
    with pytest.raises(T.TdpmError) as ei:
        T.tdpm_dt_noalloc(S, [0.1, 0.1, 0.1, 0.1], 0, 1, W, 0, 1, H, D, A)
    assert ei.value.status == T.ERR_ARG
