"""GPU: the feature extraction block (HOG pyramid) against the FP64 oracle.

On an image the library does not resample (the 8-bit pixels are exact in FP32), both sides take the gradient-channel
and orientation decisions on the same FP32 values with the same rounding, so every feature must match within FP32
accumulation error. The resample itself is checked against the oracle's FP64 area averaging. On resampled levels the
FP32 image differs from the oracle's in the last bits, so a decision can flip where two orientations (or channels)
are within rounding of each other: those levels must agree within tolerance on all but a small share of cells. Ragged
sizes (sides that are not multiples of the cell size, so that the last visible pixels repeat the border) are covered.
"""
import numpy as np
import pytest

from helpers import agreement, det_keys, device_pyramid
from oracle import hog as ohog
from paper_1707_03268_gb300 import synth

pytestmark = pytest.mark.gpu

FEAT_ATOL = 2e-5  # features are sums of at most four values truncated at 0.2, each accumulated in FP32


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def T(torch):
    from paper_1707_03268_gb300 import tdpm
    return tdpm


@pytest.fixture(scope="module")
def ctx(T):
    c = T.tdpm_create(0)
    yield c
    T.tdpm_destroy(c)


def _image(seed, h, w):
    """Smooth structure plus noise, 8-bit RGB (edges of every orientation)."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    base = 120 + 60 * np.sin(x / 7.0 + 0.3 * y / 5.0) + 40 * np.cos(y / 9.0 - x / 13.0)
    img = np.stack([base, base * 0.8 + 20, 255 - base], axis=2) + rng.normal(0, 12, size=(h, w, 3))
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


@pytest.mark.parametrize("h,w", [(61, 77), (96, 128), (131, 90)])
@pytest.mark.parametrize("sbin", [4, 8])
def test_features_of_an_unresampled_image(torch, T, ctx, h, w, sbin):
    img = _image(h * 1000 + w, h, w)
    got = T.tdpm_hog_features(ctx, torch.from_numpy(img.astype(np.float32)).cuda(), sbin).cpu().numpy()
    want = ohog.hog(img.astype(np.float32), sbin)
    assert got.shape == want.shape and got.shape[0] > 0
    np.testing.assert_allclose(got, want, rtol=0, atol=FEAT_ATOL)
    assert np.all(got[..., 31] == 0)


@pytest.mark.parametrize("scale", [1.0, 2 ** -0.1, 2 ** -0.7, 0.5, 0.37])
def test_resize_matches_the_oracle(torch, T, ctx, scale):
    rng = np.random.default_rng(4)
    img = rng.uniform(0, 255, size=(67, 93, 3)).astype(np.float32)
    got = T.tdpm_resize(ctx, torch.from_numpy(img).cuda(), scale).cpu().numpy()
    want = ohog.resize(img, scale)
    assert got.shape == want.shape
    np.testing.assert_allclose(got, want, rtol=2e-6, atol=2e-4)


def test_pyramid_matches_the_oracle(torch, T, ctx):
    img = _image(7, 240, 320)
    pyr = T.tdpm_hog_pyramid(ctx, torch.from_numpy(img).cuda(), sbin=8, lam=10, min_cells=8)
    want = ohog.hog_pyramid(img.astype(np.float32), sbin=8, lam=10, min_cells=8)
    shapes, nbytes = T.tdpm_hog_pyramid_shape(240, 320, 8, 10, 8)
    assert [tuple(l.shape[:2]) for l in want] == shapes == [tuple(l.shape[:2]) for l in pyr.levels]
    assert nbytes == sum(h * w * 32 * 4 for h, w in shapes)
    torch.cuda.synchronize()
    for j, (lv, ref) in enumerate(zip(pyr.levels, want)):
        got = lv.cpu().numpy()
        err = np.max(np.abs(got - ref), axis=2)
        if j in (0, 10):  # scale 1: not resampled, decisions on identical values
            assert np.max(err) <= FEAT_ATOL, j
        else:  # resampled: a decision may flip at a near-tie; all but a small share of cells agree
            assert np.mean(err > 1e-4) <= 0.01, (j, float(np.mean(err > 1e-4)))


def test_hog_pyramid_feeds_the_scoring_path(torch, T, ctx):
    """Image -> HOG pyramid -> scores -> detections, against the same model scored on the oracle's pyramid."""
    img = _image(11, 240, 320)
    pyr = T.tdpm_hog_pyramid(ctx, torch.from_numpy(img).cuda())
    ref_levels = ohog.hog_pyramid(img.astype(np.float32))
    ref = device_pyramid(synth.Pyramid([l.astype(np.float32) for l in ref_levels], 10), torch)
    model = synth.Model(synth.make_dpm_class(np.random.default_rng(5)))
    mid = T.tdpm_load_model(ctx, model)
    a = T.tdpm_build_pyramid_scores(ctx, mid, pyr, T.FORM_FULL, T.PREC_FP32)
    b = T.tdpm_build_pyramid_scores(ctx, mid, ref, T.FORM_FULL, T.PREC_FP32)
    sa = T.tdpm_detect(ctx, a, -np.inf)["score"]
    tau = float(np.percentile(sa, 99))
    da, db = T.tdpm_detect(ctx, a, tau), T.tdpm_detect(ctx, b, tau)
    assert len(da) > 0
    assert agreement(det_keys(da), det_keys(db)) >= 0.97
    T.tdpm_release(ctx, a)
    T.tdpm_release(ctx, b)


def test_hog_argument_errors(torch, T, ctx):
    with pytest.raises(T.TdpmError):
        T.tdpm_hog_pyramid_shape(40, 40, 8, 10, 8)      # too small for one root level
    with pytest.raises(T.TdpmError):
        T.tdpm_hog_pyramid_shape(240, 320, 6, 10, 8)    # cell size not 4, 8 or 16
    with pytest.raises(T.TdpmError):
        T.tdpm_resize(ctx, torch.zeros((8, 8, 3), device="cuda"), 1.5)


def test_repeated_pyramid_calls_replay_identically(torch, T, ctx):
    """The second call with the same buffers reuses the device tables and later ones replay a captured graph; an
    interleaved single-image call invalidates both. Every call writes the same bits."""
    img = torch.from_numpy(_image(13, 150, 200)).cuda()
    pyr = T.HogPyramid(150, 200)
    l0 = T.tdpm_kernel_launches()
    first = pyr.compute(ctx, img).flat.clone()
    per_call = T.tdpm_kernel_launches() - l0   # one resize per octave, gradients, cells, features
    assert per_call == 4                        # 150x200: every root level is in the first octave
    l0 = T.tdpm_kernel_launches()
    for _ in range(4):
        pyr.compute(ctx, img)
        torch.cuda.synchronize()
        assert torch.equal(pyr.flat, first)
    assert T.tdpm_kernel_launches() - l0 == 4 * per_call   # graph replays counted too
    T.tdpm_hog_features(ctx, img.float(), 8)
    pyr.flat.zero_()
    pyr.compute(ctx, img)
    torch.cuda.synchronize()
    assert torch.equal(pyr.flat, first)
