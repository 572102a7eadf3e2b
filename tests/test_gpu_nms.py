"""GPU: greedy non-maximum suppression of the detections (a DPM convention, not in the paper) against the oracle.

Both sides take the same detection records (those tdpm_detect returns), compute boxes and overlaps in FP64 with each
operation rounded once, and order by the same FP32 scores, so the kept sets must be identical.
"""
import numpy as np
import pytest

from helpers import device_pyramid
from oracle import oracle as orc
from paper_1707_03268_gb300 import synth

pytestmark = pytest.mark.gpu


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


def _oracle_keep(dets, model, lam, classes, overlap, cell0):
    recs = [(int(d["image"]), int(d["component"]), int(d["level"]), int(d["y"]), int(d["x"]), float(d["score"]))
            for d in dets]
    root_hw = [c.root.shape[:2] for c in model.components]
    return orc.nms(recs, root_hw, cell0, lam, overlap, classes)


@pytest.mark.parametrize("pct,overlap", [(97, 0.5), (90, 0.3), (99.5, 0.7)])
def test_nms_matches_oracle_one_image(torch, T, pct, overlap):
    ctx = T.tdpm_create(0)
    wl = synth.config_c2()
    mid = T.tdpm_load_model(ctx, wl.model)
    pyr = wl.pyramids[0]
    sid = T.tdpm_build_pyramid_scores(ctx, mid, device_pyramid(pyr, torch), T.FORM_FULL, T.PREC_FP32)
    tau = float(np.percentile(T.tdpm_detect(ctx, sid, -np.inf)["score"], pct))
    dets = T.tdpm_detect(ctx, sid, tau).copy()
    kept = T.tdpm_detect_nms(ctx, sid, tau, None, overlap, 4.0)
    want = _oracle_keep(dets, wl.model, pyr.lam, None, overlap, 4.0)
    assert 0 < len(want) < len(dets)
    np.testing.assert_array_equal(kept, dets[want])
    T.tdpm_release(ctx, sid)
    T.tdpm_destroy(ctx)


def test_nms_batch_with_classes_and_bank(torch, T):
    """A ragged batch scored with a small bank (4 classes of 6 components): groups are (image, class). Both NMS paths:
    pairwise overlap masks (up to 16,384 detections) and the per-group walk above that."""
    ctx = T.tdpm_create(0)
    rng = np.random.default_rng(61)
    comps = []
    for c in range(4):
        comps += synth.make_dpm_class(np.random.default_rng(300 + c))
    model = synth.Model(comps)
    classes = [i // 6 for i in range(len(comps))]
    mid = T.tdpm_load_model(ctx, model)
    pyrs = [synth.make_pyramid(rng, synth.pyramid_sizes(h, w), synth.LAMBDA) for (h, w) in
            [(150, 200), (240, 130), (96, 96)]]
    sid = T.tdpm_build_batch_scores(ctx, mid, [device_pyramid(p, torch) for p in pyrs], T.FORM_FULL, T.PREC_BF16X3)
    tau = float(np.percentile(T.tdpm_detect(ctx, sid, -np.inf)["score"], 98))
    dets = T.tdpm_detect(ctx, sid, tau).copy()
    for cls, overlap in ((classes, 0.5), (None, 0.5), (classes, 0.25)):
        kept = T.tdpm_detect_nms(ctx, sid, tau, cls, overlap, 4.0)
        want = _oracle_keep(dets, model, synth.LAMBDA, cls, overlap, 4.0)
        assert 0 < len(want) < len(dets)
        np.testing.assert_array_equal(kept, dets[want])
    # more than 16,384 detections: each group's CTA walks its boxes itself instead of the pairwise masks
    all_scores = np.sort(T.tdpm_detect(ctx, sid, -np.inf)["score"])
    tau_low = float(all_scores[-20000])
    dets = T.tdpm_detect(ctx, sid, tau_low).copy()
    assert len(dets) > 16384
    kept = T.tdpm_detect_nms(ctx, sid, tau_low, classes, 0.5, 4.0)
    want = _oracle_keep(dets, model, synth.LAMBDA, classes, 0.5, 4.0)
    np.testing.assert_array_equal(kept, dets[want])
    # nothing above the threshold: nothing kept
    assert len(T.tdpm_detect_nms(ctx, sid, 1e9, classes, 0.5, 4.0)) == 0
    with pytest.raises(T.TdpmError):
        T.tdpm_detect_nms(ctx, sid, tau, classes, 1.5, 4.0)
    with pytest.raises(T.TdpmError):
        T.tdpm_detect_nms(ctx, sid, tau, [-1] + classes[1:], 0.5, 4.0)
    with pytest.raises(T.TdpmError):
        T.tdpm_detect_nms(ctx, sid, tau, classes, 0.5, 0.0)
    T.tdpm_release(ctx, sid)
    T.tdpm_destroy(ctx)
