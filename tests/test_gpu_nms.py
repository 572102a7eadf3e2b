"""GPU: greedy non-maximum suppression of the detections (a DPM convention, not in the paper) against the oracle.

The inputs are exact in FP32: integer features and filters and power-of-two deformation costs make every score an
integer combination that FP32 holds exactly, so the library's detections equal the oracle's (checked), and each side
runs NMS on detections it computed itself. Both compute boxes and overlaps in FP64 with each operation rounded once
and order by the same scores (many equal: ties go to the earlier record), so the kept sets must be identical.
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


def _integer_classes(seed, n_classes):
    """DPM-shaped components (roots 5x11, 7x7, 11x5 and mirrors, eight 6x6 parts) with integer filter entries in
    [-2, 2] and power-of-two deformation coefficients."""
    rng = np.random.default_rng(seed)
    comps = []
    for c in range(n_classes):
        for comp in synth.make_dpm_class(np.random.default_rng(seed * 100 + c)):
            comp.root = rng.integers(-2, 3, size=comp.root.shape).astype(np.float32)
            for p in comp.parts:
                p.filt = rng.integers(-2, 3, size=p.filt.shape).astype(np.float32)
                p.deform = synth.make_pow2_deform(rng)
            comps.append(comp)
    return synth.Model(comps)


def _integer_pyramid(rng, h, w):
    pyr = synth.make_pyramid(rng, synth.pyramid_sizes(h, w), synth.LAMBDA)
    return synth.Pyramid([rng.integers(0, 4, size=l.shape).astype(np.float32) for l in pyr.levels], pyr.lam)


def _oracle(model, scored, tau, classes, overlap, cell0=4.0):
    """The oracle's own detections of every image (``scored``: score_pyramid per image) at tau, and the records NMS
    keeps (FP64, from the oracle)."""
    recs = []
    for i, sc in enumerate(scored):
        for d in orc.detect(sc, tau):
            recs.append((i,) + tuple(d[:5]))
    root_hw = [c.root.shape[:2] for c in model.components]
    kept = orc.nms(recs, root_hw, cell0, synth.LAMBDA, overlap, classes)
    return recs, [recs[k] for k in kept]


def _keys(dets):
    return [(int(d["image"]), int(d["component"]), int(d["level"]), int(d["y"]), int(d["x"]), float(d["score"]))
            for d in dets]


@pytest.mark.parametrize("q,overlap", [(97, 0.5), (90, 0.3), (99.5, 0.7)])
def test_nms_matches_oracle_one_image(torch, T, q, overlap):
    ctx = T.tdpm_create(0)
    model = _integer_classes(3, 1)
    pyr = _integer_pyramid(np.random.default_rng(8), 240, 320)
    mid = T.tdpm_load_model(ctx, model)
    sid = T.tdpm_build_pyramid_scores(ctx, mid, device_pyramid(pyr, torch), T.FORM_FULL, T.PREC_FP32)
    scored = orc.score_pyramid(model, pyr)
    tau = float(np.percentile(orc.all_scores(scored), q))
    recs, want = _oracle(model, [scored], tau, None, overlap)
    assert _keys(T.tdpm_detect(ctx, sid, tau)) == recs          # exact inputs: identical detections
    got = _keys(T.tdpm_detect_nms(ctx, sid, tau, None, overlap, 4.0))
    assert 0 < len(want) < len(recs)
    assert got == want
    T.tdpm_release(ctx, sid)
    T.tdpm_destroy(ctx)


def test_nms_batch_with_classes_and_bank(torch, T):
    """A ragged batch scored with a bank of 4 classes (24 components): groups are (image, class). Both NMS paths:
    pairwise overlap masks (up to 16,384 detections) and the per-group walk above that."""
    ctx = T.tdpm_create(0)
    model = _integer_classes(5, 4)
    classes = [i // 6 for i in range(len(model.components))]
    mid = T.tdpm_load_model(ctx, model)
    rng = np.random.default_rng(61)
    pyrs = [_integer_pyramid(rng, h, w) for (h, w) in [(150, 200), (240, 130), (96, 96)]]
    sid = T.tdpm_build_batch_scores(ctx, mid, [device_pyramid(p, torch) for p in pyrs], T.FORM_FULL, T.PREC_FP32)
    scored = [orc.score_pyramid(model, p) for p in pyrs]
    scores = np.concatenate([orc.all_scores(sc) for sc in scored])
    tau = float(np.percentile(scores, 98))
    for cls, overlap in ((classes, 0.5), (None, 0.5), (classes, 0.25)):
        recs, want = _oracle(model, scored, tau, cls, overlap)
        got = _keys(T.tdpm_detect_nms(ctx, sid, tau, cls, overlap, 4.0))
        assert 0 < len(want) < len(recs)
        assert got == want
    # more than 16,384 detections: each group's CTA walks its boxes itself instead of the pairwise masks
    tau_low = float(np.sort(scores)[-20000])
    recs, want = _oracle(model, scored, tau_low, classes, 0.5)
    assert len(recs) > 16384
    assert _keys(T.tdpm_detect_nms(ctx, sid, tau_low, classes, 0.5, 4.0)) == want
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
