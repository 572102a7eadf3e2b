"""GPU: several images scored in one batch give exactly what each image gives alone, and match the oracle.

Each stage runs one launch over the jobs of every level of every image; a position's arithmetic never depends on which
other levels share the launch, so the batched maps must be bit-identical to single-image builds.
"""
import numpy as np
import pytest

from helpers import agreement, det_keys, device_pyramid, rel_err
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


@pytest.fixture(scope="module")
def ctx(T):
    c = T.tdpm_create(0)
    yield c
    T.tdpm_destroy(c)


def _batch_images(seed=21):
    """Differently sized images (ragged level counts), one whose pyramid is too small for any root placement."""
    rng = np.random.default_rng(seed)
    pyrs = [synth.make_pyramid(rng, synth.pyramid_sizes(h, w), synth.LAMBDA) for (h, w) in
            [(150, 200), (240, 130), (96, 96), (180, 320)]]
    pyrs.append(synth.make_pyramid(rng, [(9, 9), (5, 5)], lam=1))
    return pyrs


def _maps(T, ctx, sid, model, n_levels, lam, image):
    # a level with no scored root position gives an empty map
    return {(c, j): T.tdpm_get_maps(ctx, sid, T.MAP_FINAL_SCORE, c, j, image=image)
            for c in range(len(model.components)) for j in range(lam, n_levels)}


@pytest.mark.parametrize("form,prec", [("full", "fp32"), ("full", "bf16x3"), ("decomposed", "bf16x3"),
                                       ("decomposed", "fp32")])
def test_batch_equals_single_images(torch, T, ctx, form, prec):
    wl = synth.config_c2()
    mid = T.tdpm_load_model(ctx, wl.model)
    f = T.FORM_FULL if form == "full" else T.FORM_DECOMPOSED
    p = T.PREC_FP32 if prec == "fp32" else T.PREC_BF16X3
    if f == T.FORM_DECOMPOSED:
        T.tdpm_decompose(ctx, mid, 8, T.DECOMP_PER_FILTER, max_iters=60, seed=1)
    pyrs = _batch_images()
    dps = [device_pyramid(py, torch) for py in pyrs]
    bsid = T.tdpm_build_batch_scores(ctx, mid, dps, f, p)
    singles = []
    for dp in dps:
        singles.append(T.tdpm_build_pyramid_scores(ctx, mid, dp, f, p))
    # thresholds low enough that every image contributes detections
    tau = float(np.percentile(T.tdpm_get_maps(ctx, singles[0], T.MAP_FINAL_SCORE, 0, synth.LAMBDA), 90))
    bdets = T.tdpm_detect(ctx, bsid, tau)
    assert np.all(np.diff(bdets["image"]) >= 0)
    for i, (py, sid) in enumerate(zip(pyrs, singles)):
        bm = _maps(T, ctx, bsid, wl.model, len(py.levels), py.lam, i)
        sm = _maps(T, ctx, sid, wl.model, len(py.levels), py.lam, 0)
        assert bm.keys() == sm.keys()
        for k in bm:
            np.testing.assert_array_equal(bm[k], sm[k])
        sd = T.tdpm_detect(ctx, sid, tau)
        mine = bdets[bdets["image"] == i]
        assert len(mine) == len(sd)
        for name in ("component", "level", "y", "x", "score", "n_parts", "part_y", "part_x"):
            np.testing.assert_array_equal(mine[name], sd[name])
        assert np.all(sd["image"] == 0)
    assert np.sum(bdets["image"] == len(pyrs) - 1) == 0   # the degenerate image has nothing to score
    for sid in singles:
        T.tdpm_release(ctx, sid)
    T.tdpm_release(ctx, bsid)


def test_batch_matches_oracle_per_image(torch, T, ctx):
    """FP32 full form, two images of one batch, against the FP64 oracle scored one image at a time."""
    wl = synth.config_c2()
    mid = T.tdpm_load_model(ctx, wl.model)
    pyrs = _batch_images(seed=5)[:2]
    sid = T.tdpm_build_batch_scores(ctx, mid, [device_pyramid(py, torch) for py in pyrs], T.FORM_FULL, T.PREC_FP32)
    all_ref = []
    for i, py in enumerate(pyrs):
        ref = orc.score_pyramid(wl.model, py)
        for m in ref:
            got = T.tdpm_get_maps(ctx, sid, T.MAP_FINAL_SCORE, m["component"], m["level"], image=i)
            assert rel_err(got, m["score"]) <= 1e-5
        all_ref.append(ref)
    tau = float(np.percentile(np.concatenate([orc.all_scores(r) for r in all_ref]), 98))
    dets = T.tdpm_detect(ctx, sid, tau)
    for i, ref in enumerate(all_ref):
        mine = dets[dets["image"] == i]
        assert agreement(det_keys(mine), det_keys(orc.detect(ref, tau))) >= 0.995
    T.tdpm_release(ctx, sid)


def test_batch_rejects_bad_image_index(torch, T, ctx):
    wl = synth.config_c1()
    mid = T.tdpm_load_model(ctx, wl.model)
    dp = device_pyramid(wl.pyramids[0], torch)
    sid = T.tdpm_build_batch_scores(ctx, mid, [dp, dp], T.FORM_FULL, T.PREC_FP32)
    a = T.tdpm_get_maps(ctx, sid, T.MAP_FINAL_SCORE, 0, 1, image=0)
    b = T.tdpm_get_maps(ctx, sid, T.MAP_FINAL_SCORE, 0, 1, image=1)
    np.testing.assert_array_equal(a, b)
    with pytest.raises(T.TdpmError):
        T.tdpm_get_maps(ctx, sid, T.MAP_FINAL_SCORE, 0, 1, image=2)
    with pytest.raises(T.TdpmError):
        T.tdpm_get_maps(ctx, sid, T.MAP_FINAL_SCORE, 0, 1, image=-1)
    with pytest.raises(T.TdpmError):
        T.tdpm_build_batch_scores(ctx, mid, [], T.FORM_FULL, T.PREC_FP32)
    T.tdpm_release(ctx, sid)


def test_component_subsets_equal_full_batch_filtered(torch, T, ctx):
    """A batch scored for a subset of components per image gives, for those components, exactly the maps and
    detections of the full batch; the others are not computed."""
    wl = synth.config_c2()
    mid = T.tdpm_load_model(ctx, wl.model)
    pyrs = _batch_images(seed=9)[:4]
    dps = [device_pyramid(py, torch) for py in pyrs]
    nc = len(wl.model.components)
    mask = np.zeros((len(pyrs), nc), dtype=np.uint8)
    mask[0, [0, 3]] = 1
    mask[1, :] = 1
    mask[2, [5]] = 1
    mask[3, [1, 2, 4]] = 1
    full = T.tdpm_build_batch_scores(ctx, mid, dps, T.FORM_FULL, T.PREC_BF16X3)
    sub = T.tdpm_build_batch_scores_subset(ctx, mid, dps, mask, T.FORM_FULL, T.PREC_BF16X3)
    tau = float(np.percentile(T.tdpm_detect(ctx, full, -np.inf)["score"], 95))
    df, ds = T.tdpm_detect(ctx, full, tau), T.tdpm_detect(ctx, sub, tau)
    keep = mask[df["image"], df["component"]].astype(bool)
    assert keep.sum() == len(ds) > 0
    for name in ("image", "component", "level", "y", "x", "score", "part_y", "part_x"):
        np.testing.assert_array_equal(df[keep][name], ds[name])
    for i, py in enumerate(pyrs):
        for c in range(nc):
            for j in range(py.lam, len(py.levels)):
                a = T.tdpm_get_maps(ctx, full, T.MAP_FINAL_SCORE, c, j, image=i)
                b = T.tdpm_get_maps(ctx, sub, T.MAP_FINAL_SCORE, c, j, image=i)
                if mask[i, c]:
                    np.testing.assert_array_equal(a, b)
                else:
                    assert b.size == 0
    T.tdpm_release(ctx, full)
    T.tdpm_release(ctx, sub)


def test_thresholds_per_image_and_component(torch, T, ctx):
    """tdpm_detect_thresholds gives exactly the records of tdpm_detect at the lowest threshold that clear their own
    (image, component) threshold, in the same order; a uniform table equals tdpm_detect."""
    wl = synth.config_c2()
    mid = T.tdpm_load_model(ctx, wl.model)
    pyrs = _batch_images(seed=13)[:3]
    sid = T.tdpm_build_batch_scores(ctx, mid, [device_pyramid(py, torch) for py in pyrs], T.FORM_FULL, T.PREC_FP32)
    nc = len(wl.model.components)
    allp = T.tdpm_detect(ctx, sid, -np.inf)
    rng = np.random.default_rng(3)
    tau = np.percentile(allp["score"], rng.uniform(80, 99.5, size=(len(pyrs), nc))).astype(np.float32)
    got = T.tdpm_detect_thresholds(ctx, sid, tau)
    low = T.tdpm_detect(ctx, sid, float(tau.min()))
    want = low[low["score"] >= tau[low["image"], low["component"]]]
    assert len(got) == len(want) > 0
    for name in ("image", "component", "level", "y", "x", "score", "part_y", "part_x"):
        np.testing.assert_array_equal(got[name], want[name])
    flat = np.full((len(pyrs), nc), float(np.median(tau)), dtype=np.float32)
    a, b = T.tdpm_detect_thresholds(ctx, sid, flat), T.tdpm_detect(ctx, sid, float(flat[0, 0]))
    np.testing.assert_array_equal(a, b)
    with pytest.raises(T.TdpmError):
        T.tdpm_detect_thresholds(ctx, sid, np.full((len(pyrs), nc), np.nan, dtype=np.float32))
    T.tdpm_release(ctx, sid)
