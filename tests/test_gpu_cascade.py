"""GPU: convolution shortening (Sec. 4 thresholds from positive examples, Algorithm 1's early exit) against the oracle.

A 6-component class model, decomposed per filter at rank 6, scores a batch of four 240x320 pyramids with planted
object instances (positives, five per component and image). The library's partial sums at the positives and its thresholds must match the oracle's within FP32
rounding; no positive may be pruned by thresholds taken from itself (the library evaluates the thresholds and the
cascade with one device function, so this holds exactly); with no thresholds the cascade is plain step 4; and on a
second pyramid the kept detections must equal the oracle's except where a score or a partial sum lies within rounding
of its threshold.
"""
import numpy as np
import pytest

from helpers import device_pyramid
from oracle import oracle as orc
from paper_1707_03268_gb300 import synth

pytestmark = pytest.mark.gpu

RANK = 6


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


def _placements(rng, model, pyr, per_comp):
    """per_comp random valid root positions of every component (so that every component gets thresholds)."""
    out = []
    for c, comp in enumerate(model.components):
        cells = []
        for j in range(pyr.lam, len(pyr.levels)):
            Y, X = orc.root_domain(pyr.sizes[j], pyr.sizes[j - pyr.lam], comp.root.shape[:2],
                                   [(p.filt.shape[:2], p.anchor) for p in comp.parts])
            cells += [(c, j, y, x) for y in range(Y) for x in range(X)]
        out += [cells[i] for i in sorted(rng.choice(len(cells), size=per_comp, replace=False))]
    return out


def _records(T, places):
    """Records of (image, component, level, y, x) placements."""
    r = np.zeros(len(places), dtype=T.DETECTION_DTYPE)
    for i, (im, c, j, y, x) in enumerate(places):
        r[i]["image"], r[i]["component"], r[i]["level"], r[i]["y"], r[i]["x"] = im, c, j, y, x
    return r


def _factors(T, ctx, mid):
    """Per-filter factors (lam, A, B, C) in model order from the library's FP64 factors (block-diagonal Lambda)."""
    n_f, n_groups = T.tdpm_model_info(ctx, mid)
    out = [None] * n_f
    for gi in range(n_groups):
        info = T.tdpm_group_info(ctx, mid, gi)
        A, B, C, Lam = T.tdpm_get_factors(ctx, mid, gi)
        for k, fid in enumerate(info["filter_ids"]):
            idx = np.nonzero(Lam[k])[0]
            out[fid] = (Lam[k, idx], A[:, idx], B[:, idx], C[:, idx])
    return out


@pytest.fixture(scope="module")
def setup(torch, T):
    ctx = T.tdpm_create(0)
    model = synth.Model(synth.make_dpm_class(np.random.default_rng(72)))
    mid = T.tdpm_load_model(ctx, model)
    T.tdpm_decompose(ctx, mid, RANK, T.DECOMP_PER_FILTER, max_iters=40, seed=3)
    rng = np.random.default_rng(71)
    sizes = synth.pyramid_sizes(240, 320)
    train, pos_train = [], []
    for im in range(4):
        base = synth.make_pyramid(rng, sizes, synth.LAMBDA)
        places = _placements(rng, model, base, 5)
        train.append(synth.plant_objects(rng, base, model, places))
        pos_train += [(im,) + p for p in places]
    base_test = synth.make_pyramid(rng, sizes, synth.LAMBDA)
    pos_test = _placements(rng, model, base_test, 2)
    test = synth.plant_objects(rng, base_test, model, pos_test)
    d_train, d_test = [device_pyramid(p, torch) for p in train], device_pyramid(test, torch)
    s_train = T.tdpm_build_batch_scores(ctx, mid, d_train, T.FORM_DECOMPOSED, T.PREC_FP32)
    s_test = T.tdpm_build_pyramid_scores(ctx, mid, d_test, T.FORM_DECOMPOSED, T.PREC_FP32)
    yield dict(ctx=ctx, model=model, mid=mid, train=train, test=test, d_train=d_train, d_test=d_test,
               s_train=s_train, s_test=s_test, pos_train=pos_train, pos_test=pos_test,
               factors=_factors(T, ctx, mid))
    T.tdpm_destroy(ctx)


def _tol(p):
    return 2e-5 * max(1.0, float(np.max(np.abs(p))))


def test_partials_and_thresholds_match_the_oracle(T, setup):
    S = setup
    recs = _records(T, S["pos_train"])
    P = T.tdpm_cascade_partials(S["ctx"], S["s_train"], S["d_train"], recs, S["mid"])
    n_slots = [1 + len(c.parts) for c in S["model"].components]
    for i, (im, *rec) in enumerate(S["pos_train"]):
        ref = orc.cascade_partials(S["model"], S["train"][im], S["factors"], tuple(rec))
        assert len(ref) == n_slots[rec[0]]
        for s, p in enumerate(ref):
            got = P[i, s, : len(p)].astype(np.float64)
            assert np.max(np.abs(got - p)) <= _tol(p), (i, s)
            assert np.all(np.isnan(P[i, s, len(p):]))
        assert np.all(np.isnan(P[i, len(ref):]))
    t = T.tdpm_cascade_thresholds(S["ctx"], S["s_train"], S["d_train"], recs, S["mid"])
    t_ref = orc.cascade_thresholds(S["model"], lambda img: S["train"][img], S["factors"], S["pos_train"])
    for fid in range(t.shape[0]):
        if fid in t_ref:
            r = t_ref[fid]
            assert np.max(np.abs(t[fid, : len(r)] - r)) <= _tol(r), fid
            assert np.all(np.isneginf(t[fid, len(r):]))
        else:
            assert np.all(np.isneginf(t[fid]))


def test_positives_survive_and_no_thresholds_is_plain_detection(T, setup):
    S = setup
    ctx = S["ctx"]
    t = T.tdpm_cascade_thresholds(ctx, S["s_train"], S["d_train"], _records(T, S["pos_train"]), S["mid"])
    kept, st = T.tdpm_detect_cascade(ctx, S["s_train"], S["d_train"], t, -np.inf)
    keys = set(zip(kept["image"].tolist(), kept["component"].tolist(), kept["level"].tolist(), kept["y"].tolist(),
                   kept["x"].tolist()))
    assert set(S["pos_train"]) <= keys
    n_all = len(T.tdpm_detect(ctx, S["s_train"], -np.inf))
    assert st["candidates"] == n_all and st["pruned"] == n_all - len(kept)
    assert st["terms_total"] == n_all * 9 * RANK and 0 < st["terms_evaluated"] <= st["terms_total"]
    # the background is pruned early: most hypotheses go, after few terms
    assert st["pruned"] > 0.5 * n_all and st["terms_evaluated"] < 0.5 * st["terms_total"]
    # no thresholds: the cascade keeps every detection, bit for bit, and evaluates every term
    none = np.full_like(t, -np.inf)
    tau = float(np.percentile(T.tdpm_detect(ctx, S["s_test"], -np.inf)["score"], 95))
    got, st0 = T.tdpm_detect_cascade(ctx, S["s_test"], [S["d_test"]], none, tau)
    np.testing.assert_array_equal(got, T.tdpm_detect(ctx, S["s_test"], tau))
    assert st0["pruned"] == 0 and st0["terms_evaluated"] == st0["terms_total"] == len(got) * 9 * RANK


def test_cascade_detections_match_the_oracle(T, setup):
    S = setup
    ctx, model = S["ctx"], S["model"]
    t = T.tdpm_cascade_thresholds(ctx, S["s_train"], S["d_train"], _records(T, S["pos_train"]), S["mid"])
    t_ref = orc.cascade_thresholds(model, lambda img: S["train"][img], S["factors"], S["pos_train"])
    rebuilt = [orc.cp_reconstruct(w, [A, B, C]) for (w, A, B, C) in S["factors"]]
    scored = orc.score_pyramid(model, S["test"], filters=rebuilt)
    smax = float(np.max(np.abs(orc.all_scores(scored))))
    tau = float(np.percentile(orc.all_scores(scored), 97))
    dets = orc.detect(scored, tau)
    keep_ref = orc.cascade_detect(model, S["test"], S["factors"], t_ref, dets)
    ref = {tuple(dets[i][:4]): dets[i][4] for i in keep_ref}
    got, st = T.tdpm_detect_cascade(ctx, S["s_test"], [S["d_test"]], t, tau)
    gkeys = set(zip(got["component"].tolist(), got["level"].tolist(), got["y"].tolist(), got["x"].tolist()))
    assert len(ref) > 0 and st["pruned"] > 0
    # every difference must sit within rounding of tau or of a cascade threshold (oracle values)
    score_of = {(m["component"], m["level"]): m["score"] for m in scored}
    unexplained = []
    for key in gkeys ^ set(ref):
        c, j, y, x = key
        s = float(score_of[(c, j)][y, x])
        near_tau = abs(s - tau) <= 2e-5 * smax
        P = orc.cascade_partials(model, S["test"], S["factors"], key)
        fid0 = sum(1 + len(cc.parts) for cc in model.components[:c])
        margins = [abs(p[q] - t_ref[fid0 + k][q]) / max(1.0, abs(t_ref[fid0 + k][q]))
                   for k, p in enumerate(P) if fid0 + k in t_ref for q in range(len(p))]
        near_thr = min(margins) <= 4e-5 if margins else False
        if not (near_tau or near_thr):
            unexplained.append(key)
    assert not unexplained, unexplained[:5]
    assert len(gkeys & set(ref)) >= 0.99 * len(gkeys | set(ref))


def test_cascade_argument_errors(torch, T, setup):
    S = setup
    ctx = S["ctx"]
    t = T.tdpm_cascade_thresholds(ctx, S["s_train"], S["d_train"], _records(T, S["pos_train"]), S["mid"])
    with pytest.raises(T.TdpmError):  # not the pyramids the scores set was built from
        T.tdpm_detect_cascade(ctx, S["s_train"], S["d_train"][:3], t, 0.0)
    with pytest.raises(T.TdpmError):
        T.tdpm_detect_cascade(ctx, S["s_test"], S["d_train"][:1], t, 0.0)
    bad = t.copy()
    bad[0, 0] = np.nan
    with pytest.raises(T.TdpmError):
        T.tdpm_detect_cascade(ctx, S["s_train"], S["d_train"], bad, 0.0)
    r = _records(T, S["pos_train"][:1])
    r[0]["component"] = 99
    with pytest.raises(T.TdpmError):
        T.tdpm_cascade_partials(ctx, S["s_train"], S["d_train"], r, S["mid"])
    # the cascade needs per-filter factors
    c2 = T.tdpm_create(0)
    mid = T.tdpm_load_model(c2, S["model"])
    T.tdpm_decompose(c2, mid, 8, T.DECOMP_JOINT, max_iters=5, seed=1)
    sid = T.tdpm_build_pyramid_scores(c2, mid, S["d_test"], T.FORM_DECOMPOSED, T.PREC_FP32)
    with pytest.raises(T.TdpmError):
        T.tdpm_detect_cascade(c2, sid, [S["d_test"]], t, 0.0)
    T.tdpm_destroy(c2)
