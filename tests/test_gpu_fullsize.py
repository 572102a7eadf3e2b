"""GPU parity at the bank workload's full size (C3: a 20-class bank of 1080 filters on one 1280x720 pyramid, 45
levels), in the configurations the benchmark times, on outputs the oracle computes one by one.

The whole bank's FP64 scores would take the oracle minutes, so it checks samples: filter responses at random
(filter, level, position) triples, from the window and the filter directly; and the complete final score maps of a
few (component, root level) pairs, with their part maps, distance transforms and assembly. Full BF16 is compared with
the oracle on BF16-rounded operands (every product exact in FP32, so only FP32 summation-order error remains);
per-filter rank 8 in split BF16 (the headline's arithmetic on the bank) with the oracle on the same factors.
"""
import numpy as np
import pytest

from helpers import rel_err
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
def c3(torch, T):
    wl = synth.config_c3()
    ctx = T.tdpm_create(0)
    mid = T.tdpm_load_model(ctx, wl.model)
    pyr = wl.pyramids[0]
    levels = [torch.from_numpy(np.ascontiguousarray(l)).cuda() for l in pyr.levels]
    yield dict(wl=wl, ctx=ctx, mid=mid, pyr=pyr, dp=T.DevicePyramid(levels, pyr.lam))
    T.tdpm_destroy(ctx)


def _bf16(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).bfloat16().float().numpy().astype(np.float64)


def _component_score(model, c, feats, lam, j, filters):
    """Oracle final score map of component c at root level j (Sec. 2 score, G11 anchors) from FP64 feature levels
    and filters (model order)."""
    comp = model.components[c]
    fid = sum(1 + len(cc.parts) for cc in model.components[:c])
    root, parts = filters[fid], filters[fid + 1: fid + 1 + len(comp.parts)]
    Y, X = orc.root_domain(feats[j].shape[:2], feats[j - lam].shape[:2], root.shape[:2],
                           [(pf.shape[:2], p.anchor) for p, pf in zip(comp.parts, parts)])
    total = orc.correlate(feats[j].astype(np.float32), root)[:Y, :X] + float(comp.bias)
    for p, pf in zip(comp.parts, parts):
        D, _, _ = orc.dt2d(orc.correlate(feats[j - lam].astype(np.float32), pf), np.asarray(p.deform, np.float64))
        total = total + D[np.ix_(p.anchor[0] + 2 * np.arange(Y), p.anchor[1] + 2 * np.arange(X))]
    return total


def test_c3_full_bf16_sampled_responses_and_score_maps(torch, T, c3):
    wl, ctx, mid, pyr = c3["wl"], c3["ctx"], c3["mid"], c3["pyr"]
    sid = T.tdpm_build_pyramid_scores(ctx, mid, c3["dp"], T.FORM_FULL, T.PREC_BF16)
    filters = wl.model.filters()
    rng = np.random.default_rng(91)
    checked = 0
    while checked < 300:
        fid = int(rng.integers(len(filters)))
        f = filters[fid]
        j = int(rng.integers(len(pyr.levels)))
        try:
            got = T.tdpm_get_maps(ctx, sid, T.MAP_FILTER_SCORE, fid, j)
        except T.TdpmError:
            continue  # this filter's role does not score this level
        if got.size == 0:
            continue  # the filter does not fit this level
        y, x = int(rng.integers(got.shape[0])), int(rng.integers(got.shape[1]))
        win = _bf16(pyr.levels[j][y:y + f.shape[0], x:x + f.shape[1]], torch)
        prod = win * _bf16(f, torch)
        assert abs(float(got[y, x]) - prod.sum()) <= 2e-5 * np.abs(prod).sum() + 1e-12, (fid, j, y, x)
        checked += 1
    # whole final score maps of three (component, level) pairs: one of each root shape, at a mid-size level
    rounded = [_bf16(l, torch) for l in pyr.levels]
    rfilters = [_bf16(f, torch) for f in filters]
    for c, j in ((6, 20), (8, 24), (64, 28)):  # roots 5x11, 7x7, 11x5
        ref = _component_score(wl.model, c, rounded, pyr.lam, j, rfilters)
        got = T.tdpm_get_maps(ctx, sid, T.MAP_FINAL_SCORE, c, j)
        assert got.shape == ref.shape
        assert rel_err(got, ref) <= 2e-5, (c, j)
    T.tdpm_release(ctx, sid)


def test_c3_per_filter_rank8_split_bf16_score_maps(torch, T, c3):
    wl, ctx, mid, pyr = c3["wl"], c3["ctx"], c3["mid"], c3["pyr"]
    T.tdpm_decompose(ctx, mid, 8, T.DECOMP_PER_FILTER, max_iters=60, seed=1)
    sid = T.tdpm_build_pyramid_scores(ctx, mid, c3["dp"], T.FORM_DECOMPOSED, T.PREC_BF16X3)
    n_f, n_groups = T.tdpm_model_info(ctx, mid)
    rebuilt = [None] * n_f
    for gi in range(n_groups):
        info = T.tdpm_group_info(ctx, mid, gi)
        A, B, C, Lam = T.tdpm_get_factors(ctx, mid, gi)
        Fk = orc.joint_reconstruct(Lam, A, B, C)
        for k, fid in enumerate(info["filter_ids"]):
            rebuilt[fid] = Fk[k]
    feats = [l.astype(np.float64) for l in pyr.levels]
    for c, j in ((3, 21), (55, 26)):
        ref = _component_score(wl.model, c, feats, pyr.lam, j, rebuilt)
        got = T.tdpm_get_maps(ctx, sid, T.MAP_FINAL_SCORE, c, j)
        assert rel_err(got, ref) <= 1e-4, (c, j)
    T.tdpm_release(ctx, sid)
