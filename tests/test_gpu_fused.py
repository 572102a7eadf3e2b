"""GPU: the fused decomposed kernels (channel stage on the tensor cores + separable passes + recombination in one
launch, Sec. 4) against the two-launch form and against the FP64 oracle.

Two fused kernels exist. The tile kernel (cells on the MMA's M dimension; every shape) issues the same MMAs per 128-row
tile as the channel-stage kernel and the same multiply-add order as the separable kernel, so it gives filter maps
bit-identical to the two-launch form; it is forced here with TDPM_ZSEP_FORM. The terms-on-M kernel (6x6 and 7x7
filters, the default for them) adds a filter's terms in another order and folds lambda_r into a_r, so its maps equal
the two-launch maps up to FP32 rounding of the sum. Filter groups of different widths are covered: rank 8, 3 (many
filters per group), 20 and 40 (groups spanning several warps of terms); the C2 model has all four compiled shapes (6x6
parts, 5x11, 7x7, 11x5 roots).
"""
import numpy as np
import pytest

from helpers import agreement, assert_same_sum, det_keys, device_pyramid, rel_err
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


def _images(seed):
    """Ragged batch: different sizes, levels narrower than a 32-column tile and shorter than a row tile."""
    rng = np.random.default_rng(seed)
    pyrs = [synth.make_pyramid(rng, synth.pyramid_sizes(h, w), synth.LAMBDA) for (h, w) in
            [(150, 200), (240, 130), (96, 96)]]
    pyrs.append(synth.make_pyramid(rng, [(40, 33), (31, 70), (17, 12), (12, 45), (8, 9), (6, 6)], lam=2))
    return pyrs


def _stage_names(T, ctx, build):
    T.tdpm_profile_reset(ctx)
    T.tdpm_profile_enable(ctx, True)
    sid = build()
    T.tdpm_profile_enable(ctx, False)
    names = set(T.tdpm_profile_read(ctx))
    return sid, names


@pytest.mark.parametrize("rank", [8, 3, 20, 40])
@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
@pytest.mark.parametrize("kernel", ["tile", "terms"])
def test_fused_equals_two_launch_form(torch, T, rank, prec, kernel, monkeypatch):
    if kernel == "tile":
        monkeypatch.setenv("TDPM_ZSEP_FORM", "0")  # the tile kernel for every shape
    ctx = T.tdpm_create(0)
    wl = synth.config_c2()
    mid = T.tdpm_load_model(ctx, wl.model)
    T.tdpm_decompose(ctx, mid, rank, T.DECOMP_PER_FILTER, max_iters=40, seed=2)
    p = T.PREC_BF16X3 if prec == "bf16x3" else T.PREC_BF16
    pyrs = _images(rank)
    dps = [device_pyramid(py, torch) for py in pyrs]
    n_f, _ = T.tdpm_model_info(ctx, mid)

    def build():
        return T.tdpm_build_batch_scores(ctx, mid, dps, T.FORM_DECOMPOSED, p)

    T.tdpm_set_fusion(ctx, True)
    fused, names_f = _stage_names(T, ctx, build)
    T.tdpm_set_fusion(ctx, False)
    plain, names_p = _stage_names(T, ctx, build)
    T.tdpm_set_fusion(ctx, True)
    assert "zsep_tc" in names_f and "zproj_tc" not in names_f and "sep" not in names_f
    assert "zsep_tc" not in names_p and {"zproj_tc", "sep"} <= names_p
    n_maps = 0
    for i, py in enumerate(pyrs):
        for fid in range(n_f):
            for j in range(len(py.levels)):
                try:
                    a = T.tdpm_get_maps(ctx, fused, T.MAP_FILTER_SCORE, fid, j, image=i)
                except T.TdpmError:
                    continue  # the filter does not fit this level or its role does not score it
                b = T.tdpm_get_maps(ctx, plain, T.MAP_FILTER_SCORE, fid, j, image=i)
                if kernel == "tile":
                    np.testing.assert_array_equal(a, b)
                else:
                    assert_same_sum(a, b)
                n_maps += 1
    assert n_maps > 100
    tau = float(np.percentile(T.tdpm_detect(ctx, plain, -np.inf)["score"], 97))
    if kernel == "tile":
        np.testing.assert_array_equal(T.tdpm_detect(ctx, fused, tau), T.tdpm_detect(ctx, plain, tau))
    else:
        assert agreement(det_keys(T.tdpm_detect(ctx, fused, tau)), det_keys(T.tdpm_detect(ctx, plain, tau))) >= 0.995
    T.tdpm_release(ctx, fused)
    T.tdpm_release(ctx, plain)
    T.tdpm_destroy(ctx)


def _factor_filters(T, ctx, mid, torch, round_c):
    """Every filter rebuilt from its factors (Lambda is block-diagonal in the per-filter mode), c_r rounded to BF16
    when round_c."""
    n_f, n_groups = T.tdpm_model_info(ctx, mid)
    filters = [None] * n_f
    for gi in range(n_groups):
        info = T.tdpm_group_info(ctx, mid, gi)
        A, B, C, Lam = T.tdpm_get_factors(ctx, mid, gi)
        if round_c:
            C = torch.from_numpy(C.astype(np.float32)).bfloat16().double().numpy()
        F = orc.joint_reconstruct(Lam, A, B, C)
        for k, fid in enumerate(info["filter_ids"]):
            filters[fid] = F[k]
    return filters


def test_fused_bf16_matches_oracle(torch, T, ctx):
    """BF16 operands through the fused kernel: against the oracle on the same BF16-rounded features and c_r (the 1-D
    passes run in FP32), and within the stated 1e-2 of the FP64 result with the unrounded factors; the detections
    agree with those of the rounded-operand oracle."""
    wl = synth.config_c2()
    pyr = wl.pyramids[0]
    mid = T.tdpm_load_model(ctx, wl.model)
    T.tdpm_decompose(ctx, mid, 16, T.DECOMP_PER_FILTER, max_iters=150, seed=3)
    T.tdpm_set_fusion(ctx, True)
    sid, names = _stage_names(T, ctx, lambda: T.tdpm_build_pyramid_scores(ctx, mid, device_pyramid(pyr, torch),
                                                                           T.FORM_DECOMPOSED, T.PREC_BF16))
    assert "zsep_tc" in names
    rounded = synth.Pyramid([torch.from_numpy(l).bfloat16().float().numpy() for l in pyr.levels], pyr.lam)
    ref_r = orc.score_pyramid(wl.model, rounded, filters=_factor_filters(T, ctx, mid, torch, True))
    ref = orc.score_pyramid(wl.model, pyr, filters=_factor_filters(T, ctx, mid, torch, False))
    for mr, m in zip(ref_r, ref):
        got = T.tdpm_get_maps(ctx, sid, T.MAP_FINAL_SCORE, m["component"], m["level"])
        assert rel_err(got, mr["score"]) <= 1e-4
        assert rel_err(got, m["score"]) <= 1e-2
    # detections against the oracle on the same rounded operands (BF16 rounding alone moves near-threshold scores)
    tau = float(np.percentile(orc.all_scores(ref_r), 99))
    assert agreement(det_keys(T.tdpm_detect(ctx, sid, tau)), det_keys(orc.detect(ref_r, tau))) >= 0.995
    T.tdpm_release(ctx, sid)


def test_unfusable_groups_fall_back(torch, T, ctx):
    """Filter shapes without a compiled fused form (3x3 here) run as two launches in the same build as fused ones,
    and both match the two-launch maps (to the rounding of the terms' sum for the terms-on-M kernel)."""
    rng = np.random.default_rng(17)
    comps = synth.make_dpm_class(rng)[:2]
    odd = synth.make_component(rng, (3, 3), [(3, 3)] * 2, kind="iid")
    model = synth.Model(comps + [odd])
    mid = T.tdpm_load_model(ctx, model)
    T.tdpm_decompose(ctx, mid, 6, T.DECOMP_PER_FILTER, max_iters=40, seed=1)
    dp = device_pyramid(synth.make_pyramid(rng, synth.pyramid_sizes(120, 160), synth.LAMBDA), torch)
    n_f, _ = T.tdpm_model_info(ctx, mid)
    T.tdpm_set_fusion(ctx, True)
    fused, names = _stage_names(T, ctx, lambda: T.tdpm_build_pyramid_scores(ctx, mid, dp, T.FORM_DECOMPOSED,
                                                                             T.PREC_BF16X3))
    assert {"zsep_tc", "zproj_tc", "sep"} <= names
    T.tdpm_set_fusion(ctx, False)
    plain = T.tdpm_build_pyramid_scores(ctx, mid, dp, T.FORM_DECOMPOSED, T.PREC_BF16X3)
    T.tdpm_set_fusion(ctx, True)
    for fid in range(n_f):
        for j in range(0, 20):
            try:
                a = T.tdpm_get_maps(ctx, fused, T.MAP_FILTER_SCORE, fid, j)
            except T.TdpmError:
                continue
            assert_same_sum(a, T.tdpm_get_maps(ctx, plain, T.MAP_FILTER_SCORE, fid, j))
    T.tdpm_release(ctx, fused)
    T.tdpm_release(ctx, plain)


@pytest.mark.parametrize("ranks", [(40, 30), (55, 36), (64, 13), (64, 32), (32, 32)])
def test_terms_kernel_matches_oracle_at_high_rank(torch, T, ctx, ranks):
    """The terms-on-M kernel with groups whose filters span several warps of terms (30 terms: four filters per
    128-term group, 40 terms: three; 13 terms: nine filters; 32 terms: four, on 6x6 parts and, at (32, 32), on 7x7
    roots), with Sec. 5's (S, T) root / part rank pairs, against the oracle on the same factors (split BF16: 1e-4 of the FP64 result), and the detections at >= 99.5% agreement. A group whose every
    filter is at its exact rank (h*w: the slice form; all of them at (55, 36)) is scored by the full form's kernel on
    the original filters, so its maps equal the full correlation's."""
    wl = synth.config_c2()
    pyr = wl.pyramids[0]
    mid = T.tdpm_load_model(ctx, wl.model)
    S, Tp = ranks
    rk = []
    for c in wl.model.components:
        rk.append(S)
        rk.extend([Tp] * len(c.parts))
    T.tdpm_decompose_ranks(ctx, mid, rk, max_iters=60, seed=4)
    for gi in range(T.tdpm_model_info(ctx, mid)[1]):
        info = T.tdpm_group_info(ctx, mid, gi)
        exact = info["h"] * info["w"]
        assert info["rank"] == sum(min(S if info["role"] == 0 else Tp, exact) for _ in info["filter_ids"])
    sid, names = _stage_names(T, ctx, lambda: T.tdpm_build_pyramid_scores(ctx, mid, device_pyramid(pyr, torch),
                                                                           T.FORM_DECOMPOSED, T.PREC_BF16X3))
    exact_roots, exact_parts = S >= 55, Tp >= 36
    assert ("zsep_tc" in names) == (not (exact_roots and exact_parts))
    assert ("corr_tc" in names) == (exact_roots or exact_parts)
    ref = orc.score_pyramid(wl.model, pyr, filters=_factor_filters(T, ctx, mid, torch, False))
    for m in ref:
        got = T.tdpm_get_maps(ctx, sid, T.MAP_FINAL_SCORE, m["component"], m["level"])
        assert rel_err(got, m["score"]) <= 1e-4
    if Tp == 36:
        n_f, _ = T.tdpm_model_info(ctx, mid)
        for fid in range(n_f):
            f = wl.model.filters()[fid]
            if f.shape[:2] != (6, 6):
                continue
            got = T.tdpm_get_maps(ctx, sid, T.MAP_FILTER_SCORE, fid, 5)
            assert rel_err(got, orc.correlate(pyr.levels[5], f.astype(np.float64))) <= 1e-4
    tau = float(np.percentile(orc.all_scores(ref), 99))
    assert agreement(det_keys(T.tdpm_detect(ctx, sid, tau)), det_keys(orc.detect(ref, tau))) >= 0.995
    T.tdpm_release(ctx, sid)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_every_fused_form_gives_the_same_maps(torch, T, prec, monkeypatch):
    """The fused kernel's forms (one CTA per item; persistent with one or two feature stages and Z buffers, forced
    through TDPM_ZSEP_FORM; a form that does not fit a shape falls back to the default) give identical maps."""
    wl = synth.config_c2()
    pyrs = _images(5)
    p = T.PREC_BF16X3 if prec == "bf16x3" else T.PREC_BF16
    results = []
    for form in ("0", "1", "2", "3", "4"):
        monkeypatch.setenv("TDPM_ZSEP_FORM", form)
        c = T.tdpm_create(0)
        mid = T.tdpm_load_model(c, wl.model)
        T.tdpm_decompose(c, mid, 8, T.DECOMP_PER_FILTER, max_iters=40, seed=2)
        n_f, _ = T.tdpm_model_info(c, mid)
        sid = T.tdpm_build_batch_scores(c, mid, [device_pyramid(py, torch) for py in pyrs], T.FORM_DECOMPOSED, p)
        maps = {}
        for i, py in enumerate(pyrs):
            for fid in range(n_f):
                for j in range(len(py.levels)):
                    try:
                        maps[(i, fid, j)] = T.tdpm_get_maps(c, sid, T.MAP_FILTER_SCORE, fid, j, image=i)
                    except T.TdpmError:
                        pass
        results.append(maps)
        T.tdpm_destroy(c)
    assert len(results[0]) > 100
    for other in results[1:]:
        assert other.keys() == results[0].keys()
        for key, a in results[0].items():
            np.testing.assert_array_equal(other[key], a)
