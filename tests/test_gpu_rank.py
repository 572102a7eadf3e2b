"""GPU: automatic rank selection (Sec. 4 rank detection) and scoring with per-filter ranks that differ.

Filters of known rank (sums of k outer products) make the smallest rank meeting the criterion unique at e = 10: one
rank below, the missing term leaves an error at least 1.5 times the threshold; at the planted rank the ALS fit is
exact to far inside it. So the library's choice (its own ALS) must equal the planted ranks and the oracle's choice
(the oracle's ALS, best of three starts). The scores of the resulting model, whose filter groups mix ranks 1 to 5,
go through the fused decomposed kernel and must equal the two-launch form bit for bit and the oracle on the same
factors within the split-BF16 tolerance.
"""
import numpy as np
import pytest

from helpers import assert_same_sum, device_pyramid, rel_err
from oracle import oracle as orc
from paper_1707_03268_gb300 import synth

pytestmark = pytest.mark.gpu

PART_RANKS = [1, 2, 3, 5, 2, 3, 1, 4]
ROOT_RANK = 4


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


def _planted_model(seed=41):
    rng = np.random.default_rng(seed)
    comp = synth.make_component(rng, (6, 11), [(6, 6)] * len(PART_RANKS), kind="dpm")
    comp.root = synth.make_filter(rng, 6, 11, "dpm", n_terms=ROOT_RANK, decay=0.8)
    for p, k in zip(comp.parts, PART_RANKS):
        p.filt = synth.make_filter(rng, 6, 6, "dpm", n_terms=k, decay=0.8)
    return synth.Model([comp])


def test_auto_rank_picks_planted_ranks_and_scores(torch, T):
    model = _planted_model()
    ctx = T.tdpm_create(0)
    mid = T.tdpm_load_model(ctx, model)
    rep, ranks = T.tdpm_decompose_auto(ctx, mid, 10.0, 12, max_iters=500, seed=1)
    filters = model.filters()  # model order: root, then parts
    assert list(ranks) == [ROOT_RANK] + PART_RANKS
    assert rep["total_rank"] == sum(ranks)
    for f, r in zip(filters, ranks):
        r_orc, met = orc.select_rank(f, 10.0, 12, max_iters=500, seed=1)
        assert met and r_orc == r
    # the library's factors meet the criterion at the chosen ranks (checked by the oracle's test)
    n_f, n_groups = T.tdpm_model_info(ctx, mid)
    rebuilt = [None] * n_f
    for gi in range(n_groups):
        info = T.tdpm_group_info(ctx, mid, gi)
        A, B, C, Lam = T.tdpm_get_factors(ctx, mid, gi)
        Fk = orc.joint_reconstruct(Lam, A, B, C)
        for k, fid in enumerate(info["filter_ids"]):
            rebuilt[fid] = Fk[k]
            assert orc.rank_criterion_holds(filters[fid], Fk[k], int(ranks[fid]), 10.0)
    # scoring with mixed ranks per filter group: fused = two-launch, and the oracle on the same factors
    pyr = synth.make_pyramid(np.random.default_rng(42), synth.pyramid_sizes(120, 160), synth.LAMBDA)
    dp = device_pyramid(pyr, torch)
    T.tdpm_set_fusion(ctx, True)
    fused = T.tdpm_build_pyramid_scores(ctx, mid, dp, T.FORM_DECOMPOSED, T.PREC_BF16X3)
    T.tdpm_set_fusion(ctx, False)
    plain = T.tdpm_build_pyramid_scores(ctx, mid, dp, T.FORM_DECOMPOSED, T.PREC_BF16X3)
    for fid in range(n_f):
        for j in range(len(pyr.levels)):
            try:
                a = T.tdpm_get_maps(ctx, fused, T.MAP_FILTER_SCORE, fid, j)
            except T.TdpmError:
                continue
            assert_same_sum(a, T.tdpm_get_maps(ctx, plain, T.MAP_FILTER_SCORE, fid, j))
    ref = orc.score_pyramid(model, pyr, filters=rebuilt)
    for m in ref:
        got = T.tdpm_get_maps(ctx, fused, T.MAP_FINAL_SCORE, m["component"], m["level"])
        assert rel_err(got, m["score"]) <= 1e-4
    T.tdpm_release(ctx, fused)
    T.tdpm_release(ctx, plain)
    with pytest.raises(T.TdpmError):
        T.tdpm_decompose_auto(ctx, mid, 0.0, 12)
    with pytest.raises(T.TdpmError):
        T.tdpm_decompose_auto(ctx, mid, 1.0, 0)
    T.tdpm_destroy(ctx)
