"""CPU checks of arithmetic rules the kernels rely on (no GPU).

The NMS overlap masks decide "intersection / area > overlap" without the FP64 division outside a narrow band: with
prod = fl(overlap * area), inter >= fl(prod * (1 + 2^-50)) implies fl(inter / area) > overlap, and
inter <= fl(prod * (1 - 2^-50)) implies the opposite. Both sides of that rule are IEEE double operations, which numpy
float64 reproduces, so the rule is checked here against the division on random and on adversarially close cases.
"""
import numpy as np


def _fast(inter, area, overlap):
    prod = overlap * area
    if inter >= prod * (1.0 + 2.0 ** -50):
        return True
    if inter <= prod * (1.0 - 2.0 ** -50):
        return False
    return inter / area > overlap


def test_nms_division_free_rule_matches_the_division():
    rng = np.random.default_rng(3)
    overlaps = [0.5, 0.3, 0.7, 0.25, 1.0 / 3.0, 0.1, 0.9, np.nextafter(0.5, 1.0), np.nextafter(0.5, 0.0)]
    n_band = 0
    for overlap in overlaps:
        for _ in range(20000):
            area = float(rng.uniform(1.0, 1e6))
            inter = float(rng.uniform(0.0, area))
            assert _fast(inter, area, overlap) == (inter / area > overlap)
        # adversarial: inter within a few ulps of overlap * area
        for _ in range(20000):
            area = float(rng.uniform(1.0, 1e6)) * float(2.0 ** rng.integers(-20, 20))
            inter = overlap * area
            for _k in range(int(rng.integers(0, 6))):
                inter = np.nextafter(inter, np.inf if rng.random() < 0.5 else -np.inf)
            inter = float(inter)
            fast = _fast(inter, area, overlap)
            exact = inter / area > overlap
            assert fast == exact, (inter, area, overlap)
            n_band += int(abs(inter - overlap * area) <= overlap * area * 2.0 ** -50)
    assert n_band > 0  # the band (where the division decides) was exercised


def test_planted_objects_line_up_with_their_filters():
    """The cascade's positive examples: a planted instance raises the root's response at the placement, and the last
    part's at its anchor (part windows may overlap; the later one is written over the earlier), far above the
    background, and touches no other level."""
    import pytest

    from oracle import oracle as orc
    from paper_1707_03268_gb300 import synth

    rng = np.random.default_rng(4)
    model = synth.Model(synth.make_dpm_class(np.random.default_rng(5))[:1])
    comp = model.components[0]
    base = synth.make_pyramid(rng, synth.pyramid_sizes(160, 200), synth.LAMBDA)
    j = synth.LAMBDA + 2
    y, x = 3, 4
    planted = synth.plant_objects(rng, base, model, [(0, j, y, x)])
    root_b = orc.correlate(base.levels[j], comp.root)
    root_p = orc.correlate(planted.levels[j], comp.root)
    assert root_p[y, x] > root_b[y, x] + 1.0 and root_p[y, x] > np.max(root_b) + 1.0
    p = comp.parts[-1]
    py, px = 2 * y + p.anchor[0], 2 * x + p.anchor[1]
    s_b = orc.correlate(base.levels[j - synth.LAMBDA], p.filt)
    s_p = orc.correlate(planted.levels[j - synth.LAMBDA], p.filt)
    assert s_p[py, px] > np.max(s_b) + 0.5
    untouched = [k for k in range(len(base.levels)) if k not in (j, j - synth.LAMBDA)]
    assert all(np.array_equal(base.levels[k], planted.levels[k]) for k in untouched)
    assert all(0.0 <= l.min() and l.max() <= 0.2 for l in planted.levels)
    with pytest.raises(AssertionError):
        synth.plant_objects(rng, base, model, [(0, j, 10 ** 4, 0)])


def test_synthetic_images_are_seeded_8bit_rgb():
    from paper_1707_03268_gb300 import synth

    a = synth.make_image(np.random.default_rng(1), 37, 53)
    b = synth.make_image(np.random.default_rng(1), 37, 53)
    assert a.dtype == np.uint8 and a.shape == (37, 53, 3) and np.array_equal(a, b)
    assert len(np.unique(a)) > 100  # structure and noise, not a flat image


def test_rank_pairs_and_class_thresholds_of_the_benchmark():
    """The benchmark's (S, T) root / part rank pairs map to per-filter ranks in model order, capped at the exact rank
    h*w; the bank's per-class thresholds (written by the oracle script) expand to one per component."""
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    from paper_1707_03268_gb300 import synth

    wl = synth.config_c2()
    r = bench.filter_ranks(wl.model, 64, 32)
    shapes = [f.shape[:2] for f in wl.model.filters()]
    assert len(r) == len(shapes)
    i = 0
    for c in wl.model.components:
        assert r[i] == c.root.shape[0] * c.root.shape[1]  # S = 64 is past every root's exact rank
        assert all(v == min(32, 36) for v in r[i + 1:i + 1 + len(c.parts)])
        i += 1 + len(c.parts)
    assert list(bench.filter_ranks(wl.model, 8, 40)[1:9]) == [36] * 8  # capped at 6 * 6
    taus = bench.load_taus("c3", 120)
    assert taus.shape == (120,) and np.all(taus[:6] == taus[0]) and taus[0] != taus[6]
    assert np.all(bench.load_taus("c2", 6) == np.float32(bench.load_tau()))
    # the ladder starts from the cheapest part rank and ends at the exact parts
    assert bench.RANK_LADDER[-1][1] == 36 and bench.AGREEMENT_BAR == 0.995
