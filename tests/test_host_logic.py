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
