"""Pins for the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test compares the oracle with something other than itself: values the paper prints, hand-worked examples,
closed forms, textbook reductions and pure-Python brute force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as orc
from oracle import tiny
from paper_1707_03268_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------------------------------------
# formula (1), Sec. 4/5
# ---------------------------------------------------------------------------------------------------------------------
def _read_gain_fixture():
    rows, bound = [], None
    with open(os.path.join(GOLDEN, "gain_formula_sec5.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "bound":
                bound = float(tok[1])
            else:
                rows.append(tuple(int(t) for t in tok))
    return rows, bound


def test_gain_formula_sec5_example():
    rows, bound = _read_gain_fixture()
    shapes = []
    for h, w, L, R, count in rows:
        shapes += [(h, w, L)] * count
    R = rows[0][3]
    g = orc.bank_gain(shapes, R)
    # "beyond 7": the bank is at 7 and the 8x8x32 parts alone are above it
    assert g >= bound - 1e-12 and g < bound + 0.2
    assert orc.gain(8, 8, 32, 6) > bound
    assert math.isclose(g, (8 * 8 * 8 * 32 + 5 * 11 * 32) / (6 * 48 * 8 + 6 * 48), rel_tol=1e-15)


def test_gain_per_filter_values():
    assert orc.gain(8, 8, 32, 6) == pytest.approx(2048 / 288)
    assert orc.gain(5, 11, 32, 6) == pytest.approx(1760 / 288)
    assert orc.gain(6, 6, 32, 8) == pytest.approx(1152 / 352)
    # memory ratio (Sec. 5, last paragraph): h*w*L numbers against R triples of vectors
    h, w, L, R = 6, 6, 32, 8
    assert (h * w * L) / (R * (h + w + L)) == orc.gain(h, w, L, R)


# ---------------------------------------------------------------------------------------------------------------------
# correlation (Sec. 2)
# ---------------------------------------------------------------------------------------------------------------------
def test_correlate_delta_filter_picks_feature():
    rng = np.random.default_rng(10)
    feat = rng.uniform(0, 0.2, size=(9, 13, 32)).astype(np.float32)
    h, w = 4, 5
    for (dy, dx, c) in [(0, 0, 0), (3, 4, 31), (1, 3, 7), (2, 0, 19)]:
        filt = np.zeros((h, w, 32))
        filt[dy, dx, c] = 1.0
        out = orc.correlate(feat, filt)
        assert out.shape == (9 - h + 1, 13 - w + 1)
        np.testing.assert_array_equal(out, feat[dy:dy + out.shape[0], dx:dx + out.shape[1], c].astype(np.float64))


def test_correlate_1x1_is_gemv():
    rng = np.random.default_rng(11)
    feat = rng.uniform(0, 0.2, size=(7, 5, 32)).astype(np.float32)
    f = rng.normal(0, 0.05, size=(1, 1, 32))
    out = orc.correlate(feat, f)
    ref = feat.reshape(-1, 32).astype(np.float64) @ f.reshape(32)
    np.testing.assert_allclose(out.ravel(), ref, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("H,W,h,w", [(5, 6, 2, 3), (4, 4, 4, 4), (6, 3, 1, 2), (3, 7, 3, 1)])
def test_correlate_matches_python_bruteforce(H, W, h, w):
    rng = np.random.default_rng(H * 100 + W * 10 + h)
    L = 3
    feat = rng.uniform(0, 0.2, size=(H, W, L)).astype(np.float32)
    filt = rng.normal(0, 0.05, size=(h, w, L))
    ref = np.array(tiny.correlate(feat.tolist(), filt.tolist()))
    np.testing.assert_allclose(orc.correlate(feat, filt), ref, rtol=1e-12, atol=1e-15)


def test_correlate_filter_larger_than_map_is_empty():
    feat = np.zeros((3, 3, 32), np.float32)
    assert orc.correlate(feat, np.zeros((4, 2, 32))).shape == (0, 2)


# ---------------------------------------------------------------------------------------------------------------------
# CP decomposition (Sec. 4)
# ---------------------------------------------------------------------------------------------------------------------
def test_separable_rank1_equals_direct_correlation():
    """Sec. 4: I o (a (x) b (x) c) = ((I o c) o a) o b (linearity of correlation)."""
    rng = np.random.default_rng(12)
    feat = rng.uniform(0, 0.2, size=(11, 14, 32)).astype(np.float32)
    a, b, c = rng.normal(size=6), rng.normal(size=5), rng.normal(size=32)
    direct = orc.correlate(feat, np.einsum("a,b,c->abc", a, b, c))
    np.testing.assert_allclose(orc.correlate_rank1(feat, a, b, c), direct, rtol=1e-12, atol=1e-13)


def test_full_rank_decomposition_is_exact_and_scores_agree():
    rng = np.random.default_rng(13)
    F = synth.make_filter(rng, 6, 6, "iid")
    w, A, B, C = orc.cp_full_rank(F)
    assert A.shape[1] == 36
    np.testing.assert_array_equal(orc.cp_reconstruct(w, [A, B, C]), F.astype(np.float64))
    feat = rng.uniform(0, 0.2, size=(12, 10, 32)).astype(np.float32)
    sep = sum(w[r] * orc.correlate_rank1(feat, A[:, r], B[:, r], C[:, r]) for r in range(A.shape[1]))
    np.testing.assert_allclose(sep, orc.correlate(feat, F), rtol=1e-11, atol=1e-13)


def _planted(rng, dims, R):
    U = [rng.standard_normal((n, R)) for n in dims]
    return U, orc.cp_reconstruct(np.ones(R), U)


def _congruence(U_true, U_est):
    """Best-matching column cosine product over a permutation (greedy; factors are generic)."""
    R = U_true[0].shape[1]
    used, worst = set(), 1.0
    for r in range(R):
        best, arg = -1.0, None
        for s in range(R):
            if s in used:
                continue
            cos = 1.0
            for ut, ue in zip(U_true, U_est):
                cos *= abs(ut[:, r] @ ue[:, s]) / (np.linalg.norm(ut[:, r]) * np.linalg.norm(ue[:, s]))
            if cos > best:
                best, arg = cos, s
        used.add(arg)
        worst = min(worst, best)
    return worst


def test_als_recovers_planted_rank_kruskal():
    """Kruskal (Sec. 4): generic factors with R <= (k_A + k_B + k_C)/2 - 1 give an essentially unique CP form, so ALS
    must reach zero error and return the planted factors up to permutation and scale."""
    rng = np.random.default_rng(14)
    dims, R = (6, 6, 32), 4
    assert R <= 0.5 * (min(6, R) + min(6, R) + min(32, R)) - 1
    U, T = _planted(rng, dims, R)
    best = None
    for seed in range(4):
        w, V, hist = orc.cp_als(T, R, max_iters=2000, tol=0.0, eps=1e-13, seed=seed)
        err = np.linalg.norm(T - orc.cp_reconstruct(w, V)) / np.linalg.norm(T)
        if best is None or err < best[0]:
            best = (err, V)
    assert best[0] <= 1e-10
    assert _congruence(U, best[1]) >= 1 - 1e-8


def test_als_rank1_converges_in_one_sweep():
    rng = np.random.default_rng(15)
    U, T = _planted(rng, (5, 7, 32), 1)
    w, V, hist = orc.cp_als(T, 1, max_iters=1, tol=0.0, seed=3)
    assert np.linalg.norm(T - orc.cp_reconstruct(w, V)) <= 1e-12 * np.linalg.norm(T)


def test_als_objective_non_increasing():
    rng = np.random.default_rng(16)
    T = rng.normal(size=(6, 6, 32))
    w, V, hist = orc.cp_als(T, 5, max_iters=60, tol=0.0, seed=1)
    h = np.array(hist)
    assert np.all(np.diff(h) <= 1e-12 * np.linalg.norm(T))
    # the least-squares fit can never beat the full residual of the best rank-0 model
    assert h[-1] < np.linalg.norm(T)


def test_als_joint_order4_planted():
    """Joint decomposition of a stacked K x h x w x 32 filter bank with shared factors and per-filter weights."""
    rng = np.random.default_rng(17)
    dims, R = (10, 6, 6, 32), 5
    U, T = _planted(rng, dims, R)
    best = 1.0
    for seed in range(4):
        w, V, hist = orc.cp_als(T, R, max_iters=3000, tol=0.0, eps=1e-13, seed=seed)
        best = min(best, np.linalg.norm(T - orc.cp_reconstruct(w, V)) / np.linalg.norm(T))
    assert best <= 1e-9
    Lam = V[0] * w
    F = orc.joint_reconstruct(Lam, V[1], V[2], V[3])
    np.testing.assert_allclose(F, T, atol=1e-9 * np.abs(T).max())


def test_rank_criterion_monotone_in_e():
    rng = np.random.default_rng(18)
    F = synth.make_filter(rng, 6, 6, "dpm")
    w, V, _ = orc.cp_als(F, 4, max_iters=200, seed=0)
    Fr = orc.cp_reconstruct(w, V)
    err = np.linalg.norm(F - Fr)
    thr = (4 * 44 / 1152) ** 2
    assert orc.rank_criterion_holds(F, Fr, 4, 1.01 * err / thr)
    assert not orc.rank_criterion_holds(F, Fr, 4, 0.99 * err / thr)


# ---------------------------------------------------------------------------------------------------------------------
# distance transform (Sec. 2 argmax equation)
# ---------------------------------------------------------------------------------------------------------------------
def test_dt1d_hand_worked_examples():
    with open(os.path.join(GOLDEN, "dt1d_hand.txt")) as fh:
        cases = [l for l in fh if l.strip() and not l.startswith("#")]
    assert len(cases) == 2
    for line in cases:
        f, coef, D, I = [np.array([float(t) for t in part.split()]) for part in line.split("|")]
        d, i = orc.dt1d(f, coef[0], coef[1])
        np.testing.assert_array_equal(d, D)
        np.testing.assert_array_equal(i, I.astype(np.int32))


@pytest.mark.parametrize("H,W", [(1, 1), (1, 7), (6, 1), (5, 6), (7, 4)])
def test_dt2d_matches_2d_bruteforce_strict(H, W):
    """Integer maps and power-of-two costs are exact in FP64: values and tie-breaks must match bit for bit."""
    rng = np.random.default_rng(H * 31 + W)
    for _ in range(3):
        S = synth.make_integer_map(rng, H, W, -6, 6).astype(np.float64)
        d = synth.make_pow2_deform(rng).astype(np.float64)
        D, Iy, Ix = orc.dt2d(S, d)
        Dref, Aref = tiny.dt2d(S.tolist(), d.tolist())
        np.testing.assert_array_equal(D, np.array(Dref))
        np.testing.assert_array_equal(np.stack([Iy, Ix], -1), np.array(Aref, dtype=np.int32).reshape(H, W, 2))


def test_dt2d_matches_2d_bruteforce_float():
    rng = np.random.default_rng(19)
    S = rng.normal(size=(6, 7))
    d = np.array([0.03, 0.05, -0.02, 0.08])
    D, Iy, Ix = orc.dt2d(S, d)
    Dref, Aref = tiny.dt2d(S.tolist(), d.tolist())
    np.testing.assert_allclose(D, np.array(Dref), rtol=0, atol=1e-14)
    np.testing.assert_array_equal(np.stack([Iy, Ix], -1), np.array(Aref, dtype=np.int32).reshape(6, 7, 2))


def test_dt2d_huge_costs_is_identity():
    rng = np.random.default_rng(20)
    S = rng.normal(size=(9, 8))
    # large quadratic terms, small linear ones: every move costs more than the map's range
    D, Iy, Ix = orc.dt2d(S, [0.5, 1e6, -0.5, 1e6])
    np.testing.assert_array_equal(D, S)
    yy, xx = np.meshgrid(np.arange(9), np.arange(8), indexing="ij")
    np.testing.assert_array_equal(Iy, yy)
    np.testing.assert_array_equal(Ix, xx)


def test_dt1d_constant_map_closed_form():
    """For a constant map the best displacement minimises lin*t + quad*t^2 over integers t in [-p, n-1-p]: the integer
    nearest to -lin/(2 quad) (the lower one on a half-way tie), clamped to the range."""
    n = 40
    # dyadic coefficients keep every cost exact, so the half-way case (-0.875, 0.125), t0 = 3.5, is a true tie
    for lin, quad in [(0.375, 0.0625), (-0.875, 0.125), (0.046875, 0.0009765625), (0.0, 0.015625), (0.125, 0.0625)]:
        D, I = orc.dt1d(np.full(n, 2.5), lin, quad)
        t0 = -lin / (2 * quad)
        t_star = math.ceil(t0 - 0.5)
        for p in range(n):
            t = min(max(t_star, -p), n - 1 - p)
            assert I[p] == p + t
            assert D[p] == pytest.approx(2.5 - (lin * t + quad * t * t), abs=1e-14)


def test_dt2d_single_spike_closed_form():
    H, W = 8, 9
    S = np.full((H, W), -1e9)
    S[5, 2] = 3.0
    d = [0.2, 0.1, -0.3, 0.05]
    D, Iy, Ix = orc.dt2d(S, d)
    for y in range(H):
        for x in range(W):
            dx, dy = 2 - x, 5 - y
            assert D[y, x] == pytest.approx(3.0 - (d[0] * dx + d[1] * dx * dx + d[2] * dy + d[3] * dy * dy), abs=1e-12)
            assert (Iy[y, x], Ix[y, x]) == (5, 2)


# ---------------------------------------------------------------------------------------------------------------------
# assembly and threshold (Sec. 2 score, Algorithm 1)
# ---------------------------------------------------------------------------------------------------------------------
def _tiny_workload(seed=21):
    rng = np.random.default_rng(seed)
    comp = synth.make_component(rng, (2, 3), [(2, 2), (3, 2)], kind="iid", bias=0.25)
    pyr = synth.make_pyramid(rng, [(10, 12), (5, 6)], lam=1)
    return synth.Model([comp]), pyr


def test_score_equals_sum_of_stated_terms_and_parts_are_optimal():
    model, pyr = _tiny_workload()
    comp = model.components[0]
    scored = orc.score_pyramid(model, pyr)
    assert len(scored) == 1
    m = scored[0]
    root_lv, part_lv = pyr.levels[1].tolist(), pyr.levels[0].tolist()
    parts = [(p.filt.tolist(), p.anchor, p.deform.tolist()) for p in comp.parts]
    Y, X = m["score"].shape
    assert Y > 0 and X > 0
    for y in range(Y):
        for x in range(X):
            pos = [(int(m["part_y"][i, y, x]), int(m["part_x"][i, y, x])) for i in range(len(parts))]
            s = tiny.hypothesis_score(root_lv, part_lv, comp.root.tolist(), parts, comp.bias, y, x, pos)
            assert s == pytest.approx(m["score"][y, x], abs=1e-12)
            # each reported part position is a best placement for its anchor (Sec. 2 argmax equation)
            for i, (filt, (vy, vx), d) in enumerate(parts):
                best = max(tiny.dot_at(part_lv, filt, qy, qx) - tiny.deform_cost(d, qx - (2 * x + vx), qy - (2 * y + vy))
                           for qy in range(len(part_lv) - len(filt) + 1) for qx in range(len(part_lv[0]) - len(filt[0]) + 1))
                got = tiny.dot_at(part_lv, filt, *pos[i]) - tiny.deform_cost(d, pos[i][1] - (2 * x + vx),
                                                                               pos[i][0] - (2 * y + vy))
                assert got == pytest.approx(best, abs=1e-12)


def test_root_domain_keeps_every_anchor_inside():
    model, pyr = _tiny_workload()
    comp = model.components[0]
    (H, W), (Hp, Wp) = pyr.sizes[1], pyr.sizes[0]
    Y, X = orc.root_domain((H, W), (Hp, Wp), comp.root.shape[:2], [(p.filt.shape[:2], p.anchor) for p in comp.parts])
    for p in comp.parts:
        hp, wp = p.filt.shape[:2]
        assert 2 * (Y - 1) + p.anchor[0] <= Hp - hp and 2 * (X - 1) + p.anchor[1] <= Wp - wp
    assert Y <= H - comp.root.shape[0] + 1 and X <= W - comp.root.shape[1] + 1
    # one more row or column would put the root or some part outside its map
    assert (Y == H - comp.root.shape[0] + 1) or any(2 * Y + p.anchor[0] > Hp - p.filt.shape[0] for p in comp.parts)
    assert (X == W - comp.root.shape[1] + 1) or any(2 * X + p.anchor[1] > Wp - p.filt.shape[1] for p in comp.parts)


def test_threshold_extremes_and_order():
    model, pyr = _tiny_workload()
    scored = orc.score_pyramid(model, pyr)
    n_all = sum(m["score"].size for m in scored)
    assert len(orc.detect(scored, -math.inf)) == n_all
    assert orc.detect(scored, math.inf) == []
    med = float(np.median(orc.all_scores(scored)))
    dets = orc.detect(scored, med)
    assert all(d[4] >= med for d in dets)
    assert dets == sorted(dets, key=lambda d: d[:4])


def test_decomposed_scores_equal_full_at_full_rank():
    """Decomposed and full scores agree when the decomposition is exact (full rank)."""
    model, pyr = _tiny_workload(22)
    full = orc.score_pyramid(model, pyr)
    filters = []
    for F in model.filters():
        w, A, B, C = orc.cp_full_rank(F)
        filters.append(orc.cp_reconstruct(w, [A, B, C]))
    dec = orc.score_pyramid(model, pyr, filters=filters)
    for a, b in zip(full, dec):
        np.testing.assert_allclose(a["score"], b["score"], rtol=0, atol=1e-13)
        np.testing.assert_array_equal(a["part_y"], b["part_y"])


def test_pyramid_shape_matches_dpm_convention():
    sizes = synth.pyramid_sizes(375, 500)
    assert len(sizes) == 36
    for j in range(synth.LAMBDA, len(sizes)):
        (H, W), (Hp, Wp) = sizes[j], sizes[j - synth.LAMBDA]
        assert Hp >= 2 * H and Wp >= 2 * W


def test_select_rank_finds_planted_rank():
    """Sec. 4 rank detection on filters of known rank k (a sum of k outer products, FP32): the criterion fails below k
    (the missing terms carry about a fifth of the norm, far above e (r (N+M+L) / NML)^2 at e = 1) and holds at k (the
    ALS fit is exact up to FP32 rounding), so the smallest r meeting it is k."""
    rng = np.random.default_rng(31)
    for k in (1, 2, 4):
        F = synth.make_filter(rng, 6, 6, "dpm", n_terms=k, decay=0.8)
        r, met = orc.select_rank(F, 1.0, 12, max_iters=500, seed=1)
        assert met and r == k, (k, r, met)


def test_select_rank_cap_and_exact_form():
    """A full-rank filter with a tiny e meets the test only with the exact slice form (r = h*w, error 0); a cap below
    h*w returns the cap, unmet."""
    rng = np.random.default_rng(32)
    F = rng.normal(0.0, 0.05, size=(2, 2, 32)).astype(np.float32)
    r, met = orc.select_rank(F, 1e-12, 10, max_iters=50)
    assert (r, met) == (4, True)
    r, met = orc.select_rank(F, 1e-12, 3, max_iters=50)
    assert (r, met) == (3, False)


def test_nms_keeps_the_best_of_overlapping_boxes():
    """Hand-made cases: the highest box of a cluster survives, a box covered by more than `overlap` of its own area
    goes, one covered by exactly half stays (strictly greater suppresses), other images and classes are independent,
    and score ties go to the earlier record."""
    root_hw = [(4, 4), (4, 4)]
    dets = [
        (0, 0, 0, 0, 0, 1.0),   # box [0,4)x[0,4) at cell 1 (level 0, cell0 = 1)
        (0, 0, 0, 0, 1, 2.0),   # [1,5): covers 3/4 of box 0 -> box 0 suppressed
        (0, 0, 0, 0, 3, 1.5),   # [3,7): overlap with box 1 is 2/4 = 0.5, not > 0.5 -> kept
        (1, 0, 0, 0, 0, 0.5),   # another image: independent
        (0, 1, 0, 0, 1, 0.1),   # another class (component 1 -> class 1): independent
        (0, 0, 0, 10, 10, 2.0), # far away, tie in score with record 1 -> both kept
    ]
    kept = orc.nms(dets, root_hw, cell0=1.0, lam=10, overlap=0.5, component_class=[0, 1])
    assert kept == [1, 2, 3, 4, 5]
    # one class for both components: record 4 overlaps record 1 (same box) and has a lower score -> suppressed
    kept = orc.nms(dets, root_hw, cell0=1.0, lam=10, overlap=0.5, component_class=[0, 0])
    assert kept == [1, 2, 3, 5]
    # level scale: level 10 with lam 10 doubles the cell, so (y, x) = (0, 1) covers [2, 10) and hides a level-0 box at
    # [2, 6) entirely (its own area is the reference)
    dets2 = [(0, 0, 10, 0, 1, 3.0), (0, 0, 0, 0, 2, 1.0)]
    assert orc.nms(dets2, root_hw, cell0=1.0, lam=10) == [0]
    # ties: the earlier record wins
    dets3 = [(0, 0, 0, 0, 0, 1.0), (0, 0, 0, 0, 0, 1.0)]
    assert orc.nms(dets3, root_hw, cell0=1.0, lam=10) == [0]


# ---------------------------------------------------------------------------------------------------------------------
# convolution shortening (Sec. 4 thresholds, Algorithm 1)
# ---------------------------------------------------------------------------------------------------------------------
def _cascade_workload(seed=31, R=3):
    model, pyr = _tiny_workload(seed)
    factors = []
    for f in model.filters():
        w, (A, B, C), _ = orc.cp_als(f.astype(np.float64), R, max_iters=60, seed=1)
        factors.append((w, A, B, C))
    comp = model.components[0]
    Y, X = orc.root_domain(pyr.sizes[1], pyr.sizes[0], comp.root.shape[:2],
                           [(p.filt.shape[:2], p.anchor) for p in comp.parts])
    recs = [(0, 1, y, x) for y in range(Y) for x in range(X)]
    return model, pyr, factors, recs


def test_cascade_partials_end_at_the_decomposed_filter_response():
    """Linearity (Sec. 4): the last partial sum of each slot is the response of the filter rebuilt from its factors, at
    the root position for the root and at the anchor for each part (direct correlation, another code path)."""
    model, pyr, factors, recs = _cascade_workload()
    comp = model.components[0]
    rebuilt = [orc.cp_reconstruct(w, [A, B, C]) for (w, A, B, C) in factors]
    root_map = orc.correlate(pyr.levels[1], rebuilt[0])
    part_maps = [orc.correlate(pyr.levels[0], rebuilt[1 + i]) for i in range(len(comp.parts))]
    for (c, j, y, x) in recs:
        P = orc.cascade_partials(model, pyr, factors, (c, j, y, x))
        assert len(P) == 1 + len(comp.parts) and all(len(p) == 3 for p in P)
        assert P[0][-1] == pytest.approx(root_map[y, x], rel=1e-12, abs=1e-12)
        for i, p in enumerate(comp.parts):
            assert P[1 + i][-1] == pytest.approx(part_maps[i][2 * y + p.anchor[0], 2 * x + p.anchor[1]],
                                                 rel=1e-12, abs=1e-12)


def test_cascade_adds_the_heaviest_term_first():
    """The first partial sum is the term of largest |lambda| alone, evaluated as three 1-D correlations."""
    model, pyr, factors, recs = _cascade_workload()
    w, A, B, C = factors[0]
    r = int(np.argmax(np.abs(w)))
    assert orc.cascade_order(w)[0] == r
    one = w[r] * orc.correlate_rank1(pyr.levels[1], A[:, r], B[:, r], C[:, r])
    for (c, j, y, x) in recs[:7]:
        assert orc.cascade_partials(model, pyr, factors, (c, j, y, x))[0][0] == pytest.approx(one[y, x], rel=1e-12,
                                                                                              abs=1e-12)
    assert orc.cascade_order(np.array([0.5, -2.0, 2.0, 1.0])) == [1, 2, 3, 0]  # ties by index


def test_cascade_thresholds_are_the_tightest_that_keep_every_positive():
    """Sec. 4: with thresholds from a set of positives no positive is pruned, and raising any single threshold above
    its value prunes at least one of them; with no thresholds the cascade keeps every detection."""
    model, pyr, factors, recs = _cascade_workload()
    rng = np.random.default_rng(5)
    pos = [recs[i] for i in rng.choice(len(recs), size=6, replace=False)]
    t = orc.cascade_thresholds(model, lambda img: pyr, factors, [(0,) + p for p in pos])
    assert sorted(t) == [0, 1, 2]
    for p in pos:
        assert orc.cascade_walk(model, pyr, factors, t, p) == (False, 9)
    for fid, tf in t.items():
        for q in range(len(tf)):
            t2 = {k: v.copy() for k, v in t.items()}
            t2[fid][q] = np.nextafter(tf[q], np.inf)
            assert any(orc.cascade_walk(model, pyr, factors, t2, p)[0] for p in pos)
    dets = orc.detect(orc.score_pyramid(model, pyr), -np.inf)
    assert orc.cascade_detect(model, pyr, factors, {}, dets) == list(range(len(dets)))
    # the walk stops at the first partial sum below its threshold and counts the terms it evaluated
    big = {0: np.array([np.inf, np.inf, np.inf])}
    assert orc.cascade_walk(model, pyr, factors, big, recs[0]) == (True, 1)
    part = {2: np.array([-np.inf, np.inf, np.inf])}
    assert orc.cascade_walk(model, pyr, factors, part, recs[0]) == (True, 3 + 3 + 2)


# ---------------------------------------------------------------------------------------------------------------------
# feature extraction block: area-averaging resize and 32-channel HOG
# ---------------------------------------------------------------------------------------------------------------------
from oracle import hog as ohog  # noqa: E402


def test_resize_identity_halving_and_mass():
    rng = np.random.default_rng(3)
    img = rng.uniform(0, 255, size=(12, 18, 3))
    assert np.array_equal(ohog.resize(img, 1.0), img)
    half = ohog.resize(img, 0.5)
    np.testing.assert_allclose(half, 0.25 * (img[0::2, 0::2] + img[1::2, 0::2] + img[0::2, 1::2] + img[1::2, 1::2]),
                               rtol=1e-13)
    const = np.full((17, 23, 3), 7.25)
    np.testing.assert_allclose(ohog.resize(const, 2 ** -0.3), 7.25, rtol=1e-13)
    # 20 -> 16 pixels at s = 0.8: the output intervals tile the input, so the mass scales by 1 / s exactly
    row = rng.uniform(0, 1, size=(1, 20, 1))
    out = ohog.resize(np.repeat(row, 5, axis=0), 0.8)
    assert out.shape == (4, 16, 1)
    assert out[0, :, 0].sum() / 0.8 == pytest.approx(row.sum(), rel=1e-13)
    # odd length halved: the last output pixel is the mean of the one input pixel its interval still covers
    odd = rng.uniform(0, 1, size=(2, 5, 1))
    assert ohog.resize(odd, 0.5)[0, 2, 0] == pytest.approx(0.5 * (odd[0, 4, 0] + odd[1, 4, 0]), rel=1e-13)


def _ramp(h, w, a, b, boost=1):
    """I = a x + b y in every channel, channel `boost` three times as steep."""
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    img = np.stack([a * x + b * y] * 3, axis=2)
    img[..., boost] = 3 * (a * x + b * y)
    return img.astype(np.float32)


@pytest.mark.parametrize("deg", [0.0, 13.0, 47.0, 95.0, 171.0, 200.0, 333.0])
def test_hog_orientation_bin_of_a_ramp(deg):
    """A ramp has one gradient (2a, 2b) (times 3 in the steepest channel, which wins) everywhere: every interior pixel
    votes into the bin whose direction o * 20 degrees is nearest to the gradient's angle modulo 180, plus 9 when the
    gradient points against it."""
    th = math.radians(deg)
    obin, mag = ohog.gradients(_ramp(12, 14, math.cos(th), math.sin(th)))
    o_near = int(round(deg / 20.0)) % 18
    want = o_near if o_near < 9 else o_near
    assert np.all(obin[1:-1, 1:-1] == want)
    assert np.allclose(mag[1:-1, 1:-1], 6.0, rtol=1e-5)   # |3 * (2 cos, 2 sin)| (FP32 image)
    assert np.all(mag[0] == 0) and np.all(mag[:, -1] == 0)


@pytest.mark.parametrize("slope,clipped", [(1.0, True), (3e-6, False)])
def test_hog_features_of_a_ramp_closed_form(slope, clipped):
    """Uniform gradient magnitude m in one bin o: every cell whose votes are complete holds h = sbin^2 m; a cell
    surrounded by such cells has four blocks of energy 4 h^2, so each normalised value is h / sqrt(4 h^2 + 1e-4),
    0.2 once truncated. Channel o and the contrast-insensitive channel o mod 9 are 0.5 * 4 * that value, the four
    texture channels that value / sqrt(18), all others 0."""
    sbin = 8
    img = _ramp(8 * 9, 8 * 8, slope * math.cos(math.radians(40)), slope * math.sin(math.radians(40)))
    f = ohog.hog(img, sbin)
    assert f.shape == (7, 6, 32)
    m = 3 * 2 * slope
    h = sbin * sbin * m
    v = h / math.sqrt(4 * h * h + 1e-4)
    assert (v > 0.2) == clipped
    v = min(v, 0.2)
    want = np.zeros(32)
    want[2] = want[18 + 2] = 2.0 * v
    want[27:31] = v / math.sqrt(18.0)
    for y in range(1, f.shape[0] - 1):
        for x in range(1, f.shape[1] - 1):
            np.testing.assert_allclose(f[y, x], want, rtol=2e-5, atol=1e-12)


def test_hog_equals_brute_force_on_a_small_image():
    rng = np.random.default_rng(8)
    img = rng.integers(0, 256, size=(21, 27, 3)).astype(np.float32)
    obin, mag = ohog.gradients(img)
    for sbin in (4, 8):
        got = ohog.hog(img, sbin)
        want = np.array(tiny.hog_features(obin.tolist(), mag.tolist(), sbin))
        assert got.shape == want.shape
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)


def test_hog_pyramid_levels():
    rng = np.random.default_rng(9)
    img = rng.integers(0, 256, size=(96, 128, 3)).astype(np.float32)
    lv = ohog.hog_pyramid(img, sbin=8, lam=3, min_cells=4)
    np.testing.assert_allclose(lv[0], ohog.hog(img, 4), rtol=1e-12)         # 2x octave, scale 1
    np.testing.assert_allclose(lv[3], ohog.hog(img, 8), rtol=1e-12)         # first root level, scale 1
    np.testing.assert_allclose(lv[4], ohog.hog(ohog.resize(img, 2 ** (-1 / 3)), 8), rtol=1e-12)
    np.testing.assert_allclose(lv[6], ohog.hog(ohog.resize(img, 0.5), 8), rtol=1e-12)
    assert all(min(l.shape[:2]) >= 4 for l in lv[3:])
    for j in range(3):   # every part level is at least twice its root level
        assert lv[j].shape[0] >= 2 * lv[3 + j].shape[0] and lv[j].shape[1] >= 2 * lv[3 + j].shape[1]
