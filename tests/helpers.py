"""Shared test utilities: move seeded inputs to the GPU, compare the CUDA path with the oracle."""
from __future__ import annotations

import math
from typing import Dict, List, Sequence, Tuple

import numpy as np

EPS32 = float(np.finfo(np.float32).eps)


def device_pyramid(pyr, torch):
    from paper_1707_03268_gb300 import tdpm
    levels = [torch.from_numpy(np.ascontiguousarray(l)).cuda() for l in pyr.levels]
    return tdpm.DevicePyramid(levels, pyr.lam)


def rel_err(got: np.ndarray, ref: np.ndarray) -> float:
    """max |got - ref| / max |ref| (the score tolerance is relative to the largest score)."""
    if ref.size == 0:
        return 0.0
    return float(np.max(np.abs(got.astype(np.float64) - ref)) / max(np.max(np.abs(ref)), 1e-30))


def dt_value(S: np.ndarray, d: Sequence[float], qy: int, qx: int, py: int, px: int) -> float:
    """FP64 value of placing the part at (qy, qx) for anchor (py, px)."""
    dx, dy = qx - px, qy - py
    return float(S[qy, qx]) - (d[0] * dx + d[1] * dx * dx + d[2] * dy + d[3] * dy * dy)


def dt_tie_tol(S: np.ndarray, d: Sequence[float], qy: int, qx: int, py: int, px: int) -> float:
    """Rounding allowance of an FP32 evaluation of one candidate: a few ulps of the terms it adds up."""
    dx, dy = qx - px, qy - py
    mag = abs(float(S[qy, qx])) + abs(d[0] * dx) + abs(d[1] * dx * dx) + abs(d[2] * dy) + abs(d[3] * dy * dy)
    return 8.0 * EPS32 * (1.0 + mag)


def check_argmax(S: np.ndarray, d, gy: np.ndarray, gx: np.ndarray, oy: np.ndarray, ox: np.ndarray,
                 py: np.ndarray, px: np.ndarray) -> Tuple[int, int]:
    """Compare GPU argmax (gy, gx) with the oracle's (oy, ox) at anchors (py, px). A differing choice is a tie when
    the oracle's FP64 value at the GPU's choice is within FP32 rounding of the maximum. Returns (ties, bad)."""
    ties = bad = 0
    diff = np.argwhere((gy != oy) | (gx != ox))
    for idx in diff:
        i = tuple(idx)
        v_best = dt_value(S, d, int(oy[i]), int(ox[i]), int(py[i]), int(px[i]))
        v_gpu = dt_value(S, d, int(gy[i]), int(gx[i]), int(py[i]), int(px[i]))
        tol = dt_tie_tol(S, d, int(gy[i]), int(gx[i]), int(py[i]), int(px[i])) + \
            dt_tie_tol(S, d, int(oy[i]), int(ox[i]), int(py[i]), int(px[i]))
        if v_best - v_gpu <= tol:
            ties += 1
        else:
            bad += 1
    return ties, bad


def det_keys(dets) -> set:
    if isinstance(dets, np.ndarray):
        return set(zip(dets["component"].tolist(), dets["level"].tolist(), dets["y"].tolist(), dets["x"].tolist()))
    return set((d[0], d[1], d[2], d[3]) for d in dets)


def agreement(a: set, b: set) -> float:
    u = a | b
    return 1.0 if not u else len(a & b) / len(u)


# Two evaluations of the same decomposed filter map in FP32 that add the same products in different orders (the sum
# over a filter's CP terms, and lambda_r folded into a_r or applied after the passes) differ by FP32 rounding only: a
# few ulps of the partial sums per term, at most about 40 terms here. Relative to the map's largest value.
SUM_ORDER_TOL = 2e-5


def assert_same_sum(a: np.ndarray, b: np.ndarray, tol: float = SUM_ORDER_TOL) -> None:
    assert a.shape == b.shape
    if b.size:
        assert rel_err(a, b.astype(np.float64)) <= tol, rel_err(a, b.astype(np.float64))
