"""Pure-Python brute force for tiny inputs -- test infrastructure, used to pin the oracle.

Nothing here calls the C oracle or numpy arithmetic: every quantity is a Python loop over Python floats, so a mistake
in the oracle's C code or its numpy glue cannot be repeated here by sharing it.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def correlate(feat, filt) -> List[List[float]]:
    """Sec. 2, f . phi(p): out[y][x] = sum_{dy,dx,c} filt[dy][dx][c] * feat[y+dy][x+dx][c] over valid placements."""
    H, W, L = len(feat), len(feat[0]), len(feat[0][0])
    h, w = len(filt), len(filt[0])
    out = []
    for y in range(H - h + 1):
        row = []
        for x in range(W - w + 1):
            acc = 0.0
            for dy in range(h):
                for dx in range(w):
                    for c in range(L):
                        acc += float(filt[dy][dx][c]) * float(feat[y + dy][x + dx][c])
            row.append(acc)
        out.append(row)
    return out


def deform_cost(d: Sequence[float], ddx: int, ddy: int) -> float:
    """d . psi with psi = (dx, dx^2, dy, dy^2), displacement = part position - anchor."""
    return float(d[0]) * ddx + float(d[1]) * ddx * ddx + float(d[2]) * ddy + float(d[3]) * ddy * ddy


def dt2d(S, d) -> Tuple[List[List[float]], List[List[Tuple[int, int]]]]:
    """Sec. 2 argmax equation over the whole map, O(n^4): for every anchor (y, x) the best (qy, qx) of
    S[qy][qx] - d . psi; among equal maxima the lexicographically smallest (qy, qx)."""
    H, W = len(S), len(S[0])
    D, A = [], []
    for y in range(H):
        drow, arow = [], []
        for x in range(W):
            best, arg = None, None
            for qy in range(H):
                for qx in range(W):
                    v = float(S[qy][qx]) - deform_cost(d, qx - x, qy - y)
                    if best is None or v > best:
                        best, arg = v, (qy, qx)
            drow.append(best)
            arow.append(arg)
        D.append(drow)
        A.append(arow)
    return D, A


def dot_at(feat, filt, y: int, x: int) -> float:
    """f . phi at one placement (top-left corner (y, x))."""
    acc = 0.0
    for dy in range(len(filt)):
        for dx in range(len(filt[0])):
            for c in range(len(filt[0][0])):
                acc += float(filt[dy][dx][c]) * float(feat[y + dy][x + dx][c])
    return acc


def hypothesis_score(root_level, part_level, root, parts, bias: float, y0: int, x0: int,
                     positions: Sequence[Tuple[int, int]]) -> float:
    """Sec. 2 score of one hypothesis {p0, p1, ..., pn}: f0 . phi(p0) + sum_i (f_i . phi(p_i) - d_i . psi(p_i, p0)) + b.
    ``parts`` = [(filt, (vy, vx), d)], part i's anchor is (2*y0 + vy, 2*x0 + vx)."""
    s = dot_at(root_level, root, y0, x0) + float(bias)
    for (filt, (vy, vx), d), (py, px) in zip(parts, positions):
        s += dot_at(part_level, filt, py, px) - deform_cost(d, px - (2 * x0 + vx), py - (2 * y0 + vy))
    return s


def hog_features(obin, mag, sbin):
    """Brute force of the HOG cell votes and features from per-pixel bins and magnitudes (nested lists): every
    visible pixel votes bilinearly into its four cells, then each interior cell is normalised by its four 2x2 blocks
    (E = sum of squared contrast-insensitive sums, N = 1 / sqrt(block E + 1e-4)), truncated at 0.2 and projected to
    18 + 9 + 4 channels plus a zero channel."""
    import math
    h, w = len(mag), len(mag[0])
    cy, cx = (2 * h + sbin) // (2 * sbin), (2 * w + sbin) // (2 * sbin)   # floor(n / sbin + 1/2)
    hist = [[[0.0] * 18 for _ in range(cx)] for _ in range(cy)]
    for y in range(1, cy * sbin - 1):
        for x in range(1, cx * sbin - 1):
            yy, xx = min(y, h - 2), min(x, w - 2)
            yp, xp = (y + 0.5) / sbin - 0.5, (x + 0.5) / sbin - 0.5
            iy, ix = math.floor(yp), math.floor(xp)
            for ty, wy in ((iy, 1.0 - (yp - iy)), (iy + 1, yp - iy)):
                for tx, wx in ((ix, 1.0 - (xp - ix)), (ix + 1, xp - ix)):
                    if 0 <= ty < cy and 0 <= tx < cx:
                        hist[ty][tx][obin[yy][xx]] += wy * wx * mag[yy][xx]
    E = [[sum((hist[a][b][o] + hist[a][b][o + 9]) ** 2 for o in range(9)) for b in range(cx)] for a in range(cy)]
    out = []
    for y in range(1, cy - 1):
        row = []
        for x in range(1, cx - 1):
            norms = []
            for a0, b0 in ((y, x), (y, x - 1), (y - 1, x), (y - 1, x - 1)):
                s = E[a0][b0] + E[a0][b0 + 1] + E[a0 + 1][b0] + E[a0 + 1][b0 + 1]
                norms.append(1.0 / math.sqrt(s + 1e-4))
            hc = hist[y][x]
            f = [0.0] * 32
            for o in range(18):
                f[o] = 0.5 * sum(min(hc[o] * n, 0.2) for n in norms)
            for o in range(9):
                f[18 + o] = 0.5 * sum(min((hc[o] + hc[o + 9]) * n, 0.2) for n in norms)
            for k, n in enumerate(norms):
                f[27 + k] = sum(min(hc[o] * n, 0.2) for o in range(18)) / math.sqrt(18.0)
            row.append(f)
        out.append(row)
    return out
