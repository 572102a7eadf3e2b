"""FP64 oracle for the DPM scoring path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import this module; it shares no
code with the CUDA library. FP32 inputs are widened to FP64 and every quantity is computed from its definition:

* ``correlate``            filter response at every valid placement (Sec. 2 score equation; Sec. 4 cost alpha)
* ``correlate_rank1``      one term of the separable form ((I o c) o a) o b (Sec. 4, I o T identity)
* ``dt1d`` / ``dt2d``      generalised distance transform with argmax, brute force (Sec. 2 argmax equation)
* ``cp_reconstruct``       sum of rank-1 tensor products (Sec. 4, CP decomposition, Fig. 2)
* ``cp_full_rank``         an exact decomposition with R = h*w slices (Sec. 4: every tensor has a CP form)
* ``cp_als``               alternating least squares, one exact least-squares solve per factor (Sec. 4, ALS cycle)
* ``gain``                 formula (1) of Sec. 4
* ``select_rank``          the rank detection of Sec. 4: the smallest r meeting the error criterion
* ``score_pyramid``        steps 1-3 for every component and root level (Sec. 2 score; Algorithm 1 steps 12-13)
* ``detect``               step 4, threshold (Algorithm 1 steps 15-16)
* ``nms``                  greedy non-maximum suppression of detections (a DPM convention; the paper has none)
* ``cascade_*``            convolution shortening (Sec. 4 thresholds t_i, Algorithm 1 steps 4-9)

Readings of points the paper leaves open (they are listed with reasons in the design notes): valid correlation with no
padding; the part level of root level j is j - lam and part i of a root at (y, x) is anchored at (2y + vy, 2x + vx);
the deformation cost is d . (dx, dx^2, dy, dy^2) with displacement = part position - anchor, over the whole part map;
among equal maxima the lexicographically smallest (row, column) wins; a root position is scored only where the root
filter and every anchored part position lie inside their maps.
"""
from __future__ import annotations

import ctypes
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import build as _build

_LIB = None
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int32)


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        L = ctypes.CDLL(_build.build())
        L.oracle_correlate.argtypes = [_fp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                       ctypes.c_int, _dp]
        L.oracle_correlate_rank1.argtypes = [_fp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp,
                                             ctypes.c_int, _dp, _dp, _dp]
        L.oracle_dt1d.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _ip]
        L.oracle_dt2d.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, _dp, _ip, _ip]
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_set_num_threads.argtypes = [ctypes.c_int]
        _LIB = L
    return _LIB


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_num_threads(n: int) -> None:
    lib().oracle_set_num_threads(int(n))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


# ----------------------------------------------------------------------------------------------------------------------
# Step 1: correlation (Sec. 2 score equation, Sec. 4)
# ----------------------------------------------------------------------------------------------------------------------
def correlate(feat: np.ndarray, filt: np.ndarray) -> np.ndarray:
    """out[y][x] = sum_{dy,dx,c} filt[dy][dx][c] * feat[y+dy][x+dx][c] over valid placements (FP64)."""
    feat = _f32(feat)
    filt = _f64(filt)
    H, W, L = feat.shape
    h, w, L2 = filt.shape
    assert L == L2
    Ho, Wo = H - h + 1, W - w + 1
    out = np.zeros((max(Ho, 0), max(Wo, 0)), dtype=np.float64)
    if Ho > 0 and Wo > 0:
        lib().oracle_correlate(_ptr(feat, _fp), H, W, L, _ptr(filt, _dp), h, w, _ptr(out, _dp))
    return out


def correlate_rank1(feat: np.ndarray, a: np.ndarray, b: np.ndarray, c: np.ndarray) -> np.ndarray:
    """((I o c) o a) o b for one rank-1 filter a (x) b (x) c, evaluated as three 1-D correlations (Sec. 4)."""
    feat = _f32(feat)
    a, b, c = _f64(a), _f64(b), _f64(c)
    H, W, L = feat.shape
    h, w = a.shape[0], b.shape[0]
    Ho, Wo = H - h + 1, W - w + 1
    out = np.zeros((max(Ho, 0), max(Wo, 0)), dtype=np.float64)
    if Ho > 0 and Wo > 0:
        scratch = np.zeros(H * W + Ho * W, dtype=np.float64)
        lib().oracle_correlate_rank1(_ptr(feat, _fp), H, W, L, _ptr(a, _dp), h, _ptr(b, _dp), w, _ptr(c, _dp),
                                     _ptr(out, _dp), _ptr(scratch, _dp))
    return out


# ----------------------------------------------------------------------------------------------------------------------
# Step 2: generalised distance transform (Sec. 2 argmax equation)
# ----------------------------------------------------------------------------------------------------------------------
def dt1d(f: np.ndarray, lin: float, quad: float) -> Tuple[np.ndarray, np.ndarray]:
    """D[p] = max_q f[q] - (lin*(q-p) + quad*(q-p)^2); I[p] = smallest maximising q."""
    f = _f64(f)
    n = f.shape[0]
    D = np.zeros(n, dtype=np.float64)
    I = np.zeros(n, dtype=np.int32)
    lib().oracle_dt1d(_ptr(f, _dp), n, float(lin), float(quad), _ptr(D, _dp), _ptr(I, _ip))
    return D, I


def dt2d(S: np.ndarray, d: Sequence[float]) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """D[y][x] = max_{qy,qx} S[qy][qx] - d . (qx-x, (qx-x)^2, qy-y, (qy-y)^2), with the argmax (Iy, Ix)."""
    S = _f64(S)
    dd = _f64(np.asarray(d, dtype=np.float64).reshape(4))
    H, W = S.shape
    D = np.zeros((H, W), dtype=np.float64)
    Iy = np.zeros((H, W), dtype=np.int32)
    Ix = np.zeros((H, W), dtype=np.int32)
    if H > 0 and W > 0:
        lib().oracle_dt2d(_ptr(S, _dp), H, W, _ptr(dd, _dp), _ptr(D, _dp), _ptr(Iy, _ip), _ptr(Ix, _ip))
    return D, Iy, Ix


# ----------------------------------------------------------------------------------------------------------------------
# Filter tensors and their CP decomposition (Sec. 4)
# ----------------------------------------------------------------------------------------------------------------------
_LETTERS = "abcdefgh"


def cp_reconstruct(weights: np.ndarray, factors: Sequence[np.ndarray]) -> np.ndarray:
    """sum_r weights[r] * u1[:, r] (x) u2[:, r] (x) ... (Sec. 4: T = a_1 (x) b_1 (x) c_1 + ... + a_R (x) b_R (x) c_R)."""
    n = len(factors)
    expr = "z," + ",".join(_LETTERS[m] + "z" for m in range(n)) + "->" + _LETTERS[:n]
    return np.einsum(expr, _f64(weights), *[_f64(u) for u in factors])


def joint_reconstruct(Lam: np.ndarray, A: np.ndarray, B: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Filters of one shape group from shared factors: F_k = sum_r Lam[k, r] a_r (x) b_r (x) c_r, shape [K][h][w][L]."""
    return np.einsum("kr,ar,br,cr->kabc", _f64(Lam), _f64(A), _f64(B), _f64(C))


def cp_full_rank(F: np.ndarray) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """An exact CP form of an h x w x L filter with R = h*w terms: a_r = e_dy, b_r = e_dx, c_r = F[dy][dx][:]."""
    F = _f64(F)
    h, w, L = F.shape
    R = h * w
    A = np.zeros((h, R))
    B = np.zeros((w, R))
    C = np.zeros((L, R))
    for dy in range(h):
        for dx in range(w):
            r = dy * w + dx
            A[dy, r] = 1.0
            B[dx, r] = 1.0
            C[:, r] = F[dy, dx, :]
    return np.ones(R), A, B, C


def _mttkrp(T: np.ndarray, U: Sequence[np.ndarray], n: int) -> np.ndarray:
    """T_(n) times the Khatri-Rao product of every factor but the n-th."""
    N = T.ndim
    others = [m for m in range(N) if m != n]
    expr = _LETTERS[:N] + "," + ",".join(_LETTERS[m] + "z" for m in others) + "->" + _LETTERS[n] + "z"
    return np.einsum(expr, T, *[U[m] for m in others], optimize=True)


def cp_als(T: np.ndarray, R: int, max_iters: int = 500, eps: float = 0.0, tol: float = 1e-10, seed: int = 0,
           init: Optional[Sequence[np.ndarray]] = None) -> Tuple[np.ndarray, List[np.ndarray], List[float]]:
    """Rank-R CP decomposition by alternating least squares (Sec. 4).

    Each cycle replaces factor n (n = 0, 1, ..., in order) by the exact least-squares minimiser of
    f = ||T - sum_r u1_r (x) u2_r (x) ...||_F with the other factors fixed: the normal equations
    U_n (Hadamard_{m != n} U_m^T U_m) = T_(n) (Khatri-Rao_{m != n} U_m), solved by least squares. The cycle stops at
    ``max_iters``, when f <= eps * ||T||_F (the paper's f < epsilon, made relative), or when f changed by at most
    tol * ||T||_F in the last cycle. Returns (weights, unit-column factors, f after every cycle).
    """
    T = _f64(T)
    N = T.ndim
    if init is None:
        rng = np.random.default_rng(seed)
        U = [rng.standard_normal((T.shape[m], R)) for m in range(N)]
    else:
        U = [_f64(u).copy() for u in init]
    normT = float(np.linalg.norm(T))
    hist: List[float] = []
    for _ in range(max_iters):
        for n in range(N):
            G = np.ones((R, R))
            for m in range(N):
                if m != n:
                    G *= U[m].T @ U[m]
            M = _mttkrp(T, U, n)
            U[n] = np.linalg.lstsq(G, M.T, rcond=None)[0].T
        # move scale into the first factor; the model (and f) is unchanged
        for m in range(1, N):
            nrm = np.linalg.norm(U[m], axis=0)
            nrm[nrm == 0] = 1.0
            U[m] = U[m] / nrm
            U[0] = U[0] * nrm
        f = float(np.linalg.norm(T - cp_reconstruct(np.ones(R), U)))
        hist.append(f)
        if f <= eps * normT:
            break
        if len(hist) > 1 and abs(hist[-2] - f) <= tol * normT:
            break
    w = np.linalg.norm(U[0], axis=0)
    w_safe = np.where(w == 0, 1.0, w)
    U[0] = U[0] / w_safe
    return w, U, hist


def gain(N: int, M: int, L: int, R: int) -> float:
    """Formula (1): NML / (R (N + M + L)), the multiplication and storage ratio of full to rank-R filters."""
    return (N * M * L) / (R * (N + M + L))


def bank_gain(shapes: Sequence[Tuple[int, int, int]], R: int) -> float:
    """Formula (1) summed over a bank: total full products over total rank-R products."""
    full = sum(n * m * l for (n, m, l) in shapes)
    dec = sum(R * (n + m + l) for (n, m, l) in shapes)
    return full / dec


def rank_criterion_holds(F: np.ndarray, F_r: np.ndarray, r: int, e: float) -> bool:
    """Sec. 4 rank detection test: ||f - CP(f, r)||_F < e * (r (N+M+L) / (N M L))^2."""
    N, M, L = F.shape
    return float(np.linalg.norm(_f64(F) - _f64(F_r))) < e * (r * (N + M + L) / (N * M * L)) ** 2


def select_rank(F: np.ndarray, e: float, max_rank: int, max_iters: int = 500, tol: float = 1e-10,
                seed: int = 0, restarts: int = 3) -> Tuple[int, bool]:
    """Sec. 4 rank detection for one filter: the smallest r = 1, 2, ... with ||f - CP(f, r)||_F < e (r (N+M+L) /
    (N M L))^2. CP(f, r) is the best of ``restarts`` runs of ``cp_als`` from seeds seed, seed + 1, ... (one ALS run
    from a random start can stall with a term unused); at r >= N*M it is the exact slice form of ``cp_full_rank``
    (error 0). Returns (r, met): met is False when no r <= max_rank meets the test (r is then max_rank)."""
    N, M, L = F.shape
    for r in range(1, max_rank + 1):
        if r >= N * M:
            w0, A0, B0, C0 = cp_full_rank(F)
            return r, rank_criterion_holds(F, cp_reconstruct(w0, [A0, B0, C0]), r, e)
        fits = []
        for s in range(restarts):
            w, U, _ = cp_als(F, r, max_iters=max_iters, tol=tol, seed=seed + s)
            Fr = cp_reconstruct(w, U)
            fits.append((float(np.linalg.norm(_f64(F) - Fr)), s, Fr))
        best = min(fits, key=lambda t: t[:2])[2]
        if rank_criterion_holds(F, best, r, e):
            return r, True
    return max_rank, False


# ----------------------------------------------------------------------------------------------------------------------
# Steps 1-4 over a pyramid (Sec. 2, Algorithm 1 without the pruning of steps 7-10)
# ----------------------------------------------------------------------------------------------------------------------
def root_domain(level_hw: Tuple[int, int], part_level_hw: Tuple[int, int], root_hw: Tuple[int, int],
                parts: Sequence[Tuple[Tuple[int, int], Tuple[int, int]]]) -> Tuple[int, int]:
    """Root positions scored at one level: (Y, X) with y < Y, x < X iff the root fits at (y, x) and every part's
    anchor (2y + vy, 2x + vx) is a valid placement of that part on the part level. ``parts`` = [((h, w), (vy, vx))]."""
    H, W = level_hw
    Hp, Wp = part_level_hw
    Y, X = H - root_hw[0] + 1, W - root_hw[1] + 1
    for (hp, wp), (vy, vx) in parts:
        Hs, Ws = Hp - hp + 1, Wp - wp + 1
        Y = min(Y, (Hs - 1 - vy) // 2 + 1 if Hs > 0 else 0)
        X = min(X, (Ws - 1 - vx) // 2 + 1 if Ws > 0 else 0)
    return max(Y, 0), max(X, 0)


def score_pyramid(model, pyramid, filters: Optional[Sequence[np.ndarray]] = None) -> List[Dict]:
    """Score every component at every root level (Sec. 2: s = f0 phi(p0) + sum_i (f_i phi(p_i) - d_i psi(p_i, p0))).

    ``filters`` (FP64, model order: root then parts of each component) replaces the model's filters, e.g. filters
    rebuilt from CP factors. Returns one dict per (component, root level) with a non-empty domain, in that order:
    component, level, score [Y][X], part_y / part_x [n_parts][Y][X] (part-level cells).
    """
    levels, lam = pyramid.levels, pyramid.lam
    out: List[Dict] = []
    fid = 0
    for c, comp in enumerate(model.components):
        n = len(comp.parts)
        if filters is None:
            root_f = comp.root.astype(np.float64)
            part_fs = [p.filt.astype(np.float64) for p in comp.parts]
        else:
            root_f = _f64(filters[fid])
            part_fs = [_f64(filters[fid + 1 + i]) for i in range(n)]
        fid += 1 + n
        for j in range(lam, len(levels)):
            l = j - lam
            Y, X = root_domain(levels[j].shape[:2], levels[l].shape[:2], root_f.shape[:2],
                               [(pf.shape[:2], p.anchor) for p, pf in zip(comp.parts, part_fs)])
            if Y <= 0 or X <= 0:
                continue
            total = correlate(levels[j], root_f)[:Y, :X] + float(comp.bias)
            part_y = np.zeros((n, Y, X), dtype=np.int32)
            part_x = np.zeros((n, Y, X), dtype=np.int32)
            for i, (p, pf) in enumerate(zip(comp.parts, part_fs)):
                S = correlate(levels[l], pf)
                D, Iy, Ix = dt2d(S, np.asarray(p.deform, dtype=np.float64))
                ys = p.anchor[0] + 2 * np.arange(Y)
                xs = p.anchor[1] + 2 * np.arange(X)
                total = total + D[np.ix_(ys, xs)]
                part_y[i] = Iy[np.ix_(ys, xs)]
                part_x[i] = Ix[np.ix_(ys, xs)]
            out.append({"component": c, "level": j, "score": total, "part_y": part_y, "part_x": part_x})
    return out


def detect(scored: Sequence[Dict], tau: float) -> List[Tuple]:
    """Step 4 (Algorithm 1 steps 15-16): every scored position with s >= tau, ordered by (component, level, y, x).
    Each detection is (component, level, y, x, score, part_y tuple, part_x tuple)."""
    dets = []
    for m in scored:
        ys, xs = np.nonzero(m["score"] >= tau)
        for y, x in zip(ys.tolist(), xs.tolist()):
            dets.append((m["component"], m["level"], y, x, float(m["score"][y, x]),
                         tuple(int(v) for v in m["part_y"][:, y, x]), tuple(int(v) for v in m["part_x"][:, y, x])))
    dets.sort(key=lambda d: (d[0], d[1], d[2], d[3]))
    return dets


def nms(dets: Sequence[Tuple], root_hw: Sequence[Tuple[int, int]], cell0: float, lam: int, overlap: float = 0.5,
        component_class: Optional[Sequence[int]] = None) -> List[int]:
    """Greedy non-maximum suppression, per (image, class). The paper has no NMS; this is the DPM convention.

    ``dets``: records (image, component, level, y, x, score), ``level`` counted within the image. A detection's box is
    its component's root filter (h0 x w0 cells, ``root_hw``) at its level, whose cells measure
    cell0 * 2 ** (level / lam) image pixels: [x c, x c + w0 c) x [y c, y c + h0 c). Within a group the detections
    are taken by score, highest first (ties: earlier record first); each one not yet suppressed is kept and
    suppresses every later one whose box it covers by more than ``overlap`` of that later box's area. Returns the
    kept records' indices, ascending. Boxes and overlaps are computed in FP64, each product and sum rounded once."""
    cls = component_class
    boxes = []
    for (img, comp, level, y, x, score) in dets:
        c = cell0 * 2.0 ** (level / lam)
        h0, w0 = root_hw[comp]
        x1, y1 = x * c, y * c
        boxes.append((x1, y1, x1 + w0 * c, y1 + h0 * c))
    groups: Dict[Tuple[int, int], List[int]] = {}
    for i, d in enumerate(dets):
        groups.setdefault((d[0], cls[d[1]] if cls is not None else 0), []).append(i)
    kept = []
    for members in groups.values():
        order = sorted(members, key=lambda i: (-dets[i][5], i))
        alive = {i: True for i in order}
        for a, i in enumerate(order):
            if not alive[i]:
                continue
            kept.append(i)
            bi = boxes[i]
            for j in order[a + 1:]:
                if not alive[j]:
                    continue
                bj = boxes[j]
                iw = min(bi[2], bj[2]) - max(bi[0], bj[0])
                ih = min(bi[3], bj[3]) - max(bi[1], bj[1])
                if iw > 0 and ih > 0 and (iw * ih) / ((bj[2] - bj[0]) * (bj[3] - bj[1])) > overlap:
                    alive[j] = False
    return sorted(kept)


def cascade_order(lam: np.ndarray) -> List[int]:
    """A filter's CP terms in the order the cascade adds them: decreasing |lambda_r|, ties by term index (reading of
    "the first i summands" of Sec. 4)."""
    return sorted(range(len(lam)), key=lambda r: (-abs(float(lam[r])), r))


def cascade_partials(model, pyramid, factors: Sequence[Tuple[np.ndarray, ...]], rec: Tuple[int, int, int, int]
                     ) -> List[np.ndarray]:
    """Partial sums of every filter of a root hypothesis (Sec. 4 formula for t_i; Algorithm 1 steps 4-6).

    ``rec`` = (component, root level j, y, x); ``factors[fid]`` = (lam [R], A [h][R], B [w][R], C [32][R]), the
    per-filter CP decomposition of filter fid (model order). Slot 0 is the root at (y, x) on level j, slot 1 + i part
    i at its anchor (2y + vy, 2x + vx) on level j - lam. Term r at window phi is
    lam_r * sum_{dy,dx,c} phi[dy][dx][c] A[dy][r] B[dx][r] C[c][r]; entry q of a slot is the sum of its first q + 1
    terms in ``cascade_order``. FP64."""
    c, j, y, x = rec
    fid = sum(1 + len(comp.parts) for comp in model.components[:c])
    comp = model.components[c]
    wins = [(j, y, x)] + [(j - pyramid.lam, 2 * y + p.anchor[0], 2 * x + p.anchor[1]) for p in comp.parts]
    out = []
    for s, (lv, y0, x0) in enumerate(wins):
        lam, A, B, C = (_f64(a) for a in factors[fid + s])
        h, w = A.shape[0], B.shape[0]
        phi = _f64(pyramid.levels[lv][y0:y0 + h, x0:x0 + w, :])
        assert phi.shape == (h, w, C.shape[0]), "window outside its level"
        terms = lam * np.einsum("ijc,ir,jr,cr->r", phi, A, B, C)
        out.append(np.cumsum(terms[cascade_order(lam)]))
    return out


def cascade_thresholds(model, pyramid_of, factors, positives: Sequence[Tuple[int, int, int, int, int]]
                       ) -> Dict[int, np.ndarray]:
    """t_q of every filter with positives (Sec. 4): the minimum over the positives of its partial sum of the first
    q + 1 terms. ``positives`` = (image, component, level, y, x); ``pyramid_of(image)`` gives that image's pyramid.
    Returns {fid: t [R_fid]}; filters of components without positives are absent (never pruned)."""
    t: Dict[int, np.ndarray] = {}
    for (img, c, j, y, x) in positives:
        fid = sum(1 + len(comp.parts) for comp in model.components[:c])
        for s, p in enumerate(cascade_partials(model, pyramid_of(img), factors, (c, j, y, x))):
            t[fid + s] = p.copy() if fid + s not in t else np.minimum(t[fid + s], p)
    return t


def cascade_walk(model, pyramid, factors, thresholds: Dict[int, np.ndarray], rec: Tuple[int, int, int, int]
                 ) -> Tuple[bool, int]:
    """Algorithm 1 steps 3-11 for one hypothesis: the filters in model order, each one's terms in cascade order,
    stopping at the first partial sum below its threshold. Returns (pruned, terms evaluated)."""
    c = rec[0]
    fid = sum(1 + len(comp.parts) for comp in model.components[:c])
    evaluated = 0
    for s, p in enumerate(cascade_partials(model, pyramid, factors, rec)):
        t = thresholds.get(fid + s)
        for q in range(len(p)):
            evaluated += 1
            if t is not None and p[q] < t[q]:
                return True, evaluated
    return False, evaluated


def cascade_detect(model, pyramid, factors, thresholds: Dict[int, np.ndarray], dets: Sequence[Tuple]) -> List[int]:
    """Algorithm 1's result set D among the step-4 detections ``dets`` (records starting (component, level, y, x),
    as ``detect`` returns them): the indices of those the cascade does not prune, ascending. A pruned hypothesis
    leaves D whatever its score, and one that survives is in D exactly when s >= tau, so D is this subset."""
    return [i for i, d in enumerate(dets) if not cascade_walk(model, pyramid, factors, thresholds, tuple(d[:4]))[0]]


def all_scores(scored: Sequence[Dict]) -> np.ndarray:
    return np.concatenate([m["score"].ravel() for m in scored]) if scored else np.zeros(0)
