"""FP64 oracle for the feature extraction block (HOG pyramid) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU legs may import this module; it shares no code
with the CUDA library. The paper takes the features as given: DPM v5 scores "some variation of HOG" (Sec. 2), and its
feature extraction block costs about a twentieth of the scoring (Sec. 2). The variation used here is the 32-channel
HOG of the DPM release the paper builds on (Felzenszwalb et al., PAMI 2010, Sec. 6: contrast-sensitive and
-insensitive orientation channels under four block normalisations, truncated at 0.2, with the analytic projection),
written from that description. Steps and the readings taken where the description leaves a choice:

* ``resize``       anti-aliased down-scaling by area averaging: pixel i of a row covers [i, i + 1); output pixel j of
                   a row scaled by s covers [j / s, (j + 1) / s) and is the mean of the input over that interval (the
                   same along columns). Output size round(n * s).
* ``gradients``    per pixel (x, y) with 1 <= x <= w - 2, 1 <= y <= h - 2: central differences dx = I[y][x+1] - I[y][x-1],
                   dy = I[y+1][x] - I[y-1][x] in each colour channel; the channel with the largest dx^2 + dy^2 wins
                   (the first on ties). Orientation: the unit directions u_o = (cos(o pi / 9), sin(o pi / 9)), o < 9;
                   the bin is the o with the largest |u_o . (dx, dy)| (the first on ties), plus 9 when that projection
                   is negative (18 contrast-sensitive bins); a pixel whose every projection is <= 0 in absolute value
                   (no gradient) votes into bin 0 with weight 0. These two decisions are taken in FP32, the precision
                   of the kernel, with each product and sum rounded once: the gradient in FP32 from the FP32 image,
                   the projections as fl(fl(u_x dx) + fl(u_y dy)) with u rounded to FP32.
* ``cells``        c = floor(n / sbin + 1/2) cells per dimension; pixel x of the visible region 1 <= x <= c sbin - 2 reads
                   the image at min(x, w - 2) (the last interior column repeats); its magnitude sqrt(dx^2 + dy^2)
                   votes bilinearly into the cells around xp = (x + 0.5) / sbin - 0.5 (and likewise in y).
* ``features``     per interior cell (the outermost ring of cells is dropped: (cy - 2) x (cx - 2) cells), with
                   E = sum_{o<9} (h_o + h_{o+9})^2 per cell and the four 2x2 blocks around the cell giving
                   N_k = 1 / sqrt(sum of their E + 1e-4): 18 channels 0.5 sum_k min(h_o N_k, 0.2), 9 channels
                   0.5 sum_k min((h_o + h_{o+9}) N_k, 0.2), 4 texture channels (1 / sqrt(18)) sum_{o<18} min(h_o N_k, 0.2),
                   and a 32nd channel that is 0.
* ``pyramid``      lam scales 2^(-i / lam) of the image (area averaging); then each further octave halves the previous
                   one. Levels 0 .. lam - 1 are the features at sbin / 2 of the first octave's images (the 2x octave
                   the parts use); root levels follow, at sbin, octave by octave, kept while both sides have at least
                   ``min_cells`` cells.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np

TRUNC = 0.2
NORM_EPS = 1e-4
N_ORIENT = 9


def _weights(n_in: int, n_out: int, s: float) -> np.ndarray:
    """Row-resampling matrix W [n_out][n_in]: W[j][i] = |[i, i + 1) and [j / s, (j + 1) / s)| * s, the mean over the
    output pixel's interval (intervals beyond the input are clipped and the mean taken over the covered part)."""
    Wm = np.zeros((n_out, n_in), dtype=np.float64)
    for j in range(n_out):
        a, b = j / s, (j + 1) / s
        b = min(b, float(n_in))
        for i in range(int(math.floor(a)), int(math.ceil(b))):
            ov = min(b, i + 1.0) - max(a, float(i))
            if ov > 0.0:
                Wm[j, i] = ov
        Wm[j] /= Wm[j].sum()
    return Wm


def resized_size(n: int, s: float) -> int:
    return int(math.floor(n * s + 0.5))


def resize(img: np.ndarray, s: float) -> np.ndarray:
    """Area-averaging resize of an H x W x C image by s <= 1 (FP64)."""
    H, W = img.shape[:2]
    Ho, Wo = resized_size(H, s), resized_size(W, s)
    Wy, Wx = _weights(H, Ho, s), _weights(W, Wo, s)
    rows = np.einsum("yi,ijc->yjc", Wy, img.astype(np.float64))     # along columns, then along rows
    return np.einsum("yjc,xj->yxc", rows, Wx)


def _orient_table() -> Tuple[np.ndarray, np.ndarray]:
    o = np.arange(N_ORIENT, dtype=np.float64)
    return np.cos(o * math.pi / N_ORIENT).astype(np.float32), np.sin(o * math.pi / N_ORIENT).astype(np.float32)


def gradients(img: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Per interior pixel: the orientation bin (int, 0..17) and the magnitude (FP64), arrays over the whole image
    (the border ring is 0). The channel and orientation choices are taken in FP32 (module docstring)."""
    im = np.asarray(img, dtype=np.float32)
    h, w, _ = im.shape
    dx = np.zeros((h, w, im.shape[2]), np.float32)
    dy = np.zeros_like(dx)
    dx[1:-1, 1:-1] = im[1:-1, 2:] - im[1:-1, :-2]
    dy[1:-1, 1:-1] = im[2:, 1:-1] - im[:-2, 1:-1]
    v = dx * dx + dy * dy                                  # FP32, each operation rounded
    ch = np.argmax(v, axis=2)                              # first maximum
    gx = np.take_along_axis(dx, ch[..., None], 2)[..., 0]
    gy = np.take_along_axis(dy, ch[..., None], 2)[..., 0]
    gv = np.take_along_axis(v, ch[..., None], 2)[..., 0]
    ux, uy = _orient_table()
    dots = ux[None, None, :] * gx[..., None] + uy[None, None, :] * gy[..., None]   # FP32
    best = np.zeros((h, w), np.float32)
    obin = np.zeros((h, w), np.int64)
    for o in range(N_ORIENT):                              # strictly larger replaces: the first maximum wins
        d = dots[..., o]
        pos = d > best
        best = np.where(pos, d, best)
        obin = np.where(pos, o, obin)
        neg = -d > best
        best = np.where(neg, -d, best)
        obin = np.where(neg, o + N_ORIENT, obin)
    mag = np.sqrt(gv.astype(np.float64))
    mag[0, :] = mag[-1, :] = 0.0
    mag[:, 0] = mag[:, -1] = 0.0
    return obin, mag


def cell_histograms(obin: np.ndarray, mag: np.ndarray, sbin: int) -> np.ndarray:
    """Bilinear votes of the visible pixels into [cy][cx][18] cells (FP64; votes added in pixel order)."""
    h, w = mag.shape
    cy, cx = (2 * h + sbin) // (2 * sbin), (2 * w + sbin) // (2 * sbin)   # floor(n / sbin + 1/2)
    hist = np.zeros((cy, cx, 2 * N_ORIENT), np.float64)
    ys = np.arange(1, cy * sbin - 1)
    xs = np.arange(1, cx * sbin - 1)
    if ys.size == 0 or xs.size == 0:
        return hist
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    yy, xx = np.minimum(Y, h - 2), np.minimum(X, w - 2)
    yp, xp = (Y + 0.5) / sbin - 0.5, (X + 0.5) / sbin - 0.5
    iy, ix = np.floor(yp).astype(np.int64), np.floor(xp).astype(np.int64)
    fy, fx = yp - iy, xp - ix
    o, m = obin[yy, xx], mag[yy, xx]
    for (ty, wy) in ((iy, 1.0 - fy), (iy + 1, fy)):
        for (tx, wx) in ((ix, 1.0 - fx), (ix + 1, fx)):
            ok = (ty >= 0) & (ty < cy) & (tx >= 0) & (tx < cx)
            np.add.at(hist, (ty[ok], tx[ok], o[ok]), (wy * wx * m)[ok])
    return hist


def features_from_hist(hist: np.ndarray) -> np.ndarray:
    """[cy - 2][cx - 2][32] features from the cell histograms (FP64)."""
    cy, cx = hist.shape[:2]
    out = np.zeros((max(cy - 2, 0), max(cx - 2, 0), 32), np.float64)
    if cy < 3 or cx < 3:
        return out
    E = np.sum((hist[..., :N_ORIENT] + hist[..., N_ORIENT:]) ** 2, axis=2)
    B = E[:-1, :-1] + E[:-1, 1:] + E[1:, :-1] + E[1:, 1:]      # B[a][b]: the 2x2 block with top-left cell (a, b)
    Nb = 1.0 / np.sqrt(B + NORM_EPS)
    # the four blocks containing interior cell (Y, X) = (y + 1, x + 1): top-left corners (Y, X), (Y, X-1), (Y-1, X),
    # (Y-1, X-1)
    norms = [Nb[1:, 1:], Nb[1:, :-1], Nb[:-1, 1:], Nb[:-1, :-1]]
    hc = hist[1:-1, 1:-1]
    ins = hc[..., :N_ORIENT] + hc[..., N_ORIENT:]
    for n in norms:
        t = np.minimum(hc * n[..., None], TRUNC)
        out[..., :2 * N_ORIENT] += 0.5 * t
        out[..., 2 * N_ORIENT:3 * N_ORIENT] += 0.5 * np.minimum(ins * n[..., None], TRUNC)
    for k, n in enumerate(norms):
        out[..., 27 + k] = np.sum(np.minimum(hc * n[..., None], TRUNC), axis=2) / math.sqrt(18.0)
    return out


def hog(img: np.ndarray, sbin: int) -> np.ndarray:
    """The 32-channel features of one image at cell size sbin."""
    obin, mag = gradients(img)
    return features_from_hist(cell_histograms(obin, mag, sbin))


def pyramid_images(img: np.ndarray, lam: int, min_side: int) -> List[List[np.ndarray]]:
    """octaves[k][i]: the image at scale 2^(-k - i / lam); octave 0 by area averaging from the image, octave k + 1
    by halving octave k, while the smaller side has at least min_side pixels."""
    octaves = [[resize(img, 2.0 ** (-i / lam)) if i else np.asarray(img, np.float64) for i in range(lam)]]
    while True:
        nxt = [resize(im, 0.5) for im in octaves[-1]]
        if min(nxt[-1].shape[:2]) < min_side and min(nxt[0].shape[:2]) < min_side:
            break
        octaves.append(nxt)
        if len(octaves) > 16:
            break
    return octaves


def hog_pyramid(img: np.ndarray, sbin: int = 8, lam: int = 10, min_cells: int = 8) -> List[np.ndarray]:
    """The feature pyramid: lam levels of the 2x octave (sbin / 2 on the first octave's images), then the root levels
    (sbin) in order of decreasing scale while both sides have at least min_cells cells."""
    octaves = pyramid_images(img, lam, (min_cells + 2) * sbin // 2)
    levels = [hog(im, sbin // 2) for im in octaves[0]]
    for ims in octaves:
        for im in ims:
            f = hog(im, sbin)
            if min(f.shape[:2]) < min_cells:
                return levels
            levels.append(f)
    return levels
