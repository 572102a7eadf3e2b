"""Seeded synthetic inputs for the DPM scoring path.

This module makes HOG-shaped feature pyramids and DPM-shaped model banks from a seed. It holds none of the
scoring arithmetic (no correlation, no distance transform, no assembly): the CUDA path's tests and benchmarks and the
FP64 oracle both consume its arrays, so neither side can bias the other through shared code.

The datasets and trained DPM release-5 models the paper evaluates on (Sec. 5) are not available; these generators
stand in for them with the same shapes and value ranges:

* features: 32 channels per cell, i.i.d. U[0, 0.2) (0.2 is the HOG truncation value);
* pyramid: DPM-style, ``lam`` levels per octave; the first ``lam`` levels form the 2x octave (cell size sbin/2) that
  part filters are evaluated on, the remaining levels are at cell size ``sbin`` and hold root positions;
* filters: h x w x 32; "iid" draws N(0, 0.05) entries, "dpm" draws a filter with a smooth, geometrically decaying CP
  spectrum (trained DPM filters are close to low rank: Sec. 5 finds ranks 6-11 within a small percentage of rank 21,
  which almost matches the full filters);
* deformation coefficients (d1, d2, d3, d4) of (dx, dx^2, dy, dy^2), each U[0.001, 0.1];
* part anchors in part-level cells relative to twice the root position, drawn so every anchored part filter lies
  inside the root's 2x footprint.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

FEAT_DIM = 32
HOG_TRUNC = 0.2
LAMBDA = 10
SBIN = 8
FILTER_STD = 0.05
DEFORM_RANGE = (0.001, 0.1)


# --------------------------------------------------------------------------------------------------------------------
# data containers (plain arrays; no behaviour)
# --------------------------------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Part:
    filt: np.ndarray            # float32 [h][w][32]
    anchor: Tuple[int, int]     # (vy, vx) in part-level cells
    deform: np.ndarray          # float32 [4] = coefficients of (dx, dx^2, dy, dy^2)


@dataclasses.dataclass
class Component:
    root: np.ndarray            # float32 [h][w][32]
    parts: List[Part]
    bias: float = 0.0


@dataclasses.dataclass
class Model:
    components: List[Component]

    def filters(self) -> List[np.ndarray]:
        """All filters in model order: component 0 root, its parts, component 1 root, ..."""
        out = []
        for c in self.components:
            out.append(c.root)
            out.extend(p.filt for p in c.parts)
        return out


@dataclasses.dataclass
class Pyramid:
    levels: List[np.ndarray]    # float32 [H][W][32] each
    lam: int                    # part level of root level j is j - lam

    @property
    def sizes(self) -> List[Tuple[int, int]]:
        return [(int(l.shape[0]), int(l.shape[1])) for l in self.levels]


# --------------------------------------------------------------------------------------------------------------------
# pyramid shapes and contents
# --------------------------------------------------------------------------------------------------------------------
def pyramid_sizes(img_h: int, img_w: int, sbin: int = SBIN, lam: int = LAMBDA,
                  min_cells: int = 8) -> List[Tuple[int, int]]:
    """Cell grid sizes (H, W) of a DPM-style pyramid for an img_h x img_w image.

    Levels 0..lam-1 are the 2x octave: scale s_m = 2^(-m/lam), cell size sbin/2. Levels lam.. are at cell size sbin with
    scale s_m, m = 0, 1, ..., kept while both sides have at least ``min_cells`` cells. Scales one octave apart are made
    by exact halving so a part level is always at least twice its root level in both dimensions.
    """
    base = [math.pow(2.0, -m / lam) for m in range(lam)]

    def scale(m: int) -> float:
        return base[m % lam] / float(1 << (m // lam))

    octave = [(int(math.floor(img_h * scale(m) * 2 / sbin)), int(math.floor(img_w * scale(m) * 2 / sbin)))
              for m in range(lam)]
    root = []
    m = 0
    while True:
        H = int(math.floor(img_h * scale(m) / sbin))
        W = int(math.floor(img_w * scale(m) / sbin))
        if min(H, W) < min_cells:
            break
        root.append((H, W))
        m += 1
    return octave + root


def make_pyramid(rng: np.random.Generator, sizes: Sequence[Tuple[int, int]], lam: int) -> Pyramid:
    levels = [rng.uniform(0.0, HOG_TRUNC, size=(H, W, FEAT_DIM)).astype(np.float32) for (H, W) in sizes]
    return Pyramid(levels=levels, lam=lam)


# --------------------------------------------------------------------------------------------------------------------
# filters and models
# --------------------------------------------------------------------------------------------------------------------
def make_filter(rng: np.random.Generator, h: int, w: int, kind: str = "iid", n_terms: int = 36,
                decay: float = 0.7) -> np.ndarray:
    """One h x w x 32 filter with entry RMS FILTER_STD.

    kind "iid": i.i.d. N(0, FILTER_STD). kind "dpm": a smooth CP spectrum, the sum of ``n_terms`` outer products of
    random unit vectors with weights decay^r, rescaled to RMS FILTER_STD (a rank-R truncation leaves roughly decay^R
    of the filter's norm).
    """
    if kind == "iid":
        return rng.normal(0.0, FILTER_STD, size=(h, w, FEAT_DIM)).astype(np.float32)
    if kind != "dpm":
        raise ValueError(kind)
    F = np.zeros((h, w, FEAT_DIM))
    for r in range(n_terms):
        a = rng.standard_normal(h); a /= np.linalg.norm(a)
        b = rng.standard_normal(w); b /= np.linalg.norm(b)
        c = rng.standard_normal(FEAT_DIM); c /= np.linalg.norm(c)
        F += (decay ** r) * a[:, None, None] * b[None, :, None] * c[None, None, :]
    F *= FILTER_STD / np.sqrt(np.mean(F * F))
    return F.astype(np.float32)


def channel_involution(seed: int = 12345) -> np.ndarray:
    """A fixed permutation pi of the 32 channels with pi(pi(c)) = c (stand-in for HOG's mirrored orientations)."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(FEAT_DIM)
    pi = np.arange(FEAT_DIM)
    for i in range(0, FEAT_DIM - 1, 2):
        a, b = perm[i], perm[i + 1]
        pi[a], pi[b] = b, a
    return pi


def mirror_filter(F: np.ndarray) -> np.ndarray:
    """Flip along x and permute channels by the fixed involution."""
    return np.ascontiguousarray(F[:, ::-1, :][:, :, channel_involution()])


def make_component(rng: np.random.Generator, root_hw: Tuple[int, int], part_hw: Sequence[Tuple[int, int]],
                   kind: str = "iid", bias: float = 0.0, **filter_kw) -> Component:
    h0, w0 = root_hw
    root = make_filter(rng, h0, w0, kind, **filter_kw)
    parts = []
    for (hp, wp) in part_hw:
        f = make_filter(rng, hp, wp, kind, **filter_kw)
        vy = int(rng.integers(0, max(0, 2 * h0 - hp) + 1))
        vx = int(rng.integers(0, max(0, 2 * w0 - wp) + 1))
        d = rng.uniform(*DEFORM_RANGE, size=4).astype(np.float32)
        parts.append(Part(filt=f, anchor=(vy, vx), deform=d))
    return Component(root=root, parts=parts, bias=float(bias))


def mirror_component(c: Component) -> Component:
    """Mirror image of a component: filters mirrored, x anchors reflected in the 2x footprint, linear x cost negated."""
    h0, w0 = c.root.shape[:2]
    parts = []
    for p in c.parts:
        hp, wp = p.filt.shape[:2]
        d = p.deform.copy()
        d[0] = -d[0]
        parts.append(Part(filt=mirror_filter(p.filt), anchor=(p.anchor[0], 2 * w0 - wp - p.anchor[1]), deform=d))
    return Component(root=mirror_filter(c.root), parts=parts, bias=c.bias)


DPM_ROOT_SHAPES = ((5, 11), (7, 7), (11, 5))
DPM_PART_SHAPE = (6, 6)
DPM_N_PARTS = 8


def make_dpm_class(rng: np.random.Generator, kind: str = "dpm", **filter_kw) -> List[Component]:
    """A DPM release-5-shaped class model: 3 components (roots 5x11, 7x7, 11x5) and their mirrors, 8 parts of 6x6."""
    comps = []
    for hw in DPM_ROOT_SHAPES:
        c = make_component(rng, hw, [DPM_PART_SHAPE] * DPM_N_PARTS, kind, **filter_kw)
        comps.append(c)
        comps.append(mirror_component(c))
    return comps


# --------------------------------------------------------------------------------------------------------------------
# images (input of the feature extraction block)
# --------------------------------------------------------------------------------------------------------------------
def make_image(rng: np.random.Generator, h: int, w: int) -> np.ndarray:
    """An 8-bit RGB image [h][w][3]: smooth oriented structure (edges in every direction) plus pixel noise."""
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    ph = rng.uniform(0, 2 * np.pi, size=4)
    base = 120 + 60 * np.sin(x / 7.0 + 0.3 * y / 5.0 + ph[0]) + 40 * np.cos(y / 9.0 - x / 13.0 + ph[1])
    img = np.stack([base, base * 0.8 + 20, 255 - base], axis=2) + rng.normal(0, 12, size=(h, w, 3))
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


# --------------------------------------------------------------------------------------------------------------------
# planted object instances (positive examples for the thresholds of Sec. 4)
# --------------------------------------------------------------------------------------------------------------------
def plant_objects(rng: np.random.Generator, pyramid: Pyramid, model: Model,
                  placements: Sequence[Tuple[int, int, int, int]], strength: float = 1.0,
                  noise: float = 0.02) -> Pyramid:
    """A copy of ``pyramid`` with an object instance at each placement (component, root level j, y, x): the root
    window at (y, x) on level j and every part window at its anchor (2y + vy, 2x + vx) on level j - lam are set to
    0.1 + 0.1 * strength * f / max|f| plus N(0, noise) per entry, clipped to [0, 0.2] (features that line up with
    the filter f). Windows are written root first, then the parts in model order, so where part windows overlap the
    later part's pattern wins. Placements must be valid root positions (the root and every anchored part inside their
    levels)."""
    levels = [l.copy() for l in pyramid.levels]
    for (c, j, y, x) in placements:
        comp = model.components[c]
        wins = [(j, y, x, comp.root)] + [(j - pyramid.lam, 2 * y + p.anchor[0], 2 * x + p.anchor[1], p.filt)
                                         for p in comp.parts]
        for (lv, y0, x0, f) in wins:
            h, w = f.shape[:2]
            L = levels[lv]
            assert 0 <= y0 and 0 <= x0 and y0 + h <= L.shape[0] and x0 + w <= L.shape[1], "placement out of range"
            pat = 0.1 + 0.1 * strength * f / np.max(np.abs(f)) + rng.normal(0.0, noise, size=f.shape)
            L[y0:y0 + h, x0:x0 + w, :] = np.clip(pat, 0.0, HOG_TRUNC).astype(np.float32)
    return Pyramid(levels=levels, lam=pyramid.lam)


# --------------------------------------------------------------------------------------------------------------------
# strict-suite inputs: values exactly representable in FP32 so that every rounding order gives the same bits
# --------------------------------------------------------------------------------------------------------------------
def make_integer_map(rng: np.random.Generator, H: int, W: int, lo: int = -64, hi: int = 64) -> np.ndarray:
    return rng.integers(lo, hi + 1, size=(H, W)).astype(np.float32)


def make_pow2_deform(rng: np.random.Generator) -> np.ndarray:
    """(d1, d2, d3, d4): linear terms +-2^-k, quadratic terms 2^-k, k in 0..4."""
    k = rng.integers(0, 5, size=4)
    d = (2.0 ** (-k)).astype(np.float32)
    sign = rng.choice([-1.0, 1.0], size=2).astype(np.float32)
    d[0] *= sign[0]
    d[2] *= sign[1]
    return d


# --------------------------------------------------------------------------------------------------------------------
# workload configurations
# --------------------------------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    model: Model
    pyramids: List[Pyramid]
    description: str


def config_c1(seed: int = 0) -> Workload:
    """Single root level of 30x40 cells with its 60x80 part level; 1 root 6x11 + 8 parts 6x6, i.i.d. N(0, 0.05)."""
    rng = np.random.default_rng(seed)
    pyr = make_pyramid(rng, [(60, 80), (30, 40)], lam=1)
    comp = make_component(rng, (6, 11), [(6, 6)] * 8, kind="iid")
    return Workload("c1_single_level_30x40", Model([comp]), [pyr],
                    "1 root level 30x40x32 + part level 60x80x32 U[0,0.2); root 6x11, 8 parts 6x6 N(0,0.05)")


def config_c2(seed: int = 1, kind: str = "dpm") -> Workload:
    """One 500x375 image (36 levels), a 6-component DPM-shaped class model with 48 parts."""
    rng = np.random.default_rng(seed)
    model = Model(make_dpm_class(rng, kind))
    pyr = make_pyramid(rng, pyramid_sizes(375, 500), lam=LAMBDA)
    return Workload("c2_dpm_class_500x375", model, [pyr],
                    "500x375 image, sbin 8, 10 levels/octave (36 levels); 6 components (roots 5x11/7x7/11x5 + "
                    "mirrors), 48 parts 6x6")


def config_c3(seed: int = 2, n_classes: int = 20, img_hw: Tuple[int, int] = (720, 1280), kind: str = "dpm") -> Workload:
    """A bank of ``n_classes`` DPM-shaped class models (1080 filters for 20 classes) on one 1280x720 image."""
    rng = np.random.default_rng(seed)
    comps = []
    for _ in range(n_classes):
        comps.extend(make_dpm_class(rng, kind))
    pyr = make_pyramid(rng, pyramid_sizes(*img_hw), lam=LAMBDA)
    return Workload(f"c3_bank{n_classes}_{img_hw[1]}x{img_hw[0]}", Model(comps), [pyr],
                    f"{n_classes}-class bank ({len(comps)} components), {img_hw[1]}x{img_hw[0]} image")


def config_c4(seed: int = 3, n_images: int = 64, n_classes: int = 20, kind: str = "dpm") -> Workload:
    """A batch of images with W ~ U{320..1280}, H ~ U{240..720}, scored by a 20-class bank."""
    rng = np.random.default_rng(seed)
    comps = []
    for _ in range(n_classes):
        comps.extend(make_dpm_class(rng, kind))
    pyrs = []
    for _ in range(n_images):
        W = int(rng.integers(320, 1281))
        H = int(rng.integers(240, 721))
        pyrs.append(make_pyramid(rng, pyramid_sizes(H, W), lam=LAMBDA))
    return Workload(f"c4_batch{n_images}_bank{n_classes}", Model(comps), pyrs,
                    f"{n_images} images W~U{{320..1280}} H~U{{240..720}}, {n_classes}-class bank")


def serving_requests(seed: int = 4, n: int = 200, rate_hz: float = 200.0,
                     sizes: Sequence[Tuple[int, int]] = ((480, 640), (720, 1280), (1080, 1920)),
                     max_classes: int = 20) -> List[dict]:
    """Poisson arrivals: each request has an arrival time, an image size and a distinct subset of class ids."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate_hz))
        hw = sizes[int(rng.integers(0, len(sizes)))]
        k = int(rng.integers(1, max_classes + 1))
        classes = sorted(int(c) for c in rng.choice(max_classes, size=k, replace=False))
        out.append({"id": i, "t_arrival": t, "img_hw": hw, "classes": classes, "seed": int(rng.integers(0, 2**31))})
    return out
