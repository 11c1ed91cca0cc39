"""Seeded synthetic slides shaped like renal needle biopsies.

The generator is counter based: every pixel value is a pure function of
(seed, y, x, channel), so any window of a slide can be produced on the CPU
without generating the rest, and the CUDA library's ``omni_synth_slide``
reproduces it byte for byte.  Randomness comes from SplitMix64 (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014; output
mixer constants as published by Vigna in splitmix64.c): value k of the stream
seeded with ``seed`` is mix(seed + (k + 1) * GAMMA).

Pixel recipe (all integer):
  * background 235 (near-white glass),
  * tissue = union of rotated ellipses (elongated cores along the long axis for
    needle biopsies, free blobs otherwise), coloured by a pink -> purple blend
    on the normalised radial depth inside the deepest covering ellipse,
  * needle-biopsy cores also hold sharp-edged structures, as kidney tissue
    holds glomeruli, tubule lumina and vessels: the slide is divided into
    512 x 512 cells; draw k = (cell row << 20 | cell column) of SplitMix64
    seeded with seed ^ STRUCT_SALT decides whether the cell holds a disc
    (low byte < 160), its type (next byte mod 3: dark purple, pale, red), its
    radius r = 64 + (7 bits) and its centre, offset from the cell centre by
    (b * 2 m) // 255 - m per axis (b the next bytes, m = 254 - r) so the disc
    stays inside its cell; tissue pixels inside the disc take the type's
    colour instead of the depth blend,
  * per-channel noise: Irwin-Hall sum of four 16-bit uniforms from one
    SplitMix64 draw, scaled to sigma ~= 5.8 and rounded to an integer,
  * clamp to [0, 255].
Ellipse parameters are drawn on the host with numpy's PCG64 and handed to both
generators as integers.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
MIX1 = np.uint64(0xBF58476D1CE4E5B9)
MIX2 = np.uint64(0x94D049BB133111EB)

BACKGROUND = 235
PINK = (232, 150, 200)
PURPLE = (150, 90, 170)
Q14 = 1 << 14
STRUCT_SALT = 0x5A17C0DE5EED
STRUCT_CELL_SHIFT = 9                      # 512 x 512 cells at 40x
STRUCT_COLOURS = ((120, 50, 140), (245, 205, 230), (195, 65, 95))


@dataclass(frozen=True)
class Ellipse:
    cy: int
    cx: int
    a: int        # semi-axis along the rotated u direction, pixels
    b: int        # semi-axis along the rotated v direction, pixels
    cos_q14: int
    sin_q14: int


@dataclass(frozen=True)
class SlideSpec:
    H: int
    W: int
    seed: int
    ellipses: tuple
    structures: bool = False     # sharp-edged discs inside the tissue (needle cores)

    def as_int_array(self) -> np.ndarray:
        """Ellipses packed as int64 rows (cy, cx, a, b, cos_q14, sin_q14)."""
        if not self.ellipses:
            return np.zeros((0, 6), np.int64)
        return np.array([[e.cy, e.cx, e.a, e.b, e.cos_q14, e.sin_q14] for e in self.ellipses],
                        np.int64)


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """Output number ``idx`` (0-based, uint64 array) of SplitMix64 seeded with ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx.astype(np.uint64) + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * MIX1
        z = (z ^ (z >> np.uint64(27))) * MIX2
        return z ^ (z >> np.uint64(31))


def _ellipse(rng, cy, cx, a, b, theta) -> Ellipse:
    return Ellipse(int(cy), int(cx), max(1, int(a)), max(1, int(b)),
                   int(round(math.cos(theta) * Q14)), int(round(math.sin(theta) * Q14)))


def make_spec(H: int, W: int, seed: int, tissue: float, layout: str, n_blobs: int) -> SlideSpec:
    """Draw ellipse geometry so the expected tissue area is ``tissue`` * H * W."""
    rng = np.random.default_rng(seed)
    ells: List[Ellipse] = []
    area = tissue * H * W
    if layout == "cores":
        # long thin cores along the long axis, stacked across the short axis
        long_is_x = W >= H
        L, Sh = (W, H) if long_is_x else (H, W)
        n = n_blobs
        for k in range(n):
            a = rng.uniform(0.38, 0.46) * L
            b = area / (n * math.pi * a)
            c_short = (k + 0.5) / n * Sh + rng.uniform(-0.05, 0.05) * Sh / n
            c_long = L / 2 + rng.uniform(-0.04, 0.04) * L
            theta = rng.uniform(-0.03, 0.03)
            if long_is_x:
                ells.append(_ellipse(rng, c_short, c_long, a, b, theta))
            else:
                ells.append(_ellipse(rng, c_long, c_short, a, b, theta + math.pi / 2))
    else:
        n = n_blobs
        for _ in range(n):
            a = math.sqrt(area / (n * math.pi)) * rng.uniform(0.8, 1.6)
            b = area / (n * math.pi * a)
            ells.append(_ellipse(rng, rng.uniform(0.1, 0.9) * H, rng.uniform(0.1, 0.9) * W,
                                 a, b, rng.uniform(0, math.pi)))
    return SlideSpec(H, W, seed, tuple(ells), structures=(layout == "cores"))


def _structures(spec: SlideSpec, ys: np.ndarray, xs: np.ndarray):
    """Type (0..2) of the structure disc covering each pixel, -1 where none."""
    sh = STRUCT_CELL_SHIFT
    cy0, cy1 = int(ys.min()) >> sh, int(ys.max()) >> sh
    cx0, cx1 = int(xs.min()) >> sh, int(xs.max()) >> sh
    cyy = np.arange(cy0, cy1 + 1, dtype=np.int64)[:, None]
    cxx = np.arange(cx0, cx1 + 1, dtype=np.int64)[None, :]
    k = ((cyy << 20) | cxx).astype(np.uint64)
    h = splitmix64(spec.seed ^ STRUCT_SALT, k)
    byte = lambda q: ((h >> np.uint64(8 * q)) & np.uint64(0xFF)).astype(np.int64)  # noqa: E731
    present = byte(0) < 160
    stype = byte(1) % 3
    r = 64 + (((h >> np.uint64(16)) & np.uint64(0x7F)).astype(np.int64))
    m = 254 - r
    half = 1 << (sh - 1)
    ccy = (cyy << sh) + half + (byte(3) * 2 * m) // 255 - m
    ccx = (cxx << sh) + half + (byte(4) * 2 * m) // 255 - m
    iy = (ys >> sh) - cy0
    ix = (xs >> sh) - cx0
    dy = ys - ccy[iy, ix]
    dx = xs - ccx[iy, ix]
    inside = present[iy, ix] & (dy * dy + dx * dx < r[iy, ix] * r[iy, ix])
    return np.where(inside, stype[iy, ix], -1)


def _depth_q8(spec: SlideSpec, ys: np.ndarray, xs: np.ndarray) -> np.ndarray:
    """Deepest normalised radial depth (0..255) over all ellipses, -1 outside tissue."""
    depth = np.full(np.broadcast(ys, xs).shape, -1, np.int64)
    for e in spec.ellipses:
        dy = ys - e.cy
        dx = xs - e.cx
        u = np.abs(dx * e.cos_q14 + dy * e.sin_q14)          # Q14
        v = np.abs(-dx * e.sin_q14 + dy * e.cos_q14)         # Q14
        uq = np.minimum((u << 2) // e.a, 1 << 20)            # Q16 ratio |u|/a
        vq = np.minimum((v << 2) // e.b, 1 << 20)
        r = uq * uq + vq * vq                                # Q32
        inside = r < (1 << 32)
        t8 = ((1 << 32) - r) >> 24
        depth = np.where(inside & (t8 > depth), t8, depth)
    return depth


def gen_window(spec: SlideSpec, y0: int, x0: int, h: int, w: int) -> np.ndarray:
    """Slide pixels [y0:y0+h, x0:x0+w] as uint8 (h, w, 3)."""
    ys = np.arange(y0, y0 + h, dtype=np.int64)[:, None]
    xs = np.arange(x0, x0 + w, dtype=np.int64)[None, :]
    depth = _depth_q8(spec, ys, xs)
    yy, xx = np.broadcast_arrays(ys, xs)
    st = _structures(spec, yy, xx) if spec.structures else np.full(depth.shape, -1, np.int64)
    out = np.empty((h, w, 3), np.uint8)
    base_idx = (ys * spec.W + xs) * 3
    for c in range(3):
        hsh = splitmix64(spec.seed, (base_idx + c).astype(np.uint64))
        s = np.zeros(hsh.shape, np.int64)
        for k in range(4):
            s += ((hsh >> np.uint64(16 * k)) & np.uint64(0xFFFF)).astype(np.int64)
        noise = ((s * 10 - 1310700 + 32768 + (32 << 16)) >> 16) - 32
        t = np.maximum(depth, 0)
        col = (PINK[c] * (256 - t) + PURPLE[c] * t + 128) >> 8
        scol = np.array([sc[c] for sc in STRUCT_COLOURS], np.int64)[np.maximum(st, 0)]
        col = np.where(st >= 0, scol, col)
        val = np.where(depth >= 0, col, BACKGROUND) + noise
        out[..., c] = np.clip(val, 0, 255).astype(np.uint8)
    return out


def gen_slide(spec: SlideSpec) -> np.ndarray:
    return gen_window(spec, 0, 0, spec.H, spec.W)


def spec_for(work) -> SlideSpec:
    return make_spec(work.H, work.W, work.seed, work.tissue, work.layout, work.n_blobs)


def gen_gt_masks(H: int, W: int, factors, class_scale, seed: int, n_per_class: int = 5):
    """Seeded binary ground-truth masks, one per class at its scale's resolution."""
    masks = []
    for c, s in enumerate(class_scale):
        f = factors[s]
        h, w = -(-H // f), -(-W // f)
        sp = make_spec(h, w, seed * 1000 + c, 0.25, "blobs", n_per_class)
        ys = np.arange(h, dtype=np.int64)[:, None]
        xs = np.arange(w, dtype=np.int64)[None, :]
        masks.append((_depth_q8(sp, ys, xs) >= 0).astype(np.uint8))
    return masks
