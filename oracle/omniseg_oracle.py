"""FP64 CPU oracle for the Omni-Seg slide-wise inference path.

TEST INFRASTRUCTURE ONLY.  This module is imported by the tests, by the
package's smoke check and by the benchmark's CPU-baseline arm.  The product
path (the CUDA library and its Python binding) never imports or calls it, and
it shares no code with that path: the only common dependency is the ``synth``
input generator, which holds none of the method's arithmetic.

It is deliberately plain: integer steps use numpy int64 / Python integers,
floating-point steps use torch float64 on the CPU, and every step is the
textbook definition of the operation in the order the method states it.

Paper: "An Accelerated Pipeline for Multi-label Renal Pathology Image
Segmentation at the Whole Slide Image Level" (Leng, Deng et al.).
  Sec. 2.1  tissue detection and patch extraction (padding, 2x2-mean pad colour,
            Otsu foreground, median blur)
  Sec. 2.2  Omni-Seg segmentation of overlapping tiles at 40x / 10x / 5x
  Sec. 2.3  slide-wise aggregation: per-class merge, foreground filter
  Sec. 3.2  parameter values (512 tiles, stride 256 at 40x, vote thresholds)
The network is the cited Omni-Seg dynamic network; its layer structure here is
the residual U-Net + GAP -> controller -> dynamic 1x1 head stated by the
workload description.  Readings taken where the text is silent are named
"[reading]" at the function that applies them.
"""
from __future__ import annotations

from fractions import Fraction
from typing import Dict, List, Sequence, Tuple

import math

import numpy as np
import torch

from synth.configs import (HEAD_CH, N_HEAD_PARAMS, THUMB, STITCH_AVG, STITCH_VOTE, WINDOW_FLAT,
                           WINDOW_TENT, WINDOW_HANN)
from synth.weights import layout

F64 = torch.float64

# ----------------------------------------------------------------------------
# Sec. 2.1: padding
# ----------------------------------------------------------------------------


def padded_dims(work, H: int | None = None, W: int | None = None) -> Tuple[int, int, int]:
    """Padded 40x canvas size and the leading border.

    [reading] Sec. 2.1 pads the slide so edge tiles are not truncated (4096 px
    in the paper; ``pad_lead`` here, default 0).  Every scale's canvas must be
    covered exactly by its P/S_s patch grid and by 32x32 thumbnail blocks, so
    the canvas is extended right/bottom to a multiple of f_s * S_s for every
    scale s (their least common multiple) and to at least f_max * P (f_max =
    largest downsample factor).
    """
    H = work.H if H is None else H
    W = work.W if W is None else W
    lead = work.pad_lead
    fmax = max(work.factors)
    unit = 1
    for s, f in enumerate(work.factors):
        assert (f * scale_stride(work, s)) % THUMB == 0
        unit = math.lcm(unit, f * scale_stride(work, s))
    minimum = -(-(fmax * work.P) // unit) * unit

    def ext(d):
        return max(-(-(d + 2 * lead) // unit) * unit, minimum)
    return ext(H), ext(W), lead


def pad_colour(rgb: np.ndarray) -> np.ndarray:
    """Sec. 2.1: pad colour = mean of the 2x2 top-left pixels, per channel.

    [reading] integer mean rounded half up: (sum + 2) >> 2.
    """
    blk = rgb[:2, :2, :].astype(np.int64).reshape(-1, 3)
    return (blk.sum(axis=0) + 2) >> 2


def pad_slide(rgb: np.ndarray, work) -> np.ndarray:
    H, W, _ = rgb.shape
    Hp, Wp, lead = padded_dims(work, H, W)
    canvas = np.empty((Hp, Wp, 3), np.uint8)
    canvas[...] = pad_colour(rgb).astype(np.uint8)
    canvas[lead:lead + H, lead:lead + W] = rgb
    return canvas


# ----------------------------------------------------------------------------
# Sec. 2.2: 40x / 10x / 5x pyramid
# ----------------------------------------------------------------------------


def half(img: np.ndarray) -> np.ndarray:
    """One 2x2 box-average step: (a + b + c + d + 2) >> 2 (round half up)."""
    a = img.astype(np.int64)
    s = a[0::2, 0::2] + a[0::2, 1::2] + a[1::2, 0::2] + a[1::2, 1::2]
    return ((s + 2) >> 2).astype(np.uint8)


def pyramid(canvas: np.ndarray, factors: Sequence[int]) -> List[np.ndarray]:
    """Image per scale index; factor f is reached by log2(f) iterated halvings."""
    out = []
    for f in factors:
        img = canvas
        g = f
        while g > 1:
            img = half(img)
            g //= 2
        out.append(img)
    return out


# ----------------------------------------------------------------------------
# Sec. 2.1: tissue detection (Otsu foreground after a median blur)
# ----------------------------------------------------------------------------


def thumbnail(canvas: np.ndarray) -> np.ndarray:
    """32x32 box mean of the 40x canvas, rounded half up: (sum + 512) >> 10."""
    Hp, Wp, _ = canvas.shape
    a = canvas.astype(np.int64).reshape(Hp // THUMB, THUMB, Wp // THUMB, THUMB, 3)
    return ((a.sum(axis=(1, 3)) + (THUMB * THUMB // 2)) >> 10).astype(np.uint8)


def grey(rgb: np.ndarray) -> np.ndarray:
    """Integer luma: (77 R + 150 G + 29 B + 128) >> 8."""
    a = rgb.astype(np.int64)
    return ((77 * a[..., 0] + 150 * a[..., 1] + 29 * a[..., 2] + 128) >> 8).astype(np.uint8)


def median_blur(img: np.ndarray, k: int) -> np.ndarray:
    """k x k median with replicated borders (k odd).

    Definition used: the median of the k*k window values is the smallest level
    v such that at least (k*k + 1) / 2 of them are <= v.  Counts come from a
    summed-area table of the indicator (img <= v), for every v in 0..255.
    """
    assert k % 2 == 1 and k >= 1
    r = k // 2
    h, w = img.shape
    pad = np.pad(img.astype(np.int64), r, mode="edge")
    need = (k * k + 1) // 2
    med = np.full((h, w), -1, np.int64)
    for v in range(256):
        ind = (pad <= v).astype(np.int64)
        sat = np.zeros((h + 2 * r + 1, w + 2 * r + 1), np.int64)
        sat[1:, 1:] = ind.cumsum(0).cumsum(1)
        cnt = sat[k:k + h, k:k + w] - sat[0:h, k:k + w] - sat[k:k + h, 0:w] + sat[0:h, 0:w]
        med = np.where((med < 0) & (cnt >= need), v, med)
    return med.astype(np.uint8)


def histogram(img: np.ndarray) -> np.ndarray:
    return np.bincount(img.ravel().astype(np.int64), minlength=256).astype(np.int64)


def otsu(hist: Sequence[int]) -> int:
    """Otsu's threshold on a 256-bin histogram (class 0 = levels <= t).

    Maximises the between-class variance w0 w1 (mu0 - mu1)^2, which for
    class-0 count W(t) and level sum S(t) equals
    (N S(t) - W(t) S_T)^2 / (N^2 W(t) (N - W(t))).  Compared exactly with
    rational arithmetic.  [reading] ties go to the smallest t; t with
    W = 0 or W = N is not a split.  Returns -1 when no split exists.
    """
    h = [int(x) for x in hist]
    N = sum(h)
    ST = sum(i * h[i] for i in range(256))
    best_t, best = -1, None
    W = S = 0
    for t in range(256):
        W += h[t]
        S += t * h[t]
        if W == 0 or W == N:
            continue
        score = Fraction((N * S - W * ST) ** 2, W * (N - W))
        if best is None or score > best:
            best, best_t = score, t
    return best_t


def tissue_mask(canvas: np.ndarray, k: int):
    """Thumbnail tissue mask: tissue = blurred grey <= Otsu threshold.

    Tissue is darker than the near-white glass, so the class below the
    threshold is the foreground.  Returns (mask bool, threshold, blurred grey,
    histogram).
    """
    g = grey(thumbnail(canvas))
    b = median_blur(g, k)
    hst = histogram(b)
    t = otsu(hst)
    return b.astype(np.int64) <= t, t, b, hst


def area_filter(mask: np.ndarray, min_area: int) -> np.ndarray:
    """[reading] Sec. 2.1's contour step on the tissue mask: a tissue region is
    a set of mask pixels connected through their 8 neighbours (a region's
    outer contour encloses exactly such a set once its holes are counted as
    part of it; only the region's own pixels are kept, holes stay background),
    and regions with fewer than ``min_area`` pixels are removed.  The paper
    names no area; 0 keeps every region (the mask unchanged).

    Written as the definition: a breadth-first flood fill from every unvisited
    tissue pixel collects one region, whose size decides whether it stays."""
    if min_area <= 0:
        return mask.copy()
    h, w = mask.shape
    seen = np.zeros((h, w), dtype=bool)
    out = np.zeros((h, w), dtype=bool)
    ys, xs = np.nonzero(mask)
    for y0, x0 in zip(ys.tolist(), xs.tolist()):
        if seen[y0, x0]:
            continue
        seen[y0, x0] = True
        region = [(y0, x0)]
        k = 0
        while k < len(region):
            y, x = region[k]
            k += 1
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    yy, xx = y + dy, x + dx
                    if 0 <= yy < h and 0 <= xx < w and mask[yy, xx] and not seen[yy, xx]:
                        seen[yy, xx] = True
                        region.append((yy, xx))
        if len(region) >= min_area:
            for (y, x) in region:
                out[y, x] = True
    return out


# ----------------------------------------------------------------------------
# Sec. 2.2: overlapping tile grid and foreground selection
# ----------------------------------------------------------------------------


def scale_stride(work, s: int) -> int:
    """Tile stride of scale s in its own pixels.  Sec. 3.2 strides the 40x
    scale by 256 and the 10x and 5x scales by 64 (8 overlapping tiles per
    axis there, 2 at 40x); an empty or zero per-scale entry means the common
    stride S."""
    st = tuple(getattr(work, "strides", ()) or ())
    return st[s] if st and st[s] else work.S


def grid(work, Hp: int, Wp: int, s: int) -> Tuple[int, int]:
    f = work.factors[s]
    hs, ws = Hp // f, Wp // f
    S = scale_stride(work, s)
    return (hs - work.P) // S + 1, (ws - work.P) // S + 1


def tile_list(work, mask: np.ndarray, Hp: int, Wp: int):
    """Foreground tiles in (scale, row, col) order.

    A tile at scale s with origin (y, x) covers 40x rows y*f .. (y+P)*f - 1,
    i.e. thumbnail rows y*f/32 .. (y+P)*f/32 - 1; it is foreground when any
    tissue thumbnail pixel lies there (or always, with the filter off).
    Returns (list of (s, y, x), list of per-scale bool flag grids).
    """
    tiles, flags = [], []
    for s, f in enumerate(work.factors):
        ny, nx = grid(work, Hp, Wp, s)
        fl = np.zeros((ny, nx), bool)
        for i in range(ny):
            for j in range(nx):
                y, x = i * scale_stride(work, s), j * scale_stride(work, s)
                if work.tissue_filter:
                    r0, r1 = y * f // THUMB, (y + work.P) * f // THUMB
                    c0, c1 = x * f // THUMB, (x + work.P) * f // THUMB
                    fg = bool(mask[r0:r1, c0:c1].any())
                else:
                    fg = True
                fl[i, j] = fg
                if fg:
                    tiles.append((s, y, x))
        flags.append(fl)
    return tiles, flags


# ----------------------------------------------------------------------------
# Sec. 2.2: Omni-Seg network (residual U-Net, GAP -> controller -> dynamic head)
# ----------------------------------------------------------------------------


def weights_f64(work, blob: np.ndarray) -> Dict[str, torch.Tensor]:
    out, off = {}, 0
    for name, shape in layout(work).items():
        n = int(np.prod(shape))
        out[name] = torch.from_numpy(blob[off:off + n].astype(np.float64)).reshape(shape)
        off += n
    assert off == blob.size
    return out


def normalise(u8: np.ndarray) -> torch.Tensor:
    """[reading] v = 2 u / 255 - 1, HWC uint8 -> (B,) C H W float64."""
    t = torch.from_numpy(np.ascontiguousarray(u8)).to(F64)
    t = t.movedim(-1, -3)
    return 2.0 * t / 255.0 - 1.0


def conv3x3(x: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    """y[o,i,j] = sum_{c,dy,dx} w[o,c,dy,dx] x[c, i+dy-1, j+dx-1], zero outside.

    x: (B, C, H, W); w: (O, C, 3, 3).  Written as the sum over the nine taps of
    (O x C) @ (C x H W) products of the shifted input.
    """
    B, C, H, W = x.shape
    xp = torch.zeros((B, C, H + 2, W + 2), dtype=F64)
    xp[:, :, 1:H + 1, 1:W + 1] = x
    y = torch.zeros((B, w.shape[0], H * W), dtype=F64)
    for dy in range(3):
        for dx in range(3):
            xs = xp[:, :, dy:dy + H, dx:dx + W].reshape(B, C, H * W)
            y = y + torch.matmul(w[:, :, dy, dx], xs)
    return y.reshape(B, w.shape[0], H, W)


def conv1x1(x: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    B, C, H, W = x.shape
    return torch.matmul(w, x.reshape(B, C, H * W)).reshape(B, w.shape[0], H, W)


def affine(z: torch.Tensor, g: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """[reading] inference-mode norm: per-channel g * z + b (folded batch norm)."""
    return z * g[None, :, None, None] + b[None, :, None, None]


def relu(z: torch.Tensor) -> torch.Tensor:
    """max(z, 0); [reading] its derivative at exactly 0 is taken as 0."""
    return torch.relu(z)


def res_block(x: torch.Tensor, p: Dict[str, torch.Tensor], pre: str) -> torch.Tensor:
    """out = ReLU(N2(conv(ReLU(N1(conv(x))))) + proj(x)); proj = 1x1 conv."""
    a = relu(affine(conv3x3(x, p[pre + ".w1"]), p[pre + ".g1"], p[pre + ".b1"]))
    z = affine(conv3x3(a, p[pre + ".w2"]), p[pre + ".g2"], p[pre + ".b2"])
    return relu(z + conv1x1(x, p[pre + ".wp"]))


def maxpool2(x: torch.Tensor) -> torch.Tensor:
    return torch.maximum(torch.maximum(x[:, :, 0::2, 0::2], x[:, :, 0::2, 1::2]),
                         torch.maximum(x[:, :, 1::2, 0::2], x[:, :, 1::2, 1::2]))


def _interp_axis(x: torch.Tensor, dim: int) -> torch.Tensor:
    """x2 linear resampling along one axis, half-pixel centres, edge clamp.

    Output index i samples source coordinate (i + 0.5) / 2 - 0.5.
    """
    R = x.shape[dim]
    out = []
    for i in range(2 * R):
        src = (i + 0.5) / 2.0 - 0.5
        i0 = int(np.floor(src))
        fr = src - i0
        a = x.select(dim, min(max(i0, 0), R - 1))
        b = x.select(dim, min(max(i0 + 1, 0), R - 1))
        out.append((1.0 - fr) * a + fr * b)
    return torch.stack(out, dim=dim)


def upsample2(x: torch.Tensor) -> torch.Tensor:
    """Bilinear x2 (align_corners = False), separable along H then W."""
    return _interp_axis(_interp_axis(x, 2), 3)


def unet(v: torch.Tensor, p: Dict[str, torch.Tensor], levels: int):
    """Encoder (maxpool between levels) and decoder (upsample, concat [up, skip]).

    Returns (y0, bottleneck, cats) where cats[l] is the decoder input of level l.
    """
    skips = []
    x = v
    for l in range(levels):
        y = res_block(x, p, f"enc{l}")
        skips.append(y)
        if l < levels - 1:
            x = maxpool2(y)
    bott = skips[-1]
    y = bott
    cats = {}
    for l in range(levels - 2, -1, -1):
        cat = torch.cat([upsample2(y), skips[l]], dim=1)   # [reading] up first, then skip
        cats[l] = cat
        y = res_block(cat, p, f"dec{l}")
    return y, bott, cats


def prehead(y0: torch.Tensor, p) -> torch.Tensor:
    """[reading] h0 = ReLU(1x1 conv base -> 8): the head input has 8 channels."""
    return relu(conv1x1(y0, p["head.w"]) + p["head.b"][None, :, None, None])


def controller(g: torch.Tensor, cls: int, scl: int, p, n_classes: int, n_scales: int):
    """theta = Wc [g; onehot(class); onehot(scale)] + bc  (153 values per patch)."""
    B = g.shape[0]
    z = torch.zeros((B, g.shape[1] + n_classes + n_scales), dtype=F64)
    z[:, :g.shape[1]] = g
    z[:, g.shape[1] + cls] = 1.0
    z[:, g.shape[1] + n_classes + scl] = 1.0
    return torch.matmul(z, p["ctrl.w"].T) + p["ctrl.b"][None, :]


def split_theta(theta: torch.Tensor):
    """[reading] 153 = W1(8x8, out x in) W2(8x8) W3(1x8) b1(8) b2(8) b3(1)."""
    W1 = theta[:, 0:64].reshape(-1, 8, 8)
    W2 = theta[:, 64:128].reshape(-1, 8, 8)
    W3 = theta[:, 128:136].reshape(-1, 1, 8)
    b1 = theta[:, 136:144]
    b2 = theta[:, 144:152]
    b3 = theta[:, 152:153]
    return W1, W2, W3, b1, b2, b3


def dynamic_head(h0: torch.Tensor, theta: torch.Tensor) -> torch.Tensor:
    """logit = W3 ReLU(W2 ReLU(W1 h0 + b1) + b2) + b3 at every pixel."""
    B, C, H, W = h0.shape
    W1, W2, W3, b1, b2, b3 = split_theta(theta)
    x = h0.reshape(B, C, H * W)
    h1 = relu(torch.matmul(W1, x) + b1[:, :, None])
    h2 = relu(torch.matmul(W2, h1) + b2[:, :, None])
    out = torch.matmul(W3, h2) + b3[:, :, None]
    return out.reshape(B, H, W)


def patch_forward(patches_u8: np.ndarray, p, work, scl: int):
    """Logits of every class at scale ``scl`` for a batch of HWC uint8 patches.

    Returns (logits (n_cls_at_scale, B, P, P) float64, class ids).
    """
    v = normalise(patches_u8)
    y0, bott, _ = unet(v, p, work.levels)
    g = bott.mean(dim=(2, 3))                         # GAP of the bottleneck
    h0 = prehead(y0, p)
    classes = [c for c, s in enumerate(work.class_scale) if s == scl]
    outs = [dynamic_head(h0, controller(g, c, scl, p, work.n_classes, work.n_scales))
            for c in classes]
    return torch.stack(outs, 0), classes


# ----------------------------------------------------------------------------
# Sec. 2.3 / 3.2: slide-wise aggregation
# ----------------------------------------------------------------------------


def window_weights(P: int, window: int) -> np.ndarray:
    """[reading] Weight of a tile's logit at tile pixel (u, v) in the overlap
    average: w = t(u) t(v) with t = 1 (flat, the plain mean of Sec. 2.3),
    t(u) = min(u + 1, P - u) (tent) or t(u) = sin^2(pi (u + 1/2) / P) (Hann).
    The paper names no window; every choice is positive at every pixel."""
    u = np.arange(P, dtype=np.float64)
    if window == WINDOW_FLAT:
        t = np.ones(P)
    elif window == WINDOW_TENT:
        t = np.minimum(u + 1.0, P - u)
    elif window == WINDOW_HANN:
        t = np.sin(np.pi * (u + 0.5) / P) ** 2
    else:
        raise ValueError(window)
    return t[:, None] * t[None, :]


def stitch(patch_logits: Dict[Tuple[int, int], np.ndarray], hs: int, ws: int, P: int,
           window: int = 0):
    """Overlap average of the processed tiles covering each pixel.

    L(x) = sum_p w_p(x) l_p(x) / sum_p w_p(x) (w = 1: the mean over cov(x)
    tiles); votes(x) = #{p : l_p(x) > 0}; pixels with no covering tile keep
    L = 0, cov = 0.  Sum in float64 in ascending tile order.
    """
    acc = np.zeros((hs, ws), np.float64)
    wsum = np.zeros((hs, ws), np.float64)
    cov = np.zeros((hs, ws), np.int64)
    votes = np.zeros((hs, ws), np.int64)
    w = window_weights(P, window)
    for (y, x) in sorted(patch_logits):
        lp = patch_logits[(y, x)]
        acc[y:y + P, x:x + P] += w * lp
        wsum[y:y + P, x:x + P] += w
        cov[y:y + P, x:x + P] += 1
        votes[y:y + P, x:x + P] += (lp > 0)
    L = np.where(cov > 0, acc / np.where(cov > 0, wsum, 1.0), 0.0)
    return L, cov, votes


def vote_margin(patch_logits: Dict[Tuple[int, int], np.ndarray], hs: int, ws: int, P: int) -> np.ndarray:
    """Smallest |l_p(x)| over the processed tiles p covering x (inf where no
    tile covers x): a vote can change only if some covering tile's logit is
    within the arithmetic error of zero."""
    m = np.full((hs, ws), np.inf)
    for (y, x), lp in patch_logits.items():
        m[y:y + P, x:x + P] = np.minimum(m[y:y + P, x:x + P], np.abs(lp))
    return m


def tissue_at_scale(mask: np.ndarray, f: int, hs: int, ws: int) -> np.ndarray:
    """Thumbnail mask sampled at scale-f pixel (y, x) -> thumb (y f / 32, x f / 32)."""
    ys = (np.arange(hs) * f) // THUMB
    xs = (np.arange(ws) * f) // THUMB
    return mask[ys[:, None], xs[None, :]]


def labels(L, cov, votes, mode: int, tissue=None) -> np.ndarray:
    """Label emission.

    average mode: cov > 0 and L > 0 (strictly).
    vote mode ([reading] of the Sec. 3.2 vote thresholds as "at least half of
    the covering tiles"): cov > 0 and 2 votes >= cov.
    Sec. 2.3: optionally AND with the tissue foreground.
    """
    if mode == STITCH_AVG:
        lab = (cov > 0) & (L > 0)
    else:
        lab = (cov > 0) & (2 * votes >= cov)
    if tissue is not None:
        lab = lab & tissue
    return lab.astype(np.uint8)


def argmax_map(Ls: Sequence[np.ndarray], class_ids: Sequence[int]) -> np.ndarray:
    """0 = background (every logit <= 0), else 1 + class id of the largest
    logit; ties go to the lower class id."""
    stack = np.stack(Ls, 0)
    best = np.argmax(stack, axis=0)               # first maximum on ties
    mx = np.max(stack, axis=0)
    ids = np.asarray(class_ids)[best] + 1
    return np.where(mx > 0, ids, 0).astype(np.uint8)


def stain(rgb: np.ndarray, maps: Sequence, factors: Sequence[int], colours, alphas) -> np.ndarray:
    """Sec. 2.3: the merged label map of every tissue type is stained onto the
    40x slide in its own colour.

    [reading] Map k (at its scale, ceil(H/f_k) x ceil(W/f_k)) covers 40x pixel
    (y, x) through pixel (y // f_k, x // f_k).  Stains are applied in map
    order; where map k is on, each channel becomes the alpha blend
    (c (256 - a_k) + colour_k a_k + 128) >> 8 with a_k in 0..256.
    """
    H, W, _ = rgb.shape
    out = rgb.astype(np.int64).copy()
    for m, f, col, a in zip(maps, factors, colours, alphas):
        if m is None:
            continue
        on = np.repeat(np.repeat(np.asarray(m) != 0, f, axis=0), f, axis=1)[:H, :W]
        c = np.asarray(col, np.int64)
        out[on] = (out[on] * (256 - a) + c * a + 128) >> 8
    return out.astype(np.uint8)


def resize_down(img: np.ndarray, r: int) -> np.ndarray:
    """Sec. 2.3: the 10x product is resized directly from the stained 40x
    image.  [reading] Resizing by r is the r x r box mean rounded half up,
    (sum + n // 2) // n over the n image pixels of the block (edge blocks of a
    ragged image have fewer)."""
    H, W, _ = img.shape
    oh, ow = -(-H // r), -(-W // r)
    out = np.zeros((oh, ow, 3), np.uint8)
    for i in range(oh):
        for j in range(ow):
            blk = img[i * r:(i + 1) * r, j * r:(j + 1) * r].reshape(-1, 3).astype(np.int64)
            n = blk.shape[0]
            out[i, j] = (blk.sum(axis=0) + n // 2) // n
    return out


# ----------------------------------------------------------------------------
# Whole path
# ----------------------------------------------------------------------------


def prepare(rgb: np.ndarray, work):
    """Stages of Sec. 2.1: pad, pyramid, tissue mask, tile list."""
    canvas = pad_slide(rgb, work)
    Hp, Wp, lead = padded_dims(work, rgb.shape[0], rgb.shape[1])
    pyr = pyramid(canvas, work.factors)
    mask, t, blurred, hst = tissue_mask(canvas, work.median_k)
    mask = area_filter(mask, getattr(work, "min_tissue_area", 0))
    tiles, flags = tile_list(work, mask, Hp, Wp)
    return dict(canvas=canvas, Hp=Hp, Wp=Wp, lead=lead, pyr=pyr, mask=mask, otsu=t,
                blurred=blurred, hist=hst, tiles=tiles, flags=flags)


def segment(rgb: np.ndarray, work, blob: np.ndarray, window=None, batch: int = 4,
            prep=None):
    """Full path: per-class stitched logits, coverage and labels at each scale.

    ``window`` = (y0, x0, h, w) in 40x padded-canvas pixels restricts the work
    to the tiles that overlap it (each scale gets the window divided by its
    factor); outputs then cover only that window.
    """
    if prep is None:
        prep = prepare(rgb, work)
    p = weights_f64(work, blob)
    Hp, Wp, P = prep["Hp"], prep["Wp"], work.P
    out = {"prep": prep, "L": {}, "cov": {}, "votes": {}, "labels": {}, "window": {}, "margin": {}}
    for s, f in enumerate(work.factors):
        hs, ws = Hp // f, Wp // f
        if window is None:
            wy0, wx0, wh, ww = 0, 0, hs, ws
        else:
            wy0, wx0, wh, ww = (window[0] // f, window[1] // f,
                                max(1, window[2] // f), max(1, window[3] // f))
        mine = [(y, x) for (ss, y, x) in prep["tiles"] if ss == s
                and y < wy0 + wh and y + P > wy0 and x < wx0 + ww and x + P > wx0]
        classes = [c for c, cs in enumerate(work.class_scale) if cs == s]
        per_class = {c: {} for c in classes}
        img = prep["pyr"][s]
        for k in range(0, len(mine), batch):
            chunk = mine[k:k + batch]
            pats = np.stack([img[y:y + P, x:x + P] for (y, x) in chunk], 0)
            lg, cls = patch_forward(pats, p, work, s)
            for ci, c in enumerate(cls):
                for bi, (y, x) in enumerate(chunk):
                    per_class[c][(y, x)] = lg[ci, bi].numpy()
        tis = tissue_at_scale(prep["mask"], f, hs, ws) if work.tissue_and else None
        for c in classes:
            L, cov, votes = stitch(per_class[c], hs, ws, P, getattr(work, "stitch_window", 0))
            sl = (slice(wy0, wy0 + wh), slice(wx0, wx0 + ww))
            out["L"][c] = L[sl]
            out["cov"][c] = cov[sl]
            out["votes"][c] = votes[sl]
            out["margin"][c] = vote_margin(per_class[c], hs, ws, P)[sl]
            out["labels"][c] = labels(L[sl], cov[sl], votes[sl], work.stitch_mode,
                                      None if tis is None else tis[sl])
        out["window"][s] = (wy0, wx0, wh, ww)
    return out


def segment_window_regions(get40, mask: np.ndarray, work, blob: np.ndarray, window,
                           Hp: int, Wp: int, batch: int = 2, scales=None):
    """The whole path restricted to a window, for slides too large to hold.

    ``get40(y0, x0, h, w)`` returns 40x padded-canvas pixels; ``mask`` is the
    slide's thumbnail tissue mask (computed by ``tissue_mask`` on the full
    slide).  Each covering tile's pixels at scale f come from its 40x footprint
    by iterated 2x2 means, which equals the same crop of the full pyramid
    because every output pixel depends only on its own f x f block.
    """
    p = weights_f64(work, blob)
    tiles, _ = tile_list(work, mask, Hp, Wp)
    P = work.P
    out = {"L": {}, "cov": {}, "labels": {}, "window": {}}
    for s, f in enumerate(work.factors):
        if scales is not None and s not in scales:
            continue
        hs, ws = Hp // f, Wp // f
        wy0, wx0, wh, ww = window[0] // f, window[1] // f, max(1, window[2] // f), max(1, window[3] // f)
        mine = [(y, x) for (ss, y, x) in tiles if ss == s
                and y < wy0 + wh and y + P > wy0 and x < wx0 + ww and x + P > wx0]
        classes = [c for c, cs in enumerate(work.class_scale) if cs == s]
        per_class = {c: {} for c in classes}
        for k in range(0, len(mine), batch):
            chunk = mine[k:k + batch]
            pats = []
            for (y, x) in chunk:
                img = get40(y * f, x * f, P * f, P * f)
                g = f
                while g > 1:
                    img = half(img)
                    g //= 2
                pats.append(img)
            lg, cls = patch_forward(np.stack(pats, 0), p, work, s)
            for ci, c in enumerate(cls):
                for bi, (y, x) in enumerate(chunk):
                    per_class[c][(y, x)] = lg[ci, bi].numpy()
        # stitch only the window: shift tile origins into window coordinates
        tis = tissue_at_scale(mask, f, hs, ws)[wy0:wy0 + wh, wx0:wx0 + ww] if work.tissue_and else None
        wt = window_weights(P, getattr(work, "stitch_window", 0))
        for c in classes:
            acc = np.zeros((wh, ww), np.float64)
            wsum = np.zeros((wh, ww), np.float64)
            cov = np.zeros((wh, ww), np.int64)
            votes = np.zeros((wh, ww), np.int64)
            for (y, x) in sorted(per_class[c]):
                lp = per_class[c][(y, x)]
                ya, yb = max(y, wy0), min(y + P, wy0 + wh)
                xa, xb = max(x, wx0), min(x + P, wx0 + ww)
                sub = lp[ya - y:yb - y, xa - x:xb - x]
                wsub = wt[ya - y:yb - y, xa - x:xb - x]
                acc[ya - wy0:yb - wy0, xa - wx0:xb - wx0] += wsub * sub
                wsum[ya - wy0:yb - wy0, xa - wx0:xb - wx0] += wsub
                cov[ya - wy0:yb - wy0, xa - wx0:xb - wx0] += 1
                votes[ya - wy0:yb - wy0, xa - wx0:xb - wx0] += (sub > 0)
            L = np.where(cov > 0, acc / np.where(cov > 0, wsum, 1.0), 0.0)
            out["L"][c] = L
            out["cov"][c] = cov
            out["labels"][c] = labels(L, cov, votes, work.stitch_mode, tis)
        out["window"][s] = (wy0, wx0, wh, ww)
    return out


# ----------------------------------------------------------------------------
# Differentiation: stitched soft-Dice + BCE and its gradient
# ----------------------------------------------------------------------------

GRAD_PARAMS = ("ctrl.w", "ctrl.b", "head.w", "head.b", "dec0.w1", "dec0.g1", "dec0.b1",
               "dec0.w2", "dec0.g2", "dec0.b2", "dec0.wp")


def dice_bce(L: torch.Tensor, g: torch.Tensor) -> torch.Tensor:
    """[reading] soft-Dice (smooth 1) + mean BCE on the stitched logits of one class.

    dice = 1 - (2 sum(sig(L) g) + 1) / (sum sig(L) + sum g + 1)
    bce  = mean(max(L, 0) - g L + log(1 + exp(-|L|)))
    """
    sg = torch.sigmoid(L)
    dice = 1.0 - (2.0 * (sg * g).sum() + 1.0) / (sg.sum() + g.sum() + 1.0)
    bce = (torch.clamp(L, min=0.0) - g * L + torch.log1p(torch.exp(-L.abs()))).mean()
    return dice + bce


class DiffProblem:
    """Forward of the differentiated sub-chain on cached constants.

    The gradient stops at the GAP feature and at the decoder-level-0 input
    (both are computed once from the frozen encoder/decoder and held fixed), so
    the loss is a function of the controller, the pre-head and the last
    decoder block only.
    """

    def __init__(self, rgb, work, blob, gts, batch: int = 4):
        self.work = work
        self.prep = prepare(rgb, work)
        self.p = weights_f64(work, blob)
        self.gts = [torch.from_numpy(g.astype(np.float64)) for g in gts]
        Hp, Wp, P = self.prep["Hp"], self.prep["Wp"], work.P
        self.cache = []     # (scale, [(y, x)], cat0 (B,3C,P,P), g (B, Cb))
        for s, f in enumerate(work.factors):
            mine = [(y, x) for (ss, y, x) in self.prep["tiles"] if ss == s]
            img = self.prep["pyr"][s]
            for k in range(0, len(mine), batch):
                chunk = mine[k:k + batch]
                pats = np.stack([img[y:y + P, x:x + P] for (y, x) in chunk], 0)
                with torch.no_grad():
                    _, bott, cats = unet(normalise(pats), self.p, work.levels)
                self.cache.append((s, chunk, cats[0], bott.mean(dim=(2, 3))))

    def loss(self, q: Dict[str, torch.Tensor]) -> torch.Tensor:
        """Loss as a function of the parameters in ``q`` (others from the blob)."""
        work = self.work
        p = dict(self.p)
        p.update(q)
        Hp, Wp, P = self.prep["Hp"], self.prep["Wp"], work.P
        acc = {}
        cov = {}
        for c, s in enumerate(work.class_scale):
            f = work.factors[s]
            acc[c] = torch.zeros((Hp // f, Wp // f), dtype=F64)
            cov[c] = torch.zeros((Hp // f, Wp // f), dtype=F64)
        for (s, chunk, cat0, g) in self.cache:
            y0 = res_block(cat0, p, "dec0")
            h0 = prehead(y0, p)
            for c in [c for c, cs in enumerate(work.class_scale) if cs == s]:
                lg = dynamic_head(h0, controller(g, c, s, p, work.n_classes, work.n_scales))
                for bi, (y, x) in enumerate(chunk):
                    acc[c][y:y + P, x:x + P] += lg[bi]
                    cov[c][y:y + P, x:x + P] += 1.0
        total = torch.zeros((), dtype=F64)
        for c in range(work.n_classes):
            L = torch.where(cov[c] > 0, acc[c] / torch.clamp(cov[c], min=1.0),
                            torch.zeros_like(acc[c]))
            H, W = self.gts[c].shape
            total = total + dice_bce(L[:H, :W], self.gts[c])
        return total / work.n_classes

    def loss_heads_only(self, q: Dict[str, torch.Tensor]) -> torch.Tensor:
        """loss(q) for q holding only controller / pre-head parameters: the last
        decoder block's output does not depend on them, so it is computed once
        (with the blob's values) and reused; the value equals loss(q)."""
        assert all(k.startswith("ctrl.") or k.startswith("head.") for k in q)
        if not hasattr(self, "_y0"):
            with torch.no_grad():
                self._y0 = [res_block(cat0, self.p, "dec0") for (_, _, cat0, _) in self.cache]
        return self.loss_from_y0(q, self._y0)

    def loss_from_y0(self, q: Dict[str, torch.Tensor], y0s) -> torch.Tensor:
        """loss with the last decoder block's output of every cached batch given
        (y0s[k] for self.cache[k]) and the controller / pre-head parameters in q
        (others from the blob)."""
        assert all(k.startswith("ctrl.") or k.startswith("head.") for k in q)
        work = self.work
        p = dict(self.p)
        p.update(q)
        Hp, Wp, P = self.prep["Hp"], self.prep["Wp"], work.P
        acc, cov = {}, {}
        for c, s in enumerate(work.class_scale):
            f = work.factors[s]
            acc[c] = torch.zeros((Hp // f, Wp // f), dtype=F64)
            cov[c] = torch.zeros((Hp // f, Wp // f), dtype=F64)
        for (s, chunk, _, g), y0 in zip(self.cache, y0s):
            h0 = prehead(y0, p)
            for c in [c for c, cs in enumerate(work.class_scale) if cs == s]:
                lg = dynamic_head(h0, controller(g, c, s, p, work.n_classes, work.n_scales))
                for bi, (y, x) in enumerate(chunk):
                    acc[c][y:y + P, x:x + P] += lg[bi]
                    cov[c][y:y + P, x:x + P] += 1.0
        total = torch.zeros((), dtype=F64)
        for c in range(work.n_classes):
            L = torch.where(cov[c] > 0, acc[c] / torch.clamp(cov[c], min=1.0), torch.zeros_like(acc[c]))
            H, W = self.gts[c].shape
            total = total + dice_bce(L[:H, :W], self.gts[c])
        return total / work.n_classes

    def params(self) -> Dict[str, torch.Tensor]:
        return {k: self.p[k].clone() for k in GRAD_PARAMS}

    def loss_and_grads_by_batch(self):
        """The same loss and gradient as loss_and_grads, one batch of tiles in
        memory at a time: the chain rule through the overlap average written
        out.  Pass 1 (no autograd) stitches every class's logits and takes
        G = dloss/dL; pass 2 recomputes each batch's tile logits l_p with
        autograd and back-propagates sum_p sum_x G(x) l_p(x) / cov(x), which
        has the batch's share of the gradient."""
        work = self.work
        q = {k: v.clone().requires_grad_(True) for k, v in self.params().items()}
        Hp, Wp, P = self.prep["Hp"], self.prep["Wp"], work.P
        acc, cov = {}, {}
        for c, s in enumerate(work.class_scale):
            f = work.factors[s]
            acc[c] = torch.zeros((Hp // f, Wp // f), dtype=F64)
            cov[c] = torch.zeros((Hp // f, Wp // f), dtype=F64)

        def batch_logits(p, s, cat0, g):
            h0 = prehead(res_block(cat0, p, "dec0"), p)
            return {c: dynamic_head(h0, controller(g, c, s, p, work.n_classes, work.n_scales))
                    for c in [c for c, cs in enumerate(work.class_scale) if cs == s]}

        p = dict(self.p)
        p.update({k: v.detach() for k, v in q.items()})
        with torch.no_grad():
            for (s, chunk, cat0, g) in self.cache:
                for c, lg in batch_logits(p, s, cat0, g).items():
                    for bi, (y, x) in enumerate(chunk):
                        acc[c][y:y + P, x:x + P] += lg[bi]
                        cov[c][y:y + P, x:x + P] += 1.0
        Ls = {c: torch.where(cov[c] > 0, acc[c] / torch.clamp(cov[c], min=1.0),
                             torch.zeros_like(acc[c])).requires_grad_(True) for c in acc}
        total = torch.zeros((), dtype=F64)
        for c in range(work.n_classes):
            H, W = self.gts[c].shape
            total = total + dice_bce(Ls[c][:H, :W], self.gts[c])
        total = total / work.n_classes
        total.backward()
        G = {c: torch.where(cov[c] > 0, Ls[c].grad / torch.clamp(cov[c], min=1.0), torch.zeros_like(cov[c]))
             for c in Ls}
        p = dict(self.p)
        p.update(q)
        for (s, chunk, cat0, g) in self.cache:
            part = torch.zeros((), dtype=F64)
            for c, lg in batch_logits(p, s, cat0, g).items():
                for bi, (y, x) in enumerate(chunk):
                    part = part + (G[c][y:y + P, x:x + P] * lg[bi]).sum()
            part.backward()
        return float(total.detach()), {k: v.grad.detach().clone() for k, v in q.items()}

    def loss_and_grads(self):
        q = {k: v.clone().requires_grad_(True) for k, v in self.params().items()}
        L = self.loss(q)
        L.backward()
        return float(L.detach()), {k: v.grad.detach().clone() for k, v in q.items()}
