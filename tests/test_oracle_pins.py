"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against brute force on tiny inputs, a closed form,
an invariant, a library routine computing the same textbook operation by a
different formulation, or a value the paper prints (tests/golden/).
"""
import json
import math
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import synth
from oracle import omniseg_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_params.json")
F64 = torch.float64


def rng(seed=0):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- padding, pyramid


def test_pad_colour_is_rounded_2x2_mean():
    img = np.zeros((4, 4, 3), np.uint8)
    img[0, 0] = (10, 0, 255)
    img[0, 1] = (11, 1, 255)
    img[1, 0] = (12, 2, 254)
    img[1, 1] = (13, 2, 254)
    # sums 46, 5, 1018 -> means 11.5, 1.25, 254.5 -> round half up 12, 1, 255
    assert O.pad_colour(img).tolist() == [12, 1, 255]


def test_padded_dims_cover_every_scale_grid():
    for w in (synth.TINY, synth.NEEDLE, synth.DIFF, synth.LARGE, synth.NEEDLE_PAPER,
              synth.NEEDLE_PAPER.with_(H=5000, W=9000)):
        Hp, Wp, lead = O.padded_dims(w)
        strides = w.strides or (w.S,) * w.n_scales
        for f, S in zip(w.factors, strides):
            for d in (Hp, Wp):
                assert d % f == 0 and (d // f - w.P) % S == 0 and d // f >= w.P
        assert Hp % synth.THUMB == 0 and Wp % synth.THUMB == 0
    # needle / large need no padding (their sizes already sit on the grid)
    assert O.padded_dims(synth.NEEDLE)[:2] == (16384, 49152)
    assert O.padded_dims(synth.LARGE)[:2] == (32768, 98304)
    # a ragged size is extended, and the paper's 4096 border adds to both sides
    w = synth.NEEDLE.with_(H=5000, W=9000)
    assert O.padded_dims(w)[:2] == (6144, 10240)
    w2 = w.with_(pad_lead=4096)
    Hp, Wp, lead = O.padded_dims(w2)
    assert lead == 4096 and Hp >= 5000 + 8192 and Wp >= 9000 + 8192
    # per-scale strides 256 / 64 / 64 (Sec. 3.2): units 256, 4 * 64, 8 * 64 -> 512,
    # at least 8 * 512 = 4096: 5000 -> 5120, 9000 -> 9216
    assert O.padded_dims(synth.NEEDLE_PAPER.with_(H=5000, W=9000))[:2] == (5120, 9216)


def test_pad_slide_places_image_and_colour():
    w = synth.NEEDLE.with_(H=300, W=700, pad_lead=64, S=64, P=128)
    img = rng().integers(0, 256, (300, 700, 3)).astype(np.uint8)
    c = O.pad_slide(img, w)
    assert np.array_equal(c[64:364, 64:764], img)
    col = O.pad_colour(img)
    assert (c[:64] == col).all() and (c[364:] == col).all() and (c[:, 764:] == col).all()


def test_half_brute_force_and_constant():
    img = rng(1).integers(0, 256, (6, 8, 3)).astype(np.uint8)
    h = O.half(img)
    for i in range(3):
        for j in range(4):
            for c in range(3):
                s = sum(int(img[2 * i + a, 2 * j + b, c]) for a in (0, 1) for b in (0, 1))
                assert h[i, j, c] == (s + 2) // 4
    const = np.full((64, 64, 3), 201, np.uint8)
    for p in O.pyramid(const, (1, 2, 4, 8)):
        assert (p == 201).all()
    assert [p.shape[0] for p in O.pyramid(const, (1, 4, 8))] == [64, 16, 8]


# ---------------------------------------------------------------- tissue detection


def test_thumbnail_and_grey_closed_forms():
    canvas = rng(2).integers(0, 256, (64, 96, 3)).astype(np.uint8)
    t = O.thumbnail(canvas)
    assert t.shape == (2, 3, 3)
    blk = canvas[32:64, 64:96, 1].astype(np.int64).sum()
    assert t[1, 2, 1] == (blk + 512) // 1024
    assert O.grey(np.array([[[255, 255, 255]]], np.uint8))[0, 0] == 255
    assert O.grey(np.array([[[0, 0, 0]]], np.uint8))[0, 0] == 0
    assert O.grey(np.array([[[100, 50, 200]]], np.uint8))[0, 0] == (7700 + 7500 + 5800 + 128) >> 8


@pytest.mark.parametrize("k", [1, 3, 5, 7])
def test_median_blur_brute_force_and_scipy(k):
    scipy_nd = pytest.importorskip("scipy.ndimage")
    img = rng(k).integers(0, 256, (9, 11)).astype(np.uint8)
    m = O.median_blur(img, k)
    r = k // 2
    pad = np.pad(img, r, mode="edge")
    for i in range(9):
        for j in range(11):
            assert m[i, j] == int(np.median(pad[i:i + k, j:j + k]))
    assert np.array_equal(m, scipy_nd.median_filter(img, size=k, mode="nearest"))


def _otsu_float(hist):
    """Textbook Otsu: maximise w0 w1 (mu0 - mu1)^2 over t, first max wins."""
    h = np.asarray(hist, np.float64)
    N = h.sum()
    lev = np.arange(256)
    best, bt = -1.0, -1
    for t in range(256):
        w0 = h[:t + 1].sum() / N
        w1 = 1.0 - w0
        if h[:t + 1].sum() == 0 or h[:t + 1].sum() == N:
            continue
        mu0 = (lev[:t + 1] * h[:t + 1]).sum() / h[:t + 1].sum()
        mu1 = (lev[t + 1:] * h[t + 1:]).sum() / h[t + 1:].sum()
        v = w0 * w1 * (mu0 - mu1) ** 2
        if v > best * (1 + 1e-12):
            best, bt = v, t
    return bt


def test_otsu_two_levels_and_textbook():
    h = np.zeros(256, np.int64)
    h[60] = 700
    h[230] = 300
    t = O.otsu(h)
    assert 60 <= t < 230
    assert t == 60            # every t in [60, 229] gives the same split; smallest wins
    for s in range(20):
        hh = rng(100 + s).integers(0, 50, 256)
        hh[rng(200 + s).integers(0, 256, 100)] = 0
        assert O.otsu(hh) == _otsu_float(hh)
    assert O.otsu(np.eye(256, dtype=np.int64)[17] * 1000) == -1     # one level: no split


def test_tissue_mask_finds_dark_blobs():
    img = np.full((256, 256, 3), 235, np.uint8)
    img[64:192, 32:128] = (150, 90, 170)
    mask, t, _, _ = O.tissue_mask(img, 3)
    assert mask.shape == (8, 8)
    # a 3x3 median removes the block's corners (4 of 9 window pixels) only
    assert mask[3:5, 1:4].all() and mask[2:6, 2].all() and not mask[:, 5:].any()
    assert not mask[2, 1] and not mask[5, 3]


# ---------------------------------------------------------------- tiling


def test_tile_counts_closed_form():
    for w, expect in ((synth.TINY, [49]), (synth.NEEDLE, [63 * 191, 15 * 47, 7 * 23]),
                      (synth.DIFF, [225, 9, 1]), (synth.LARGE, [63 * 191, 15 * 47, 7 * 23])):
        Hp, Wp, _ = O.padded_dims(w)
        got = [int(np.prod(O.grid(w, Hp, Wp, s))) for s in range(w.n_scales)]
        assert got == expect, (w.name, got)
    assert sum([63 * 191, 15 * 47, 7 * 23]) == 12899
    # Sec. 3.2 strides: the 10x canvas 4096 x 12288 holds (4096 - 512) / 64 + 1 = 57
    # by (12288 - 512) / 64 + 1 = 185 tiles, the 5x canvas 2048 x 6144 25 by 89
    w = synth.NEEDLE_PAPER
    Hp, Wp, _ = O.padded_dims(w)
    assert (Hp, Wp) == (16384, 49152)
    assert [O.grid(w, Hp, Wp, s) for s in range(3)] == [(63, 191), (57, 185), (25, 89)]


def test_per_scale_strides_tile_positions_and_overlap():
    """Tile origins step by each scale's own stride; an interior pixel is
    covered by (P / S_s)^2 tiles: 4 at 40x, 64 at 10x and 5x (Sec. 3.2 counts
    2 and 8 per axis).  Equal per-scale strides reproduce the common-stride
    tiling exactly."""
    w = synth.NEEDLE_PAPER.with_(H=8192, W=8192, tissue_filter=False)
    Hp, Wp, _ = O.padded_dims(w)
    mask = np.ones((Hp // 32, Wp // 32), bool)
    tiles, flags = O.tile_list(w, mask, Hp, Wp)
    for s, (f, S) in enumerate(zip(w.factors, (256, 64, 64))):
        ts = [(y, x) for (q, y, x) in tiles if q == s]
        ys, xs = sorted({y for y, _ in ts}), sorted({x for _, x in ts})
        assert ys == list(range(0, Hp // f - w.P + 1, S))
        assert xs == list(range(0, Wp // f - w.P + 1, S))
        cy, cx = Hp // f // 2 + 3, Wp // f // 2 + 5
        n = sum(1 for y, x in ts if y <= cy < y + w.P and x <= cx < x + w.P)
        assert n == (w.P // S) ** 2
    assert [len([t for t in tiles if t[0] == s]) for s in range(3)] == [
        (Hp // 256 - 1) * (Wp // 256 - 1),
        ((Hp // 4 - 512) // 64 + 1) * ((Wp // 4 - 512) // 64 + 1),
        ((Hp // 8 - 512) // 64 + 1) * ((Wp // 8 - 512) // 64 + 1)]
    same = synth.NEEDLE.with_(H=8192, W=8192)
    m2 = rng(5).random((Hp // 32, Wp // 32)) < 0.01
    a = O.tile_list(same, m2, Hp, Wp)
    b = O.tile_list(same.with_(strides=(256, 256, 256)), m2, Hp, Wp)
    assert a[0] == b[0] and all(np.array_equal(x, y) for x, y in zip(a[1], b[1]))


@pytest.mark.parametrize("strides", [(256, 256, 256), (256, 64, 64)])
def test_tile_list_foreground_brute_force(strides):
    w = synth.NEEDLE.with_(H=2048, W=4096, P=512, S=256, tissue_filter=True, strides=strides)
    Hp, Wp, _ = O.padded_dims(w)
    mask = np.zeros((Hp // 32, Wp // 32), bool)
    mask[10, 70] = True          # 40x pixel rows 320..351, cols 2240..2271
    tiles, flags = O.tile_list(w, mask, Hp, Wp)
    for s, f in enumerate(w.factors):
        S = strides[s]
        ny, nx = O.grid(w, Hp, Wp, s)
        for i in range(ny):
            for j in range(nx):
                y0, x0 = i * S * f, j * S * f             # 40x footprint
                y1, x1 = y0 + w.P * f, x0 + w.P * f
                hit = y0 <= 320 < y1 and x0 <= 2240 < x1
                assert flags[s][i, j] == hit
    assert tiles == sorted(tiles)
    assert all(flags[s][y // strides[s], x // strides[s]] for (s, y, x) in tiles)


# ---------------------------------------------------------------- network pieces


def test_conv3x3_brute_force():
    x = torch.from_numpy(rng(3).standard_normal((2, 3, 5, 6)))
    w = torch.from_numpy(rng(4).standard_normal((4, 3, 3, 3)))
    y = O.conv3x3(x, w)
    for b in range(2):
        for o in range(4):
            for i in range(5):
                for j in range(6):
                    s = 0.0
                    for c in range(3):
                        for dy in range(3):
                            for dx in range(3):
                                ii, jj = i + dy - 1, j + dx - 1
                                if 0 <= ii < 5 and 0 <= jj < 6:
                                    s += float(w[o, c, dy, dx]) * float(x[b, c, ii, jj])
                    assert abs(float(y[b, o, i, j]) - s) < 1e-12


def test_conv_matches_library_conv2d():
    x = torch.from_numpy(rng(5).standard_normal((2, 16, 12, 10)))
    w = torch.from_numpy(rng(6).standard_normal((8, 16, 3, 3)))
    torch.testing.assert_close(O.conv3x3(x, w), F.conv2d(x, w, padding=1), rtol=0, atol=1e-12)
    wp = torch.from_numpy(rng(7).standard_normal((8, 16)))
    torch.testing.assert_close(O.conv1x1(x, wp), F.conv2d(x, wp[:, :, None, None]),
                               rtol=0, atol=1e-12)


def test_upsample_bilinear_library_and_constant():
    x = torch.from_numpy(rng(8).standard_normal((2, 3, 4, 5)))
    ref = F.interpolate(x, scale_factor=2, mode="bilinear", align_corners=False)
    torch.testing.assert_close(O.upsample2(x), ref, rtol=0, atol=1e-14)
    c = torch.full((1, 2, 6, 6), 3.25, dtype=F64)
    assert torch.equal(O.upsample2(c), torch.full((1, 2, 12, 12), 3.25, dtype=F64))
    # interior weights 0.25 / 0.75
    v = torch.arange(4, dtype=F64).reshape(1, 1, 1, 4).expand(1, 1, 2, 4).contiguous()
    u = O.upsample2(v)[0, 0, 0]
    assert u.tolist() == [0.0, 0.25, 0.75, 1.25, 1.75, 2.25, 2.75, 3.0]


def test_maxpool_library():
    x = torch.from_numpy(rng(9).standard_normal((2, 3, 8, 6)))
    torch.testing.assert_close(O.maxpool2(x), F.max_pool2d(x, 2), rtol=0, atol=0)


def _torch_unet(v, p, levels):
    """Independent model from standard torch layers (conv2d / interpolate / max_pool2d)."""
    def block(x, pre):
        a = F.relu(F.conv2d(x, p[pre + ".w1"], padding=1) * p[pre + ".g1"].view(1, -1, 1, 1)
                   + p[pre + ".b1"].view(1, -1, 1, 1))
        z = (F.conv2d(a, p[pre + ".w2"], padding=1) * p[pre + ".g2"].view(1, -1, 1, 1)
             + p[pre + ".b2"].view(1, -1, 1, 1))
        return F.relu(z + F.conv2d(x, p[pre + ".wp"][:, :, None, None]))
    skips, x = [], v
    for l in range(levels):
        y = block(x, f"enc{l}")
        skips.append(y)
        x = F.max_pool2d(y, 2)
    y = skips[-1]
    for l in range(levels - 2, -1, -1):
        y = block(torch.cat([F.interpolate(y, scale_factor=2, mode="bilinear",
                                           align_corners=False), skips[l]], 1), f"dec{l}")
    return y, skips[-1]


def test_unet_matches_independent_torch_model():
    w = synth.TINY
    p = O.weights_f64(w, synth.gen_weights(w))
    patch = rng(10).integers(0, 256, (2, 32, 32, 3)).astype(np.uint8)
    v = O.normalise(patch)
    y0, bott, _ = O.unet(v, p, w.levels)
    r0, rb = _torch_unet(v, p, w.levels)
    torch.testing.assert_close(y0, r0, rtol=0, atol=1e-10)
    torch.testing.assert_close(bott, rb, rtol=0, atol=1e-10)
    assert float(v.min()) >= -1.0 and float(v.max()) <= 1.0
    assert torch.equal(O.normalise(np.array([[[0, 255, 51]]], np.uint8))[:, 0, 0],
                       torch.tensor([-1.0, 1.0, -0.6], dtype=F64))


def test_one_hot_controller_reproduces_explicit_head():
    """With the GAP columns of Wc zeroed, theta is the sum of the class column,
    the scale column and the bias; the dynamic head must equal three explicit
    1x1 convolutions built from those numbers."""
    w = synth.NEEDLE
    p = O.weights_f64(w, synth.gen_weights(w))
    Cb = w.widths[-1]
    p = dict(p)
    wc = p["ctrl.w"].clone()
    wc[:, :Cb] = 0.0
    p["ctrl.w"] = wc
    p["ctrl.b"] = torch.from_numpy(rng(11).standard_normal(153))
    g = torch.from_numpy(rng(12).standard_normal((3, Cb)))
    h0 = torch.from_numpy(rng(13).standard_normal((3, 8, 7, 9)))
    for cls, scl in ((0, 0), (3, 1), (5, 2)):
        theta = O.controller(g, cls, scl, p, w.n_classes, w.n_scales)
        col = wc[:, Cb + cls] + wc[:, Cb + w.n_classes + scl] + p["ctrl.b"]
        torch.testing.assert_close(theta, col[None].expand(3, -1), rtol=0, atol=0)
        W1 = col[0:64].reshape(8, 8)
        W2 = col[64:128].reshape(8, 8)
        W3 = col[128:136].reshape(1, 8)
        b1, b2, b3 = col[136:144], col[144:152], col[152:153]
        ref = F.conv2d(h0, W1[:, :, None, None], b1).relu()
        ref = F.conv2d(ref, W2[:, :, None, None], b2).relu()
        ref = F.conv2d(ref, W3[:, :, None, None], b3)[:, 0]
        torch.testing.assert_close(O.dynamic_head(h0, theta), ref, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- stitching, labels


def test_stitch_reconstructs_known_canvas_exactly():
    hs, ws, P, S = 96, 128, 32, 16
    canvas = rng(14).integers(-512, 512, (hs, ws)) / 64.0       # dyadic: sums are exact
    tiles = {(y, x): canvas[y:y + P, x:x + P].copy()
             for y in range(0, hs - P + 1, S) for x in range(0, ws - P + 1, S)}
    L, cov, votes = O.stitch(tiles, hs, ws, P)
    assert np.array_equal(L, canvas)
    # interior coverage is (P/S)^2; corners 1
    assert cov[40, 40] == 4 and cov[0, 0] == 1 and cov[0, 40] == 2
    # votes brute force
    for (yy, xx) in ((5, 5), (40, 60), (95, 127)):
        v = sum(1 for (y, x), t in tiles.items()
                if y <= yy < y + P and x <= xx < x + P and t[yy - y, xx - x] > 0)
        assert votes[yy, xx] == v


def test_stitch_constant_field_and_missing_tiles():
    tiles = {(0, 0): np.full((8, 8), 2.5), (0, 4): np.full((8, 8), 2.5)}
    L, cov, _ = O.stitch(tiles, 12, 12, 8)
    assert (L[:8, :12] == 2.5).all() and (L[8:] == 0).all() and (cov[8:] == 0).all()


@pytest.mark.parametrize("window", [synth.WINDOW_TENT, synth.WINDOW_HANN])
def test_weighted_stitch_constant_and_known_canvas(window):
    """A weighted average of equal values is that value: a constant field
    stays constant and tiles cut from a canvas re-stitch to it (exactly for
    the integer tent weights and dyadic values, to rounding for Hann)."""
    hs, ws, P, S = 96, 128, 32, 16
    canvas = rng(15).integers(-512, 512, (hs, ws)) / 64.0
    tiles = {(y, x): canvas[y:y + P, x:x + P].copy()
             for y in range(0, hs - P + 1, S) for x in range(0, ws - P + 1, S)}
    L, cov, _ = O.stitch(tiles, hs, ws, P, window)
    if window == synth.WINDOW_TENT:
        assert np.array_equal(L, canvas)
    else:
        assert np.abs(L - canvas).max() < 1e-12
    assert cov[40, 40] == 4
    const = {k: np.full((P, P), -1.75) for k in tiles}
    Lc, _, _ = O.stitch(const, hs, ws, P, window)
    assert np.abs(Lc + 1.75).max() < 1e-12


def test_weighted_stitch_hand_values():
    """P = 4, two tiles at x = 0 and x = 2 holding 3 and 6.  Tent weights per
    axis are 1, 2, 2, 1: pixel x = 2 sees weights 2 (first tile) and 1, so
    L = (2*3 + 6) / 3 = 4; pixel x = 3 sees 1 and 2, L = 5.  Hann weights
    sin^2(pi (u + 1/2) / 4) of the two tiles sum to 1 there (sin^2 + cos^2),
    so L = 3 cos^2(pi/8) + 6 sin^2(pi/8) = 3 + 1.5 (1 - sqrt(2)/2).  The flat
    window gives the plain mean 4.5."""
    tiles = {(0, 0): np.full((4, 4), 3.0), (0, 2): np.full((4, 4), 6.0)}
    Lt, cov, _ = O.stitch(tiles, 4, 6, 4, synth.WINDOW_TENT)
    assert Lt[1, 2] == 4.0 and Lt[1, 3] == 5.0 and Lt[1, 0] == 3.0 and Lt[1, 5] == 6.0
    assert cov[1].tolist() == [1, 1, 2, 2, 1, 1]
    Lh, _, _ = O.stitch(tiles, 4, 6, 4, synth.WINDOW_HANN)
    assert abs(Lh[2, 2] - (3 + 1.5 * (1 - np.sqrt(2) / 2))) < 1e-12
    assert abs(Lh[2, 3] - (6 - 1.5 * (1 - np.sqrt(2) / 2))) < 1e-12
    Lf, _, _ = O.stitch(tiles, 4, 6, 4, synth.WINDOW_FLAT)
    assert Lf[0, 2] == 4.5 and Lf[0, 3] == 4.5


def test_hann_window_is_a_partition_of_unity_at_half_overlap():
    """With S = P / 2 every interior pixel's four Hann weights sum to 1."""
    P, S = 16, 8
    w = O.window_weights(P, synth.WINDOW_HANN)
    tot = np.zeros((64, 64))
    for y in range(0, 64 - P + 1, S):
        for x in range(0, 64 - P + 1, S):
            tot[y:y + P, x:x + P] += w
    assert np.abs(tot[S:-S, S:-S] - 1.0).max() < 1e-14
    assert np.array_equal(O.window_weights(P, synth.WINDOW_FLAT), np.ones((P, P)))


def test_overlap_counts_match_paper():
    g = json.load(open(GOLDEN))
    P = g["tile_size"]["value"]
    for stride, overlaps, thr in ((g["stride_40x"]["value"], g["overlaps_40x"]["value"],
                                   g["vote_threshold_40x"]["value"]),
                                  (g["stride_10x_5x"]["value"], g["overlaps_10x_5x"]["value"],
                                   g["vote_threshold_10x_5x"]["value"])):
        n = 8 * P // stride
        tiles = {(0, x): np.ones((P, P)) for x in range(0, n * stride - P + 1, stride)}
        _, cov, _ = O.stitch(tiles, P, n * stride, P)
        assert cov[0, n * stride // 2] == overlaps          # one axis: P / S tiles
        # the vote reading "at least half" gives the paper's thresholds
        assert (overlaps + 1) // 2 == thr


def test_labels_modes_and_argmax():
    L = np.array([[0.0, 1e-9, -1.0, 2.0]])
    cov = np.array([[1, 1, 0, 3]])
    votes = np.array([[0, 1, 0, 1]])
    assert O.labels(L, cov, votes, synth.STITCH_AVG).tolist() == [[0, 1, 0, 1]]
    assert O.labels(L, cov, votes, synth.STITCH_VOTE).tolist() == [[0, 1, 0, 0]]
    tis = np.array([[True, False, True, True]])
    assert O.labels(L, cov, votes, synth.STITCH_AVG, tis).tolist() == [[0, 0, 0, 1]]
    a = O.argmax_map([np.array([[1.0, -1.0, 2.0]]), np.array([[1.0, -2.0, 3.0]])], [4, 5])
    assert a.tolist() == [[5, 0, 6]]


def test_needle_head_offsets_are_the_calibrated_ones():
    """The needle workloads' per-class head offsets are the values the oracle
    calibration (tests/golden/make_head_offsets.py) wrote, and each class's
    threshold left between 1% and 99% of the calibration tiles' tissue pixels
    positive (every class informative)."""
    g = json.load(open(os.path.join(os.path.dirname(GOLDEN), "head_offsets.json")))
    assert tuple(synth.NEEDLE.head_offsets) == tuple(g["head_offsets"])
    assert tuple(synth.LARGE.head_offsets) == tuple(g["head_offsets"])
    for c, row in g["classes"].items():
        assert 0.01 <= row["positive_fraction_in_tissue"] <= 0.99, (c, row)
        assert abs(row["offset"] + row["threshold"]) < 1e-12


def test_per_class_offsets_shift_only_their_class():
    """A class's offset enters theta[152] (the head's final bias) through that
    class's one-hot input only: with the GAP zeroed, the controller output of
    class c differs from the zero-offset network's exactly by offset_c in
    entry 152 and nowhere else."""
    w = synth.small_variant(synth.NEEDLE, H=256, W=256, P=64, S=32, base=4, levels=3,
                            head_offsets=(0.5, -1.25, 2.0, 0.0, 3.0, -0.75))
    w0 = w.with_(head_offsets=())
    p = O.weights_f64(w, synth.gen_weights(w))
    p0 = O.weights_f64(w0, synth.gen_weights(w0))
    g = torch.zeros((1, w.widths[-1]), dtype=F64)
    for c, s in enumerate(w.class_scale):
        d = O.controller(g, c, s, p, w.n_classes, w.n_scales) - O.controller(g, c, s, p0, w.n_classes, w.n_scales)
        expect = torch.zeros_like(d)
        expect[0, 152] = float(np.float32(w.head_offsets[c]) + p0["ctrl.w"][152, w.widths[-1] + c].float()) \
            - float(p0["ctrl.w"][152, w.widths[-1] + c])
        assert torch.allclose(d, expect, atol=1e-7), c


def test_vote_margin_brute_force():
    """The vote margin is, pixel by pixel, the smallest |logit| among the tiles
    whose footprint contains the pixel (counted by scanning every tile)."""
    r = rng(22)
    P, hs, ws = 4, 9, 11
    tiles = {(y, x): r.standard_normal((P, P)) for (y, x) in [(0, 0), (2, 2), (4, 6), (5, 7), (0, 6)]}
    m = O.vote_margin(tiles, hs, ws, P)
    for y in range(hs):
        for x in range(ws):
            vals = [abs(lp[y - ty, x - tx]) for (ty, tx), lp in tiles.items()
                    if ty <= y < ty + P and tx <= x < tx + P]
            assert m[y, x] == (min(vals) if vals else np.inf), (y, x)


def test_tissue_at_scale_brute_force_footprint():
    """A scale-f pixel (y, x) covers the 40x pixels [y f, (y + 1) f) x [x f, (x + 1) f);
    for f dividing the 32-pixel thumbnail cell the whole footprint lies in one
    cell, found here by scanning the cells, and the pixel takes that cell's
    mask value.  The mask has distinct neighbouring cells so an off-by-one in
    either axis changes the result."""
    r = rng(21)
    mask = r.random((7, 9)) < 0.5
    mask[0, 0], mask[0, 1], mask[1, 0] = True, False, False
    for f in (1, 2, 4, 8):
        hs, ws = 7 * 32 // f, 9 * 32 // f
        got = O.tissue_at_scale(mask, f, hs, ws)
        assert got.shape == (hs, ws)
        for y in range(hs):
            cy = [cy for cy in range(7) if all(32 * cy <= yy < 32 * (cy + 1) for yy in range(y * f, (y + 1) * f))]
            assert len(cy) == 1
            for x in range(ws):
                cx = [cx for cx in range(9)
                      if all(32 * cx <= xx < 32 * (cx + 1) for xx in range(x * f, (x + 1) * f))]
                assert len(cx) == 1
                assert got[y, x] == mask[cy[0], cx[0]], (f, y, x)


# ---------------------------------------------------------------- loss, gradient


def test_dice_bce_closed_form():
    n = 10
    L = torch.zeros(n, dtype=F64)
    g = torch.ones(n, dtype=F64)
    v = O.dice_bce(L, g)
    dice = 1 - (2 * 0.5 * n + 1) / (0.5 * n + n + 1)
    assert abs(float(v) - (dice + math.log(2))) < 1e-14
    L = torch.tensor([-3.0, 0.5, 2.0, 7.0], dtype=F64)
    g = torch.tensor([0.0, 1.0, 0.0, 1.0], dtype=F64)
    s = torch.sigmoid(L)
    naive = (-(g * torch.log(s) + (1 - g) * torch.log(1 - s))).mean()
    dice = 1 - (2 * (s * g).sum() + 1) / (s.sum() + g.sum() + 1)
    assert abs(float(O.dice_bce(L, g)) - float(naive + dice)) < 1e-14


@pytest.mark.slow
def test_gradient_matches_central_differences():
    w = synth.small_variant(synth.DIFF, H=256, W=256, P=64, S=32, base=4, levels=3,
                            max_batch=16)
    rgb = synth.gen_slide(synth.spec_for(w))
    gts = synth.gen_gt_masks(w.H, w.W, w.factors, w.class_scale, seed=7)
    prob = O.DiffProblem(rgb, w, synth.gen_weights(w), gts)
    loss, grads = prob.loss_and_grads()
    base = prob.params()
    r = rng(8)
    eps = 1e-6
    names = list(base)
    checked = 0
    for trial in range(48):
        name = names[trial % len(names)]
        idx = tuple(int(r.integers(0, s)) for s in base[name].shape)
        qp = {k: v.clone() for k, v in base.items()}
        qm = {k: v.clone() for k, v in base.items()}
        qp[name][idx] += eps
        qm[name][idx] -= eps
        with torch.no_grad():
            fd = (float(prob.loss(qp)) - float(prob.loss(qm))) / (2 * eps)
        an = float(grads[name][idx])
        # central differences at eps = 1e-6 carry ~1e-10 absolute round-off, so
        # entries far below the tensor's largest are compared against 1e-5 * max
        scale = max(abs(fd), 1e-5 * float(grads[name].abs().max()), 1e-9)
        assert abs(an - fd) / scale < 1e-4, (name, idx, an, fd)
        checked += 1
    assert checked == 48


def test_heads_only_loss_equals_full_loss():
    """The head-only evaluation (last block output reused) gives the same loss
    as the full sub-chain for controller / pre-head perturbations."""
    w = synth.small_variant(synth.DIFF, H=256, W=256, P=64, S=32, base=4, levels=3, max_batch=16)
    rgb = synth.gen_slide(synth.spec_for(w))
    gts = synth.gen_gt_masks(w.H, w.W, w.factors, w.class_scale, seed=7)
    prob = O.DiffProblem(rgb, w, synth.gen_weights(w), gts)
    base = prob.params()
    r = rng(9)
    for name in ("ctrl.w", "ctrl.b", "head.w", "head.b"):
        q = {name: base[name] + 1e-3 * torch.from_numpy(r.standard_normal(tuple(base[name].shape)))}
        with torch.no_grad():
            a, b = float(prob.loss(q)), float(prob.loss_heads_only(q))
        assert abs(a - b) <= 1e-13 * max(1.0, abs(a)), (name, a, b)


def test_gradient_by_batch_equals_one_pass_autograd():
    """The batch-by-batch gradient (chain rule through the overlap average
    written out) equals autograd over the whole stitched loss."""
    w = synth.small_variant(synth.DIFF, H=256, W=256, P=64, S=32, base=4, levels=3, max_batch=16)
    rgb = synth.gen_slide(synth.spec_for(w))
    gts = synth.gen_gt_masks(w.H, w.W, w.factors, w.class_scale, seed=7)
    prob = O.DiffProblem(rgb, w, synth.gen_weights(w), gts)
    l1, g1 = prob.loss_and_grads()
    l2, g2 = prob.loss_and_grads_by_batch()
    assert abs(l1 - l2) <= 1e-13 * abs(l1)
    for k in g1:
        assert torch.allclose(g1[k], g2[k], rtol=1e-10, atol=1e-13 * float(g1[k].abs().max())), k


def test_diff_workload_fd_golden_matches_autograd():
    """tests/golden/diff_fd.json (make_diff_fd.py): on the differentiation
    workload itself, the oracle's autograd gradient equals FP64 central
    differences at 64 seeded parameters, entry by entry."""
    p = os.path.join(os.path.dirname(GOLDEN), "diff_fd.json")
    g = json.load(open(p))
    assert len(g["draws"]) == 64
    assert len({d["name"] for d in g["draws"]}) == len(O.GRAD_PARAMS)
    for d in g["draws"]:
        floor = 1e-4 * d["tensor_max_abs_grad"]
        assert abs(d["autograd"] - d["fd"]) <= 1e-4 * max(abs(d["fd"]), floor), d


def test_window_from_regions_equals_whole_slide():
    """Evaluating a window from 40x regions (pyramid crops built per tile) gives
    exactly the whole-slide evaluation restricted to that window."""
    w = synth.NEEDLE.with_(H=1024, W=1536, P=128, S=64, base=8, levels=3, median_k=5)
    spec = synth.make_spec(1024, 1536, 3, 0.45, "cores", 3)
    rgb = synth.gen_slide(spec)
    blob = synth.gen_weights(w)
    win = (256, 512, 256, 256)
    full = O.segment(rgb, w, blob, window=win, batch=8)
    prep = full["prep"]
    reg = O.segment_window_regions(lambda y, x, h, ww: prep["canvas"][y:y + h, x:x + ww], prep["mask"],
                                   w, blob, win, prep["Hp"], prep["Wp"], batch=8)
    for c in range(w.n_classes):
        assert np.array_equal(full["L"][c], reg["L"][c])
        assert np.array_equal(full["cov"][c], reg["cov"][c])
        assert np.array_equal(full["labels"][c], reg["labels"][c])
    assert any(full["cov"][c].max() > 0 for c in full["cov"])


# ---------------------------------------------------------------- input generator


def test_needle_cores_hold_structure_discs_inside_tissue_only():
    """Needle-biopsy slides carry the sharp-edged structure discs inside their
    cores (each disc inside its 512-px cell, every structure pixel on tissue);
    blob slides carry none."""
    from synth import slides as S
    spec = synth.spec_for(synth.NEEDLE)
    assert spec.structures and not synth.spec_for(synth.TINY).structures
    ys = np.arange(5120, 7168, dtype=np.int64)[:, None]
    xs = np.arange(24576, 26624, dtype=np.int64)[None, :]
    yy, xx = np.broadcast_arrays(ys, xs)
    st = S._structures(spec, yy, xx)
    depth = S._depth_q8(spec, ys, xs)
    inside = (st >= 0) & (depth >= 0)
    assert inside.mean() > 0.05 and set(np.unique(st[inside]).tolist()) == {0, 1, 2}
    img = synth.gen_window(spec, 5120, 24576, 2048, 2048).astype(np.int64)
    for t, col in enumerate(S.STRUCT_COLOURS):
        m = (st == t) & (depth >= 0)
        mean = img[m].mean(axis=0)
        assert np.all(np.abs(mean - np.array(col)) < 2.0), (t, mean)


def test_generator_windows_are_consistent():
    spec = synth.make_spec(300, 500, 5, 0.4, "cores", 3)
    full = synth.gen_slide(spec)
    assert np.array_equal(synth.gen_window(spec, 37, 111, 50, 70), full[37:87, 111:181])
    bg = full[full.min(axis=2) > 225]
    assert abs(bg.mean() - 235) < 2 and bg.std() > 3


# ---------------------------------------------------------------- stained products (Sec. 2.3)


def test_stain_hand_values_identities_and_order():
    """(100, 200, 50) stained red (255, 0, 0) at alpha 128: (100*128 + 255*128 +
    128) >> 8 = 178, (200*128 + 128) >> 8 = 100, (50*128 + 128) >> 8 = 25.
    Alpha 0 leaves the slide, alpha 256 paints the colour, later maps paint
    over earlier ones."""
    rgb = np.zeros((4, 4, 3), np.uint8)
    rgb[...] = (100, 200, 50)
    on = np.ones((4, 4), np.uint8)
    assert O.stain(rgb, [on], [1], [(255, 0, 0)], [128])[0, 0].tolist() == [178, 100, 25]
    assert np.array_equal(O.stain(rgb, [on], [1], [(255, 0, 0)], [0]), rgb)
    assert O.stain(rgb, [on], [1], [(7, 8, 9)], [256])[2, 3].tolist() == [7, 8, 9]
    two = O.stain(rgb, [on, on], [1, 1], [(7, 8, 9), (1, 2, 3)], [256, 256])
    assert (two.reshape(-1, 3) == (1, 2, 3)).all()
    assert np.array_equal(O.stain(rgb, [None], [1], [(1, 2, 3)], [256]), rgb)


def test_stain_maps_lower_scales_by_their_factor():
    """A 10x map pixel (1, 2) covers 40x rows 4..7 and columns 8..11 exactly
    (brute force over the slide)."""
    rgb = rng(21).integers(0, 256, (13, 17, 3)).astype(np.uint8)
    m = np.zeros((4, 5), np.uint8)
    m[1, 2] = 1
    out = O.stain(rgb, [m], [4], [(0, 0, 0)], [256])
    for y in range(13):
        for x in range(17):
            inside = 4 <= y < 8 and 8 <= x < 12
            assert out[y, x].tolist() == ([0, 0, 0] if inside else rgb[y, x].tolist())


def test_resize_down_rounding_edges_and_pyramid():
    """Box mean rounded half up: eight 5s and eight 0s in a 4 x 4 block give
    (40 + 8) // 16 = 3; a 5 x 7 image resized by 4 is 2 x 2, its corner block
    averaging the 1 x 3 remaining pixels; a constant-block image resizes
    exactly; resizing by 2 equals the pyramid's 2 x 2 mean."""
    img = np.zeros((4, 4, 3), np.uint8)
    img[:2] = 5
    assert O.resize_down(img, 4)[0, 0].tolist() == [3, 3, 3]
    r = rng(22).integers(0, 256, (5, 7, 3)).astype(np.uint8)
    d = O.resize_down(r, 4)
    assert d.shape == (2, 2, 3)
    blk = r[4:5, 4:7].reshape(-1, 3).astype(np.int64)
    assert d[1, 1].tolist() == ((blk.sum(0) + 1) // 3).tolist()
    blk = r[0:4, 4:7].reshape(-1, 3).astype(np.int64)
    assert d[0, 1].tolist() == ((blk.sum(0) + 6) // 12).tolist()
    c = np.repeat(np.repeat(rng(23).integers(0, 256, (3, 5, 3)), 8, 0), 8, 1).astype(np.uint8)
    assert np.array_equal(O.resize_down(c, 8), c[::8, ::8])
    e = rng(24).integers(0, 256, (16, 24, 3)).astype(np.uint8)
    assert np.array_equal(O.resize_down(e, 2), O.half(e))


def test_area_filter_pins():
    """Sec. 2.1's contour step as read here (8-connected tissue regions under
    min_area pixels removed): hand cases fix the connectivity and the hole
    handling; on random masks the kept pixels equal scipy's 8-connected
    labelling with its region sizes (an independent library routine)."""
    ndi = pytest.importorskip("scipy.ndimage")
    m = np.zeros((6, 6), bool)
    m[1, 1] = m[2, 2] = True                       # diagonal contact: one region of 2
    assert O.area_filter(m, 2).sum() == 2 and O.area_filter(m, 3).sum() == 0
    ring = np.zeros((5, 5), bool)
    ring[1:4, 1:4] = True
    ring[2, 2] = False                             # 8 pixels around a hole: one region of 8
    assert np.array_equal(O.area_filter(ring, 8), ring) and not O.area_filter(ring, 9).any()
    assert np.array_equal(O.area_filter(ring, 0), ring)
    rng = np.random.default_rng(5)
    for trial in range(6):
        mask = rng.random((40, 57)) < 0.35 + 0.05 * trial
        lab, n = ndi.label(mask, structure=np.ones((3, 3), int))
        sizes = np.bincount(lab.ravel())
        for a in (1, 3, 7, 20):
            want = mask & (sizes[lab] >= a)
            assert np.array_equal(O.area_filter(mask, a), want), (trial, a)
