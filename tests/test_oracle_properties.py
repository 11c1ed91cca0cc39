"""Randomised invariants of the oracle (CPU): stitching, staining, resizing,
median blur, tiling and the network pieces obey properties that hold for
any input, so a misapplied weight, a wrong index or a dropped term in the
oracle shows up on inputs no fixed case covers."""
import numpy as np
import pytest

import synth
from oracle import omniseg_oracle as O

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings

WINDOWS = [synth.WINDOW_FLAT, synth.WINDOW_TENT, synth.WINDOW_HANN]


@st.composite
def tile_sets(draw):
    P = draw(st.sampled_from([4, 8, 12]))
    S = draw(st.sampled_from([s for s in (2, 4, 6, 8) if P % s == 0]))
    ny, nx = draw(st.integers(1, 4)), draw(st.integers(1, 4))
    hs, ws = (ny - 1) * S + P, (nx - 1) * S + P
    keep = draw(st.lists(st.booleans(), min_size=ny * nx, max_size=ny * nx))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    g = np.random.default_rng(seed)
    tiles = {(i * S, j * S): g.standard_normal((P, P))
             for i in range(ny) for j in range(nx) if keep[i * nx + j]}
    return tiles, hs, ws, P


@settings(max_examples=60, deadline=None)
@given(tile_sets(), st.sampled_from(WINDOWS))
def test_stitch_is_a_convex_combination_of_covering_tiles(ts, window):
    """Where covered, the stitched logit lies between the smallest and largest
    covering tile logit; coverage and votes equal brute-force counts;
    uncovered pixels are exactly 0."""
    tiles, hs, ws, P = ts
    L, cov, votes = O.stitch(tiles, hs, ws, P, window)
    for y in range(hs):
        for x in range(ws):
            vals = [t[y - ty, x - tx] for (ty, tx), t in tiles.items()
                    if ty <= y < ty + P and tx <= x < tx + P]
            assert cov[y, x] == len(vals)
            assert votes[y, x] == sum(v > 0 for v in vals)
            if vals:
                assert min(vals) - 1e-12 <= L[y, x] <= max(vals) + 1e-12
            else:
                assert L[y, x] == 0.0


@settings(max_examples=40, deadline=None)
@given(tile_sets(), st.sampled_from(WINDOWS), st.floats(-5, 5), st.floats(0.5, 3))
def test_stitch_commutes_with_affine_maps(ts, window, b, a):
    """A weighted average commutes with l -> a l + b on every covered pixel."""
    tiles, hs, ws, P = ts
    L, cov, _ = O.stitch(tiles, hs, ws, P, window)
    L2, _, _ = O.stitch({k: a * v + b for k, v in tiles.items()}, hs, ws, P, window)
    m = cov > 0
    assert np.allclose(L2[m], a * L[m] + b, atol=1e-9)


@settings(max_examples=40, deadline=None)
@given(st.integers(1, 19), st.integers(1, 19), st.sampled_from([2, 4, 8]), st.integers(0, 2 ** 31 - 1))
def test_resize_stays_within_block_range(H, W, r, seed):
    """Every resized pixel lies between its block's smallest and largest value
    per channel, and the output is ceil(H / r) x ceil(W / r)."""
    img = np.random.default_rng(seed).integers(0, 256, (H, W, 3)).astype(np.uint8)
    d = O.resize_down(img, r)
    assert d.shape == (-(-H // r), -(-W // r), 3)
    for i in range(d.shape[0]):
        for j in range(d.shape[1]):
            blk = img[i * r:(i + 1) * r, j * r:(j + 1) * r].reshape(-1, 3)
            assert (blk.min(0) <= d[i, j]).all() and (d[i, j] <= blk.max(0)).all()


@settings(max_examples=40, deadline=None)
@given(st.integers(1, 17), st.integers(1, 17), st.integers(0, 2 ** 31 - 1))
def test_stain_opaque_maps_paint_the_last_class(H, W, seed):
    """With every alpha 256 a pixel takes the colour of the last map that is
    on there (maps at factors 1, 2 and 4), else keeps the slide's colour;
    with every alpha 0 the slide is unchanged."""
    g = np.random.default_rng(seed)
    rgb = g.integers(0, 256, (H, W, 3)).astype(np.uint8)
    factors = [1, 2, 4]
    maps = [(g.random((-(-H // f), -(-W // f))) < 0.4).astype(np.uint8) for f in factors]
    cols = [tuple(int(v) for v in g.integers(0, 256, 3)) for _ in factors]
    out = O.stain(rgb, maps, factors, cols, [256] * 3)
    for y in range(H):
        for x in range(W):
            want = rgb[y, x].tolist()
            for m, f, c in zip(maps, factors, cols):
                if m[y // f, x // f]:
                    want = list(c)
            assert out[y, x].tolist() == want
    assert np.array_equal(O.stain(rgb, maps, factors, cols, [0] * 3), rgb)


@settings(max_examples=30, deadline=None)
@given(st.integers(1, 24), st.integers(1, 24), st.sampled_from([1, 3, 5]), st.integers(0, 2 ** 31 - 1))
def test_median_blur_stays_within_its_window(H, W, k, seed):
    """Each blurred value lies between the smallest and largest value of its
    replicate-bordered k x k window, and a constant image is unchanged."""
    img = np.random.default_rng(seed).integers(0, 256, (H, W)).astype(np.uint8)
    b = O.median_blur(img, k)
    r = k // 2
    pad = np.pad(img, r, mode="edge")
    for y in range(H):
        for x in range(W):
            win = pad[y:y + k, x:x + k]
            assert win.min() <= b[y, x] <= win.max()
    c = np.full((H, W), 77, np.uint8)
    assert np.array_equal(O.median_blur(c, k), c)


@settings(max_examples=30, deadline=None)
@given(st.sampled_from([(1,), (1, 4), (1, 4, 8)]), st.integers(1, 3), st.integers(1, 3))
def test_tile_list_full_and_empty_masks(factors, hy, wx):
    """With a tissue mask covering everything every grid tile is foreground;
    with an empty mask none is; the list is ordered by scale, row, column."""
    P, S = 64, 32
    w = synth.TINY.with_(factors=factors, P=P, S=S, H=256 * hy, W=256 * wx, tissue_filter=True,
                         class_scale=(0,))
    Hp, Wp, _ = O.padded_dims(w)
    full, _ = O.tile_list(w, np.ones((Hp // 32, Wp // 32), bool), Hp, Wp)
    empty, _ = O.tile_list(w, np.zeros((Hp // 32, Wp // 32), bool), Hp, Wp)
    assert len(full) == sum(int(np.prod(O.grid(w, Hp, Wp, s))) for s in range(len(factors)))
    assert empty == [] and full == sorted(full)


@settings(max_examples=25, deadline=None)
@given(st.integers(1, 6), st.integers(1, 6), st.integers(0, 2 ** 31 - 1))
def test_upsample_commutes_with_flips_and_is_linear(H, W, seed):
    """Half-pixel bilinear x2 with edge clamp is symmetric: flipping the input
    along an axis flips the output; it is linear; its outputs stay within the
    input's range (convex weights)."""
    import torch
    g = torch.Generator().manual_seed(seed)
    x = torch.randn((1, 2, H, W), generator=g, dtype=torch.float64)
    y = torch.randn((1, 2, H, W), generator=g, dtype=torch.float64)
    u = O.upsample2(x)
    for d in (2, 3):
        assert torch.allclose(O.upsample2(x.flip(d)), u.flip(d), atol=1e-12)
    assert torch.allclose(O.upsample2(2.0 * x - y), 2.0 * u - O.upsample2(y), atol=1e-12)
    assert u.shape == (1, 2, 2 * H, 2 * W)
    assert float(u.min()) >= float(x.min()) - 1e-12 and float(u.max()) <= float(x.max()) + 1e-12


@settings(max_examples=25, deadline=None)
@given(st.integers(1, 6), st.integers(1, 6), st.integers(1, 3), st.integers(1, 3), st.integers(0, 2 ** 31 - 1))
def test_conv3x3_flip_equivariance_and_linearity(H, W, C, O_, seed):
    """Flipping the input and the kernel along an axis flips the output (zero
    padding is symmetric); the conv is linear in the input and the weights."""
    import torch
    g = torch.Generator().manual_seed(seed)
    x = torch.randn((2, C, H, W), generator=g, dtype=torch.float64)
    x2 = torch.randn((2, C, H, W), generator=g, dtype=torch.float64)
    w = torch.randn((O_, C, 3, 3), generator=g, dtype=torch.float64)
    w2 = torch.randn((O_, C, 3, 3), generator=g, dtype=torch.float64)
    y = O.conv3x3(x, w)
    for d in (2, 3):
        assert torch.allclose(O.conv3x3(x.flip(d), w.flip(d)), y.flip(d), atol=1e-12)
    assert torch.allclose(O.conv3x3(x + 3.0 * x2, w), y + 3.0 * O.conv3x3(x2, w), atol=1e-10)
    assert torch.allclose(O.conv3x3(x, w - w2), y - O.conv3x3(x, w2), atol=1e-10)


@settings(max_examples=25, deadline=None)
@given(st.integers(1, 5), st.integers(1, 5), st.integers(0, 2 ** 31 - 1))
def test_maxpool_picks_the_window_maximum(H, W, seed):
    """Each pooled value is one of its 2 x 2 window's values and not below any."""
    import torch
    g = torch.Generator().manual_seed(seed)
    x = torch.randn((1, 3, 2 * H, 2 * W), generator=g, dtype=torch.float64)
    m = O.maxpool2(x)
    win = x.reshape(1, 3, H, 2, W, 2).permute(0, 1, 2, 4, 3, 5).reshape(1, 3, H, W, 4)
    assert torch.equal(m, win.max(dim=-1).values)


@settings(max_examples=25, deadline=None)
@given(st.integers(1, 4), st.integers(0, 2 ** 31 - 1))
def test_dynamic_head_is_per_tile(B, seed):
    """Tile b's logits depend only on tile b's features and parameters:
    permuting the batch permutes the output."""
    import torch
    g = torch.Generator().manual_seed(seed)
    h0 = torch.relu(torch.randn((B, 8, 3, 5), generator=g, dtype=torch.float64))
    th = torch.randn((B, synth.N_HEAD_PARAMS), generator=g, dtype=torch.float64)
    out = O.dynamic_head(h0, th)
    perm = torch.randperm(B, generator=g)
    assert torch.allclose(O.dynamic_head(h0[perm], th[perm]), out[perm], atol=1e-12)
