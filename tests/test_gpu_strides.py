"""Overlap variants through the whole GPU path.  Per-scale tile strides
(Sec. 3.2: 256 at 40x, 64 at 10x and 5x, majority vote): the tile lists
equal the oracle's, the FP32 maps match the FP64 oracle on a window, the
tensor-core precisions agree with FP32, and the needle slide tiles to the
oracle's stored counts.  Weighted overlap averages (tent and Hann windows)
match the oracle's."""
import json
import os

import numpy as np
import pytest
import torch

import synth
from oracle import omniseg_oracle as O

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LOGIT_TOL = 1e-4

# 128-pixel tiles strided 64 at 40x and 16 at 10x and 5x: two overlapping
# tiles per axis at 40x, eight at the coarser scales, as in Sec. 3.2
SMALL = synth.NEEDLE.with_(P=128, S=64, levels=3, median_k=5, max_batch=8, H=1024, W=1536,
                           strides=(64, 16, 16), stitch_mode=synth.STITCH_VOTE)


@pytest.fixture(scope="module")
def api():
    from paper_2305_14566_gb300.build import build
    build()
    from paper_2305_14566_gb300 import api as A
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return A


@pytest.fixture(scope="module")
def slide():
    spec = synth.make_spec(SMALL.H, SMALL.W, 36, 0.5, "cores", 3)
    return synth.gen_slide(spec)


def test_tile_list_matches_oracle(api, slide):
    """Tissue mask, per-scale flags and the (scale, y, x) list equal the
    oracle's, bit for bit; the grids are 15 x 23, 9 x 17 and 1 x 5."""
    seg = api.Segmenter(SMALL, synth.gen_weights(SMALL))
    sz = seg.query(SMALL.H, SMALL.W)
    assert [(sz.grid_h[s], sz.grid_w[s]) for s in range(3)] == [(15, 23), (9, 17), (1, 5)]
    t = seg.tile_slide(torch.from_numpy(slide).cuda())
    torch.cuda.synchronize()
    prep = O.prepare(slide, SMALL)
    n = int(t["counts"][0].item())
    assert n == len(prep["tiles"])
    assert [tuple(r) for r in t["tiles"][:n].cpu().tolist()] == [tuple(q) for q in prep["tiles"]]
    flags = np.concatenate([f.ravel() for f in prep["flags"]]).astype(np.uint8)
    assert np.array_equal(t["flags"][:flags.size].cpu().numpy(), flags)
    assert np.array_equal(t["tissue"].cpu().numpy().astype(bool), prep["mask"])
    seg.close()


def test_vote_maps_fp32_against_oracle(api, slide):
    """Coverage equals the oracle's (up to 64 tiles at 10x), logits agree
    within 1e-4 and labels equal the oracle's except where a covering tile's
    logit is within 1e-3 of zero (its vote may differ) and that one vote
    decides the label (2 votes - coverage in [-2, 1])."""
    blob = synth.gen_weights(SMALL)
    seg = api.Segmenter(SMALL, blob)
    out = seg.segment(torch.from_numpy(slide).cuda(), logits=True, coverage=True)
    torch.cuda.synchronize()
    orc = O.segment(slide, SMALL, blob, window=(256, 512, 256, 256), batch=8)
    assert int(orc["cov"][2].max()) == 64 and int(orc["cov"][0].max()) == 4
    for c, s in enumerate(SMALL.class_scale):
        wy, wx, wh, ww = orc["window"][s]
        cov = out["coverage"][s][wy:wy + wh, wx:wx + ww].cpu().numpy().astype(np.int64)
        assert np.array_equal(cov, orc["cov"][c]), c
        g = out["logits"][c][wy:wy + wh, wx:wx + ww].double().cpu().numpy()
        assert np.abs(g - orc["L"][c]).max() <= LOGIT_TOL, c
        gl = out["labels"][c][wy:wy + wh, wx:wx + ww].cpu().numpy()
        m = 2 * orc["votes"][c] - orc["cov"][c]
        bad = gl != orc["labels"][c]
        assert not (bad & ((m < -2) | (m > 1))).any(), c
        assert not (bad & (orc["margin"][c] >= 1e-3)).any(), (c, int(bad.sum()))
    seg.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_tensor_core_precisions_agree_with_fp32(api, slide, prec):
    """The tensor-core path with per-scale strides labels at least 99.5% of
    every class's pixels as the FP32 path does (majority votes over up to 64
    tiles absorb most rounding)."""
    from paper_2305_14566_gb300 import _lib as L
    blob = synth.gen_weights(SMALL)
    rgb = torch.from_numpy(slide).cuda()
    s32 = api.Segmenter(SMALL, blob)
    o32 = s32.segment(rgb)
    o32 = {c: t.clone() for c, t in o32["labels"].items()}
    s32.close()
    seg = api.Segmenter(SMALL, blob, precision=L.BF16 if prec == "bf16" else L.FP16)
    out = seg.segment(rgb)
    torch.cuda.synchronize()
    for c in o32:
        ag = float((out["labels"][c] == o32[c]).float().mean().item())
        print("%s class %d agreement %.5f" % (prec, c, ag))
        assert ag >= 0.995, (c, ag)
    seg.close()


def test_needle_slide_tiles_to_the_oracle_counts(api):
    """The 16384 x 49152 needle slide with strides 256 / 64 / 64 gives the
    oracle's stored foreground counts per scale (grids 63 x 191, 57 x 185,
    25 x 89) and its stored tissue mask."""
    gold = json.load(open(os.path.join(GOLDEN, "needle_tiles.json")))
    m = np.load(os.path.join(GOLDEN, "needle_tissue_mask.npz"))
    mask = np.unpackbits(m["bits"])[:int(np.prod(m["shape"]))].reshape(m["shape"]).astype(bool)
    w = synth.NEEDLE_PAPER
    assert list(w.strides) == gold["paper_strides"]
    rgb = api.synth_slide(synth.spec_for(w))
    t = api.tile_slide_noalloc(w, rgb)
    torch.cuda.synchronize()
    counts = t["counts"].cpu().tolist()
    assert counts[1:] == gold["paper_strides_tiles_per_scale"]
    assert counts[0] == gold["paper_strides_tiles_total"]
    assert np.array_equal(t["tissue"].cpu().numpy().astype(bool), mask)


@pytest.mark.parametrize("window", [synth.WINDOW_TENT, synth.WINDOW_HANN])
@pytest.mark.parametrize("strides", [(), (64, 16, 16)])
def test_windowed_average_fp32_against_oracle(api, slide, window, strides):
    """L = sum_p w_p l_p / sum_p w_p with a tent or Hann tile window: logits
    within 1e-4 of the oracle, labels equal wherever |L| >= 1e-3, coverage
    exact; the flat-window run of the same slide differs (the window is used)."""
    w = SMALL.with_(strides=strides, stitch_window=window, stitch_mode=synth.STITCH_AVG)
    blob = synth.gen_weights(w)
    rgb = torch.from_numpy(slide).cuda()
    seg = api.Segmenter(w, blob)
    out = seg.segment(rgb, logits=True, coverage=True)
    out = {k: {c: t.clone() for c, t in d.items()} for k, d in out.items()}
    seg.close()
    flat = api.Segmenter(w.with_(stitch_window=synth.WINDOW_FLAT), blob)
    fo = flat.segment(rgb, logits=True)
    torch.cuda.synchronize()
    orc = O.segment(slide, w, blob, window=(256, 512, 256, 256), batch=8)
    for c, s in enumerate(w.class_scale):
        wy, wx, wh, ww = orc["window"][s]
        g = out["logits"][c][wy:wy + wh, wx:wx + ww].double().cpu().numpy()
        o = orc["L"][c]
        assert np.abs(g - o).max() <= LOGIT_TOL, c
        gl = out["labels"][c][wy:wy + wh, wx:wx + ww].cpu().numpy()
        assert not ((gl != orc["labels"][c]) & (np.abs(o) >= 1e-3)).any(), c
        cov = out["coverage"][s][wy:wy + wh, wx:wx + ww].cpu().numpy().astype(np.int64)
        assert np.array_equal(cov, orc["cov"][c]), c
    assert any(not torch.equal(out["logits"][c], fo["logits"][c]) for c in fo["logits"])
    flat.close()


def test_backward_refuses_a_weighted_window(api):
    """omni_backward differentiates the flat overlap average only; a context
    with a tent window gets OMNI_EINVAL and a message, nothing launches."""
    from paper_2305_14566_gb300 import _lib as L
    w = synth.DIFF.with_(H=512, W=512, stitch_window=synth.WINDOW_TENT)
    seg = api.Segmenter(w, synth.gen_weights(w))
    rgb = torch.full((512, 512, 3), 200, dtype=torch.uint8, device="cuda")
    sz = seg.query(512, 512)
    gts = [torch.zeros((sz.out_h[s], sz.out_w[s]), dtype=torch.uint8, device="cuda")
           for s in w.class_scale]
    with pytest.raises(L.OmniError) as e:
        seg.backward(rgb, gts)
    assert e.value.status == L.EINVAL and "flat" in str(e.value)
    seg.close()
