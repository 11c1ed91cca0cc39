"""Edge cases of the whole path on the GPU: a slide without any foreground
tile, a slide smaller than one tile, the vote stitch mode against the FP64
oracle, and properties that must hold exactly: results do not depend on the
batch size, and a run restricted to some scales and classes reproduces the
full run's maps for them."""
import numpy as np
import pytest
import torch

import synth
from oracle import omniseg_oracle as O

pytestmark = pytest.mark.gpu

LOGIT_TOL = 1e-4
LABEL_BAND = 1e-3


@pytest.fixture(scope="module")
def api():
    from paper_2305_14566_gb300.build import build
    build()
    from paper_2305_14566_gb300 import api as A
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return A


def _prec(name):
    from paper_2305_14566_gb300 import _lib as L
    return {"fp32": L.FP32, "bf16": L.BF16, "fp16": L.FP16}[name]


# a base-32, 3-level network on 128-pixel tiles: every tensor-core variant applies
SMALL = synth.NEEDLE.with_(P=128, S=64, levels=3, median_k=5, max_batch=8)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_background_slide_segments_to_empty_maps(api, prec):
    """A slide of plain glass has no tissue, hence no tile at any scale: every
    label, logit, coverage and argmax value is 0 and nothing fails."""
    w = SMALL.with_(H=1024, W=2048)
    rgb = torch.full((1024, 2048, 3), 235, dtype=torch.uint8, device="cuda")
    seg = api.Segmenter(w, synth.gen_weights(w), precision=_prec(prec))
    t = seg.tile_slide(rgb)
    assert int(t["counts"].sum().item()) == 0
    out = seg.segment(rgb, logits=True, coverage=True, argmax=True)
    torch.cuda.synchronize()
    for k in out["labels"]:
        assert int(out["labels"][k].count_nonzero().item()) == 0
        assert int(out["logits"][k].count_nonzero().item()) == 0
    for s in out["coverage"]:
        assert int(out["coverage"][s].count_nonzero().item()) == 0
        assert int(out["argmax"][s].count_nonzero().item()) == 0
    seg.close()


def test_slide_smaller_than_one_tile_fp32_against_oracle(api):
    """A 100 x 150 slide is padded to the tile grid (1024 x 1024 at 40x for
    8 x 128-pixel tiles at 5x); the maps are cropped back to 100 x 150 (10x:
    25 x 38, 5x: 13 x 19) and match the oracle."""
    w = SMALL.with_(H=100, W=150)
    spec = synth.make_spec(100, 150, 31, 0.5, "blobs", 2)
    rgb_np = synth.gen_slide(spec)
    blob = synth.gen_weights(w)
    seg = api.Segmenter(w, blob)
    sz = seg.query(100, 150)
    assert (sz.Hp, sz.Wp) == (1024, 1024)
    out = seg.segment(torch.from_numpy(rgb_np).cuda(), logits=True, coverage=True)
    torch.cuda.synchronize()
    orc = O.segment(rgb_np, w, blob, batch=8)
    for c, s in enumerate(w.class_scale):
        f = w.factors[s]
        oh, ow = -(-100 // f), -(-150 // f)
        g = out["logits"][c].double().cpu().numpy()
        assert g.shape == (oh, ow)
        o = orc["L"][c][:oh, :ow]
        assert np.abs(g - o).max() <= LOGIT_TOL, c
        gl = out["labels"][c].cpu().numpy()
        bad = gl != orc["labels"][c][:oh, :ow]
        assert not (bad & (np.abs(o) >= LABEL_BAND)).any(), c
        cov = out["coverage"][s].cpu().numpy().astype(np.int64)
        assert np.array_equal(cov, orc["cov"][c][:oh, :ow])
    seg.close()


def test_vote_stitch_mode_fp32_against_oracle(api):
    """Vote stitching (a pixel is positive when at least half of its covering
    tiles say so): labels equal the oracle's except where a covering tile's
    logit is within 1e-3 of zero (its vote may differ) and that one vote
    decides the label (2 votes - coverage in [-2, 1])."""
    w = SMALL.with_(H=1024, W=1536, stitch_mode=synth.STITCH_VOTE)
    spec = synth.make_spec(1024, 1536, 33, 0.5, "cores", 3)
    rgb_np = synth.gen_slide(spec)
    blob = synth.gen_weights(w)
    seg = api.Segmenter(w, blob)
    out = seg.segment(torch.from_numpy(rgb_np).cuda(), logits=True, coverage=True)
    torch.cuda.synchronize()
    orc = O.segment(rgb_np, w, blob, window=(256, 512, 256, 256), batch=8)
    n_pos = 0
    for c, s in enumerate(w.class_scale):
        wy, wx, wh, ww = orc["window"][s]
        gl = out["labels"][c][wy:wy + wh, wx:wx + ww].cpu().numpy()
        ol = orc["labels"][c]
        m = 2 * orc["votes"][c] - orc["cov"][c]
        bad = gl != ol
        assert not (bad & ((m < -2) | (m > 1))).any(), c
        assert not (bad & (orc["margin"][c] >= 1e-3)).any(), (c, int(bad.sum()))
        n_pos += int(ol.sum())
        g = out["logits"][c][wy:wy + wh, wx:wx + ww].double().cpu().numpy()
        assert np.abs(g - orc["L"][c]).max() <= LOGIT_TOL
    assert n_pos > 0, "the window should hold positive votes"
    seg.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_results_do_not_depend_on_batch_size(api, prec):
    """Tiles are independent: the same slide through batches of 3 and of 16
    tiles gives bit-identical logits and labels (default kernels)."""
    w = SMALL.with_(H=1024, W=1536)
    spec = synth.make_spec(1024, 1536, 34, 0.5, "cores", 3)
    rgb = torch.from_numpy(synth.gen_slide(spec)).cuda()
    blob = synth.gen_weights(w)
    res = []
    for mb in (3, 16):
        seg = api.Segmenter(w.with_(max_batch=mb), blob, precision=_prec(prec))
        o = seg.segment(rgb, logits=True)
        torch.cuda.synchronize()
        res.append({k: {c: t.clone() for c, t in d.items()} for k, d in o.items()})
        seg.close()
    for c in res[0]["logits"]:
        assert torch.equal(res[0]["logits"][c], res[1]["logits"][c]), c
        assert torch.equal(res[0]["labels"][c], res[1]["labels"][c]), c


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_scale_and_class_subsets_match_the_full_run(api, prec):
    """Segmenting only the 10x scale's classes, or a single 40x class (one
    dynamic head per tile), reproduces the full run's maps bit for bit."""
    w = SMALL.with_(H=1024, W=1536)
    spec = synth.make_spec(1024, 1536, 35, 0.5, "cores", 3)
    rgb = torch.from_numpy(synth.gen_slide(spec)).cuda()
    blob = synth.gen_weights(w)
    seg = api.Segmenter(w, blob, precision=_prec(prec))
    full = seg.segment(rgb, logits=True)
    full = {k: {c: t.clone() for c, t in d.items()} for k, d in full.items()}
    part = seg.segment(rgb, scales=[1], classes=[2, 3], logits=True)
    one = seg.segment(rgb, scales=[0], classes=[0], logits=True)
    torch.cuda.synchronize()
    assert sorted(part["labels"]) == [2, 3] and sorted(one["labels"]) == [0]
    for c in (2, 3):
        assert torch.equal(part["logits"][c], full["logits"][c]), c
        assert torch.equal(part["labels"][c], full["labels"][c]), c
    assert torch.equal(one["logits"][0], full["logits"][0])
    assert torch.equal(one["labels"][0], full["labels"][0])
    seg.close()
