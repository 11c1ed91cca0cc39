"""The stained 40x product and the image resized from it (Sec. 2.3) against
the oracle, bit for bit: random class maps at 40x, 10x and 5x on ragged and
aligned slides, padded rows, every resize factor, and the label maps of a
real segmentation run."""
import numpy as np
import pytest
import torch

import synth
from oracle import omniseg_oracle as O

pytestmark = pytest.mark.gpu

COLOURS = [(230, 25, 75), (60, 180, 75), (255, 225, 25), (0, 130, 200), (245, 130, 48), (145, 30, 180)]


@pytest.fixture(scope="module")
def api():
    from paper_2305_14566_gb300.build import build
    build()
    from paper_2305_14566_gb300 import api as A
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return A


def _maps(H, W, factors, seed):
    g = np.random.default_rng(seed)
    return [(g.random((-(-H // f), -(-W // f))) < 0.3).astype(np.uint8) for f in factors]


@pytest.mark.parametrize("H,W,down,pad", [(1000, 1500, 4, 0), (1024, 1536, 4, 0), (999, 1501, 8, 0),
                                          (517, 263, 2, 0), (1000, 1500, 4, 12)])
def test_stain_and_resize_match_oracle(api, H, W, down, pad):
    factors = [1, 1, 4, 4, 8, 8]
    alphas = [128, 96, 200, 256, 64, 0]
    maps = _maps(H, W, factors, H + W + down)
    rgb_np = np.random.default_rng(H * W).integers(0, 256, (H, W, 3)).astype(np.uint8)
    full = torch.zeros((H, W * 3 + pad), dtype=torch.uint8, device="cuda")
    full[:, :W * 3] = torch.from_numpy(rgb_np.reshape(H, W * 3)).cuda()
    rgb = full[:, :W * 3].view(H, W, 3) if pad == 0 else torch.as_strided(full, (H, W, 3), (W * 3 + pad, 3, 1))
    labels = {c: torch.from_numpy(m).cuda() for c, m in enumerate(maps)}
    fac = {c: f for c, f in enumerate(factors)}
    s40, sd = api.stain(rgb, labels, fac, colours=COLOURS, alpha=alphas, down=down)
    torch.cuda.synchronize()
    o40 = O.stain(rgb_np, maps, factors, COLOURS, alphas)
    assert np.array_equal(s40.cpu().numpy(), o40)
    assert np.array_equal(sd.cpu().numpy(), O.resize_down(o40, down))
    # each output alone equals the joint run
    _, sd2 = api.stain(rgb, labels, fac, colours=COLOURS, alpha=alphas, down=down, want40=False)
    s402, _ = api.stain(rgb, labels, fac, colours=COLOURS, alpha=alphas, want_down=False)
    torch.cuda.synchronize()
    assert torch.equal(sd2, sd) and torch.equal(s402, s40)


def test_stain_of_segmented_slide(api):
    """The label maps of a segmentation run stained with the default colours
    at alpha 128, and the 10x product, equal the oracle's on the same maps."""
    w = synth.NEEDLE.with_(P=128, S=64, levels=3, median_k=5, max_batch=8, H=1024, W=1536)
    spec = synth.make_spec(w.H, w.W, 37, 0.5, "cores", 3)
    rgb_np = synth.gen_slide(spec)
    rgb = torch.from_numpy(rgb_np).cuda()
    seg = api.Segmenter(w, synth.gen_weights(w))
    out = seg.segment(rgb)
    fac = {c: w.factors[s] for c, s in enumerate(w.class_scale)}
    s40, s10 = api.stain(rgb, out["labels"], fac)
    torch.cuda.synchronize()
    ids = sorted(out["labels"])
    maps = [out["labels"][c].cpu().numpy() for c in ids]
    assert sum(int(m.sum()) for m in maps) > 0
    o40 = O.stain(rgb_np, maps, [fac[c] for c in ids], [api.STAIN_COLOURS[c] for c in ids], [128] * len(ids))
    assert np.array_equal(s40.cpu().numpy(), o40)
    assert np.array_equal(s10.cpu().numpy(), O.resize_down(o40, 4))
    seg.close()


def test_stain_rejects_bad_arguments(api):
    """Bad factor, alpha or resize factor: OMNI_EINVAL before any launch."""
    from paper_2305_14566_gb300 import _lib as L
    rgb = torch.zeros((64, 64, 3), dtype=torch.uint8, device="cuda")
    m = {0: torch.zeros((64, 64), dtype=torch.uint8, device="cuda")}
    for kw in ({"down": 3}, {"alpha": 300}):
        with pytest.raises(L.OmniError):
            api.stain(rgb, m, {0: 1}, **kw)
    with pytest.raises(L.OmniError):
        api.stain(rgb, m, {0: 3})
