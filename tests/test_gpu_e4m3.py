"""The 8-bit experiment of the network's convolutions: one residual-U-Net
conv layer on E4M3 operands (omni_conv_layer with OMNI_E4M3: one activation
scale s_x = max|x| / 448, per-output-channel weight scales, kind::f8f6f4 MMAs
with FP32 accumulation) against the oracle's FP64 conv of the same BF16
activations and FP32 weights.

Bound, from the format alone: E4M3 keeps 3 mantissa bits, so rounding v / s
moves it by at most 2^-4 of itself in the normal range and by 2^-10 below
2^-6 (half the subnormal spacing 2^-9), i.e. |dv| <= 2^-4 |v| + 2^-10 s.  With
A = sum |w||x|, X = sum |x| and W = sum |w| over the 9 cin products of an
output, |d conv| <= (2^-3 + 2^-8) A + 2^-10 (1 + 2^-4)(s_w X + s_x W)
+ 2^-20 s_w s_x 9 cin; times g, plus the BF16 rounding of the output
(2^-8 of it) and 1e-5 g A for the FP32 accumulation.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import omniseg_oracle as O

pytestmark = pytest.mark.gpu

E4M3_SHAPES = [(32, 128, 256), (16, 256, 512), (64, 128, 128)]


@pytest.fixture(scope="module")
def api():
    from paper_2305_14566_gb300.build import build
    build()
    from paper_2305_14566_gb300 import api as A
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return A


def _case(R, cin, cout, B=2):
    rng = np.random.default_rng(2000 + R + cin + cout)
    x = np.abs(rng.standard_normal((B, R, R, cin))).astype(np.float32)
    xb = torch.from_numpy(x).to(torch.bfloat16)                  # the layer's BF16 activations
    x64 = xb.to(torch.float64).permute(0, 3, 1, 2)
    w = (rng.standard_normal((cout, cin, 3, 3)) * np.sqrt(2 / (9 * cin))).astype(np.float32)
    g = rng.uniform(0.9, 1.1, cout).astype(np.float32)
    b = rng.uniform(-0.05, 0.05, cout).astype(np.float32)
    w64 = torch.from_numpy(w.astype(np.float64))
    z = O.affine(O.conv3x3(x64, w64), torch.from_numpy(g.astype(np.float64)),
                 torch.from_numpy(b.astype(np.float64)))
    ref = O.relu(z).permute(0, 2, 3, 1).numpy()
    # the bound's sums
    A = O.conv3x3(x64.abs(), w64.abs()).permute(0, 2, 3, 1).numpy()
    X = O.conv3x3(x64.abs(), torch.ones((1, cin, 3, 3), dtype=torch.float64)).permute(0, 2, 3, 1).numpy()
    W = np.abs(w.astype(np.float64)).reshape(cout, -1).sum(1)
    s_x = float(x64.abs().max()) / 448.0
    s_w = np.abs(w.astype(np.float64)).reshape(cout, -1).max(1) / 448.0
    dconv = ((2.0 ** -3 + 2.0 ** -8) * A + 2.0 ** -10 * (1 + 2.0 ** -4) * (s_w * X + s_x * W)
             + 2.0 ** -20 * s_w * s_x * 9 * cin)
    bound = g * (dconv + 1e-5 * A) * (1 + 2.0 ** -8) + 2.0 ** -8 * np.abs(ref)
    return xb, w, g, b, ref, bound


def _run(api, L, xb, R, cin, cout, w, g, b, config):
    y = torch.full((xb.shape[0], R, R, cout), float("nan"), dtype=torch.bfloat16, device="cuda")
    api.conv_layer(L.E4M3, xb.cuda(), R, cin, cout, w, g, b, y, config=config)
    torch.cuda.synchronize()
    return y


@pytest.mark.parametrize("R,cin,cout", E4M3_SHAPES)
def test_e4m3_layer_within_the_format_bound(api, R, cin, cout):
    """Every E4M3 configuration (per-tap kernel on one CTA or CTA pairs, N tile
    128 / 256) stays within the bound derived from the format, and all of them
    give the same bits (each output sums the same K = 32 products in the same
    order)."""
    from paper_2305_14566_gb300 import _lib as L
    xb, w, g, b, ref, bound = _case(R, cin, cout)
    outs = []
    for kind in (0, 8):
        for bn in (128, 256):
            if bn > cout or cout % bn:
                continue
            y = _run(api, L, xb, R, cin, cout, w, g, b, (kind, bn, 128, 0))
            got = y.float().cpu().numpy()
            assert np.isfinite(got).all(), (kind, bn)
            err = np.abs(got - ref)
            assert (err <= bound).all(), (kind, bn, float((err - bound).max()))
            outs.append(y)
    for y in outs[1:]:
        assert torch.equal(y, outs[0])
    got = outs[0].float().cpu().numpy()
    rel = np.sqrt(np.mean((got - ref) ** 2) / np.mean(ref ** 2))
    print("e4m3 R=%d cin=%d cout=%d rms rel err %.4f max err/bound %.3f" %
          (R, cin, cout, rel, float((np.abs(got - ref) / bound).max())))
    # against the oracle the 8-bit operands cost about 2^-5 relative (RMS)
    assert rel < 2.0 ** -4


def test_e4m3_layer_refuses_unsupported_shapes(api):
    """cin not a multiple of 128, a residual projection or a configuration
    outside the per-tap E4M3 kernels is refused before any launch."""
    from paper_2305_14566_gb300 import _lib as L
    xb, w, g, b, _, _ = _case(32, 128, 256)
    y = torch.empty((2, 32, 32, 256), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(RuntimeError):
        api.conv_layer(L.E4M3, xb[..., :64].contiguous().cuda(), 32, 64, 256, w[:, :64], g, b, y)
    with pytest.raises(RuntimeError):
        api.conv_layer(L.E4M3, xb.cuda(), 32, 128, 256, w, g, b, y, config=(3, 256, 128, 0))
    r = torch.zeros((2, 32, 32, 128), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(RuntimeError):
        api.conv_layer(L.E4M3, xb.cuda(), 32, 128, 256, w, g, b, y, r=r, cr=128,
                       wp=np.zeros((256, 128), np.float32))
    # the context still works
    y2 = _run(api, L, xb, 32, 128, 256, w, g, b, None)
    assert torch.isfinite(y2.float()).all()


def _agree_dice(a, b):
    a = a > 0
    b = b > 0
    den = int(a.sum() + b.sum())
    return float((a == b).mean()), (1.0 if den == 0 else 2.0 * float((a & b).sum()) / den)


def test_e4m3_network_against_fp32(api):
    """The network with the E4M3 experiment on (the first convs of the deeper
    levels, cin and cout multiples of 128, on 8-bit operands) against the FP32
    path: labels are reported (the 16-bit bar does not apply) and must agree on
    most pixels; the logits differ from the BF16 run's, and switching the
    experiment off gives the BF16 run's bits back.  A non-BF16 segmenter
    refuses it."""
    from paper_2305_14566_gb300 import _lib as L
    w = synth.NEEDLE.with_(H=2048, W=4096, P=256, S=128, median_k=5, max_batch=16)
    rgb = api.synth_slide(synth.make_spec(2048, 4096, 44, 0.5, "cores", 3))
    blob = synth.gen_weights(w)
    seg = api.Segmenter(w, blob, precision=L.BF16)

    def run():
        o = seg.segment(rgb, logits=True)
        torch.cuda.synchronize()
        return {n: {c: t.clone() for c, t in d.items()} for n, d in o.items() if n in ("labels", "logits")}

    ob = run()
    seg.set_e4m3(True)
    o8 = run()
    seg.set_e4m3(False)
    ob2 = run()
    seg.close()
    seg32 = api.Segmenter(w, blob, precision=L.FP32)
    o = seg32.segment(rgb, logits=True)
    torch.cuda.synchronize()
    l32 = {c: t.cpu().numpy() for c, t in o["labels"].items()}
    seg32.close()
    for c in ob["logits"]:
        assert torch.equal(ob2["logits"][c], ob["logits"][c]), c
        assert not torch.equal(o8["logits"][c], ob["logits"][c]), c
        ag8, dc8 = _agree_dice(o8["labels"][c].cpu().numpy(), l32[c])
        agb, dcb = _agree_dice(ob["labels"][c].cpu().numpy(), l32[c])
        d = (o8["logits"][c] - ob["logits"][c]).abs()
        print("e4m3 network class %d vs fp32: agree %.6f dice %.5f (bf16: %.6f / %.5f), max|dL| vs bf16 %.3f" %
              (c, ag8, dc8, agb, dcb, float(d.max())))
        assert ag8 >= 0.9, (c, ag8)
    s16 = api.Segmenter(w, blob, precision=L.FP16)
    with pytest.raises(RuntimeError):
        s16.set_e4m3(True)
    s16.close()
