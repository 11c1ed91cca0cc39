"""BF16 tcgen05 path against the FP64 oracle.

Layer level: one fused conv (implicit GEMM on the tensor cores) against the
oracle's FP64 conv evaluated on the same BF16-rounded operands, so the only
differences are FP32 accumulation order and the final BF16 rounding of the
output (relative 2^-8).

Whole path: label agreement and per-class Dice of the BF16 labels against the
oracle's (FP64) labels, and the logit error statistics.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import omniseg_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2305_14566_gb300.build import build
    build()
    from paper_2305_14566_gb300 import api as A
    assert torch.cuda.is_available()
    return A


def bf16_round(a: np.ndarray) -> np.ndarray:
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).bfloat16().float().numpy()


# (R, cin, cout, cr): every kernel variant (N tile 32..256, channel chunk 32 / 64,
# with and without the projection segment, several N tiles, rows of 16..256)
SHAPES = [(16, 32, 32, 32), (32, 64, 128, 0), (64, 64, 256, 0), (32, 256, 512, 0),
          (128, 32, 64, 32), (64, 128, 256, 128), (256, 96, 32, 96), (32, 768, 256, 768),
          (16, 512, 512, 256), (32, 32, 32, 0)]


@pytest.mark.parametrize("R,cin,cout,cr", SHAPES)
def test_conv_layer_bf16(api, R, cin, cout, cr):
    from paper_2305_14566_gb300 import _lib as L
    rng = np.random.default_rng(1000 + R + cin + cout + cr)
    B = 2
    x = bf16_round(np.abs(rng.standard_normal((B, R, R, cin))))
    w = bf16_round(rng.standard_normal((cout, cin, 3, 3)) * np.sqrt(2 / (9 * cin)))
    g = rng.uniform(0.9, 1.1, cout).astype(np.float32)
    b = rng.uniform(-0.05, 0.05, cout).astype(np.float32)
    r = bf16_round(np.abs(rng.standard_normal((B, R, R, cr)))) if cr else None
    wp = bf16_round(rng.standard_normal((cout, cr)) * np.sqrt(1 / cr)) if cr else None
    xd = torch.from_numpy(x).cuda().bfloat16()
    rd = torch.from_numpy(r).cuda().bfloat16() if cr else None
    y = torch.full((B, R, R, cout), float("nan"), dtype=torch.bfloat16, device="cuda")
    api.conv_layer(L.BF16, xd, R, cin, cout, w, g, b, y, rd, cr, wp)
    got = y.float().cpu().numpy()
    xt = torch.from_numpy(x.astype(np.float64)).permute(0, 3, 1, 2)
    z = O.affine(O.conv3x3(xt, torch.from_numpy(w.astype(np.float64))),
                 torch.from_numpy(g.astype(np.float64)), torch.from_numpy(b.astype(np.float64)))
    if cr:
        z = z + O.conv1x1(torch.from_numpy(r.astype(np.float64)).permute(0, 3, 1, 2),
                          torch.from_numpy(wp.astype(np.float64)))
    ref = O.relu(z).permute(0, 2, 3, 1).numpy()
    assert np.isfinite(got).all()
    err = np.abs(got - ref)
    bound = 2.0 ** -8 * np.abs(ref) + 1e-4 * np.sqrt(9 * cin + cr)
    assert (err <= bound).all(), (float(err.max()), float((err - bound).max()))


def _stats(gpu_lab, gpu_L, orc_lab, orc_L):
    agree = float((gpu_lab == orc_lab).mean())
    inter = float(((gpu_lab > 0) & (orc_lab > 0)).sum())
    den = float((gpu_lab > 0).sum() + (orc_lab > 0).sum())
    dice = 1.0 if den == 0 else 2 * inter / den
    d = np.abs(gpu_L - orc_L)
    return agree, dice, float(d.max()), float(np.percentile(d, 99)), int((orc_lab > 0).sum())


def test_bf16_whole_path_window_against_oracle(api):
    """The needle network (base 32, 5 levels, 3 scales, 6 heads) with 256 px
    tiles at stride 128 on a 2048 x 2048 slide with tissue filtering."""
    from paper_2305_14566_gb300 import _lib as L
    w = synth.NEEDLE.with_(H=2048, W=2048, P=256, S=128, median_k=5, max_batch=16)
    spec = synth.make_spec(2048, 2048, 41, 0.5, "cores", 3)
    rgb_np = synth.gen_slide(spec)
    blob = synth.gen_weights(w)
    seg = api.Segmenter(w, blob, precision=L.BF16)
    out = seg.segment(torch.from_numpy(rgb_np).cuda(), logits=True, coverage=True)
    torch.cuda.synchronize()
    orc = O.segment(rgb_np, w, blob, window=(640, 768, 512, 512), batch=8)
    rows = []
    for c, s in enumerate(w.class_scale):
        wy, wx, wh, ww = orc["window"][s]
        gl = out["labels"][c][wy:wy + wh, wx:wx + ww].cpu().numpy()
        gL = out["logits"][c][wy:wy + wh, wx:wx + ww].double().cpu().numpy()
        rows.append((c,) + _stats(gl, gL, orc["labels"][c], orc["L"][c]))
        cov = out["coverage"][s][wy:wy + wh, wx:wx + ww].cpu().numpy().astype(np.int64)
        assert np.array_equal(cov, orc["cov"][c])
    for row in rows:
        print("class %d agree %.5f dice %.5f max|dL| %.3e p99|dL| %.3e positives %d" % row)
    agree_all = np.mean([r[1] for r in rows])
    assert agree_all >= 0.999, rows
    for r in rows:
        if r[5] >= 2000:
            assert r[2] >= 0.995, r
    seg.close()
