"""Hand-written backward (omni_backward) against the FP64 oracle's gradient.

The oracle's gradient is torch autograd over its FP64 forward of the same
sub-chain; it is itself pinned by central finite differences in
tests/test_oracle_pins.py.  The bar is 1e-3 relative: for every gradient
tensor, max |g_gpu - g_oracle| <= 1e-3 * max |g_oracle|.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import omniseg_oracle as O

pytestmark = pytest.mark.gpu

NAME = {"ctrl.w": "ctrl_w", "ctrl.b": "ctrl_b", "head.w": "head_w", "head.b": "head_b",
        "dec0.w1": "dec0_w1", "dec0.g1": "dec0_g1", "dec0.b1": "dec0_b1", "dec0.w2": "dec0_w2",
        "dec0.g2": "dec0_g2", "dec0.b2": "dec0_b2", "dec0.wp": "dec0_wp"}


@pytest.fixture(scope="module")
def api():
    from paper_2305_14566_gb300.build import build
    build()
    from paper_2305_14566_gb300 import api as A
    assert torch.cuda.is_available()
    return A


def _run(api, w, batch):
    rgb_np = synth.gen_slide(synth.spec_for(w))
    gts = synth.gen_gt_masks(w.H, w.W, w.factors, w.class_scale, seed=7)
    blob = synth.gen_weights(w)
    seg = api.Segmenter(w, blob, max_batch=batch)
    loss, grads = seg.backward(torch.from_numpy(rgb_np).cuda(), [torch.from_numpy(g).cuda() for g in gts])
    loss2, grads2 = seg.backward(torch.from_numpy(rgb_np).cuda(), [torch.from_numpy(g).cuda() for g in gts])
    torch.cuda.synchronize()
    # deterministic: a second call gives identical bits
    assert torch.equal(loss, loss2)
    for k in grads:
        assert torch.equal(grads[k], grads2[k]), k
    prob = O.DiffProblem(rgb_np, w, blob, gts)
    ol, og = prob.loss_and_grads()
    seg.close()
    return float(loss), {k: v.double().cpu().numpy() for k, v in grads.items()}, ol, og


def _compare(gl, gg, ol, og):
    assert abs(gl - ol) <= 1e-5 * abs(ol), (gl, ol)
    for name, ref in og.items():
        ref = ref.numpy()
        got = gg[NAME[name]]
        assert got.shape == ref.shape, name
        err = np.abs(got - ref).max()
        scale = np.abs(ref).max()
        print("%-8s max|g| %.3e max err %.3e rel %.2e" % (name, scale, err, err / max(scale, 1e-30)))
        assert err <= 1e-3 * scale, name


def test_backward_small_network_matches_oracle(api):
    """The differentiation workload's slide, scales and tiling (2048^2, 256 px
    tiles at stride 128, 235 tiles, 6 classes) with a narrow U-Net."""
    w = synth.DIFF.with_(base=8, levels=3)
    _compare(*_run(api, w, 16))


def test_backward_diff_workload_matches_oracle(api):
    """The differentiation workload itself (base 32, 5 levels)."""
    _compare(*_run(api, synth.DIFF, 32))
