"""Hand-written backward (omni_backward) against the FP64 oracle's gradient.

The oracle's gradient is torch autograd over its FP64 forward of the same
sub-chain; it is itself pinned by central finite differences in
tests/test_oracle_pins.py.  The bar is 1e-3 relative: for every gradient
tensor, max |g_gpu - g_oracle| <= 1e-3 * max |g_oracle|.
"""
import json
import os

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
    """The differentiation workload itself (base 32, 5 levels): every gradient
    tensor against the oracle's autograd gradient (max-norm relative 1e-3), and
    entry by entry against FP64 central differences at 64 seeded parameters
    (tests/golden/diff_fd.json): |g - fd| <= 1e-3 max(|fd|, 1e-3 max|g_tensor|),
    the floor covering entries far below their tensor's largest, where FP32
    accumulation order dominates."""
    gl, gg, ol, og = _run(api, synth.DIFF, 32)
    _compare(gl, gg, ol, og)
    fdg = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "diff_fd.json")))
    worst = 0.0
    for d in fdg["draws"]:
        got = float(gg[NAME[d["name"]]][tuple(d["index"])])
        scale = max(abs(d["fd"]), 1e-3 * d["tensor_max_abs_grad"])
        worst = max(worst, abs(got - d["fd"]) / scale)
        assert abs(got - d["fd"]) <= 1e-3 * scale, (d, got)
    print("64 FD entries: worst relative error %.2e" % worst)


def test_omniseg_loss_autograd_matches_backward_and_tracks_params(api):
    """OmniSegLoss through torch.autograd: p.grad equals omni_backward's
    gradients; after a parameter update the next forward uses the updated
    values (the oracle's loss and gradient at those values); a wrongly shaped
    parameter is refused."""
    from paper_2305_14566_gb300 import _lib as L
    w = synth.DIFF.with_(base=8, levels=3)
    rgb_np = synth.gen_slide(synth.spec_for(w))
    gts_np = synth.gen_gt_masks(w.H, w.W, w.factors, w.class_scale, seed=7)
    blob = synth.gen_weights(w)
    rgb = torch.from_numpy(rgb_np).cuda()
    gts = [torch.from_numpy(g).cuda() for g in gts_np]
    seg = api.Segmenter(w, blob, max_batch=16)
    offs = seg.grad_offsets()
    shapes = seg.grad_shapes()
    params = [torch.from_numpy(blob[offs[k]:offs[k] + int(np.prod(shapes[k]))].reshape(shapes[k]).copy())
              .cuda().requires_grad_(True) for k in L.GRAD_FIELDS]
    loss = api.OmniSegLoss.apply(seg, rgb, gts, *params)
    loss.backward()
    _, ref = seg.backward(rgb, gts)
    torch.cuda.synchronize()
    for k, p in zip(L.GRAD_FIELDS, params):
        assert torch.equal(p.grad, ref[k]), k
    # one SGD step on three bias vectors; loss and gradients must follow the new values
    with torch.no_grad():
        for k, p in zip(L.GRAD_FIELDS, params):
            if k in ("ctrl_b", "head_b", "dec0_b2"):
                p -= 0.5 * p.grad
            p.grad = None
    loss2 = api.OmniSegLoss.apply(seg, rgb, gts, *params)
    loss2.backward()
    torch.cuda.synchronize()
    blob2 = blob.copy()
    for k, p in zip(L.GRAD_FIELDS, params):
        blob2[offs[k]:offs[k] + p.numel()] = p.detach().cpu().numpy().ravel()
    assert np.array_equal(seg.blob, blob2)
    prob = O.DiffProblem(rgb_np, w, blob2, gts_np)
    ol, og = prob.loss_and_grads()
    assert abs(float(loss2) - ol) <= 1e-5 * abs(ol), (float(loss2), ol)
    assert float(loss2) != float(loss)
    for name, ref_g in og.items():
        got = params[L.GRAD_FIELDS.index(NAME[name])].grad.double().cpu().numpy()
        ref_g = ref_g.numpy()
        assert np.abs(got - ref_g).max() <= 1e-3 * np.abs(ref_g).max(), name
    bad = list(params)
    bad[0] = torch.zeros(3, 3, device="cuda")
    with pytest.raises(ValueError):
        api.OmniSegLoss.apply(seg, rgb, gts, *bad)
    seg.close()


def test_finetuning_loop_lowers_the_stitched_loss(api):
    """A fine-tuning loop over the differentiated sub-chain (controller,
    pre-head, last decoder block): torch.optim.Adam on the OmniSegLoss
    parameters, one forward + backward + step per iteration on the
    differentiation workload's slide and masks.  The stitched soft-Dice + BCE
    loss falls over the iterations, and the last value equals the oracle's
    loss at the updated weights."""
    from paper_2305_14566_gb300 import _lib as L
    w = synth.DIFF.with_(base=8, levels=3)
    rgb_np = synth.gen_slide(synth.spec_for(w))
    gts_np = synth.gen_gt_masks(w.H, w.W, w.factors, w.class_scale, seed=7)
    blob = synth.gen_weights(w)
    rgb = torch.from_numpy(rgb_np).cuda()
    gts = [torch.from_numpy(g).cuda() for g in gts_np]
    seg = api.Segmenter(w, blob, max_batch=16)
    offs, shapes = seg.grad_offsets(), seg.grad_shapes()
    params = [torch.from_numpy(blob[offs[k]:offs[k] + int(np.prod(shapes[k]))].reshape(shapes[k]).copy())
              .cuda().requires_grad_(True) for k in L.GRAD_FIELDS]
    opt = torch.optim.Adam(params, lr=1e-3)
    losses = []
    for it in range(8):
        opt.zero_grad()
        loss = api.OmniSegLoss.apply(seg, rgb, gts, *params)
        loss.backward()
        opt.step()
        losses.append(float(loss))
    final = float(api.OmniSegLoss.apply(seg, rgb, gts, *params))
    torch.cuda.synchronize()
    print("fine-tuning losses", ["%.5f" % v for v in losses], "final %.5f" % final)
    assert final < losses[0] and losses[-1] < losses[0], losses
    blob2 = blob.copy()
    for k, p in zip(L.GRAD_FIELDS, params):
        blob2[offs[k]:offs[k] + p.numel()] = p.detach().cpu().numpy().ravel()
    ol = float(O.DiffProblem(rgb_np, w, blob2, gts_np).loss({}))
    assert abs(final - ol) <= 1e-5 * abs(ol), (final, ol)
    seg.close()
