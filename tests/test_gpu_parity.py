"""GPU path (through the C ABI) against the FP64 oracle.

Integer stages (generator, pyramid-derived tile lists, Otsu, tissue mask) are
compared bit for bit; the FP32 network path within 1e-4 absolute on the
stitched logits, with labels allowed to differ only where the oracle's
|logit| < 1e-3.
"""
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


def _check_window(gpu, orc, work, window_by_scale):
    """Compare GPU full-slide outputs with an oracle window result."""
    worst = 0.0
    for c, s in enumerate(work.class_scale):
        if c not in orc["L"]:
            continue
        wy, wx, wh, ww = orc["window"][s]
        g = gpu["logits"][c][wy:wy + wh, wx:wx + ww].double().cpu().numpy()
        o = orc["L"][c]
        d = np.abs(g - o)
        worst = max(worst, float(d.max()))
        assert d.max() <= LOGIT_TOL, (c, float(d.max()))
        gl = gpu["labels"][c][wy:wy + wh, wx:wx + ww].cpu().numpy()
        bad = gl != orc["labels"][c]
        assert not (bad & (np.abs(o) >= LABEL_BAND)).any(), c
        if s in gpu["coverage"]:
            cov = gpu["coverage"][s][wy:wy + wh, wx:wx + ww].cpu().numpy().astype(np.int64)
            assert np.array_equal(cov, orc["cov"][c])
    return worst


# ---------------------------------------------------------------- generator


def test_synth_generator_bit_exact(api):
    spec = synth.spec_for(synth.TINY)
    g = api.synth_slide(spec).cpu().numpy()
    assert np.array_equal(g, synth.gen_slide(spec))
    spec = synth.spec_for(synth.NEEDLE)
    assert spec.structures
    for (y0, x0, h, w) in ((0, 0, 64, 96), (5000, 20000, 300, 257), (5632, 24576, 1024, 1536),
                           (16384 - 37, 49152 - 53, 37, 53)):
        g = api.synth_slide(spec, y0, x0, h, w).cpu().numpy()
        assert np.array_equal(g, synth.gen_window(spec, y0, x0, h, w)), (y0, x0)


# ---------------------------------------------------------------- tiling (Sec. 2.1)


def _tile_compare(api, work, rgb_np):
    seg = api.Segmenter(work, synth.gen_weights(work))
    rgb = torch.from_numpy(rgb_np).cuda()
    t = seg.tile_slide(rgb)
    torch.cuda.synchronize()
    prep = O.prepare(rgb_np, work)
    n = int(t["counts"][0])
    got = [tuple(x) for x in t["tiles"][:n].cpu().numpy().tolist()]
    assert got == prep["tiles"]
    per = [sum(1 for q in prep["tiles"] if q[0] == s) for s in range(work.n_scales)]
    assert t["counts"][1:].cpu().numpy().tolist() == per
    assert int(t["otsu"][0]) == prep["otsu"]
    assert np.array_equal(t["tissue"].cpu().numpy().astype(bool), prep["mask"])
    flags = np.concatenate([f.ravel() for f in prep["flags"]])
    assert np.array_equal(t["flags"].cpu().numpy()[:flags.size].astype(bool), flags)
    seg.close()
    return prep


def test_tile_slide_tiny(api):
    w = synth.TINY
    _tile_compare(api, w, synth.gen_slide(synth.spec_for(w)))


def test_tile_slide_ragged_with_filter_and_padding(api):
    w = synth.NEEDLE.with_(H=3000, W=5000, median_k=5, max_batch=2)
    spec = synth.make_spec(3000, 5000, 33, 0.3, "cores", 3)
    prep = _tile_compare(api, w, synth.gen_slide(spec))
    assert 0 < len(prep["tiles"]) < sum(int(np.prod(f.shape)) for f in prep["flags"])


def _specks_slide():
    """Glass with one large dark tissue region and small dark specks of 2 x 2
    to 6 x 6 thumbnail cells (64..192 px at 40x), some touching diagonally."""
    rng = np.random.default_rng(9)
    rgb = np.full((3072, 4096, 3), 232, np.uint8)
    rgb += rng.integers(0, 12, rgb.shape, dtype=np.uint8)
    rgb[640:2432, 512:2560] = (150, 80, 140)                       # the biopsy core
    for k, (cy, cx, r) in enumerate([(300, 3000, 2), (900, 3300, 3), (2000, 3500, 4), (2700, 3000, 6),
                                     (2800, 300, 3), (200, 200, 2)]):
        rgb[cy:cy + 32 * r, cx:cx + 32 * r] = (140, 70, 130)
    rgb[1500:1564, 3700:3764] = (140, 70, 130)                     # two 2 x 2 specks touching at a corner
    rgb[1564:1628, 3764:3828] = (140, 70, 130)
    return rgb


@pytest.mark.parametrize("min_area", [0, 5, 12, 30])
def test_tile_slide_area_filter_matches_oracle(api, min_area):
    """Sec. 2.1 contour step: 8-connected tissue regions of the thumbnail mask
    under min_area pixels are removed before tiling; mask, flags and tile list
    bit-exact against the oracle, with specks on both sides of each area."""
    w = synth.NEEDLE.with_(H=3072, W=4096, median_k=3, max_batch=2, min_tissue_area=min_area)
    prep = _tile_compare(api, w, _specks_slide())
    base = O.prepare(_specks_slide(), w.with_(min_tissue_area=0))
    if min_area:
        assert prep["mask"].sum() < base["mask"].sum()
    else:
        assert np.array_equal(prep["mask"], base["mask"])


def test_tile_slide_constant_slide_has_no_tiles(api):
    w = synth.NEEDLE.with_(H=2048, W=2048, median_k=3, max_batch=2)
    rgb = np.full((2048, 2048, 3), 235, np.uint8)
    prep = _tile_compare(api, w, rgb)
    assert prep["tiles"] == [] and prep["otsu"] == -1


def test_tile_slide_needle_full_size(api):
    """Full 16384 x 49152 needle slide generated on the device; the oracle's
    thumbnail is evaluated band by band (it is a per-32x32-block definition)."""
    w = synth.NEEDLE
    spec = synth.spec_for(w)
    rgb = api.synth_slide(spec)
    seg = api.Segmenter(w, synth.gen_weights(w))
    t = seg.tile_slide(rgb)
    host = rgb.cpu().numpy()
    del rgb
    thumb = np.concatenate([O.thumbnail(host[y:y + 1024]) for y in range(0, w.H, 1024)], 0)
    g = O.grey(thumb)
    b = O.median_blur(g, w.median_k)
    thr = O.otsu(O.histogram(b))
    mask = b.astype(np.int64) <= thr
    tiles, flags = O.tile_list(w, mask, w.H, w.W)
    assert int(t["otsu"][0]) == thr
    assert np.array_equal(t["tissue"].cpu().numpy().astype(bool), mask)
    n = int(t["counts"][0])
    assert n == len(tiles) and 0.2 < n / 12899 < 0.9
    assert [tuple(x) for x in t["tiles"][:n].cpu().numpy().tolist()] == tiles
    seg.close()


# ---------------------------------------------------------------- one fused conv layer


@pytest.mark.parametrize("R,cin,cout,cr", [(16, 16, 32, 8), (32, 24, 8, 24), (8, 64, 64, 0)])
def test_conv_layer_fp32(api, R, cin, cout, cr):
    from paper_2305_14566_gb300 import _lib as L
    rng = np.random.default_rng(R + cin)
    B = 3
    x = rng.standard_normal((B, R, R, cin)).astype(np.float32)
    w = (rng.standard_normal((cout, cin, 3, 3)) * np.sqrt(2 / (9 * cin))).astype(np.float32)
    g = rng.uniform(0.9, 1.1, cout).astype(np.float32)
    b = rng.uniform(-0.05, 0.05, cout).astype(np.float32)
    r = rng.standard_normal((B, R, R, cr)).astype(np.float32) if cr else None
    wp = (rng.standard_normal((cout, cr)) * np.sqrt(2 / cr)).astype(np.float32) if cr else None
    y = torch.zeros((B, R, R, cout), dtype=torch.float32, device="cuda")
    api.conv_layer(L.FP32, torch.from_numpy(x).cuda(), R, cin, cout, w, g, b, y,
                   None if r is None else torch.from_numpy(r).cuda(), cr, wp)
    xt = torch.from_numpy(x.astype(np.float64)).permute(0, 3, 1, 2)
    z = O.affine(O.conv3x3(xt, torch.from_numpy(w.astype(np.float64))),
                 torch.from_numpy(g.astype(np.float64)), torch.from_numpy(b.astype(np.float64)))
    if cr:
        z = z + O.conv1x1(torch.from_numpy(r.astype(np.float64)).permute(0, 3, 1, 2),
                          torch.from_numpy(wp.astype(np.float64)))
    ref = O.relu(z).permute(0, 2, 3, 1).numpy()
    assert np.abs(y.cpu().numpy() - ref).max() < 2e-5


# ---------------------------------------------------------------- whole path, FP32


def test_tiny_fp32_end_to_end(api):
    w = synth.TINY
    rgb_np = synth.gen_slide(synth.spec_for(w))
    blob = synth.gen_weights(w)
    seg = api.Segmenter(w, blob)
    out = seg.segment(torch.from_numpy(rgb_np).cuda(), logits=True, coverage=True, argmax=True)
    torch.cuda.synchronize()
    orc = O.segment(rgb_np, w, blob, batch=16)
    worst = _check_window(out, orc, w, None)
    assert worst < LOGIT_TOL
    am = O.argmax_map([orc["L"][0], orc["L"][1]], [0, 1])
    ga = out["argmax"][0].cpu().numpy()
    close = np.abs(orc["L"][0] - orc["L"][1]) < LABEL_BAND
    near0 = np.maximum(orc["L"][0], orc["L"][1]) < LABEL_BAND
    assert not ((ga != am) & ~close & ~near0).any()
    assert seg.launch_count() > 0
    seg.close()


def test_needle_network_small_tiles_fp32_window(api):
    """The needle network (base 32, 5 levels, 3 scales, 6 heads) with 128 px
    tiles on a ragged slide with tissue filtering, padding and tissue AND."""
    w = synth.NEEDLE.with_(H=700, W=1400, P=128, S=64, median_k=5, max_batch=8)
    spec = synth.make_spec(700, 1400, 21, 0.45, "cores", 3)
    rgb_np = synth.gen_slide(spec)
    blob = synth.gen_weights(w)
    seg = api.Segmenter(w, blob)
    out = seg.segment(torch.from_numpy(rgb_np).cuda(), logits=True, coverage=True)
    torch.cuda.synchronize()
    orc = O.segment(rgb_np, w, blob, window=(256, 512, 256, 256), batch=8)
    _check_window(out, orc, w, None)
    # the window holds tissue and processed tiles at every scale
    assert orc["prep"]["mask"][8:16, 16:24].any()
    assert all(orc["cov"][c].max() > 0 for c in orc["cov"])
    seg.close()


def test_needle_network_unpadded_slide_fp32_window(api):
    """A slide whose size already sits on the tile grid: the 40x canvas is the
    caller's buffer and the 10x / 5x canvases are the first workspace regions."""
    w = synth.NEEDLE.with_(H=1024, W=1536, P=128, S=64, median_k=5, max_batch=8)
    spec = synth.make_spec(1024, 1536, 22, 0.45, "cores", 3)
    rgb_np = synth.gen_slide(spec)
    blob = synth.gen_weights(w)
    seg = api.Segmenter(w, blob)
    assert seg.query(1024, 1536).Hp == 1024
    out = seg.segment(torch.from_numpy(rgb_np).cuda(), logits=True, coverage=True)
    torch.cuda.synchronize()
    orc = O.segment(rgb_np, w, blob, window=(512, 768, 256, 256), batch=8)
    _check_window(out, orc, w, None)
    seg.close()


def test_host_buffers_match_device_path(api):
    w = synth.TINY
    rgb_np = synth.gen_slide(synth.spec_for(w))
    seg = api.Segmenter(w, synth.gen_weights(w))
    dev = seg.segment(torch.from_numpy(rgb_np).cuda())
    hosts = {c: torch.zeros((512, 512), dtype=torch.uint8).pin_memory() for c in range(2)}
    seg.segment_host(torch.from_numpy(rgb_np).pin_memory(), hosts)
    for c in range(2):
        assert torch.equal(hosts[c], dev["labels"][c].cpu())
    seg.close()


def test_host_buffers_banded_downloads_with_graphs(api):
    """Host-buffer path on a three-scale slide with many stitch bands and
    batches: labels downloaded band by band on the context's copy stream equal
    the device path's, eagerly and through a captured, replayed CUDA graph."""
    from paper_2305_14566_gb300 import _lib as L
    w = synth.NEEDLE.with_(H=2048, W=4096, P=256, S=128, median_k=5, max_batch=16)
    spec = synth.make_spec(2048, 4096, 51, 0.5, "cores", 3)
    rgb_np = synth.gen_slide(spec)
    seg = api.Segmenter(w, synth.gen_weights(w), precision=L.BF16)
    dev = seg.segment(torch.from_numpy(rgb_np).cuda())
    torch.cuda.synchronize()
    dev = {c: t.cpu() for c, t in dev["labels"].items()}
    assert sum(int(t.sum()) for t in dev.values()) > 0
    rgb_h = torch.from_numpy(rgb_np).pin_memory()
    seg.set_graphs(True)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    hosts = {c: torch.empty(tuple(t.shape), dtype=torch.uint8).pin_memory() for c, t in dev.items()}
    for call in range(3):                 # eager, capture + launch, replay (same buffers: same key)
        for t in hosts.values():
            t.fill_(7)
        with torch.cuda.stream(stream):
            seg.segment_host(rgb_h, hosts)
        for c in dev:
            assert torch.equal(hosts[c], dev[c]), (call, c)
    seg.close()
