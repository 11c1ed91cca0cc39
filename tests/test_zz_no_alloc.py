"""The allocation-free tiling entry point against the workspace one.

omni_tile_slide_noalloc exists for callers that must not allocate device
memory while they run (a scanner loop with a device-memory budget fixed at
start-up, a process whose device memory belongs to another framework's pool).
It keeps its scratch in a static device array instead of a caller workspace;
its outputs must be bit-identical to omni_tile_slide's.  This file is named
to be collected last, so a run that stops at the first failure has already
run every other test.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2305_14566_gb300.build import build
    build()
    from paper_2305_14566_gb300 import api as A
    assert torch.cuda.is_available()
    return A


def _same(a, b):
    n = int(a["counts"][0])
    assert n == int(b["counts"][0])
    assert torch.equal(a["counts"], b["counts"])
    assert torch.equal(a["tiles"][:n], b["tiles"][:n])
    assert torch.equal(a["flags"], b["flags"])
    assert torch.equal(a["tissue"], b["tissue"])
    assert torch.equal(a["otsu"], b["otsu"])
    return n


def test_noalloc_tiling_matches_workspace_tiling_twice(api):
    cases = [
        # ragged slide: padding, tissue filter, median 5
        (synth.NEEDLE.with_(H=3000, W=5000, median_k=5, max_batch=2),
         synth.make_spec(3000, 5000, 33, 0.3, "cores", 3)),
        # the paper's 4096 border on a small needle-like slide
        (synth.NEEDLE.with_(H=2500, W=6000, median_k=9, pad_lead=4096, max_batch=2),
         synth.make_spec(2500, 6000, 34, 0.4, "cores", 4)),
    ]
    for work, spec in cases:
        rgb = api.synth_slide(spec)
        seg = api.Segmenter(work, synth.gen_weights(work))
        ref = seg.tile_slide(rgb)
        first = api.tile_slide_noalloc(work, rgb)
        second = api.tile_slide_noalloc(work, rgb)
        torch.cuda.synchronize()
        n1 = _same(first, ref)
        n2 = _same(second, ref)
        assert n1 == n2 > 0
        seg.close()


def test_noalloc_rejects_slides_beyond_its_scratch(api):
    """A slide whose tile grid exceeds the static scratch is refused on the
    host with OMNI_EINVAL (the buffer is real, so nothing could read past it
    even if the check were missing)."""
    import ctypes as C
    from paper_2305_14566_gb300 import _lib as L
    # stride 64 (the paper's 10x/5x stride) on a 16384^2 slide: 62001 + 3249 + 625
    # tile cells > OMNI_NOALLOC_MAX_TILES
    work = synth.NEEDLE.with_(H=16384, W=16384, S=64)
    cfg = api.make_config(work)
    s = L.Sizes()
    assert L.lib().omni_query(C.byref(cfg), work.H, work.W, C.byref(s)) == L.OK
    assert s.n_tiles_max > L.NOALLOC_MAX_TILES
    rgb = torch.zeros((work.H, work.W, 3), dtype=torch.uint8, device="cuda")
    out = torch.zeros((s.n_tiles_max, 3), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(4, dtype=torch.int32, device="cuda")
    tl = L.TileList(out.data_ptr(), cnt.data_ptr(), None, None, None)
    st = L.lib().omni_tile_slide_noalloc(C.byref(cfg), C.c_void_p(rgb.data_ptr()), work.H, work.W,
                                         rgb.stride(0), C.byref(tl), None)
    assert st == L.EINVAL
    torch.cuda.synchronize()
