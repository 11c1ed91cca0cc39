"""Several slides per call (omni_segment_slides): the foreground tiles of all
slides share network batches per scale; every slide's labels and logits must
equal its own omni_segment_slide call bit for bit, eagerly and through a
captured, replayed CUDA graph."""
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


# ragged sizes: padded right/bottom, different grids per slide, one slide
# smaller than the coarsest scale's tile footprint
SIZES = [(2048, 3000, 61), (1500, 2048, 62), (1024, 4096, 63), (2048, 2048, 64), (700, 900, 65)]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_slides_share_batches_and_match_single_calls(api, prec):
    from paper_2305_14566_gb300 import _lib as L
    w = synth.NEEDLE.with_(P=256, S=128, median_k=5, max_batch=16)
    precision = L.FP32 if prec == "fp32" else L.BF16
    rgbs = [api.synth_slide(synth.make_spec(h, wd, sd, 0.5, "cores", 3)) for (h, wd, sd) in SIZES]
    blob = synth.gen_weights(w)
    seg = api.Segmenter(w, blob, precision=precision)
    singles = []
    for r in rgbs:
        o = seg.segment(r, logits=True)
        singles.append({k: {c: t.clone() for c, t in d.items()} for k, d in o.items() if k in ("labels", "logits")})
    torch.cuda.synchronize()
    assert sum(int(t.sum()) for o in singles for t in o["labels"].values()) > 0
    seg.set_graphs(True)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    outs = None
    for call in range(3):                # eager, capture + launch, replay
        with torch.cuda.stream(stream):
            outs = seg.segment_many(rgbs, outs=outs, logits=True)
        torch.cuda.synchronize()
        for i, (o, ref) in enumerate(zip(outs, singles)):
            for c in ref["labels"]:
                assert torch.equal(o["labels"][c], ref["labels"][c]), (call, i, c)
                assert torch.equal(o["logits"][c], ref["logits"][c]), (call, i, c)
        times = seg.slide_times()
        assert len(times) == len(rgbs) and all(t > 0 for t in times), times
    seg.close()
