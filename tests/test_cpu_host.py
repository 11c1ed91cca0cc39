"""Host-side checks that need no GPU: the C ABI library loads and exports every
declared entry point, configuration validation, sizes and FLOP counts."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import synth
from oracle import omniseg_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2305_14566_gb300 import _lib
    from paper_2305_14566_gb300.build import build
    build()
    _lib.lib()
    return _lib


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "omniseg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(omni_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(L):
    syms = declared_symbols()
    assert "omni_segment_slide" in syms and "omni_tile_slide" in syms
    lib = C.CDLL(L.LIB_PATH)
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing
    assert set(L.EXPORTS) <= set(syms)


def _cfg(L, work, **kw):
    from paper_2305_14566_gb300.api import make_config
    c = make_config(work)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def test_weights_count_matches_blob_layout(L):
    for w in (synth.TINY, synth.NEEDLE, synth.DIFF):
        c = _cfg(L, w)
        assert L.lib().omni_weights_count(C.byref(c)) == synth.n_params(w)
        assert synth.gen_weights(w).size == synth.n_params(w)


@pytest.mark.parametrize("field,value", [("levels", 1), ("base", 12), ("stride", 100),
                                         ("median_k", 4), ("max_batch", 0), ("pad_lead", 3),
                                         ("n_classes", 17), ("stitch_window", 3),
                                         ("stitch_window", -1)])
def test_invalid_configs_rejected_without_device(L, field, value):
    c = _cfg(L, synth.NEEDLE, **{field: value})
    ctx = C.c_void_p()
    assert L.lib().omni_create(C.byref(c), C.byref(ctx)) == L.EINVAL
    assert not ctx.value
    s = L.Sizes()
    assert L.lib().omni_query(C.byref(c), 1000, 1000, C.byref(s)) == L.EINVAL


@pytest.mark.parametrize("s,value", [(1, 100), (0, 16), (2, -64), (1, 1024)])
def test_bad_scale_strides_rejected(L, s, value):
    """A per-scale stride must divide P (512), be a multiple of 4, and put tile
    borders on 32-pixel thumbnail cells (16 at 40x does not)."""
    c = _cfg(L, synth.NEEDLE_PAPER)
    c.scale_stride[s] = value
    sz = L.Sizes()
    assert L.lib().omni_query(C.byref(c), 1000, 1000, C.byref(sz)) == L.EINVAL


def test_bad_factors_rejected(L):
    c = _cfg(L, synth.NEEDLE)
    c.factors[1] = 3
    s = L.Sizes()
    assert L.lib().omni_query(C.byref(c), 1000, 1000, C.byref(s)) == L.EINVAL
    c = _cfg(L, synth.NEEDLE)
    c.class_scale[0] = 5
    assert L.lib().omni_query(C.byref(c), 1000, 1000, C.byref(s)) == L.EINVAL


@pytest.mark.parametrize("work,H,W", [(synth.TINY, 512, 512), (synth.NEEDLE, 16384, 49152),
                                      (synth.DIFF, 2048, 2048), (synth.LARGE, 32768, 98304),
                                      (synth.NEEDLE, 5000, 9000), (synth.NEEDLE, 300, 700),
                                      (synth.NEEDLE_PAPER, 16384, 49152),
                                      (synth.NEEDLE_PAPER, 5000, 9000)])
def test_query_sizes_match_oracle(L, work, H, W):
    c = _cfg(L, work)
    s = L.Sizes()
    assert L.lib().omni_query(C.byref(c), H, W, C.byref(s)) == L.OK
    Hp, Wp, lead = O.padded_dims(work, H, W)
    assert (s.Hp, s.Wp) == (Hp, Wp)
    assert (s.thumb_h, s.thumb_w) == (Hp // 32, Wp // 32)
    for k, f in enumerate(work.factors):
        assert (s.grid_h[k], s.grid_w[k]) == O.grid(work, Hp, Wp, k)
        assert (s.out_h[k], s.out_w[k]) == (-(-H // f), -(-W // f))
    assert s.n_tiles_max == sum(int(np.prod(O.grid(work, Hp, Wp, k)))
                                for k in range(work.n_scales))
    assert s.workspace_bytes >= s.tile_workspace_bytes > 0


def test_flops_per_tile_needle():
    """119.15 GFLOP of convolution per 512x512 tile of the base-32, 5-level U-Net."""
    from paper_2305_14566_gb300 import _lib as L
    c = _cfg(L, synth.NEEDLE)
    s = L.Sizes()
    assert L.lib().omni_query(C.byref(c), 16384, 49152, C.byref(s)) == 0
    # independent count from the weight shapes: 2 * R^2 * (#weights of each conv)
    lay = synth.layout(synth.NEEDLE)
    fl = 0
    for name, shape in lay.items():
        if name.split(".")[1] in ("w1", "w2", "wp") and name[:3] in ("enc", "dec"):
            l = int(name[3])
            R = 512 >> l
            fl += 2 * R * R * int(np.prod(shape))
    assert s.flops_per_tile == fl
    assert abs(fl / 1e9 - 119.15) < 0.05


def test_workload_padding_matches_config_sizes():
    assert O.padded_dims(synth.TINY)[:2] == (512, 512)
    assert O.padded_dims(synth.DIFF)[:2] == (2048, 2048)


@pytest.mark.parametrize("case", ["down", "factor", "alpha", "no_output", "stride", "n_maps"])
def test_stain_rejects_bad_arguments_without_device(L, case):
    """omni_stain checks sizes, factors, alphas, resize factor and strides on
    the host and returns OMNI_EINVAL before touching the device (the
    pointers below are never dereferenced)."""
    fake = C.c_void_p(0x1000)
    maps = (C.c_void_p * 1)(fake)
    fac = np.array([1], np.int32)
    col = np.array([1, 2, 3], np.uint8)
    alp = np.array([128], np.int32)
    args = dict(H=64, W=64, rs=192, n=1, fac=fac, alp=alp, out40=fake, os=192, down=4, outd=fake, ds=48)
    if case == "down":
        args["down"] = 3
    elif case == "factor":
        args["fac"] = np.array([3], np.int32)
    elif case == "alpha":
        args["alp"] = np.array([257], np.int32)
    elif case == "no_output":
        args["out40"] = None
        args["outd"] = None
    elif case == "stride":
        args["rs"] = 100
    elif case == "n_maps":
        args["n"] = 17
    st = L.lib().omni_stain(fake, args["H"], args["W"], args["rs"], args["n"], maps,
                            args["fac"].ctypes.data_as(C.c_void_p), col.ctypes.data_as(C.c_void_p),
                            args["alp"].ctypes.data_as(C.c_void_p), args["out40"], args["os"],
                            args["down"], args["outd"], args["ds"], None)
    assert st == L.EINVAL


def test_head_calibration_rule_picks_the_emptiest_band():
    """The needle heads' calibration rule (tests/golden/make_head_offsets.py):
    on a two-mode response it places the threshold in the empty gap between
    the modes (no response within 0.05 of it, half the pixels positive); on
    one Gaussian mode it moves to the low tail, the candidate range's end
    (99% positive), where the fewest responses crowd the threshold."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_head_offsets", os.path.join(os.path.dirname(__file__), "golden", "make_head_offsets.py"))
    M = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(M)
    rng = np.random.default_rng(3)
    two = np.concatenate([rng.normal(-2.0, 0.3, 20000), rng.normal(2.0, 0.3, 20000)])
    t, near, pos = M.least_crowded(two)
    assert -0.8 < t < 0.8 and near == 0.0 and abs(pos - 0.5) < 1e-3, (t, near, pos)
    one = rng.normal(-4.0, 1.0, 40000)
    t, near, pos = M.least_crowded(one)
    assert abs(pos - 0.99) < 2e-3 and t < -6.0, (t, near, pos)
