"""ctypes binding of libomniseg.so (argument marshalling only).

Every function here forwards to the C entry point of the same name declared
in include/omniseg.h.  Loading fails loudly when the library has not been
built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

MAX_SCALES = 4
MAX_CLASSES = 16
MAX_SLIDES = 16

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EWEIGHTS, ESTATE = 0, -1, -2, -3, -4, -5, -6
FP32, BF16, FP16 = 0, 1, 2
E4M3 = 3          # omni_conv_layer only: the 8-bit experiment
STITCH_AVG, STITCH_VOTE = 0, 1
NOALLOC_MAX_THUMB_PX = 4 << 20
NOALLOC_MAX_TILES = 1 << 16

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libomniseg.so")

EXPORTS = ("omni_create", "omni_destroy", "omni_last_error", "omni_weights_count",
           "omni_load_weights", "omni_query", "omni_tile_slide", "omni_segment_slide",
           "omni_segment_slide_host", "omni_synth_slide", "omni_conv_layer", "omni_set_timing",
           "omni_get_timing", "omni_last_launch_count", "omni_get_launch_times",
           "omni_tile_slide_noalloc", "omni_backward", "omni_backward_workspace",
           "omni_set_autotune", "omni_set_e4m3", "omni_set_graphs", "omni_set_fusion", "omni_get_tuned",
           "omni_stain", "omni_query_slides", "omni_segment_slides", "omni_conv_candidates", "omni_set_conv_kind")


class Config(C.Structure):
    _fields_ = [("patch", C.c_int32), ("stride", C.c_int32), ("levels", C.c_int32),
                ("base", C.c_int32), ("n_scales", C.c_int32),
                ("factors", C.c_int32 * MAX_SCALES), ("n_classes", C.c_int32),
                ("class_scale", C.c_int32 * MAX_CLASSES), ("precision", C.c_int32),
                ("stitch_mode", C.c_int32), ("tissue_filter", C.c_int32),
                ("tissue_and", C.c_int32), ("pad_lead", C.c_int32), ("median_k", C.c_int32),
                ("max_batch", C.c_int32), ("scale_stride", C.c_int32 * MAX_SCALES),
                ("stitch_window", C.c_int32), ("min_tissue_area", C.c_int32)]


class Sizes(C.Structure):
    _fields_ = [("Hp", C.c_int32), ("Wp", C.c_int32), ("thumb_h", C.c_int32),
                ("thumb_w", C.c_int32), ("grid_h", C.c_int32 * MAX_SCALES),
                ("grid_w", C.c_int32 * MAX_SCALES), ("n_tiles_max", C.c_int32),
                ("out_h", C.c_int32 * MAX_SCALES), ("out_w", C.c_int32 * MAX_SCALES),
                ("tile_workspace_bytes", C.c_uint64), ("workspace_bytes", C.c_uint64),
                ("flops_per_tile", C.c_uint64)]


class TileList(C.Structure):
    _fields_ = [("tiles", C.c_void_p), ("counts", C.c_void_p), ("flags", C.c_void_p),
                ("tissue", C.c_void_p), ("otsu", C.c_void_p)]


GRAD_FIELDS = ("ctrl_w", "ctrl_b", "head_w", "head_b", "dec0_w1", "dec0_g1", "dec0_b1", "dec0_w2",
               "dec0_g2", "dec0_b2", "dec0_wp")


class Grads(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in GRAD_FIELDS]


class Outputs(C.Structure):
    _fields_ = [("labels", C.c_void_p * MAX_CLASSES), ("logits", C.c_void_p * MAX_CLASSES),
                ("coverage", C.c_void_p * MAX_SCALES), ("argmax", C.c_void_p * MAX_SCALES)]


_lib = None


def lib() -> C.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_2305_14566_gb300.build.build() "
                           "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, u32, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
    sig = {
        "omni_create": (i32, [C.POINTER(Config), C.POINTER(vp)]),
        "omni_destroy": (None, [vp]),
        "omni_last_error": (C.c_char_p, [vp]),
        "omni_weights_count": (i64, [C.POINTER(Config)]),
        "omni_load_weights": (i32, [vp, vp, i64]),
        "omni_query": (i32, [C.POINTER(Config), i32, i32, C.POINTER(Sizes)]),
        "omni_tile_slide": (i32, [vp, vp, i32, i32, i64, vp, u64, C.POINTER(TileList), vp]),
        "omni_segment_slide": (i32, [vp, vp, i32, i32, i64, u32, u32, vp, u64,
                                     C.POINTER(Outputs), vp]),
        "omni_segment_slide_host": (i32, [vp, vp, i32, i32, i64, u32, u32, vp, u64,
                                          C.POINTER(vp), vp]),
        "omni_synth_slide": (i32, [vp, i32, u64, i32, i32, i32, i32, i32, i32, vp, i64, vp]),
        "omni_stain": (i32, [vp, i32, i32, i64, i32, C.POINTER(vp), vp, vp, vp, vp, i64, i32, vp,
                             i64, vp]),
        "omni_conv_layer": (i32, [i32, i32, i32, i32, i32, vp, i32, i32, vp, vp, vp, vp, i32,
                                  i32, i32, vp, vp, i32, i32, vp, i32, vp, vp]),
        "omni_conv_candidates": (i32, [i32, i32, i32, i32, vp, i32]),
        "omni_set_conv_kind": (i32, [vp, i32]),
        "omni_set_timing": (i32, [vp, i32]),
        "omni_get_timing": (i32, [vp, i32, C.POINTER(C.c_double), C.POINTER(i64),
                                  C.POINTER(C.c_double)]),
        "omni_last_launch_count": (i64, [vp]),
        "omni_get_launch_times": (i64, [vp, i64, vp, vp, vp, vp]),
        "omni_tile_slide_noalloc": (i32, [C.POINTER(Config), vp, i32, i32, i64,
                                          C.POINTER(TileList), vp]),
        "omni_backward_workspace": (u64, [C.POINTER(Config), i32, i32]),
        "omni_set_autotune": (i32, [vp, i32]),
        "omni_set_e4m3": (i32, [vp, i32]),
        "omni_set_graphs": (i32, [vp, i32]),
        "omni_set_fusion": (i32, [vp, i32]),
        "omni_get_tuned": (i32, [vp, vp, i32]),
        "omni_backward": (i32, [vp, vp, i32, i32, i64, C.POINTER(vp), vp, u64, vp, C.POINTER(Grads), vp]),
        "omni_query_slides": (i32, [C.POINTER(Config), i32, vp, vp, C.POINTER(u64)]),
        "omni_segment_slides": (i32, [vp, i32, vp, vp, vp, vp, u32, u32, vp, u64, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class OmniError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"omniseg status {status}: {msg}")
        self.status = status


def check(status: int, ctx=None, what: str = "") -> None:
    if status != OK:
        msg = lib().omni_last_error(ctx).decode() if ctx else what
        raise OmniError(status, msg or what)
