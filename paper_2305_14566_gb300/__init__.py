"""GB300 (sm_103a) Omni-Seg slide-wise inference: tiling, residual U-Net with a
class/scale-conditioned dynamic head, and atomic-free overlap stitching.

The compute path is the CUDA library ``libomniseg.so`` (C ABI in
include/omniseg.h); this package only marshals arguments to it.
"""
from . import _lib  # noqa: F401
from ._lib import FP32, BF16, FP16, STITCH_AVG, STITCH_VOTE, OmniError  # noqa: F401

