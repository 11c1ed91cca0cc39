"""Seeded random-init weights for the residual U-Net, pre-head and controller.

No trained Omni-Seg checkpoint is available, so every parameter is drawn from
a seeded numpy PCG64 stream and stored as one flat little-endian float32 blob.
The blob order below is the file format read by ``omni_load_weights`` and by
the oracle; it is a layout description, not arithmetic of the method.

Blob order (C_l = base * 2**l, L = levels, conv weights OIHW):
  encoder l = 0 .. L-1, cin = 3 if l == 0 else C_{l-1}, cout = C_l:
      w1[cout][cin][3][3] g1[cout] b1[cout] w2[cout][cout][3][3] g2[cout] b2[cout]
      wp[cout][cin]                           (1x1 projection on the residual)
  decoder l = L-2 .. 0, cin = 3 * C_l (concat of upsampled C_{l+1} and skip C_l):
      w1[cout][cin][3][3] g1 b1 w2[cout][cout][3][3] g2 b2 wp[cout][cin]
  pre-head   wh[8][C_0] bh[8]
  controller wc[153][C_{L-1} + n_classes + n_scales] bc[153]

Init: convolutions and projections He-normal N(0, 2 / fan_in); norm scale
g ~ U[0.9, 1.1], norm shift b ~ U[-0.05, 0.05]; pre-head He-normal with its
bias ~ U[-0.05, 0.05]; controller He-normal with zero bias.  The second norm
scale and the projection of every residual block are multiplied by 1/sqrt(2)
so that the two branches of each residual sum add up to the variance of one
(the residual-gain reading), which keeps activations and logits O(1) through
the 2L-1 blocks.

Head calibration.  Random weights give the head's output no trained decision
threshold: it is negative everywhere.  The controller bias of theta[152] (the
head's final bias b3) is the workload's ``head_offset``, and
``head_offsets[c]`` is added to the controller weight that carries class c's
one-hot input into theta[152], so each class gets its own threshold.  The
needle workloads use per-class offsets placed at the valley of each class's
in-tissue response (tests/golden/make_head_offsets.py); the differentiation
workload uses one offset of 3.3, the tiny one 0.
"""
from __future__ import annotations

import math
from collections import OrderedDict
from typing import Dict, List, Tuple

import numpy as np

from .configs import HEAD_CH, N_HEAD_PARAMS

RES_GAIN = 1.0 / math.sqrt(2.0)


def layout(work) -> "OrderedDict[str, Tuple[int, ...]]":
    """Name -> shape of every tensor in blob order."""
    C = work.widths
    L = work.levels
    out: "OrderedDict[str, Tuple[int, ...]]" = OrderedDict()

    def block(prefix, cin, cout):
        out[prefix + ".w1"] = (cout, cin, 3, 3)
        out[prefix + ".g1"] = (cout,)
        out[prefix + ".b1"] = (cout,)
        out[prefix + ".w2"] = (cout, cout, 3, 3)
        out[prefix + ".g2"] = (cout,)
        out[prefix + ".b2"] = (cout,)
        out[prefix + ".wp"] = (cout, cin)

    for l in range(L):
        block(f"enc{l}", 3 if l == 0 else C[l - 1], C[l])
    for l in range(L - 2, -1, -1):
        block(f"dec{l}", 3 * C[l], C[l])
    out["head.w"] = (HEAD_CH, C[0])
    out["head.b"] = (HEAD_CH,)
    out["ctrl.w"] = (N_HEAD_PARAMS, work.ctrl_in)
    out["ctrl.b"] = (N_HEAD_PARAMS,)
    return out


def n_params(work) -> int:
    return int(sum(int(np.prod(s)) for s in layout(work).values()))


def gen_weights(work, seed: int | None = None) -> np.ndarray:
    """Flat float32 blob in the order of ``layout(work)``."""
    rng = np.random.default_rng(work.weights_seed if seed is None else seed)
    parts: List[np.ndarray] = []
    for name, shape in layout(work).items():
        kind = name.split(".")[1]
        if kind in ("w1", "w2", "wp", "w"):
            fan_in = int(np.prod(shape[1:]))
            t = rng.standard_normal(shape) * math.sqrt(2.0 / fan_in)
            if kind == "wp":
                t = t * RES_GAIN
        elif kind in ("g1", "g2"):
            t = rng.uniform(0.9, 1.1, shape)
            if kind == "g2":
                t = t * RES_GAIN
        elif kind in ("b1", "b2") or name == "head.b":
            t = rng.uniform(-0.05, 0.05, shape)
        else:  # ctrl.b
            t = np.zeros(shape)
            t[-1] = getattr(work, "head_offset", 0.0)
        if name == "ctrl.w" and getattr(work, "head_offsets", ()):
            # class c's one-hot input reaches theta[152] (the head's final
            # bias b3) through column C_{L-1} + c: a per-class threshold
            cb = work.widths[-1]
            for c, off in enumerate(work.head_offsets):
                t[-1, cb + c] += off
        parts.append(np.asarray(t, np.float32).ravel())
    return np.concatenate(parts).astype(np.float32)


def unpack(work, blob: np.ndarray) -> Dict[str, np.ndarray]:
    """Split a flat blob into named arrays (views, float32)."""
    out = {}
    off = 0
    for name, shape in layout(work).items():
        n = int(np.prod(shape))
        out[name] = blob[off:off + n].reshape(shape)
        off += n
    if off != blob.size:
        raise ValueError(f"weights blob has {blob.size} floats, layout needs {off}")
    return out
