"""Workload descriptions for the Omni-Seg slide-wise inference path.

Each workload fixes the slide geometry, the magnifications, the patch grid
(patch size P, stride S), the U-Net width/depth and the class heads.  These are
plain shape descriptions shared by the oracle, the tests and the benchmark;
they hold none of the method's arithmetic.

Magnifications are given as integer downsample factors relative to 40x
(1 = 40x, 4 = 10x, 8 = 5x), the three scales used for prediction in the
paper's segmentation stage (Sec. 2.2).  Classes are ordered so that two heads
sit at every scale (PTC, VES at 40x; PT, DT at 10x; TUFT, CAP at 5x), following
the tissue/magnification pairing given in Sec. 1 (capillaries at 40x, tubules
at 10x, glomeruli at 5x).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Tuple

HEAD_CH = 8            # dynamic head width: 1x1 convs 8 -> 8 -> 8 -> 1
N_HEAD_PARAMS = 8 * 8 + 8 * 8 + 8 + 8 + 8 + 1   # = 153 generated per (patch, class)
THUMB = 32             # tissue-detection thumbnail: 32x32 box at 40x
CLASS_NAMES = ("PTC", "VES", "PT", "DT", "TUFT", "CAP")

STITCH_AVG = 0
STITCH_VOTE = 1
WINDOW_FLAT = 0        # overlap-average weight per tile pixel: 1
WINDOW_TENT = 1        # min(u + 1, P - u) per axis
WINDOW_HANN = 2        # sin^2(pi (u + 1/2) / P) per axis


@dataclass(frozen=True)
class Workload:
    name: str
    H: int
    W: int
    seed: int                      # slide generator seed
    tissue: float                  # target tissue fraction
    layout: str                    # "cores" (needle biopsy) | "blobs"
    n_blobs: int
    factors: Tuple[int, ...]       # downsample factor per scale index
    P: int
    S: int
    base: int
    levels: int
    class_scale: Tuple[int, ...]   # scale index of every class
    weights_seed: int
    tissue_filter: bool = True     # drop background patches (Sec. 2.1)
    tissue_and: bool = True        # AND labels with the tissue mask (Sec. 2.3)
    stitch_mode: int = STITCH_AVG
    median_k: int = 59
    pad_lead: int = 0              # the paper's 4096 border; 0 for these workloads
    max_batch: int = 32
    head_offset: float = 0.0       # controller bias of the head's final bias b3 (weights init)
    head_offsets: Tuple[float, ...] = ()   # per-class addition to b3 through the class one-hot
    strides: Tuple[int, ...] = ()  # per-scale tile stride; () or 0 = S (Sec. 3.2: 256, 64, 64)
    stitch_window: int = WINDOW_FLAT
    min_tissue_area: int = 0       # drop 8-connected tissue regions under this many thumbnail px

    @property
    def n_classes(self) -> int:
        return len(self.class_scale)

    @property
    def n_scales(self) -> int:
        return len(self.factors)

    def stride(self, s: int) -> int:
        """Tile stride of scale index s, in that scale's pixels."""
        return self.strides[s] if self.strides and self.strides[s] else self.S

    @property
    def widths(self) -> List[int]:
        return [self.base << l for l in range(self.levels)]

    @property
    def ctrl_in(self) -> int:
        return self.widths[-1] + self.n_classes + self.n_scales

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


TINY = Workload(
    name="tiny", H=512, W=512, seed=0, tissue=0.35, layout="blobs", n_blobs=8,
    factors=(1,), P=128, S=64, base=8, levels=3, class_scale=(0, 0),
    weights_seed=10, tissue_filter=False, tissue_and=False, max_batch=49)

# Per-class head calibration of the needle network (weights seed 11): class c's
# threshold is the one with the fewest in-tissue raw responses within 0.05 of
# it (relative to the tissue and to its positives) on calibration tiles of the
# oracle, written by tests/golden/make_head_offsets.py into
# tests/golden/head_offsets.json (a CPU test keeps the two equal).
NEEDLE_HEAD_OFFSETS = (6.8456, 7.3584, 6.974, 6.0431, 7.3029, 6.2199)

NEEDLE = Workload(
    name="needle", H=16384, W=49152, seed=1, tissue=0.40, layout="cores", n_blobs=4,
    factors=(1, 4, 8), P=512, S=256, base=32, levels=5,
    class_scale=(0, 0, 1, 1, 2, 2), weights_seed=11, max_batch=256,
    head_offsets=NEEDLE_HEAD_OFFSETS)

DIFF = Workload(
    name="diff", H=2048, W=2048, seed=7, tissue=0.40, layout="blobs", n_blobs=6,
    factors=(1, 4, 8), P=256, S=128, base=32, levels=5,
    class_scale=(0, 0, 1, 1, 2, 2), weights_seed=12, tissue_filter=False,
    tissue_and=False, max_batch=64, head_offset=3.3)

LARGE = Workload(
    name="large", H=32768, W=98304, seed=200, tissue=0.35, layout="cores", n_blobs=4,
    factors=(1, 4, 8), P=1024, S=512, base=32, levels=5,
    class_scale=(0, 0, 1, 1, 2, 2), weights_seed=11, max_batch=8,
    head_offsets=NEEDLE_HEAD_OFFSETS)


# The paper's own overlap setting (Sec. 3.2): 40x tiles strided by 256 (two
# overlapping tiles per axis, vote threshold 1), 10x and 5x tiles by 64 (eight
# per axis, threshold 4), labels by majority vote.
NEEDLE_PAPER = NEEDLE.with_(name="needle_paper", strides=(256, 64, 64), stitch_mode=STITCH_VOTE)


def ragged_workloads(n: int = 12, seed0: int = 100) -> List[Workload]:
    """Twelve slides: long side ~U[8192, 49152], aspect ~U[1, 4], tissue ~U[0.2, 0.6]."""
    import numpy as np
    out = []
    for k in range(n):
        rng = np.random.default_rng(seed0 + k)
        long_side = int(rng.integers(8192, 49152 + 1))
        aspect = float(rng.uniform(1.0, 4.0))
        short = max(1024, int(long_side / aspect))
        tissue = float(rng.uniform(0.2, 0.6))
        out.append(NEEDLE.with_(name=f"ragged{k}", H=short, W=long_side, seed=seed0 + k,
                                tissue=tissue, n_blobs=int(rng.integers(3, 6))))
    return out


def small_variant(w: Workload, H: int, W: int, P: int, S: int, base: int, levels: int,
                  **kw) -> Workload:
    """Same method and scales at a size the FP64 oracle finishes in seconds."""
    return w.with_(name=w.name + "_small", H=H, W=W, P=P, S=S, base=base, levels=levels, **kw)
