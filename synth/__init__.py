"""Seeded synthetic inputs (slides, ground-truth masks, random-init weights).

Shared by the FP64 oracle, the tests and the benchmark.  Nothing here
computes any step of the segmentation method; it only produces inputs.
"""
from .configs import (TINY, NEEDLE, NEEDLE_PAPER, DIFF, LARGE, Workload, ragged_workloads, small_variant,
                      HEAD_CH, N_HEAD_PARAMS, THUMB, CLASS_NAMES, STITCH_AVG, STITCH_VOTE,
                      WINDOW_FLAT, WINDOW_TENT, WINDOW_HANN)
from .slides import (SlideSpec, Ellipse, make_spec, spec_for, gen_window, gen_slide,
                     gen_gt_masks, splitmix64)
from .weights import gen_weights, layout, unpack, n_params
