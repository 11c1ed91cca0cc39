"""Write needle_crop.npz: the FP64 oracle's segmentation of one 2048 x 2048
crop of the 16384 x 49152 needle-biopsy slide at 40x, with the matching
512 x 512 window at 10x and 256 x 256 at 5x (the crop origin is a multiple of
2048, so every scale's window starts on its tile grid).

The crop is drawn with a fixed seed among the 2048-aligned crops that hold
the centre line of tissue core 2 within the middle third of its length and
whose thumbnail tissue fraction lies in [0.4, 0.8] (deep tissue, the tissue
edge and glass in one window).  Every
processed tile that overlaps the window (81 at 40x, 9 at 10x, 4 at 5x when
all are foreground) runs through the
oracle's network and the window is stitched from them
(oracle.segment_window_regions), with the tissue AND of the workload.

Stored per class c: labels (bit-packed), the pixels where |L| < 1e-3
(bit-packed; the only places an FP32 path may disagree), and the stitched
logits on a 128 x 128 subsample (stride 16 at 40x, 4 at 10x, 2 at 5x).
Calls only the input generator and the FP64 oracle.
Run: python tests/golden/make_needle_crop.py   (~15 min)
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import omniseg_oracle as O  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
CROP = 2048
CORE = 2
SEED = 2048


def load_mask():
    g = np.load(os.path.join(HERE, "needle_tissue_mask.npz"))
    n = int(np.prod(g["shape"]))
    return np.unpackbits(g["bits"])[:n].reshape(g["shape"]).astype(bool)


def pick_crop(w, spec, mask):
    e = spec.ellipses[CORE]
    cands = []
    for y0 in range(0, w.H - CROP + 1, CROP):
        for x0 in range(0, w.W - CROP + 1, CROP):
            if not (y0 <= e.cy < y0 + CROP) or abs(x0 + CROP // 2 - e.cx) > e.a / 3:
                continue
            frac = float(mask[y0 // 32:(y0 + CROP) // 32, x0 // 32:(x0 + CROP) // 32].mean())
            if 0.4 <= frac <= 0.8:
                cands.append((y0, x0, frac))
    rng = np.random.default_rng(SEED)
    return cands[int(rng.integers(0, len(cands)))]


def main():
    w = synth.NEEDLE
    spec = synth.spec_for(w)
    blob = synth.gen_weights(w)
    mask = load_mask()
    y0, x0, frac = pick_crop(w, spec, mask)
    print("crop", y0, x0, "tissue fraction", frac, flush=True)
    orc = O.segment_window_regions(lambda y, x, h, ww: synth.gen_window(spec, y, x, h, ww), mask, w, blob,
                                   (y0, x0, CROP, CROP), w.H, w.W, batch=2)
    arrs = {"origin": np.array([y0, x0]), "size": np.array([CROP]),
            "head_offsets": np.array(w.head_offsets, np.float64)}
    meta = {}
    for c, s in enumerate(w.class_scale):
        L = orc["L"][c]
        lab = orc["labels"][c].astype(np.uint8)
        k = L.shape[0] // 128
        arrs[f"win{c}"] = np.array(orc["window"][s])
        arrs[f"shape{c}"] = np.array(L.shape)
        arrs[f"labels{c}"] = np.packbits(lab.ravel())
        arrs[f"nearzero{c}"] = np.packbits((np.abs(L) < 1e-3).astype(np.uint8).ravel())
        arrs[f"sub{c}"] = np.array([k])
        arrs[f"L{c}"] = L[::k, ::k].astype(np.float32)
        meta[c] = {"positives": int(lab.sum()), "pixels": int(lab.size),
                   "near_zero": int((np.abs(L) < 1e-3).sum())}
        print(c, meta[c], flush=True)
    np.savez_compressed(os.path.join(HERE, "needle_crop.npz"), **arrs)
    print(json.dumps({"origin": [y0, x0], "tissue_fraction": frac, "classes": meta}))


if __name__ == "__main__":
    main()
