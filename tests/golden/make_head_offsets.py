"""Write head_offsets.json: the per-class threshold of the dynamic head for the
needle-biopsy network (synth.NEEDLE, weights seed 11), from the FP64 oracle.

No trained checkpoint exists, so the network's raw head output carries no
trained decision threshold: with random weights it is negative everywhere and
varies smoothly inside tissue.  A class's label decision is well conditioned
only where few pixels respond near its threshold.  This script therefore
places class c's threshold at the valley of its raw response:

  1. calibration tiles: at each scale, vertical strips of tiles across tissue
     cores 0 and 3 of the needle slide (the test crops lie on core 2);
  2. raw response: the oracle's stitched-free tile logits of class c with
     every offset zero, at the tile pixels that the slide's tissue mask marks
     as tissue (the labels are ANDed with that mask);
  3. threshold t_c: the smallest value of the histogram of those responses,
     smoothed by a 9-bin moving average over 400 bins spanning their
     0.5%..99.5% quantiles, among bins between their 5% and 95% quantiles;
  4. offset_c = -t_c, added to the head's final bias through class c's
     one-hot input (synth.weights).

Calls only the input generator and the FP64 oracle.  The tissue mask is the
oracle's (tests/golden/needle_tissue_mask.npz, written by
make_needle_tiles.py).  Run: python tests/golden/make_head_offsets.py  (~10 min)
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
# strips per scale: (core, x position as a fraction of the core's half length)
STRIPS = {0: [(0, -0.3), (3, -0.3)],
          1: [(0, -0.3), (0, 0.3), (3, -0.3), (3, 0.3)],
          2: [(0, -0.45), (0, -0.15), (0, 0.15), (0, 0.45), (3, -0.45), (3, -0.15), (3, 0.15), (3, 0.45)]}


def load_mask():
    g = np.load(os.path.join(HERE, "needle_tissue_mask.npz"))
    n = int(np.prod(g["shape"]))
    return np.unpackbits(g["bits"])[:n].reshape(g["shape"]).astype(bool)


def strip_tiles(w, spec, s, core, frac):
    """Tile origins (scale pixels) of a vertical strip crossing the core."""
    f, P, S = w.factors[s], w.P, w.stride(s)
    e = spec.ellipses[core]
    step = S * f
    x40 = int((e.cx + frac * e.a) // step) * step
    out = []
    for y40 in range(0, w.H - P * f + 1, step):
        if y40 + P * f > e.cy - e.b and y40 < e.cy + e.b:
            out.append((y40 // f, x40 // f))
    return out


def valley(x, bins=400, smooth=9, lo_q=0.05, hi_q=0.95):
    lo, hi = np.quantile(x, [0.005, 0.995])
    h, edges = np.histogram(x, bins=bins, range=(lo, hi))
    hs = np.convolve(h, np.ones(smooth) / smooth, mode="same")
    centres = 0.5 * (edges[1:] + edges[:-1])
    a, b = np.quantile(x, [lo_q, hi_q])
    inside = (centres > a) & (centres < b)
    i = int(np.argmin(np.where(inside, hs, np.inf)))
    return float(centres[i]), float(hs[i] / hs.max())


def main():
    base = synth.NEEDLE.with_(head_offsets=(), head_offset=0.0)
    spec = synth.spec_for(base)
    p = O.weights_f64(base, synth.gen_weights(base))
    mask = load_mask()
    out = {"_source": "oracle responses of synth.NEEDLE with zero head offsets "
                      "(tests/golden/make_head_offsets.py)", "classes": {}}
    offsets = [0.0] * base.n_classes
    for s, f in enumerate(base.factors):
        P = base.P
        hs, ws = base.H // f, base.W // f
        tis = O.tissue_at_scale(mask, f, hs, ws)
        tiles = sorted({t for (core, frac) in STRIPS[s] for t in strip_tiles(base, spec, s, core, frac)})
        cls = [c for c, cs in enumerate(base.class_scale) if cs == s]
        vals = {c: [] for c in cls}
        for (y, x) in tiles:
            img = synth.gen_window(spec, y * f, x * f, P * f, P * f)
            g = f
            while g > 1:
                img = O.half(img)
                g //= 2
            lg, ids = O.patch_forward(img[None], p, base, s)
            m = tis[y:y + P, x:x + P]
            for k, c in enumerate(ids):
                vals[c].append(lg[k, 0].numpy()[m])
        for c in cls:
            v = np.concatenate(vals[c])
            t, dens = valley(v)
            offsets[c] = -t
            out["classes"][str(c)] = {"scale": s, "name": synth.CLASS_NAMES[c], "threshold": t,
                                      "offset": -t, "relative_density_at_threshold": dens,
                                      "tiles": len(tiles), "tissue_pixels": int(v.size),
                                      "positive_fraction_in_tissue": float(np.mean(v > t))}
            print(json.dumps({c: out["classes"][str(c)]}), flush=True)
    out["head_offsets"] = [round(o, 4) for o in offsets]
    with open(os.path.join(HERE, "head_offsets.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out["head_offsets"]))


if __name__ == "__main__":
    main()
