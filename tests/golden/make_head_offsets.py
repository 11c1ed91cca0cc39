"""Write head_offsets.json: the per-class threshold of the dynamic head for the
needle-biopsy network (synth.NEEDLE, weights seed 11), from the FP64 oracle.

No trained checkpoint exists, so the network's raw head output carries no
trained decision threshold: with random weights it is negative everywhere and
varies smoothly inside tissue.  A class's label decision is well conditioned
only where few pixels respond close to its threshold: a pixel whose raw
response lies within a small band around the threshold can change label under
a small perturbation of its logit, a pixel outside it cannot.  This script
places class c's threshold where that band holds the fewest pixels relative
to what the label comparison can absorb:

  1. calibration tiles: at each scale, vertical strips of tiles across tissue
     cores 0 and 3 of the needle slide (the test crops lie on core 2);
  2. raw response: the oracle's stitched-free tile logits of class c with
     every offset zero, at the tile pixels that the slide's tissue mask marks
     as tissue (the labels are ANDed with that mask);
  3. candidates: the responses' quantiles at 400 evenly spaced levels from 1%
     to 99% (so 1% to 99% of the tissue pixels end up positive) and the
     midpoints between neighbouring ones;
  4. for each candidate t: near(t) = share of tissue pixels whose response
     lies within DELTA = 0.05 of t, pos(t) = share above t, and
     score(t) = max(near / 0.001, near / (0.01 pos)): near against 0.1% of
     the tissue and against 1% of the positives (a Dice loss of 0.005 is a
     flipped share of 1% of the positives);
  5. threshold t_c: the candidate of least score; offset_c = -t_c, added to
     the head's final bias through class c's one-hot input (synth.weights).

With this random network the in-tissue responses have no deep interior
valley: at 10x and 5x they are smooth and unimodal (standard deviation about
0.5 against 1.7 at 40x), so the least crowded thresholds lie in the low tail
and label 97-99% of the tissue positive.  Restricted to 5%..95% positive, the
best 5x thresholds still have 1.3-2.4% of the tissue within 0.05, where
16-bit storage of the activations (logit noise of a few hundredths) flips
more than 0.1% of the labels.

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


DELTA = 0.05


def least_crowded(x, lo_q=0.01, hi_q=0.99, n=400):
    """Threshold of least score (see the module docstring) among the quantiles
    of the responses x; returns (threshold, near share, positive share)."""
    v = np.sort(np.asarray(x, np.float64))
    best = None
    q = np.quantile(v, np.linspace(lo_q, hi_q, n))
    for t in np.concatenate([q, 0.5 * (q[1:] + q[:-1])]):
        near = (np.searchsorted(v, t + DELTA, "right") - np.searchsorted(v, t - DELTA, "left")) / v.size
        pos = 1.0 - np.searchsorted(v, t, "right") / v.size
        score = max(near / 0.001, near / (0.01 * pos))
        if best is None or score < best[0]:
            best = (score, float(t), float(near), float(pos))
    return best[1], best[2], best[3]


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
            t, near, pos = least_crowded(v)
            offsets[c] = -t
            out["classes"][str(c)] = {"scale": s, "name": synth.CLASS_NAMES[c], "threshold": t,
                                      "offset": -t, "share_within_delta": near, "delta": DELTA,
                                      "tiles": len(tiles), "tissue_pixels": int(v.size),
                                      "positive_fraction_in_tissue": pos}
            print(json.dumps({c: out["classes"][str(c)]}), flush=True)
    out["head_offsets"] = [round(o, 4) for o in offsets]
    with open(os.path.join(HERE, "head_offsets.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out["head_offsets"]))


if __name__ == "__main__":
    main()
