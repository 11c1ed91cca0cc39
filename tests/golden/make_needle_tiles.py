"""Write needle_tiles.json (the oracle's tissue threshold and foreground tile
counts, with the common stride and with the per-scale strides of Sec. 3.2)
and needle_tissue_mask.npz (its 512 x 1536 tissue mask, bit-packed)
for the 16384 x 49152 needle-biopsy workload.

Calls only the input generator and the FP64 oracle.  The slide is generated
on the CPU in bands of 1024 rows; the oracle's thumbnail is a per-32x32-block
definition, so the bands' thumbnails concatenate to the slide's.
Run: python tests/golden/make_needle_tiles.py   (several minutes)
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import omniseg_oracle as O  # noqa: E402


def main():
    w = synth.NEEDLE
    spec = synth.spec_for(w)
    bands = [O.thumbnail(synth.gen_window(spec, y, 0, 1024, w.W)) for y in range(0, w.H, 1024)]
    thumb = np.concatenate(bands, 0)
    b = O.median_blur(O.grey(thumb), w.median_k)
    t = O.otsu(O.histogram(b))
    mask = b.astype(np.int64) <= t
    tiles, flags = O.tile_list(w, mask, w.H, w.W)
    per = [sum(1 for q in tiles if q[0] == s) for s in range(w.n_scales)]
    # the same slide tiled with the per-scale strides of Sec. 3.2 (256 / 64 / 64)
    wp = synth.NEEDLE_PAPER
    ptiles, pflags = O.tile_list(wp, mask, *O.padded_dims(wp)[:2])
    pper = [sum(1 for q in ptiles if q[0] == s) for s in range(wp.n_scales)]
    out = {"_source": "oracle tile list of synth.NEEDLE (tests/golden/make_needle_tiles.py)",
           "otsu": int(t), "tissue_fraction": float(mask.mean()),
           "tiles_per_scale": per, "tiles_total": len(tiles),
           "grid_per_scale": [int(f.size) for f in flags],
           "paper_strides": list(wp.strides),
           "paper_strides_tiles_per_scale": pper, "paper_strides_tiles_total": len(ptiles),
           "paper_strides_grid_per_scale": [int(f.size) for f in pflags]}
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "needle_tiles.json"), "w") as f:
        json.dump(out, f, indent=1)
    np.savez_compressed(os.path.join(here, "needle_tissue_mask.npz"), shape=np.array(mask.shape),
                        bits=np.packbits(mask.astype(np.uint8).ravel()))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
