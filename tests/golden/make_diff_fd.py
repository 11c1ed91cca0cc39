"""Write diff_fd.json: FP64 central finite differences of the stitched
soft-Dice + BCE loss of the differentiation workload (synth.DIFF: 2048 x 2048
slide, 256-px tiles at stride 128, 235 tiles, base-32 5-level network, six
ground-truth masks) at 64 seeded parameters of the differentiated sub-chain
(controller, pre-head, last decoder block), next to the oracle's autograd
gradient at the same entries.

  fd = (loss(p + eps e_i) - loss(p - eps e_i)) / (2 eps),  eps = 1e-6
Parameters: draw k (k = 0..63) takes tensor k mod 11 of the sub-chain (in
oracle.GRAD_PARAMS order) and a uniformly drawn entry of it (numpy PCG64,
seed 8).  A draw whose difference quotients at eps and eps / 4 disagree by
more than 1e-4 relative straddles a ReLU kink and is redrawn (logged).
Calls only the input generator and the FP64 oracle.
Run: python tests/golden/make_diff_fd.py   (about half an hour on 8 cores)
"""
import json
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import omniseg_oracle as O  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
EPS = 1e-6
N_DRAWS = 64


def main():
    w = synth.DIFF
    t0 = time.time()
    rgb = synth.gen_slide(synth.spec_for(w))
    gts = synth.gen_gt_masks(w.H, w.W, w.factors, w.class_scale, seed=7)
    prob = O.DiffProblem(rgb, w, synth.gen_weights(w), gts)
    loss, grads = prob.loss_and_grads_by_batch()
    print("autograd done %.0fs loss %.12f" % (time.time() - t0, loss), flush=True)
    base = prob.params()
    names = list(O.GRAD_PARAMS)
    rng = np.random.default_rng(8)

    def quotient(name, idx, eps):
        qp = {name: base[name].clone()}
        qm = {name: base[name].clone()}
        qp[name][idx] += eps
        qm[name][idx] -= eps
        fn = prob.loss_heads_only if name.startswith(("ctrl.", "head.")) else prob.loss
        with torch.no_grad():
            return (float(fn(qp)) - float(fn(qm))) / (2 * eps)

    rows, redrawn = [], []
    k = 0
    while len(rows) < N_DRAWS:
        name = names[k % len(names)]
        idx = tuple(int(rng.integers(0, s)) for s in base[name].shape)
        fd = quotient(name, idx, EPS)
        fd4 = quotient(name, idx, EPS / 4)
        if abs(fd - fd4) > 1e-4 * max(abs(fd), 1e-8):
            redrawn.append({"name": name, "index": list(idx), "fd": fd, "fd_eps_quarter": fd4})
            print("redrawn (kink)", name, idx, fd, fd4, flush=True)
            continue
        rows.append({"name": name, "index": list(idx), "fd": fd, "autograd": float(grads[name][idx]),
                     "tensor_max_abs_grad": float(grads[name].abs().max())})
        print(len(rows), name, idx, "fd %.10e ag %.10e  %.0fs" % (fd, rows[-1]["autograd"], time.time() - t0),
              flush=True)
        k += 1
    out = {"_source": "oracle central differences on synth.DIFF (tests/golden/make_diff_fd.py)",
           "eps": EPS, "loss": loss, "draws": rows, "redrawn": redrawn}
    with open(os.path.join(HERE, "diff_fd.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
