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

Evaluation.  Controller and pre-head entries go through the oracle's
loss_heads_only.  An entry of the last decoder block changes one channel of
one of its convolutions, so the block's output at p +- eps e_i is rebuilt
from the unperturbed block's cached conv1, conv2 and projection outputs by
redoing only that channel (the block's own definition, out = ReLU(N2(conv2(
ReLU(N1(conv1(x))))) + proj(x)), split along the changed channel):
  w1[o,i,dy,dx]: conv1's channel o gains eps times the shifted input channel
      i; then as for g1 / b1;
  g1[o], b1[o]: channel o of ReLU(N1(conv1 x)) is recomputed and conv2 is
      corrected by conv2 restricted to input channel o applied to that
      channel's change;
  w2[o,i,dy,dx]: conv2's channel o gains eps times the shifted channel i of
      ReLU(N1(conv1 x));
  g2[o], b2[o]: N2 of channel o;  wp[o,i]: proj channel o gains eps x_i.
Every draw checks its rebuilt block output against the oracle's res_block
with the perturbed tensor on the first cached batch (max abs difference
below 1e-12 or the script stops), and loss_from_y0 is the oracle's.
Calls only the input generator and the FP64 oracle.
Run: python tests/golden/make_diff_fd.py   (about an hour on 8 cores, 30 GB)
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


class BlockCache:
    """Unperturbed conv1, conv2 and projection outputs of the last decoder
    block for every cached batch of the problem."""

    def __init__(self, prob):
        self.prob = prob
        p = prob.p
        self.c1, self.c2, self.px = [], [], []
        with torch.no_grad():
            for (_, _, cat0, _) in prob.cache:
                c1 = O.conv3x3(cat0, p["dec0.w1"])
                self.c1.append(c1)
                self.c2.append(O.conv3x3(O.relu(O.affine(c1, p["dec0.g1"], p["dec0.b1"])), p["dec0.w2"]))
                self.px.append(O.conv1x1(cat0, p["dec0.wp"]))

    @staticmethod
    def _tap(d, dy, dx, dtype):
        """3x3 kernel with d at (dy, dx): conv3x3 with it shifts its input."""
        t = torch.zeros((1, 1, 3, 3), dtype=dtype)
        t[0, 0, dy, dx] = d
        return t

    def y0(self, k, name, idx, d):
        """Block output of cached batch k with entry idx of tensor name moved by d."""
        p = self.prob.p
        cat0 = self.prob.cache[k][2]
        c2, px = self.c2[k], self.px[k]
        g2, b2 = p["dec0.g2"], p["dec0.b2"]
        c1 = self.c1[k]
        if name in ("dec0.w1", "dec0.g1", "dec0.b1"):
            o = idx[0]
            c1o = c1[:, o:o + 1]
            g1o = p["dec0.g1"][o:o + 1].clone()
            b1o = p["dec0.b1"][o:o + 1].clone()
            a_old = O.relu(O.affine(c1o, g1o, b1o))
            if name == "dec0.w1":
                i = idx[1]
                c1o = c1o + O.conv3x3(cat0[:, i:i + 1], self._tap(d, idx[2], idx[3], c1o.dtype))
            elif name == "dec0.g1":
                g1o[0] += d
            else:
                b1o[0] += d
            a_new = O.relu(O.affine(c1o, g1o, b1o))
            c2 = c2 + O.conv3x3(a_new - a_old, p["dec0.w2"][:, o:o + 1])
        elif name == "dec0.w2":
            o, i = idx[0], idx[1]
            a_i = O.relu(O.affine(c1[:, i:i + 1], p["dec0.g1"][i:i + 1], p["dec0.b1"][i:i + 1]))
            c2 = c2.clone()
            c2[:, o:o + 1] += O.conv3x3(a_i, self._tap(d, idx[2], idx[3], a_i.dtype))
        elif name in ("dec0.g2", "dec0.b2"):
            g2, b2 = g2.clone(), b2.clone()
            (g2 if name == "dec0.g2" else b2)[idx[0]] += d
        elif name == "dec0.wp":
            o, i = idx
            px = px.clone()
            px[:, o] += d * cat0[:, i]
        else:
            raise ValueError(name)
        return O.relu(O.affine(c2, g2, b2) + px)

    def loss(self, name, idx, d):
        with torch.no_grad():
            ys = [self.y0(k, name, idx, d) for k in range(len(self.prob.cache))]
            # self-check on the first batch against the block's own definition
            q = dict(self.prob.p)
            q[name] = q[name].clone()
            q[name][idx] += d
            full = O.res_block(self.prob.cache[0][2], q, "dec0")
            err = float((full - ys[0]).abs().max())
            if err > 1e-12:
                raise RuntimeError("rebuilt block output differs from res_block: %s %s %g" % (name, idx, err))
            return float(self.prob.loss_from_y0({}, ys))


def main():
    w = synth.DIFF
    t0 = time.time()
    rgb = synth.gen_slide(synth.spec_for(w))
    gts = synth.gen_gt_masks(w.H, w.W, w.factors, w.class_scale, seed=7)
    prob = O.DiffProblem(rgb, w, synth.gen_weights(w), gts)
    loss, grads = prob.loss_and_grads_by_batch()
    print("autograd done %.0fs loss %.12f" % (time.time() - t0, loss), flush=True)
    blk = BlockCache(prob)
    base = prob.params()
    names = list(O.GRAD_PARAMS)
    rng = np.random.default_rng(8)

    def quotient(name, idx, eps):
        if name.startswith(("ctrl.", "head.")):
            qp = {name: base[name].clone()}
            qm = {name: base[name].clone()}
            qp[name][idx] += eps
            qm[name][idx] -= eps
            with torch.no_grad():
                return (float(prob.loss_heads_only(qp)) - float(prob.loss_heads_only(qm))) / (2 * eps)
        return (blk.loss(name, idx, eps) - blk.loss(name, idx, -eps)) / (2 * eps)

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
