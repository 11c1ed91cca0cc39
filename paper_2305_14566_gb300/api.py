"""Thin Python layer over the C ABI: torch tensors in, torch tensors out.

PyTorch provides device memory and streams only; every step of the path runs
in the library's CUDA kernels.  Names follow include/omniseg.h.
"""
from __future__ import annotations

import ctypes as C
from typing import Dict, Optional, Sequence

import numpy as np
import torch

from . import _lib as L


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream: Optional[torch.cuda.Stream] = None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_config(work, precision: int = L.FP32, max_batch: Optional[int] = None) -> L.Config:
    """omni_config for a workload description (see synth.configs.Workload)."""
    c = L.Config()
    c.patch, c.stride, c.levels, c.base = work.P, work.S, work.levels, work.base
    c.n_scales = len(work.factors)
    for i, f in enumerate(work.factors):
        c.factors[i] = f
    c.n_classes = len(work.class_scale)
    for i, s in enumerate(work.class_scale):
        c.class_scale[i] = s
    c.precision = precision
    c.stitch_mode = work.stitch_mode
    c.tissue_filter = int(work.tissue_filter)
    c.tissue_and = int(work.tissue_and)
    c.pad_lead = work.pad_lead
    c.median_k = work.median_k
    c.max_batch = max_batch if max_batch is not None else work.max_batch
    for i in range(c.n_scales):
        c.scale_stride[i] = work.stride(i)
    c.stitch_window = work.stitch_window
    c.min_tissue_area = getattr(work, "min_tissue_area", 0)
    return c


class Segmenter:
    """One library context: configuration + device weights."""

    def __init__(self, work, blob: np.ndarray, precision: int = L.FP32,
                 max_batch: Optional[int] = None):
        self.lib = L.lib()
        self.work = work
        self.cfg = make_config(work, precision, max_batch)
        self.ctx = C.c_void_p()
        st = self.lib.omni_create(C.byref(self.cfg), C.byref(self.ctx))
        L.check(st, None, "omni_create rejected the configuration")
        self.blob = None
        self.load_weights(blob)
        self._ws: Optional[torch.Tensor] = None
        self._stamps: Optional[torch.Tensor] = None
        self._stamps_n = 0

    def load_weights(self, blob: np.ndarray):
        """omni_load_weights: replace the context's weights (a flat FP32 blob in
        the layout of omniseg.h); the segmenter keeps a host copy."""
        blob = np.array(blob, dtype=np.float32, copy=True).ravel()
        L.check(self.lib.omni_load_weights(self.ctx, blob.ctypes.data_as(C.c_void_p), blob.size),
                self.ctx)
        self.blob = blob

    def close(self):
        if self.ctx:
            self.lib.omni_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ sizes
    def query(self, H: int, W: int) -> L.Sizes:
        s = L.Sizes()
        L.check(self.lib.omni_query(C.byref(self.cfg), H, W, C.byref(s)), None, "omni_query: bad size")
        return s

    def workspace(self, nbytes: int, device) -> torch.Tensor:
        if self._ws is None or self._ws.numel() < nbytes or self._ws.device != torch.device(device):
            self._ws = None
            self._ws = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
        return self._ws

    # ------------------------------------------------------------------ Sec. 2.1
    def tile_slide(self, rgb: torch.Tensor) -> Dict[str, torch.Tensor]:
        """Tiles, per-scale counts/flags, tissue mask and Otsu threshold."""
        H, W, _ = rgb.shape
        sz = self.query(H, W)
        dev = rgb.device
        n = sz.n_tiles_max
        out = dict(tiles=torch.zeros((n, 3), dtype=torch.int32, device=dev),
                   counts=torch.zeros(1 + self.cfg.n_scales, dtype=torch.int32, device=dev),
                   flags=torch.zeros(n, dtype=torch.uint8, device=dev),
                   tissue=torch.zeros((sz.thumb_h, sz.thumb_w), dtype=torch.uint8, device=dev),
                   otsu=torch.zeros(1, dtype=torch.int32, device=dev))
        tl = L.TileList(out["tiles"].data_ptr(), out["counts"].data_ptr(), out["flags"].data_ptr(),
                        out["tissue"].data_ptr(), out["otsu"].data_ptr())
        ws = self.workspace(sz.tile_workspace_bytes, dev)
        L.check(self.lib.omni_tile_slide(self.ctx, _ptr(rgb), H, W, rgb.stride(0), _ptr(ws),
                                         ws.numel(), C.byref(tl), _stream()), self.ctx)
        return out

    # ------------------------------------------------------------------ whole path
    def segment(self, rgb: torch.Tensor, scales: Optional[Sequence[int]] = None,
                classes: Optional[Sequence[int]] = None, logits: bool = False,
                coverage: bool = False, argmax: bool = False,
                out: Optional[Dict] = None) -> Dict:
        """Label maps (and optional logits / coverage / argmax) per class.

        Returns {"labels": {c: u8 tensor}, "logits": {c: f32}, "coverage": {s: u16},
        "argmax": {s: u8}}.  Pass ``out`` (a previous result) to reuse its buffers.
        """
        H, W, _ = rgb.shape
        sz = self.query(H, W)
        dev = rgb.device
        cfg = self.cfg
        scales = list(range(cfg.n_scales)) if scales is None else list(scales)
        classes = [k for k in range(cfg.n_classes) if classes is None or k in classes]
        smask = sum(1 << s for s in scales)
        cmask = sum(1 << k for k in classes)
        if out is None:
            out = {"labels": {}, "logits": {}, "coverage": {}, "argmax": {}}
            for k in classes:
                s = cfg.class_scale[k]
                if s not in scales:
                    continue
                shp = (sz.out_h[s], sz.out_w[s])
                out["labels"][k] = torch.empty(shp, dtype=torch.uint8, device=dev)
                if logits:
                    out["logits"][k] = torch.empty(shp, dtype=torch.float32, device=dev)
            for s in scales:
                shp = (sz.out_h[s], sz.out_w[s])
                if coverage:
                    out["coverage"][s] = torch.empty(shp, dtype=torch.int16, device=dev)
                if argmax:
                    out["argmax"][s] = torch.empty(shp, dtype=torch.uint8, device=dev)
        o = L.Outputs()
        for k, t in out["labels"].items():
            o.labels[k] = t.data_ptr()
        for k, t in out["logits"].items():
            o.logits[k] = t.data_ptr()
        for s, t in out["coverage"].items():
            o.coverage[s] = t.data_ptr()
        for s, t in out["argmax"].items():
            o.argmax[s] = t.data_ptr()
        ws = self.workspace(sz.workspace_bytes, dev)
        L.check(self.lib.omni_segment_slide(self.ctx, _ptr(rgb), H, W, rgb.stride(0), smask, cmask,
                                            _ptr(ws), ws.numel(), C.byref(o), _stream()), self.ctx)
        return out

    def segment_many(self, rgbs: Sequence[torch.Tensor], outs: Optional[Sequence[Dict]] = None,
                     logits: bool = False) -> list:
        """omni_segment_slides: several slides in one call, their tiles packed
        into shared network batches per scale.  Returns one {"labels": ...,
        "logits": ...} dict per slide (pass ``outs`` to reuse buffers)."""
        n = len(rgbs)
        dev = rgbs[0].device
        cfg = self.cfg
        Hs = np.array([int(r.shape[0]) for r in rgbs], np.int32)
        Ws = np.array([int(r.shape[1]) for r in rgbs], np.int32)
        strides = np.array([int(r.stride(0)) for r in rgbs], np.int64)
        nbytes = C.c_uint64()
        L.check(self.lib.omni_query_slides(C.byref(cfg), n, Hs.ctypes.data_as(C.c_void_p),
                                           Ws.ctypes.data_as(C.c_void_p), C.byref(nbytes)),
                None, "omni_query_slides: bad sizes")
        if outs is None:
            outs = []
            for r in rgbs:
                sz = self.query(int(r.shape[0]), int(r.shape[1]))
                o = {"labels": {}, "logits": {}}
                for k in range(cfg.n_classes):
                    s = cfg.class_scale[k]
                    shp = (sz.out_h[s], sz.out_w[s])
                    o["labels"][k] = torch.empty(shp, dtype=torch.uint8, device=dev)
                    if logits:
                        o["logits"][k] = torch.empty(shp, dtype=torch.float32, device=dev)
                outs.append(o)
        arr = (L.Outputs * n)()
        for i, o in enumerate(outs):
            for k, t in o["labels"].items():
                arr[i].labels[k] = t.data_ptr()
            for k, t in o.get("logits", {}).items():
                arr[i].logits[k] = t.data_ptr()
        ptrs = (C.c_void_p * n)(*[r.data_ptr() for r in rgbs])
        ws = self.workspace(nbytes.value, dev)
        if self._stamps is None or self._stamps.numel() < n + 1 or self._stamps.device != dev:
            self._stamps = torch.zeros(L.MAX_SLIDES + 1, dtype=torch.int64, device=dev)
        self._stamps_n = n
        L.check(self.lib.omni_segment_slides(self.ctx, n, ptrs, Hs.ctypes.data_as(C.c_void_p),
                                             Ws.ctypes.data_as(C.c_void_p), strides.ctypes.data_as(C.c_void_p),
                                             (1 << cfg.n_scales) - 1, (1 << cfg.n_classes) - 1, _ptr(ws),
                                             ws.numel(), arr, _ptr(self._stamps), _stream()), self.ctx)
        return list(outs)

    def slide_times(self):
        """Per-slide completion times (ms after the post-tiling chain's start)
        of the last segment_many call, from the device clock stamps it wrote
        (waits for the current stream)."""
        t = self._stamps[:self._stamps_n + 1].cpu().numpy().astype(np.uint64)
        return [float((t[1 + i] - t[0]) / 1e6) for i in range(self._stamps_n)]

    def segment_host(self, rgb_host: torch.Tensor, labels_host: Dict[int, torch.Tensor],
                     device="cuda") -> Dict[int, torch.Tensor]:
        """Whole path from a HOST slide into HOST label buffers (copies included)."""
        H, W, _ = rgb_host.shape
        sz = self.query(H, W)
        ws = self.workspace(sz.workspace_bytes, device)
        arr = (C.c_void_p * L.MAX_CLASSES)()
        cmask = 0
        for k, t in labels_host.items():
            arr[k] = t.data_ptr()
            cmask |= 1 << k
        smask = (1 << self.cfg.n_scales) - 1
        L.check(self.lib.omni_segment_slide_host(self.ctx, _ptr(rgb_host), H, W, rgb_host.stride(0),
                                                 smask, cmask, _ptr(ws), ws.numel(), arr,
                                                 _stream()), self.ctx)
        return labels_host

    # ------------------------------------------------------------------ loss + backward
    def grad_shapes(self):
        w = self.work
        C0, zdim = w.base, w.widths[-1] + w.n_classes + w.n_scales
        return {"ctrl_w": (153, zdim), "ctrl_b": (153,), "head_w": (8, C0), "head_b": (8,),
                "dec0_w1": (C0, 3 * C0, 3, 3), "dec0_g1": (C0,), "dec0_b1": (C0,),
                "dec0_w2": (C0, C0, 3, 3), "dec0_g2": (C0,), "dec0_b2": (C0,),
                "dec0_wp": (C0, 3 * C0)}

    def grad_offsets(self):
        """Blob offset of every differentiated tensor.  The blob ends with the
        last decoder block (w1 g1 b1 w2 g2 b2 wp), the pre-head (w, b) and the
        controller (w, b), in that order."""
        order = ("dec0_w1", "dec0_g1", "dec0_b1", "dec0_w2", "dec0_g2", "dec0_b2", "dec0_wp",
                 "head_w", "head_b", "ctrl_w", "ctrl_b")
        shapes = self.grad_shapes()
        n_tail = sum(int(np.prod(shapes[k])) for k in order)
        off = self.blob.size - n_tail
        out = {}
        for k in order:
            out[k] = off
            off += int(np.prod(shapes[k]))
        return out

    def backward(self, rgb: torch.Tensor, gts):
        """Stitched soft-Dice + BCE loss of one slide and its gradients (omni_backward).

        ``gts``: one uint8 device tensor per class at its scale's label-map size.
        Returns (loss tensor [1], {name: FP32 gradient tensor}).
        """
        H, W, _ = rgb.shape
        dev = rgb.device
        nbytes = int(self.lib.omni_backward_workspace(C.byref(self.cfg), H, W))
        if nbytes == 0:
            raise L.OmniError(L.EINVAL, "omni_backward_workspace: bad configuration or size")
        ws = self.workspace(nbytes, dev)
        grads = {k: torch.zeros(v, dtype=torch.float32, device=dev) for k, v in self.grad_shapes().items()}
        g = L.Grads(*[grads[k].data_ptr() for k in L.GRAD_FIELDS])
        gt_arr = (C.c_void_p * len(gts))(*[t.data_ptr() for t in gts])
        loss = torch.zeros(1, dtype=torch.float32, device=dev)
        L.check(self.lib.omni_backward(self.ctx, _ptr(rgb), H, W, rgb.stride(0), gt_arr, _ptr(ws),
                                       ws.numel(), _ptr(loss), C.byref(g), _stream()), self.ctx)
        return loss, grads

    # ------------------------------------------------------------------ timing
    def set_timing(self, on: bool = True):
        L.check(self.lib.omni_set_timing(self.ctx, int(on)), self.ctx)

    def timing(self, kind: int):
        ms, n, work = C.c_double(), C.c_int64(), C.c_double()
        L.check(self.lib.omni_get_timing(self.ctx, kind, C.byref(ms), C.byref(n), C.byref(work)),
                self.ctx)
        return ms.value, n.value, work.value

    def set_autotune(self, on: bool = True):
        L.check(self.lib.omni_set_autotune(self.ctx, int(on)), self.ctx)

    def set_e4m3(self, on: bool = True):
        """E4M3 experiment: the first convs of the deeper levels (cin, cout
        multiples of 128) run on E4M3 operands (BF16 segmenters only)."""
        L.check(self.lib.omni_set_e4m3(self.ctx, int(on)), self.ctx)

    def set_conv_kind(self, kind: int = -1):
        """Force one tensor-core kernel kind on every layer that has it (-1: default)."""
        L.check(self.lib.omni_set_conv_kind(self.ctx, int(kind)), self.ctx)

    def set_graphs(self, on: bool = True):
        L.check(self.lib.omni_set_graphs(self.ctx, int(on)), self.ctx)

    def set_fusion(self, on: bool = True):
        """Epilogue fusion of the encoder max-pool and of the pre-head + heads (default on)."""
        L.check(self.lib.omni_set_fusion(self.ctx, int(on)), self.ctx)

    def tuned(self):
        """[(R, cin, cout, cr, res_kind, batch, kind, N tile, chunk, stages)] chosen by the autotuner."""
        n = self.lib.omni_get_tuned(self.ctx, None, 0)
        rows = np.zeros((max(n, 1), 10), np.int32)
        self.lib.omni_get_tuned(self.ctx, rows.ctypes.data_as(C.c_void_p), n)
        return [tuple(int(v) for v in r) for r in rows[:n]]

    def launch_count(self) -> int:
        return int(self.lib.omni_last_launch_count(self.ctx))

    def launch_times(self, max_n: int = 1 << 16):
        """(ms, kind, tag, work) arrays of every timed launch of the last call."""
        ms = np.zeros(max_n, np.float64)
        kinds = np.zeros(max_n, np.int32)
        tags = np.zeros(max_n, np.int32)
        work = np.zeros(max_n, np.float64)
        n = self.lib.omni_get_launch_times(self.ctx, max_n, ms.ctypes.data_as(C.c_void_p),
                                           kinds.ctypes.data_as(C.c_void_p),
                                           tags.ctypes.data_as(C.c_void_p),
                                           work.ctypes.data_as(C.c_void_p))
        if n < 0:
            raise L.OmniError(L.ECUDA, "omni_get_launch_times failed")
        return ms[:n], kinds[:n], tags[:n], work[:n]


class OmniSegLoss(torch.autograd.Function):
    """loss = OmniSegLoss.apply(segmenter, rgb, gts, *params): the stitched
    soft-Dice + BCE loss as a differentiable function of the controller, the
    pre-head and the last decoder block (in the order of _lib.GRAD_FIELDS).

    The parameter tensors are the source of truth: each must have the shape of
    its gradient (``Segmenter.grad_shapes``), and when any differs from the
    weights loaded into ``segmenter`` (an optimizer stepped them), forward
    writes them into the segmenter's blob and reloads it before evaluating, so
    loss and gradients always belong to the values passed in.  Forward and
    backward both come from one omni_backward call."""

    @staticmethod
    def forward(ctx, seg, rgb, gts, *params):
        names = L.GRAD_FIELDS
        if len(params) != len(names):
            raise ValueError("OmniSegLoss takes %d parameter tensors (%s), got %d"
                             % (len(names), ", ".join(names), len(params)))
        shapes = seg.grad_shapes()
        offs = seg.grad_offsets()
        blob = None
        for k, p in zip(names, params):
            if tuple(p.shape) != tuple(shapes[k]):
                raise ValueError("parameter %s has shape %s, the network needs %s"
                                 % (k, tuple(p.shape), tuple(shapes[k])))
            v = p.detach().to("cpu", torch.float32).contiguous().numpy().ravel()
            cur = seg.blob[offs[k]:offs[k] + v.size]
            if not np.array_equal(v, cur):
                if blob is None:
                    blob = seg.blob.copy()
                blob[offs[k]:offs[k] + v.size] = v
        if blob is not None:
            seg.load_weights(blob)
        loss, grads = seg.backward(rgb, gts)
        ctx.grads = [grads[k] for k in names]
        return loss[0]

    @staticmethod
    def backward(ctx, gout):
        return (None, None, None) + tuple(gout * g for g in ctx.grads)


def tile_slide_noalloc(work, rgb: torch.Tensor) -> Dict[str, torch.Tensor]:
    """omni_tile_slide_noalloc: tiling with the library's static scratch
    (no workspace, no device allocation inside the call)."""
    cfg = make_config(work)
    H, W, _ = rgb.shape
    s = L.Sizes()
    L.check(L.lib().omni_query(C.byref(cfg), H, W, C.byref(s)), None, "omni_query: bad size")
    dev = rgb.device
    n = s.n_tiles_max
    out = dict(tiles=torch.zeros((n, 3), dtype=torch.int32, device=dev),
               counts=torch.zeros(1 + cfg.n_scales, dtype=torch.int32, device=dev),
               flags=torch.zeros(n, dtype=torch.uint8, device=dev),
               tissue=torch.zeros((s.thumb_h, s.thumb_w), dtype=torch.uint8, device=dev),
               otsu=torch.zeros(1, dtype=torch.int32, device=dev))
    tl = L.TileList(out["tiles"].data_ptr(), out["counts"].data_ptr(), out["flags"].data_ptr(),
                    out["tissue"].data_ptr(), out["otsu"].data_ptr())
    L.check(L.lib().omni_tile_slide_noalloc(C.byref(cfg), _ptr(rgb), H, W, rgb.stride(0),
                                            C.byref(tl), _stream()),
            None, "omni_tile_slide_noalloc rejected the call")
    return out


# Class colours of the stained product (PTC, VES, PT, DT, TUFT, CAP), 50% opacity.
STAIN_COLOURS = ((230, 25, 75), (60, 180, 75), (255, 225, 25), (0, 130, 200), (245, 130, 48),
                 (145, 30, 180))


def stain(rgb: torch.Tensor, labels: Dict[int, torch.Tensor], factors: Dict[int, int],
          colours=None, alpha=128, out40: Optional[torch.Tensor] = None, down: int = 4,
          outd: Optional[torch.Tensor] = None, want40: bool = True, want_down: bool = True):
    """omni_stain: stain the class label maps onto the 40x slide (Sec. 2.3) and
    resize the stained image by ``down`` (the 10x product for 4).

    ``labels``: class id -> u8 device map at that class's scale; ``factors``:
    class id -> its downsample factor.  Maps are applied in ascending class id.
    Returns (stained 40x image or None, resized image or None)."""
    H, W, _ = rgb.shape
    ids = sorted(labels)
    n = len(ids)
    cols = colours if colours is not None else [STAIN_COLOURS[c % len(STAIN_COLOURS)] for c in ids]
    alphas = alpha if isinstance(alpha, (list, tuple)) else [alpha] * n
    dev = rgb.device
    if want40 and out40 is None:
        out40 = torch.empty((H, W, 3), dtype=torch.uint8, device=dev)
    if want_down and outd is None:
        outd = torch.empty((-(-H // down), -(-W // down), 3), dtype=torch.uint8, device=dev)
    maps = (C.c_void_p * max(n, 1))(*[labels[c].data_ptr() for c in ids])
    fac = np.array([factors[c] for c in ids] or [1], dtype=np.int32)
    col = np.array(cols or [(0, 0, 0)], dtype=np.uint8).reshape(-1)
    alp = np.array(alphas or [0], dtype=np.int32)
    L.check(L.lib().omni_stain(_ptr(rgb), H, W, rgb.stride(0), n, maps,
                               fac.ctypes.data_as(C.c_void_p), col.ctypes.data_as(C.c_void_p),
                               alp.ctypes.data_as(C.c_void_p),
                               _ptr(out40) if want40 else None, out40.stride(0) if want40 else 0,
                               down, _ptr(outd) if want_down else None,
                               outd.stride(0) if want_down else 0, _stream()),
            None, "omni_stain: bad arguments")
    return (out40 if want40 else None), (outd if want_down else None)


def synth_slide(spec, y0: int = 0, x0: int = 0, h: Optional[int] = None,
                w: Optional[int] = None, device="cuda", out: Optional[torch.Tensor] = None):
    """Window of a seeded synthetic slide generated on the device."""
    h = spec.H if h is None else h
    w = spec.W if w is None else w
    if out is None:
        out = torch.empty((h, w, 3), dtype=torch.uint8, device=device)
    ell = np.ascontiguousarray(spec.as_int_array(), dtype=np.int64)
    st = L.lib().omni_synth_slide(ell.ctypes.data_as(C.c_void_p), ell.shape[0],
                                  C.c_uint64(spec.seed & 0xFFFFFFFFFFFFFFFF), int(spec.structures), spec.W,
                                  y0, x0, h, w, _ptr(out), out.stride(0), _stream())
    L.check(st, None, "omni_synth_slide failed")
    return out


def conv_layer(precision: int, x: torch.Tensor, R: int, cin: int, cout: int, w: np.ndarray,
               g: np.ndarray, b: np.ndarray, y: torch.Tensor, r: Optional[torch.Tensor] = None,
               cr: int = 0, wp: Optional[np.ndarray] = None, x_cs=None, x_co=0, r_cs=None,
               r_co=0, y_cs=None, y_co=0, repeat: int = 1, config=None) -> float:
    """One fused conv layer through omni_conv_layer; returns ms per launch.
    config: None (default kernel choice) or a (kind, N tile, chunk, stages)
    row of conv_candidates.  precision E4M3 (the 8-bit experiment): x and y
    BF16, no residual, config (0 or 8, 128 or 256, 128, 0)."""
    B = x.shape[0]
    w = np.ascontiguousarray(w, np.float32)
    g = np.ascontiguousarray(g, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    wpp = None if wp is None else np.ascontiguousarray(wp, np.float32)
    cfg = None if config is None else np.ascontiguousarray(config, np.int32)
    ms = C.c_float(0.0)
    st = L.lib().omni_conv_layer(
        precision, B, R, cin, cout, _ptr(x), x_cs or cin, x_co, w.ctypes.data_as(C.c_void_p),
        g.ctypes.data_as(C.c_void_p), b.ctypes.data_as(C.c_void_p), _ptr(r), r_cs or cr, r_co, cr,
        None if wpp is None else wpp.ctypes.data_as(C.c_void_p), _ptr(y), y_cs or cout, y_co,
        None if cfg is None else cfg.ctypes.data_as(C.c_void_p), repeat, C.byref(ms), _stream())
    L.check(st, None, "omni_conv_layer failed")
    return ms.value


def conv_candidates(R: int, cin: int, cout: int, cr: int = 0):
    """Legal tensor-core configurations of a conv shape: (kind, N tile, chunk, stages) rows."""
    rows = np.zeros((16, 4), np.int32)
    n = L.lib().omni_conv_candidates(R, cin, cout, cr, rows.ctypes.data_as(C.c_void_p), 16)
    return [tuple(int(v) for v in rows[i]) for i in range(n)]
