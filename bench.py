"""Benchmark: segmented slide Mpx/s on the needle-biopsy workload.

One step = one call of omni_segment_slide on a 16384 x 49152 synthetic 40x
slide (805.3 Mpx): tiling, pyramid, the residual U-Net + dynamic heads on every
foreground tile at 40x / 10x / 5x, and stitching + labels for all 6 classes.
The slide (2.4 GB) is larger than L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORK = synth.NEEDLE


def describe(w) -> str:
    if w.strides:
        st = "strides " + "/".join(str(x) for x in w.strides) + " per scale, majority vote"
    else:
        st = f"stride {w.S}"
    return (f"needle-biopsy slide {w.H}x{w.W} at 40x, scales 40x/10x/5x, tiles "
            f"{w.P} {st}, residual U-Net base {w.base} x {w.levels} levels, "
            f"6 class heads, tissue filter on")


WORKLOAD = describe(WORK)
METRIC = "segmented slide Mpx/s (6 classes x 3 scales)"


def code_digest(path):
    """SHA-256 of a C++ source with its comments and runs of white space
    removed: the counters depend on the code, not on how it is commented."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return hashlib.sha256(" ".join(text.split()).encode()).hexdigest()


def conv_traffic(bf16, tiles_per_step, conv_launches_per_step):
    """DRAM bytes of the conv kernels from the committed ncu counters (per
    foreground tile), valid only while the conv code is the one captured."""
    p = os.path.join(ROOT, "profiles", "conv_traffic_needle_bf16.json")
    src = os.path.join(ROOT, "paper_2305_14566_gb300", "csrc", "conv_tc_impl.cuh")
    if not bf16 or not os.path.exists(p) or conv_launches_per_step <= 0:
        return None, None
    d = json.load(open(p))
    if code_digest(src) != d.get("conv_code_sha256"):
        return None, None
    per_step = d["bytes_per_tile"] * tiles_per_step
    return per_step / conv_launches_per_step, per_step


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        if self.p is None:
            return None
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        loaded = [r[0] for r in rows]
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(value: float, device="cpu") -> float:
    """Largest value over all ranks of the current process group (or the value
    itself without one): the step time of a multi-GPU run is its slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(mpx_per_rank: float, ms_step_max: float, world: int) -> float:
    """Whole-job throughput: every rank segments its own slide (weak scaling),
    so the job processes world * mpx_per_rank per slowest-rank step."""
    return mpx_per_rank * world / (ms_step_max / 1e3)


def tag_name(t: int) -> str:
    if t < 100:
        return f"conv enc{t // 10}.{t % 10 + 1}"
    if t < 200:
        return f"conv dec{(t - 100) // 10}.{t % 10 + 1}"
    if t == 401:
        return "gap+controller"
    names = {2: "maxpool", 3: "upsample", 4: "gap", 5: "head", 6: "stitch", 7: "prep"}
    return names.get(t // 100, str(t))


def summarize(ms, tags, work, steps):
    """Per-layer device time per step (ms) and achieved TFLOP/s for convs."""
    out = {}
    for t in sorted(set(int(x) for x in tags)):
        m = tags == t
        k = tag_name(t)
        e = out.setdefault(k, {"ms": 0.0, "launches": 0, "flop": 0.0})
        e["ms"] += float(ms[m].sum()) / steps
        e["launches"] += int(m.sum()) // steps
        e["flop"] += float(work[m].sum()) / steps
    for e in out.values():
        e["tflops"] = round(e["flop"] / (e["ms"] / 1e3) / 1e12, 1) if e["flop"] and e["ms"] else None
        e["ms"] = round(e["ms"], 2)
        del e["flop"]
    return out


def run_layer(args):
    """One fused conv layer (same kernel as the slide path) launched back to
    back: the small case used for the tensor-core kernel's ncu capture."""
    import torch
    from paper_2305_14566_gb300.build import build
    build()
    from paper_2305_14566_gb300 import api, _lib
    vals = [int(v) for v in args.layer.split(",")]
    R, cin, cout, cr, B, rep = vals[:6]
    config = tuple(vals[6:10]) if len(vals) == 10 else None   # kind, N tile, chunk, stages
    rng = np.random.default_rng(0)
    prec = {"bf16": _lib.BF16, "fp16": _lib.FP16, "fp32": _lib.FP32, "e4m3": _lib.E4M3}[args.precision]
    dt = {"bf16": torch.bfloat16, "fp16": torch.float16, "fp32": torch.float32,
          "e4m3": torch.bfloat16}[args.precision]      # E4M3: BF16 activations in and out
    x = torch.rand((B, R, R, cin), device="cuda").to(dt)
    r = torch.rand((B, R, R, cr), device="cuda").to(dt) if cr else None
    y = torch.empty((B, R, R, cout), device="cuda", dtype=dt)
    w = (rng.standard_normal((cout, cin, 3, 3)) * np.sqrt(2 / (9 * cin))).astype(np.float32)
    g = np.ones(cout, np.float32)
    b = np.zeros(cout, np.float32)
    wp = (rng.standard_normal((cout, cr)) * np.sqrt(1 / cr)).astype(np.float32) if cr else None
    api.conv_layer(prec, x, R, cin, cout, w, g, b, y, r, cr, wp, repeat=1, config=config)
    ms = api.conv_layer(prec, x, R, cin, cout, w, g, b, y, r, cr, wp, repeat=rep, config=config)
    fl = 2.0 * B * R * R * cout * (9 * cin + cr)
    pk, src = peaks()
    tf = fl / (ms / 1e3) / 1e12
    line = {"layer": {"R": R, "cin": cin, "cout": cout, "cr": cr, "B": B,
                      "config": list(config) if config else "default"},
            "precision": args.precision, "ms_per_launch": ms, "tflops": tf,
            "frac_of_bf16_burst": tf / pk["bf16_tflops"], "peak_source": src}
    if prec == _lib.E4M3:
        # E4M3 peak: the measured BF16 burst times the nominal 4.5 / 2.25 ratio
        line["frac_of_e4m3_burst"] = tf / (2.0 * pk["bf16_tflops"])
    print(json.dumps(line))


def run_ragged(args, api, _lib, dev, prec):
    """Twelve synthetic slides (long side U[8192, 49152], aspect U[1, 4], tissue
    U[0.2, 0.6]); one step segments all of them in ONE omni_segment_slides
    call: every slide is tiled, then the foreground tiles of all slides share
    the network batches of each scale, and the whole post-tiling chain is one
    captured CUDA graph.  Per-slide latency = completion of the slide's last
    stitch band after the chain's start (events inside the graph)."""
    import torch
    works = synth.ragged_workloads()
    blob = synth.gen_weights(works[0])
    seg = api.Segmenter(works[0], blob, precision=prec)
    if prec != _lib.FP32 and not args.no_autotune:
        seg.set_autotune(True)
    rgbs = [api.synth_slide(synth.spec_for(w), device=dev) for w in works]
    outs = seg.segment_many(rgbs)            # tunes every conv shape
    torch.cuda.synchronize()
    seg.set_graphs(True)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        for _ in range(max(2, args.warmup)):  # the second call captures the graph
            seg.segment_many(rgbs, outs=outs)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        per = []
        with Clocks(0) as clk:
            e0.record()
            for _ in range(args.steps):
                seg.segment_many(rgbs, outs=outs)
            e1.record()
            torch.cuda.synchronize()
        # per-slide completion stamps of one more (untimed) step
        seg.segment_many(rgbs, outs=outs)
        per.append(seg.slide_times())
    total_ms = e0.elapsed_time(e1) / args.steps
    mpx = sum(w.H * w.W for w in works) / 1e6
    lat = np.mean(np.array(per), axis=0) if per else None
    print(json.dumps({"metric": "ragged 12-slide segmentation Mpx/s", "value": mpx / (total_ms / 1e3),
                      "unit": "Mpx/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": total_ms, "higher_is_better": True, "dtype": args.precision,
                      "data": "synthetic",
                      "config": {"workload": "12 ragged needle-like slides, seeds 100-111, one "
                                             "omni_segment_slides call per step (tiles of all slides "
                                             "share batches; one CUDA graph after tiling)",
                                 "slides": [[w.H, w.W, round(w.tissue, 3)] for w in works]},
                      "per_slide_done_ms": None if lat is None else [round(float(v), 2) for v in lat],
                      "clocks": clk.summary()}))
    seg.close()


def run_large(args, api, _lib, dev, prec):
    """The large throughput sweep: four 32768x98304 needle-biopsy slides (35% tissue,
    seeds 200-203) with 1024-px tiles at stride 512; one step segments all four.
    With --compare-fp32 the first slide is also segmented by the plain FP32 path
    and the per-class label agreement and Dice against it are reported."""
    import torch
    works = [synth.LARGE.with_(name=f"large{k}", seed=200 + k) for k in range(4)]
    blob = synth.gen_weights(works[0])
    seg = api.Segmenter(works[0], blob, precision=prec)
    if prec != _lib.FP32 and not args.no_autotune:
        seg.set_autotune(True)
    if args.e4m3:
        seg.set_e4m3(True)
    seg.workspace(seg.query(works[0].H, works[0].W).workspace_bytes, dev)
    rgbs = [api.synth_slide(synth.spec_for(w), device=dev) for w in works]
    outs = [seg.segment(r) for r in rgbs]
    torch.cuda.synchronize()
    for _ in range(max(0, args.warmup - 1)):
        for r, o in zip(rgbs, outs):
            seg.segment(r, out=o)
    torch.cuda.synchronize()
    seg.set_timing(True)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        t0.record()
        for _ in range(args.steps):
            for r, o in zip(rgbs, outs):
                seg.segment(r, out=o)
        t1.record()
        torch.cuda.synchronize()
    conv_ms, conv_n, conv_flops = seg.timing(0)
    seg.set_timing(False)
    ms_step = t0.elapsed_time(t1) / args.steps
    mpx = sum(w.H * w.W for w in works) / 1e6
    pk, src = peaks()
    peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
    achieved = conv_flops / (conv_ms / 1e3) / 1e12 if conv_ms else None
    line = {"metric": "large 4-slide segmentation Mpx/s", "value": mpx / (ms_step / 1e3), "unit": "Mpx/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "4 needle-biopsy slides 32768x98304 at 40x, 35% tissue, tiles 1024 "
                                   "stride 512, base 32 x 5 levels, 6 heads", "slides_mpx": mpx,
                       "tiles_per_step": int(round(conv_flops / args.steps /
                                                   seg.query(works[0].H, works[0].W).flops_per_tile))},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak if achieved else None, "traffic": None,
                         "kernel": "conv (all U-Net layers)", "peak_source": f"bf16 dense sustained ({src})"},
            "memory": {"workspace_bytes": int(seg.query(works[0].H, works[0].W).workspace_bytes),
                       "max_batch": int(works[0].max_batch)},
            "clocks": clk.summary()}
    if args.e4m3:
        line["e4m3"] = ("experiment: enc3.1, enc4.1, dec2.1 and dec3.1 on E4M3 operands (per-call "
                        "activation scale, per-channel weight scales), the rest BF16")
    if args.compare_fp32 and prec != _lib.FP32:
        keep = {c: t.clone() for c, t in outs[0]["labels"].items()}
        seg.close()
        seg._ws = None                     # the BF16 workspace
        del outs, seg
        rgbs = rgbs[:1]
        torch.cuda.empty_cache()
        seg32 = api.Segmenter(works[0], blob, precision=_lib.FP32)
        o32 = seg32.segment(rgbs[0])
        torch.cuda.synchronize()
        rows = []
        for c, lab in keep.items():
            a, b = lab > 0, o32["labels"][c] > 0
            den = int(a.sum().item() + b.sum().item())
            inter = int((a & b).sum().item())
            rows.append({"class": int(c), "agree": float((a == b).float().mean().item()),
                         "dice": 1.0 if den == 0 else 2.0 * inter / den, "positives_fp32": int(b.sum().item())})
        line["labels_vs_fp32_slide0"] = rows
        seg32.close()
    else:
        seg.close()
    print(json.dumps(line))


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _crop_origin():
    """40x origin of the needle crop the oracle tests use (written by
    tests/golden/make_needle_crop.py), else a fixed tissue-rich one."""
    p = os.path.join(ROOT, "tests", "golden", "needle_crop.npz")
    if os.path.exists(p):
        d = np.load(p)
        return int(d["origin"][0]), int(d["origin"][1])
    return 8192, 24576


def oracle_sample(per_scale: int = 1):
    """The FP64 oracle on a bounded sample of the needle workload: ``per_scale``
    foreground tiles of every scale taken from the 2048 x 2048 crop (U-Net,
    GAP, controller and the scale's two heads, then the stitch of those
    tiles).  Returns (seconds per tile per scale, the sample's description)."""
    import torch
    from oracle import omniseg_oracle as O
    torch.set_num_threads(_host_cores())
    spec = synth.spec_for(WORK)
    blob = synth.gen_weights(WORK)
    p = O.weights_f64(WORK, blob)
    y0, x0 = _crop_origin()
    per = []
    for s, f in enumerate(WORK.factors):
        P, S = WORK.P, WORK.stride(s)
        span = P * f
        # tiles whose 40x footprint starts inside the crop, on the scale's grid
        ty = (y0 // (S * f)) * S * f
        tiles = [(ty // f, (x0 // (S * f)) * S * f // f + k * S) for k in range(per_scale)]
        # the synthetic 40x windows are inputs: generated before the clock starts
        wins = [synth.gen_window(spec, y * f, x * f, span, span) for (y, x) in tiles]
        t0 = time.perf_counter()
        lg = {}
        for (y, x), img in zip(tiles, wins):
            g = f
            while g > 1:
                img = O.half(img)
                g //= 2
            out, _ = O.patch_forward(img[None], p, WORK, s)
            lg[(0, x - tiles[0][1])] = out[0, 0].numpy()
        O.stitch(lg, P, P + S * (per_scale - 1), P)
        per.append((time.perf_counter() - t0) / len(tiles))
    return per, (f"{per_scale} tile(s) of each scale (40x, 10x, 5x) from the 2048x2048 needle crop at "
                 f"{y0},{x0}: FP64 pyramid halvings, U-Net, GAP, controller, the scale's two heads and "
                 f"their stitch (the synthetic input windows are generated outside the timing)")


def oracle_slide_rate(per_tile_s):
    """Mpx/s the oracle would reach on the whole needle slide: the measured time
    per tile of each scale times the slide's foreground tiles of that scale
    (the oracle's own counts, tests/golden/needle_tiles.json)."""
    gold = os.path.join(ROOT, "tests", "golden", "needle_tiles.json")
    counts = json.load(open(gold))["tiles_per_scale"]
    secs = sum(t * n for t, n in zip(per_tile_s, counts))
    return WORK.H * WORK.W / 1e6 / secs, counts


def cpu_baseline():
    oracle_sample()                      # warm-up pass: first-call allocation and thread start-up
    per, sample = oracle_sample()
    v, counts = oracle_slide_rate(per)
    return {"value": v, "unit": "Mpx/s", "cores": _host_cores(), "kind": "oracle",
            "sample": sample + "; seconds per tile " + ", ".join(f"{t:.2f}" for t in per) +
                      f", scaled by the slide's {'/'.join(str(n) for n in counts)} foreground tiles"}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores.  Each step times
    one tile of every scale of the needle crop and converts it to the slide
    rate; W untimed steps, then K timed ones; the value is their median."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample()
    vals, sample = [], ""
    for _ in range(args.steps):
        per, sample = oracle_sample()
        vals.append(oracle_slide_rate(per)[0])
    v = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mpx/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"kind": "oracle", "cores": _host_cores(), "sample": sample,
                             "value": v, "unit": "Mpx/s"},
            "e2e": {"value": v, "unit": "Mpx/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp16", "fp32", "e4m3"],
                    help="e4m3: the 8-bit experiment, --layer only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true",
                    help="skip the step of the plain FP32 path that the line reports as fp32_plain")
    ap.add_argument("--e4m3", action="store_true",
                    help="with --large: the E4M3 experiment (the deeper levels' first convs on 8-bit operands)")
    ap.add_argument("--compare-fp32", action="store_true",
                    help="--large: also segment the first slide with the FP32 path and compare labels")
    ap.add_argument("--ragged", action="store_true",
                    help="the 12-slide ragged workload: per-slide latency and aggregate Mpx/s")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--large", action="store_true",
                    help="the large sweep: four 32768x98304 slides, 1024-px tiles (its own JSON line)")
    ap.add_argument("--workload", default="needle", choices=["needle", "small"],
                    help="small: a 2048x8192 slice of the needle configuration, for multi-pass ncu "
                         "captures that must stay a few GB (never a bench line)")
    ap.add_argument("--paper-strides", action="store_true",
                    help="the needle slide tiled with the per-scale strides of Sec. 3.2 (256 at 40x, "
                         "64 at 10x and 5x) and majority-vote labels (its own JSON line)")
    ap.add_argument("--profile-step", action="store_true",
                    help="one slide step after the tuning call, bracketed by cudaProfilerStart/Stop "
                         "(for ncu --profile-from-start off)")
    ap.add_argument("--max-batch", type=int, default=0, help="tiles per network batch (0: the workload's)")
    ap.add_argument("--layer", default=None,
                    help="R,cin,cout,cr,B,repeat[,kind,N tile,chunk,stages]: time one fused conv layer "
                         "instead (optionally one tensor-core configuration of omni_conv_candidates)")
    args = ap.parse_args()
    if args.layer:
        run_layer(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist
    from paper_2305_14566_gb300.build import build
    build()
    from paper_2305_14566_gb300 import api, _lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    if args.precision == "e4m3":
        raise SystemExit("--precision e4m3 is the layer experiment: use it with --layer")
    prec = {"bf16": _lib.BF16, "fp16": _lib.FP16, "fp32": _lib.FP32}[args.precision]

    if args.ragged:
        run_ragged(args, api, _lib, dev, prec)
        return
    if args.large:
        run_large(args, api, _lib, dev, prec)
        return
    base_work = synth.NEEDLE_PAPER if args.paper_strides else WORK
    work = base_work if args.workload == "needle" else base_work.with_(name="needle_small", H=2048, W=8192)
    if work is not base_work and not args.profile_step:
        raise SystemExit("--workload small is for --profile-step captures only")
    spec = synth.spec_for(work)
    rgb = api.synth_slide(spec, device=dev)
    blob = synth.gen_weights(work)
    seg = api.Segmenter(work, blob, precision=prec, max_batch=args.max_batch or None)
    if prec != _lib.FP32 and not args.no_autotune:
        seg.set_autotune(True)          # the first (untimed) call tunes every conv shape
    out = seg.segment(rgb)
    torch.cuda.synchronize()
    if args.profile_step:
        # one step after tuning, bracketed for `ncu --profile-from-start off`
        seg.segment(rgb, out=out)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        seg.segment(rgb, out=out)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile_step": True, "workload": work.name, "launches": seg.launch_count()}))
        seg.close()
        return

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        seg.segment(rgb, out=out)
    barrier()
    # eager steps with per-launch CUDA events (the library records them on the
    # launching stream): per-layer breakdown, conv roofline, stitch bandwidth
    n_inst = max(1, min(args.steps, 3))
    seg.set_timing(True)
    i0 = torch.cuda.Event(enable_timing=True)
    i1 = torch.cuda.Event(enable_timing=True)
    i0.record()
    for _ in range(n_inst):
        seg.segment(rgb, out=out)
    i1.record()
    barrier()
    conv_ms, conv_n, conv_flops = seg.timing(0)
    st_ms, _, st_bytes = seg.timing(1)
    ms_l, kinds_l, tags_l, work_l = seg.launch_times()
    seg.set_timing(False)
    eager_ms = i0.elapsed_time(i1) / n_inst
    mpx = work.H * work.W / 1e6
    breakdown = summarize(ms_l, tags_l, work_l, n_inst)

    # the timed steps: tiling, then the network and stitch replayed from the
    # CUDA graph the library captured on the second call (on a created stream;
    # the legacy default stream cannot be captured)
    seg.set_graphs(True)
    gstream = torch.cuda.Stream()
    gstream.wait_stream(torch.cuda.current_stream())
    launches = 0
    with torch.cuda.stream(gstream):
        for _ in range(2 + args.warmup):
            seg.segment(rgb, out=out)      # key, capture, then W warm-up replays
        barrier()
        with Clocks(local) as clk:
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            barrier()
            t0.record()
            for _ in range(args.steps):
                seg.segment(rgb, out=out)
                launches += seg.launch_count()
            t1.record()
            barrier()
    seg.set_graphs(False)
    clocks = clk.summary()
    ms_step = max_over_ranks(t0.elapsed_time(t1) / args.steps, device=dev)
    value = whole_job_value(mpx, ms_step, world)

    pk, src = peaks()
    if prec != _lib.FP32:
        # FP16 and BF16 share the kind::f16 tensor-core rate
        peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
        bound, peak_note = "tensor", f"bf16 dense sustained ({src}); fp16 runs at the same rate"
    else:
        peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        bound, peak_note = "alu", "FP32 FFMA: 152 SMs x 128 lanes x 2 x max SM clock"
    conv_per_launch_ms = conv_ms / max(conv_n, 1)
    achieved = (conv_flops / max(conv_n, 1)) / (conv_per_launch_ms / 1e3) / 1e12
    tiles_step = int(round(conv_flops / n_inst / seg.query(work.H, work.W).flops_per_tile))
    traffic, traffic_step = conv_traffic(prec == _lib.BF16, tiles_step, conv_n / n_inst)
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": "conv (all U-Net layers)",
            "peak_source": peak_note,
            "traffic_note": ("DRAM bytes per conv launch, averaged over a step; from the ncu counters of a "
                             "2048x8192 slice scaled by foreground tiles" if traffic else
                             "no ncu counters for this conv build / precision"),
            "traffic_per_step": traffic_step,
            "share_of_step": conv_ms / n_inst / eager_ms}
    stitch = {"achieved_gbs": st_bytes / (st_ms / 1e3) / 1e9 if st_ms else None,
              "peak_gbs": pk["hbm_gbs"], "ms_per_step": st_ms / n_inst}

    eager = {"value": mpx * world / (eager_ms / 1e3), "unit": "Mpx/s", "ms_per_step": eager_ms,
             "steps": n_inst, "note": "eager launches with per-launch events (breakdown, roofline)"}

    # the stained 40x product and its 10x resize (Sec. 2.3), one HBM pass
    fac = {c: work.factors[s] for c, s in enumerate(work.class_scale)}
    s40, s10 = api.stain(rgb, out["labels"], fac)
    for _ in range(2):
        api.stain(rgb, out["labels"], fac, out40=s40, outd=s10)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        api.stain(rgb, out["labels"], fac, out40=s40, outd=s10)
    e1.record()
    torch.cuda.synchronize()
    st_ms1 = e0.elapsed_time(e1) / 3
    st_b = 2 * rgb.numel() + s10.numel() + sum(t.numel() for t in out["labels"].values())
    stain = {"ms": st_ms1, "bytes": int(st_b), "achieved_gbs": st_b / (st_ms1 / 1e3) / 1e9,
             "peak_gbs": pk["hbm_gbs"], "frac": st_b / (st_ms1 / 1e3) / 1e9 / pk["hbm_gbs"],
             "note": "omni_stain: 6 class maps onto the 40x slide + the 4x4-resized 10x image; "
                     "outside the timed step"}
    del s40, s10

    # end to end through the host-buffer entry point (pinned host memory)
    rgb_h = rgb.cpu().pin_memory()
    labs = {c: torch.empty(tuple(out["labels"][c].shape), dtype=torch.uint8).pin_memory()
            for c in out["labels"]}
    seg.segment_host(rgb_h, labs, device=dev)
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        seg.segment_host(rgb_h, labs, device=dev)
    barrier()
    e2e_s = (time.perf_counter() - w0) / e2e_steps
    e2e = {"value": mpx * world / e2e_s, "unit": "Mpx/s",
           "h2d_bytes_per_step": int(rgb_h.numel()),
           "d2h_bytes_per_step": int(sum(t.numel() for t in labs.values()))}
    del rgb_h, labs

    tuned_rows = [list(t) for t in seg.tuned()]
    fp32 = None
    if not args.no_fp32 and prec != _lib.FP32 and world == 1:
        # the plain FP32 path (FFMA convs, no tensor cores) on the same slide:
        # one untimed step, one step timed with events on the launching stream
        seg.close()
        seg._ws = None
        torch.cuda.empty_cache()
        seg32 = api.Segmenter(work, blob, precision=_lib.FP32)
        o32 = seg32.segment(rgb)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record()
        seg32.segment(rgb, out=o32)
        f1.record()
        torch.cuda.synchronize()
        ms32 = f0.elapsed_time(f1)
        fp32 = {"value": mpx / (ms32 / 1e3), "unit": "Mpx/s", "steps": 1, "ms_per_step": ms32,
                "speedup_of_value": value / (mpx / (ms32 / 1e3)),
                "note": "plain FP32 path (FFMA implicit GEMM on the CUDA cores), same slide"}
        seg32.close()
        del o32

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Mpx/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": args.precision, "data": "synthetic",
                "config": {"workload": describe(work), "slide_px": work.H * work.W,
                           "l2": "no flush: inputs (2.4 GB slide) larger than L2",
                           "parallelism": f"replicas x{world}",
                           "tiles_per_step": tiles_step},
                "roofline": roof, "stitch": stitch, "stain": stain, "e2e": e2e, "gpu_launches": int(launches),
                "memory": {"workspace_bytes": int(seg.query(work.H, work.W).workspace_bytes),
                           "max_batch": int(args.max_batch or work.max_batch),
                           "note": "device workspace of one slide call (batch activations, tile-logit ring "
                                   "of the banded stitch, pyramid, tiling); the slide and outputs are the "
                                   "caller's"},
                "breakdown": breakdown, "eager": eager,
                "autotuned": tuned_rows,
                "clocks": clocks}
        if fp32 is not None:
            line["fp32_plain"] = fp32
        if world == 1 and not args.no_cpu_baseline and not args.paper_strides:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line))
    seg.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
