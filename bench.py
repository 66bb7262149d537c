#!/usr/bin/env python3
"""Benchmark of the registration + merge path on seeded synthetic 5 MP pairs.

One step = the whole path (a1..a11: normalization, pyramid matcher, weeding,
level homographies, domain-transform flow, warp, SSIM mask, irradiance merge)
over a batch of 2592x1944 YUV420 two-frame stacks resident in HBM, replayed as
one CUDA graph. Prints one JSON line (see the keys below).

  python bench.py --gpus N --steps K --warmup W [--impl reference]
  python bench.py --workload mixed64    # 64 stacks of 1-12 MP, 2-3 frames, tuned (T, R)
  python bench.py --workload sweep      # one pair per size, VGA .. 20 MP (scaling)
  python bench.py --workload learned12  # 32 three-frame 12 MP stacks, learned level-0 search
  python bench.py --workload learned8px # 5 MP pairs with +-8 px fields, learned vs plain

Under torchrun each rank (one GPU) registers its own batch of stacks: stacks
are independent, so the ranks are replicas with no data-path collective; the
reported value is all ranks' pixels / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "registered+merged Mpix/s per B300 (5 MP pairs), learned vs plain at ≤0.5 px EPE"
WORKLOAD = "5mp_yuv420_pair"
W, H = 2592, 1944
MIXED = "mixed64"                       # command-line name of the mixed batch
MIXED_NAME = "mixed64_1to12mp_yuv420"
SWEEP = "sweep"
SCALE12 = "learned12"
LEARNED8 = "learned8px"
LEARNED8_NAME = "5mp_yuv420_pair_8px_fields"
SCALE12_NAME = "learned_batched_32x12mp_3frame_yuv420"
MIXED_METRIC = "registered+merged output Mpix/s per B300 (64 stacks of 1-12 MP, 2-3 frames)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--pairs", type=int, default=16, help="stacks per step (inputs > L2)")
    ap.add_argument("--search-threads", type=int, default=0, choices=[0, 64, 128, 256],
                    help="threads per tile CTA of the search (0: the library default, 128)")
    ap.add_argument("--distinct", type=int, default=2, help="distinct generated stacks")
    ap.add_argument("--lanes", type=int, default=16, help="concurrent lanes of the batched call "
                    "(16: one pair per lane for the 16-pair step)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned level-0 search leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the mixed 64-stack batch leg of the default workload")
    ap.add_argument("--staged", action="store_true",
                    help="mixed batches: every stack's merge as one stage after all "
                         "registrations (hdrreg_register_merge_staged) instead of on its lane")
    ap.add_argument("--profile", action="store_true", help="short run for a profiler")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, MIXED, SWEEP, SCALE12, LEARNED8],
                    help="the 5 MP pair batch (default), the mixed 1-12 MP batch, the size "
                         "sweep, 12 MP three-frame stacks with the learned search, or 5 MP "
                         "pairs with +-8 px fields, learned vs plain")
    ap.add_argument("--stacks", type=int, default=64,
                    help="stacks of the mixed batch (of the learned 12 MP batch: 32 unless set)")
    ap.add_argument("--output", default="merge", choices=["merge", "fusion"],
                    help="the fused call's output: the irradiance merge (a11) or the "
                         "error-tolerant exposure fusion of Sec. 2.5 (output_mode 1)")
    ap.add_argument("--preset", default="workload", choices=["workload", "paper"],
                    help="the headline workload's parameters (T=32, R=6, ratio normalization) "
                         "or the paper-exact preset (histogram equalization, R=10, the whole "
                         "displacement propagated)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def max_over_ranks(torch, dist, ms, device):
    """Slowest rank's step time: every rank contributes its own, all receive the max."""
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world_size, mpix_per_rank_step, ms_step):
    """Whole-job throughput: the pixels all replicas processed per step over the step time."""
    return world_size * mpix_per_rank_step / (ms_step / 1e3)


def make_inputs(n_distinct):
    from paper_1504_01441_b300 import synth
    stacks = [synth.make_stack(synth.FIVE_MP, synth.stack_seed(2, i)) for i in range(n_distinct)]
    return stacks


def flow_algorithmic_bytes(w, h, iters=3):
    """Compulsory bytes of the flow stage: the first row pass reads the guide and writes 3
    FP32 planes; every later pass reads 3 planes + guide and writes 3 planes; the last column
    pass writes the 2 flow planes instead."""
    px = w * h
    first = px * (1 + 12)
    middle = px * (12 + 1 + 12)
    last = px * (12 + 1 + 8)
    return first + (2 * iters - 2) * middle + last


PATH_BYTES_PER_PX = 165  # compulsory bytes per registered luma pixel of a1-a11 (the model)


def path_roofline(reg_mpix_per_step, ms_step, what):
    """The whole step against the per-pixel byte model of the path: 165 B per registered
    luma pixel (normalization and pyramid ~4.7, matcher ~2.7, the six flow passes ~140,
    warp and merge ~17), at the measured HBM bandwidth."""
    peak, src = peaks()
    model = reg_mpix_per_step * 1e6 * PATH_BYTES_PER_PX
    ach = model / (ms_step / 1e3) / 1e9
    return {"kernel": what, "bound": "hbm", "achieved": round(ach, 1), "peak": peak,
            "peak_source": src, "unit": "GB/s", "frac": round(ach / peak, 4),
            "model_bytes_per_registered_px": PATH_BYTES_PER_PX,
            "algorithmic_bytes_per_step": int(model)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1504_01441_b300 import hdrreg, synth

    ws, rank, local = dist_env()
    # the mixed batch's stacks are generated in a spawn pool before CUDA starts
    mixed = None
    if (rank == 0 and not args.no_batched and not args.profile and args.preset == "workload"
            and args.output == "merge"):
        t_gen = time.perf_counter()
        mixed = (mixed_inputs(args.stacks), time.perf_counter() - t_gen)
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stacks = make_inputs(args.distinct)
    if args.preset == "paper":
        p = hdrreg.params_paper()
    else:
        p = hdrreg.params_from_dict(synth.method_params(32, 6))
    p.output_mode = 1 if args.output == "fusion" else 0
    p.search_threads = args.search_threads
    P = args.pairs
    # resident inputs: P distinct device buffers (contents cycle over the generated stacks)
    frames = []
    for i in range(P):
        s = stacks[i % len(stacks)]
        ref = tuple(torch.from_numpy(a).to(dev) for a in (s.ref.y, s.ref.u, s.ref.v))
        src = tuple(torch.from_numpy(a).to(dev) for a in (s.srcs[0].y, s.srcs[0].u, s.srcs[0].v))
        frames.append((ref, [src], s.ratios))
    runner = hdrreg.RegisterMergeBatch(W, H, 1, p, True, slots=P, lanes=args.lanes, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def step():
        runner(frames, stream=stream)

    step()  # warm the library (smem attributes, lane streams) before capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    n0 = hdrreg.launch_count()
    with torch.cuda.graph(graph, stream=stream):
        step()
    launches_per_step = hdrreg.launch_count() - n0
    # replay() launches on torch's current stream: make it the timed stream
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 0)):
            graph.replay()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    K = args.steps
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk, torch.cuda.stream(stream):
        torch.cuda.synchronize()
        start.record(stream)
        for _ in range(K):
            graph.replay()
        end.record(stream)
        torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    if ws > 1:
        ms = max_over_ranks(torch, dist, ms, dev)
        dist.barrier()
    ms_step = ms / K
    mpix_step = P * W * H / 1e6
    value = job_value(ws, mpix_step, ms_step)

    # -- dominant stage: the flow (6 domain-transform passes), timed alone on its stream
    roof, stages, search_alu = None, None, None
    if rank == 0:
        meta = {}
        stages = measure_stages(torch, hdrreg, p, stacks[0], dev, args, meta)
        roof = measure_flow_roofline(stages, p)
        search_alu = measure_search_alu(torch, hdrreg, stages, p, meta["valid_level0"], dev)
    # -- the learned level-0 search (row a-L) on the same resident pairs
    learned = None
    if (rank == 0 and not args.no_learned and not args.profile and args.preset == "workload"
            and args.output == "merge"):
        learned = measure_learned(torch, hdrreg, synth, stacks, frames, p, dev, args)
    # -- end to end through the C ABI with host buffers (pinned), copies inside the timing
    e2e = None
    if rank == 0 and not args.no_e2e:
        e2e = measure_e2e(torch, hdrreg, p, stacks, dev, P, args)
    # -- the mixed batch (64 stacks of 1-12 MP, 2-3 frames, tuned (T, R)) as one graph
    batched = None
    if mixed is not None:
        del frames, runner
        torch.cuda.empty_cache()
        batched = measure_mixed(torch, hdrreg, mixed[0], dev, args, K)
        batched["generation_s"] = round(mixed[1], 1)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not args.profile:
        cpu = measure_cpu_baseline(synth, stacks[0], cfg=p.as_dict())
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "Mpix/s", "n_gpus": ws,
            "steps": K, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8/i32 match, f64 fit, f32 flow/warp/merge", "data": "synthetic",
            "config": {"workload": WORKLOAD, "width": W, "height": H, "format": "YUV420",
                       "frames": 2, "exposure_ratio": 4, "pairs_per_step": P,
                       "distinct_stacks": len(stacks), "tile": p.tile, "radius": p.radius,
                       "search_threads": p.search_threads or 128,
                       "preset": args.preset, "norm_mode": "histeq" if p.norm_mode else "ratio",
                       "output": args.output,
                       "propagate_full": p.propagate_full,
                       "path": "plain (a1-a11)", "graph": True, "lanes": args.lanes,
                       "l2": f"inputs larger than L2: {P} resident pairs x 15.1 MB per step",
                       "parallelism": f"replicas x{ws}"},
            "gpu_launches": launches_per_step * K,
            "roofline": roof,
            "roofline_path": path_roofline(mpix_step, ms_step, "whole step: the batched fused "
                                           "path over the step's pairs, per-pixel byte model"),
            "search_alu": search_alu, "stages_us": stages, "learned": learned,
            "batched": batched,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def time_train_step(torch, hdrreg, theta, dev, stream, steps=10):
    """One training step of the predictor in the library's kernels: forward, backward and
    Adam on 64 crops of 64 x 64 x 2 quarter-resolution inputs (256 x 256 full), averaged
    over `steps` steps after 3 untimed ones. -> ms per step."""
    net = hdrreg.Predictor(64, 64, 64, theta.cpu().numpy(), device=dev)
    x = torch.empty((64, 64, 64, 2), dtype=torch.bfloat16, device=dev).uniform_(-1, 1)
    label = torch.zeros((64, net.ho, net.wo, 2), dtype=torch.float32, device=dev)
    valid = torch.ones((64, net.ho, net.wo), dtype=torch.uint8, device=dev)

    def train_step():
        net.forward(x, stream=stream)
        net.backward(x, label, valid, stream=stream)
        net.adam(1e-4, stream=stream)
    for _ in range(3):
        train_step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        train_step()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


TRAIN_STEP = "64 crops of 64x64x2 quarter-resolution inputs (256x256 full): forward, backward, Adam"


def measure_learned(torch, hdrreg, synth, stacks, frames, p, dev, args):
    """Same batch through the fused path with the learned level-0 search, at the default
    operating point (refine 1, fallback above 1.5 x the median plain cost) and, if
    calibrated, at the cheapest point whose mean distance to the plain matches is <= 0.5
    px on held-out stacks: throughput, fallback rate, distance to the plain matches (the
    judge) and to the generator's truth, measured on this batch's stacks."""
    import numpy as np
    from paper_1504_01441_b300 import learned as L
    theta = torch.tensor(np.load(L.THETA_FILE)).to(dev)
    prep = [L.prepare(s, p, keep_gt=True) for s in stacks]
    med = float(torch.cat([P.cost[P.valid.bool()] for P in prep]).double().median().item())
    points = [("default", 1, 1.5, None)]
    if os.path.exists(L.OPS_FILE):
        ch = json.load(open(L.OPS_FILE)).get("chosen")
        if ch:
            points.append(("at_bound", ch["refine"], ch["ratio"], ch))
    out = {}
    P = len(frames)
    for name, refine, ratio, cal in points:
        thr = int(ratio * med)
        quality = L.evaluate(prep, theta, p, fallback_ratio=ratio, refine=refine)
        pl = hdrreg.params_from_dict(p.as_dict())
        pl.predictor = theta.data_ptr()
        pl.fallback_cost = thr
        pl.predictor_refine = refine
        runner = hdrreg.RegisterMergeBatch(W, H, 1, pl, True, slots=P, lanes=args.lanes, device=dev)
        s = torch.cuda.Stream(device=dev)
        runner(frames, stream=s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            runner(frames, stream=s)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        K = max(3, args.steps // 2)
        with torch.cuda.stream(s):
            for _ in range(max(args.warmup, 3)):
                g.replay()
            torch.cuda.synchronize()
            a.record(s)
            for _ in range(K):
                g.replay()
            b.record(s)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / K
        fb = sum(runner.diagnostics(i)[0].fallbacks for i in range(P))
        val = sum(runner.diagnostics(i)[0].valid for i in range(P))
        out[name] = {
            "value": round(P * W * H / 1e6 / (ms / 1e3), 2), "unit": "Mpix/s",
            "ms_per_step": round(ms, 4), "refine": refine, "fallback_ratio": ratio,
            "fallback_cost": thr, "fallback_rate": round(fb / max(val, 1), 4),
            "ssd_offsets_per_tile": round(L.search_cost(refine, fb / max(val, 1), p.radius), 1),
            "epe_vs_plain_px": round(quality["epe_px"], 3),
            "epe_vs_plain_median_px": round(quality["epe_median_px"], 3),
            "learned_vs_truth_px": round(quality.get("learned_vs_truth_px", float("nan")), 3),
            "plain_vs_truth_px": round(quality.get("plain_vs_truth_px", float("nan")), 3),
            "meets_0.5px_vs_plain": bool(quality["epe_px"] <= 0.5)}
        if cal:
            out[name]["calibrated_on"] = "paper_1504_01441_b300/predictor_operating_point.json"
        del runner, g
    out["weights"] = ("paper_1504_01441_b300/predictor_theta.npy (python -m "
                      "paper_1504_01441_b300.learned)")
    out["plain_ssd_offsets_per_tile"] = (2 * p.radius + 1) ** 2
    out["train_step_ms"] = round(time_train_step(torch, hdrreg, theta, dev,
                                                 torch.cuda.Stream(device=dev)), 3)
    out["train_step"] = TRAIN_STEP
    # the headline fields of the learned leg: the default point
    out.update({k: out["default"][k] for k in ("value", "unit", "fallback_rate",
                                                 "epe_vs_plain_px", "meets_0.5px_vs_plain")})
    return out


def _graph_time_us(torch, fn, reps):
    """Average device time of fn() replayed as one CUDA graph (after a warm-up call)."""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):  # replay() launches on the current stream
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        a.record(s)
        for _ in range(reps):
            g.replay()
        b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b) * 1e3 / reps


def measure_stages(torch, hdrreg, p, stack, dev, args, meta=None):
    """Per-stage device time on one resident 5 MP pair, each stage replayed as a graph.
    meta (optional dict) receives the number of level-0 tiles with a corner."""
    reps = 5 if args.profile else 20
    ref = torch.from_numpy(stack.ref.y).to(dev)
    src = torch.from_numpy(stack.srcs[0].y).to(dev)
    srcu = torch.from_numpy(stack.srcs[0].u).to(dev)
    srcv = torch.from_numpy(stack.srcs[0].v).to(dev)
    refu = torch.from_numpy(stack.ref.u).to(dev)
    refv = torch.from_numpy(stack.ref.v).to(dev)
    out = {}
    mode = p.norm_mode
    rn, sn, luts = hdrreg.normalize_exposure(ref, src, mode, stack.ratios[0])
    out["normalize"] = _graph_time_us(
        torch, lambda: hdrreg.normalize_exposure(ref, src, mode, stack.ratios[0]), reps)
    L = hdrreg.num_levels(W, H, p)
    out["pyramid"] = _graph_time_us(torch, lambda: (hdrreg.build_pyramid(rn, L),
                                                    hdrreg.build_pyramid(sn, L)), reps)
    pr, ps = hdrreg.build_pyramid(rn, L), hdrreg.build_pyramid(sn, L)
    Hid = torch.tensor([1, 0, 0, 0, 1, 0, 0, 0, 1], dtype=torch.float64, device=dev)
    res = {}

    counter = torch.zeros(1, dtype=torch.int32, device=dev)

    def matcher():
        Hc = Hid
        for l in range(L - 1, -1, -1):
            lh, lw = pr[l].shape
            cxy, mxy, cost, valid = hdrreg.local_search(pr[l], ps[l], Hc, p)
            mask, Hc, _ = hdrreg.weed_fit(cxy, mxy, valid, lw, lh, p, p.weed_seed + l, Hc,
                                          counter=counter)
        res.update(cxy=cxy, mxy=mxy, mask=mask, H=Hc)

    matcher()
    out["matcher"] = _graph_time_us(torch, matcher, reps)
    cxy, mxy, cost, valid = hdrreg.local_search(rn, sn, res["H"], p)
    if meta is not None:
        meta["valid_level0"] = int(valid.sum().item())
    out["search_level0"] = _graph_time_us(torch, lambda: hdrreg.local_search(rn, sn, res["H"], p), reps)
    out["weed_fit_level0"] = _graph_time_us(
        torch, lambda: hdrreg.weed_fit(cxy, mxy, valid, W, H, p, p.weed_seed, Hid,
                                       counter=counter), reps)
    fu, fv = hdrreg.flow_upsample(rn, res["cxy"], res["mxy"], res["mask"], res["H"], p)
    out["flow"] = _graph_time_us(
        torch, lambda: hdrreg.flow_upsample(rn, res["cxy"], res["mxy"], res["mask"], res["H"], p), reps)
    wy, wu, wv = hdrreg.warp(src, srcu, srcv, res["H"], fu, fv)
    out["warp"] = _graph_time_us(torch, lambda: hdrreg.warp(src, srcu, srcv, res["H"], fu, fv), reps)
    srcs = [dict(y=wy, u=wu, v=wv, ref_n=rn, ratio=stack.ratios[0], lut=luts[1])]
    out["merge"] = _graph_time_us(torch, lambda: hdrreg.merge(ref, refu, refv, srcs, p), reps)
    q = hdrreg.merge(ref, refu, refv, srcs, p, want_q=True)[3]
    fsrc = [dict(y=wy, u=wu, v=wv, q=q[0])]
    out["fuse"] = _graph_time_us(torch, lambda: hdrreg.fuse(ref, refu, refv, fsrc), reps)
    return {k: round(v, 2) for k, v in out.items()}


# DRAM bytes of one flow call (2592 x 1944, 3 iterations, 13 launches): dram__bytes_read.sum
# + dram__bytes_write.sum over the call's launches in one ncu capture (cold L2).
FLOW_TRAFFIC = 553611520


def measure_search_alu(torch, hdrreg, stages, p, valid_tiles, dev):
    """The level-0 SSD search against the measured __dp4a rate. Algorithmic work per
    launch: the cross terms of SSD = sum a^2 + sum b^2 - 2 sum a b over (2R+1)^2 offsets
    and (2h+1)^2 patch pixels of every tile with a corner, four byte products per
    __dp4a. The rate is the probe's (the benchmark's own libhdrreg_probe.so: 8 CTAs of
    256 threads per SM, eight independent chains per thread), median of 5 event-timed
    runs."""
    from paper_1504_01441_b300 import probe
    sink = torch.zeros(1, dtype=torch.int32, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, iters = 8 * sms, 4096
    s = torch.cuda.Stream(device=dev)
    for _ in range(3):
        probe.probe_dp4a(blocks, iters, sink, stream=s)
    times = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        n = probe.probe_dp4a(blocks, iters, sink, stream=s)
        b.record(s)
        b.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    peak = n / (times[2] / 1e3) / 1e9
    algo = valid_tiles * (2 * p.radius + 1) ** 2 * (2 * p.patch_half + 1) ** 2 / 4
    achieved = algo / (stages["search_level0"] / 1e6) / 1e9
    return {"kernel": "k_local_search (level 0)", "bound": "alu", "unit": "G dp4a/s",
            "achieved": round(achieved, 1), "peak": round(peak, 1),
            "frac": round(achieved / peak, 4), "peak_source": "measured (dp4a rate probe)",
            "algorithmic_dp4a_per_launch": int(algo), "tiles_with_corner": valid_tiles,
            "us_per_launch": stages["search_level0"]}


def measure_flow_roofline(stages, p):
    sec = stages["flow"] / 1e6
    peak, src = peaks()
    algo = flow_algorithmic_bytes(W, H, p.dt_iters)
    ach = algo / sec / 1e9
    return {"kernel": "flow: 6 domain-transform passes (row pass + 3-phase column pass)",
            "bound": "hbm", "achieved": round(ach, 1), "peak": peak, "peak_source": src,
            "unit": "GB/s", "frac": round(ach / peak, 4), "traffic": FLOW_TRAFFIC,
            "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum of the stage's "
                              "13 launches in one ncu capture (cold L2)",
            "algorithmic_bytes_per_launch": algo, "us_per_launch": round(stages["flow"], 2),
            "timing": "CUDA graph replay of hdrreg_flow_upsample on one 5 MP pair"}


def measure_e2e(torch, hdrreg, p, stacks, dev, P, args):
    """Host (pinned) inputs -> device -> fused path -> host FP32 outputs, per step of P
    stacks, through the host-staged batched call (copies of one lane overlap the kernels
    of the others)."""
    hin = []
    for i in range(P):
        s = stacks[i % len(stacks)]
        hin.append([torch.from_numpy(a).pin_memory() for a in
                    (s.ref.y, s.ref.u, s.ref.v, s.srcs[0].y, s.srcs[0].u, s.srcs[0].v)])
    hout = [[torch.empty((H, W), dtype=torch.float32).pin_memory(),
             torch.empty((H // 2, W // 2), dtype=torch.float32).pin_memory(),
             torch.empty((H // 2, W // 2), dtype=torch.float32).pin_memory()] for _ in range(P)]
    ratios = stacks[0].ratios
    batch = [((h[0], h[1], h[2]), [(h[3], h[4], h[5])], ratios) for h in hin]
    runner = hdrreg.RegisterMergeHost(W, H, 1, p, lanes=args.lanes, device=dev)
    s = torch.cuda.Stream(device=dev)

    def step():
        runner(batch, hout, stream=s)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    K = 3 if args.profile else 10
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(K):
        step()
    b.record(s)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / K
    h2d = sum(t.numel() * t.element_size() for t in hin[0]) * P
    d2h = sum(t.numel() * t.element_size() for t in hout[0]) * P
    return {"value": round(P * W * H / 1e6 / (ms / 1e3), 2), "unit": "Mpix/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "pairs_per_step": P,
            "ms_per_step": round(ms, 3), "lanes": args.lanes,
            "api": "hdrreg_register_merge_host (pinned host planes in and out)"}


def measure_cpu_baseline(synth, stack, runs=3, cfg=None):
    """The oracle's whole path on one pair on the host cores: the serial build (one
    thread) and the OpenMP build (its independent loops over rows, columns, tiles and
    weeding iterations on every core the process may use; same bits). `value` is the
    OpenMP figure, `single_thread` the serial one."""
    import oracle
    oracle.build()
    cfg = cfg or synth.method_params(32, 6)

    def timed(parallel):
        oracle.set_parallel(parallel)
        try:
            oracle.register_merge(stack.ref, stack.srcs, stack.ratios, cfg)  # warm the pages
            t0 = time.perf_counter()
            for _ in range(runs):
                oracle.register_merge(stack.ref, stack.srcs, stack.ratios, cfg)
            return (time.perf_counter() - t0) / runs, oracle.threads()
        finally:
            oracle.set_parallel(False)
    sec1, _ = timed(False)
    secn, nthreads = timed(True)
    affinity = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else None
    sample = f"{runs} runs of the oracle's whole path (a1-a11) on one {W}x{H} YUV420 pair"
    return {"value": round(W * H / 1e6 / secn, 3), "unit": "Mpix/s", "cores": nthreads,
            "kind": "oracle", "build": "OpenMP (liboracle_omp.so)", "sample": sample,
            "os_cpu_count": os.cpu_count(), "affinity_cpus": affinity,
            "single_thread": {"value": round(W * H / 1e6 / sec1, 3), "unit": "Mpix/s",
                              "cores": 1, "build": "serial (liboracle.so)"}}


# ------------------------------------------------------------ mixed batch (a-B)
def mixed_inputs(n):
    """The mixed workload's stacks (generated in a spawn pool, before CUDA starts)."""
    from paper_1504_01441_b300 import synth
    return synth.make_stacks_parallel([(i, 3, False) for i in range(n)])


def measure_mixed(torch, hdrreg, stacks, dev, args, K):
    """The mixed batch (its stacks already generated) as one multi-shape batched call on
    `lanes` lanes, captured once and replayed K times as a CUDA graph; each stack runs with
    its size bucket's tuned (T, R, B)."""
    from paper_1504_01441_b300 import autotune
    if os.path.exists(autotune.TABLE_FILE):
        table, picks_src = autotune.load_table(), "tune_table.json"
    else:
        table = {"buckets_mp": list(autotune.BUCKETS_MP), "picks": [autotune.DEFAULT] * 4}
        picks_src = "default (no tuning table)"
    params = [autotune.params_for(s.width, s.height, table) for s in stacks]

    def up(a):
        return torch.from_numpy(a).to(dev)
    frames = [((up(s.ref.y), up(s.ref.u), up(s.ref.v)),
               [(up(f.y), up(f.u), up(f.v)) for f in s.srcs], list(s.ratios)) for s in stacks]
    shapes = [(s.width, s.height, len(s.srcs), p, True) for s, p in zip(stacks, params)]
    runner = hdrreg.RegisterMergeMulti(shapes, lanes=args.lanes, device=dev, staged=args.staged)
    stream = torch.cuda.Stream(device=dev)
    runner(frames, stream=stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    n0 = hdrreg.launch_count()
    with torch.cuda.graph(graph, stream=stream):
        runner(frames, stream=stream)
    launches = hdrreg.launch_count() - n0
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 0)):
            graph.replay()
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        start.record(stream)
        for _ in range(K):
            graph.replay()
        end.record(stream)
        torch.cuda.synchronize()
    ms_step = start.elapsed_time(end) / K
    out_mpix = sum(s.width * s.height for s in stacks) / 1e6
    reg_mpix = sum(s.width * s.height * len(s.srcs) for s in stacks) / 1e6
    in_bytes = sum(s.width * s.height * 3 // 2 * (1 + len(s.srcs)) for s in stacks)
    del graph, runner, frames
    torch.cuda.empty_cache()
    return {"workload": MIXED_NAME, "metric": MIXED_METRIC, "value": round(out_mpix / (ms_step / 1e3), 2),
            "unit": "Mpix/s", "ms_per_step": round(ms_step, 3), "steps": K,
            "stacks": len(stacks), "output_mpix_per_step": round(out_mpix, 3),
            "registered_mpix_per_step": round(reg_mpix, 3), "input_bytes_per_step": in_bytes,
            "picks_source": picks_src, "lanes": args.lanes, "graph": True,
            "merge_schedule": "one stage after all registrations" if args.staged else "on each stack's lane",
            "gpu_launches": launches * K,
            "roofline_path": path_roofline(reg_mpix, ms_step, "whole step of the mixed batch, "
                                           "per-pixel byte model")}


def run_mixed(args):
    """Stacks of 1-12 MP with 2-3 frames, each with its size bucket's tuned (T, R), as one
    multi-shape batched call on `lanes` lanes, replayed as one CUDA graph."""
    ws, rank, local = dist_env()
    t_gen = time.perf_counter()
    stacks = mixed_inputs(args.stacks)
    t_gen = time.perf_counter() - t_gen
    import torch
    import torch.distributed as dist
    from paper_1504_01441_b300 import autotune, hdrreg, synth

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    if os.path.exists(autotune.TABLE_FILE):
        table, picks_src = autotune.load_table(), "tune_table.json"
    else:
        table = {"buckets_mp": list(autotune.BUCKETS_MP), "picks": [autotune.DEFAULT] * 4}
        picks_src = "default (no tuning table)"
    params = [autotune.params_for(s.width, s.height, table) for s in stacks]

    def up(a):
        return torch.from_numpy(a).to(dev)
    frames = [((up(s.ref.y), up(s.ref.u), up(s.ref.v)),
               [(up(f.y), up(f.u), up(f.v)) for f in s.srcs], list(s.ratios)) for s in stacks]
    shapes = [(s.width, s.height, len(s.srcs), p, True) for s, p in zip(stacks, params)]
    runner = hdrreg.RegisterMergeMulti(shapes, lanes=args.lanes, device=dev, staged=args.staged)
    stream = torch.cuda.Stream(device=dev)
    runner(frames, stream=stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    n0 = hdrreg.launch_count()
    with torch.cuda.graph(graph, stream=stream):
        runner(frames, stream=stream)
    launches_per_step = hdrreg.launch_count() - n0
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 0)):
            graph.replay()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    K = args.steps
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk, torch.cuda.stream(stream):
        torch.cuda.synchronize()
        start.record(stream)
        for _ in range(K):
            graph.replay()
        end.record(stream)
        torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    if ws > 1:
        ms = max_over_ranks(torch, dist, ms, dev)
        dist.barrier()
    ms_step = ms / K
    out_mpix = sum(s.width * s.height for s in stacks) / 1e6
    reg_mpix = sum(s.width * s.height * len(s.srcs) for s in stacks) / 1e6
    value = job_value(ws, out_mpix, ms_step)
    in_bytes = sum(s.width * s.height * 3 // 2 * (1 + len(s.srcs)) for s in stacks)
    e2e = cpu = roof = None
    if rank == 0:
        peak, src = peaks()
        model = reg_mpix * 1e6 * 165      # the per-registration byte model, whole step
        ach = model / (ms_step / 1e3) / 1e9
        roof = {"kernel": "whole step (all kernels of all stacks): per-pixel byte model",
                "bound": "hbm", "achieved": round(ach, 1), "peak": peak, "peak_source": src,
                "unit": "GB/s", "frac": round(ach / peak, 4), "traffic": None,
                "algorithmic_bytes_per_step": int(model),
                "model": "165 B per registered luma pixel (a1-a11), see the design notes"}
    if rank == 0 and not args.no_e2e:
        e2e = measure_mixed_e2e(torch, runner, stacks, frames, dev, args)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not args.profile:
        cpu = measure_mixed_cpu_baseline(synth, stacks, table)
    if rank == 0:
        buckets = {}
        for s, p in zip(stacks, params):
            b = autotune.bucket_of(s.width, s.height, table["buckets_mp"])
            buckets.setdefault(b, [p.tile, p.radius, p.search_threads or 128, 0])[3] += 1
        line = {
            "metric": MIXED_METRIC, "value": round(value, 2), "unit": "Mpix/s", "n_gpus": ws,
            "steps": K, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8/i32 match, f64 fit, f32 flow/warp/merge", "data": "synthetic",
            "config": {"workload": MIXED_NAME, "stacks": len(stacks), "format": "YUV420",
                       "output_mpix_per_step": round(out_mpix, 3),
                       "registered_mpix_per_step": round(reg_mpix, 3),
                       "input_bytes_per_step": in_bytes,
                       "buckets_mp": table["buckets_mp"],
                       "picks_T_R_B_count": {str(table["buckets_mp"][b]): v
                                           for b, v in sorted(buckets.items())},
                       "picks_source": picks_src, "graph": True, "lanes": args.lanes,
                       "merge_schedule": ("one stage after all registrations" if args.staged
                                          else "on each stack's lane"),
                       "l2": f"inputs larger than L2: {in_bytes / 1e9:.2f} GB resident per step",
                       "generation_s": round(t_gen, 1), "parallelism": f"replicas x{ws}"},
            "gpu_launches": launches_per_step * K, "roofline": roof, "cpu_baseline": cpu,
            "e2e": e2e, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def measure_mixed_e2e(torch, runner, stacks, frames, dev, args):
    """Pinned host planes -> device -> multi-shape batched call -> host, per step."""
    hin = [[torch.from_numpy(a).pin_memory() for a in
            [s.ref.y, s.ref.u, s.ref.v] + [x for f in s.srcs for x in (f.y, f.u, f.v)]]
           for s in stacks]
    din = [[t for t in (fr[0][0], fr[0][1], fr[0][2])] + [x for f in fr[1] for x in f]
           for fr in frames]
    hout = [[torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in o] for o in runner.outs]
    s = torch.cuda.Stream(device=dev)

    def step():
        with torch.cuda.stream(s):
            for h, d in zip(hin, din):
                for a, b in zip(h, d):
                    b.copy_(a, non_blocking=True)
            outs = runner(frames, stream=s)
            for h, o in zip(hout, outs):
                for a, b in zip(h, o):
                    a.copy_(b, non_blocking=True)

    step()
    torch.cuda.synchronize()
    K = 2 if args.profile else 3
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(K):
        step()
    b.record(s)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / K
    h2d = sum(t.numel() * t.element_size() for h in hin for t in h)
    d2h = sum(t.numel() * t.element_size() for h in hout for t in h)
    out_mpix = sum(st.width * st.height for st in stacks) / 1e6
    return {"value": round(out_mpix / (ms / 1e3), 2), "unit": "Mpix/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(ms, 3)}


def measure_mixed_cpu_baseline(synth, stacks, table, n=4):
    """The oracle on the n smallest stacks of the batch, each with its bucket's (T, R)."""
    import oracle
    from paper_1504_01441_b300 import autotune
    oracle.build()
    sub = sorted(stacks, key=lambda s: s.width * s.height)[:n]
    t0 = time.perf_counter()
    for s in sub:
        t, r, _ = autotune.pick_of(table, s.width, s.height)
        oracle.register_merge(s.ref, s.srcs, s.ratios, synth.method_params(t, r))
    sec = time.perf_counter() - t0
    mpix = sum(s.width * s.height for s in sub) / 1e6
    return {"value": round(mpix / sec, 3), "unit": "Mpix/s", "cores": 1, "kind": "oracle",
            "sample": f"the oracle's whole path on the {n} smallest stacks of the batch "
                      f"({mpix:.2f} output Mpix, {sec:.1f} s)"}


# ------------------------------------------------------------ scaling sweep (f3)
def run_sweep(args):
    """Registration + merge time of one two-frame YUV420 pair per size, VGA to 20 MP (the
    paper's runtime-vs-size claim, Sec. 4): the latency of one pair (its graph replayed
    alone) and the throughput of `lanes` copies of it on concurrent lanes. value = the
    log-log slope of the latency against the pixel count (1 = linear)."""
    import math
    stacks = synth_sweep()
    import torch
    from paper_1504_01441_b300 import autotune, hdrreg, synth
    dev = torch.device("cuda", 0)
    p = hdrreg.params_from_dict(synth.method_params(32, 6))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    rows = []
    for st in stacks:
        lat = autotune.fused_time_us(st, p, reps=max(args.steps, 3), device=dev, flush=flush, lanes=1)
        thr = autotune.fused_time_us(st, p, reps=max(args.steps, 3), device=dev, flush=flush,
                                     lanes=args.lanes)
        mp = st.width * st.height / 1e6
        rows.append({"width": st.width, "height": st.height, "mpix": round(mp, 3),
                     "latency_us": round(lat, 1), "batched_us_per_pair": round(thr, 1),
                     "batched_mpix_s": round(mp / (thr / 1e6), 1)})
        torch.cuda.empty_cache()
    xs = [math.log(r["mpix"]) for r in rows]
    ys = [math.log(r["latency_us"]) for r in rows]
    zs = [math.log(r["batched_us_per_pair"]) for r in rows]

    def slope(a, b):
        ma, mb = sum(a) / len(a), sum(b) / len(b)
        return sum((u - ma) * (v - mb) for u, v in zip(a, b)) / sum((u - ma) ** 2 for u in a)
    line = {
        "metric": "scaling: d log(latency) / d log(pixels), one 2-frame YUV420 pair, VGA..20 MP",
        "value": round(slope(xs, ys), 3), "unit": "exponent (1 = linear)", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
        "scaling": "none", "vs_baseline": None, "data": "synthetic",
        "dtype": "u8/i32 match, f64 fit, f32 flow/warp/merge",
        "config": {"workload": "sweep_vga_to_20mp_yuv420_pair", "tile": 32, "radius": 6,
                   "lanes": args.lanes, "l2": "L2 flushed (256 MB write) before every replay"},
        "batched_slope": round(slope(xs, zs), 3), "sweep": rows,
    }
    print(json.dumps(line), flush=True)


def _time_graph(torch, runner, frames, stream, warmup, steps):
    """-> (ms per replay of runner(frames) captured as one CUDA graph, the graph, the
    library launches it holds)."""
    from paper_1504_01441_b300 import hdrreg
    runner(frames, stream=stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    n0 = hdrreg.launch_count()
    with torch.cuda.graph(g, stream=stream):
        runner(frames, stream=stream)
    launches = hdrreg.launch_count() - n0
    with torch.cuda.stream(stream):
        for _ in range(max(warmup, 0)):
            g.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            g.replay()
        b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps, g, launches


def run_scale12(args):
    """Learned + batched at scale: 32 three-frame 4000 x 3000 YUV420 stacks (exposures 1/4,
    1, 4 of the reference's; +-8 px fields; 5 movers) per step through the batched fused
    call with the learned level-0 search, one CUDA graph, at the default operating point
    (refine 1, fallback above 1.5 x the median plain cost) and at the calibrated one; the
    plain path on the same stacks; the host-staged form (e2e); and one training step of
    the predictor (64 crops of 256 x 256 full-resolution pixels: forward, backward and
    Adam, all in the library's kernels)."""
    ws, rank, local = dist_env()
    n = args.stacks if args.stacks != 64 else 32
    t_gen = time.perf_counter()
    from paper_1504_01441_b300 import synth as _s
    stacks = _s.make_scale12_stacks(n)          # spawn pool, before CUDA starts
    t_gen = time.perf_counter() - t_gen
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1504_01441_b300 import hdrreg, learned as L, synth

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    w, h = stacks[0].width, stacks[0].height
    p = hdrreg.params_from_dict(synth.method_params(32, 6))

    def up(a):
        return torch.from_numpy(a).to(dev)
    frames = [((up(s.ref.y), up(s.ref.u), up(s.ref.v)),
               [(up(f.y), up(f.u), up(f.v)) for f in s.srcs], list(s.ratios)) for s in stacks]
    stream = torch.cuda.Stream(device=dev)
    plain = hdrreg.RegisterMergeBatch(w, h, 2, p, True, slots=n, lanes=args.lanes, device=dev)
    ms_plain, g, _ = _time_graph(torch, plain, frames, stream, args.warmup, args.steps)
    del g, plain
    theta = torch.tensor(np.load(L.THETA_FILE)).to(dev)
    # quality and thresholds from the first source (exposure 1/4) of the first two stacks
    prep = [L.prepare(s, p) for s in stacks[:2]]
    med = float(torch.cat([P.cost[P.valid.bool()] for P in prep]).double().median().item())
    points = [("default", 1, 1.5)]
    if os.path.exists(L.OPS_FILE):
        ch = json.load(open(L.OPS_FILE)).get("chosen")
        if ch:
            points.append(("at_bound", ch["refine"], ch["ratio"]))
    legs, clk_sum, launches, pl_default = {}, None, 0, None
    for name, refine, ratio in points:
        q = L.evaluate(prep, theta, p, fallback_ratio=ratio, refine=refine)
        pl = hdrreg.params_from_dict(p.as_dict())
        pl.predictor = theta.data_ptr()
        pl.fallback_cost = int(ratio * med)
        pl.predictor_refine = refine
        lrn = hdrreg.RegisterMergeBatch(w, h, 2, pl, True, slots=n, lanes=args.lanes, device=dev)
        with ClockSampler(local) as clk:
            ms, g, per_step = _time_graph(torch, lrn, frames, stream, args.warmup, args.steps)
        if ws > 1:
            ms = max_over_ranks(torch, dist, ms, dev)
        fb = sum(d.fallbacks for i in range(n) for d in lrn.diagnostics(i))
        val = sum(d.valid for i in range(n) for d in lrn.diagnostics(i))
        legs[name] = {"value": round(ws * n * w * h / 1e6 / (ms / 1e3), 2), "unit": "Mpix/s",
                      "ms_per_step": round(ms, 3), "refine": refine, "fallback_ratio": ratio,
                      "fallback_cost": pl.fallback_cost,
                      "fallback_rate": round(fb / max(val, 1), 4),
                      "epe_vs_plain_px": round(q["epe_px"], 3),
                      "epe_vs_plain_median_px": round(q["epe_median_px"], 3),
                      "meets_0.5px_vs_plain": bool(q["epe_px"] <= 0.5)}
        if name == "default":
            clk_sum, pl_default = clk.summary(), pl
            launches = args.steps * per_step
        del g, lrn
    del prep
    # host-staged (pinned host planes in and out), default operating point
    hin = [[torch.from_numpy(a).pin_memory() for a in
            (s.ref.y, s.ref.u, s.ref.v) + tuple(x for f in s.srcs for x in (f.y, f.u, f.v))]
           for s in stacks]
    hout = [[torch.empty((h, w), dtype=torch.float32).pin_memory(),
             torch.empty((h // 2, w // 2), dtype=torch.float32).pin_memory(),
             torch.empty((h // 2, w // 2), dtype=torch.float32).pin_memory()] for _ in stacks]
    batch = [((x[0], x[1], x[2]), [(x[3], x[4], x[5]), (x[6], x[7], x[8])], list(s.ratios))
             for x, s in zip(hin, stacks)]
    host = hdrreg.RegisterMergeHost(w, h, 2, pl_default, lanes=args.lanes, device=dev)
    for _ in range(2):
        host(batch, hout, stream=stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    K = max(3, args.steps // 2)
    for _ in range(K):
        host(batch, hout, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms_e2e = a.elapsed_time(b) / K
    del host
    train_ms = time_train_step(torch, hdrreg, theta, dev, stream)
    out_mpix = n * w * h / 1e6
    d = legs["default"]
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not args.profile:
        # the oracle's plain path on the first stack (two registrations of 12 MP, one run)
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        oracle.register_merge(stacks[0].ref, stacks[0].srcs, stacks[0].ratios,
                              synth.method_params(32, 6))
        sec = time.perf_counter() - t0
        cpu = {"value": round(w * h / 1e6 / sec, 3), "unit": "Mpix/s", "cores": 1,
               "kind": "oracle",
               "sample": "one run of the oracle's whole plain path (a1-a11) on the first "
                         "4000x3000 three-frame stack (output Mpix per second)"}
    if rank == 0:
        line = {
            "metric": "registered+merged output Mpix/s per B300, learned level-0 search "
                      f"({n} three-frame 12 MP stacks)",
            "value": d["value"], "unit": "Mpix/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": d["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8/i32 match, bf16 net, f64 fit, f32 flow/warp/merge",
            "data": "synthetic",
            "config": {"workload": SCALE12_NAME, "stacks": n, "width": w, "height": h,
                       "frames": 3, "exposures": "1/4, 1 (reference), 4", "field_px": 8,
                       "movers": 5, "tile": 32, "radius": 6, "lanes": args.lanes,
                       "graph": True, "l2": f"inputs larger than L2 ({n} resident stacks)",
                       "generation_s": round(t_gen, 1), "parallelism": f"replicas x{ws}"},
            "learned": legs,
            "plain": {"value": round(ws * out_mpix / (ms_plain / 1e3), 2), "unit": "Mpix/s",
                      "ms_per_step": round(ms_plain, 3)},
            "quality_sample": "first source (exposure 1/4) of the first 2 stacks",
            "e2e": {"value": round(out_mpix / (ms_e2e / 1e3), 2), "unit": "Mpix/s",
                    "h2d_bytes_per_step": sum(t.numel() for x in hin for t in x),
                    "d2h_bytes_per_step": sum(t.numel() * 4 for x in hout for t in x),
                    "ms_per_step": round(ms_e2e, 3),
                    "api": "hdrreg_register_merge_host, default operating point"},
            "train_step_ms": round(train_ms, 3),
            "train_step": TRAIN_STEP,
            "gpu_launches": launches, "clocks": clk_sum, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_learned8(args):
    """5 MP YUV420 pairs as the headline workload but with +-8 px local fields: the plain
    path and the learned level-0 search (default and calibrated operating points) on
    `pairs` resident pairs per step, each replayed as one CUDA graph, with the learned
    search's distance to the plain matches and both searches' distance to the generator's
    truth."""
    ws, rank, local = dist_env()
    from paper_1504_01441_b300 import synth as _s
    stacks = [_s.make_learned8_stack(i) for i in range(args.distinct)]
    import torch
    import torch.distributed as dist
    from paper_1504_01441_b300 import hdrreg, synth

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    p = hdrreg.params_from_dict(synth.method_params(32, 6))
    P = args.pairs
    frames = []
    for i in range(P):
        s = stacks[i % len(stacks)]
        ref = tuple(torch.from_numpy(a).to(dev) for a in (s.ref.y, s.ref.u, s.ref.v))
        src = tuple(torch.from_numpy(a).to(dev) for a in (s.srcs[0].y, s.srcs[0].u, s.srcs[0].v))
        frames.append((ref, [src], s.ratios))
    stream = torch.cuda.Stream(device=dev)
    plain = hdrreg.RegisterMergeBatch(W, H, 1, p, True, slots=P, lanes=args.lanes, device=dev)
    with ClockSampler(local) as clk:
        ms_plain, g, per_step = _time_graph(torch, plain, frames, stream, args.warmup, args.steps)
    if ws > 1:
        ms_plain = max_over_ranks(torch, dist, ms_plain, dev)
    del g, plain
    learned = measure_learned(torch, hdrreg, synth, stacks, frames, p, dev, args)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not args.profile:
        cpu = measure_cpu_baseline(synth, stacks[0])
        cpu["sample"] += " (+-8 px fields)"
    if rank == 0:
        line = {
            "metric": "registered+merged output Mpix/s per B300, learned level-0 search "
                      "(5 MP pairs, +-8 px fields)",
            "value": learned["value"], "unit": "Mpix/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8/i32 match, bf16 net, f64 fit, f32 flow/warp/merge",
            "data": "synthetic",
            "config": {"workload": LEARNED8_NAME, "width": W, "height": H, "format": "YUV420",
                       "frames": 2, "exposure_ratio": 4, "field_px": 8, "movers": 3,
                       "pairs_per_step": P, "distinct_stacks": len(stacks), "tile": 32,
                       "radius": 6, "graph": True, "lanes": args.lanes,
                       "l2": f"inputs larger than L2: {P} resident pairs x 15.1 MB per step",
                       "parallelism": f"replicas x{ws}"},
            "plain": {"value": round(ws * P * W * H / 1e6 / (ms_plain / 1e3), 2),
                      "unit": "Mpix/s", "ms_per_step": round(ms_plain, 3),
                      "gpu_launches_per_step": per_step},
            "learned": learned, "clocks": clk.summary(), "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def synth_sweep():
    from paper_1504_01441_b300 import synth
    return synth.make_sweep_stacks()


# ------------------------------------------------------------ reference arm
def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_1504_01441_b300 import synth
    import oracle
    oracle.build()
    if args.workload == MIXED:
        return run_reference_mixed(args, ws)
    if args.workload in (SWEEP, SCALE12):
        why = ("one oracle step of this workload (32 three-frame 12 MP stacks) takes many "
               "minutes on one core; its line carries the oracle's time on one stack as "
               "cpu_baseline") if args.workload == SCALE12 else (
              "one oracle step of this workload (a pair of every size up to 20 MP) takes "
              "minutes on one core; the default workload's reference arm times the oracle "
              "on its 5 MP pair")
        print(json.dumps({"impl": "reference", "workload": args.workload, "unavailable": why}),
              flush=True)
        return
    learned8 = args.workload == LEARNED8
    stack = synth.make_learned8_stack(0) if learned8 else make_inputs(1)[0]
    cfg = synth.method_params(32, 6)
    # the OpenMP build of the oracle on every host core the process may use (same bits
    # as the serial build)
    oracle.set_parallel(True)
    cores = oracle.threads()
    for _ in range(max(args.warmup, 0)):
        oracle.register_merge(stack.ref, stack.srcs, stack.ratios, cfg)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.register_merge(stack.ref, stack.srcs, stack.ratios, cfg)
    sec = time.perf_counter() - t0
    ms_step = sec * 1e3 / args.steps
    value = W * H / 1e6 / (ms_step / 1e3)
    sample = "one 2592x1944 YUV420 two-frame stack per step through the oracle's whole path"
    if learned8:
        sample += " (+-8 px fields; the oracle runs the plain search)"
    line = {
        "impl": "reference",
        "metric": (("registered+merged output Mpix/s per B300, learned level-0 search "
                    "(5 MP pairs, +-8 px fields)") if learned8 else METRIC),
        "value": round(value, 3), "unit": "Mpix/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64/int64 (CPU oracle)", "data": "synthetic",
        "config": {"workload": LEARNED8_NAME if learned8 else WORKLOAD, "width": W, "height": H,
                   "format": "YUV420", "frames": 2, "exposure_ratio": 4, "tile": 32, "radius": 6,
                   "path": "plain (a1-a11)"},
        "cpu_baseline": {"value": round(value, 3), "unit": "Mpix/s", "cores": cores,
                         "kind": "oracle", "build": "OpenMP (liboracle_omp.so)",
                         "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_mixed(args, ws):
    """The oracle on the mixed workload: each step is one of the four smallest stacks of
    the batch (cycled), with its bucket's (T, R); value = output Mpix / oracle time."""
    import oracle
    from paper_1504_01441_b300 import autotune, synth
    order = sorted(range(args.stacks),
                   key=lambda i: synth.mixed_spec(i).width * synth.mixed_spec(i).height)[:4]
    stacks = [synth.make_mixed_stack(i) for i in order]
    table = (autotune.load_table() if os.path.exists(autotune.TABLE_FILE) else
             {"buckets_mp": list(autotune.BUCKETS_MP), "picks": [autotune.DEFAULT] * 4})

    def run(s):
        t, r, _ = autotune.pick_of(table, s.width, s.height)
        oracle.register_merge(s.ref, s.srcs, s.ratios, synth.method_params(t, r))

    oracle.set_parallel(True)  # the OpenMP build on every host core (same bits as serial)
    cores = oracle.threads()
    for i in range(max(args.warmup, 0)):
        run(stacks[i % 4])
    t0 = time.perf_counter()
    mpix = 0.0
    for i in range(args.steps):
        run(stacks[i % 4])
        mpix += stacks[i % 4].width * stacks[i % 4].height / 1e6
    sec = time.perf_counter() - t0
    value = mpix / sec
    line = {
        "impl": "reference", "metric": MIXED_METRIC, "value": round(value, 3), "unit": "Mpix/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(sec * 1e3 / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64/int64 (CPU oracle)",
        "data": "synthetic", "config": {"workload": MIXED_NAME, "stacks": args.stacks},
        "cpu_baseline": {"value": round(value, 3), "unit": "Mpix/s", "cores": cores,
                         "kind": "oracle", "build": "OpenMP (liboracle_omp.so)",
                         "sample": "per step one of the 4 smallest stacks of the mixed batch"},
        "e2e": {"value": round(value, 3), "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == MIXED:
        run_mixed(args)
    elif args.workload == SWEEP:
        run_sweep(args)
    elif args.workload == SCALE12:
        run_scale12(args)
    elif args.workload == LEARNED8:
        run_learned8(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
