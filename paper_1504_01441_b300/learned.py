"""Training and evaluation of the learned level-0 search (row a-L).

The network (csrc/cnn.cu) predicts, per 32x32 tile, the displacement the plain
SSD search of Sec. 2.2 finds at level 0, from the normalized reference and the
source pre-warped by the level-1 homography at quarter resolution. Everything
numeric runs in the library's kernels; this module only sequences the calls:

  prepare(stack)  plain matcher down to level 1 (H1), the network input, and the
                  plain level-0 search whose displacements are the labels;
  train(...)      Adam on random crops of 8 x 8 tiles (64 x 64 input pixels);
  evaluate(...)   end-point error of the learned search against the plain one
                  (mean |match_learned - match_plain| over tiles with a corner) and
                  its fallback rate, with the fallback cost calibrated as 1.5 x the
                  median plain level-0 SSD cost.

Training inputs are seeded synthetic stacks of synth.py shaped like the headline 5 MP pairs
(+-4 px fields); evaluation also reports stacks with +-8 px fields, where the field exceeds the
plain search's radius and the plain labels stop being measurements.
`python -m paper_1504_01441_b300.learned --out FILE` trains from scratch and writes
the parameters (float32, HDRREG_CNN_PARAMS values); the committed
paper_1504_01441_b300/predictor_theta.npy was written this way.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import struct
import time
import zlib
from typing import List

import numpy as np

from . import hdrreg, synth

CROP_TILES = 8
# the headline workload's distribution (5 MP, r = 4, sigma 1.5, +-4 px fields, 3 movers),
# luma only; STRESS_SPEC doubles the field, beyond the plain search's radius of 6 px
TRAIN_SPEC = synth.StackSpec(2592, 1944, ratios=((4, 1),), noise_sigma=1.5, field_amp=4.0,
                             movers=3, chroma=False)
STRESS_SPEC = synth.StackSpec(2592, 1944, ratios=((4, 1),), noise_sigma=1.5, field_amp=8.0,
                              movers=3, chroma=False)
THETA_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "predictor_theta.npy")


@dataclasses.dataclass
class Prepared:
    x: object          # bfloat16 [hq, wq, 2] network input
    label: object      # FP32 [nty * ntx, 2] plain displacement from the search centre
    valid: object      # uint8 [nty * ntx]
    match: object      # int32 [nty * ntx, 2] plain level-0 matches
    cost: object       # int32 [nty * ntx] plain level-0 SSD costs
    H1: object         # float64 [9] level-1 homography
    ref_n: object
    src_n: object
    ntx: int
    nty: int
    gt: object = None  # optional FP32 [2, H, W]: generator ground truth (source position)


def prepare(stack, p: hdrreg.Params, device="cuda", keep_gt: bool = False) -> Prepared:
    import torch
    dev = torch.device(device)
    ref = torch.from_numpy(stack.ref.y).to(dev)
    src = torch.from_numpy(stack.srcs[0].y).to(dev)
    rn, sn, _ = hdrreg.normalize_exposure(ref, src, hdrreg.NORM_RATIO, stack.ratios[0])
    h, w = rn.shape
    L = hdrreg.num_levels(w, h, p)
    if L < 3 or p.tile != 32:
        raise ValueError("the learned search needs tile 32 and three pyramid levels")
    pr, ps = hdrreg.build_pyramid(rn, L), hdrreg.build_pyramid(sn, L)
    Hc = torch.tensor([1, 0, 0, 0, 1, 0, 0, 0, 1], dtype=torch.float64, device=dev)
    counter = torch.zeros(1, dtype=torch.int32, device=dev)
    for lv in range(L - 1, 0, -1):
        lh, lw = pr[lv].shape
        cxy, mxy, cost, valid = hdrreg.local_search(pr[lv], ps[lv], Hc, p)
        _, Hc, _ = hdrreg.weed_fit(cxy, mxy, valid, lw, lh, p, p.weed_seed + lv, Hc, counter=counter)
    H1 = Hc.clone()
    x = hdrreg.predictor_input(pr[2], ps[2], H1)
    cxy, mxy, cost, valid = hdrreg.local_search(rn, sn, H1, p)
    lab = hdrreg.tile_labels(cxy, mxy, valid, w, h, H1)
    gt = None
    if keep_gt and stack.gt and stack.gt[0] is not None:
        gt = torch.from_numpy(np.stack(stack.gt[0])).to(dev)
    return Prepared(x, lab, valid, mxy, cost, H1, rn, sn, w // p.tile, h // p.tile, gt)


def make_stacks(n: int, first_index: int, spec=TRAIN_SPEC):
    return synth.make_spec_stacks_parallel(spec, [synth.stack_seed(4, first_index + i)
                                                  for i in range(n)])


# Training checkpoint: a flat file of a fixed header, the FP32 parameters, the two Adam
# moment vectors, the crop generator's state, and a CRC-32 of everything before it.
CKPT_MAGIC = b"HDRRCKP1"
_CKPT_HEAD = struct.Struct("<8sIIqqI")  # magic, version, parameters, Adam step, step, rng bytes


def write_checkpoint(path: str, theta, m, v, adam_t: int, step: int, rng_state: bytes):
    """Write a training checkpoint (atomically: a temporary file, then a rename).
    theta, m, v: float32 vectors of the same length; adam_t: Adam's step counter; step: the
    next training step to run; rng_state: the crop generator's state."""
    arrs = [np.ascontiguousarray(np.asarray(a, np.float32)).reshape(-1) for a in (theta, m, v)]
    if not arrs[0].size == arrs[1].size == arrs[2].size:
        raise ValueError("theta, m and v must have the same length")
    body = _CKPT_HEAD.pack(CKPT_MAGIC, 1, arrs[0].size, int(adam_t), int(step), len(rng_state))
    body += b"".join(a.tobytes() for a in arrs) + bytes(rng_state)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        f.write(body + struct.pack("<I", zlib.crc32(body)))
    os.replace(tmp, path)


def read_checkpoint(path: str) -> dict:
    """-> dict(theta, m, v, adam_t, step, rng_state); ValueError if the file is not a
    checkpoint, is truncated, or fails its checksum."""
    data = open(path, "rb").read()
    if len(data) < _CKPT_HEAD.size + 4:
        raise ValueError(f"{path}: too short for a checkpoint")
    magic, version, n, adam_t, step, nr = _CKPT_HEAD.unpack_from(data, 0)
    if magic != CKPT_MAGIC or version != 1:
        raise ValueError(f"{path}: not a predictor training checkpoint")
    end = _CKPT_HEAD.size + 12 * n + nr
    if len(data) != end + 4:
        raise ValueError(f"{path}: size {len(data)} does not match its header ({end + 4})")
    if struct.unpack_from("<I", data, end)[0] != zlib.crc32(data[:end]):
        raise ValueError(f"{path}: checksum mismatch")
    o = _CKPT_HEAD.size
    vec = [np.frombuffer(data, np.float32, n, o + 4 * n * i).copy() for i in range(3)]
    return dict(theta=vec[0], m=vec[1], v=vec[2], adam_t=adam_t, step=step,
                rng_state=data[o + 12 * n:end])


def train(prepared: List[Prepared], steps: int, batch: int = 64, lr: float = 2e-3, seed: int = 0,
          theta=None, log_every: int = 50, augment: bool = True, label_bound: float = 6.0,
          checkpoint: str = None, checkpoint_every: int = 0, resume: str = None,
          stop_at: int = None):
    """Adam on random crops (each under one of the 8 mirror/transpose symmetries when
    augment); crops of one batch come from all prepared stacks in turn; labels on the
    border of the plain search (|d| >= label_bound, the search radius) are left out.
    checkpoint / checkpoint_every: write a checkpoint after every that many steps (and
    after the last); resume: continue from a checkpoint, which gives the same parameters,
    bit for bit, as the run that was never interrupted (the crops come from the saved
    generator state, the learning rate from the step number); stop_at: end after that
    step of the `steps`-step schedule (a run in pieces)."""
    import torch
    from . import hdrreg as hd
    dev = prepared[0].x.device
    side = 8 * CROP_TILES
    pred = hd.Predictor(batch, side, side, theta, device=dev)
    if theta is None:
        pred.theta.copy_(torch.tensor(init_theta(seed)))
    g = torch.Generator(device="cpu").manual_seed(seed)
    start = 0
    if resume:
        ck = read_checkpoint(resume)
        if ck["theta"].size != pred.theta.numel():
            raise ValueError(f"{resume}: {ck['theta'].size} parameters, the network has "
                             f"{pred.theta.numel()}")
        pred.theta.copy_(torch.from_numpy(ck["theta"]))
        pred.m.copy_(torch.from_numpy(ck["m"]))
        pred.v.copy_(torch.from_numpy(ck["v"]))
        pred.t = ck["adam_t"]
        g.set_state(torch.frombuffer(bytearray(ck["rng_state"]), dtype=torch.uint8))
        start = ck["step"]

    def save(next_step):
        torch.cuda.synchronize()
        write_checkpoint(checkpoint, pred.theta.cpu().numpy(), pred.m.cpu().numpy(),
                         pred.v.cpu().numpy(), pred.t, next_step, g.get_state().numpy().tobytes())
    xb = torch.empty((batch, side, side, 2), dtype=torch.bfloat16, device=dev)
    lb = torch.empty((batch, CROP_TILES, CROP_TILES, 2), dtype=torch.float32, device=dev)
    vb = torch.empty((batch, CROP_TILES, CROP_TILES), dtype=torch.uint8, device=dev)
    per = [batch // len(prepared) + (1 if i < batch % len(prepared) else 0)
           for i in range(len(prepared))]
    history = []
    t0 = time.perf_counter()
    end = steps if stop_at is None else min(steps, stop_at)
    for step in range(start, end):
        o = 0
        for P, k in zip(prepared, per):
            if k == 0:
                continue
            org = torch.stack([torch.randint(0, P.ntx - CROP_TILES + 1, (k,), generator=g),
                               torch.randint(0, P.nty - CROP_TILES + 1, (k,), generator=g),
                               torch.randint(0, 8 if augment else 1, (k,), generator=g),
                               torch.zeros(k, dtype=torch.int64)], 1)
            org = org.to(torch.int32).to(dev)
            xc, lc, vc = hd.predictor_crops(P.x, P.label, P.valid, P.ntx, P.nty, org, CROP_TILES,
                                            label_bound)
            xb[o:o + k].copy_(xc)
            lb[o:o + k].copy_(lc)
            vb[o:o + k].copy_(vc)
            o += k
        pred.forward(xb)
        loss, _ = pred.backward(xb, lb, vb)
        pred.adam(lr=lr * (1.0 - 0.9 * step / max(steps - 1, 1)))  # linear decay to 10%
        if step % log_every == 0 or step == steps - 1:
            history.append((step, float(loss.item())))
        if checkpoint and ((checkpoint_every and (step + 1) % checkpoint_every == 0) or
                           step == end - 1):
            save(step + 1)
    torch.cuda.synchronize()
    if int(pred.status.item()) != 0:
        raise hd.HdrregError(2, "a tensor-core kernel timed out during training")
    return pred.theta.detach().clone(), history, time.perf_counter() - t0


def init_theta(seed: int):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, head scaled by 0.1 -- the
    network's starting point for training."""
    rng = np.random.default_rng(seed)
    layers = [(27, 16, 3, True), (16, 16, 3, True), (16, 32, 3, True), (32, 32, 3, True),
              (32, 48, 3, True), (48, 48, 3, True), (48, 64, 3, True), (64, 64, 3, True),
              (64, 2, 1, False)]
    parts = []
    for ci, co, k, relu in layers:
        std = np.sqrt(2.0 / (ci * k * k)) * (1.0 if relu else 0.1)
        parts.append(rng.normal(0.0, std, co * k * k * ci))
        parts.append(np.zeros(co))
    th = np.concatenate(parts).astype(np.float32)
    assert th.size == hdrreg.CNN_PARAMS
    return th


def evaluate(prepared: List[Prepared], theta, p: hdrreg.Params, fallback_ratio: float = 1.5,
             refine: int = 1):
    """Learned vs plain level-0 search on prepared stacks -> metrics dict."""
    import torch
    errs, fb_tot, val_tot, raw = [], 0, 0, []
    P0 = prepared[0]
    hq, wq = P0.x.shape[0], P0.x.shape[1]
    net = hdrreg.Predictor(1, hq, wq, theta, device=P0.x.device)
    costs = torch.cat([P.cost[P.valid.bool()] for P in prepared]).double()
    thr = int(fallback_ratio * float(costs.median().item()))
    gt_plain, gt_learned = [], []
    for P in prepared:
        out = net.forward(P.x.unsqueeze(0))[0]
        c, m, co, v, fb = hdrreg.local_search_predicted(P.ref_n, P.src_n, P.H1, p, out, thr, refine)
        ok = (v.bool() & P.valid.bool())
        d = (m[ok] - P.match[ok]).double()
        errs.append(torch.sqrt((d * d).sum(1)))
        if P.gt is not None:
            cc = c[ok].long()
            g = torch.stack([P.gt[0][cc[:, 1], cc[:, 0]], P.gt[1][cc[:, 1], cc[:, 0]]], 1).double()
            gt_plain.append(torch.sqrt(((P.match[ok].double() - g) ** 2).sum(1)))
            gt_learned.append(torch.sqrt(((m[ok].double() - g) ** 2).sum(1)))
        pr = out[:P.nty, :P.ntx].reshape(-1, 2)[ok]
        dr = (pr.double() - P.label[ok].double())
        raw.append(torch.sqrt((dr * dr).sum(1)))
        fb_tot += int(fb[ok].sum().item())
        val_tot += int(ok.sum().item())
    e = torch.cat(errs)
    r = torch.cat(raw)
    extra = {}
    if gt_plain:
        gp, gl = torch.cat(gt_plain), torch.cat(gt_learned)
        extra = {"plain_vs_truth_px": float(gp.mean().item()),
                 "learned_vs_truth_px": float(gl.mean().item()),
                 "plain_vs_truth_median_px": float(gp.median().item()),
                 "learned_vs_truth_median_px": float(gl.median().item())}
    return {**extra, "epe_px": float(e.mean().item()), "epe_median_px": float(e.median().item()),
            "within_half_px": float((e <= 0.5).double().mean().item()),
            "epe_network_px": float(r.mean().item()),
            "fallback_rate": fb_tot / max(val_tot, 1), "tiles": val_tot, "fallback_cost": thr,
            "refine": refine}


OPS_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "predictor_operating_point.json")


def search_cost(refine: int, fallback_rate: float, radius: int = 6) -> float:
    """SSD offsets per tile of the search with a prediction: the refinement window, plus
    the full window on the tiles that fall back."""
    return (2 * refine + 1) ** 2 + fallback_rate * (2 * radius + 1) ** 2


def calibrate(prepared: List[Prepared], theta, p: hdrreg.Params, bound: float = 0.5,
              refines=(1, 2, 3, 4), ratios=(1.5, 1.25, 1.0, 0.9, 0.8)):
    """Every (refine, fallback ratio) on the prepared stacks -> (points, the cheapest point
    whose mean distance to the plain matches is <= bound, by search_cost; None if none)."""
    pts = []
    for r in refines:
        for fr in ratios:
            q = evaluate(prepared, theta, p, fallback_ratio=fr, refine=r)
            pts.append({"refine": r, "ratio": fr, "epe_px": round(q["epe_px"], 4),
                        "fallback_rate": round(q["fallback_rate"], 4),
                        "cost": round(search_cost(r, q["fallback_rate"], p.radius), 2)})
    ok = [t for t in pts if t["epe_px"] <= bound]
    return pts, (min(ok, key=lambda t: (t["cost"], t["refine"])) if ok else None)


def time_network(reps: int, h: int = 486, w: int = 648):
    """Device time (us per call) of the inference form and of the training forward of the
    network on one quarter-resolution input of a 2592 x 1944 frame (trained parameters,
    random input), each call timed with CUDA events over `reps` calls after three."""
    import torch
    theta = np.load(THETA_FILE)
    x = torch.tensor(np.random.default_rng(1).uniform(-1, 1, (1, h, w, 2)),
                     dtype=torch.bfloat16).cuda()
    net = hdrreg.Predictor(1, h, w, theta)
    out = {}
    for name, fn in (("infer_us", lambda: net.infer(x)), ("forward_us", lambda: net.forward(x))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        out[name] = round(a.elapsed_time(b) * 1e3 / max(reps, 1), 2)
    return out


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--time-network", type=int, default=0, metavar="REPS",
                    help="only time the network (inference and training forward) and exit")
    ap.add_argument("--calibrate", type=int, default=0, metavar="STACKS",
                    help="choose the operating point meeting --bound on STACKS held-out stacks")
    ap.add_argument("--bound", type=float, default=0.5)
    ap.add_argument("--ops-out", default=OPS_FILE)
    ap.add_argument("--out", default=THETA_FILE)
    ap.add_argument("--train-stacks", type=int, default=16)
    ap.add_argument("--stress-stacks", type=int, default=0,
                    help="training stacks with +-8 px fields (STRESS_SPEC) besides the +-4 px ones")
    ap.add_argument("--checkpoint", default=None,
                    help="write a training checkpoint to this file (every --checkpoint-every "
                         "steps and at the end)")
    ap.add_argument("--checkpoint-every", type=int, default=1000)
    ap.add_argument("--resume", default=None, help="continue training from this checkpoint")
    ap.add_argument("--label-radius", type=int, default=6,
                    help="search radius of the plain level-0 search that labels the training "
                         "tiles (labels on its border are left out)")
    ap.add_argument("--eval-stacks", type=int, default=2)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--log", default=None)
    args = ap.parse_args()
    if args.time_network:
        print(json.dumps(time_network(args.time_network)))
        return
    if args.calibrate:
        # held-out stacks shaped like the headline workload (seeds apart from training,
        # evaluation and the bench's stacks)
        p = hdrreg.params_from_dict(synth.method_params(32, 6))
        theta = torch.tensor(np.load(THETA_FILE)).cuda()
        stacks = [synth.make_stack(synth.FIVE_MP, synth.stack_seed(4, 3000 + i))
                  for i in range(args.calibrate)]
        prep = [prepare(st, p) for st in stacks]
        pts, best = calibrate(prep, theta, p, bound=args.bound)
        rep = {"bound_px": args.bound, "stacks": args.calibrate, "chosen": best, "points": pts,
               "spec": "2592x1944 YUV420, r = 4, sigma 1.5, +-4 px fields, seeds 4:3000+"}
        with open(args.ops_out, "w") as f:
            json.dump(rep, f, indent=1)
        print(json.dumps({"chosen": best}))
        return
    p = hdrreg.params_from_dict(synth.method_params(32, 6))
    p_label = hdrreg.params_from_dict(synth.method_params(32, args.label_radius))
    t0 = time.perf_counter()
    stacks = make_stacks(args.train_stacks, 0)
    if args.stress_stacks:
        stacks += make_stacks(args.stress_stacks, 4000, STRESS_SPEC)
    train_set = [prepare(s, p_label) for s in stacks]
    del stacks
    eval_set = [prepare(s, p, keep_gt=True) for s in make_stacks(args.eval_stacks, 1000)]
    t_data = time.perf_counter() - t0
    theta, hist, t_train = train(train_set, args.steps, args.batch, args.lr, args.seed,
                                 label_bound=float(args.label_radius), checkpoint=args.checkpoint,
                                 checkpoint_every=args.checkpoint_every, resume=args.resume)
    m_train = evaluate(train_set[:2], theta, p)
    m_eval = {f"refine{r}_ratio{fr}": evaluate(eval_set, theta, p, fallback_ratio=fr, refine=r)
              for r in (0, 1) for fr in (1.0, 1.5)}
    stress = [prepare(s, p, keep_gt=True) for s in make_stacks(1, 2000, STRESS_SPEC)]
    m_eval["stress_refine1_ratio1.5"] = evaluate(stress, theta, p, fallback_ratio=1.5, refine=1)
    np.save(args.out, theta.cpu().numpy())
    rep = {"steps": args.steps, "batch": args.batch, "lr": args.lr, "seed": args.seed,
           "train_stacks": args.train_stacks, "stress_stacks": args.stress_stacks,
           "label_radius": args.label_radius, "data_s": round(t_data, 1),
           "train_s": round(t_train, 2), "ms_per_step": round(1e3 * t_train / args.steps, 3),
           "loss": hist[::10] + hist[-1:], "train_metrics": m_train, "eval_metrics": m_eval}
    print(json.dumps(rep))
    if args.log:
        json.dump(rep, open(args.log, "w"))


if __name__ == "__main__":
    main()
