"""Tile size T, search radius R and search block shape B per image-size bucket for
batches of mixed stacks.

The paper runs one tile size and one search radius for its 5 MP pairs (Sec. 2.6,
Sec. 3). A batch that mixes 1-12 MP stacks can do better per size: small images
have fewer tiles to amortize a wide search, large ones more. For every size bucket
this module measures each candidate (T, R) on seeded generator stacks of that
bucket:

  * time: device time per stack of the batched fused call with one copy of the stack
    on each of four lanes, as stacks of a bucket run in a batch (CUDA-graph replay,
    CUDA events, L2 flushed before every replay);
  * error: the end-point error of the registration H^0 + F (Eq. 3 homography plus
    the dense residual flow of Sec. 2.4) against the generator's ground-truth map,
    averaged over the reference pixels whose true source position lies inside the
    source image;

and keeps the fastest candidate whose error is no larger than that of the default
(T = 32, R = 6). A second stage then times the chosen (T, R) with each block shape of
the tile search -- B threads per tile CTA, 64, 128 or 256 -- and keeps the fastest;
the search's results are exact integers that do not depend on B, so the error stays
that of the first stage. The selection rules and the bucket lookup are plain host code
(`pick`, `pick_block`, `bucket_of`, `pick_of`); measuring needs the GPU. `python -m
paper_1504_01441_b300.autotune` writes the table next to this file, where
`load_table` finds it (`--blocks-only` re-runs the second stage on an existing table).
"""
from __future__ import annotations

import json
import os
from typing import Dict, List, Optional, Sequence, Tuple

BUCKETS_MP = (2.0, 4.0, 8.0, 12.0)          # upper bounds of the luma-area buckets
TILES = (16, 24, 32, 48)
RADII = (3, 4, 5, 6, 7, 8)
DEFAULT = (32, 6)
BLOCKS = (64, 128, 256)                     # threads per tile CTA of the search
DEFAULT_BLOCK = 128
TABLE_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_table.json")


def candidates() -> List[Tuple[int, int]]:
    return [(t, r) for t in TILES for r in RADII]


def bucket_of(w: int, h: int, buckets: Sequence[float] = BUCKETS_MP) -> int:
    """Index of the first bucket whose bound holds w*h megapixels (the last one beyond)."""
    mp = w * h / 1e6
    for i, b in enumerate(buckets):
        if mp <= b:
            return i
    return len(buckets) - 1


def pick(results: Dict[Tuple[int, int], Tuple[float, float]],
         default: Tuple[int, int] = DEFAULT) -> Tuple[int, int]:
    """results: (T, R) -> (time, error). The fastest candidate whose error is <= the
    default's; ties in time go to the smaller (T, R). The default must be measured."""
    if default not in results:
        raise ValueError("the default candidate was not measured")
    bound = results[default][1]
    ok = [(tr, te) for tr, te in results.items() if te[1] <= bound]
    return min(ok, key=lambda kv: (kv[1][0], kv[0]))[0]


def pick_block(times: Dict[int, float]) -> int:
    """times: block shape B -> time. The fastest; ties go to the smaller B."""
    if not times:
        raise ValueError("no block shape was measured")
    return min(times.items(), key=lambda kv: (kv[1], kv[0]))[0]


def pick_of(table: Dict, w: int, h: int) -> Tuple[int, int, int]:
    """(T, R, B) of a w x h stack's bucket; a table without block shapes gives B = 0 (the
    library's default, 128)."""
    pk = tuple(table["picks"][bucket_of(w, h, table["buckets_mp"])])
    return (pk[0], pk[1], pk[2] if len(pk) > 2 else 0)


def params_for(w: int, h: int, table: Dict, **over):
    """Library parameters of a w x h stack: the method's defaults with the (T, R, B) of
    its bucket from a tuning table (as returned by load_table)."""
    from . import hdrreg, synth
    t, r, b = pick_of(table, w, h)
    return hdrreg.params_from_dict(synth.method_params(tile=t, radius=r, search_threads=b,
                                                       **over))


def load_table(path: str = TABLE_FILE) -> Dict:
    with open(path) as f:
        table = json.load(f)
    table["picks"] = [tuple(x) for x in table["picks"]]
    return table


# ------------------------------------------------------------------ GPU measurement
def registration_epe(stack, p, device="cuda") -> float:
    """Mean end-point error (pixels) of H^0 + F against the generator ground truth over
    all sources of `stack`, from the library's step calls (a1-a8, the same kernels the
    fused call runs)."""
    import torch
    from . import hdrreg
    dev = torch.device(device)
    ref = torch.from_numpy(stack.ref.y).to(dev)
    h, w = ref.shape
    L = hdrreg.num_levels(w, h, p)
    ys, xs = torch.meshgrid(torch.arange(h, device=dev, dtype=torch.float64),
                            torch.arange(w, device=dev, dtype=torch.float64), indexing="ij")
    xn, yn = (2 * xs - (w - 1)) / w, (2 * ys - (h - 1)) / w
    errs = []
    for k, src_f in enumerate(stack.srcs):
        src = torch.from_numpy(src_f.y).to(dev)
        rn, sn, _ = hdrreg.normalize_exposure(ref, src, hdrreg.NORM_RATIO, stack.ratios[k])
        pr, ps = hdrreg.build_pyramid(rn, L), hdrreg.build_pyramid(sn, L)
        Hc = torch.tensor([1, 0, 0, 0, 1, 0, 0, 0, 1], dtype=torch.float64, device=dev)
        counter = torch.zeros(1, dtype=torch.int32, device=dev)
        for lv in range(L - 1, -1, -1):
            lh, lw = pr[lv].shape
            cxy, mxy, _, valid = hdrreg.local_search(pr[lv], ps[lv], Hc, p)
            if hdrreg.lib().hdrreg_weed_fit_supported(valid.numel()):
                mask, Hc, _ = hdrreg.weed_fit(cxy, mxy, valid, lw, lh, p, p.weed_seed + lv, Hc,
                                              counter=counter)
            else:   # beyond the one-launch plan: the workspace weeding, then the fit
                mask = hdrreg.weed(cxy, mxy, valid, lw, lh, p, p.weed_seed + lv)
                Hc, _ = hdrreg.fit_homography(cxy, mxy, mask, lw, lh, Hc)
        fu, fv = hdrreg.flow_upsample(rn, cxy, mxy, mask, Hc, p)
        H = Hc.view(3, 3)
        den = H[2, 0] * xn + H[2, 1] * yn + H[2, 2]
        hx = ((H[0, 0] * xn + H[0, 1] * yn + H[0, 2]) / den * w + (w - 1)) / 2
        hy = ((H[1, 0] * xn + H[1, 1] * yn + H[1, 2]) / den * w + (h - 1)) / 2
        gx = torch.from_numpy(stack.gt[k][0]).to(dev).double()
        gy = torch.from_numpy(stack.gt[k][1]).to(dev).double()
        inside = (gx >= 0) & (gx <= w - 1) & (gy >= 0) & (gy <= h - 1)
        e = torch.hypot(hx + fu.double() - gx, hy + fv.double() - gy)[inside]
        errs.append(e)
    return float(torch.cat(errs).mean().item())


def _device_stack(stack, device):
    import torch
    def t(a):
        return None if a is None else torch.from_numpy(a).to(device)
    ref = (t(stack.ref.y), t(stack.ref.u), t(stack.ref.v))
    srcs = [(t(s.y), t(s.u), t(s.v)) for s in stack.srcs]
    return ref, srcs, list(stack.ratios)


def fused_time_us(stack, p, reps: int = 5, device="cuda", flush=None, lanes: int = 4) -> float:
    """Device time (us) per stack of the batched fused call on `lanes` copies of `stack`
    (one per lane, as stacks of one bucket run in a batch), replayed from a CUDA graph
    with L2 flushed (a write larger than L2) before each replay; the median replay over
    `lanes`."""
    import torch
    from . import hdrreg
    copies = [_device_stack(stack, device) for _ in range(lanes)]
    h, w = copies[0][0][0].shape
    rm = hdrreg.RegisterMergeBatch(w, h, len(stack.srcs), p, copies[0][0][1] is not None,
                                   slots=lanes, lanes=lanes, device=device)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        rm(copies, stream=s)                     # first call raises kernel smem limits
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rm(copies, stream=s)
    if flush is None:
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    times = []
    with torch.cuda.stream(s):
        for i in range(reps + 1):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            g.replay()
            b.record(s)
            b.synchronize()
            if i:
                times.append(a.elapsed_time(b) * 1e3 / lanes)
    times.sort()
    return times[len(times) // 2]


def tuning_jobs(per_bucket: int = 2, buckets: Sequence[float] = BUCKETS_MP):
    """(stack_index, config_index, with_gt) of the tuning stacks: seeded mixed-workload
    stacks (with ground truth) drawn until every bucket has `per_bucket` of them. They
    use stack indices from 10000 up, apart from those of the measured batch."""
    from . import synth
    need = [per_bucket] * len(buckets)
    jobs, i = [], 10000
    while any(need):
        sp = synth.mixed_spec(i)
        b = bucket_of(sp.width, sp.height, buckets)
        if need[b]:
            need[b] -= 1
            jobs.append((i, 3, True))
        i += 1
    return jobs


def _by_bucket(stacks, buckets):
    groups: List[list] = [[] for _ in buckets]
    for st in stacks:
        groups[bucket_of(st.width, st.height, buckets)].append(st)
    return groups


def tune_blocks(stacks, picks: Sequence[Sequence[int]], blocks: Sequence[int] = BLOCKS,
                reps: int = 5, buckets: Sequence[float] = BUCKETS_MP, device="cuda", log=None,
                flush=None):
    """Second stage: the (T, R) pick of every bucket timed with each block shape of the
    search; -> ([T, R, B] per bucket, {bucket: {B: us}})."""
    import torch
    from . import hdrreg, synth
    if flush is None:
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    out, meas = [], []
    for b, group in enumerate(_by_bucket(stacks, buckets)):
        t, r = picks[b][0], picks[b][1]
        if not group:
            out.append([t, r, DEFAULT_BLOCK])
            meas.append({})
            continue
        times = {}
        for nt in blocks:
            p = hdrreg.params_from_dict(synth.method_params(tile=t, radius=r, search_threads=nt))
            times[nt] = sum(fused_time_us(st, p, reps, device, flush) for st in group) / len(group)
            if log:
                log(f"bucket <= {buckets[b]} MP: T={t} R={r} B={nt}: {times[nt]:.1f} us")
        out.append([t, r, pick_block(times)])
        meas.append({str(k): round(v, 2) for k, v in times.items()})
    return out, meas


def tune(stacks, cands: Optional[Sequence[Tuple[int, int]]] = None, reps: int = 5,
         buckets: Sequence[float] = BUCKETS_MP, device="cuda", log=None,
         blocks: Sequence[int] = BLOCKS) -> Dict:
    """Measure every candidate on the stacks of each bucket, then the block shapes of
    the pick; -> table dict."""
    import torch
    from . import hdrreg, synth
    cands = list(cands or candidates())
    if DEFAULT not in cands:
        cands.append(DEFAULT)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    picks, meas = [], []
    for b, group in enumerate(_by_bucket(stacks, buckets)):
        if not group:
            picks.append(DEFAULT)
            meas.append({})
            continue
        res = {}
        for t, r in cands:
            p = hdrreg.params_from_dict(synth.method_params(tile=t, radius=r))
            us = sum(fused_time_us(st, p, reps, device, flush) for st in group) / len(group)
            epe = sum(registration_epe(st, p, device) for st in group) / len(group)
            res[(t, r)] = (us, epe)
            if log:
                log(f"bucket <= {buckets[b]} MP: T={t} R={r}: {us:.1f} us, EPE {epe:.4f} px")
        picks.append(pick(res))
        meas.append({f"{t},{r}": [round(v[0], 2), round(v[1], 5)] for (t, r), v in res.items()})
    picks3, bmeas = tune_blocks(stacks, picks, blocks, reps, buckets, device, log, flush)
    return {"buckets_mp": list(buckets), "picks": picks3,
            "default": list(DEFAULT), "measurements": meas, "block_measurements": bmeas,
            "stacks": [[st.width, st.height, len(st.srcs), st.seed] for st in stacks],
            "device": torch.cuda.get_device_name(device), "reps": reps, "lanes": 4}


def main():
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--per-bucket", type=int, default=2)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--out", default=TABLE_FILE)
    ap.add_argument("--blocks-only", action="store_true",
                    help="keep the (T, R) picks of the existing table; time the block shapes")
    a = ap.parse_args()
    from . import synth
    stacks = synth.make_stacks_parallel(tuning_jobs(a.per_bucket))   # before any CUDA call
    log = lambda m: print(m, flush=True)
    if a.blocks_only:
        table = load_table()
        picks3, bmeas = tune_blocks(stacks, table["picks"], reps=a.reps,
                                    buckets=table["buckets_mp"], log=log)
        table["picks"], table["block_measurements"] = picks3, bmeas
    else:
        table = tune(stacks, reps=a.reps, log=log)
    with open(a.out, "w") as f:
        json.dump(table, f, indent=1)
    print(json.dumps({"picks": table["picks"], "buckets_mp": table["buckets_mp"]}))


if __name__ == "__main__":
    main()
