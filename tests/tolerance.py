"""The FP32 parity rule of the GPU tests, one helper for every test file.

Every FP32 output element (flow, warp, SSIM mask, merge, fusion) must satisfy

    |gpu - oracle| <= rel * max(|oracle|, 1)        (rel = 1e-4)

element by element: the relative error of the element, with a floor of one unit
(1 DN, 1 px, an SSIM of 1) below which the error is absolute. The maximum and the
99.99th percentile of the per-element ratio |gpu - oracle| / max(|oracle|, 1) are
printed with every check.

``exclude`` names elements whose value depends on a discrete decision that the GPU
takes from FP32 sample positions and the oracle from float64 ones, and that the
oracle itself shows to flip within a bound far above the FP32 error (see
``oracle.clip_fragile``). Those elements are left out of the rule and reported
separately: how many there were and how many of them broke the rule.
"""
import numpy as np

REL = 1e-4


def rel_ratio(gpu, orc):
    """per-element |gpu - oracle| / max(|oracle|, 1), float64"""
    g = np.asarray(gpu, np.float64)
    o = np.asarray(orc, np.float64)
    return np.abs(g - o) / np.maximum(np.abs(o), 1.0)


def check_rel(gpu, orc, what, rel=REL, exclude=None, max_excluded_frac=1e-3):
    """Assert the per-element rule; returns the largest per-element ratio."""
    g = np.asarray(gpu, np.float64)
    o = np.asarray(orc, np.float64)
    assert g.shape == o.shape, f"{what}: shape {g.shape} vs {o.shape}"
    r = rel_ratio(g, o)
    nonfinite = ~np.isfinite(g)
    r[nonfinite] = np.inf
    keep = np.ones(r.shape, bool) if exclude is None else ~np.asarray(exclude, bool)
    rk = r[keep]
    worst = float(rk.max()) if rk.size else 0.0
    p9999 = float(np.quantile(rk, 0.9999)) if rk.size else 0.0
    bad = rk > rel
    msg = f"{what}: per-element max {worst:.3e}, 99.99th percentile {p9999:.3e} (limit {rel:.0e})"
    if rk.size and bad.any():
        ri = np.where(keep.ravel())[0][int(np.argmax(rk))]
        idx = np.unravel_index(int(ri), r.shape)
        msg += (f"; {int(bad.sum())} of {rk.size} elements above the limit, worst at {idx}: "
                f"gpu {g[idx]!r} oracle {o[idx]!r}")
    if exclude is not None:
        nex = int((~keep).sum())
        nex_bad = int((r[~keep] > rel).sum())
        msg += (f"; {nex} elements on a fragile clip decision left out, {nex_bad} of them "
                f"above the limit")
        assert nex <= max_excluded_frac * r.size, msg
    print(msg)
    assert not nonfinite.any(), msg
    assert not bad.any(), msg
    return worst


def chroma_exclude(exclude_y):
    """a chroma element is left out when any luma element of its 2x2 block is"""
    if exclude_y is None:
        return None
    e = np.asarray(exclude_y, bool)
    h, w = e.shape
    e = e[: h // 2 * 2, : w // 2 * 2]
    return e[0::2, 0::2] | e[0::2, 1::2] | e[1::2, 0::2] | e[1::2, 1::2]


# Half-side, in pixels, of the square around each sample position inside which the
# oracle's clip decision must not change for the pixel to be compared. The GPU's sample
# positions differ from the oracle's by the float32 flow's error plus the float32
# evaluation of H0. The flow itself is held to 1e-4 * max(|F|, 1), i.e. 1e-3 px for
# flows up to 10 px (measured on the 5 MP pair: below 6e-5 px), so 1e-3 px is the bound.
# On the 2592 x 1944 headline pair 132 of 5.04 M pixels are fragile at this bound.
FRAGILE_DELTA = 1e-3


def fused_fragile(orc, stack, out, cfg, delta=FRAGILE_DELTA):
    """Reference pixels where the clip decision of any source's warped sample is fragile
    (``oracle.clip_fragile`` around the oracle's own sample positions H0(p) + F(p)).
    ``out`` is ``orc.register_merge(..., want_intermediates=True)``."""
    ex = None
    for k, s in enumerate(stack.srcs):
        H = np.eye(3) if cfg.get("propagate_full") else out["H0"][k]
        f = orc.clip_fragile(s.y, H, out["flow_u"][k], out["flow_v"][k], delta)
        ex = f if ex is None else ex | f
    return ex


def check_merged(orc, stack, out, cfg, planes, what="merge"):
    """The fused path's merged planes (y and, for YUV420, u and v; numpy or torch) against
    the oracle's, per element, with the fragile clip decisions left out and reported."""
    ex = fused_fragile(orc, stack, out, cfg)
    for name, g in zip("yuv", planes):
        if g is None or out.get(name) is None:
            continue
        g = g.cpu().numpy() if hasattr(g, "cpu") else g
        if name == "y":
            check_rel(g, out[name], f"{what} {name}", exclude=ex)
        else:  # one fragile luma sample leaves out the chroma element of its 2x2 block
            check_rel(g, out[name], f"{what} {name}", exclude=chroma_exclude(ex),
                      max_excluded_frac=4e-3)


def oracle_tail(orc, stack, out, cfg, flows=None, output="merge", use_contrast=True,
                jitter=None):
    """The oracle's steps after the flow (a9 warp, a10 mask, then the a11 merge or the
    exposure fusion), from the oracle's own H0 and the given per-source flows (default:
    the oracle's). ``jitter`` (a numpy Generator) moves every warped value that is not a
    whole number by one unit of FP32 rounding (relative 2^-24) up or down at random, as
    computing and storing it in FP32 can (whole numbers, from equal taps or whole-pixel
    positions, are exact in FP32).
    -> (y, u, v) float64 planes."""
    from oracle import fusion as F
    ref = stack.ref
    chroma = ref.u is not None
    warped, qs, clips, ratios = [], [], [], []
    for k, s in enumerate(stack.srcs):
        num, den = stack.ratios[k]
        fu, fv = flows[k] if flows is not None else (out["flow_u"][k], out["flow_v"][k])
        if cfg["norm_mode"] == 0:
            ref_n, _ = orc.normalize_ratio(ref.y, s.y, num, den)
            gain, lut = (den / num if num < den else 1.0), None
        else:
            ref_n, gain, lut = orc.histeq_lut(ref.y)[ref.y], 1.0, orc.histeq_lut(s.y)
        H = np.eye(3) if cfg.get("propagate_full") else out["H0"][k]
        wy, wu, wv, clip = orc.warp(s.y, s.u if chroma else None, s.v if chroma else None, H,
                                    fu, fv, want_clip=True)
        if jitter is not None:
            # integer-valued samples (equal taps, whole-pixel positions) are exact in FP32
            def j(a):
                if a is None:
                    return None
                step = 2.0 ** -24 * jitter.choice((-1.0, 1.0), a.shape)
                return np.where(a == np.rint(a), a, a * (1.0 + step))
            wy, wu, wv = j(wy), j(wu), j(wv)
        qs.append(orc.ghost_mask(ref_n, wy, cfg["norm_mode"], gain, lut, cfg["ssim_sigma"],
                                 cfg["ssim_radius"]))
        warped.append((wy, wu, wv))
        clips.append(clip)
        ratios.append(num / den)
    if output == "fusion":
        return F.fuse(ref.y, ref.u, ref.v, warped, qs, use_contrast=use_contrast,
                      sigma=cfg["we_sigma"])
    return orc.merge(ref.y, ref.u, ref.v, warped, qs, ratios, we_sigma=cfg["we_sigma"],
                     clips=clips)


def flow_sensitivity(orc, stack, out, cfg, output="merge", use_contrast=True, rel=REL,
                     random_trials=2, value_trials=2, seed=0):
    """Per plane, how far the oracle's own end-to-end output moves when every source's
    flow moves by what the flow's parity rule allows, d = rel * max(|F|, 1) per component:
    the largest change over the four uniform diagonal shifts (+-d, +-d), over
    ``random_trials`` fields of independent per-pixel signs (+-d), which is what moves
    the differences of neighbouring samples (the fusion's contrast weight), and over
    ``value_trials`` draws of FP32-sized jitter on the warped values (``oracle_tail``).
    The GPU's flow is held only to that bound and its warped values are FP32, so the output
    is determined only to this amount beyond its own rule.
    -> (the oracle's planes, the per-element movement)."""
    rng = np.random.default_rng(seed)
    orc.set_parallel(True)  # the OpenMP build: same bits, less waiting
    try:
        base = oracle_tail(orc, stack, out, cfg, None, output, use_contrast)
        sens = [np.zeros_like(b) if b is not None else None for b in base]
        shifts = [(sx, sy) for sx in (-1.0, 1.0) for sy in (-1.0, 1.0)]
        shifts += ["random"] * random_trials
        for sh in shifts:
            flows = []
            for k in range(len(stack.srcs)):
                fu, fv = out["flow_u"][k], out["flow_v"][k]
                if sh == "random":
                    sx = rng.choice((-1.0, 1.0), fu.shape)
                    sy = rng.choice((-1.0, 1.0), fv.shape)
                else:
                    sx, sy = sh
                flows.append((fu + sx * rel * np.maximum(np.abs(fu), 1.0),
                              fv + sy * rel * np.maximum(np.abs(fv), 1.0)))
            moved = oracle_tail(orc, stack, out, cfg, flows, output, use_contrast)
            for i, (m, b) in enumerate(zip(moved, base)):
                if b is not None:
                    sens[i] = np.maximum(sens[i], np.abs(m - b))
        for _ in range(value_trials):
            moved = oracle_tail(orc, stack, out, cfg, None, output, use_contrast, jitter=rng)
            for i, (m, b) in enumerate(zip(moved, base)):
                if b is not None:
                    sens[i] = np.maximum(sens[i], np.abs(m - b))
    finally:
        orc.set_parallel(False)
    return base, sens


def check_end_to_end(gpu, orc_plane, sens, what, rel=REL, exclude=None, max_excluded_frac=1e-3):
    """|gpu - oracle| <= rel * max(|oracle|, 1) + 4 sens, element by element: the rule plus
    four times the output's movement under the flow's own tolerance (``flow_sensitivity``:
    eight perturbations estimate the largest movement from below; on the exposure fusion the
    worst element measured 1.4 x twice the estimate, so the factor is 4), with the fragile
    clip decisions (``exclude``) left out and counted. Reports how many elements needed the
    second term."""
    g = np.asarray(gpu, np.float64)
    o = np.asarray(orc_plane, np.float64)
    keep = np.ones(o.shape, bool) if exclude is None else ~np.asarray(exclude, bool)
    d = np.abs(g - o)[keep]
    rule = rel * np.maximum(np.abs(o), 1.0)[keep]
    bound = rule + 4.0 * np.asarray(sens)[keep]
    ratio = d / bound
    beyond_rule = int((d > rule).sum())
    nex = int((~keep).sum())
    msg = (f"{what}: per-element max |g-o| / (rule + 4 x flow sensitivity) {ratio.max():.3e}; "
           f"{beyond_rule} of {d.size} elements beyond the bare rule (max "
           f"{(d / rule).max():.3e}), within the flow-propagated bound; {nex} elements on a "
           f"fragile clip decision left out")
    print(msg)
    assert np.isfinite(g).all(), msg
    assert nex <= max_excluded_frac * o.size, msg
    assert (d <= bound).all(), msg + f"; {int((d > bound).sum())} beyond the bound"
