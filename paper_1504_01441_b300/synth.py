"""Seeded synthetic exposure stacks shaped like the paper's two-shot 5 MP / VGA pairs.

This module only *makes inputs*: it renders a procedural scene, exposes it at
several exposure times, moves the camera and a few objects between shots, and
adds sensor noise. It contains none of the registration or merge arithmetic of
the method, so it may feed both the CPU oracle and the CUDA path.

Scene recipe (all draws from one seeded PCG64 stream):
  * background: constant luma U(0, 40), chroma 0;
  * 200 Gaussian blobs composited front-to-back with alpha = exp(-r^2 / 2 s^2)
    (support 4 s), s ~ U(4, W/20);
  * 50 axis-aligned hard-edged rectangles, side ~ U(8, W/8), rendered with 4x4
    supersampling of the indicator;
  * primitive luma 255 * u**2.5 with u ~ U(0, 1): a dark-skewed histogram like an
    expose-to-the-right short exposure (Sec. 2.1) so that the x4 frame saturates
    only in the highlights; chroma offsets U(-20, 20) per primitive;
  * "movers": 64x64 rectangles painted last, displaced independently in every
    source frame by U(-16, 16) px.

Geometry of source frame k: a map B_k from source pixel q to scene coordinates,
B_k(q) = c + s R(theta) (q - c) + t + f(q) with s = 1 +- 2 %, theta = +-1 deg,
t = +-8 px, and f a smooth field interpolated (bicubic Lagrange) from a 4x4
grid of U(-A, A) values. The reference frame uses the identity map.

Exposure: frame value = clip(round(r_k * S(B_k(q)) + n)), n ~ N(0, sigma^2),
with r_k the exposure ratio t_k / t_ref (chroma: 128 + r_k * C + n).
Ground truth: for every reference pixel p the source position B_k^{-1}(p)
(Newton iterations in float64), used only to report end-point error.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 0x15040144100


@dataclasses.dataclass
class Frame:
    y: np.ndarray                      # uint8 [H, W]
    u: Optional[np.ndarray] = None     # uint8 [H/2, W/2] or None (luma-only stacks)
    v: Optional[np.ndarray] = None


@dataclasses.dataclass
class Stack:
    ref: Frame
    srcs: List[Frame]
    ratios: List[Tuple[int, int]]      # exposure ratio t_src / t_ref of every source, as num/den
    gt: List[Optional[Tuple[np.ndarray, np.ndarray]]]  # per source: (x, y) float32 [H, W] or None
    width: int
    height: int
    seed: int


@dataclasses.dataclass
class StackSpec:
    width: int
    height: int
    ratios: Sequence[Tuple[int, int]] = ((4, 1),)
    noise_sigma: float = 1.0
    field_amp: float = 3.0
    movers: int = 1
    chroma: bool = True
    n_blobs: int = 200
    n_rects: int = 50
    scale_pct: float = 0.02
    rot_deg: float = 1.0
    shift_px: float = 8.0
    mover_size: int = 64
    mover_shift: float = 16.0
    with_gt: bool = True
    scene_gain: float = 1.0   # scales every primitive's luma (a dark scene: < 1)


# The two single-stack workloads: a VGA luma pair (T=16, R=4) and the paper's
# 5 MP YUV420 pair (T=32, R=6).
VGA_LUMA = StackSpec(640, 480, ratios=((4, 1),), noise_sigma=1.0, field_amp=3.0,
                     movers=1, chroma=False)
FIVE_MP = StackSpec(2592, 1944, ratios=((4, 1),), noise_sigma=1.5, field_amp=4.0,
                    movers=3, chroma=True)


class _Geometry:
    """Source-pixel -> scene-coordinate map B(q) = similarity(q) + f(q)."""

    def __init__(self, rng: np.random.Generator, w: int, h: int, spec: StackSpec,
                 identity: bool):
        self.w, self.h = w, h
        self.cx, self.cy = (w - 1) / 2.0, (h - 1) / 2.0
        if identity:
            self.s, self.th, self.tx, self.ty = 1.0, 0.0, 0.0, 0.0
            self.gx = np.zeros((4, 4))
            self.gy = np.zeros((4, 4))
        else:
            self.s = 1.0 + rng.uniform(-spec.scale_pct, spec.scale_pct)
            self.th = math.radians(rng.uniform(-spec.rot_deg, spec.rot_deg))
            self.tx = rng.uniform(-spec.shift_px, spec.shift_px)
            self.ty = rng.uniform(-spec.shift_px, spec.shift_px)
            a = spec.field_amp
            self.gx = rng.uniform(-a, a, size=(4, 4))
            self.gy = rng.uniform(-a, a, size=(4, 4))
        self.identity = identity
        c, s = math.cos(self.th), math.sin(self.th)
        self.a11, self.a12 = self.s * c, -self.s * s
        self.a21, self.a22 = self.s * s, self.s * c

    @staticmethod
    def _monomial(g):
        """Coefficients c[b, a] of sum_ij g[j, i] L_i(u) L_j(v) as sum_ab c[b, a] u^a v^b,
        where L_i is the cubic Lagrange basis on the nodes 0, 1, 2, 3."""
        # rows: Lagrange basis polynomial i; columns: coefficient of t^a
        m = np.array([[1.0, -11.0 / 6.0, 1.0, -1.0 / 6.0],
                      [0.0, 3.0, -5.0 / 2.0, 1.0 / 2.0],
                      [0.0, -3.0 / 2.0, 2.0, -1.0 / 2.0],
                      [0.0, 1.0 / 3.0, -1.0 / 2.0, 1.0 / 6.0]])
        return m.T @ g @ m   # [b, a]: (v^b) x (u^a)

    def _coeffs(self):
        if not hasattr(self, "_cx"):
            self._cx = self._monomial(self.gx.T).T
            self._cy = self._monomial(self.gy.T).T
        return self._cx, self._cy

    def field(self, qx, qy, deriv=False):
        sx = 3.0 / max(self.w - 1, 1)
        sy = 3.0 / max(self.h - 1, 1)
        u, v = qx * sx, qy * sy
        out = []
        for c in self._coeffs():
            # c[b, a] multiplies u^a v^b; Horner in u per power of v, then in v
            p = [((c[b, 3] * u + c[b, 2]) * u + c[b, 1]) * u + c[b, 0] for b in range(4)]
            val = ((p[3] * v + p[2]) * v + p[1]) * v + p[0]
            if deriv:
                pu = [(3.0 * c[b, 3] * u + 2.0 * c[b, 2]) * u + c[b, 1] for b in range(4)]
                du = (((pu[3] * v + pu[2]) * v + pu[1]) * v + pu[0]) * sx
                dv = ((3.0 * p[3] * v + 2.0 * p[2]) * v + p[1]) * sy
                out.append((val, du, dv))
            else:
                out.append(val)
        if deriv:
            (fx, fxx, fxy), (fy, fyx, fyy) = out
            return fx, fy, fxx, fxy, fyx, fyy
        return out[0], out[1]

    def __call__(self, qx, qy):
        if self.identity:
            return qx, qy
        dx, dy = qx - self.cx, qy - self.cy
        bx = self.cx + self.a11 * dx + self.a12 * dy + self.tx
        by = self.cy + self.a21 * dx + self.a22 * dy + self.ty
        fx, fy = self.field(qx, qy)
        return bx + fx, by + fy

    def inverse(self, px, py, iters=4):
        """Newton solve of B(q) = p for every p (float64)."""
        if self.identity:
            return px.copy(), py.copy()
        det = self.a11 * self.a22 - self.a12 * self.a21
        rx, ry = px - self.cx - self.tx, py - self.cy - self.ty
        qx = self.cx + (self.a22 * rx - self.a12 * ry) / det
        qy = self.cy + (-self.a21 * rx + self.a11 * ry) / det
        for _ in range(iters):
            dx, dy = qx - self.cx, qy - self.cy
            fx, fy, fxx, fxy, fyx, fyy = self.field(qx, qy, deriv=True)
            ex = self.cx + self.a11 * dx + self.a12 * dy + self.tx + fx - px
            ey = self.cy + self.a21 * dx + self.a22 * dy + self.ty + fy - py
            j11, j12 = self.a11 + fxx, self.a12 + fxy
            j21, j22 = self.a21 + fyx, self.a22 + fyy
            d = j11 * j22 - j12 * j21
            qx = qx - (j22 * ex - j12 * ey) / d
            qy = qy - (-j21 * ex + j11 * ey) / d
        return qx, qy

    def max_disp(self):
        corners = np.array([[0, 0], [self.w - 1, 0], [0, self.h - 1], [self.w - 1, self.h - 1]],
                           dtype=np.float64)
        bx, by = self(corners[:, 0], corners[:, 1])
        d = np.hypot(bx - corners[:, 0], by - corners[:, 1]).max()
        return float(d + 4.0 * np.abs(self.gx).max() + 4.0 * np.abs(self.gy).max() + 2.0)


def _draw_scene(rng: np.random.Generator, w: int, h: int, spec: StackSpec):
    g = spec.scene_gain
    bg = rng.uniform(0.0, 40.0) * g
    blobs = []
    for _ in range(spec.n_blobs):
        cx, cy = rng.uniform(0, w), rng.uniform(0, h)
        s = rng.uniform(4.0, max(w / 20.0, 4.5))
        a = 255.0 * rng.uniform() ** 2.5 * g
        cu, cv = rng.uniform(-20, 20) * g, rng.uniform(-20, 20) * g
        blobs.append((cx, cy, s, a, cu, cv))
    rects = []
    for _ in range(spec.n_rects):
        rw = rng.uniform(8.0, max(w / 8.0, 9.0))
        rh = rng.uniform(8.0, max(w / 8.0, 9.0))
        x0, y0 = rng.uniform(-rw / 2, w - rw / 2), rng.uniform(-rh / 2, h - rh / 2)
        a = 255.0 * rng.uniform() ** 2.5 * g
        cu, cv = rng.uniform(-20, 20) * g, rng.uniform(-20, 20) * g
        rects.append((x0, y0, x0 + rw, y0 + rh, a, cu, cv))
    movers = []
    for _ in range(spec.movers):
        m = spec.mover_size
        x0, y0 = rng.uniform(m, max(w - 2 * m, m + 1)), rng.uniform(m, max(h - 2 * m, m + 1))
        a = 255.0 * rng.uniform() ** 2.5 * g
        cu, cv = rng.uniform(-20, 20) * g, rng.uniform(-20, 20) * g
        movers.append((x0, y0, x0 + m, y0 + m, a, cu, cv))
    return bg, blobs, rects, movers


_SS = (np.arange(4) + 0.5) / 4.0 - 0.5   # 4x4 supersampling offsets


def _render(geom: _Geometry, scene, mover_shifts, out_w, out_h, step, offset, chroma):
    """Render the scene sampled at B(step*i + offset) for an out_h x out_w grid.

    Returns luma (float64) or the (U, V) chroma offsets when chroma=True.
    """
    bg, blobs, rects, movers = scene
    margin = geom.max_disp() + 2.0 * step
    qx1 = np.arange(out_w, dtype=np.float64) * step + offset
    qy1 = np.arange(out_h, dtype=np.float64) * step + offset
    qx, qy = np.meshgrid(qx1, qy1)
    bx, by = geom(qx, qy)
    if chroma:
        outs = [np.zeros((out_h, out_w)), np.zeros((out_h, out_w))]
    else:
        outs = [np.full((out_h, out_w), bg)]

    def box(x0, y0, x1, y1):
        i0 = max(int(math.floor((x0 - margin - offset) / step)), 0)
        i1 = min(int(math.ceil((x1 + margin - offset) / step)) + 1, out_w)
        j0 = max(int(math.floor((y0 - margin - offset) / step)), 0)
        j1 = min(int(math.ceil((y1 + margin - offset) / step)) + 1, out_h)
        return j0, j1, i0, i1

    for (cx, cy, s, a, cu, cv) in blobs:
        j0, j1, i0, i1 = box(cx - 4 * s, cy - 4 * s, cx + 4 * s, cy + 4 * s)
        if j0 >= j1 or i0 >= i1:
            continue
        ex, ey = bx[j0:j1, i0:i1] - cx, by[j0:j1, i0:i1] - cy
        r2 = ex * ex + ey * ey
        al = np.exp(-r2 / (2 * s * s))
        al[r2 > 16 * s * s] = 0.0
        vals = (cu, cv) if chroma else (a,)
        for o, val in zip(outs, vals):
            sub = o[j0:j1, i0:i1]
            sub += al * (val - sub)

    def paint_rect(x0, y0, x1, y1, vals):
        j0, j1, i0, i1 = box(x0, y0, x1, y1)
        if j0 >= j1 or i0 >= i1:
            return
        sqx, sqy = qx[j0:j1, i0:i1], qy[j0:j1, i0:i1]
        cov = np.zeros(sqx.shape)
        for oy in _SS:
            for ox in _SS:
                sx, sy = geom(sqx + ox * step, sqy + oy * step)
                cov += ((sx >= x0) & (sx < x1) & (sy >= y0) & (sy < y1))
        cov /= 16.0
        for o, val in zip(outs, vals):
            sub = o[j0:j1, i0:i1]
            sub += cov * (val - sub)

    for (x0, y0, x1, y1, a, cu, cv) in rects:
        paint_rect(x0, y0, x1, y1, (cu, cv) if chroma else (a,))
    for k, (x0, y0, x1, y1, a, cu, cv) in enumerate(movers):
        dx, dy = mover_shifts[k]
        paint_rect(x0 + dx, y0 + dy, x1 + dx, y1 + dy, (cu, cv) if chroma else (a,))
    if chroma:
        return outs[0], outs[1]
    return np.clip(outs[0], 0.0, 255.0)


def _expose(rng, signal, ratio, sigma, bias=0.0):
    v = bias + ratio * signal + rng.normal(0.0, sigma, size=signal.shape)
    return np.clip(np.rint(v), 0, 255).astype(np.uint8)


def make_stack(spec: StackSpec, seed: int) -> Stack:
    """Render one reference frame plus one source frame per entry of spec.ratios."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w, h = spec.width, spec.height
    if spec.chroma and (w % 2 or h % 2):
        raise ValueError("YUV420 stacks need even width and height")
    scene = _draw_scene(rng, w, h, spec)
    n_movers = len(scene[3])

    def frame(geom, shifts, ratio):
        lum = _render(geom, scene, shifts, w, h, 1.0, 0.0, False)
        y = _expose(rng, lum, ratio, spec.noise_sigma)
        if not spec.chroma:
            return Frame(y)
        cu, cv = _render(geom, scene, shifts, w // 2, h // 2, 2.0, 0.5, True)
        return Frame(y, _expose(rng, cu, ratio, spec.noise_sigma, 128.0),
                     _expose(rng, cv, ratio, spec.noise_sigma, 128.0))

    ident = _Geometry(rng, w, h, spec, identity=True)
    ref = frame(ident, [(0.0, 0.0)] * n_movers, 1.0)
    srcs, gts = [], []
    for (num, den) in spec.ratios:
        geom = _Geometry(rng, w, h, spec, identity=False)
        shifts = [tuple(rng.uniform(-spec.mover_shift, spec.mover_shift, size=2))
                  for _ in range(n_movers)]
        srcs.append(frame(geom, shifts, num / den))
        if spec.with_gt:
            px, py = np.meshgrid(np.arange(w, dtype=np.float64), np.arange(h, dtype=np.float64))
            gx, gy = geom.inverse(px, py)
            gts.append((gx.astype(np.float32), gy.astype(np.float32)))
        else:
            gts.append(None)
    return Stack(ref, srcs, [tuple(r) for r in spec.ratios], gts, w, h, seed)


def stack_seed(config_index: int, stack_index: int = 0) -> int:
    return SEED_BASE + 1000 * config_index + stack_index


def random_flow(rng: np.random.Generator, w: int, h: int, amp: float, grid: int = 5):
    """A smooth synthetic displacement field (float32 u, v) for isolated warp/merge tests."""
    gx = rng.uniform(-amp, amp, size=(grid, grid))
    gy = rng.uniform(-amp, amp, size=(grid, grid))
    xs = np.linspace(0, grid - 1, w)
    ys = np.linspace(0, grid - 1, h)
    def interp(g):
        rows = np.stack([np.interp(xs, np.arange(grid), g[j]) for j in range(grid)])
        return np.stack([np.interp(ys, np.arange(grid), rows[:, i]) for i in range(w)], axis=1)
    return interp(gx).astype(np.float32), interp(gy).astype(np.float32)


def random_homography(rng: np.random.Generator, scale=0.02, rot_deg=1.0, shift_n=0.006,
                      persp=0.002):
    """A near-identity 3x3 homography in normalized coordinates (h22 = 1)."""
    s = 1.0 + rng.uniform(-scale, scale)
    th = math.radians(rng.uniform(-rot_deg, rot_deg))
    c, si = math.cos(th), math.sin(th)
    H = np.array([[s * c, -s * si, rng.uniform(-shift_n, shift_n)],
                  [s * si, s * c, rng.uniform(-shift_n, shift_n)],
                  [rng.uniform(-persp, persp), rng.uniform(-persp, persp), 1.0]])
    return H


# --------------------------------------------------------------------------
# Method parameters of the workloads (inputs, like the frames). Paper values:
# 21x21 patches, up to 5 levels, levels >= 100 px, candidate grid spacing T/16
# (Sec. 2.6), sigma_s = 400 (Sec. 2.6); the rest are readings of silences.
def method_params(tile: int = 32, radius: int = 6, **over) -> dict:
    p = dict(tile=tile, radius=radius, patch_half=10, levels_max=5, min_level_size=100,
             grid_half=4, quad=10, corner_thresh=2, weed_iters=512, weed_delta_min=8,
             weed_delta_div=20, norm_mode=0, dt_iters=3, ssim_radius=5, propagate_full=0,
             weed_eps=1.5, sigma_s=400.0, sigma_r=0.5, ssim_sigma=1.5, we_sigma=0.2,
             flow_eps=1e-20, weed_seed=0x1504014410, output_mode=0, search_threads=0)
    p.update(over)
    return p


def mixed_spec(stack_index: int, config_index: int = 3, with_gt: bool = False) -> StackSpec:
    """One stack of the mixed batch workload: luma area U(1, 12) MP, aspect 4:3 or 16:9
    (even sides), 2 or 3 frames, YUV420, noise 1.5 DN, +-4 px local field, 3 movers. The
    reference is the darkest frame; every other frame draws its ratio from {2, 4, 8}.
    The draws come from their own PCG64 stream seeded by the stack's seed, so a stack's
    shape does not depend on which other stacks are made."""
    rng = np.random.Generator(np.random.PCG64(stack_seed(config_index, stack_index) ^ 0x5EED))
    area = rng.uniform(1.0, 12.0) * 1e6
    aspect = (4.0 / 3.0) if rng.uniform() < 0.5 else (16.0 / 9.0)
    nsrc = 1 if rng.uniform() < 0.5 else 2
    ratios = tuple((int(rng.choice((2, 4, 8))), 1) for _ in range(nsrc))
    w = 2 * int(round(math.sqrt(area * aspect) / 2.0))
    h = 2 * int(round(w / aspect / 2.0))
    return StackSpec(w, h, ratios=ratios, noise_sigma=1.5, field_amp=4.0, movers=3,
                     chroma=True, with_gt=with_gt)


def make_mixed_stack(stack_index: int, config_index: int = 3, with_gt: bool = False) -> Stack:
    return make_stack(mixed_spec(stack_index, config_index, with_gt),
                      stack_seed(config_index, stack_index))


def dark_spec(stops: int, width: int = 640, height: int = 480) -> StackSpec:
    """A scene 2^stops darker than the headline one, seen by a dark reference (values
    mostly below 255 / 2^stops, noise 1 DN) and a source 2^stops brighter (a normal
    exposure): the reference lies `stops` stops under the source."""
    return StackSpec(width, height, ratios=((2 ** stops, 1),), noise_sigma=1.0, field_amp=3.0,
                     movers=1, chroma=False, scene_gain=1.0 / 2 ** stops)


# The learned search on 5 MP pairs with +-8 px local fields (the headline recipe otherwise).
LEARNED8_SPEC = StackSpec(2592, 1944, ratios=((4, 1),), noise_sigma=1.5, field_amp=8.0,
                          movers=3, chroma=True)


def make_learned8_stack(stack_index: int) -> Stack:
    """Seeds from index 50000 up: apart from the predictor's training stacks."""
    return make_stack(LEARNED8_SPEC, stack_seed(4, 50000 + stack_index))


# Learned + batched at scale: 4000 x 3000 three-frame stacks, exposures 1/4, 1 and 4 times
# the reference's (the r = 1 frame is the reference), +-8 px local fields, 5 movers.
SCALE12_SPEC = StackSpec(4000, 3000, ratios=((1, 4), (4, 1)), noise_sigma=1.5, field_amp=8.0,
                         movers=5, chroma=True, with_gt=False)


def make_scale12_stack(stack_index: int) -> Stack:
    return make_stack(SCALE12_SPEC, stack_seed(5, stack_index))


def make_scale12_stacks(n: int, processes=None):
    """make_scale12_stack for stacks 0..n-1 in a spawn-started process pool."""
    import multiprocessing as mp
    import os
    k = processes or min(n, os.cpu_count() or 1)
    if k <= 1:
        return [make_scale12_stack(i) for i in range(n)]
    with mp.get_context("spawn").Pool(k) as pool:
        return pool.map(make_scale12_stack, range(n))


# Sizes of the scaling sweep: 4:3 frames from VGA to 20 MP (widths multiples of 32).
SWEEP_SIZES = ((640, 480), (1280, 960), (1600, 1200), (2048, 1536), (2592, 1944), (3264, 2448),
               (4000, 3000), (4608, 3456), (5184, 3888))


def sweep_spec(w: int, h: int) -> StackSpec:
    """The headline pair recipe (ratio 4, noise 1.5 DN, +-4 px fields, 3 movers, YUV420)
    at another size."""
    return dataclasses.replace(FIVE_MP, width=w, height=h, with_gt=False)


def make_sweep_stack(w: int, h: int) -> Stack:
    return make_stack(sweep_spec(w, h), stack_seed(6, w))


def make_sweep_stacks(sizes=SWEEP_SIZES, processes=None):
    """make_sweep_stack for every size in a spawn-started process pool."""
    import multiprocessing as mp
    import os
    n = processes or min(len(sizes), os.cpu_count() or 1)
    if n <= 1:
        return [make_sweep_stack(w, h) for w, h in sizes]
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.starmap(make_sweep_stack, sizes)


def make_stacks_parallel(jobs, processes=None):
    """make_mixed_stack over (stack_index, config_index, with_gt) jobs in a spawn-started
    process pool (safe after CUDA is initialized); returns the stacks in job order."""
    import multiprocessing as mp
    import os
    jobs = list(jobs)
    n = processes or min(len(jobs), os.cpu_count() or 1)
    if n <= 1:
        return [make_mixed_stack(*j) for j in jobs]
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.starmap(make_mixed_stack, jobs)


def make_spec_stacks_parallel(spec: StackSpec, seeds, processes=None):
    """make_stack(spec, seed) for every seed in a spawn-started process pool; returns the
    stacks in seed order."""
    import multiprocessing as mp
    import os
    seeds = list(seeds)
    n = processes or min(len(seeds), os.cpu_count() or 1)
    if n <= 1:
        return [make_stack(spec, sd) for sd in seeds]
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.starmap(make_stack, [(spec, sd) for sd in seeds])


WORKLOADS = {
    "vga_luma_pair": (VGA_LUMA, dict(tile=16, radius=4)),
    "5mp_yuv420_pair": (FIVE_MP, dict(tile=32, radius=6)),
}
