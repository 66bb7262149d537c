"""Oracle of the error-tolerant exposure fusion output (row f1): plain float64 numpy.

TEST INFRASTRUCTURE ONLY -- imported by tests/, __graft_entry__.smoke() and the CPU
legs of bench.py, never by the product path.

Sec. 2.5 of the paper fuses the registered stack with the exposure fusion of Mertens et
al. (2007), adding the SSIM map of each registered source as a fourth weight next to
contrast, colour saturation and well-exposedness. Written from those definitions:

  weights   W_k(p) = C_k(p)^wc * WE(Z_k(p)) * Q_k(p) + 1e-12, normalized over the frames,
            C_k = |4 I(p) - I(p-x) - I(p+x) - I(p-y) - I(p+y)| (the absolute Laplacian of
            the luma I = Z / 255, edges replicated), WE(z) = exp(-(z/255 - 0.5)^2 / (2
            sigma^2)), Q_k the SSIM quality map (1 for the reference); colour saturation
            has no luma counterpart and is left out;
  pyramids  Burt and Adelson's: REDUCE filters with g = [1, 4, 6, 4, 1] / 16 along x and
            y (coordinates clamped to the image) and keeps the even samples (sizes
            ceil(n / 2)); EXPAND interpolates back: along one axis, output 2k is
            (c[k-1] + 6 c[k] + c[k+1]) / 8 and output 2k+1 is (c[k] + c[k+1]) / 2 (coarse
            indices clamped), i.e. 4 * sum g(i) g(j) c((x-i)/2, (y-j)/2) over the integer
            positions; levels n = floor(log2(min(w, h))) (at least 1);
  blending  R^l = sum_k G{W_k}^l * L{I_k}^l with L^l = G^l - EXPAND(G^{l+1}) below the top
            level and L = G at the top; the output collapses R from the top down,
            O^l = R^l + EXPAND(O^{l+1});
  chroma    (U - 128) / 255 and (V - 128) / 255 at half resolution, blended with the 2x2
            means of the normalized luma weights;
  output    255 * O (luma) and 255 * O (chroma, signed offsets like the merge's).
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np

G5 = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0


def n_levels(w: int, h: int) -> int:
    return max(1, int(math.floor(math.log2(min(w, h)))))


def reduce_axis(a: np.ndarray, axis: int) -> np.ndarray:
    """Filter with G5 along `axis` (clamped coordinates) and keep the even samples:
    out[k] = sum_i G5[i] a[clamp(2k + i)], i = -2..2."""
    a = np.moveaxis(np.asarray(a, np.float64), axis, 0)
    n = a.shape[0]
    k = np.arange((n + 1) // 2)
    out = sum(G5[i + 2] * a[np.clip(2 * k + i, 0, n - 1)] for i in range(-2, 3))
    return np.moveaxis(out, 0, axis)


def expand_axis(c: np.ndarray, n: int, axis: int) -> np.ndarray:
    """Interpolate `c` (coarse) to length n along `axis`: out[2k] = (c[k-1] + 6 c[k] +
    c[k+1]) / 8, out[2k+1] = (c[k] + c[k+1]) / 2, coarse indices clamped."""
    c = np.moveaxis(np.asarray(c, np.float64), axis, 0)
    m = c.shape[0]
    x = np.arange(n)
    k = x // 2
    cl = lambda j: c[np.clip(j, 0, m - 1)]
    even = (cl(k - 1) + 6.0 * cl(k) + cl(k + 1)) / 8.0
    odd = (cl(k) + cl(k + 1)) / 2.0
    sel = (x % 2 == 0).reshape((n,) + (1,) * (c.ndim - 1))
    return np.moveaxis(np.where(sel, even, odd), 0, axis)


def reduce2(a):
    return reduce_axis(reduce_axis(a, 1), 0)


def expand2(c, shape):
    return expand_axis(expand_axis(c, shape[1], 1), shape[0], 0)


def gaussian_pyramid(a, levels: int) -> List[np.ndarray]:
    pyr = [np.asarray(a, np.float64)]
    for _ in range(levels - 1):
        pyr.append(reduce2(pyr[-1]))
    return pyr


def laplacian_pyramid(a, levels: int) -> List[np.ndarray]:
    g = gaussian_pyramid(a, levels)
    return [g[l] - expand2(g[l + 1], g[l].shape) for l in range(levels - 1)] + [g[-1]]


def collapse(lap: Sequence[np.ndarray]) -> np.ndarray:
    out = lap[-1]
    for l in range(len(lap) - 2, -1, -1):
        out = lap[l] + expand2(out, lap[l].shape)
    return out


def contrast(i: np.ndarray) -> np.ndarray:
    """|4 I(p) - sum of the 4 neighbours| with replicated edges."""
    p = np.pad(np.asarray(i, np.float64), 1, mode="edge")
    return np.abs(4.0 * p[1:-1, 1:-1] - p[:-2, 1:-1] - p[2:, 1:-1] - p[1:-1, :-2] - p[1:-1, 2:])


def well_exposedness(z, sigma=0.2):
    t = np.asarray(z, np.float64) / 255.0 - 0.5
    return np.exp(-(t * t) / (2.0 * sigma * sigma))


def weights(zs: Sequence[np.ndarray], qs: Sequence[Optional[np.ndarray]], use_contrast=True,
            sigma=0.2) -> List[np.ndarray]:
    """Normalized fusion weights of the frames (luma values 0..255; q None = 1)."""
    ws = []
    for z, q in zip(zs, qs):
        wk = well_exposedness(z, sigma)
        if use_contrast:
            wk = wk * contrast(np.asarray(z, np.float64) / 255.0)
        if q is not None:
            wk = wk * q
        ws.append(wk + 1e-12)
    tot = sum(ws)
    return [wk / tot for wk in ws]


def blend(images: Sequence[np.ndarray], wts: Sequence[np.ndarray], levels: int) -> np.ndarray:
    r = None
    for img, wk in zip(images, wts):
        lp = laplacian_pyramid(img, levels)
        gw = gaussian_pyramid(wk, levels)
        term = [gw[l] * lp[l] for l in range(levels)]
        r = term if r is None else [a + b for a, b in zip(r, term)]
    return collapse(r)


def fuse(ref_y, ref_u, ref_v, warped, qs, use_contrast=True, sigma=0.2):
    """ref_*: reference planes (0..255; u, v None for luma only); warped: list of (y, u, v)
    warped sources (0..255); qs: their SSIM maps. -> (Y, U - 128, V - 128) fused, float64."""
    h, w = np.asarray(ref_y).shape
    lv = n_levels(w, h)
    zs = [np.asarray(ref_y, np.float64)] + [np.asarray(s[0], np.float64) for s in warped]
    wts = weights(zs, [None] + list(qs), use_contrast, sigma)
    y = 255.0 * blend([z / 255.0 for z in zs], wts, lv)
    if ref_u is None:
        return y, None, None
    cw, ch = w // 2, h // 2
    wc = [wk[:2 * ch, :2 * cw].reshape(ch, 2, cw, 2).mean(axis=(1, 3)) for wk in wts]
    lc = n_levels(cw, ch)
    us = [np.asarray(ref_u, np.float64)] + [np.asarray(s[1], np.float64) for s in warped]
    vs = [np.asarray(ref_v, np.float64)] + [np.asarray(s[2], np.float64) for s in warped]
    u = 255.0 * blend([(c - 128.0) / 255.0 for c in us], wc, lc)
    v = 255.0 * blend([(c - 128.0) / 255.0 for c in vs], wc, lc)
    return y, u, v
