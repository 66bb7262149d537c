"""Pins of the exposure-fusion oracle (oracle/fusion.py, row f1) against definitions it
does not share code with: scipy's filters for REDUCE and EXPAND, exactness of linear
interpolation, the reconstruction identity of Laplacian pyramids, linearity of the
blend, and the weight formulas at points with known values."""
import math

import numpy as np
import pytest
from scipy import ndimage

from oracle import fusion as F


def test_levels():
    assert F.n_levels(640, 480) == 8 and F.n_levels(2592, 1944) == 10 and F.n_levels(3, 1) == 1


@pytest.mark.parametrize("shape", [(37, 50), (16, 16), (9, 5)])
def test_reduce_is_the_binomial_filter_with_replicated_edges(shape):
    a = np.random.default_rng(1).random(shape)
    want = ndimage.correlate1d(a, F.G5, axis=1, mode="nearest")[:, ::2]
    want = ndimage.correlate1d(want, F.G5, axis=0, mode="nearest")[::2, :]
    assert np.abs(F.reduce2(a) - want).max() < 1e-14


def test_expand_is_four_times_the_filter_of_the_zero_inserted_image_inside():
    rng = np.random.default_rng(2)
    c = rng.random((20, 24))
    n0, n1 = 40, 48
    up = np.zeros((n0, n1))
    up[::2, ::2] = c
    want = 4.0 * ndimage.correlate(up, np.outer(F.G5, F.G5), mode="constant")
    got = F.expand2(c, (n0, n1))
    assert np.abs(got[3:-3, 3:-3] - want[3:-3, 3:-3]).max() < 1e-14


def test_expand_reproduces_constants_and_ramps():
    c = np.full((7, 9), 3.25)
    assert np.abs(F.expand2(c, (14, 17)) - 3.25).max() < 1e-15
    k = np.arange(10, dtype=float)
    e = F.expand_axis(k, 19, 0)
    # x / 2, exact away from the clamped ends (output 0 reads c[-1] -> c[0])
    assert np.abs(e[1:18] - np.arange(1, 18) / 2.0).max() < 1e-15


def test_laplacian_pyramid_reconstructs_exactly():
    a = np.random.default_rng(3).random((61, 83))
    lv = F.n_levels(83, 61)
    assert np.abs(F.collapse(F.laplacian_pyramid(a, lv)) - a).max() < 1e-13


def test_blend_is_linear():
    rng = np.random.default_rng(4)
    a, b = rng.random((33, 47)), rng.random((33, 47))
    half = np.full((33, 47), 0.5)
    out = F.blend([a, b], [half, half], F.n_levels(47, 33))
    assert np.abs(out - 0.5 * (a + b)).max() < 1e-13
    out = F.blend([a, a], [rng.random((33, 47)), rng.random((33, 47))], F.n_levels(47, 33))
    s = F.blend([a], [np.ones((33, 47))], F.n_levels(47, 33))
    assert np.abs(s - a).max() < 1e-13


def test_weight_formulas():
    assert F.well_exposedness(127.5) == 1.0
    assert math.isclose(F.well_exposedness(0.0), math.exp(-0.25 / 0.08), rel_tol=1e-15)
    x = np.arange(12, dtype=float)
    ramp = np.tile(x, (9, 1)) * 0.01 + np.arange(9)[:, None] * 0.02
    assert np.abs(F.contrast(ramp)[1:-1, 1:-1]).max() < 1e-15  # the Laplacian of a plane
    spot = np.zeros((7, 7))
    spot[3, 3] = 0.5
    c = F.contrast(spot)
    assert c[3, 3] == 2.0 and c[2, 3] == c[4, 3] == c[3, 2] == c[3, 4] == 0.5 and c[0, 0] == 0
    rng = np.random.default_rng(5)
    zs = [rng.uniform(0, 255, (10, 12)) for _ in range(3)]
    ws = F.weights(zs, [None, rng.random((10, 12)), np.zeros((10, 12))])
    assert np.abs(sum(ws) - 1.0).max() < 1e-15
    assert ws[2].max() < 1e-9  # a zero SSIM map removes the frame


def test_fuse_of_identical_frames_and_a_dominant_frame():
    rng = np.random.default_rng(6)
    y = rng.uniform(0, 255, (48, 64))
    u = rng.uniform(0, 255, (24, 32))
    v = rng.uniform(0, 255, (24, 32))
    fy, fu, fv = F.fuse(y, u, v, [(y, u, v)], [rng.random((48, 64))])
    assert np.abs(fy - y).max() < 1e-9
    assert np.abs(fu - (u - 128.0)).max() < 1e-9 and np.abs(fv - (v - 128.0)).max() < 1e-9
    # a source with SSIM 0 everywhere: the output is the reference
    y2 = rng.uniform(0, 255, (48, 64))
    fy, _, _ = F.fuse(y, None, None, [(y2, None, None)], [np.zeros((48, 64))])
    assert np.abs(fy - y).max() < 1e-6


def test_contrast_vanishes_on_planes_and_the_floor_then_decides():
    # the discrete Laplacian of a plane is 0 (up to binary64 rounding) away from the border,
    # so on two planar frames with equal well-exposedness the normalized weights are set by
    # the 1e-12 floor alone: one half each
    y, x = np.mgrid[0:24, 0:32].astype(np.float64)
    a = 40.0 + 1.75 * x + 0.5 * y
    b = 90.0 + 0.25 * x - 1.125 * y
    ca = F.contrast(a / 255.0)[1:-1, 1:-1]
    cb = F.contrast(b / 255.0)[1:-1, 1:-1]
    assert np.abs(ca).max() < 1e-14 and np.abs(cb).max() < 1e-14
    w = F.weights([a, b], [None, np.ones_like(b)], use_contrast=True)
    we_a, we_b = F.well_exposedness(a), F.well_exposedness(b)
    inner = (slice(1, -1), slice(1, -1))
    # contrast * well-exposedness is far below the floor, so the ratio is the floor's (1:1)
    assert np.all(ca * we_a[inner] < 1e-13) and np.all(cb * we_b[inner] < 1e-13)
    assert np.allclose(w[0][inner], 0.5, atol=1e-3) and np.allclose(w[0][inner] + w[1][inner], 1.0)
