"""Pins of the learned-predictor oracle (oracle/cnn.py) against definitions it does not
share code with: brute-force convolution loops, central finite differences, closed forms
of trivial networks, explicit bfloat16 neighbours, and a hand-worked Adam step."""
import numpy as np
import pytest

from oracle import cnn


def conv_brute(x, W, b, s):
    n, h, w, ci = x.shape
    co, k, _, _ = W.shape
    p = k // 2
    ho, wo = (h + 2 * p - k) // s + 1, (w + 2 * p - k) // s + 1
    y = np.zeros((n, ho, wo, co))
    for a in range(n):
        for i in range(ho):
            for j in range(wo):
                for o in range(co):
                    acc = b[o]
                    for ky in range(k):
                        for kx in range(k):
                            yy, xx = s * i + ky - p, s * j + kx - p
                            if 0 <= yy < h and 0 <= xx < w:
                                acc += float(np.dot(W[o, ky, kx, :], x[a, yy, xx, :]))
                    y[a, i, j, o] = acc
    return y


@pytest.mark.parametrize("stride,k,h,w", [(1, 3, 5, 7), (2, 3, 7, 6), (1, 1, 4, 3), (2, 3, 1, 1)])
def test_conv_forward_brute_force(stride, k, h, w):
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, h, w, 3))
    W = rng.normal(size=(4, k, k, 3))
    b = rng.normal(size=4)
    assert np.allclose(cnn.conv_forward(x, W, b, stride), conv_brute(x, W, b, stride), atol=1e-12)


def test_stride_two_reads_2i_plus_ky_minus_1():
    x = np.zeros((1, 8, 8, 1))
    x[0, 5, 3, 0] = 1.0
    W = np.zeros((1, 3, 3, 1))
    W[0, 2, 0, 0] = 1.0  # tap ky = 2, kx = 0 reads (2i + 1, 2j - 1)
    y = cnn.conv_forward(x, W, np.zeros(1), 2)
    assert y.shape == (1, 4, 4, 1)
    assert y[0, 2, 2, 0] == 1.0 and y.sum() == 1.0


@pytest.mark.parametrize("stride", [1, 2])
def test_conv_backward_finite_differences(stride):
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 5, 6, 2))
    W = rng.normal(size=(3, 3, 3, 2))
    b = rng.normal(size=3)
    G = rng.normal(size=cnn.conv_forward(x, W, b, stride).shape)
    f = lambda x_, W_, b_: float((cnn.conv_forward(x_, W_, b_, stride) * G).sum())
    dx, dW, db = cnn.conv_backward(x, W, G, stride)
    e = 1e-6
    for arr, grad in ((x, dx), (W, dW), (b, db)):
        for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(6)]:
            d = np.zeros_like(arr)
            d[idx] = e
            args = [x, W, b]
            pos = [a is arr for a in args].index(True)
            ap, am = list(args), list(args)
            ap[pos], am[pos] = arr + d, arr - d
            num = (f(*ap) - f(*am)) / (2 * e)
            assert num == pytest.approx(grad[idx], rel=1e-6, abs=1e-8)


TINY = [(2, 3, 3, 1, True), (3, 4, 3, 2, True), (4, 2, 1, 1, False)]


def test_network_gradient_finite_differences():
    rng = np.random.default_rng(3)
    theta = rng.normal(0, 0.5, cnn.n_params(TINY))
    x = rng.normal(size=(2, 6, 5, 2))
    out, _ = cnn.forward(theta, x, layers=TINY, feature_stage=False)
    label = rng.normal(size=out.shape)
    valid = rng.random(out.shape[:3]) > 0.3

    def loss(t):
        o, _ = cnn.forward(t, x, layers=TINY, feature_stage=False)
        return cnn.loss_and_grad_out(o, label, valid)[0]

    out, cache = cnn.forward(theta, x, layers=TINY, feature_stage=False)
    L, dout = cnn.loss_and_grad_out(out, label, valid)
    g = cnn.backward(cache, dout, layers=TINY)
    e = 1e-6
    for i in rng.choice(theta.size, 25, replace=False):
        d = np.zeros_like(theta)
        d[i] = e
        num = (loss(theta + d) - loss(theta - d)) / (2 * e)
        assert num == pytest.approx(g[i], rel=1e-5, abs=1e-9)


def test_zero_weights_give_head_bias_and_param_count():
    assert cnn.n_params() == 119538
    theta = np.zeros(cnn.n_params())
    theta[-2:] = [1.5, -0.25]
    out, _ = cnn.forward(theta, np.random.default_rng(4).normal(size=(1, 16, 24, 2)))
    assert out.shape == (1, 2, 3, 2)
    assert np.all(out[..., 0] == 1.5) and np.all(out[..., 1] == -0.25)


def bf16_neighbours(v):
    """The two bfloat16 values around float32 v by truncating the low 16 bits."""
    u = np.float32(v).view(np.uint32)
    lo = np.uint32(u & 0xFFFF0000)
    hi = np.uint32(lo + 0x10000)
    return lo.view(np.float32), hi.view(np.float32), lo


def test_bf16_round_nearest_ties_to_even():
    rng = np.random.default_rng(5)
    vals = np.concatenate([rng.normal(size=200).astype(np.float32),
                           np.float32([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.0 - 2.0 ** -7,
                                       0.0, 3.0e-39])])
    got = cnn.bf16_round(vals)
    for v, g in zip(vals, got):
        lo, hi, lob = bf16_neighbours(v)
        dl, dh = abs(float(v) - float(lo)), abs(float(hi) - float(v))
        want = lo if dl < dh else hi if dh < dl else (lo if (int(lob) >> 16) % 2 == 0 else hi)
        assert g == float(want), v
    assert cnn.bf16_round(np.float32(1.0 + 2.0 ** -8)) == 1.0          # tie to even (down)
    assert cnn.bf16_round(np.float32(1.0 + 3 * 2.0 ** -8)) == 1.0 + 2.0 ** -6   # tie to even (up)


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 0.0])
    th, m, v = cnn.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, lr=0.01)
    # t = 1: m_hat = g, v_hat = g^2, update = lr g / (|g| + eps)
    want = -0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(th, want, rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_loss_is_mean_over_valid_cells():
    out = np.zeros((1, 1, 3, 2))
    label = np.array([[[[1.0, 0.0], [0.0, 2.0], [5.0, 5.0]]]])
    L, d = cnn.loss_and_grad_out(out, label, np.array([[[True, True, False]]]))
    assert L == pytest.approx((1.0 + 4.0) / 2)
    assert np.allclose(d[0, 0, 2], 0.0) and np.allclose(d[0, 0, 1], [0.0, -2.0])


def test_features_are_a_local_ssd_cost_volume():
    rng = np.random.default_rng(6)
    x = rng.uniform(-1, 1, (2, 5, 7, 2))
    f = cnn.features(x)
    assert f.shape == (2, 5, 7, 27)
    assert np.array_equal(f[..., 0], x[..., 0]) and np.array_equal(f[..., 1], x[..., 1])
    for _ in range(40):
        nb, y, xx = rng.integers(0, 2), rng.integers(0, 5), rng.integers(0, 7)
        v, u = rng.integers(-2, 3), rng.integers(-2, 3)
        bv = x[nb, y + v, xx + u, 1] if (0 <= y + v < 5 and 0 <= xx + u < 7) else 0.0
        k = 2 + (v + 2) * 5 + (u + 2)
        assert f[nb, y, xx, k] == -(x[nb, y, xx, 0] - bv) ** 2
    # a source equal to the reference shifted by (u, v) = (1, -1) zeroes that channel inside
    a = rng.uniform(-1, 1, (1, 9, 9))
    b = np.zeros_like(a)
    b[:, :8, 1:] = a[:, 1:, :8]  # b(p + (1, -1)) = a(p)
    f = cnn.features(np.stack([a, b], -1))
    assert np.all(f[0, 1:, :8, 2 + (-1 + 2) * 5 + (1 + 2)] == 0)
