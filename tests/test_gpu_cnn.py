"""Learned displacement predictor (row a-L) on the GPU against the float64 oracle
(oracle/cnn.py with the same bfloat16 rounding points): forward output and every stored
activation, loss, the gradient of every layer's weights and biases, the Adam step, and a
loss that falls under training.

Forward. The oracle rounds the same stored values to bfloat16, so the two differ only
where FP32 and FP64 accumulation land on opposite sides of a bfloat16 rounding boundary
(one step = 2^-8 relative), compounding over nine layers: max-norm relative 2e-2 on the
output. Such a difference can also flip a ReLU whose pre-activation is within rounding of
zero (observed: one or two per layer in a thousand), which changes that element's gradient
entirely. Backward is checked twice. (1) Against the oracle's whole chain on its own
forward: the oracle's loss gradient and backward on the oracle's activations, so nothing
of the GPU's forward enters the expected values. Two bfloat16 chains whose pre-activations
differ by FP32 accumulation error round some values to neighbouring bfloat16 numbers, and
that cascades: the oracle's own chain, given noise of relative size 2^-20 on its
pre-activations, moves its weight gradients by up to 3-12 % (relative L2 per layer, the
largest over eight noise draws). The bound is twice that movement, per layer, and at least
1e-2.
(2) The backward kernels alone: the oracle's backward on the activations the GPU stored
(read back through hdrreg_cnn_activation), so the ReLU masks agree and the remaining
difference is accumulation order plus bfloat16 rounding of the output gradients at nine
layers: relative L2 1e-2 and max-norm relative 3e-2. The Adam step is FP32 arithmetic on
identical inputs: 1e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_01441_b300 import build, hdrreg
    build.build()
    return hdrreg


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def named_slices():
    """(layer, 'weights' | 'biases', slice of the flat parameter vector), in order"""
    return [(i, part, sl) for i, (sw, sb) in enumerate(layer_slices())
            for part, sl in (("weights", sw), ("biases", sb))]


def all_slices():
    return [sl for _, _, sl in named_slices()]


def n_slices():
    return len(named_slices())


def layer_slices():
    from oracle import cnn
    out, o = [], 0
    for ci, co, k, s, r in cnn.LAYERS:
        nw = co * k * k * ci
        out.append((slice(o, o + nw), slice(o + nw, o + nw + co)))
        o += nw + co
    return out


@pytest.mark.parametrize("n,h,w", [(2, 24, 40), (1, 61, 33), (1, 64, 64), (2, 40, 32)])
def test_forward_and_gradients_match_oracle(hd, n, h, w):
    from oracle import cnn
    rng = np.random.default_rng(n * 100 + h + w)
    theta = cnn.init_params(7)
    theta[cnn.n_params() - 2:] = [0.3, -0.2]  # nonzero head bias
    xb = torch.tensor(rng.uniform(-1, 1, (n, h, w, 2)), dtype=torch.bfloat16)
    P = hd.Predictor(n, h, w, theta)
    out = P.forward(xb.cuda()).cpu().numpy()
    o_or, (params, acts) = cnn.forward(theta, xb.double().numpy(), bf16=True)
    assert out.shape == o_or.shape
    assert rel(out, o_or) <= 2e-2
    # every stored activation within bfloat16 rounding of the oracle's, bar rare flips
    gacts = [P.activation(-1).cpu().numpy().reshape(acts[0].shape)]
    assert np.array_equal(gacts[0], acts[0])  # the feature stage is exact
    for i in range(len(cnn.LAYERS) - 1):
        a = P.activation(i).cpu().numpy().reshape(acts[i + 1].shape)
        assert rel_l2(a, acts[i + 1]) <= 1e-2, f"activation {i}"
        gacts.append(a)
    label = rng.normal(size=out.shape).astype(np.float32)
    valid = (rng.random(out.shape[:3]) > 0.25).astype(np.uint8)
    loss, grad = P.backward(xb.cuda(), torch.tensor(label).cuda(), torch.tensor(valid).cuda())
    torch.cuda.synchronize()
    assert int(P.status.item()) == 0
    L, dout = cnn.loss_and_grad_out(out.astype(np.float64), label, valid.astype(bool))
    assert float(loss.item()) == pytest.approx(L, rel=1e-5)
    g = grad.cpu().numpy()
    # (1) independent of the GPU forward: the oracle's backward on the oracle's own
    # activations and output (the whole chain float64 with the same bfloat16 rounding
    # points), so a forward error below the forward tolerance still shows here
    L_or, dout_or = cnn.loss_and_grad_out(o_or, label, valid.astype(bool))
    assert float(loss.item()) == pytest.approx(L_or, rel=2e-2)
    g_ind = cnn.backward((params, acts), dout_or, bf16=True)
    # (2) the backward kernels alone: the oracle's backward on the activations the GPU
    # stored, so the ReLU masks agree element by element
    g_or = cnn.backward((params, gacts + [out.astype(np.float64)]), dout, bf16=True)
    # How far the oracle's own bfloat16 chain moves when its pre-activations carry noise of
    # the size of FP32 accumulation (relative 2^-20): values then round to neighbouring
    # bfloat16 numbers, and the difference cascades through the layers. Any FP32-accumulating
    # implementation differs from the float64 chain by that much, so the independent check
    # allows twice the largest movement over eight noise draws (and at least 1e-2): whether
    # a value crosses a bfloat16 boundary is all or nothing, so the movement varies from
    # draw to draw (layer 4 of the 2 x 40 x 32 case: 1e-2 to 7.5e-2 over eight draws).
    div = np.zeros(n_slices())
    for t in range(8):
        nr = np.random.default_rng(1000 + t)
        o2, c2 = cnn.forward(theta, xb.double().numpy(), bf16=True,
                             perturb=lambda z: z * (1.0 + 2.0 ** -20 * nr.standard_normal(z.shape)))
        g2 = cnn.backward(c2, cnn.loss_and_grad_out(o2, label, valid.astype(bool))[1], bf16=True)
        div = np.maximum(div, [rel_l2(g2[sl], g_ind[sl]) for sl in all_slices()])
    for j, (i, part, sl) in enumerate(named_slices()):
        e = rel_l2(g[sl], g_ind[sl])
        print(f"layer {i} {part}: relative L2 {e:.2e} against the oracle's own chain (that "
              f"chain moves {div[j]:.2e} under accumulation noise), {rel_l2(g[sl], g_or[sl]):.2e} "
              f"on the GPU's activations")
        assert e <= max(1e-2, 2.0 * div[j]), f"layer {i} {part} (independent chain)"
    for i, (sw, sb) in enumerate(layer_slices()):
        for part, sl in (("weights", sw), ("biases", sb)):
            assert rel_l2(g[sl], g_or[sl]) <= 1e-2, f"layer {i} {part}"
            assert rel(g[sl], g_or[sl]) <= 3e-2, f"layer {i} {part}"


def test_adam_matches_oracle(hd):
    from oracle import cnn
    rng = np.random.default_rng(4)
    P = hd.Predictor(1, 16, 16, cnn.init_params(1))
    th = P.theta.cpu().numpy().astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for t in (1, 2, 3):
        g = rng.normal(size=th.size).astype(np.float32)
        P.grad.copy_(torch.tensor(g))
        P.adam(lr=1e-3)
        th, m, v = cnn.adam_step(th, m, v, g.astype(np.float64), t, lr=1e-3)
        torch.cuda.synchronize()
        d = P.theta.cpu().numpy() - th
        assert np.abs(d).max() <= 1e-5 * np.abs(th).max() + 1e-7


def test_training_reduces_the_loss(hd):
    from oracle import cnn
    rng = np.random.default_rng(11)
    n, h, w = 8, 32, 32
    x = rng.uniform(-1, 1, (n, h, w, 2))
    xb = torch.tensor(x, dtype=torch.bfloat16).cuda()
    P = hd.Predictor(n, h, w, cnn.init_params(2))
    # a learnable target: the mean of channel 1 minus channel 0 over each output cell's 8x8 block
    blk = (x[..., 1] - x[..., 0]).reshape(n, 4, 8, 4, 8).mean(axis=(2, 4))
    label = np.stack([blk, -blk], -1).astype(np.float32) * 4
    lab, val = torch.tensor(label).cuda(), torch.ones((n, 4, 4), dtype=torch.uint8).cuda()
    losses = []
    for _ in range(60):
        P.forward(xb)
        loss, _ = P.backward(xb, lab, val)
        losses.append(float(loss.item()))
        P.adam(lr=3e-3)
    assert int(P.status.item()) == 0
    assert losses[-1] < 0.3 * losses[0], losses[::10]


@pytest.mark.parametrize("n,h,w", [(2, 24, 40), (1, 61, 33), (1, 130, 70), (3, 47, 29)])
def test_inference_form_matches_oracle_and_training_forward(hd, n, h, w):
    # implicit-GEMM convolutions (inputs gathered per tap, several M tiles, a ragged
    # last tile): same network, FP32 sums in another order than the im2col GEMMs
    from oracle import cnn
    rng = np.random.default_rng(n * 1000 + h + w)
    theta = cnn.init_params(11)
    theta[cnn.n_params() - 2:] = [-0.1, 0.25]
    xb = torch.tensor(rng.uniform(-1, 1, (n, h, w, 2)), dtype=torch.bfloat16)
    P = hd.Predictor(n, h, w, theta)
    got = P.infer(xb.cuda())
    fwd = P.forward(xb.cuda())
    torch.cuda.synchronize()
    assert int(P.status.item()) == 0
    got, fwd = got.cpu().numpy(), fwd.cpu().numpy()
    o_or, _ = cnn.forward(theta, xb.double().numpy(), bf16=True)
    assert got.shape == o_or.shape
    assert rel(got, o_or) <= 2e-2
    assert rel(got, fwd) <= 2e-2
    assert rel_l2(got, fwd) <= 5e-3


def test_inference_form_at_the_predictor_size(hd):
    # the quarter-resolution input of a 2592 x 1944 frame (648 x 486, 2461 M tiles at the
    # first layer) with the trained parameters: equals the training forward up to order
    from paper_1504_01441_b300 import learned
    theta = np.load(learned.THETA_FILE)
    rng = np.random.default_rng(5)
    xb = torch.tensor(rng.uniform(-1, 1, (1, 486, 648, 2)), dtype=torch.bfloat16).cuda()
    P = hd.Predictor(1, 486, 648, theta)
    got = P.infer(xb).cpu().numpy()
    fwd = P.forward(xb).cpu().numpy()
    assert int(P.status.item()) == 0
    assert rel(got, fwd) <= 2e-2 and rel_l2(got, fwd) <= 5e-3
