"""The learned and batched path at scale: three-frame 4000 x 3000 YUV420 stacks with
exposures 1/4, 1 and 4 of the reference's (the r = 1 frame is the reference, the other
two are registered to it), +-8 px local fields and 5 movers, through the batched fused
call with the learned level-0 search.

* the batched call (eager and replayed from a CUDA graph) gives the planes, H^0 bits and
  fallback counts of one fused call per stack;
* for both sources, the fused call's learned level 0 equals its step calls (predictor
  input, inference network, search with the prediction and fallback, then the level's
  weeding and fit, Eq. 3-4) bit for bit in H^0, with both branches of the fallback taken.
The step calls themselves are held to the oracle at smaller sizes (the learned-search
tests); here the sizes are the workload's own.
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


@pytest.fixture(scope="module")
def stacks():
    from paper_1504_01441_b300 import synth
    return synth.make_scale12_stacks(2)


def dev(a):
    return None if a is None else torch.as_tensor(np.ascontiguousarray(a)).cuda()


def frames(st):
    return ((dev(st.ref.y), dev(st.ref.u), dev(st.ref.v)),
            [(dev(f.y), dev(f.u), dev(f.v)) for f in st.srcs], list(st.ratios))


def plain_params(hd):
    from paper_1504_01441_b300 import synth
    return hd.params_from_dict(synth.method_params(32, 6))


def level0_inputs(hd, st, k, p):
    """Normalized level 0 of source k, the pyramids and H^1 from the step calls."""
    ref, src = dev(st.ref.y), dev(st.srcs[k].y)
    rn, sn, _ = hd.normalize_exposure(ref, src, hd.NORM_RATIO, st.ratios[k])
    h, w = rn.shape
    L = hd.num_levels(w, h, p)
    pr, ps = hd.build_pyramid(rn, L), hd.build_pyramid(sn, L)
    Hc = torch.tensor([1, 0, 0, 0, 1, 0, 0, 0, 1], dtype=torch.float64).cuda()
    counter = torch.zeros(1, dtype=torch.int32).cuda()
    for lv in range(L - 1, 0, -1):
        lh, lw = pr[lv].shape
        cxy, mxy, _, valid = hd.local_search(pr[lv], ps[lv], Hc, p)
        Hc = weed_and_fit(hd, cxy, mxy, valid, lw, lh, p, lv, Hc, counter)
    return rn, sn, pr, ps, Hc, counter


def weed_and_fit(hd, cxy, mxy, valid, w, h, p, lv, Hc, counter):
    """The level's weeding and fit as the fused call runs them: in one launch when the
    level fits it, else the workspace weeding followed by the fit."""
    if hd.lib().hdrreg_weed_fit_supported(valid.numel()):
        _, H, _ = hd.weed_fit(cxy, mxy, valid, w, h, p, p.weed_seed + lv, Hc, counter=counter)
        return H
    mask = hd.weed(cxy, mxy, valid, w, h, p, p.weed_seed + lv)
    H, _ = hd.fit_homography(cxy, mxy, mask, w, h, Hc)
    return H


@pytest.fixture(scope="module")
def learned_params(hd, stacks):
    """The trained predictor with the fallback threshold at the median plain level-0 cost
    of the first stack's first source, so that both branches occur."""
    from paper_1504_01441_b300 import learned
    p = plain_params(hd)
    theta = torch.tensor(np.load(learned.THETA_FILE)).cuda()
    rn, sn, _, _, Hc, _ = level0_inputs(hd, stacks[0], 0, p)
    _, _, cost, valid = hd.local_search(rn, sn, Hc, p)
    thr = int(cost[valid.bool()].double().median().item())
    p.predictor = theta.data_ptr()
    p.fallback_cost = thr
    p.predictor_refine = 1
    return p, theta


def test_stack_shape_and_exposures(stacks):
    st = stacks[0]
    assert (st.width, st.height) == (4000, 3000) and len(st.srcs) == 2
    assert [tuple(r) for r in st.ratios] == [(1, 4), (4, 1)]
    m0, m1, m2 = st.ref.y.mean(), st.srcs[0].y.mean(), st.srcs[1].y.mean()
    assert m1 < m0 < m2


def test_learned_batch_equals_single_calls(hd, stacks, learned_params):
    p, _ = learned_params
    fr = [frames(st) for st in stacks]
    singles = []
    for f in fr:
        planes, rm = hd.register_merge(f[0], f[1], f[2], p)
        singles.append(([x.clone() for x in planes], rm.diagnostics()))
    w, h = stacks[0].width, stacks[0].height
    bm = hd.RegisterMergeBatch(w, h, 2, p, True, slots=2, lanes=2)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        outs = bm(fr, stream=s)
    s.synchronize()

    def check(outs, what):
        for i, (planes, diags) in enumerate(singles):
            for a, b in zip(outs[i], planes):
                assert torch.equal(a, b), f"stack {i} {what}"
            got = bm.diagnostics(i)
            for k in range(2):
                assert np.array_equal(np.array(got[k].H0[:]).view(np.uint64),
                                      np.array(diags[k].H0[:]).view(np.uint64)), (i, k, what)
                assert got[k].fallbacks == diags[k].fallbacks >= 0, (i, k, what)
    check(outs, "eager")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        outs = bm(fr, stream=s)
    for o in outs:
        for x in o:
            x.zero_()
    with torch.cuda.stream(s):
        g.replay()
    s.synchronize()
    check(outs, "graph replay")


@pytest.mark.parametrize("k", [0, 1])
def test_fused_learned_level0_equals_step_calls_at_12mp(hd, stacks, learned_params, k):
    p, theta = learned_params
    st = stacks[1]
    rn, sn, pr, ps, Hc, counter = level0_inputs(hd, st, k, p)
    h, w = rn.shape
    x = hd.predictor_input(pr[2], ps[2], Hc)
    net = hd.Predictor(1, x.shape[0], x.shape[1], theta)
    pred = net.infer(x.unsqueeze(0))[0]
    cxy, mxy, cost, valid, fb = hd.local_search_predicted(rn, sn, Hc, p, pred, p.fallback_cost,
                                                          refine=p.predictor_refine)
    H0 = weed_and_fit(hd, cxy, mxy, valid, w, h, p, 0, Hc, counter)
    nfb = int(fb[valid.bool()].sum().item())
    assert 0 < nfb < int(valid.sum().item())
    f = frames(st)
    _, rm = hd.register_merge(f[0], f[1], f[2], p)
    d = rm.diagnostics()[k]
    assert np.array_equal(np.array(d.H0[:]).view(np.uint64), H0.cpu().numpy().view(np.uint64))
    assert d.fallbacks == nfb
