"""Learned level-0 search (row a-L) pieces on the GPU against the oracle: the
quarter-resolution network input, tile labels, training crops, the search with a
predicted displacement and its fallback, and the fused path wired with a
predictor. Integer outputs (labels, matches, costs, fallback flags) are bit-exact;
the bfloat16 network input is within one bfloat16 step (1/64) of the float64 value."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tolerance import check_merged
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_01441_b300 import build, hdrreg
    build.build()
    return hdrreg


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def cfg(tile=16, radius=4, **kw):
    from paper_1504_01441_b300 import synth
    return synth.method_params(tile, radius, **kw)


@pytest.fixture(scope="module")
def level_pair(orc):
    from paper_1504_01441_b300 import synth
    st = synth.make_stack(synth.VGA_LUMA, synth.stack_seed(1))
    rn, sn = orc.normalize_ratio(st.ref.y, st.srcs[0].y, 4, 1)
    return rn, sn


def test_predictor_input_matches_oracle(hd, orc, level_pair):
    rn, sn = level_pair
    rq, sq = orc.pyramid(rn, 3)[2], orc.pyramid(sn, 3)[2]
    H = np.array([[1.01, 0.02, 0.03], [-0.015, 0.99, -0.02], [0.01, -0.008, 1.0]])
    x = hd.predictor_input(dev(rq), dev(sq), dev(H.reshape(9))).float().cpu().numpy()
    want = orc.predictor_input(rq, sq, H)
    assert x.shape == want.shape
    # values in [-1, 1] stored as bfloat16: half a unit in the last place is at most 2^-9
    # (for |v| in [0.5, 1)), plus the FP32 evaluation of the sample (~1e-6)
    err = np.abs(x - want).max()
    print(f"predictor input max error {err:.3e} (bound {2.0 ** -9 + 1e-5:.3e})")
    assert err <= 2.0 ** -9 + 1e-5


def test_tile_labels_bit_exact(hd, orc, level_pair):
    rn, sn = level_pair
    c = cfg()
    H = np.array([[1.0, 0.004, 0.01], [0.0, 1.0, -0.012], [0.0, 0.0, 1.0]])
    cxy, valid, _ = orc.pick_corners(rn, c)
    _, mxy, _ = orc.search(rn, sn, H, c, cxy, valid)
    lab = hd.tile_labels(dev(cxy), dev(mxy), dev(valid), 640, 480, dev(H.reshape(9)))
    assert np.array_equal(lab.cpu().numpy(), orc.tile_labels(cxy, mxy, valid, 640, 480, H))


def test_search_predicted_bit_exact(hd, orc, level_pair):
    rn, sn = level_pair
    c = cfg()
    p = hd.params_from_dict(c)
    H = np.array([[1.0, 0.004, 0.01], [0.0, 1.0, -0.012], [0.0, 0.0, 1.0]])
    cxy, valid, _ = orc.pick_corners(rn, c)
    _, mxy, cost = orc.search(rn, sn, H, c, cxy, valid)
    lab = orc.tile_labels(cxy, mxy, valid, 640, 480, H)
    rng = np.random.default_rng(3)
    pred = (lab + rng.normal(0, 0.8, lab.shape) + (rng.random(lab.shape) < 0.15) * 6).astype(np.float32)
    thr = int(np.median(cost[valid.astype(bool)]) * 1.5)
    ntx = 640 // 16
    grid = np.zeros((480 // 16 + 1, ntx + 3, 2), np.float32)  # wider than the tile grid
    grid[:30, :ntx] = pred.reshape(30, ntx, 2)
    for refine in (0, 1, 2):
        om, oc, ofb = orc.search_predicted(rn, sn, H, c, cxy, valid, pred, thr, refine)
        assert 0 < int(ofb.sum()) < int(valid.sum())  # both branches exercised
        for nt in (0, 64, 128):    # every block shape of the search
            p.search_threads = nt
            gc, gm, gcost, gv, gfb = hd.local_search_predicted(dev(rn), dev(sn), dev(H.reshape(9)),
                                                               p, dev(grid), thr, refine)
            assert np.array_equal(gc.cpu().numpy(), cxy) and np.array_equal(gv.cpu().numpy(), valid)
            assert np.array_equal(gm.cpu().numpy(), om), (refine, nt)
            assert np.array_equal(gcost.cpu().numpy().view(np.uint32), oc), (refine, nt)
            assert np.array_equal(gfb.cpu().numpy(), ofb), (refine, nt)


def test_crops_are_the_covered_tiles(hd):
    rng = np.random.default_rng(5)
    hq, wq, ntx, nty = 40, 56, 7, 5
    x = torch.tensor(rng.normal(size=(hq, wq, 2)), dtype=torch.bfloat16)
    lab = rng.normal(size=(nty * ntx, 2)).astype(np.float32)
    val = (rng.random(nty * ntx) > 0.3).astype(np.uint8)
    org = np.array([[0, 0, s, 0] for s in range(8)] + [[3, 1, 0, 0], [4, 2, 5, 0]], np.int32)
    bound = 1.5
    xc, lc, vc = hd.predictor_crops(x.cuda(), dev(lab), dev(val), ntx, nty, dev(org), crop_tiles=3,
                                    label_bound=bound)
    xc, lc, vc = xc.cpu(), lc.cpu().numpy(), vc.cpu().numpy()
    L = lab.reshape(nty, ntx, 2)
    V = val.reshape(nty, ntx).astype(bool) & (np.abs(L) < bound).all(-1)
    for b, (tx, ty, sym, _) in enumerate(org):
        xs = x[8 * ty:8 * ty + 24, 8 * tx:8 * tx + 24]
        ls, vs = L[ty:ty + 3, tx:tx + 3].copy(), V[ty:ty + 3, tx:tx + 3]
        # the symmetry as numpy operations on the crop: transpose, then mirror rows, then columns
        def apply(a, is_vec):
            if sym & 4:
                a = a.transpose(1, 0, 2) if a.ndim == 3 else a.T
            if sym & 2:
                a = a[::-1]
            if sym & 1:
                a = a[:, ::-1]
            return a
        # output (i, j) reads source crop_src(i, j): the inverse maps, applied to the source
        def inv(a):
            if sym & 1:
                a = a[:, ::-1]
            if sym & 2:
                a = a[::-1]
            if sym & 4:
                a = a.transpose(1, 0, 2) if a.ndim == 3 else a.T
            return a
        assert torch.equal(xc[b], torch.from_numpy(np.ascontiguousarray(inv(xs.float().numpy()))).bfloat16())
        lw = inv(ls)
        d = lw.copy()
        if sym & 4:
            d = d[..., ::-1]
        mx = (sym & 2) if (sym & 4) else (sym & 1)
        my = (sym & 1) if (sym & 4) else (sym & 2)
        if mx:
            d[..., 0] = -d[..., 0]
        if my:
            d[..., 1] = -d[..., 1]
        vw = inv(vs)
        assert np.array_equal(vc[b].astype(bool), vw), sym
        assert np.array_equal(lc[b][vw], d[vw]), sym
        assert np.all(lc[b][~vw] == 0)


def test_fused_learned_path_with_zero_fallback_cost_equals_plain(hd):
    from oracle import cnn
    from paper_1504_01441_b300 import synth
    st = synth.make_stack(synth.VGA_LUMA, synth.stack_seed(1))
    c = cfg(32, 6)  # the network predicts one displacement per 32 x 32 tile
    p = hd.params_from_dict(c)
    ref = (dev(st.ref.y), None, None)
    srcs = [(dev(st.srcs[0].y), None, None)]
    (y0, _, _), rm0 = hd.register_merge(ref, srcs, st.ratios, p)
    y0 = y0.clone()
    d0 = rm0.diagnostics()[0]
    theta = torch.tensor(cnn.init_params(9)).cuda()
    p.predictor = theta.data_ptr()
    p.fallback_cost = 0  # every prediction with a nonzero SSD falls back: the plain result
    (y1, _, _), rm1 = hd.register_merge(ref, srcs, st.ratios, p)
    d1 = rm1.diagnostics()[0]
    assert d0.fallbacks == -1 and d1.fallbacks == d1.valid
    assert list(d1.H0) == list(d0.H0)
    assert torch.equal(y1, y0)
    p.fallback_cost = 2 ** 32 - 1  # every prediction accepted
    (y2, _, _), rm2 = hd.register_merge(ref, srcs, st.ratios, p)
    d2 = rm2.diagnostics()[0]
    assert d2.fallbacks == 0 and np.isfinite(y2.cpu().numpy()).all()


def test_fused_learned_path_equals_its_step_calls(hd):
    # the fused call's learned level 0 = predictor input -> inference network -> search
    # with the prediction (threshold near the median cost, so both branches occur),
    # then the level fit: the same H0 bits and the same number of fallbacks
    from paper_1504_01441_b300 import learned, synth
    st = synth.make_stack(synth.VGA_LUMA, synth.stack_seed(1))
    p = hd.params_from_dict(cfg(32, 6))
    theta = torch.tensor(np.load(learned.THETA_FILE)).cuda()
    ref, src = dev(st.ref.y), dev(st.srcs[0].y)
    rn, sn, _ = hd.normalize_exposure(ref, src, hd.NORM_RATIO, st.ratios[0])
    h, w = rn.shape
    L = hd.num_levels(w, h, p)
    pr, ps = hd.build_pyramid(rn, L), hd.build_pyramid(sn, L)
    Hc = torch.tensor([1, 0, 0, 0, 1, 0, 0, 0, 1], dtype=torch.float64).cuda()
    counter = torch.zeros(1, dtype=torch.int32).cuda()
    for lv in range(L - 1, 0, -1):
        lh, lw = pr[lv].shape
        cxy, mxy, cost, valid = hd.local_search(pr[lv], ps[lv], Hc, p)
        _, Hc, _ = hd.weed_fit(cxy, mxy, valid, lw, lh, p, p.weed_seed + lv, Hc, counter=counter)
    _, _, c_plain, v_plain = hd.local_search(rn, sn, Hc, p)
    thr = int(c_plain[v_plain.bool()].double().median().item())
    x = hd.predictor_input(pr[2], ps[2], Hc)
    net = hd.Predictor(1, x.shape[0], x.shape[1], theta)
    pred = net.infer(x.unsqueeze(0))[0]
    cxy, mxy, cost, valid, fb = hd.local_search_predicted(rn, sn, Hc, p, pred, thr, refine=1)
    _, H0, _ = hd.weed_fit(cxy, mxy, valid, w, h, p, p.weed_seed, Hc, counter=counter)
    nfb = int(fb[valid.bool()].sum().item())
    assert 0 < nfb < int(valid.sum().item())
    p.predictor = theta.data_ptr()
    p.fallback_cost = thr
    p.predictor_refine = 1
    _, rm = hd.register_merge((ref, None, None), [(src, None, None)], st.ratios, p)
    d = rm.diagnostics()[0]
    assert np.array_equal(np.array(d.H0[:]).view(np.uint64), H0.cpu().numpy().view(np.uint64))
    assert d.fallbacks == nfb


def test_learned_merge_error_against_the_oracle_at_8px_fields(hd, orc):
    # The merge error of the learned path against the float64 oracle, on one 5 MP YUV420
    # pair with +-8 px local fields. The plain fused call is at parity with the oracle
    # (per element within 1e-4 * max(|oracle|, 1)). The learned call (default operating
    # point: r = 1, fallback above 1.5 x the median plain cost) changes level-0 matches,
    # so its merged image is held to the oracle's plain merge by an error budget instead:
    # the mean absolute luma difference and the share of pixels more than 2 DN apart.
    from paper_1504_01441_b300 import learned, synth
    st = synth.make_learned8_stack(0)
    c = cfg(32, 6)
    want = orc.register_merge(st.ref, st.srcs, st.ratios, c, want_intermediates=True)
    p = hd.params_from_dict(c)
    ref = (dev(st.ref.y), dev(st.ref.u), dev(st.ref.v))
    srcs = [(dev(st.srcs[0].y), dev(st.srcs[0].u), dev(st.srcs[0].v))]
    (y0, u0, v0), _ = hd.register_merge(ref, srcs, st.ratios, p)
    torch.cuda.synchronize()
    check_merged(orc, st, want, c, (y0, u0, v0), "plain fused merge")
    prep = learned.prepare(st, p)
    thr = int(1.5 * float(prep.cost[prep.valid.bool()].double().median().item()))
    theta = torch.tensor(np.load(learned.THETA_FILE)).cuda()
    p.predictor = theta.data_ptr()
    p.fallback_cost = thr
    p.predictor_refine = 1
    (y1, _, _), rm = hd.register_merge(ref, srcs, st.ratios, p)
    d = rm.diagnostics()[0]
    diff = np.abs(y1.cpu().numpy() - want["y"])
    mean_abs, share2 = float(diff.mean()), float((diff > 2.0).mean())
    print(f"learned vs oracle: mean |dY| {mean_abs:.4f} DN, > 2 DN on {100 * share2:.3f} % "
          f"of pixels, fallback {d.fallbacks}/{d.valid}")
    assert 0 < d.fallbacks < d.valid
    # measured on a B300: 0.113 DN and 0.38 % (fallback on 283 of 1853 tiles)
    assert mean_abs <= 0.25 and share2 <= 0.01


def test_learned_search_gains_over_plain_beyond_the_search_radius(hd):
    # What the trained network buys, against the generator's truth. On +-8 px fields (seeds
    # apart from training) some tiles' true match lies outside the level-0 window: the truth
    # at the corner minus the search centre (from the level-1 homography) exceeds R = 6 in x
    # or y, so the plain search cannot reach it. The learned search (prediction, +-1
    # refinement, plain search where the residual cost exceeds 1.5 x the median plain cost;
    # the network was trained on labels of a radius-12 plain search) must land closer to the
    # truth on those tiles, and over all tiles, than the plain search does.
    from paper_1504_01441_b300 import learned, synth
    p = hd.params_from_dict(cfg(32, 6))
    theta = torch.tensor(np.load(learned.THETA_FILE)).cuda()
    plain_far, learned_far, plain_all, learned_all, fell = [], [], [], [], 0
    for i in range(2):
        P = learned.prepare(synth.make_learned8_stack(i), p, keep_gt=True)
        net = hd.Predictor(1, P.x.shape[0], P.x.shape[1], theta)
        pred = net.infer(P.x.unsqueeze(0))[0]
        thr = int(1.5 * float(P.cost[P.valid.bool()].double().median().item()))
        c, m, _, v, fb = hd.local_search_predicted(P.ref_n, P.src_n, P.H1, p, pred, thr, refine=1)
        ok = (v.bool() & P.valid.bool()).cpu().numpy()
        corner = c.cpu().numpy()[ok].astype(np.int64)
        gt = P.gt.cpu().numpy()
        truth = np.stack([gt[0][corner[:, 1], corner[:, 0]], gt[1][corner[:, 1], corner[:, 0]]], 1)
        mp = P.match.cpu().numpy()[ok].astype(np.float64)
        ml = m.cpu().numpy()[ok].astype(np.float64)
        centre = mp - P.label.cpu().numpy()[ok]        # label = plain match - search centre
        far = (np.abs(truth - centre) > p.radius).any(1)
        ep, el = np.hypot(*(mp - truth).T), np.hypot(*(ml - truth).T)
        plain_far.append(ep[far])
        learned_far.append(el[far])
        plain_all.append(ep)
        learned_all.append(el)
        fell += int(fb.cpu().numpy()[ok].sum())
    pf, lf = np.concatenate(plain_far), np.concatenate(learned_far)
    pa, la = np.concatenate(plain_all), np.concatenate(learned_all)
    print(f"tiles beyond the radius: {pf.size} of {pa.size}; end-point error against the "
          f"generator's truth there: plain {pf.mean():.3f} px, learned {lf.mean():.3f} px; "
          f"over all tiles: plain {pa.mean():.3f} px, learned {la.mean():.3f} px; "
          f"fallback on {fell} tiles")
    # measured on a B300 with the committed network: 167 of 3,730 tiles beyond the radius,
    # plain 5.72 px, learned 5.07 px there; over all tiles plain 3.02 px, learned 1.69 px
    assert pf.size >= 20
    assert lf.mean() < 0.95 * pf.mean()   # beyond the window the plain search cannot reach
    assert la.mean() < 0.75 * pa.mean()   # and over every tile with a corner


def test_training_resumes_from_a_checkpoint_bit_for_bit(hd, tmp_path):
    # six Adam steps in one run against three steps, a checkpoint, and three more steps in
    # a fresh predictor resumed from it: the same parameters, bit for bit
    from paper_1504_01441_b300 import learned, synth
    p = hd.params_from_dict(cfg(32, 6))
    prep = [learned.prepare(synth.make_stack(synth.VGA_LUMA, synth.stack_seed(1)), p)]
    whole, _, _ = learned.train(prep, 6, batch=8, seed=3, log_every=1)
    ck = str(tmp_path / "ck.bin")
    learned.train(prep, 6, batch=8, seed=3, log_every=1, checkpoint=ck, stop_at=3)
    state = learned.read_checkpoint(ck)
    assert state["step"] == 3 and state["adam_t"] == 3
    assert not np.array_equal(state["theta"], whole.cpu().numpy())
    resumed, _, _ = learned.train(prep, 6, batch=8, seed=3, log_every=1, resume=ck)
    assert torch.equal(resumed, whole)
