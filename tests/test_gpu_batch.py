"""GPU: the mixed-size batch (row a-B) and its tuner.

A batch of stacks of different sizes, frame counts and (T, R) must give, bit for bit,
what one fused call per stack gives (those are checked against the oracle in the
parity tests), also when replayed from a CUDA graph, and a member of the batch must
match the oracle run with the same parameters. The tuner's error measure must agree
with the same error computed from the oracle's homography and flow.
"""
import os

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
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


def dev_stack(s):
    return ((dev(s.ref.y), dev(s.ref.u), dev(s.ref.v)),
            [(dev(f.y), dev(f.u), dev(f.v)) for f in s.srcs], list(s.ratios))


def check_against_oracle(orc, stack, c, outs, diags):
    out = orc.register_merge(stack.ref, stack.srcs, stack.ratios, c, want_intermediates=True)
    for k, d in enumerate(diags):
        assert np.array_equal(np.array(d.H0[:]).view(np.uint64),
                              out["H0"][k].reshape(9).view(np.uint64)), f"H0 of source {k}"
    torch.cuda.synchronize()
    check_merged(orc, stack, out, c, outs)


def run_multi_case(hd, stacks, cfgs, lanes):
    """multi call vs one fused call per stack, eagerly and from a CUDA graph."""
    params = [hd.params_from_dict(c) for c in cfgs]
    dstacks = [dev_stack(s) for s in stacks]
    single = []
    for (ref, srcs, ratios), p in zip(dstacks, params):
        (y, u, v), rm = hd.register_merge(ref, srcs, ratios, p)
        single.append(([t.clone() if t is not None else None for t in (y, u, v)],
                       [d.H0[:] for d in rm.diagnostics()]))
    shapes = [(s.width, s.height, len(s.srcs), p, s.ref.u is not None)
              for s, p in zip(stacks, params)]
    mm = hd.RegisterMergeMulti(shapes, lanes=lanes)
    outs = mm(dstacks)
    torch.cuda.synchronize()
    for i, (o, (want, h0)) in enumerate(zip(outs, single)):
        for a, b in zip(o, want):
            assert (a is None and b is None) or torch.equal(a, b), f"stack {i}"
        assert [d.H0[:] for d in mm.diagnostics(i)] == h0, f"H0 of stack {i}"
    for o in outs:
        for t in o:
            if t is not None:
                t.zero_()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        mm(dstacks, stream=s)
    with torch.cuda.stream(s):
        g.replay()
    torch.cuda.synchronize()
    for i, (o, (want, _)) in enumerate(zip(outs, single)):
        for a, b in zip(o, want):
            assert (a is None and b is None) or torch.equal(a, b), f"stack {i} (graph replay)"
    return mm, outs


def test_multi_shapes_equal_single_calls_and_captures(hd, orc):
    from paper_1504_01441_b300 import synth
    specs = [synth.StackSpec(320, 240, ratios=((4, 1),), movers=1, chroma=True),
             synth.StackSpec(352, 288, ratios=((2, 1), (8, 1)), movers=1, chroma=True),
             synth.StackSpec(482, 322, ratios=((4, 1),), movers=1, chroma=True),
             synth.StackSpec(256, 192, ratios=((1, 4), (4, 1)), movers=1, chroma=False),
             synth.StackSpec(640, 360, ratios=((8, 1),), movers=2, chroma=True)]
    stacks = [synth.make_stack(sp, 90 + i) for i, sp in enumerate(specs)]
    tr = [(16, 4), (24, 3), (16, 5), (16, 3), (32, 6)]
    cfgs = [synth.method_params(t, r) for t, r in tr]
    mm, outs = run_multi_case(hd, stacks, cfgs, lanes=3)
    check_against_oracle(orc, stacks[1], cfgs[1], outs[1], mm.diagnostics(1))
    check_against_oracle(orc, stacks[3], cfgs[3], outs[3], mm.diagnostics(3))


def test_staged_merges_equal_the_lane_form_and_capture(hd):
    # the same mixed stacks with every merge as one stage after all registrations
    # (persistent launches over the tiles of every stack): the same bits as the lane form,
    # eagerly and replayed from a CUDA graph
    from paper_1504_01441_b300 import synth
    specs = [synth.StackSpec(320, 240, ratios=((4, 1),), movers=1, chroma=True),
             synth.StackSpec(352, 288, ratios=((2, 1), (8, 1)), movers=1, chroma=True),
             synth.StackSpec(256, 192, ratios=((1, 4), (4, 1)), movers=1, chroma=False),
             synth.StackSpec(482, 322, ratios=((4, 1),), movers=1, chroma=True)]
    stacks = [synth.make_stack(sp, 190 + i) for i, sp in enumerate(specs)]
    params = [hd.params_from_dict(synth.method_params(t, r))
              for t, r in [(16, 4), (24, 3), (16, 3), (16, 5)]]
    params[1].norm_mode = hd.NORM_HISTEQ
    dstacks = [dev_stack(s) for s in stacks]
    shapes = [(s.width, s.height, len(s.srcs), p, s.ref.u is not None)
              for s, p in zip(stacks, params)]
    lanes_form = hd.RegisterMergeMulti(shapes, lanes=3)
    want = [[t.clone() if t is not None else None for t in o] for o in lanes_form(dstacks)]
    staged = hd.RegisterMergeMulti(shapes, lanes=3, staged=True)
    outs = staged(dstacks)
    torch.cuda.synchronize()
    for i, (o, w_) in enumerate(zip(outs, want)):
        for a, b in zip(o, w_):
            assert (a is None and b is None) or torch.equal(a, b), f"stack {i}"
        assert ([d.H0[:] for d in staged.diagnostics(i)] ==
                [d.H0[:] for d in lanes_form.diagnostics(i)])
    for o in outs:
        for t in o:
            if t is not None:
                t.zero_()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        staged(dstacks, stream=s)
    with torch.cuda.stream(s):
        g.replay()
    torch.cuda.synchronize()
    for i, (o, w_) in enumerate(zip(outs, want)):
        for a, b in zip(o, w_):
            assert (a is None and b is None) or torch.equal(a, b), f"stack {i} (graph replay)"


def test_multi_one_lane_and_more_lanes_than_stacks(hd):
    from paper_1504_01441_b300 import synth
    specs = [synth.StackSpec(320, 240, ratios=((4, 1),), movers=1, chroma=True),
             synth.StackSpec(288, 224, ratios=((2, 1), (2, 1)), movers=1, chroma=True)]
    stacks = [synth.make_stack(sp, 95 + i) for i, sp in enumerate(specs)]
    cfgs = [synth.method_params(16, 4), synth.method_params(24, 5)]
    run_multi_case(hd, stacks, cfgs, lanes=1)
    run_multi_case(hd, stacks, cfgs, lanes=hd.MAX_LANES)


def _picks():
    from paper_1504_01441_b300 import autotune
    if os.path.exists(autotune.TABLE_FILE):
        return autotune.load_table()
    return {"buckets_mp": list(autotune.BUCKETS_MP), "picks": [autotune.DEFAULT] * 4}


def test_mixed_workload_members_at_full_size(hd, orc):
    # three stacks of the 64-stack mixed workload (the smallest, a 1-source one, and an
    # 8 MP one) with their bucket's (T, R): batch == single calls; the smallest against
    # the oracle run with the same picks
    from paper_1504_01441_b300 import autotune, synth
    table = _picks()
    idx = [53, 49, 0]
    stacks = synth.make_stacks_parallel([(i, 3, False) for i in idx], processes=1)
    cfgs = []
    for s in stacks:
        t, r, b = autotune.pick_of(table, s.width, s.height)
        cfgs.append(synth.method_params(t, r, search_threads=b))
    mm, outs = run_multi_case(hd, stacks, cfgs, lanes=2)
    check_against_oracle(orc, stacks[0], cfgs[0], outs[0], mm.diagnostics(0))


def test_registration_error_matches_the_oracle(hd, orc, vga_stack):
    # the tuner's error of H^0 + F against the generator truth, from the GPU step calls,
    # equals the same error computed from the oracle's homography and flow
    from paper_1504_01441_b300 import autotune, synth
    s = vga_stack
    c = synth.method_params(16, 4)
    gpu = autotune.registration_epe(s, hd.params_from_dict(c))
    out = orc.register_merge(s.ref, s.srcs, s.ratios, c, want_intermediates=True)
    h, w = s.ref.y.shape
    H = out["H0"][0]
    ys, xs = np.mgrid[0:h, 0:w].astype(float)
    xn, yn = (2 * xs - (w - 1)) / w, (2 * ys - (h - 1)) / w
    V = np.einsum("ij,jhw->ihw", H, np.stack([xn, yn, np.ones_like(xn)]))
    hx, hy = (V[0] / V[2] * w + (w - 1)) / 2, (V[1] / V[2] * w + (h - 1)) / 2
    gx, gy = s.gt[0]
    inside = (gx >= 0) & (gx <= w - 1) & (gy >= 0) & (gy <= h - 1)
    want = np.hypot(hx + out["flow_u"][0] - gx, hy + out["flow_v"][0] - gy)[inside].mean()
    print(f"EPE gpu {gpu:.6f} oracle {want:.6f}")
    assert abs(gpu - want) <= 1e-4 * max(want, 1.0)
    assert want < 1.0


def test_tuner_on_a_small_candidate_set(hd, vga_stack):
    from paper_1504_01441_b300 import autotune
    cands = [(16, 3), (16, 4), (24, 4)]
    table = autotune.tune([vga_stack], cands=cands, reps=2)
    meas = table["measurements"][0]
    assert set(meas) == {"16,3", "16,4", "24,4", "32,6"}
    assert all(v[0] > 0 and 0 <= v[1] < 5 for v in meas.values())
    t, r, b = table["picks"][0]
    chosen = meas[f"{t},{r}"]
    assert chosen[1] <= meas["32,6"][1]
    assert all(v[0] >= chosen[0] for v in meas.values() if v[1] <= meas["32,6"][1])
    bm = table["block_measurements"][0]
    assert set(bm) == {"64", "128", "256"} and bm[str(b)] == min(bm.values())
    assert table["picks"][1:] == [list(autotune.DEFAULT) + [128]] * 3   # buckets without stacks


@pytest.mark.parametrize("lanes", [1, 3])
def test_host_staged_batch_equals_device_batch(hd, lanes):
    # stacks in page-locked host memory, staged through the lanes by the library: the
    # same bits as the batched call on device-resident stacks
    from paper_1504_01441_b300 import synth
    spec = synth.StackSpec(320, 240, ratios=((4, 1), (2, 1)), noise_sigma=1.0, field_amp=2.0,
                           movers=1, chroma=True)
    stacks = [synth.make_stack(spec, 120 + i) for i in range(5)]
    p = hd.params_from_dict(synth.method_params(16, 4))
    dstacks = [dev_stack(s) for s in stacks]
    ref_batch = hd.RegisterMergeBatch(320, 240, 2, p, True, slots=5, lanes=lanes)
    want = [[t.clone() for t in o] for o in ref_batch(dstacks)]

    def pin(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hstacks = [((pin(s.ref.y), pin(s.ref.u), pin(s.ref.v)),
                [(pin(f.y), pin(f.u), pin(f.v)) for f in s.srcs], list(s.ratios)) for s in stacks]
    outs = [(torch.full((240, 320), -1.0).pin_memory(), torch.full((120, 160), -1.0).pin_memory(),
             torch.full((120, 160), -1.0).pin_memory()) for _ in stacks]
    runner = hd.RegisterMergeHost(320, 240, 2, p, lanes=lanes)
    s = torch.cuda.Stream()
    runner(hstacks, outs, stream=s)
    s.synchronize()
    for i, (o, w) in enumerate(zip(outs, want)):
        for a, b in zip(o, w):
            assert torch.equal(a, b.cpu()), f"stack {i}"
