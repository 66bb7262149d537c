"""Host logic of the mixed-size batch (row a-B): the tuner's selection rule and size
buckets, the mixed-workload stack recipe, and the lane plan's workspace sizes. No GPU."""
import ctypes as C
import math

import pytest

from paper_1504_01441_b300 import autotune, synth


def test_pick_takes_the_fastest_candidate_no_worse_than_the_default():
    res = {(32, 6): (100.0, 0.80), (16, 3): (40.0, 0.95), (24, 4): (60.0, 0.79),
           (48, 3): (50.0, 0.80), (48, 8): (200.0, 0.50)}
    # (16, 3) is faster but less accurate; (48, 3) ties the default's error and wins
    assert autotune.pick(res) == (48, 3)
    res[(24, 3)] = (50.0, 0.70)          # equal time: the smaller (T, R) wins
    assert autotune.pick(res) == (24, 3)
    assert autotune.pick({(32, 6): (1.0, 9.0)}) == (32, 6)
    with pytest.raises(ValueError):
        autotune.pick({(16, 3): (1.0, 0.1)})


def test_pick_block_takes_the_fastest_shape():
    assert autotune.pick_block({64: 30.0, 128: 25.0, 256: 27.0}) == 128
    assert autotune.pick_block({64: 25.0, 128: 25.0, 256: 27.0}) == 64   # tie: smaller B
    with pytest.raises(ValueError):
        autotune.pick_block({})


def test_every_block_shape_is_valid_for_the_library():
    from paper_1504_01441_b300 import build, hdrreg
    build.build()
    for nt in (0,) + autotune.BLOCKS:
        p = hdrreg.params_from_dict(synth.method_params(search_threads=nt))
        assert hdrreg.lib().hdrreg_validate_params(C.byref(p)) == 0, nt
    for nt in (32, 96, 512, -1):    # the C side sees the field where ctypes puts it
        p = hdrreg.params_from_dict(synth.method_params(search_threads=nt))
        assert hdrreg.lib().hdrreg_validate_params(C.byref(p)) == 1, nt


def test_bucket_bounds():
    assert autotune.bucket_of(1000, 1000) == 0            # 1.0 MP
    assert autotune.bucket_of(2000, 1000) == 0            # exactly 2 MP
    assert autotune.bucket_of(2000, 1001) == 1
    assert autotune.bucket_of(4000, 2000) == 2
    assert autotune.bucket_of(4000, 3000) == 3
    assert autotune.bucket_of(8000, 6000) == 3            # beyond the last bound: last bucket


def test_candidate_grid_is_valid_for_the_library():
    from paper_1504_01441_b300 import build, hdrreg
    build.build()
    assert len(autotune.candidates()) == 24 and autotune.DEFAULT in autotune.candidates()
    for t, r in autotune.candidates():
        p = hdrreg.params_from_dict(synth.method_params(tile=t, radius=r))
        assert hdrreg.lib().hdrreg_validate_params(C.byref(p)) == 0, (t, r)


def test_mixed_workload_recipe():
    specs = [synth.mixed_spec(i) for i in range(64)]
    areas = [s.width * s.height / 1e6 for s in specs]
    assert all(0.99 <= a <= 12.02 for a in areas)
    assert all(s.width % 2 == 0 and s.height % 2 == 0 and s.chroma for s in specs)
    aspects = [s.width / s.height for s in specs]
    assert all(min(abs(a - 4 / 3), abs(a - 16 / 9)) < 0.01 for a in aspects)
    n43 = sum(abs(a - 4 / 3) < 0.01 for a in aspects)
    assert 16 <= n43 <= 48
    assert {len(s.ratios) for s in specs} == {1, 2}
    assert {r for s in specs for r in s.ratios} <= {(2, 1), (4, 1), (8, 1)}
    assert all(s.noise_sigma == 1.5 and s.field_amp == 4.0 and s.movers == 3 for s in specs)
    # a stack's shape is a function of its own index only
    assert synth.mixed_spec(5) == specs[5]
    assert synth.mixed_spec(5, config_index=4) != specs[5]


def test_tuning_stacks_cover_every_bucket_apart_from_the_batch():
    jobs = autotune.tuning_jobs(per_bucket=2)
    assert len(jobs) == 2 * len(autotune.BUCKETS_MP)
    buckets = [autotune.bucket_of(synth.mixed_spec(i).width, synth.mixed_spec(i).height)
               for i, _, _ in jobs]
    assert sorted(buckets) == sorted(list(range(len(autotune.BUCKETS_MP))) * 2)
    assert all(i >= 10000 and gt for i, _, gt in jobs)


def test_params_for_uses_the_bucket_pick():
    from paper_1504_01441_b300 import build
    build.build()
    table = {"buckets_mp": [2.0, 4.0, 8.0, 12.0], "picks": [(16, 3), (24, 4), (32, 5), (48, 6)]}
    assert (autotune.params_for(1600, 1200, table).tile,
            autotune.params_for(1600, 1200, table).radius) == (16, 3)
    p = autotune.params_for(4000, 3000, table)
    assert (p.tile, p.radius, p.patch_half, p.search_threads) == (48, 6, 10, 0)
    table["picks"] = [(16, 3, 64), (24, 4, 128), (32, 5, 256), (48, 6, 128)]
    assert autotune.pick_of(table, 1600, 1200) == (16, 3, 64)
    p = autotune.params_for(4000, 3000, table)
    assert (p.tile, p.radius, p.search_threads) == (48, 6, 128)


def _stack_ex(hd, shapes):
    arr = (hd.StackEx * len(shapes))()
    keep = []
    for i, (w, h, n, t, r) in enumerate(shapes):
        p = hd.params_from_dict(synth.method_params(tile=t, radius=r))
        keep.append(p)
        arr[i].w, arr[i].h, arr[i].nsrc = w, h, n
        arr[i].p = C.pointer(p)
    return arr, keep


def test_multi_workspace_follows_the_lane_plan():
    from paper_1504_01441_b300 import build, hdrreg as hd
    build.build()
    lib = hd.lib()
    shapes = [(3840, 2160, 2, 48, 6), (1600, 1200, 1, 16, 3), (2592, 1944, 1, 32, 6),
              (1024, 768, 2, 24, 4), (4000, 3000, 1, 32, 5)]
    arr, keep = _stack_ex(hd, shapes)
    one = [hd.register_merge_workspace_size(w, h, n, keep[i])
           for i, (w, h, n, _, _) in enumerate(shapes)]
    al = [256 * math.ceil(x / 256) for x in one]
    assert lib.hdrreg_register_merge_multi_workspace_size(arr, 5, 1) == max(al)
    assert lib.hdrreg_register_merge_multi_workspace_size(arr, 5, 8) == sum(al)
    # two lanes, longest first (w*h*nsrc): 0 -> A, 4 -> B, 2 -> B, 3 -> A, 1 -> B
    two = lib.hdrreg_register_merge_multi_workspace_size(arr, 5, 2)
    assert two == max(al[0], al[3]) + max(al[4], al[2], al[1])
    assert lib.hdrreg_register_merge_multi_workspace_size(arr, 5, 0) == 0
    assert lib.hdrreg_register_merge_multi_workspace_size(arr, 5, hd.MAX_LANES + 1) == 0
    assert lib.hdrreg_register_merge_multi_workspace_size(None, 0, 2) == 0


def test_multi_argument_errors():
    from paper_1504_01441_b300 import build, hdrreg as hd
    build.build()
    lib = hd.lib()
    arr, keep = _stack_ex(hd, [(64, 64, 1, 16, 3)])
    assert lib.hdrreg_register_merge_multi(None, 0, 2, None, 0, None) == 0   # nothing to do
    assert lib.hdrreg_register_merge_multi(None, 2, 2, None, 0, None) == 1
    assert lib.hdrreg_register_merge_multi(arr, 1, 0, None, 0, None) == 1
    f = hd.Frame(None, None, None)
    arr[0].s.ref = C.pointer(f)
    assert lib.hdrreg_register_merge_multi(arr, 1, 2, None, 0, None) == 1   # NULL planes
    assert b"stack 0" in lib.hdrreg_last_error()


def test_learned_operating_point_is_the_cheapest_within_the_bound(monkeypatch):
    from paper_1504_01441_b300 import learned
    assert learned.search_cost(1, 0.0) == 9 and learned.search_cost(0, 1.0) == 1 + 169
    table = {(1, 1.5): (2.4, 0.09), (1, 1.0): (1.0, 0.58), (2, 1.0): (0.45, 0.60),
             (4, 1.0): (0.47, 0.51), (4, 1.5): (0.9, 0.08)}

    def fake(prep, theta, p, fallback_ratio, refine):
        e, fb = table.get((refine, fallback_ratio), (9.0, 0.0))
        return {"epe_px": e, "fallback_rate": fb}
    monkeypatch.setattr(learned, "evaluate", fake)

    class P:
        radius = 6
    pts, best = learned.calibrate([], None, P(), refines=(1, 2, 4), ratios=(1.5, 1.0))
    assert len(pts) == 6
    # (2, 1.0): 25 + 0.60 * 169 = 126.4 < (4, 1.0): 81 + 0.51 * 169 = 167.2
    assert (best["refine"], best["ratio"]) == (2, 1.0)
    _, none = learned.calibrate([], None, P(), refines=(1,), ratios=(1.5,), bound=0.5)
    assert none is None
