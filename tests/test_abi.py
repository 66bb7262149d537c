"""The C-ABI library loads and exports everything include/hdrreg.h declares; host
logic (defaults, validation, sizes) works without a GPU. No call here reaches a
kernel launch: every invalid argument is rejected on the host first.
"""
import ctypes as C
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hd():
    from paper_1504_01441_b300 import build, hdrreg
    build.build()
    return hdrreg


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hdrreg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hdrreg_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(hd):
    lib = hd.lib()
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(hd.EXPORTS)


def test_version_and_defaults_follow_the_paper(hd):
    assert "sm_103a" in hd.version()
    p = hd.params()
    c = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    assert p.levels_max == c["levels_max"] and p.min_level_size == c["min_level_size_px"]
    assert 2 * p.patch_half + 1 == c["patch_side"] and p.radius == c["max_search_radius"]
    assert p.sigma_s == c["sigma_s"]
    assert hd.lib().hdrreg_validate_params(C.byref(p)) == 0


def test_param_fields_match_the_workload_parameter_sets(hd):
    from paper_1504_01441_b300 import synth
    d = synth.method_params(32, 6)
    p = hd.params_from_dict(d)
    assert p.as_dict() == {k: v for k, v in d.items()}


@pytest.mark.parametrize("field,value", [("tile", 7), ("tile", 130), ("radius", 0), ("radius", 16),
                                         ("patch_half", 0), ("levels_max", 9), ("grid_half", 9),
                                         ("quad", 0), ("corner_thresh", -1), ("dt_iters", 0),
                                         ("ssim_radius", 4), ("norm_mode", 2), ("sigma_r", 0.0),
                                         ("weed_delta_div", 0), ("weed_iters", -1)])
def test_invalid_params_rejected(hd, field, value):
    p = hd.params(**{field: value})
    assert hd.lib().hdrreg_validate_params(C.byref(p)) == 1
    assert hd.lib().hdrreg_last_error()


def test_grid_must_stay_inside_the_tile(hd):
    # T=16 -> step 1, K=8 reaches the tile border: rejected; K=7 fine
    assert hd.lib().hdrreg_validate_params(C.byref(hd.params(tile=16, grid_half=8))) == 1
    assert hd.lib().hdrreg_validate_params(C.byref(hd.params(tile=16, grid_half=7))) == 0


@pytest.mark.parametrize("w,h,L", [(2592, 1944, 5), (640, 480, 3), (199, 400, 1), (4000, 3000, 5)])
def test_levels_match_oracle_rule(hd, w, h, L):
    assert hd.num_levels(w, h, hd.params()) == L


def test_sizes(hd):
    lib = hd.lib()
    assert hd.num_tiles(2592, 1944, 32) == 81 * 60
    assert lib.hdrreg_pyramid_bytes(2592, 1944, 5) == sum((2592 >> l) * (1944 >> l) for l in range(1, 5))
    assert lib.hdrreg_flow_workspace_size(2592, 1944) >= 3 * 2592 * 1944 * 4
    assert lib.hdrreg_flow_workspace_size(0, 10) == 0
    p = hd.params(tile=32, radius=6)
    ws = hd.register_merge_workspace_size(2592, 1944, 1, p)
    assert ws > 5 * 2592 * 1944 * 4
    assert hd.register_merge_workspace_size(2592, 1944, 5, p) == 0      # too many sources
    assert lib.hdrreg_normalize_workspace_size(0) == 0 and lib.hdrreg_normalize_workspace_size(1) > 0


def test_diag_layout_matches_the_header(hd):
    # hdrreg_diag: 9 binary64 then 8 int32 (levels .. fallbacks, flow_status, reserved)
    assert C.sizeof(hd.Diag) == 9 * 8 + 8 * 4
    assert hd.Diag.flow_status.offset == 9 * 8 + 6 * 4


def test_null_and_size_errors_return_before_any_launch(hd):
    lib = hd.lib()
    p = hd.params()
    assert lib.hdrreg_local_search(None, None, 64, 64, None, C.byref(p), None, None, None, None,
                                   None) == 1
    assert lib.hdrreg_normalize_exposure(None, None, 64, 64, 0, 4, 1, None, None, None, None, 0,
                                         None) == 1
    f = hd.Frame(None, None, None)
    o = hd.PlanesF32(None, None, None)
    assert lib.hdrreg_warp(C.byref(f), 64, 64, None, None, None, C.byref(o), None, None) == 1
    assert lib.hdrreg_register_merge(C.byref(f), 64, 64, 1, None, None, None, C.byref(p), None, 0,
                                     C.byref(o), None, None) == 1
    assert lib.hdrreg_fit_homography(None, None, None, -1, 10, 10, None, None, None, None) == 1
    assert b"NULL" in lib.hdrreg_last_error() or b"range" in lib.hdrreg_last_error()


def test_batch_sizes_and_argument_errors(hd):
    lib = hd.lib()
    p = hd.params(tile=32, radius=6)
    one = hd.register_merge_workspace_size(2592, 1944, 1, p)
    four = lib.hdrreg_register_merge_batch_workspace_size(2592, 1944, 1, 4, C.byref(p))
    assert four >= 4 * one and four < 4 * (one + 256)
    assert lib.hdrreg_register_merge_batch_workspace_size(2592, 1944, 1, 0, C.byref(p)) == 0
    assert lib.hdrreg_register_merge_batch_workspace_size(2592, 1944, 1, hd.MAX_LANES + 1,
                                                          C.byref(p)) == 0
    # rejected on the host: bad lane count, negative count, missing stack array, NULL planes
    assert lib.hdrreg_register_merge_batch(None, 0, 64, 64, 1, 0, C.byref(p), None, 0, None) == 1
    assert lib.hdrreg_register_merge_batch(None, -1, 64, 64, 1, 2, C.byref(p), None, 0, None) == 1
    assert lib.hdrreg_register_merge_batch(None, 3, 64, 64, 1, 2, C.byref(p), None, 0, None) == 1
    f = hd.Frame(None, None, None)
    st = (hd.Stack * 1)()
    st[0].ref = C.pointer(f)
    assert lib.hdrreg_register_merge_batch(st, 1, 64, 64, 1, 2, C.byref(p), None, 0, None) == 1
    assert b"stack 0" in lib.hdrreg_last_error()
    # an empty batch with a workspace check only
    assert lib.hdrreg_register_merge_batch(None, 0, 64, 64, 1, 2, C.byref(p), None, 0, None) == 6


def test_python_binding_refuses_cpu_tensors(hd):
    import torch
    with pytest.raises(ValueError):
        hd._ptr(torch.zeros(4))


def test_host_staged_batch_sizes_and_errors(hd):
    lib = hd.lib()
    p = hd.params(tile=32, radius=6)
    one = hd.register_merge_workspace_size(2592, 1944, 1, p)
    n4 = lib.hdrreg_register_merge_host_workspace_size(2592, 1944, 1, 4, C.byref(p))
    staging = 2592 * 1944 * (1.5 * 2 + 6)
    assert n4 >= 4 * (one + staging) and n4 < 4 * (one + staging + 16 * 256 + 4096)
    assert lib.hdrreg_register_merge_host_workspace_size(2592, 1944, 1, 0, C.byref(p)) == 0
    assert lib.hdrreg_register_merge_host_workspace_size(2592, 1944, 0, 2, C.byref(p)) == 0
    assert lib.hdrreg_register_merge_host(None, 3, 64, 64, 1, 2, C.byref(p), None, 0, None) == 1
    assert lib.hdrreg_register_merge_host(None, 0, 64, 64, 1, 0, C.byref(p), None, 0, None) == 1
    f = hd.Frame(None, None, None)
    st = (hd.Stack * 1)()
    st[0].ref = C.pointer(f)
    assert lib.hdrreg_register_merge_host(st, 1, 64, 64, 1, 2, C.byref(p), None, 0, None) == 1
    assert b"stack 0" in lib.hdrreg_last_error()
    assert lib.hdrreg_register_merge_host(None, 0, 64, 64, 1, 2, C.byref(p), None, 0, None) == 6


def test_paper_preset_and_defaults(hd):
    d, p = hd.params(), hd.params_paper()
    # the paper equalizes the frames' histograms before matching (Sec. 3)
    assert d.norm_mode == hd.NORM_HISTEQ and p.norm_mode == hd.NORM_HISTEQ
    # the preset spreads the corners' whole displacement (Sec. 2.4); the default the residual
    assert d.propagate_full == 0 and p.propagate_full == 1
    dd, pd = d.as_dict(), p.as_dict()
    assert {k for k in dd if dd[k] != pd[k]} == {"propagate_full"}
    assert hd.lib().hdrreg_validate_params(C.byref(p)) == 0


def test_rate_probe_is_a_separate_library():
    # the benchmark's dp4a rate probe lives in its own library, not in the C ABI of the
    # registration library; its argument checks return before any launch
    from paper_1504_01441_b300 import build, probe
    build.build()
    import ctypes as C2
    main = C2.CDLL(build.LIB)
    assert not hasattr(main, "hdrreg_probe_dp4a")
    lib = probe.lib()
    sink = C2.c_uint32(0)
    assert lib.hdrreg_probe_dp4a(0, 16, C2.byref(sink), None) == 1
    assert lib.hdrreg_probe_dp4a(148, 0, C2.byref(sink), None) == 1
    assert lib.hdrreg_probe_dp4a(148, 16, None, None) == 1
