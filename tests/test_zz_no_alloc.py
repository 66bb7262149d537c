"""hdrreg_weed_static: the weeding step for callers that cannot allocate device
memory (for example a real-time pipeline that allows no allocation after
start-up, or a plugin whose host owns all device memory).

It keeps its scratch in a fixed array inside the library instead of a
caller-provided workspace. This test calls it through the C ABI on two calls in
a row with different inputs and checks each mask against hdrreg_weed (the
workspace entry point) bit for bit: the masks are integer outputs, so the
tolerance the other tests use for them is exact equality. It also checks that
sizes beyond the array's capacity are rejected before anything is launched.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_weed_static_matches_the_workspace_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_01441_b300 import build, hdrreg, synth
    build.build()
    lib = hdrreg.lib()
    st = synth.make_stack(synth.VGA_LUMA, synth.stack_seed(1))
    p = hdrreg.params_from_dict(synth.method_params(16, 4))
    ref = torch.from_numpy(st.ref.y).cuda()
    src = torch.from_numpy(st.srcs[0].y).cuda()
    rn, sn, _ = hdrreg.normalize_exposure(ref, src, hdrreg.NORM_RATIO, st.ratios[0])
    H = torch.tensor([1, 0, 0, 0, 1, 0, 0, 0, 1], dtype=torch.float64, device="cuda")
    cxy, mxy, cost, valid = hdrreg.local_search(rn, sn, H, p)
    h, w = rn.shape
    stream = torch.cuda.current_stream().cuda_stream

    # two calls in a row on different inputs: the whole frame, then its first half of the
    # tiles with another seed (the second call must not see the first call's scratch)
    cases = [(valid.numel(), 11, 0, p.weed_iters), (valid.numel() // 2, 12, 5, 300)]
    for n, seed, it0, it1 in cases:
        c, m, v = cxy[:n].contiguous(), mxy[:n].contiguous(), valid[:n].contiguous()
        want = hdrreg.weed(c, m, v, w, h, p, seed, it0, it1)
        got = torch.zeros_like(want)
        status = lib.hdrreg_weed_static(c.data_ptr(), m.data_ptr(), v.data_ptr(), n, w, h,
                                        C.byref(p), C.c_uint64(seed), it0, it1, got.data_ptr(),
                                        stream)
        assert status == 0, lib.hdrreg_last_error().decode()
        torch.cuda.synchronize()
        assert int(want.count_nonzero()) > 0
        assert torch.equal(got, want)

    # beyond the static capacity: a clear error and no launch
    too_many = 8192 + 1
    assert lib.hdrreg_weed_static(None, None, None, too_many, w, h, C.byref(p), C.c_uint64(1), 0,
                                  10, None, stream) == 1
    assert b"8192" in lib.hdrreg_last_error()
