"""GPU: the error-tolerant exposure fusion (row f1) against the oracle (oracle/fusion.py).

The fusion step on identical inputs (reference planes, warped FP32 planes, SSIM maps)
must match within 1e-4 * max(|oracle|, 1) element by element -- the FP32
pyramids against float64. The fused call with output_mode 1 is compared with the oracle's
registration (its warped planes and SSIM maps) followed by the oracle's fusion.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tolerance import check_end_to_end, check_rel, flow_sensitivity
pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def hd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_01441_b300 import build, hdrreg
    build.build()
    return hdrreg


def d(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda()


@pytest.mark.parametrize("w,h,nsrc,contrast,chroma", [(334, 250, 1, True, True),
                                                       (256, 192, 2, True, True),
                                                       (161, 97, 1, False, False),
                                                       (640, 480, 2, False, True)])
def test_fuse_step_matches_oracle(hd, w, h, nsrc, contrast, chroma):
    from oracle import fusion as F
    from paper_1504_01441_b300 import synth
    rng = np.random.default_rng(w + h + nsrc)
    ry = rng.integers(0, 256, (h, w), dtype=np.uint8)
    ru = rng.integers(0, 256, (h // 2, w // 2), dtype=np.uint8) if chroma else None
    rv = rng.integers(0, 256, (h // 2, w // 2), dtype=np.uint8) if chroma else None
    srcs, warped, qs = [], [], []
    for _ in range(nsrc):
        y = rng.uniform(0, 255, (h, w)).astype(np.float32)
        u = rng.uniform(0, 255, (h // 2, w // 2)).astype(np.float32) if chroma else None
        v = rng.uniform(0, 255, (h // 2, w // 2)).astype(np.float32) if chroma else None
        q = rng.uniform(0, 1, (h, w)).astype(np.float32)
        srcs.append(dict(y=d(y), u=d(u) if chroma else None, v=d(v) if chroma else None, q=d(q)))
        warped.append((y, u, v))
        qs.append(q)
    gy, gu, gv = hd.fuse(d(ry), d(ru) if chroma else None, d(rv) if chroma else None, srcs,
                         use_contrast=contrast)
    oy, ou, ov = F.fuse(ry, ru, rv, warped, qs, use_contrast=contrast)
    torch.cuda.synchronize()
    check_rel(gy.cpu().numpy(), oy, "y")
    if chroma:
        check_rel(gu.cpu().numpy(), ou, "u")
        check_rel(gv.cpu().numpy(), ov, "v")


@pytest.mark.parametrize("mode", [1, 2])
def test_fused_call_with_exposure_fusion(hd, orc, small_yuv_stack, mode):
    from oracle import fusion as F
    from paper_1504_01441_b300 import synth
    st = small_yuv_stack
    c = synth.method_params(16, 4, output_mode=mode)
    p = hd.params_from_dict(c)
    (y, u, v), rm = hd.register_merge((d(st.ref.y), d(st.ref.u), d(st.ref.v)),
                                      [(d(f.y), d(f.u), d(f.v)) for f in st.srcs], st.ratios, p)
    torch.cuda.synchronize()
    out = orc.register_merge(st.ref, st.srcs, st.ratios, c, want_intermediates=True)
    diag = rm.diagnostics()
    warped, qs = [], []
    for k, f in enumerate(st.srcs):
        assert np.array_equal(np.array(diag[k].H0[:]).view(np.uint64),
                              out["H0"][k].reshape(9).view(np.uint64))
        wy, wu, wv = orc.warp(f.y, f.u, f.v, out["H0"][k], out["flow_u"][k], out["flow_v"][k])
        warped.append((wy, wu, wv))
        qs.append(out["q"][k])
    oy, ou, ov = F.fuse(st.ref.y, st.ref.u, st.ref.v, warped, qs, use_contrast=(mode == 1))
    # end to end the fusion weights (contrast ratios) amplify the FP32 flow's error, so the
    # planes are held to the rule plus the oracle fusion's own movement under the flow's
    # tolerance; the fusion step itself meets the bare rule on identical inputs (above)
    base, sens = flow_sensitivity(orc, st, out, c, output="fusion", use_contrast=(mode == 1))
    assert np.array_equal(base[0], oy)
    for name, g, o, sn in (("y", y, oy, sens[0]), ("u", u, ou, sens[1]), ("v", v, ov, sens[2])):
        check_end_to_end(g.cpu().numpy(), o, sn, name)


def test_fused_exposure_fusion_at_5mp(hd, orc):
    # the fusion output of the fused call on the 2592 x 1944 YUV420 pair of the batch
    # workload (T = 32, R = 6), against the oracle's registration followed by the oracle
    # fusion: same H0 bits, planes within the parity tolerance
    from oracle import fusion as F
    from paper_1504_01441_b300 import synth
    st = synth.make_stack(synth.FIVE_MP, synth.stack_seed(2, 0))
    c = synth.method_params(32, 6, output_mode=1)
    p = hd.params_from_dict(c)
    (y, u, v), rm = hd.register_merge((d(st.ref.y), d(st.ref.u), d(st.ref.v)),
                                      [(d(f.y), d(f.u), d(f.v)) for f in st.srcs], st.ratios, p)
    torch.cuda.synchronize()
    out = orc.register_merge(st.ref, st.srcs, st.ratios, c, want_intermediates=True)
    f = st.srcs[0]
    assert np.array_equal(np.array(rm.diagnostics()[0].H0[:]).view(np.uint64),
                          out["H0"][0].reshape(9).view(np.uint64))
    wy, wu, wv = orc.warp(f.y, f.u, f.v, out["H0"][0], out["flow_u"][0], out["flow_v"][0])
    oy, ou, ov = F.fuse(st.ref.y, st.ref.u, st.ref.v, [(wy, wu, wv)], [out["q"][0]])
    base, sens = flow_sensitivity(orc, st, out, c, output="fusion")
    assert np.array_equal(base[0], oy)
    for name, g, o, sn in (("y", y, oy, sens[0]), ("u", u, ou, sens[1]), ("v", v, ov, sens[2])):
        check_end_to_end(g.cpu().numpy(), o, sn, name)


def test_fuse_contrast_on_smooth_fp32_frames(hd):
    # two smooth warped-like FP32 frames (planes with slopes of 1/3 and 1/7, rounded to
    # FP32) and a flat reference: the contrasts are the rounding residue of the planes, a
    # few 1e-6 DN, and the normalized weights are their ratio. The step call must evaluate
    # |4 z - sum of the neighbours| on the FP32 values as the oracle does, not with FP32
    # rounding of its own.
    from oracle import fusion as F
    h, w = 96, 128
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    ref = np.full((h, w), 60, np.uint8)
    s1 = (80.0 + x / 3.0 + y / 7.0).astype(np.float32)
    s2 = (150.0 - x / 7.0 + y / 3.0).astype(np.float32)
    q = np.full((h, w), 0.75, np.float32)
    srcs = [dict(y=d(s), q=d(q)) for s in (s1, s2)]
    gy, _, _ = hd.fuse(d(ref), None, None, srcs, use_contrast=True)
    oy, _, _ = F.fuse(ref, None, None, [(s1, None, None), (s2, None, None)], [q, q],
                      use_contrast=True)
    torch.cuda.synchronize()
    check_rel(gy.cpu().numpy(), oy, "y")
