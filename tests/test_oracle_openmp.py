"""The OpenMP build of the oracle (liboracle_omp.so, the multi-core CPU baseline) gives
the same bits as the serial build: every output element is computed by the same
operations in the same order, and the weeding union does not depend on the order of
its iterations (Sec. 2.3)."""
import numpy as np
import pytest


@pytest.fixture
def both(orc):
    orc.build()
    yield orc
    orc.set_parallel(False)


def run(orc, parallel, fn):
    orc.set_parallel(parallel)
    try:
        return fn()
    finally:
        orc.set_parallel(False)


def same(a, b):
    if isinstance(a, dict):
        return a.keys() == b.keys() and all(same(a[k], b[k]) for k in a)
    if isinstance(a, (list, tuple)):
        return len(a) == len(b) and all(same(x, y) for x, y in zip(a, b))
    if a is None:
        return b is None
    a, b = np.asarray(a), np.asarray(b)
    return a.dtype == b.dtype and a.shape == b.shape and a.tobytes() == b.tobytes()


def test_openmp_build_uses_threads(both):
    assert run(both, True, both.threads) >= 1
    assert both.threads() == 1


@pytest.mark.parametrize("which", ["vga", "yuv3"])
def test_register_merge_same_bits(both, vga_stack, which):
    from paper_1504_01441_b300 import synth
    if which == "vga":
        st, c = vga_stack, synth.method_params(16, 4)
    else:
        spec = synth.StackSpec(256, 192, ratios=((1, 4), (4, 1)), noise_sigma=1.0,
                               field_amp=2.0, movers=1, chroma=True, n_blobs=40, n_rects=10)
        st, c = synth.make_stack(spec, 33), synth.method_params(16, 4, norm_mode=1)
    f = lambda: both.register_merge(st.ref, st.srcs, st.ratios, c, want_intermediates=True)
    assert same(run(both, False, f), run(both, True, f))


def test_weeding_same_bits(both, vga_stack):
    from paper_1504_01441_b300 import synth
    c = synth.method_params(16, 4)
    rn, sn = both.normalize_ratio(vga_stack.ref.y, vga_stack.srcs[0].y, 4, 1)
    m = both.match(rn, sn, c)
    f = lambda: both.weed(m["corner_xy"], m["match_xy"], m["valid"], 640, 480, c,
                          c["weed_seed"], 0, 2048)
    a, b = run(both, False, f), run(both, True, f)
    assert same(a, b)
