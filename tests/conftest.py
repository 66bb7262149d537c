import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size workload")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def vga_stack():
    from paper_1504_01441_b300 import synth
    return synth.make_stack(synth.VGA_LUMA, synth.stack_seed(1))


@pytest.fixture(scope="session")
def small_yuv_stack():
    from paper_1504_01441_b300 import synth
    spec = synth.StackSpec(320, 240, ratios=((4, 1),), noise_sigma=1.0, field_amp=3.0, movers=1,
                           chroma=True)
    return synth.make_stack(spec, synth.stack_seed(9))
