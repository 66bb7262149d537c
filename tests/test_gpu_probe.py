"""GPU: the benchmark's integer dot-product rate probe (libhdrreg_probe.so) launches,
finishes, and counts the operations it issues."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_dp4a_rate_probe_runs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_01441_b300 import build, probe
    build.build()
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    n = probe.probe_dp4a(148, 64, sink)
    torch.cuda.synchronize()
    assert n == 148 * 256 * 64 * 8
