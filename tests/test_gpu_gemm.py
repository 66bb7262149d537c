"""Tensor-core bf16 product (row a-L building block) against float64 numpy.

Integer-valued operands (multiples of 1/4 in [-2, 2]) make every product and every
FP32 partial sum exact, so those cases must match bit for bit; random normal
operands must match within the FP32 accumulation error."""
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


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (300, 48, 200), (77, 128, 24), (513, 200, 136),
                                   (64, 32, 8), (129, 64, 1000)])
def test_gemm_exact_on_quarter_integers(hd, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.integers(-8, 9, (M, K)) / 4.0
    B = rng.integers(-8, 9, (N, K)) / 4.0
    C, st = hd.gemm_bf16(torch.tensor(A, dtype=torch.bfloat16).cuda(),
                         torch.tensor(B, dtype=torch.bfloat16).cuda())
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(C.cpu().numpy().astype(np.float64), A @ B.T)


def test_gemm_random_within_fp32_accumulation(hd):
    rng = np.random.default_rng(9)
    M, N, K = 1000, 64, 576
    A = torch.tensor(rng.normal(size=(M, K)), dtype=torch.bfloat16)
    B = torch.tensor(rng.normal(size=(N, K)), dtype=torch.bfloat16)
    C, st = hd.gemm_bf16(A.cuda(), B.cuda())
    want = A.double().numpy() @ B.double().numpy().T
    got = C.cpu().numpy()
    assert int(st.item()) == 0
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max() + 1e-4


def test_gemm_rejects_misaligned_rows(hd):
    A = torch.zeros((16, 12), dtype=torch.bfloat16, device="cuda")  # lda = 12 (not a multiple of 8)
    B = torch.zeros((16, 12), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(hd.HdrregError):
        hd.gemm_bf16(A, B)
