"""The fifth-generation tensor-core building block (tcgen05 BF16 MMA with
the FP32 accumulator in tensor memory) against a float64 matrix product of
the same BF16 values."""
import numpy as np
import pytest

from paper_2603_29785_gb300 import qtam

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,K,flags", [(256, 128, 0), (128, 256, 0), (16, 16, 0), (256, 256, 1), (64, 48, 2),
                                       (144, 128, 3), (128, 256, 4), (256, 128, 5), (32, 32, 4)])
def test_tc_gemm_matches_float64(N, K, flags):
    g = torch.Generator().manual_seed(N * 1000 + K * 10 + flags)
    A = torch.randn((128, K), generator=g).to(torch.bfloat16)
    B = torch.randn((N, K), generator=g).to(torch.bfloat16)
    D = torch.full((128, N), float("nan"), dtype=torch.float32, device="cuda")
    Ad, Bd = A.cuda().contiguous(), B.cuda().contiguous()
    qtam.qtam_tc_gemm_check(Ad, Bd, D, N, K, flags)
    torch.cuda.synchronize()
    a = A.double().numpy() * (-1 if flags & 1 else 1)
    b = B.double().numpy() * (-1 if flags & 2 else 1)
    ref = a @ b.T
    got = D.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got))
    # FP32 accumulation of K exact BF16 products
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref)) * np.sqrt(K)


def test_tc_gemm_rejects_bad_shapes():
    A = torch.zeros((128, 32), dtype=torch.bfloat16, device="cuda")
    D = torch.zeros((128, 32), dtype=torch.float32, device="cuda")
    for N, K in ((8, 32), (32, 24), (272, 32), (32, 512)):
        with pytest.raises(qtam.QtamError):
            qtam.qtam_tc_gemm_check(A, A, D, N, K)


def test_tc_bounded_wait_reports_timeout_and_context_survives():
    """A completion that never comes (no MMA issued): the clock-bounded wait
    gives up after ~1 ms, the timeout is counted, tensor memory is released and
    the next tensor-core call runs normally."""
    A = torch.zeros((128, 32), dtype=torch.bfloat16, device="cuda")
    D = torch.full((128, 32), 7.0, dtype=torch.float32, device="cuda")
    before = qtam.qtam_tc_status()
    qtam.qtam_tc_gemm_check(A, A, D, 32, 32, 8)
    torch.cuda.synchronize()
    assert qtam.qtam_tc_status() == before + 1
    assert torch.all(D == 7.0)                      # nothing was read back from tensor memory
    test_tc_gemm_matches_float64(128, 64, 0)        # the context and the tensor memory are usable
