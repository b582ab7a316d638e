"""The tcgen05 GEMM kernel against a PyTorch FP32 matmul of the same BF16 operands."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 128, 512), (1000, 512, 512), (77, 16, 512),
                                   (513, 64, 4096), (4096, 512, 64), (128, 256, 128)])
def test_gemm_matches_torch(prlib, cuda, M, N, K):
    import torch
    from paper_2312_04830_gb300 import binding
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 13 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).to(cuda)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).to(cuda)
    D, err = binding.gemm_bf16(A, B)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = A.float() @ B.float().T
    # FP32 accumulation of exact BF16 products: differences are summation order only
    tol = 1e-5 * (K ** 0.5) * ref.abs().max().item() + 1e-6
    assert (D - ref).abs().max().item() <= tol
