"""The tensor-core dense layer (tcgen05, FP32 accumulation in tensor memory)
against a plain PyTorch FP32 computation of the same operation on the same
BF16 inputs.  Shapes span several tiles, ragged M and N, K below one
pipeline stage, and the bias + GELU epilogue."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_01421_gb300 import binding
    binding.build()
    return torch, binding


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (300, 256, 256), (1000, 387, 256),
                                   (77, 256, 16), (513, 130, 136), (4096, 256, 256)])
def test_gemm_matches_fp32_reference(env, M, N, K):
    torch, binding = env
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N)
    A = (torch.randn(M, K, generator=g) * 0.5).to(torch.bfloat16).cuda()
    Bt = (torch.randn(N, K, generator=g) * 0.1).to(torch.bfloat16).cuda()
    C32, _ = binding.gemm_bf16(A, Bt)
    ref = A.double().cpu() @ Bt.double().cpu().T
    err = (C32.double().cpu() - ref).abs().max().item()
    scale = ref.abs().max().item()
    assert err <= 1e-5 * max(1.0, scale) * max(1, K // 16)


def test_gemm_bias_gelu_epilogue(env):
    torch, binding = env
    g = torch.Generator(device="cpu").manual_seed(3)
    M, N, K = 260, 256, 64
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    Bt = (torch.randn(N, K, generator=g) * 0.2).to(torch.bfloat16).cuda()
    bias = torch.randn(N, generator=g).float().cuda()
    C32, C16 = binding.gemm_bf16(A, Bt, bias=bias, act=1, out32=True, out16=True)
    pre = A.double().cpu() @ Bt.double().cpu().T + bias.double().cpu()
    assert torch.allclose(C32.double().cpu(), pre, rtol=1e-5, atol=1e-4)
    post = torch.nn.functional.gelu(pre, approximate="tanh")
    assert torch.allclose(C16.double().cpu(), post, rtol=1e-2, atol=1e-2)
