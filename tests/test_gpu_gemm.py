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


# --- FP8 E4M3 operands (tcgen05.mma kind::f8f6f4) ---------------------------

def _e4m3(torch, x):
    """E4M3 bytes of x: nearest even, saturated to +-448 (torch's conversion
    after a clamp)."""
    return x.float().clamp(-448.0, 448.0).to(torch.float8_e4m3fn).view(torch.uint8)


def _dec(torch, b):
    return b.view(torch.float8_e4m3fn).float()


def _e4m3_step(x):
    # spacing of E4M3 numbers at |x| (3 mantissa bits, subnormal step 2^-9)
    e = np.floor(np.log2(np.maximum(np.abs(x), 2.0 ** -6)))
    return 2.0 ** (e - 3)


@pytest.mark.parametrize("M,N,K", [(128, 64, 128), (300, 256, 256), (1000, 392, 256),
                                   (77, 256, 16), (513, 130, 144), (4096, 256, 256)])
def test_gemm_fp8_matches_reference(env, M, N, K):
    # the products of E4M3 numbers are exact in FP32; the accumulation order
    # of the tensor core is not fixed, so the bound is relative to sum |a b|
    torch, binding = env
    g = torch.Generator(device="cpu").manual_seed(M * 5 + N)
    A8 = _e4m3(torch, torch.randn(M, K, generator=g) * 40)
    B8 = _e4m3(torch, torch.randn(N, K, generator=g) * 40)
    a_scale = 0.0123
    b_scale = torch.rand(N, generator=g) * 0.01 + 0.001
    bias = torch.randn(N, generator=g)
    C32, C16, C8 = binding.gemm_fp8(A8.cuda(), a_scale, B8.cuda(), b_scale.cuda(),
                                    bias=bias.cuda())
    assert C16 is None and C8 is None
    a, b = _dec(torch, A8).double(), _dec(torch, B8).double()
    s = (torch.tensor(a_scale, dtype=torch.float32) * b_scale).double()
    ref = (a @ b.T) * s + bias.double()
    mag = (a.abs() @ b.abs().T) * s
    err = (C32.cpu().double() - ref).abs()
    assert bool((err <= 2.0 ** -10 * mag + 1e-5 * (1 + ref.abs())).all()), err.max().item()


def test_gemm_fp8_outputs_and_epilogue(env):
    torch, binding = env
    g = torch.Generator(device="cpu").manual_seed(9)
    M, N, K = 700, 256, 256
    A8 = _e4m3(torch, torch.randn(M, K, generator=g) * 20).cuda()
    B8 = _e4m3(torch, torch.randn(N, K, generator=g) * 20).cuda()
    bs = (torch.rand(N, generator=g) * 0.002 + 0.001).cuda()
    bias = torch.randn(N, generator=g).cuda()
    inv = float(np.float32(1.0) / np.float32(0.02))
    # identity: C8 is exactly the E4M3 conversion of the FP32 output times inv
    C32, C16, C8 = binding.gemm_fp8(A8, 0.05, B8, bs, bias=bias, act=0, out32=True,
                                    out16=True, out8_inv_scale=inv)
    c32 = C32.cpu()
    assert torch.equal(C8.cpu(), _e4m3(torch, c32 * torch.tensor(inv, dtype=torch.float32)))
    assert torch.equal(C16.cpu(), c32.to(torch.bfloat16))
    # GELU: C16 and C8 hold the activated value (within one rounding step of
    # the tanh-form GELU of the FP32 pre-activation)
    C32g, C16g, C8g = binding.gemm_fp8(A8, 0.05, B8, bs, bias=bias, act=1, out32=True,
                                       out16=True, out8_inv_scale=inv)
    assert torch.equal(C32g.cpu(), c32)
    post = torch.nn.functional.gelu(c32.double(), approximate="tanh")
    assert torch.allclose(C16g.cpu().double(), post, rtol=1e-2, atol=1e-3)
    want = (post * inv).clamp(-448, 448).numpy()
    got = _dec(torch, C8g.cpu()).double().numpy()
    assert np.all(np.abs(got - want) <= _e4m3_step(want) + 1e-9)
    # saturation: values far beyond 448 / inv come out as +-448
    C32s, _, C8s = binding.gemm_fp8(A8, 50.0, B8, bs, act=0, out32=True, out8_inv_scale=inv)
    big = (C32s.cpu() * inv).abs() > 464
    assert bool(big.any())
    assert bool((_dec(torch, C8s.cpu())[big].abs() == 448).all())


def test_bf16_layer_with_fp8_output(env):
    torch, binding = env
    g = torch.Generator(device="cpu").manual_seed(4)
    M, N, K = 333, 256, 16
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    Bt = (torch.randn(N, K, generator=g) * 0.5).to(torch.bfloat16).cuda()
    bias = torch.randn(N, generator=g).float().cuda()
    inv = float(np.float32(1.0) / np.float32(0.01))
    C32, _ = binding.gemm_bf16(A, Bt, bias=bias, act=0, out32=True)
    C8 = binding.gemm_bf16_to_fp8(A, Bt, inv, bias=bias, act=0)
    assert torch.equal(C8.cpu(), _e4m3(torch, C32.cpu() * torch.tensor(inv, dtype=torch.float32)))


def test_fp8_quantisation_helpers(env):
    torch, binding = env
    g = torch.Generator(device="cpu").manual_seed(5)
    W = torch.randn(300, 256, generator=g) * torch.exp(torch.randn(300, 1, generator=g))
    W[5] = 0.0
    W8, sc = binding.quant_fp8_rows(W.cuda())
    sc_ref = W.abs().amax(1) / 448.0
    sc_ref[5] = 1.0
    assert torch.equal(sc.cpu(), sc_ref)
    assert torch.equal(W8.cpu(), _e4m3(torch, W / sc_ref[:, None]))
    # every row uses the full range: its largest entry quantises to +-448
    assert bool((_dec(torch, W8.cpu()).abs().amax(1)[torch.arange(300) != 5] == 448).all())
    x = (torch.randn(100_003, generator=g) * 3).to(torch.bfloat16)
    assert binding.absmax_bf16(x.cuda()) == x.float().abs().max().item()
    inv = float(np.float32(1.0) / np.float32(0.005))
    x8 = binding.quant_fp8_bf16(x.cuda(), inv)
    assert torch.equal(x8.cpu(), _e4m3(torch, x.float() * torch.tensor(inv, dtype=torch.float32)))
