"""tcgen05 tensor-core GEMM building block (bf16 x bf16 -> FP32 in TMEM)
against an FP64 reference of the same bf16 operands.  Each bf16 product is
exact in FP32, so the only error is FP32 accumulation (bounded by K u32)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K,batch", [(128, 128, 64, 1), (200, 130, 200, 3), (64, 300, 1024, 2),
                                         (1000, 1000, 512, 1)])
def test_tc_gemm_bf16(gbf, M, N, K, batch):
    import torch

    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn((batch, M, K), device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn((batch, N, K), device="cuda", generator=g).to(torch.bfloat16)
    C, rc = gbf.tc_gemm_bf16(A, B)
    torch.cuda.synchronize()
    assert rc == 0, gbf.last_error()
    ref = torch.einsum("bmk,bnk->bnm", A.double(), B.double())
    err = (C.double() - ref).abs().max().item()
    scale = torch.einsum("bmk,bnk->bnm", A.double().abs(), B.double().abs()).max().item()
    assert err <= 2 * K * 6e-8 * scale, (err, scale)
