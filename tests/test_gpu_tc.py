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


def colmajor_batch(torch, mats):
    """(batch, cols, rows) contiguous storage of column-major matrices."""
    return torch.stack([x.t().contiguous() for x in mats])


@pytest.mark.parametrize("S,prec", [(7, 0), (3, 1), (3, 0), (4, 1), (-3, 1), (1, 1)])
@pytest.mark.parametrize("m,n,k,batch", [(1, 1, 1, 1), (37, 33, 7, 2), (200, 100, 32, 1), (1000, 300, 32, 3),
                                         (65, 129, 17, 2)])
@pytest.mark.parametrize("opa,opb", [("N", "N"), ("C", "N"), ("T", "C")])
@pytest.mark.parametrize("alpha,beta", [(-1.0, 1), (1.0, 0)])
def test_zgemm_sliced(gbf, S, prec, m, n, k, batch, opa, opb, alpha, beta):
    import torch

    dt = torch.complex128 if prec == 0 else torch.complex64
    g = torch.Generator(device="cuda").manual_seed(m + 3 * n + 7 * k)
    def rnd(r, c):
        return torch.complex(torch.randn((r, c), device="cuda", dtype=torch.float64, generator=g),
                             torch.randn((r, c), device="cuda", dtype=torch.float64, generator=g))
    As = [rnd(m, k) if opa == "N" else rnd(k, m) for _ in range(batch)]
    Bs = [rnd(k, n) if opb == "N" else rnd(n, k) for _ in range(batch)]
    Cs = [rnd(m, n) for _ in range(batch)]
    A = colmajor_batch(torch, As).to(dt)
    B = colmajor_batch(torch, Bs).to(dt)
    Cd = colmajor_batch(torch, Cs).to(dt)
    op = {"N": lambda x: x, "T": lambda x: x.t(), "C": lambda x: x.conj().t()}
    ref = [alpha * (op[opa](a.to(dt).to(torch.complex128)) @ op[opb](b.to(dt).to(torch.complex128)))
           + (beta * c.to(dt).to(torch.complex128)) for a, b, c in zip(As, Bs, Cs)]
    rc = gbf.zgemm_sliced(opa, opb, A, B, Cd, alpha=alpha, beta=beta, S=S)
    torch.cuda.synchronize()
    assert rc == 0, gbf.last_error()
    got = [Cd[i].t().to(torch.complex128) for i in range(batch)]
    # S = 1: 3xTF32 products (about 2^-22 relative each) accumulated in FP32
    tol = (4e-14 if S == 7 else 2e-6) * k
    if prec == 1:
        tol = max(tol, 1e-6 * k)   # FP32 output rounding
    for gt, rf in zip(got, ref):
        assert (gt - rf).abs().max().item() <= tol * (1 + rf.abs().max().item()), (gt - rf).abs().max().item()


@pytest.mark.parametrize("cplx", [0, 1])
@pytest.mark.parametrize("m,n,k,batch", [(1, 1, 1, 1), (37, 33, 7, 2), (200, 100, 100, 1), (300, 70, 257, 2),
                                         (130, 300, 1000, 1)])
@pytest.mark.parametrize("opa,opb", [("N", "N"), ("T", "N"), ("C", "N"), ("N", "C")])
@pytest.mark.parametrize("alpha,beta", [(-1.0, 1), (1.0, 0)])
def test_gemm_sliced_any_k(gbf, cplx, m, n, k, batch, opa, opb, alpha, beta):
    """FP64-class sliced GEMM for any k against an FP64 product: error within a
    few units of k * 2^-53 * max|A| max|B| (8 digits: 56 bits per operand)."""
    import torch

    g = torch.Generator(device="cuda").manual_seed(11 * m + 5 * n + k + cplx)

    def rnd(r, c):
        x = torch.randn((r, c), device="cuda", dtype=torch.float64, generator=g)
        if cplx:
            x = torch.complex(x, torch.randn((r, c), device="cuda", dtype=torch.float64, generator=g))
        return x

    As = [rnd(m, k) if opa == "N" else rnd(k, m) for _ in range(batch)]
    Bs = [rnd(k, n) if opb == "N" else rnd(n, k) for _ in range(batch)]
    Cs = [rnd(m, n) for _ in range(batch)]
    A, B, Cd = colmajor_batch(torch, As), colmajor_batch(torch, Bs), colmajor_batch(torch, Cs)
    op = {"N": lambda x: x, "T": lambda x: x.t(), "C": lambda x: x.conj().t()}
    ref = [alpha * (op[opa](a) @ op[opb](b)) + beta * c for a, b, c in zip(As, Bs, Cs)]
    rc = gbf.gemm_sliced(opa, opb, A, B, Cd, alpha=alpha, beta=beta)
    torch.cuda.synchronize()
    assert rc == 0, gbf.last_error()
    kr = (2 if cplx else 1) * k
    for i in range(batch):
        got = Cd[i].t()
        scale = As[i].abs().max().item() * Bs[i].abs().max().item()
        tol = 4 * kr * 2.0 ** -53 * scale + 2.0 ** -52 * ref[i].abs().max().item()
        assert (got - ref[i]).abs().max().item() <= tol, ((got - ref[i]).abs().max().item(), tol)


def test_tf32_engine_needs_complex_fp32(gbf):
    """S = 1 (3xTF32) is the FP32-factor engine: an FP64 call is refused
    before anything is launched."""
    import torch

    A = torch.zeros((1, 8, 32), dtype=torch.complex128, device="cuda")
    B = torch.zeros((1, 32, 8), dtype=torch.complex128, device="cuda")
    C = torch.zeros((1, 32, 32), dtype=torch.complex128, device="cuda")
    rc = gbf.zgemm_sliced("N", "N", A, B, C, alpha=1.0, beta=0, S=1)
    torch.cuda.synchronize()
    assert rc != 0 and "3xTF32" in gbf.last_error()


@pytest.mark.parametrize("m,n,k,batch", [(1, 1, 1, 1), (37, 33, 7, 2), (200, 100, 100, 1), (300, 70, 257, 2),
                                         (130, 300, 1000, 1), (2048, 300, 2048, 2)])
@pytest.mark.parametrize("opa,opb", [("N", "N"), ("T", "N"), ("C", "N"), ("N", "C")])
@pytest.mark.parametrize("alpha,beta", [(-1.0, 1), (1.0, 0)])
def test_cgemm_tf32_any_k(gbf, m, n, k, batch, opa, opb, alpha, beta):
    """3xTF32 complex FP32 GEMM for any k (the FP32 factors' recursive solve
    updates) against an FP64 product of the same complex64 operands: each
    product is exact to about 2^-22 relative and the FP32 accumulation over
    the real embedding's 2k terms adds about sqrt(2k) 2^-24; the bound below
    is a few units of 2k 2^-22 max|A| max|B| plus the FP32 rounding of C."""
    import torch

    g = torch.Generator(device="cuda").manual_seed(13 * m + 7 * n + k)

    def rnd(r, c):
        return torch.complex(torch.randn((r, c), device="cuda", dtype=torch.float32, generator=g),
                             torch.randn((r, c), device="cuda", dtype=torch.float32, generator=g))

    As = [rnd(m, k) if opa == "N" else rnd(k, m) for _ in range(batch)]
    Bs = [rnd(k, n) if opb == "N" else rnd(n, k) for _ in range(batch)]
    Cs = [rnd(m, n) for _ in range(batch)]
    A, B, Cd = colmajor_batch(torch, As), colmajor_batch(torch, Bs), colmajor_batch(torch, Cs)
    op = {"N": lambda x: x, "T": lambda x: x.t(), "C": lambda x: x.conj().t()}
    w = torch.complex128
    ref = [alpha * (op[opa](a.to(w)) @ op[opb](b.to(w))) + beta * c.to(w) for a, b, c in zip(As, Bs, Cs)]
    rc = gbf.cgemm_tf32(opa, opb, A, B, Cd, alpha=alpha, beta=beta)
    torch.cuda.synchronize()
    assert rc == 0, gbf.last_error()
    for i in range(batch):
        got = Cd[i].t().to(w)
        scale = As[i].abs().max().item() * Bs[i].abs().max().item()
        tol = 4 * (2 * k) * 2.0 ** -22 * scale + 2.0 ** -23 * ref[i].abs().max().item()
        assert (got - ref[i]).abs().max().item() <= tol, ((got - ref[i]).abs().max().item(), tol)


def test_bounded_wait_times_out_and_gpu_stays_usable(gbf):
    """The time-out path of the engine's bounded waits: a wait on a barrier
    that nothing completes runs out after the given polls and reports -5;
    the next sliced GEMM on the same stream is correct."""
    import torch

    L = gbf.lib()
    st = torch.cuda.current_stream()
    sp = gbf._stream_ptr(st)
    assert L.gbf_wait_probe(sp, 1000) == -5
    assert "timed out" in gbf.last_error()
    assert L.gbf_wait_probe(sp, 0) == -101
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randn((64, 32), device="cuda", dtype=torch.complex128, generator=g)
    B = torch.randn((32, 48), device="cuda", dtype=torch.complex128, generator=g)
    Cd = colmajor_batch(torch, [torch.zeros((64, 48), device="cuda", dtype=torch.complex128)])
    ref = A @ B
    rc = gbf.zgemm_sliced("N", "N", colmajor_batch(torch, [A]), colmajor_batch(torch, [B]), Cd, alpha=1.0, beta=0,
                          S=7)
    torch.cuda.synchronize()
    assert rc == 0, gbf.last_error()
    assert (Cd[0].t() - ref).abs().max().item() <= 4e-14 * 32 * (1 + ref.abs().max().item())
