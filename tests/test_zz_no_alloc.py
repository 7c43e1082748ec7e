"""The sliced tensor-core GEMM entry that allocates no device memory
(gbf_zgemm_sliced_noalloc), for callers that cannot allocate during the call.

Both entries run the same kernels on the same inputs with the same launch
shapes (the workspace size only gates the call), so the no-allocation entry
must give exactly (bit for bit) what the allocating entry (gbf_zgemm_sliced,
caller-provided workspace) gives, on consecutive calls that reuse its fixed
scratch array; a warm call must not lower the device's free memory; and it
must refuse a problem whose scratch would not fit, without launching anything.  This file is collected
last and also passes when run alone in a fresh process (its first call then
does the one-time lookup of the array's device address)."""
import pytest

pytestmark = pytest.mark.gpu


def _rnd(torch, g, r, c):
    return torch.complex(torch.randn((r, c), device="cuda", dtype=torch.float64, generator=g),
                         torch.randn((r, c), device="cuda", dtype=torch.float64, generator=g))


def _case(torch, seed, m, n, k, batch, opa, opb, dt):
    g = torch.Generator(device="cuda").manual_seed(seed)
    As = [_rnd(torch, g, m, k) if opa == "N" else _rnd(torch, g, k, m) for _ in range(batch)]
    Bs = [_rnd(torch, g, k, n) if opb == "N" else _rnd(torch, g, n, k) for _ in range(batch)]
    Cs = [_rnd(torch, g, m, n) for _ in range(batch)]
    pack = lambda xs: torch.stack([x.t().contiguous() for x in xs]).to(dt)  # noqa: E731
    return pack(As), pack(Bs), pack(Cs)


CALLS = [
    # (seed, m, n, k, batch, opa, opb, alpha, beta, S, complex dtype)
    (11, 300, 200, 32, 2, "N", "C", -1.0, 1, 7, "complex128"),
    (12, 129, 65, 17, 1, "C", "N", 1.0, 0, 3, "complex64"),
    (13, 150, 90, 32, 2, "N", "N", -1.0, 1, 1, "complex64"),
]


def test_noalloc_matches_allocating_entry_on_consecutive_calls(gbf):
    import torch

    for seed, m, n, k, batch, opa, opb, alpha, beta, S, dts in CALLS:
        dt = getattr(torch, dts)
        A, B, C0 = _case(torch, seed, m, n, k, batch, opa, opb, dt)
        C_ref = C0.clone()
        C_new = C0.clone()
        assert gbf.zgemm_sliced(opa, opb, A, B, C_ref, alpha=alpha, beta=beta, S=S) == 0, gbf.last_error()
        rc = gbf.zgemm_sliced_noalloc(opa, opb, A, B, C_new, alpha=alpha, beta=beta, S=S)
        torch.cuda.synchronize()
        assert rc == 0, gbf.last_error()
        torch.cuda.synchronize()
        assert torch.equal(C_new, C_ref), (seed, S, dts)


def test_noalloc_warm_call_takes_no_device_memory(gbf):
    import torch

    seed, m, n, k, batch, opa, opb, alpha, beta, S, dts = CALLS[0]
    A, B, C0 = _case(torch, seed, m, n, k, batch, opa, opb, getattr(torch, dts))
    C = C0.clone()
    assert gbf.zgemm_sliced_noalloc(opa, opb, A, B, C, alpha=alpha, beta=beta, S=S) == 0, gbf.last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert gbf.zgemm_sliced_noalloc(opa, opb, A, B, C, alpha=alpha, beta=beta, S=S) == 0, gbf.last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (2 << 20), (free0, free1)


def test_noalloc_rejects_problems_beyond_its_scratch(gbf):
    import torch

    lim = gbf.lib().gbf_zgemm_sliced_noalloc_max()
    assert 0 < lim < (64 << 20)
    m = n = 8192
    batch = 4
    assert gbf.lib().gbf_zgemm_sliced_work(m, n, batch, 7) > lim
    dummy = torch.zeros((1, 1, 1), dtype=torch.complex128, device="cuda")
    rc = gbf.lib().gbf_zgemm_sliced_noalloc(None, 0, 7, b"N", b"N", m, n, 8, 1.0, dummy.data_ptr(), m, 0,
                                            dummy.data_ptr(), 8, 0, 0, dummy.data_ptr(), m, 0, batch)
    assert rc == -7
    assert "scratch" in gbf.last_error()
