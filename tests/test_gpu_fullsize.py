"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (device-pointer driver, inputs resident on the GPU):
  * n=4096 real symmetric generalized (M0=300, Ne=8): M against the Sylvester
    inertia count and the oracle's eigenvalues (stored by
    tests/golden/make_golden.py from the oracle alone), per-pair residuals;
  * n=8192 complex Hermitian (M0=240, Ne=16, mixed and FP64 paths): eigenvalues
    against the generated spectrum (A = U diag(lam) U^H exactly), residuals.
"""
import json
import os

import numpy as np
import pytest

from paper_1203_4031_gb300 import workloads as W

from feast_check import TOL_E, TOL_R, compare_eigs

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden", "real_generalized_n4096.json")


def gpu_residuals(A, B, X, E, torch):
    R = A @ X - ((B @ X) if B is not None else X) * E[None, :]
    nA = torch.linalg.matrix_norm(A, ord=1)
    return (torch.linalg.vector_norm(R, dim=0) / (nA * torch.linalg.vector_norm(X, dim=0))).cpu().numpy()


@pytest.fixture(scope="module")
def cfg2(gbf):
    import torch

    p = W.dense_real_generalized()
    A = gbf.fortran(torch.from_numpy(np.ascontiguousarray(p.A)).cuda())
    B = gbf.fortran(torch.from_numpy(np.ascontiguousarray(p.B)).cuda())
    return p, A, B


@pytest.mark.parametrize("prec,engine", [(0, 0), (1, 0), (0, 1)])
def test_real_generalized_4096(gbf, cfg2, prec, engine):
    import torch

    p, A, B = cfg2
    fpm = p.apply_fpm(gbf.gbf_init())
    fpm[41] = prec
    fpm[43] = engine
    h = gbf.Handle()
    r = gbf.feast_dev(A, B, p.emin, p.emax, p.m0, fpm=fpm, handle=h)
    torch.cuda.synchronize()
    assert r["info"] == 0, gbf.last_error()
    M = r["M"]
    assert M == 200
    E = r["E"][:M]
    X = r["X"][:, :M]
    rel = gpu_residuals(A, B, X, E, torch)
    assert rel.max() < TOL_R
    G = X.t() @ (B @ X)
    assert (G - torch.eye(M, dtype=G.dtype, device=G.device)).abs().max().item() < 1e-10
    with open(GOLD) as f:
        gold = json.load(f)
    assert gold["M"] == M and gold["sylvester_count"] == M
    assert compare_eigs(E.cpu().numpy(), np.array(gold["E"]), p.emin, p.emax) < TOL_E
    h.close()


@pytest.mark.parametrize("prec", [1, 0])
def test_complex_hermitian_8192(gbf, prec):
    import torch

    p = W.dense_complex_hermitian()
    A = gbf.fortran(torch.from_numpy(np.ascontiguousarray(p.A)).cuda())
    fpm = p.apply_fpm(gbf.gbf_init())
    fpm[41] = prec
    h = gbf.Handle()
    r = gbf.feast_dev(A, None, p.emin, p.emax, p.m0, fpm=fpm, handle=h)
    torch.cuda.synchronize()
    assert r["info"] == 0, gbf.last_error()
    lam = p.spectrum
    ref = lam[(lam >= p.emin) & (lam <= p.emax)]
    M = r["M"]
    assert M == len(ref)
    E = r["E"][:M]
    assert compare_eigs(E.cpu().numpy(), ref, p.emin, p.emax) < TOL_E
    rel = gpu_residuals(A, None, r["X"][:, :M], E.to(torch.complex128), torch)
    assert rel.max() < TOL_R
    h.close()
