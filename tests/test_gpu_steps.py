"""GPU parity of single hot-path rows through the C ABI, against the oracle:
  a2+a3  gbf_factor_dev (S_e = z_e B - A, LU with partial pivoting, all nodes)
  a5     gbf_solve_dev (S_e^{-1} R and S_e^{-H} R from the stored factors)
  a8     gbf_heev_dev (Jacobi reduced eigensolver)
Sizes span several 32/64 tiles and ragged tails."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

ZNE = np.array([0.3 + 0.7j, -1.1 + 0.2j, 2.0 + 1.5j])


def herm(n, cplx, seed, spd=False):
    r = np.random.default_rng(seed)
    M = r.standard_normal((n, n)) + (1j * r.standard_normal((n, n)) if cplx else 0)
    if spd:
        return M @ M.conj().T / n + np.eye(n)
    return 0.5 * (M + M.conj().T)


def cuda(a):
    import torch

    import paper_1203_4031_gb300 as g

    return g.fortran(torch.from_numpy(np.ascontiguousarray(a)).cuda())


@pytest.fixture(scope="module")
def handle(gbf):
    h = gbf.Handle()
    yield h
    h.close()


@pytest.mark.parametrize("n", [1, 7, 33, 64, 65, 127, 200])
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("prec", [0, 1])
def test_factor_and_solve(gbf, handle, n, cplx, gen, prec):
    A = herm(n, cplx, seed=n)
    B = herm(n, cplx, seed=n + 1000, spd=True) if gen else None
    rc = gbf.gbf_factor_dev(handle, cuda(A), cuda(B) if gen else None, ZNE, prec=prec)
    assert rc == 0, gbf.last_error()
    r = np.random.default_rng(7)
    nrhs = 1 if n == 1 else 13
    rhs = r.standard_normal((n, nrhs)) + 1j * r.standard_normal((n, nrhs))
    Bm = np.eye(n) if B is None else B
    tol = 1e-11 if prec == 0 else 2e-4
    for trans in (0, 1):
        Y, rc = gbf.gbf_solve_dev(handle, cuda(rhs), len(ZNE), trans=trans)
        assert rc == 0, gbf.last_error()
        Y = Y.cpu().numpy()
        for e, z in enumerate(ZNE):
            S = z * Bm - A
            lu, ipiv, info = oracle.zgetrf(S)
            assert info == 0
            ref = oracle.zgetrs(lu, ipiv, rhs, trans=trans)
            got = Y[e].T
            err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
            assert err < tol, (e, trans, err)


@pytest.mark.parametrize("n", [1000, 2048])
@pytest.mark.parametrize("prec", [0, 1])
def test_factor_and_solve_large(gbf, handle, n, prec):
    """Sizes where the solves recurse with large-K products on the tensor
    cores (sliced for FP64 factors, 3xTF32 for FP32 ones), both solve
    directions, against an FP64 dense solve of the same shifted systems."""
    A = herm(n, True, seed=n)
    rc = gbf.gbf_factor_dev(handle, cuda(A), None, ZNE, prec=prec)
    assert rc == 0, gbf.last_error()
    r = np.random.default_rng(9)
    rhs = r.standard_normal((n, 40)) + 1j * r.standard_normal((n, 40))
    # backward error ||S y - r|| / (||S|| ||y||) per column: a few units of
    # the factors' rounding (FP64-class, or FP32 for prec 1) times sqrt(n)
    tol = 1e-13 if prec == 0 else 2e-6
    for trans in (0, 1):
        Y, rc = gbf.gbf_solve_dev(handle, cuda(rhs), len(ZNE), trans=trans)
        assert rc == 0, gbf.last_error()
        Y = Y.cpu().numpy()
        for e, z in enumerate(ZNE):
            S = z * np.eye(n) - A
            Sop = S.conj().T if trans else S
            y = Y[e].T
            bwd = np.linalg.norm(Sop @ y - rhs, axis=0) / (np.linalg.norm(Sop, 1) * np.linalg.norm(y, axis=0))
            assert bwd.max() < tol, (e, trans, bwd.max())


@pytest.mark.parametrize("uplo", ["L", "U"])
def test_factor_uplo(gbf, handle, uplo):
    n = 45
    A = herm(n, True, 3)
    B = herm(n, True, 4, spd=True)
    tri = np.tril if uplo == "L" else np.triu
    mask = tri(np.ones((n, n), dtype=bool))
    Ag = np.where(mask, A, 7.0 + 7.0j)
    Bg = np.where(mask, B, -3.0 + 1.0j)
    assert gbf.gbf_factor_dev(handle, cuda(Ag), cuda(Bg), ZNE, prec=0, uplo=uplo) == 0
    rhs = np.random.default_rng(1).standard_normal((n, 4)) + 0j
    Y, rc = gbf.gbf_solve_dev(handle, cuda(rhs), len(ZNE))
    Y = Y.cpu().numpy()
    for e, z in enumerate(ZNE):
        ref = np.linalg.solve(z * B - A, rhs)
        assert np.max(np.abs(Y[e].T - ref)) < 1e-11 * np.max(np.abs(ref))


def test_factor_zero_pivot_reported(gbf, handle):
    n = 16
    A = np.zeros((n, n))
    B = np.zeros((n, n))   # S_e = 0: every pivot is zero
    rc = gbf.gbf_factor_dev(handle, cuda(A), cuda(B), ZNE, prec=0)
    assert rc == -2


@pytest.mark.parametrize("m", [1, 2, 5, 16, 17, 64, 97, 300])
@pytest.mark.parametrize("cplx", [False, True])
def test_reduced_eigensolver(gbf, handle, m, cplx):
    H = herm(m, cplx, seed=m + 50)
    w, V, rc = gbf.gbf_heev_dev(handle, cuda(H))
    assert rc == 0, gbf.last_error()
    w = w.cpu().numpy()
    V = V.cpu().numpy()
    wo, Vo, _ = oracle.jacobi_eigh(H)
    scale = max(1.0, np.abs(wo).max())
    assert np.max(np.abs(w - wo)) < 1e-13 * scale * max(1, m / 16)
    assert np.max(np.abs(V.conj().T @ V - np.eye(m))) < 1e-12
    assert np.max(np.abs(H @ V - V * w)) < 1e-12 * scale * max(1, m / 16)


def test_reduced_eigensolver_degenerate(gbf, handle):
    H = np.diag([2.0, 2.0, 2.0, -1.0, 5.0])
    w, V, rc = gbf.gbf_heev_dev(handle, cuda(H))
    assert rc == 0
    assert np.allclose(w.cpu().numpy(), [-1, 2, 2, 2, 5], atol=0)
