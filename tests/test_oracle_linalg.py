"""Pins for the oracle's dense kernels: LU with partial pivoting and its
solves (RCI cases 10/11/21), the Jacobi reduced eigensolver, the Sylvester
inertia count and SplitMix64.  Each is checked against an independent
library routine or a mathematical identity."""
import numpy as np
import pytest

import oracle
from paper_1203_4031_gb300 import workloads as W


def rand_c(n, m, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal((n, m)) + 1j * r.standard_normal((n, m))


@pytest.mark.parametrize("n", [1, 2, 7, 33, 64])
def test_zgetrf_reconstructs(n):
    S = rand_c(n, n, n)
    lu, ipiv, info = oracle.zgetrf(S)
    assert info == 0
    L = np.tril(lu, -1) + np.eye(n)
    U = np.triu(lu)
    P = np.eye(n)[list(range(n))]
    PS = S.copy()
    for k in range(n):
        PS[[k, ipiv[k]]] = PS[[ipiv[k], k]]
    assert np.allclose(L @ U, PS, atol=1e-12 * np.abs(S).max() * n)
    # partial pivoting on |re|+|im|: |l| <= cabs1(a)/|p| <= cabs1(p)/|p| <= sqrt(2)
    assert np.all(np.abs(L) <= np.sqrt(2.0) * (1 + 1e-15))
    del P


@pytest.mark.parametrize("n,m", [(1, 1), (5, 3), (40, 7), (64, 1)])
def test_zgetrs_and_adjoint(n, m):
    S = rand_c(n, n, 100 + n)
    b = rand_c(n, m, 200 + n)
    lu, ipiv, _ = oracle.zgetrf(S)
    x = oracle.zgetrs(lu, ipiv, b, trans=0)
    xh = oracle.zgetrs(lu, ipiv, b, trans=1)
    assert np.allclose(x, np.linalg.solve(S, b), rtol=1e-11, atol=1e-11)
    assert np.allclose(xh, np.linalg.solve(S.conj().T, b), rtol=1e-11, atol=1e-11)


def test_zgetrf_singular_reports_column():
    S = np.ones((3, 3), dtype=complex)
    _, _, info = oracle.zgetrf(S)
    assert info == 2


@pytest.mark.parametrize("n", [1, 2, 9, 40])
@pytest.mark.parametrize("cplx", [False, True])
def test_jacobi_matches_eigh(n, cplx):
    r = np.random.default_rng(n + 10 * cplx)
    M = r.standard_normal((n, n)) + (1j * r.standard_normal((n, n)) if cplx else 0)
    H = 0.5 * (M + M.conj().T)
    w, V, sweeps = oracle.jacobi_eigh(H)
    assert sweeps >= 0
    assert np.allclose(w, np.linalg.eigvalsh(H), atol=1e-13 * max(1, np.abs(H).max()))
    assert np.allclose(V.conj().T @ V, np.eye(n), atol=1e-13)
    assert np.allclose(H @ V, V * w, atol=1e-12)
    if not cplx:
        assert np.abs(V.imag).max() == 0.0


def test_jacobi_degenerate_and_diagonal():
    w, V, _ = oracle.jacobi_eigh(np.diag([3.0, 1.0, 2.0, 1.0]))
    assert np.allclose(w, [1, 1, 2, 3])
    H = np.ones((4, 4))   # eigenvalues 0,0,0,4
    w, V, _ = oracle.jacobi_eigh(H)
    assert np.allclose(w, [0, 0, 0, 4], atol=1e-14)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("cplx", [False, True])
def test_inertia_matches_eigvalsh(seed, cplx):
    r = np.random.default_rng(seed)
    n = 30 + seed
    M = r.standard_normal((n, n)) + (1j * r.standard_normal((n, n)) if cplx else 0)
    H = 0.5 * (M + M.conj().T)
    neg, zero = oracle.inertia_neg(H)
    assert neg == int(np.sum(np.linalg.eigvalsh(H) < 0))
    assert zero == 0


def test_inertia_two_by_two_pivots():
    # zero diagonal forces 2x2 Bunch-Kaufman pivots
    H = np.array([[0, 1, 0, 0], [1, 0, 0, 0], [0, 0, 0, 2], [0, 0, 2, 0]], dtype=float)
    assert oracle.inertia_neg(H)[0] == 2
    H = np.array([[0, 1j], [-1j, 0]])
    assert oracle.inertia_neg(H)[0] == 1


def test_sylvester_count_generalized():
    p = W.dense_real_generalized(n=120, count=10, m0=15)
    import scipy.linalg as sl

    w = sl.eigh(p.A, p.B, eigvals_only=True)
    for a, b in [(p.emin, p.emax), (-0.3, 0.1), (0.2, 0.9)]:
        assert oracle.eigcount(p.A, p.B, a, b) == int(np.sum((w >= a) & (w <= b)))


def test_splitmix64_published_sequence():
    """First outputs of SplitMix64 from state 0 (Steele, Lea & Flood 2014)."""
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [oracle.splitmix64(0, i) for i in range(3)] == expect
    assert [int(v) for v in W.splitmix64(0, np.arange(3))] == expect
