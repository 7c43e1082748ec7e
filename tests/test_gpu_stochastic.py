"""GPU parity of the stochastic eigenvalue count (fpm(14)=2, the guide's
"Stochastic estimate" section) through the C ABI against the oracle on the
same seeded inputs: generated probes bit-exact, the running mean res(1:M0)
element by element, M; FP64 and mixed (fpm(42)=1) paths, all four problem
kinds, ragged sizes, one probe.  At the n=4096 generalized benchmark size
(device-pointer driver, as the benchmark times it) every probe's quadratic
form is checked against the spectral theorem: y^T f(B^-1 A) y =
sum_i f(lambda_i) (v_i^T B y)(v_i^T y) for the B-orthonormal eigenvectors
v_i, with f the quadrature's rational function."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_1203_4031_gb300 import workloads as W

from feast_check import gapped_pencil, rademacher

pytestmark = pytest.mark.gpu

# (herm, gen, n, inside, m0, ne, prec)
CASES = [
    (False, False, 333, 12, 37, 8, 0),
    (False, True, 300, 9, 24, 3, 1),
    (True, False, 257, 10, 19, 8, 0),
    (True, True, 200, 7, 16, 8, 1),
    (False, True, 1000, 30, 64, 8, 0),
    (True, True, 640, 20, 40, 4, 0),
    (False, True, 65, 4, 1, 8, 0),
    (True, False, 16, 2, 3, 8, 1),
]


def _fpm(f, ne, prec, user=False):
    f[1] = ne
    f[13] = 2
    f[41] = prec
    if user:
        f[4] = 1
    return f


@pytest.mark.parametrize("herm,gen,n,inside,m0,ne,prec", CASES)
def test_stochastic_count_matches_oracle(gbf, herm, gen, n, inside, m0, ne, prec):
    A, B, V, lam = gapped_pencil(n, inside, herm, gen, seed=1000 + n + 7 * herm + gen)
    r = gbf.feast_host(A, B, -1.0, 1.0, m0, fpm=_fpm(gbf.gbf_init(), ne, prec), hermitian=herm)
    ref = oracle.feast(A, B, -1.0, 1.0, m0, fpm=_fpm(oracle.feastinit(), ne, 0), hermitian=herm)
    assert r["info"] == 5 == ref["info"], gbf.last_error()
    assert r["loop"] == 0
    assert np.array_equal(r["X"], ref["X"])                 # the probes, bit for bit
    assert np.array_equal(np.real(r["X"]), rademacher(n, m0))
    assert not np.any(r["E"])
    # FP64: Q to rounding; mixed: the first contour runs on FP32 factors
    tol = (1e-9 if prec == 0 else 5e-3) * (1.0 + np.abs(ref["res"]).max())
    assert np.max(np.abs(r["res"] - ref["res"])) <= tol
    if abs(ref["res"][-1] - np.floor(ref["res"][-1]) - 0.5) > tol:
        assert r["M"] == ref["M"]


@pytest.mark.parametrize("herm", [False, True])
def test_stochastic_count_with_caller_probes(gbf, herm):
    """fpm(5)=1: the caller's X are the probes (complex unit-modulus ones for
    the Hermitian kind, so the conjugate in y^H q matters)."""
    n, m0 = 180, 12
    A, B, V, lam = gapped_pencil(n, 8, herm, True, seed=55 + herm)
    g = np.random.default_rng(8)
    Y = np.exp(2j * np.pi * g.uniform(size=(n, m0))) if herm else np.sign(g.standard_normal((n, m0)))
    r = gbf.feast_host(A, B, -1.0, 1.0, m0, fpm=_fpm(gbf.gbf_init(), 8, 0, True), X0=Y, hermitian=herm)
    ref = oracle.feast(A, B, -1.0, 1.0, m0, fpm=_fpm(oracle.feastinit(), 8, 0, True), X0=Y, hermitian=herm)
    assert r["info"] == 5 == ref["info"], gbf.last_error()
    assert np.array_equal(r["X"], Y)
    assert np.max(np.abs(r["res"] - ref["res"])) <= 1e-9 * (1.0 + np.abs(ref["res"]).max())
    assert r["M"] == ref["M"]


def test_stochastic_count_real_generalized_4096(gbf):
    """Benchmark size, device pointers, 3 nodes (the guide's suggestion for
    the estimate), 64 probes, FP64 factors so the forms hold to rounding."""
    import torch

    p = W.dense_real_generalized()
    n, m0, ne = p.A.shape[0], 64, 3
    A = gbf.fortran(torch.from_numpy(np.ascontiguousarray(p.A)).cuda())
    B = gbf.fortran(torch.from_numpy(np.ascontiguousarray(p.B)).cuda())
    h = gbf.Handle()
    r = gbf.feast_dev(A, B, p.emin, p.emax, m0, fpm=_fpm(gbf.gbf_init(), ne, 0), handle=h)
    torch.cuda.synchronize()
    h.close()
    assert r["info"] == 5, gbf.last_error()
    Y = r["X"].cpu().numpy()
    assert np.array_equal(Y, rademacher(n, m0))
    res = r["res"].cpu().numpy()
    t = res * np.arange(1, m0 + 1) - np.r_[0.0, res[:-1] * np.arange(1, m0)]
    lam, V = sl.eigh(p.A, p.B)
    f = oracle.rational(p.emin, p.emax, ne, lam)
    expect = np.einsum("i,ij,ij->j", f, V.T @ (p.B @ Y), V.T @ Y)
    assert np.max(np.abs(t - expect)) <= 1e-7 * (1.0 + np.abs(expect).max())
    assert r["M"] == max(0, int(np.floor(res[-1] + 0.5)))
