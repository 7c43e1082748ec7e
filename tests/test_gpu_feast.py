"""GPU parity of the whole hot path (all rows a1..a10) through the C ABI
against the oracle on the same seeded inputs: the guide's hello world, the
Laplacian workload (n=500, closed-form spectrum), brute-force small problems
of every kind, the filtered subspace after one contour, the info codes and
the storage / entry-point variants.  FP64 path (fpm(42)=0) and mixed path
(fpm(42)=1) both."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_1203_4031_gb300 import workloads as W

from feast_check import (TOL_E, TOL_R, alpha, b_orth_error, compare_eigs, residuals,
                         vector_alignment)

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def fpm_for(g, prec, overrides=None):
    f = g.gbf_init()
    f[41] = prec
    for k, v in (overrides or {}).items():
        f[k - 1] = v
    return f


@pytest.mark.parametrize("prec", [0, 1])
def test_hello_world(gbf, prec):
    gold = json.load(open(os.path.join(GOLD, "helloworld.json")))
    A = np.array(gold["A"])
    r = gbf.feast_host(A, None, gold["emin"], gold["emax"], gold["M0"], fpm=fpm_for(gbf, prec))
    e = gold["expected"]
    assert r["info"] == 0 and r["M"] == 2 and r["loop"] == 0 and r["epsout"] == 1.0
    assert np.allclose(r["E"], e["E"], atol=1e-14)
    assert np.max(r["res"]) < 1e-14
    assert np.allclose(np.abs(r["X"]), e["X_abs"], atol=1e-14)
    assert np.sign(r["X"][0, 0]) == np.sign(r["X"][1, 0])
    assert np.sign(r["X"][0, 1]) != np.sign(r["X"][1, 1])


@pytest.mark.parametrize("prec", [0, 1])
def test_laplacian_n500(gbf, prec):
    p = W.laplacian()
    fpm = p.apply_fpm(fpm_for(gbf, prec))
    r = gbf.feast_host(p.A, None, p.emin, p.emax, p.m0, fpm=fpm)
    assert r["info"] == 0, gbf.last_error()
    M = r["M"]
    assert M in (51, 52)
    lam = p.spectrum
    ref = lam[(lam >= p.emin - 1e-12) & (lam <= p.emax + 1e-12)][:M]
    assert compare_eigs(r["E"][:M], ref, p.emin, p.emax) < TOL_E
    X = r["X"][:, :M]
    assert np.max(residuals(p.A, None, X, r["E"][:M])) < TOL_R
    assert b_orth_error(None, X) < 1e-12
    fo = p.apply_fpm(oracle.feastinit())
    o = oracle.feast(p.A, None, p.emin, p.emax, p.m0, fpm=fo)
    # lambda_167 = 1 + 2e-16 lies on Emax: it may be counted on either side
    Mc = min(M, o["M"])
    assert abs(M - o["M"]) <= 1
    if M != o["M"]:
        extra = (r["E"][Mc] if M > Mc else o["E"][Mc])
        assert abs(extra - p.emax) < 1e-12 * p.emax
    assert compare_eigs(r["E"][:Mc], o["E"][:Mc], p.emin, p.emax) < TOL_E
    # the boundary eigenvalue may also be counted in one loop and out in the
    # next, and the trace test then waits for two loops with equal counts:
    # only the loop limit binds here (loop counts are compared on an interval
    # with no eigenvalue near its ends, below)
    assert 1 <= r["loop"] <= fpm[3]
    assert vector_alignment(None, X[:, :Mc], o["X"][:, :Mc], o["E"][:Mc]) > 1 - 1e-9


@pytest.mark.parametrize("prec", [0, 1])
def test_laplacian_n500_interior(gbf, prec):
    """[0.5, 0.999]: 51 eigenvalues, none within 1e-3 of either end."""
    p = W.laplacian(emax=0.999)
    fpm = p.apply_fpm(fpm_for(gbf, prec))
    r = gbf.feast_host(p.A, None, p.emin, p.emax, p.m0, fpm=fpm)
    assert r["info"] == 0, gbf.last_error()
    lam = p.spectrum
    ref = lam[(lam >= p.emin) & (lam <= p.emax)]
    assert r["M"] == len(ref) == 51
    X = r["X"][:, :51]
    assert compare_eigs(r["E"][:51], ref, p.emin, p.emax) < TOL_E
    assert np.max(residuals(p.A, None, X, r["E"][:51])) < TOL_R
    o = oracle.feast(p.A, None, p.emin, p.emax, p.m0, fpm=p.apply_fpm(oracle.feastinit()))
    assert o["M"] == 51
    assert compare_eigs(r["E"][:51], o["E"][:51], p.emin, p.emax) < TOL_E
    if prec == 0:   # trace-criterion stops may differ by one loop with rounding order
        assert abs(r["loop"] - o["loop"]) <= 1
    assert vector_alignment(None, X, o["X"][:, :51], o["E"][:51]) > 1 - 1e-9


def small_problem(herm, gen, n, count, seed):
    r = np.random.default_rng(seed)
    M = r.standard_normal((n, n)) + (1j * r.standard_normal((n, n)) if herm else 0)
    A = 0.5 * (M + M.conj().T)
    B = None
    if gen:
        G = r.standard_normal((n, n)) + (1j * r.standard_normal((n, n)) if herm else 0)
        B = G @ G.conj().T / n + np.eye(n)
    w = sl.eigh(A, B, eigvals_only=True)
    mid = n // 2
    emin = 0.5 * (w[mid - 1] + w[mid])
    emax = 0.5 * (w[mid - 1 + count] + w[mid + count])
    return A, B, emin, emax, w


CASES = [(False, False, 40, 8, 14), (False, True, 97, 12, 20), (True, False, 65, 9, 16),
         (True, True, 130, 15, 24), (False, True, 300, 30, 45), (True, True, 257, 20, 32)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("herm,gen,n,count,m0", CASES)
def test_small_problems_vs_oracle(gbf, prec, herm, gen, n, count, m0):
    A, B, emin, emax, w = small_problem(herm, gen, n, count, seed=n)
    r = gbf.feast_host(A, B, emin, emax, m0, fpm=fpm_for(gbf, prec, {3: 12}), hermitian=herm)
    assert r["info"] == 0, (r["info"], gbf.last_error())
    o = oracle.feast(A, B, emin, emax, m0, fpm=oracle.feastinit(), hermitian=herm)
    assert r["M"] == o["M"] == count
    assert compare_eigs(r["E"][:count], o["E"][:count], emin, emax) < TOL_E
    ref = w[(w >= emin) & (w <= emax)]
    assert compare_eigs(r["E"][:count], ref, emin, emax) < TOL_E
    X = r["X"][:, :count]
    assert np.max(residuals(A, B, X, r["E"][:count])) < TOL_R
    assert b_orth_error(B, X) < 1e-11
    assert vector_alignment(B, X, o["X"][:, :count], o["E"][:count]) > 1 - 1e-8
    if prec == 0:
        assert r["loop"] == o["loop"]


@pytest.mark.parametrize("herm,gen", [(False, False), (False, True), (True, False), (True, True)])
def test_subspace_after_one_contour(gbf, herm, gen):
    """fpm(14)=1 with a given subspace (fpm(5)=1): Q element by element."""
    n, m0 = 70, 9
    A, B, emin, emax, _ = small_problem(herm, gen, n, 5, seed=3 + 2 * herm + gen)
    r0 = np.random.default_rng(11)
    Y = r0.standard_normal((n, m0)) + (1j * r0.standard_normal((n, m0)) if herm else 0)
    f = fpm_for(gbf, 0, {5: 1, 14: 1})
    r = gbf.feast_host(A, B, emin, emax, m0, fpm=f, X0=Y, hermitian=herm)
    assert r["info"] == 4
    fo = oracle.feastinit()
    fo[4] = 1
    fo[13] = 1
    o = oracle.feast(A, B, emin, emax, m0, fpm=fo, X0=Y, hermitian=herm)
    assert o["info"] == 4
    scale = np.abs(o["X"]).max()
    assert np.max(np.abs(r["X"] - o["X"])) < 1e-11 * scale


def test_info_codes_on_gpu(gbf):
    A = np.diag(np.arange(1.0, 11.0))
    assert gbf.feast_host(A, None, 3.2, 3.8, 3)["info"] == 1
    assert gbf.feast_host(A, None, 0.5, 5.5, 3)["info"] == 3
    f = fpm_for(gbf, 0, {4: 0, 6: 0})
    assert gbf.feast_host(A, None, 0.5, 3.5, 5, fpm=f)["info"] == 2
    f = fpm_for(gbf, 0, {14: 1})
    r = gbf.feast_host(A, None, 0.5, 3.5, 5, fpm=f)
    assert r["info"] == 4 and r["loop"] == 0
    Aneg = np.diag(np.r_[1.0, 2.0, -3.0, np.arange(4.0, 11.0)])
    Bbad = np.diag(np.r_[1.0, 1.0, -1.0, np.ones(7)])
    assert gbf.feast_host(Aneg, Bbad, 0.5, 3.5, 6)["info"] == -3
    # non-finite entries: the inner solver reports -2 (Table tab_info)
    for bad in (np.nan, np.inf, -np.inf):
        An = A.copy()
        An[2, 6] = An[6, 2] = bad
        assert gbf.feast_host(An, None, 0.5, 3.5, 5)["info"] == -2
        Bn = np.eye(10)
        Bn[3, 3] = bad
        for prec in (0, 1):
            assert gbf.feast_host(A, Bn, 0.5, 3.5, 5, fpm=fpm_for(gbf, prec))["info"] == -2


@pytest.mark.parametrize("uplo", ["L", "U"])
def test_uplo_storage(gbf, uplo):
    A, B, emin, emax, _ = small_problem(True, True, 60, 6, seed=21)
    rf = gbf.feast_host(A, B, emin, emax, 12)
    tri = np.tril if uplo == "L" else np.triu
    mask = tri(np.ones_like(A, dtype=bool))
    r = gbf.feast_host(np.where(mask, A, 5 + 5j), np.where(mask, B, -2 - 1j), emin, emax, 12, uplo=uplo)
    assert r["info"] == 0 and r["M"] == rf["M"] == 6
    assert compare_eigs(r["E"][:6], rf["E"][:6], emin, emax) < 1e-13


def test_device_entry_matches_host_entry(gbf):
    import torch

    A, B, emin, emax, _ = small_problem(False, True, 150, 10, seed=5)
    rh = gbf.feast_host(A, B, emin, emax, 16)
    h = gbf.Handle()
    At = gbf.fortran(torch.from_numpy(A).cuda())
    Bt = gbf.fortran(torch.from_numpy(B).cuda())
    rd = gbf.feast_dev(At, Bt, emin, emax, 16, handle=h)
    torch.cuda.synchronize()
    assert rd["info"] == rh["info"] == 0 and rd["M"] == rh["M"] and rd["loop"] == rh["loop"]
    assert np.array_equal(rd["E"].cpu().numpy(), rh["E"])
    assert np.array_equal(rd["X"].cpu().numpy(), rh["X"])
    h.close()


def test_expert_nodes_match_default(gbf):
    A, B, emin, emax, _ = small_problem(True, False, 80, 7, seed=8)
    z, w = gbf.gbf_contour(emin, emax, 8)
    r1 = gbf.feast_host(A, B, emin, emax, 12)
    r2 = gbf.feast_host(A, B, emin, emax, 12, Zne=z, Wne=w)
    assert r2["info"] == 0 and np.array_equal(r1["E"], r2["E"])


def test_trapezoid_and_ellipse(gbf):
    A, B, emin, emax, w = small_problem(False, True, 90, 8, seed=12)
    for over in ({16: 1, 2: 10}, {18: 60}):
        r = gbf.feast_host(A, B, emin, emax, 14, fpm=fpm_for(gbf, 0, over))
        o = oracle.feast(A, B, emin, emax, 14, fpm=W.Problem("x", False, A, B, emin, emax, 14,
                                                              fpm=over).apply_fpm(oracle.feastinit()))
        assert r["info"] == o["info"] == 0
        assert compare_eigs(r["E"][:8], o["E"][:8], emin, emax) < TOL_E


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,count", [(300, 15), (800, 40)])
def test_spurious_cases_vs_oracle(gbf, prec, n, count):
    """Dense generalized spectrum around a symmetric interval: spurious inside
    Ritz pairs must be flagged (res = -1, at the end) on both sides alike."""
    p = W.dense_real_generalized(n=n, count=count, m0=int(1.5 * count))
    r = gbf.feast_host(p.A, p.B, p.emin, p.emax, p.m0, fpm=p.apply_fpm(fpm_for(gbf, prec)))
    o = oracle.feast(p.A, p.B, p.emin, p.emax, p.m0, fpm=p.apply_fpm(oracle.feastinit()), hermitian=False)
    assert r["info"] == o["info"] == 0
    assert r["M"] == o["M"] == count
    assert compare_eigs(r["E"][:count], o["E"][:count], p.emin, p.emax) < TOL_E
    X = r["X"][:, :count]
    assert np.max(residuals(p.A, p.B, X, r["E"][:count])) < TOL_R
    if prec == 0:
        assert r["loop"] == o["loop"]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("herm,gen,n,count,m0", [(False, True, 300, 30, 45), (True, True, 257, 20, 32)])
def test_cuda_core_engine_vs_oracle(gbf, prec, herm, gen, n, count, m0):
    """fpm(44)=1: complex GEMMs of factor/solve on CUDA cores instead of the
    sliced tensor-core engine; same parity bar."""
    A, B, emin, emax, w = small_problem(herm, gen, n, count, seed=n)
    r = gbf.feast_host(A, B, emin, emax, m0, fpm=fpm_for(gbf, prec, {3: 12, 44: 1}), hermitian=herm)
    assert r["info"] == 0, (r["info"], gbf.last_error())
    o = oracle.feast(A, B, emin, emax, m0, fpm=oracle.feastinit(), hermitian=herm)
    assert r["M"] == o["M"] == count
    assert compare_eigs(r["E"][:count], o["E"][:count], emin, emax) < TOL_E
    assert np.max(residuals(A, B, r["X"][:, :count], r["E"][:count])) < TOL_R
