"""Pins for the oracle FEAST driver: the guide's hello-world output, closed
form spectra, brute-force eigendecompositions on small problems, the
filtered subspace Q against its spectral definition, Sylvester counts and
the info codes of Table tab_info."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_1203_4031_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def run(p, **kw):
    fpm = p.apply_fpm(oracle.feastinit())
    for k, v in kw.pop("fpm", {}).items():
        fpm[k - 1] = v
    return oracle.feast(p.A, p.B, p.emin, p.emax, kw.pop("m0", p.m0), fpm=fpm,
                        hermitian=p.hermitian, **kw)


def test_hello_world_golden():
    g = json.load(open(os.path.join(GOLD, "helloworld.json")))
    A = np.array(g["A"])
    fpm = oracle.feastinit()
    r = oracle.feast(A, None, g["emin"], g["emax"], g["M0"], fpm=fpm)
    e = g["expected"]
    assert r["info"] == e["info"] and r["M"] == e["M"] and r["loop"] == e["loop"]
    assert r["epsout"] == e["epsout"]
    assert np.allclose(r["E"], e["E"], rtol=0, atol=1e-14)
    assert abs(np.sum(r["E"][: r["M"]]) - e["trace"]) < 1e-13
    assert np.max(r["res"][: r["M"]]) < 1e-14
    X = r["X"]
    assert np.allclose(np.abs(X), e["X_abs"], atol=1e-14)
    assert np.sign(X[0, 0]) == np.sign(X[1, 0])
    assert np.sign(X[0, 1]) != np.sign(X[1, 1])


def test_laplacian_closed_form():
    """Config: n=500 Laplacian, [0.5,1], M0=80, Ne=8, trace criterion 1e-12."""
    p = W.laplacian()
    r = run(p)
    assert r["info"] == 0
    lam = p.spectrum
    strict = lam[(lam > 0.5 + 1e-12) & (lam < 1.0 - 1e-12)]
    assert len(strict) == 51
    assert r["M"] in (51, 52)          # lambda_167 = 1 + 2e-16 sits on Emax
    E = np.sort(r["E"][: r["M"]])
    ref = lam[(lam >= 0.5 - 1e-12) & (lam <= 1.0 + 1e-12)][: r["M"]]
    assert np.max(np.abs(E - ref)) < 1e-13
    assert r["epsout"] < 1e-12 and 1 <= r["loop"] <= 20
    X = r["X"][:, : r["M"]]
    assert np.allclose(X.T @ X, np.eye(r["M"]), atol=1e-12)


CASES = [
    # (hermitian, generalized, n, interval-count, m0)
    (False, False, 40, 8, 14),
    (False, True, 48, 6, 12),
    (True, False, 37, 9, 16),
    (True, True, 64, 10, 18),
]


def small_problem(herm, gen, n, count, seed):
    r = np.random.default_rng(seed)
    M = r.standard_normal((n, n)) + (1j * r.standard_normal((n, n)) if herm else 0)
    A = np.asfortranarray(0.5 * (M + M.conj().T))
    B = None
    if gen:
        G = r.standard_normal((n, n)) + (1j * r.standard_normal((n, n)) if herm else 0)
        B = np.asfortranarray(G @ G.conj().T / n + np.eye(n))
    w = sl.eigh(A, B, eigvals_only=True)
    mid = n // 2
    emin = 0.5 * (w[mid - 1] + w[mid])
    emax = 0.5 * (w[mid - 1 + count] + w[mid + count])
    return A, B, emin, emax, w


@pytest.mark.parametrize("herm,gen,n,count,m0", CASES)
def test_bruteforce_small(herm, gen, n, count, m0):
    A, B, emin, emax, w = small_problem(herm, gen, n, count, seed=n)
    fpm = oracle.feastinit()
    r = oracle.feast(A, B, emin, emax, m0, fpm=fpm, hermitian=herm)
    assert r["info"] == 0, r
    ref = w[(w >= emin) & (w <= emax)]
    assert r["M"] == len(ref) == count
    assert np.allclose(r["E"][: r["M"]], ref, rtol=0, atol=1e-11 * np.abs(w).max())
    X = r["X"][:, : r["M"]]
    Bm = np.eye(n) if B is None else B
    assert np.allclose(X.conj().T @ Bm @ X, np.eye(count), atol=1e-11)
    R = A @ X - Bm @ X * r["E"][: r["M"]]
    assert np.max(np.linalg.norm(R, axis=0)) < 1e-9
    assert oracle.eigcount(A, B, emin, emax) == count
    # paper's residual definition, Table tab_common
    alpha = max(abs(emin), abs(emax))
    res = np.sum(np.abs(R), axis=0) / np.sum(np.abs(alpha * (Bm @ X)), axis=0)
    # both are at rounding level: agree to rounding (AX via (AQ)W vs A(QW))
    assert np.allclose(r["res"][: r["M"]], res, rtol=1e-2, atol=1e-15)


@pytest.mark.parametrize("herm,gen", [(False, False), (False, True), (True, False), (True, True)])
def test_subspace_is_filtered_projection(herm, gen):
    """fpm(14)=1 returns Q after one contour.  By the spectral theorem
    Q = V f(Lambda) V^H B Y (V B-orthonormal), f the rational filter; this
    route uses no LU and no quadrature solve."""
    n, m0 = 30, 7
    A, B, emin, emax, _ = small_problem(herm, gen, n, 4, seed=7 + 2 * herm + gen)
    r0 = np.random.default_rng(3)
    Y = r0.standard_normal((n, m0)) + (1j * r0.standard_normal((n, m0)) if herm else 0)
    fpm = oracle.feastinit()
    fpm[4] = 1   # fpm(5): user subspace
    fpm[13] = 1  # fpm(14): return Q
    r = oracle.feast(A, B, emin, emax, m0, fpm=fpm, X0=Y, hermitian=herm)
    assert r["info"] == 4
    lam, V = sl.eigh(A, B)
    Bm = np.eye(n) if B is None else B
    f = oracle.rational(emin, emax, 8, lam)
    Qref = V @ (f[:, None] * (V.conj().T @ (Bm @ Y)))
    assert np.allclose(r["X"], Qref, rtol=0, atol=1e-11 * np.abs(Qref).max())


def test_exact_subspace_converges_at_loop0():
    A, B, emin, emax, w = small_problem(False, True, 40, 5, seed=11)
    lam, V = sl.eigh(A, B)
    sel = (lam >= emin) & (lam <= emax)
    X0 = np.concatenate([V[:, sel], V[:, ~sel][:, :4]], axis=1)
    fpm = oracle.feastinit()
    fpm[4] = 1
    r = oracle.feast(A, B, emin, emax, X0.shape[1], fpm=fpm, X0=X0)
    assert r["info"] == 0 and r["loop"] == 0 and r["M"] == 5


def test_uplo_variants_agree():
    A, B, emin, emax, _ = small_problem(True, True, 24, 4, seed=5)
    rf = oracle.feast(A, B, emin, emax, 8, hermitian=True)
    for uplo, tri in (("L", np.tril), ("U", np.triu)):
        garbage = np.full_like(A, 9.0 + 9.0j)
        Ap = np.where(tri(np.ones_like(A, dtype=bool)), A, garbage)
        Bp = np.where(tri(np.ones_like(B, dtype=bool)), B, garbage)
        r = oracle.feast(Ap, Bp, emin, emax, 8, hermitian=True, uplo=uplo)
        assert r["M"] == rf["M"]
        assert np.allclose(r["E"][: r["M"]], rf["E"][: rf["M"]], atol=1e-12)


def test_info_codes():
    A = np.diag(np.arange(1.0, 11.0))
    ok = oracle.feastinit()
    assert oracle.feast(A[:0, :0], None, 0, 1, 1)["info"] == 202
    assert oracle.feast(A, None, 0, 5, 0)["info"] == 201
    assert oracle.feast(A, None, 0, 5, 11)["info"] == 201
    assert oracle.feast(A, None, 5, 5, 4)["info"] == 200
    for idx, bad, code in [(1, 21, 102), (1, 0, 102), (2, -1, 103), (3, -1, 104),
                           (4, 2, 105), (5, 3, 106), (13, 3, 114), (15, 2, 116),
                           (17, 0, 118)]:
        f = ok.copy()
        f[idx] = bad
        assert oracle.feast(A, None, 0.5, 3.5, 5, fpm=f)["info"] == code
    # trapezoidal accepts any positive node count
    f = ok.copy()
    f[15] = 1
    f[1] = 21
    assert oracle.feast(A, None, 0.5, 3.5, 5, fpm=f)["info"] == 0
    # no eigenvalue in the interval
    assert oracle.feast(A, None, 3.2, 3.8, 3)["info"] == 1
    # M0 too small: 5 eigenvalues inside, M0 = 3
    assert oracle.feast(A, None, 0.5, 5.5, 3)["info"] == 3
    # no convergence within fpm(4)=0 loops with the trace criterion
    f = ok.copy()
    f[3] = 0
    f[5] = 0
    assert oracle.feast(A, None, 0.5, 3.5, 5, fpm=f)["info"] == 2
    # B not positive definite: the pencil eigenvalue 3 = (-3)/(-1) lies in
    # the interval, its eigenvector has negative B-norm
    Aneg = np.diag(np.r_[1.0, 2.0, -3.0, np.arange(4.0, 11.0)])
    Bbad = np.diag(np.r_[1.0, 1.0, -1.0, np.ones(7)])
    assert oracle.feast(Aneg, Bbad, 0.5, 3.5, 6)["info"] == -3


def test_fpm14_stops_after_one_contour():
    A = np.diag(np.arange(1.0, 11.0))
    f = oracle.feastinit()
    f[13] = 1
    r = oracle.feast(A, None, 0.5, 3.5, 5, fpm=f)
    assert r["info"] == 4 and r["loop"] == 0


@pytest.mark.parametrize("n,count", [(300, 15), (800, 40)])
def test_spurious_ritz_pairs_leave_the_count(n, count):
    """Symmetric interval in a dense generalized spectrum: mixtures of outside
    eigenvectors from both sides produce Ritz values inside with residual ~1.
    They must not be counted (Table tab_common: spurious pairs go to the end
    with res = -1); M then equals the Sylvester count and the eigenvalues
    match a library generalized eigensolver."""
    p = W.dense_real_generalized(n=n, count=count, m0=int(1.5 * count))
    r = run(p)
    assert r["info"] == 0 and r["loop"] <= 5
    assert r["M"] == count == oracle.eigcount(p.A, p.B, p.emin, p.emax)
    w = sl.eigh(p.A, p.B, eigvals_only=True)
    ref = w[(w >= p.emin) & (w <= p.emax)]
    assert np.max(np.abs(r["E"][:count] - ref)) < 1e-12 * max(abs(p.emin), abs(p.emax))
    res = r["res"][: r["m0"]]
    flagged = np.where(res == -1.0)[0]
    if flagged.size:
        assert flagged.min() >= r["m0"] - flagged.size      # at the end
        Ef = r["E"][flagged]
        assert np.all((Ef >= p.emin) & (Ef <= p.emax))      # only inside pairs are flagged
