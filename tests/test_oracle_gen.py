"""Pins for the non-Hermitian FEAST oracle (oracle/feast_gen.py).

The guide prints neither the full-contour quadrature nor the dual-subspace
iteration; these tests pin the oracle against facts fixed by mathematics:
the closed form of the trapezoidal filter on a circle, the Hermitian
half-contour rule it must reduce to on the real axis, the exact spectral
projectors of a matrix with a known eigendecomposition, brute-force
eigenvalues, and the bi-orthonormality and residual definitions of Table
tab_common."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from oracle import feast_gen as G
from paper_1203_4031_gb300 import workloads as W


# ------------------------------------------------------------ contour --
@pytest.mark.parametrize("qtype", [0, 1])
@pytest.mark.parametrize("ratio,angle", [(100, 0), (50, 0), (30, 40), (180, -120)])
def test_nodes_on_the_ellipse(qtype, ratio, angle):
    emid, r = 0.3 - 0.2j, 1.7
    z, w = G.gcontour(emid, r, 12, qtype, ratio, angle)
    u = (z - emid) * np.exp(-1j * np.deg2rad(angle)) / r
    assert np.allclose(u.real ** 2 + (u.imag / (ratio / 100)) ** 2, 1.0, atol=1e-14)
    # weights are the tangent (z' / i) times the angle rule's weight / 2
    z0, _ = G.gcontour(0.0, 1.0, 12, qtype, 100, 0)
    t = np.angle(z0) % (2 * np.pi)
    tang = r * np.exp(1j * np.deg2rad(angle)) * (ratio / 100 * np.cos(t) + 1j * np.sin(t))
    om = np.polynomial.legendre.leggauss(12)[1] if qtype == 0 else np.full(12, 2 / 12)
    assert np.allclose(w, 0.5 * om * tang, atol=1e-14)


@pytest.mark.parametrize("ne", [2, 3, 8, 16, 17])
def test_trapezoid_circle_closed_form(ne):
    """Trapezoidal points on a circle are the roots of u^N = -1, for which
    (1/N) sum u_e / (u_e - u) = 1 / (1 + u^N) exactly."""
    emid, r = -0.4 + 0.25j, 0.8
    z, w = G.gcontour(emid, r, ne, 1)
    lam = emid + r * np.array([0.0, 0.3 + 0.2j, -0.7j, 0.95, 1.05j, 1.3 - 0.4j, 2.5, -4 + 3j])
    u = (lam - emid) / r
    assert np.allclose(G.grationalx(z, w, lam), 1.0 / (1.0 + u ** ne), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("k", [2, 4, 8])
@pytest.mark.parametrize("ratio", [100, 40])
def test_real_axis_matches_hermitian_half_contour(k, ratio):
    """For a real centre, the trapezoidal full contour with 2k points holds
    the Hermitian half contour's k points and their mirror images, so its
    filter on the real axis equals the Hermitian rational function."""
    emin, emax = -0.5, 1.5
    z, w = G.gcontour(0.5 * (emin + emax), 0.5 * (emax - emin), 2 * k, 1, ratio, 0)
    lam = np.linspace(-2.0, 3.0, 41)
    f_full = G.grationalx(z, w, lam)
    f_half = oracle.rational(emin, emax, k, lam, qtype=1, ratio=ratio)
    assert np.allclose(f_full.imag, 0.0, atol=1e-14)
    assert np.allclose(f_full.real, f_half, atol=1e-14)


@pytest.mark.parametrize("qtype", [0, 1])
def test_conjugate_symmetry_and_centre(qtype):
    z, w = G.gcontour(0.25, 2.0, 10, qtype)
    assert np.allclose(z[::-1], np.conj(z), atol=1e-15)
    assert np.allclose(w[::-1], np.conj(w), atol=1e-15)
    assert np.all(z[:5].imag > 0)
    # f(Emid) = sum omega / 2 = 1 on a circle
    assert abs(G.grationalx(z, w, [0.25])[0] - 1.0) < 1e-14


@pytest.mark.parametrize("qtype", [0, 1])
def test_filter_tends_to_indicator(qtype):
    emid, r = 1.0 + 1.0j, 0.5
    z, w = G.gcontour(emid, r, 64, qtype, 60, 30)
    rng = np.random.default_rng(5)
    pts = emid + 1.2 * r * (rng.uniform(-1, 1, 400) + 1j * rng.uniform(-1, 1, 400))
    ins = G.inside(pts, emid, r, 60, 30)
    u = (pts - emid) * np.exp(-1j * np.deg2rad(30)) / r
    d = np.sqrt(u.real ** 2 + (u.imag / 0.6) ** 2)
    far = np.abs(d - 1.0) > 0.45
    f = G.grationalx(z, w, pts)
    assert np.all(np.abs(f[ins & far] - 1.0) < 1e-4)
    assert np.all(np.abs(f[~ins & far]) < 1e-4)


# --------------------------------------------------- one contour (Q) --
@pytest.mark.parametrize("qtype", [0, 1])
def test_first_subspaces_are_the_filtered_projectors(qtype):
    """fpm(14)=1 returns Q and Q^ after one contour.  With A = S D S^{-1}
    known exactly: Q = S f(D) S^{-1} Y and Q^ = S^{-H} conj(f(D)) S^H Y."""
    n, m0 = 60, 8
    rng = np.random.default_rng(1)
    S = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 4 * np.eye(n)
    d = rng.uniform(-1, 1, n) + 1j * rng.uniform(-1, 1, n)
    A = S @ np.diag(d) @ np.linalg.inv(S)
    fpm = G.feastinit_gen()
    fpm[13] = 1
    fpm[16] = qtype
    fpm[7] = 12
    emid, r = 0.1 + 0.1j, 0.6
    o = G.feast_gen(A, None, emid, r, m0, fpm)
    assert o["info"] == 4
    z, w = G.gcontour(emid, r, 12, qtype)
    f = G.grationalx(z, w, d)
    Y = G.initial_subspace(n, m0)
    Si = np.linalg.inv(S)
    Q = S @ (f[:, None] * (Si @ Y))
    Qh = Si.conj().T @ (np.conj(f)[:, None] * (S.conj().T @ Y))
    assert np.allclose(o["X"][:, :m0], Q, atol=1e-10 * np.abs(Q).max())
    assert np.allclose(o["X"][:, m0:], Qh, atol=1e-10 * np.abs(Qh).max())


# --------------------------------------------------- full iteration --
def _check_known(P, o, tol=1e-11):
    m0 = P.m0
    M = o["M"]
    assert o["info"] == 0, o["info"]
    assert M == P.count
    exact = P.spectrum[G.inside(P.spectrum, P.emid, P.r)]
    got = o["E"][:M]
    for lam in exact:       # every exact eigenvalue inside is found once
        assert np.min(np.abs(got - lam)) < tol
    assert np.max(o["res"][:M]) < 1e-10 and np.max(o["res"][m0:m0 + M]) < 1e-10
    assert o["biorth"] < 1e-12
    # inside ones first, in ascending (Re, Im)
    key = np.lexsort((got.imag, got.real))
    assert np.all(key == np.arange(M))
    # the residual definition of Table tab_common, recomputed
    A = P.A.astype(np.complex128)
    B = np.eye(P.n) if P.B is None else P.B.astype(np.complex128)
    X, Xh = o["X"][:, :M], o["X"][:, m0:m0 + M]
    alpha = abs(P.emid) + P.r
    rr = np.sum(np.abs(A @ X - (B @ X) * got), axis=0) / np.sum(np.abs(alpha * (B @ X)), axis=0)
    rl = (np.sum(np.abs(A.conj().T @ Xh - (B.conj().T @ Xh) * got.conj()), axis=0)
          / np.sum(np.abs(alpha * (B.conj().T @ Xh)), axis=0))
    assert np.allclose(rr, o["res"][:M], rtol=1e-3, atol=1e-14)
    assert np.allclose(rl, o["res"][m0:m0 + M], rtol=1e-3, atol=1e-14)
    assert np.allclose(Xh.conj().T @ B @ X, np.eye(M), atol=1e-11)
    assert np.allclose(np.linalg.norm(X, axis=0), 1.0, atol=1e-13)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("gen", [False, True])
def test_known_spectrum(cplx, gen):
    P = W.dense_nonsymmetric(160, count=9, m0=14, complex_=cplx, generalized=gen)
    fpm = P.apply_fpm(G.feastinit_gen())
    _check_known(P, G.feast_gen(P.A, P.B, P.emid, P.r, P.m0, fpm))


def test_real_problem_conjugate_pairs():
    P = W.dense_nonsymmetric(160, count=12, m0=18, emid=0.2 + 0.0j, seed=77)
    o = G.feast_gen(P.A, P.B, P.emid, P.r, P.m0, P.apply_fpm(G.feastinit_gen()))
    E = o["E"][:o["M"]]
    for lam in E[np.abs(E.imag) > 1e-8]:
        assert np.min(np.abs(E - np.conj(lam))) < 1e-12


@pytest.mark.parametrize("crit", [0, 1])
@pytest.mark.parametrize("qtype", [0, 1])
def test_brute_force_random_dense(crit, qtype):
    """A random complex matrix (no structure): the eigenvalues inside a
    circle match the library's dense eigenvalues."""
    n = 48
    rng = np.random.default_rng(3)
    A = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    lam = np.linalg.eigvals(A)
    emid = 0.1 - 0.05j
    dist = np.sort(np.abs(lam - emid))
    r = 0.5 * (dist[5] + dist[6])
    fpm = G.feastinit_gen()
    fpm[5] = crit
    fpm[16] = qtype
    fpm[7] = 24
    o = G.feast_gen(A, None, emid, r, 12, fpm)
    assert o["info"] == 0 and o["M"] == 6
    for l in lam[np.abs(lam - emid) < r]:
        assert np.min(np.abs(o["E"][:6] - l)) < 1e-11


def test_info_no_eigenvalue_and_small_subspace():
    P = W.dense_nonsymmetric(100, count=8, m0=12, complex_=True)
    fpm = P.apply_fpm(G.feastinit_gen())
    o = G.feast_gen(P.A, None, 5.0 + 5.0j, 0.5, 8, fpm)
    assert o["info"] == 1 and o["M"] == 0
    o = G.feast_gen(P.A, None, P.emid, P.r, 5, fpm)
    assert o["info"] == 3


def test_initial_subspace_is_the_hermitian_oracles():
    """Same SplitMix64 entries as the C oracle's complex initial subspace."""
    Y = G.initial_subspace(5, 3)
    u = lambda k: (oracle.splitmix64(G.SUBSPACE_SEED, k) >> 11) * (2.0 / 9007199254740992.0) - 1.0
    for j in range(3):
        for i in range(5):
            t = i + 5 * j
            assert Y[i, j] == complex(u(2 * t), u(2 * t + 1))


@pytest.mark.parametrize("gen", [False, True])
def test_hermitian_pencil_matches_hermitian_oracle(gen):
    """On a Hermitian A (and Hermitian positive definite B) every eigenvalue
    is real, so the non-Hermitian iteration on a circle centred on the real
    axis must find exactly the Hermitian oracle's eigenvalues in the
    diameter's interval, with right and left vectors alike."""
    n = 90
    rng = np.random.default_rng(11)
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = 0.5 * (X + X.conj().T) / np.sqrt(n)
    B = None
    if gen:
        Y = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        B = np.eye(n) + 0.05 * (Y @ Y.conj().T) / n
    w = sla.eigvalsh(A, B)
    emid = 0.05
    d = np.sort(np.abs(w - emid))
    r = 0.5 * (d[7] + d[8])
    ref = oracle.feast(A, B, emid - r, emid + r, 12, hermitian=True)
    assert ref["info"] == 0 and ref["M"] == 8
    fpm = G.feastinit_gen()
    fpm[7] = 24
    # M0 = 14: the sparse real spectrum leaves most of the 6 extra columns
    # with filter values at rounding level; the numerical-range cut keeps
    # the pencil regular (m0 returned below 14)
    o = G.feast_gen(A, B, emid, r, 14, fpm)
    assert o["info"] == 0 and o["M"] == 8 and 8 <= o["m0"] <= 14
    E = o["E"][:8]
    assert np.max(np.abs(E.imag)) < 1e-12
    assert np.max(np.abs(np.sort(E.real) - ref["E"][:8])) < 1e-12
    # a Hermitian pencil's left eigenvectors are its right ones: x^_j is a
    # multiple of x_j (distinct eigenvalues)
    Xr, Xl = o["X"][:, :8], o["X"][:, 14:22]
    for j in range(8):
        x, y = Xr[:, j], Xl[:, j]
        cosang = abs(np.vdot(x, y)) / (np.linalg.norm(x) * np.linalg.norm(y))
        assert abs(cosang - 1.0) < 1e-9


@pytest.mark.parametrize("cplx", [False, True])
def test_large_subspace_keeps_the_pencil_regular(cplx):
    """M0 = 16 for 6 eigenvalues inside: without the numerical-range cut the
    reduced pencil turns singular (non-finite Ritz values); with it the
    iteration converges to the known eigenvalues."""
    P = W.dense_nonsymmetric(300, count=6, m0=16, complex_=cplx, generalized=True, seed=13)
    o = G.feast_gen(P.A, P.B, P.emid, P.r, P.m0, P.apply_fpm(G.feastinit_gen()))
    assert o["info"] == 0 and o["M"] == 6
    for lam in P.spectrum[G.inside(P.spectrum, P.emid, P.r)]:
        assert np.min(np.abs(o["E"][:6] - lam)) < 1e-12
    assert np.max(o["res"][:6]) < 1e-10 and np.max(o["res"][16:22]) < 1e-10


def test_range_basis_is_orthonormal_and_drops_noise():
    rng = np.random.default_rng(2)
    U = np.linalg.qr(rng.standard_normal((50, 5)) + 1j * rng.standard_normal((50, 5)))[0]
    M = U @ np.diag([3.0, 1.0, 0.5, 1e-3, 2.0]) @ (rng.standard_normal((5, 8)))
    M[:, 7] += 1e-9 * rng.standard_normal(50)       # a direction far below the Gram's resolution
    Bq, k = G._range_basis(M)
    assert k == 5
    assert np.allclose(Bq.conj().T @ Bq, np.eye(5), atol=1e-10)
    assert np.allclose(Bq @ (Bq.conj().T @ U), U, atol=1e-8)


@pytest.mark.parametrize("delta", [1e-5, 1e-6])
def test_nearly_defective_pair_is_kept(delta):
    """A 2 x 2 block [[0, 1], [0, delta]] inside the circle: its two
    eigenvectors are nearly parallel (angle ~ delta), so the filtered
    subspace has a direction with a tiny Gram eigenvalue (~delta^2) that
    belongs to the wanted span; the numerical-range cut must keep it."""
    rng = np.random.default_rng(7)
    n = 60
    T = np.diag(rng.uniform(1.0, 3.0, n)).astype(complex)
    T[0, 0], T[1, 1], T[0, 1] = 0.0, delta, 1.0
    U = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))[0]
    A = U @ T @ U.conj().T
    fpm = G.feastinit_gen()
    o = G.feast_gen(A, None, 0.0, 0.5, 4, fpm)
    assert o["info"] == 0 and o["M"] == 2 and o["m0"] == 4
    assert np.min(np.abs(o["E"][:2])) < 1e-9 and np.min(np.abs(o["E"][:2] - delta)) < 1e-9
