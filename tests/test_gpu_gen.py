"""Non-Hermitian FEAST on the GPU (gbf_dgegv_dev / gbf_zgegv_dev) against the
oracle (oracle/feast_gen.py) and against pencils with a known spectrum.

Eigenvalues are unique and compared element by element (each oracle value
matched to the nearest GPU value, all within 1e-10 relative to alpha);
eigenvectors are unique only up to scale, so they are checked through what
is unique: the residuals of Table tab_common (both below the 1e-10 gate),
unit right vectors, and the bi-orthonormality X^^H B X = I of the pairs
inside."""
import numpy as np
import pytest
import torch

from oracle import feast_gen as G
from paper_1203_4031_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_E = 1e-10


def _dev(a):
    if a is None:
        return None
    t = torch.as_tensor(np.asfortranarray(a))
    return t.t().contiguous().t().cuda()


def _run(gbf, P, fpm, h, X=None):
    out = gbf.feast_gen_dev(_dev(P.A), _dev(P.B), P.emid, P.r, P.m0, fpm, X=X, handle=h)
    torch.cuda.synchronize()
    return out


def _check_outputs(P, o, fpm, exact=None):
    m0, M = P.m0, o["M"]
    E = o["E"].cpu().numpy()
    res = o["res"].cpu().numpy()
    alpha = abs(P.emid) + P.r
    assert o["info"] == 0, (o["info"], M, o["loop"])
    if exact is not None:
        assert M == len(exact)
        for lam in exact:
            assert np.min(np.abs(E[:M] - lam)) < TOL_E * alpha
    assert np.all(G.inside(E[:M], P.emid, P.r, fpm[17], fpm[18]))
    assert not np.any(G.inside(E[M:], P.emid, P.r, fpm[17], fpm[18]))
    key = np.lexsort((E[:M].imag, E[:M].real))
    assert np.all(key == np.arange(M))
    assert np.max(res[:M]) < 1e-10 and np.max(res[m0:m0 + M]) < 1e-10
    X = o["X"]
    Xr, Xl = X[:, :M], X[:, m0:m0 + M]
    assert torch.allclose(torch.linalg.vector_norm(Xr, dim=0), torch.ones(M, dtype=torch.float64, device="cuda"),
                          atol=1e-12)
    B = torch.eye(P.n, dtype=torch.complex128, device="cuda") if P.B is None else _dev(P.B).to(torch.complex128)
    Gm = Xl.conj().T @ (B @ Xr)
    assert torch.max(torch.abs(Gm - torch.eye(M, dtype=torch.complex128, device="cuda"))).item() < 1e-10
    assert o["biorth"] is not None and o["biorth"] < 1e-10
    # residuals recomputed from the returned vectors (definition of Table tab_common)
    A = _dev(P.A).to(torch.complex128)
    Et = o["E"][:M]
    rr = (torch.sum(torch.abs(A @ Xr - (B @ Xr) * Et), 0) / torch.sum(torch.abs(alpha * (B @ Xr)), 0))
    assert torch.max(rr).item() < 1e-10


@pytest.mark.parametrize("n", [40, 130, 200])
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("prec", [0, 1])
def test_parity_with_oracle(gbf, n, cplx, gen, prec):
    """FP64 factors (prec 0) and FP32 factors with the FP64 residual
    correction (prec 1, fpm(42)=1) against the FP64 oracle."""
    P = W.dense_nonsymmetric(n, count=max(3, n // 20), m0=max(6, n // 12), complex_=cplx, generalized=gen)
    fpm = P.apply_fpm(gbf.gbf_init())
    fpm[41] = prec
    h = gbf.Handle()
    o = _run(gbf, P, fpm, h)
    ref = G.feast_gen(P.A, P.B, P.emid, P.r, P.m0, P.apply_fpm(G.feastinit_gen()))
    assert ref["info"] == 0
    exact = ref["E"][:ref["M"]]
    _check_outputs(P, o, fpm, exact)
    assert abs(o["loop"] - ref["loop"]) <= (1 if prec == 0 else 2)
    known = P.spectrum[G.inside(P.spectrum, P.emid, P.r)]
    for lam in known:
        assert np.min(np.abs(o["E"].cpu().numpy()[:o["M"]] - lam)) < TOL_E
    h.close()


@pytest.mark.parametrize("qtype", [0, 1])
@pytest.mark.parametrize("cplx", [False, True])
def test_first_contour_subspaces_match_oracle(gbf, qtype, cplx):
    """fpm(14)=1: Q and Q^ after one contour, element by element (the real
    problem takes the conjugate-pair path on the GPU, all nodes in the
    oracle)."""
    P = W.dense_nonsymmetric(150, count=8, m0=12, complex_=cplx, generalized=True, seed=11)
    fpm = P.apply_fpm(gbf.gbf_init())
    fpm[13] = 1
    fpm[16] = qtype
    o = _run(gbf, P, fpm, gbf.Handle())
    assert o["info"] == 4
    fo = P.apply_fpm(G.feastinit_gen())
    fo[13] = 1
    fo[16] = qtype
    ref = G.feast_gen(P.A, P.B, P.emid, P.r, P.m0, fo)
    Xg = o["X"].cpu().numpy()
    for part in (slice(0, P.m0), slice(P.m0, 2 * P.m0)):
        a, b = Xg[:, part], ref["X"][:, part]
        assert np.max(np.abs(a - b)) <= 1e-11 * np.max(np.abs(b))


def test_conjugate_pair_path_equals_complex_path(gbf):
    """A real problem (fpm(8)/2 factorisations) and the same matrices passed
    as complex (all fpm(8) nodes factored) give the same eigenpairs."""
    P = W.dense_nonsymmetric(256, count=12, m0=20, generalized=True, seed=5)
    fpm = P.apply_fpm(gbf.gbf_init())
    o1 = _run(gbf, P, fpm, gbf.Handle())
    Pc = W.GeneralProblem(P.name, True, P.A.astype(np.complex128), P.B.astype(np.complex128), P.emid, P.r, P.m0,
                          P.spectrum, P.count)
    o2 = _run(gbf, Pc, fpm, gbf.Handle())
    assert o1["info"] == 0 and o2["info"] == 0 and o1["M"] == o2["M"] == 12
    E1, E2 = o1["E"].cpu().numpy()[:12], o2["E"].cpu().numpy()[:12]
    for lam in E2:
        assert np.min(np.abs(E1 - lam)) < 1e-12
    assert abs(o1["loop"] - o2["loop"]) <= 1


@pytest.mark.parametrize("qtype,ratio,angle,crit,m0", [(0, 100, 0, 1, 16), (1, 60, 25, 1, 12), (1, 100, 0, 0, 16),
                                                       (0, 150, -90, 0, 24)])
def test_contour_shapes_and_criteria(gbf, qtype, ratio, angle, crit, m0):
    """Gauss and trapezoidal rules on circles and rotated ellipses, residual
    and trace criteria (M0 about 1.5 times the count inside, as the guide
    advises)."""
    P = W.dense_nonsymmetric(180, count=10, m0=m0, complex_=True, seed=9)
    fpm = P.apply_fpm(gbf.gbf_init())
    fpm[16], fpm[17], fpm[18], fpm[5] = qtype, ratio, angle, crit
    fpm[7] = 24
    h = gbf.Handle()
    o = _run(gbf, P, fpm, h)
    fo = P.apply_fpm(G.feastinit_gen())
    fo[16], fo[17], fo[18], fo[5], fo[7] = qtype, ratio, angle, crit, 24
    ref = G.feast_gen(P.A, P.B, P.emid, P.r, P.m0, fo)
    assert o["info"] == ref["info"] == 0
    assert o["M"] == ref["M"]
    E = o["E"].cpu().numpy()
    for lam in ref["E"][:ref["M"]]:
        assert np.min(np.abs(E[:o["M"]] - lam)) < TOL_E
    if crit == 1:
        _check_outputs(P, o, fpm, ref["E"][:ref["M"]])
    h.close()


def test_restart_from_returned_vectors(gbf):
    P = W.dense_nonsymmetric(160, count=9, m0=14, complex_=False, seed=3)
    fpm = P.apply_fpm(gbf.gbf_init())
    h = gbf.Handle()
    o = _run(gbf, P, fpm, h)
    assert o["info"] == 0 and o["loop"] >= 1
    fpm[4] = 1
    o2 = _run(gbf, P, fpm, h, X=o["X"].clone())
    assert o2["info"] == 0 and o2["loop"] <= 1 and o2["M"] == o["M"]
    E1, E2 = o["E"].cpu().numpy()[:o["M"]], o2["E"].cpu().numpy()[:o["M"]]
    assert np.max(np.abs(E1 - E2)) < 1e-12


def test_info_codes(gbf):
    P = W.dense_nonsymmetric(100, count=8, m0=12, complex_=True)
    fpm = P.apply_fpm(gbf.gbf_init())
    h = gbf.Handle()
    A = _dev(P.A)
    o = gbf.feast_gen_dev(A, None, 5.0 + 5.0j, 0.5, 8, fpm, handle=h)
    assert o["info"] == 1 and o["M"] == 0
    o = gbf.feast_gen_dev(A, None, P.emid, P.r, 5, fpm, handle=h)
    assert o["info"] == 3
    o = gbf.feast_gen_dev(A, None, P.emid, 0.0, 12, fpm, handle=h)
    assert o["info"] == 200
    o = gbf.feast_gen_dev(A, None, P.emid, P.r, 101, fpm, handle=h)
    assert o["info"] == 201
    bad = fpm.copy()
    bad[41] = 2
    assert gbf.feast_gen_dev(A, None, P.emid, P.r, 12, bad, handle=h)["info"] == 142
    bad = fpm.copy()
    bad[16] = 3
    assert gbf.feast_gen_dev(A, None, P.emid, P.r, 12, bad, handle=h)["info"] == 117
    An = A.clone()
    An[3, 7] = float("nan")
    o = gbf.feast_gen_dev(An, None, P.emid, P.r, 12, fpm, handle=h)
    assert o["info"] == -2
    # the context stays usable
    o = gbf.feast_gen_dev(A, None, P.emid, P.r, 12, fpm, handle=h)
    assert o["info"] == 0 and o["M"] == 8
    h.close()


@pytest.mark.parametrize("n,m0", [(1, 1), (2, 2), (5, 3), (33, 33)])
def test_tiny_and_full_subspace(gbf, n, m0):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    lam = np.linalg.eigvals(A)
    emid = complex(np.mean(lam))
    r = 1.05 * float(np.max(np.abs(lam - emid))) + 1e-3
    fpm = gbf.gbf_init()
    fpm[7] = 32
    o = gbf.feast_gen_dev(_dev(A), None, emid, r, m0, fpm, handle=gbf.Handle())
    torch.cuda.synchronize()
    if m0 < n:
        assert o["info"] == 3
        return
    assert o["info"] == 0 and o["M"] == n
    E = o["E"].cpu().numpy()
    for l in lam:
        assert np.min(np.abs(E - l)) < 1e-10 * max(1.0, abs(l))


@pytest.mark.parametrize("prec", [0, 1])
def test_known_spectrum_n2048(gbf, prec):
    """A larger real non-symmetric pencil (several LU tiles, a ragged
    subspace): eigenvalues against the construction's spectrum, residuals
    and bi-orthonormality through the outputs, FP64 and FP32 factors."""
    P = W.dense_nonsymmetric(2048, count=24, m0=40, generalized=True, seed=21)
    fpm = P.apply_fpm(gbf.gbf_init())
    fpm[41] = prec
    o = _run(gbf, P, fpm, gbf.Handle())
    known = P.spectrum[G.inside(P.spectrum, P.emid, P.r)]
    _check_outputs(P, o, fpm, known)


@pytest.mark.parametrize("cplx", [False, True])
def test_host_entry_and_expert_nodes(gbf, cplx):
    """The host-array drivers equal the device ones bit for bit; the expert
    form with the rule's own nodes and weights equals the default; custom
    nodes (Gauss, 24 points, passed by the caller) reach the same pairs."""
    P = W.dense_nonsymmetric(140, count=8, m0=13, complex_=cplx, generalized=True, seed=4)
    fpm = P.apply_fpm(gbf.gbf_init())
    h = gbf.Handle()
    od = _run(gbf, P, fpm, h)
    oh = gbf.feast_gen_host(P.A, P.B, P.emid, P.r, P.m0, fpm)
    assert oh["info"] == od["info"] == 0 and oh["M"] == od["M"] and oh["loop"] == od["loop"]
    assert np.array_equal(oh["E"], od["E"].cpu().numpy())
    assert np.array_equal(oh["res"], od["res"].cpu().numpy())
    assert np.array_equal(oh["X"], od["X"].cpu().numpy())
    z, w = gbf.gbf_gcontour(P.emid, P.r, 16, 1, 100, 0)
    ox = gbf.feast_gen_host(P.A, P.B, P.emid, P.r, P.m0, fpm, Zne=z, Wne=w)
    assert ox["info"] == 0 and ox["M"] == od["M"]
    Ed = od["E"].cpu().numpy()[:od["M"]]
    for lam in ox["E"][:ox["M"]]:
        assert np.min(np.abs(Ed - lam)) < 1e-12
    z, w = G.gcontour(P.emid, P.r, 24, 0)
    f2 = fpm.copy()
    f2[7] = 24
    og = gbf.feast_gen_host(P.A, P.B, P.emid, P.r, P.m0, f2, Zne=z, Wne=w)
    assert og["info"] == 0 and og["M"] == od["M"]
    for lam in og["E"][:og["M"]]:
        assert np.min(np.abs(Ed - lam)) < 1e-10
    h.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("cplx", [False, True])
def test_large_subspace_sparse_spectrum(gbf, prec, cplx):
    """M0 well above the count (here 2.7 times): the columns of Q for the
    eigenvalues far outside carry filter values far below the solves'
    rounding level.  From the second loop on they are formed in the
    residual-correction form, exact relative to their own size, so the
    reduced pencil stays regular and the pairs inside converge."""
    P = W.dense_nonsymmetric(300, count=6, m0=16, complex_=cplx, generalized=True, seed=13)
    fpm = P.apply_fpm(gbf.gbf_init())
    fpm[41] = prec
    o = _run(gbf, P, fpm, gbf.Handle())
    known = P.spectrum[G.inside(P.spectrum, P.emid, P.r)]
    _check_outputs(P, o, fpm, known)


def test_nearly_defective_pair(gbf):
    """A 2 x 2 block [[0, 1], [0, 1e-6]] inside the circle: nearly parallel
    eigenvectors, a tiny Gram eigenvalue in the wanted span; both
    eigenvalues found, as by the oracle."""
    rng = np.random.default_rng(7)
    n = 60
    T = np.diag(rng.uniform(1.0, 3.0, n)).astype(complex)
    T[0, 0], T[1, 1], T[0, 1] = 0.0, 1e-6, 1.0
    U = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))[0]
    A = U @ T @ U.conj().T
    fpm = gbf.gbf_init()
    o = gbf.feast_gen_dev(_dev(A), None, 0.0, 0.5, 4, fpm, handle=gbf.Handle())
    torch.cuda.synchronize()
    ref = G.feast_gen(A, None, 0.0, 0.5, 4, G.feastinit_gen())
    assert ref["info"] == 0 and o["info"] == 0 and o["M"] == 2
    E = o["E"].cpu().numpy()[:2]
    assert np.min(np.abs(E)) < 1e-9 and np.min(np.abs(E - 1e-6)) < 1e-9
