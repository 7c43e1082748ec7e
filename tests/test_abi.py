"""C-ABI boundary checks that need no GPU: the library builds, loads and
exports every symbol include/gbfeast.h declares; host-only entry points
(feastinit defaults, contour, rational filter, argument validation) match
the oracle and the guide's tables."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import paper_1203_4031_gb300 as g

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "gbfeast.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gbf_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = g.load()
    names = declared_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name


def test_version_and_error_text():
    assert g.version() >= 100
    assert isinstance(g.last_error(), str)


def test_feastinit_defaults_table():
    """Table tab_fpm defaults (fpm[i-1] = fpm(i))."""
    fpm = g.gbf_init()
    expect = {2: 8, 3: 12, 4: 20, 6: 1, 7: 5, 8: 16, 17: 1, 18: 100}
    for i in range(1, 65):
        assert fpm[i - 1] == expect.get(i, 0), i
    assert np.array_equal(fpm, oracle.feastinit())


@pytest.mark.parametrize("ne", [1, 2, 8, 16, 20, 56])
@pytest.mark.parametrize("qtype,ratio", [(0, 100), (1, 100), (0, 50), (1, 200)])
def test_contour_matches_oracle(ne, qtype, ratio):
    for emin, emax in [(-5.0, 5.0), (0.5, 1.0), (-0.0023589538297558448, 0.0023589538297558448)]:
        z, w = g.gbf_contour(emin, emax, ne, qtype, ratio)
        zo, wo = oracle.contour(emin, emax, ne, qtype, ratio)
        scale = emax - emin
        assert np.max(np.abs(z - zo)) <= 4e-16 * scale * 4 + 1e-300
        assert np.max(np.abs(w - wo)) <= 4e-16 * scale * 4 + 1e-300


@pytest.mark.parametrize("ne", [8, 16])
def test_rational_matches_oracle_and_invariants(ne):
    x = np.linspace(-2.0, 3.0, 101)
    f = g.gbf_rational(-0.5, 1.5, ne, x)
    fo = oracle.rational(-0.5, 1.5, ne, x)
    assert np.max(np.abs(f - fo)) < 1e-14
    fc = g.gbf_rational(-0.5, 1.5, ne, np.array([0.5, -0.5, 1.5]))
    assert abs(fc[0] - 1) < 1e-14 and abs(fc[1] - 0.5) < 1e-13 and abs(fc[2] - 0.5) < 1e-13
    z, w = g.gbf_contour(-0.5, 1.5, ne)
    assert np.max(np.abs(g.gbf_rationalx(z, w, x) - f)) == 0.0


def test_contour_info_codes():
    L = g.load()
    z = np.zeros(16)
    w = np.zeros(16)
    dp = C.POINTER(C.c_double)
    zp, wp = z.ctypes.data_as(dp), w.ctypes.data_as(dp)
    assert L.gbf_contour(1.0, 1.0, 8, 0, 100, zp, wp) == 200
    assert L.gbf_contour(0.0, 1.0, 0, 0, 100, zp, wp) == 102
    assert L.gbf_contour(0.0, 1.0, 8, 2, 100, zp, wp) == 116
    assert L.gbf_contour(0.0, 1.0, 8, 0, 0, zp, wp) == 118


def test_driver_argument_validation_without_gpu():
    """Codes of Table tab_info that are decided before any device work."""
    A = np.diag(np.arange(1.0, 11.0))
    r = g.feast_host(A[:0, :0].reshape(0, 0), None, 0, 1, 1)
    assert r["info"] == 202
    assert g.feast_host(A, None, 0.0, 5.0, 0)["info"] == 201
    assert g.feast_host(A, None, 0.0, 5.0, 11)["info"] == 201
    assert g.feast_host(A, None, 5.0, 5.0, 4)["info"] == 200
    assert g.feast_host(A, None, 0.0, 5.0, 4, uplo="X")["info"] == -101
    base = g.gbf_init()
    for idx, bad, code in [(1, 21, 102), (1, 0, 102), (2, -1, 103), (3, -1, 104), (4, 2, 105),
                           (5, 3, 106), (13, 3, 114), (15, 2, 116), (17, 0, 118), (41, 2, 142),
                           (42, 5, 143), (43, 2, 144)]:
        f = base.copy()
        f[idx] = bad
        assert g.feast_host(A, None, 0.5, 3.5, 5, fpm=f)["info"] == code, (idx, bad)


def test_gen_driver_argument_validation_without_gpu():
    """Non-Hermitian drivers: the codes decided before any device work."""
    A = np.diag(np.arange(1.0, 11.0)) + np.triu(np.ones((10, 10)), 1)
    assert g.feast_gen_host(A[:0, :0].reshape(0, 0), None, 0.0, 1.0, 1)["info"] == 202
    assert g.feast_gen_host(A, None, 2.0, 1.5, 0)["info"] == 201
    assert g.feast_gen_host(A, None, 2.0, 1.5, 11)["info"] == 201
    assert g.feast_gen_host(A, None, 2.0, 0.0, 4)["info"] == 200
    assert g.feast_gen_host(A, None, 2.0, -1.0, 4)["info"] == 200
    base = g.gbf_init()
    for idx, bad, code in [(2, -1, 103), (2, 17, 103), (3, -1, 104), (4, 2, 105), (5, 3, 106), (7, 0, 108),
                           (7, 2000, 108), (13, 2, 114), (16, 2, 117), (17, 0, 118), (18, 181, 119),
                           (18, -181, 119), (41, 2, 142), (42, 5, 143), (43, 2, 144)]:
        f = base.copy()
        f[idx] = bad
        assert g.feast_gen_host(A, None, 2.0 + 0.5j, 1.5, 5, fpm=f)["info"] == code, (idx, bad)


def test_tensor_core_workspace_sizes():
    """Workspace sizes are host arithmetic on the operand layouts: S digit
    planes of bf16 (64 per embedded row) plus one 8-byte scale slot per row
    and column for the sliced engine; for S = 1 (3xTF32), hi and lo planes
    of 2 K-chunks x 32 FP32 per embedded row of A and per column of B."""
    L = g.load()
    L.gbf_zgemm_sliced_work.restype = C.c_size_t
    L.gbf_zgemm_sliced_work.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
    al = lambda v: (v + 255) & ~255  # noqa: E731
    for m, n, b in [(1, 1, 1), (300, 200, 2), (4096, 4096, 8), (8191, 241, 16)]:
        assert L.gbf_zgemm_sliced_work(m, n, b, 1) == al(2 * b * 2 * 2 * m * 32 * 4) + al(2 * b * 2 * n * 32 * 4)
        for S in (7, 4, 3, -3):
            s = abs(S)
            assert L.gbf_zgemm_sliced_work(m, n, b, S) == (al(s * b * 2 * m * 64 * 2) + al(s * b * n * 64 * 2)
                                                            + al(b * 2 * m * 8) + al(b * n * 8))


# ------------------------------------------------ non-Hermitian contour --
@pytest.mark.parametrize("ne", [1, 2, 7, 16, 40])
@pytest.mark.parametrize("qtype,ratio,angle", [(0, 100, 0), (1, 100, 0), (0, 50, 30), (1, 170, -135)])
def test_gcontour_matches_oracle(ne, qtype, ratio, angle):
    from oracle import feast_gen as G

    for emid, r in [(0.0, 1.0), (0.3 - 0.2j, 1.7), (-4.0 + 2.0j, 0.01)]:
        z, w = g.gbf_gcontour(emid, r, ne, qtype, ratio, angle)
        zo, wo = G.gcontour(emid, r, ne, qtype, ratio, angle)
        scale = abs(emid) + r
        assert np.max(np.abs(z - zo)) <= 1e-15 * scale * 16
        assert np.max(np.abs(w - wo)) <= 1e-15 * r * 16
        lam = emid + r * np.array([0.1 + 0.2j, 0.9, -1.3j, 2.0 + 1.0j])
        f = g.gbf_grationalx(z, w, lam)
        assert np.allclose(f, G.grationalx(zo, wo, lam), rtol=1e-10 * (abs(emid) + r) / r, atol=1e-14)


def test_gcontour_info_codes():
    L = g.load()
    z = np.zeros(32)
    w = np.zeros(32)
    zp, wp = C.c_void_p(z.ctypes.data), C.c_void_p(w.ctypes.data)
    assert L.gbf_gcontour(0.0, 0.0, 0.0, 8, 1, 100, 0, zp, wp) == 200
    assert L.gbf_gcontour(0.0, 0.0, 1.0, 0, 1, 100, 0, zp, wp) == 108
    assert L.gbf_gcontour(0.0, 0.0, 1.0, 8, 2, 100, 0, zp, wp) == 117
    assert L.gbf_gcontour(0.0, 0.0, 1.0, 8, 1, 0, 0, zp, wp) == 118
    assert L.gbf_gcontour(0.0, 0.0, 1.0, 8, 1, 100, 181, zp, wp) == 119
