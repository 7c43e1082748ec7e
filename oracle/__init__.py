"""Plain FP64 CPU FEAST oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  The CUDA product path
(``paper_1203_4031_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``feast_oracle.c`` (see its header for the guide
sections each routine restates); this module only marshals numpy arrays
through ctypes and expands the ``UPLO`` storage convention of the dense
interfaces ("Matrix storage" section: 'F' full, 'L' lower, 'U' upper).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
        vp = C.c_void_p
        L.ora_gauss_legendre.argtypes = [C.c_int, dp, dp]
        L.ora_contour.argtypes = [C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, vp, vp]
        L.ora_rationalx.argtypes = [vp, vp, C.c_int, dp, C.c_int, dp]
        L.ora_zgetrf.argtypes = [C.c_int, vp, C.c_int, ip]
        L.ora_zgetrs.argtypes = [C.c_int, C.c_int, C.c_int, vp, C.c_int, ip, vp, C.c_int]
        L.ora_zheev_jacobi.argtypes = [C.c_int, vp, C.c_int, dp, vp, C.c_int]
        L.ora_inertia_neg.argtypes = [C.c_int, vp, C.c_int, C.POINTER(C.c_long)]
        L.ora_inertia_neg.restype = C.c_long
        L.ora_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        L.ora_splitmix64.restype = C.c_uint64
        L.ora_feast.argtypes = [C.c_int, C.c_int, vp, C.c_int, vp, C.c_int, ip,
                                C.c_double, C.c_double, C.c_int, vp, vp, vp, dp, dp,
                                ip, ip, dp, ip, ip, C.c_int]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _v(a):
    return C.c_void_p(a.ctypes.data)


def _zf(a):
    """Fortran-ordered complex128 copy."""
    return np.asfortranarray(np.array(a, dtype=np.complex128))


def feastinit():
    """Defaults of Table tab_fpm (fpm[i-1] = fpm(i))."""
    fpm = np.zeros(64, dtype=np.int32)
    fpm[1] = 8      # fpm(2) contour points (half contour)
    fpm[2] = 12     # fpm(3) eps = 1e-12
    fpm[3] = 20     # fpm(4) max refinement loops
    fpm[5] = 1      # fpm(6) residual-based convergence
    fpm[6] = 5      # fpm(7) single precision eps exponent
    fpm[7] = 16     # fpm(8) full-contour points (non-Hermitian)
    fpm[16] = 1     # fpm(17) non-Hermitian quadrature
    fpm[17] = 100   # fpm(18) ellipse ratio (circle)
    return fpm


def gauss_legendre(ne):
    x = np.zeros(ne)
    w = np.zeros(ne)
    if lib().ora_gauss_legendre(ne, _d(x), _d(w)) != 0:
        raise ValueError("ne must be >= 1")
    return x, w


def contour(emin, emax, ne, qtype=0, ratio=100):
    z = np.zeros(ne, dtype=np.complex128)
    w = np.zeros(ne, dtype=np.complex128)
    rc = lib().ora_contour(float(emin), float(emax), int(ne), int(qtype), int(ratio), _v(z), _v(w))
    if rc != 0:
        raise ValueError(f"ora_contour failed ({rc})")
    return z, w


def rationalx(zne, wne, eig):
    zne = np.ascontiguousarray(zne, dtype=np.complex128)
    wne = np.ascontiguousarray(wne, dtype=np.complex128)
    eig = np.ascontiguousarray(eig, dtype=np.float64)
    f = np.zeros(eig.shape[0])
    lib().ora_rationalx(_v(zne), _v(wne), len(zne), _d(eig), eig.shape[0], _d(f))
    return f


def rational(emin, emax, ne, eig, qtype=0, ratio=100):
    z, w = contour(emin, emax, ne, qtype, ratio)
    return rationalx(z, w, eig)


def zgetrf(S):
    a = _zf(S)
    n = a.shape[0]
    ipiv = np.zeros(n, dtype=np.int32)
    info = lib().ora_zgetrf(n, _v(a), n, _i(ipiv))
    return a, ipiv, info


def zgetrs(lu, ipiv, b, trans=0):
    b = _zf(b)
    if b.ndim == 1:
        b = b.reshape(-1, 1, order="F")
    n = lu.shape[0]
    lib().ora_zgetrs(int(trans), n, b.shape[1], _v(lu), n, _i(ipiv), _v(b), n)
    return b


def jacobi_eigh(H):
    a = _zf(H)
    n = a.shape[0]
    w = np.zeros(n)
    v = np.zeros((n, n), dtype=np.complex128, order="F")
    sweeps = lib().ora_zheev_jacobi(n, _v(a), n, _d(w), _v(v), n)
    return w, v, sweeps


def inertia_neg(H):
    """(#negative, #zero pivots) of a Hermitian matrix."""
    a = _zf(H)
    z = C.c_long(0)
    neg = lib().ora_inertia_neg(a.shape[0], _v(a), a.shape[0], C.byref(z))
    return int(neg), int(z.value)


def eigcount(A, B, a, b):
    """Sylvester count of pencil eigenvalues in [a, b]: nu(A-bB) - nu(A-aB)."""
    A = np.asarray(A)
    Bm = np.eye(A.shape[0]) if B is None else np.asarray(B)
    return inertia_neg(A - b * Bm)[0] - inertia_neg(A - a * Bm)[0]


def splitmix64(seed, i):
    return int(lib().ora_splitmix64(C.c_uint64(seed), C.c_uint64(i)))


def expand_uplo(M, uplo):
    """Full Hermitian matrix from the triangle UPLO references."""
    M = np.array(M)
    if uplo in ("F", "f"):
        return M
    if uplo in ("L", "l"):
        low = np.tril(M, -1)
    elif uplo in ("U", "u"):
        low = np.triu(M, 1).conj().T
    else:
        raise ValueError("uplo must be F, L or U")
    d = np.diag(np.real(np.diag(M))) if np.iscomplexobj(M) else np.diag(np.diag(M))
    return low + d + low.conj().T


def feast(A, B, emin, emax, m0, fpm=None, X0=None, zne=None, wne=None,
          hermitian=None, uplo="F", nthreads=None):
    """Run the oracle FEAST.  Returns a dict with E, X, res, M, loop, epsout,
    m0 (kept subspace size) and info, in the layout of Table tab_common."""
    if fpm is None:
        fpm = feastinit()
    fpm = np.ascontiguousarray(fpm, dtype=np.int32)
    if hermitian is None:
        hermitian = np.iscomplexobj(A) or (B is not None and np.iscomplexobj(B))
    A = _zf(expand_uplo(A, uplo))
    n = A.shape[0]
    Bf = None if B is None else _zf(expand_uplo(B, uplo))
    X = np.zeros((max(n, 1), max(int(m0), 1)), dtype=np.complex128, order="F")
    if X0 is not None:
        X[:, :] = X0
    E = np.zeros(max(int(m0), 1))
    res = np.zeros(max(int(m0), 1))
    M = C.c_int(0)
    loop = C.c_int(0)
    eps = C.c_double(0)
    m0o = C.c_int(0)
    info = C.c_int(0)
    zp = wp = None
    if zne is not None:
        zne = np.ascontiguousarray(zne, dtype=np.complex128)
        wne = np.ascontiguousarray(wne, dtype=np.complex128)
        zp, wp = _v(zne), _v(wne)
    if nthreads is None:
        nthreads = int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))
    lib().ora_feast(1 if hermitian else 0, n, _v(A), n,
                    None if Bf is None else _v(Bf), n, _i(fpm),
                    float(emin), float(emax), int(m0), zp, wp, _v(X), _d(E), _d(res),
                    C.byref(M), C.byref(loop), C.byref(eps), C.byref(m0o),
                    C.byref(info), int(nthreads))
    Xo = X if hermitian else X.real.copy(order="F")
    return dict(E=E, X=Xo, res=res, M=M.value, loop=loop.value, epsout=eps.value,
                m0=m0o.value, info=info.value, fpm=fpm)
