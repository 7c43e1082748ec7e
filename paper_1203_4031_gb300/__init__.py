"""Python binding of libgbfeast (include/gbfeast.h): argument marshalling only.

Every function forwards to the C ABI of the same name; all arithmetic runs in
the CUDA library.  Host-pointer drivers take numpy arrays; ``*_dev`` entry
points take CUDA tensors (torch) in column-major layout (stride (1, ld)).
There is no fallback: if the library cannot be built or loaded, ``load()``
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def load(build: bool = True):
    """Load (building first if needed) libgbfeast.so; raises on failure."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libgbfeast.so not found at {path}")
    L = C.CDLL(path)
    vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)
    L.gbf_version.restype = C.c_int
    L.gbf_last_error.restype = C.c_char_p
    L.gbf_launch_count.restype = C.c_longlong
    L.gbf_create.argtypes = [C.POINTER(vp)]
    L.gbf_destroy.argtypes = [vp]
    L.gbf_init.argtypes = [ip]
    L.gbf_contour.argtypes = [C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, dp, dp]
    L.gbf_rational.argtypes = [C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, dp, C.c_int, dp]
    L.gbf_rationalx.argtypes = [dp, dp, C.c_int, dp, C.c_int, dp]
    host_ev = [C.c_char, C.c_int, vp, C.c_int, ip, dp, ip, C.c_double, C.c_double, ip, vp, vp, ip, vp, ip]
    host_gv = [C.c_char, C.c_int, vp, C.c_int, vp, C.c_int, ip, dp, ip, C.c_double, C.c_double, ip, vp, vp,
               ip, vp, ip]
    for name in ("gbf_dsyev", "gbf_zheev"):
        getattr(L, name).argtypes = host_ev
    for name in ("gbf_dsygv", "gbf_zhegv"):
        getattr(L, name).argtypes = host_gv
    for name in ("gbf_dsygvx", "gbf_zhegvx"):
        getattr(L, name).argtypes = host_gv + [vp, vp]
    dev = [vp, vp, C.c_char, C.c_int, vp, C.c_int, vp, C.c_int, ip, dp, ip, C.c_double, C.c_double, ip, vp, vp,
           ip, vp, ip, vp, vp]
    L.gbf_dsygv_dev.argtypes = dev
    L.gbf_zhegv_dev.argtypes = dev
    L.gbf_dsygv_dev_shard.argtypes = dev + [vp]
    L.gbf_zhegv_dev_shard.argtypes = dev + [vp]
    L.gbf_shard_nodes.argtypes = [C.c_int, C.c_int, C.c_int, ip, ip]
    gen = [vp, vp, C.c_int, vp, C.c_int, vp, C.c_int, ip, dp, ip, C.c_double, C.c_double, C.c_double, ip, vp, vp,
           ip, vp, ip, vp, vp]
    L.gbf_dgegv_dev.argtypes = gen
    L.gbf_zgegv_dev.argtypes = gen
    gen_host = [C.c_int, vp, C.c_int, vp, C.c_int, ip, dp, ip, C.c_double, C.c_double, C.c_double, ip, vp, vp, ip,
                vp, ip, vp, vp]
    L.gbf_dgegv.argtypes = gen_host
    L.gbf_zgegv.argtypes = gen_host
    L.gbf_gcontour.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp]
    L.gbf_grationalx.argtypes = [vp, vp, C.c_int, vp, C.c_int, vp]
    L.gbf_wait_probe.argtypes = [vp, C.c_long]
    L.gbf_biorth_defect.argtypes = [vp]
    L.gbf_biorth_defect.restype = C.c_double
    L.gbf_factor_dev.argtypes = [vp, vp, C.c_int, C.c_int, C.c_char, C.c_int, vp, C.c_int, vp, C.c_int, C.c_int, vp]
    L.gbf_solve_dev.argtypes = [vp, vp, C.c_int, C.c_int, vp, vp]
    L.gbf_heev_dev.argtypes = [vp, vp, C.c_int, C.c_int, vp, vp, vp]
    L.gbf_problem_bytes.argtypes = [C.POINTER(Problem)]
    L.gbf_problem_bytes.restype = C.c_size_t
    L.gbf_batch_solve.argtypes = [vp, vp, C.c_int, C.POINTER(Problem), C.POINTER(Result), C.c_int]
    L.gbf_server_create.argtypes = [C.c_size_t, C.c_int, C.POINTER(vp)]
    L.gbf_server_submit.argtypes = [vp, C.POINTER(Problem), C.POINTER(C.c_ulonglong)]
    L.gbf_server_poll.argtypes = [vp, C.c_ulonglong, C.POINTER(Result)]
    L.gbf_server_wait.argtypes = [vp, C.c_ulonglong, C.POINTER(Result)]
    L.gbf_server_stats.argtypes = [vp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t), C.POINTER(C.c_int),
                                   C.POINTER(C.c_int)]
    L.gbf_server_destroy.argtypes = [vp]
    L.gbf_tc_gemm_bf16.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, C.c_long, C.c_long, vp]
    L.gbf_zgemm_sliced_work.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
    L.gbf_zgemm_sliced_work.restype = C.c_size_t
    L.gbf_zgemm_sliced.argtypes = [vp, C.c_int, C.c_int, C.c_char, C.c_char, C.c_int, C.c_int, C.c_int, C.c_double,
                                   vp, C.c_long, C.c_long, vp, C.c_long, C.c_long, C.c_int, vp, C.c_long, C.c_long,
                                   C.c_int, vp, C.c_size_t, vp]
    L.gbf_gemm_sliced_work.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
    L.gbf_gemm_sliced_work.restype = C.c_size_t
    L.gbf_gemm_sliced.argtypes = [vp, C.c_int, C.c_char, C.c_char, C.c_int, C.c_int, C.c_int, C.c_double, vp,
                                  C.c_long, C.c_long, vp, C.c_long, C.c_long, C.c_int, vp, C.c_long, C.c_long,
                                  C.c_int, vp, C.c_size_t, vp]
    L.gbf_cgemm_tf32_work.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
    L.gbf_cgemm_tf32_work.restype = C.c_size_t
    L.gbf_cgemm_tf32.argtypes = [vp, C.c_char, C.c_char, C.c_int, C.c_int, C.c_int, C.c_double, vp, C.c_long,
                                 C.c_long, vp, C.c_long, C.c_long, C.c_int, vp, C.c_long, C.c_long, C.c_int, vp,
                                 C.c_size_t, vp]
    L.gbf_zgemm_sliced_noalloc_max.restype = C.c_size_t
    L.gbf_zgemm_sliced_noalloc.argtypes = [vp, C.c_int, C.c_int, C.c_char, C.c_char, C.c_int, C.c_int, C.c_int,
                                           C.c_double, vp, C.c_long, C.c_long, vp, C.c_long, C.c_long, C.c_int, vp,
                                           C.c_long, C.c_long, C.c_int]
    L.gbf_profile.argtypes = [C.c_int]
    L.gbf_profile_name.restype = C.c_char_p
    L.gbf_profile_read.argtypes = [C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    _lib = L
    return L


def lib():
    return load()


# ------------------------------------------------------------- ABI structs --
class Problem(C.Structure):
    """gbf_problem (include/gbfeast.h)."""
    _fields_ = [("kind", C.c_int), ("uplo", C.c_char), ("n", C.c_int), ("dA", C.c_void_p), ("lda", C.c_int),
                ("dB", C.c_void_p), ("ldb", C.c_int), ("emin", C.c_double), ("emax", C.c_double),
                ("m0", C.c_int), ("fpm", C.c_int * 64), ("dE", C.c_void_p), ("dX", C.c_void_p),
                ("dres", C.c_void_p), ("Zne", C.c_void_p), ("Wne", C.c_void_p)]


class Result(C.Structure):
    """gbf_result (include/gbfeast.h)."""
    _fields_ = [("info", C.c_int), ("M", C.c_int), ("loop", C.c_int), ("m0", C.c_int), ("epsout", C.c_double),
                ("queue_ms", C.c_double), ("run_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# ------------------------------------------------------------------ helpers --
def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _fortran(a, dtype):
    return np.asfortranarray(np.asarray(a, dtype=dtype))


def fortran(t):
    """Column-major view-copy of a 2-D torch tensor (stride (1, rows))."""
    return t.t().contiguous().t()


def _check_colmajor(t, rows):
    if t.dim() != 2 or t.stride(0) != 1 or t.stride(1) < rows:
        raise ValueError("expected a column-major CUDA tensor (use paper_1203_4031_gb300.fortran)")
    return t.stride(1)


def version():
    return lib().gbf_version()


def last_error():
    return lib().gbf_last_error().decode()


def launch_count():
    return lib().gbf_launch_count()


def gbf_init():
    fpm = np.zeros(64, dtype=np.int32)
    lib().gbf_init(_ip(fpm))
    return fpm


def gbf_contour(emin, emax, ne, fpm16=0, fpm18=100):
    z = np.zeros(ne, dtype=np.complex128)
    w = np.zeros(ne, dtype=np.complex128)
    rc = lib().gbf_contour(float(emin), float(emax), int(ne), int(fpm16), int(fpm18),
                           z.ctypes.data_as(C.POINTER(C.c_double)), w.ctypes.data_as(C.POINTER(C.c_double)))
    if rc:
        raise ValueError(f"gbf_contour: info {rc}")
    return z, w


def gbf_rational(emin, emax, ne, eig, fpm16=0, fpm18=100):
    eig = np.ascontiguousarray(eig, dtype=np.float64)
    f = np.zeros(eig.shape[0])
    rc = lib().gbf_rational(float(emin), float(emax), int(ne), int(fpm16), int(fpm18), _dp(eig), eig.shape[0],
                            _dp(f))
    if rc:
        raise ValueError(f"gbf_rational: info {rc}")
    return f


def gbf_rationalx(zne, wne, eig):
    zne = np.ascontiguousarray(zne, dtype=np.complex128)
    wne = np.ascontiguousarray(wne, dtype=np.complex128)
    eig = np.ascontiguousarray(eig, dtype=np.float64)
    f = np.zeros(eig.shape[0])
    lib().gbf_rationalx(zne.ctypes.data_as(C.POINTER(C.c_double)), wne.ctypes.data_as(C.POINTER(C.c_double)),
                        len(zne), _dp(eig), eig.shape[0], _dp(f))
    return f


class Handle:
    """Owner of a gbf_handle (device workspace cache)."""

    def __init__(self):
        h = C.c_void_p()
        rc = lib().gbf_create(C.byref(h))
        if rc:
            raise RuntimeError(f"gbf_create failed ({rc}): {last_error()}")
        self.h = h

    def close(self):
        if self.h:
            lib().gbf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _scalars():
    return (C.c_double(0.0), C.c_int(0), C.c_int(0), C.c_int(0))


def feast_host(A, B, emin, emax, m0, fpm=None, X0=None, uplo="F", hermitian=None, Zne=None, Wne=None):
    """Host-pointer drivers gbf_{dsyev,dsygv,zheev,zhegv}[x]; returns a dict
    with E, X, res, M, loop, epsout, m0 (kept subspace) and info."""
    if fpm is None:
        fpm = gbf_init()
    fpm = np.ascontiguousarray(fpm, dtype=np.int32).copy()
    if hermitian is None:
        hermitian = np.iscomplexobj(A) or (B is not None and np.iscomplexobj(B))
    dt = np.complex128 if hermitian else np.float64
    A = _fortran(A, dt)
    n = A.shape[0]
    Bf = None if B is None else _fortran(B, dt)
    X = np.zeros((n, m0), dtype=dt, order="F")
    if X0 is not None:
        X[:, :] = X0
    E = np.zeros(m0)
    res = np.zeros(m0)
    eps, loop, M, info = _scalars()
    M0 = C.c_int(int(m0))
    u = C.c_char(uplo.encode())
    L = lib()
    args_tail = (_ip(fpm), C.byref(eps), C.byref(loop), float(emin), float(emax), C.byref(M0), _ptr(E), _ptr(X),
                 C.byref(M), _ptr(res), C.byref(info))
    if Zne is not None:
        zne = np.ascontiguousarray(Zne, dtype=np.complex128)
        wne = np.ascontiguousarray(Wne, dtype=np.complex128)
        Bp = Bf if Bf is not None else None
        fn = L.gbf_zhegvx if hermitian else L.gbf_dsygvx
        fn(u, n, _ptr(A), n, _ptr(Bp), n, *args_tail, _ptr(zne), _ptr(wne))
    elif Bf is None:
        (L.gbf_zheev if hermitian else L.gbf_dsyev)(u, n, _ptr(A), n, *args_tail)
    else:
        (L.gbf_zhegv if hermitian else L.gbf_dsygv)(u, n, _ptr(A), n, _ptr(Bf), n, *args_tail)
    return dict(E=E, X=X, res=res, M=M.value, loop=loop.value, epsout=eps.value, m0=M0.value, info=info.value)


def feast_dev(A, B, emin, emax, m0, fpm=None, E=None, X=None, res=None, uplo="F", handle=None, stream=None,
              Zne=None, Wne=None):
    """Device-pointer drivers gbf_dsygv_dev / gbf_zhegv_dev on torch CUDA
    tensors (A, B column-major; B None for the standard problem).  E, X, res
    are allocated if not given (X is read when fpm(5)=1)."""
    import torch

    if fpm is None:
        fpm = gbf_init()
    fpm = np.ascontiguousarray(fpm, dtype=np.int32).copy()
    herm = A.is_complex()
    n = A.shape[0]
    lda = _check_colmajor(A, n)
    ldb = _check_colmajor(B, n) if B is not None else n
    dev = A.device
    if E is None:
        E = torch.zeros(m0, dtype=torch.float64, device=dev)
    if res is None:
        res = torch.zeros(m0, dtype=torch.float64, device=dev)
    if X is None:
        X = torch.zeros((m0, n), dtype=A.dtype, device=dev).t()
    eps, loop, M, info = _scalars()
    M0 = C.c_int(int(m0))
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    sp = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    zp = wp = None
    if Zne is not None:
        zne = np.ascontiguousarray(Zne, dtype=np.complex128)
        wne = np.ascontiguousarray(Wne, dtype=np.complex128)
        zp, wp = _ptr(zne), _ptr(wne)
    fn = lib().gbf_zhegv_dev if herm else lib().gbf_dsygv_dev
    fn(handle.h if handle is not None else None, sp, C.c_char(uplo.encode()), n, _ptr(A), lda, _ptr(B), ldb,
       _ip(fpm), C.byref(eps), C.byref(loop), float(emin), float(emax), C.byref(M0), _ptr(E), _ptr(X),
       C.byref(M), _ptr(res), C.byref(info), zp, wp)
    return dict(E=E, X=X, res=res, M=M.value, loop=loop.value, epsout=eps.value, m0=M0.value, info=info.value)


def gbf_gcontour(emid, r, ne, fpm17=1, fpm18=100, fpm19=0):
    """Full-contour nodes and weights of the non-Hermitian drivers."""
    z = np.zeros(ne, dtype=np.complex128)
    w = np.zeros(ne, dtype=np.complex128)
    emid = complex(emid)
    rc = lib().gbf_gcontour(emid.real, emid.imag, float(r), int(ne), int(fpm17), int(fpm18), int(fpm19), _ptr(z),
                            _ptr(w))
    if rc:
        raise ValueError(f"gbf_gcontour failed ({rc})")
    return z, w


def gbf_grationalx(zne, wne, eig):
    """f(eig) = sum_e w_e / (z_e - eig) for complex eig (host)."""
    zne = np.ascontiguousarray(zne, dtype=np.complex128)
    wne = np.ascontiguousarray(wne, dtype=np.complex128)
    eig = np.ascontiguousarray(eig, dtype=np.complex128)
    f = np.zeros(eig.shape[0], dtype=np.complex128)
    lib().gbf_grationalx(_ptr(zne), _ptr(wne), len(zne), _ptr(eig), eig.shape[0], _ptr(f))
    return f


def feast_gen_dev(A, B, emid, r, m0, fpm=None, X=None, handle=None, stream=None, Zne=None, Wne=None):
    """Non-Hermitian drivers gbf_dgegv_dev (real A, B) / gbf_zgegv_dev
    (complex) on torch CUDA tensors (column-major; B None for the standard
    problem).  Returns E (m0 complex), X (n x 2 m0 complex: right, then left
    vectors; read as the initial guesses when fpm(5)=1), res (2 m0), M, loop,
    epsout, info and the bi-orthonormality defect of a converged solve."""
    import torch

    if fpm is None:
        fpm = gbf_init()
    fpm = np.ascontiguousarray(fpm, dtype=np.int32).copy()
    cplx = A.is_complex()
    n = A.shape[0]
    lda = _check_colmajor(A, n)
    ldb = _check_colmajor(B, n) if B is not None else n
    dev = A.device
    E = torch.zeros(m0, dtype=torch.complex128, device=dev)
    res = torch.zeros(2 * m0, dtype=torch.float64, device=dev)
    if X is None:
        X = torch.zeros((2 * m0, n), dtype=torch.complex128, device=dev).t()
    elif X.stride(0) != 1 or X.stride(1) != n or X.dtype != torch.complex128:
        raise ValueError("X must be complex128, column-major n x 2 m0 with ld n")
    eps, loop, M, info = _scalars()
    M0 = C.c_int(int(m0))
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    sp = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    zp = wp = None
    if Zne is not None:
        zne = np.ascontiguousarray(Zne, dtype=np.complex128)
        wne = np.ascontiguousarray(Wne, dtype=np.complex128)
        zp, wp = _ptr(zne), _ptr(wne)
    emid = complex(emid)
    fn = lib().gbf_zgegv_dev if cplx else lib().gbf_dgegv_dev
    h = handle.h if handle is not None else None
    fn(h, sp, n, _ptr(A), lda, _ptr(B), ldb, _ip(fpm), C.byref(eps), C.byref(loop), emid.real, emid.imag,
       float(r), C.byref(M0), _ptr(E), _ptr(X), C.byref(M), _ptr(res), C.byref(info), zp, wp)
    bi = lib().gbf_biorth_defect(h) if h is not None else None
    return dict(E=E, X=X, res=res, M=M.value, loop=loop.value, epsout=eps.value, info=info.value, biorth=bi)


def feast_gen_host(A, B, emid, r, m0, fpm=None, X0=None, Zne=None, Wne=None):
    """Host-array non-Hermitian drivers gbf_dgegv / gbf_zgegv (numpy A, B;
    B None for the standard problem; Zne, Wne for the expert form).  Returns
    E (m0 complex), X (n x 2 m0 complex), res (2 m0), M, loop, epsout, info."""
    if fpm is None:
        fpm = gbf_init()
    fpm = np.ascontiguousarray(fpm, dtype=np.int32).copy()
    cplx = np.iscomplexobj(A) or (B is not None and np.iscomplexobj(B))
    dt = np.complex128 if cplx else np.float64
    A = _fortran(A, dt)
    n = A.shape[0]
    Bf = None if B is None else _fortran(B, dt)
    X = np.zeros((n, 2 * m0), dtype=np.complex128, order="F")
    if X0 is not None:
        X[:, :] = X0
    E = np.zeros(m0, dtype=np.complex128)
    res = np.zeros(2 * m0)
    eps, loop, M, info = _scalars()
    M0 = C.c_int(int(m0))
    zp = wp = None
    if Zne is not None:
        zne = np.ascontiguousarray(Zne, dtype=np.complex128)
        wne = np.ascontiguousarray(Wne, dtype=np.complex128)
        zp, wp = _ptr(zne), _ptr(wne)
    emid = complex(emid)
    fn = lib().gbf_zgegv if cplx else lib().gbf_dgegv
    fn(n, _ptr(A), n, _ptr(Bf), n, _ip(fpm), C.byref(eps), C.byref(loop), emid.real, emid.imag, float(r),
       C.byref(M0), _ptr(E), _ptr(X), C.byref(M), _ptr(res), C.byref(info), zp, wp)
    return dict(E=E, X=X, res=res, M=M.value, loop=loop.value, epsout=eps.value, info=info.value)


def gbf_factor_dev(handle, A, B, zne, prec=0, uplo="F", stream=None):
    import torch

    n = A.shape[0]
    lda = _check_colmajor(A, n)
    ldb = _check_colmajor(B, n) if B is not None else n
    zne = np.ascontiguousarray(zne, dtype=np.complex128)
    if stream is None:
        stream = torch.cuda.current_stream(A.device)
    return lib().gbf_factor_dev(handle.h if handle else None, C.c_void_p(stream.cuda_stream),
                                1 if A.is_complex() else 0, int(prec), C.c_char(uplo.encode()), n, _ptr(A), lda,
                                _ptr(B), ldb, len(zne), _ptr(zne))


def gbf_solve_dev(handle, rhs, ne, trans=0, stream=None):
    """rhs: complex128 CUDA tensor n x nrhs (column-major); returns the
    ne x n x nrhs node solutions as a (ne, nrhs, n) tensor (so [e].t() is
    the n x nrhs block) and the return code."""
    import torch

    n, nrhs = rhs.shape
    _check_colmajor(rhs, n)
    Y = torch.zeros((ne, nrhs, n), dtype=torch.complex128, device=rhs.device)
    if stream is None:
        stream = torch.cuda.current_stream(rhs.device)
    rc = lib().gbf_solve_dev(handle.h if handle else None, C.c_void_p(stream.cuda_stream), int(trans), nrhs,
                             _ptr(rhs), _ptr(Y))
    return Y, rc


def gbf_heev_dev(handle, A, stream=None):
    """A: m x m CUDA tensor (float64 or complex128, column-major), overwritten.
    Returns (w, V, rc)."""
    import torch

    m = A.shape[0]
    _check_colmajor(A, m)
    w = torch.zeros(m, dtype=torch.float64, device=A.device)
    V = torch.zeros((m, m), dtype=A.dtype, device=A.device).t()
    if stream is None:
        stream = torch.cuda.current_stream(A.device)
    rc = lib().gbf_heev_dev(handle.h if handle else None, C.c_void_p(stream.cuda_stream),
                            1 if A.is_complex() else 0, m, _ptr(A), _ptr(w), _ptr(V))
    return w, V, rc


# ------------------------------------------------- independent problems --
class DeviceProblem:
    """A problem whose inputs and outputs live in CUDA tensors (kept alive
    here while the library uses them)."""

    def __init__(self, A, B, emin, emax, m0, fpm=None, uplo="F"):
        import torch

        if fpm is None:
            fpm = gbf_init()
        n = A.shape[0]
        self.A, self.B = A, B
        lda = _check_colmajor(A, n)
        ldb = _check_colmajor(B, n) if B is not None else n
        self.E = torch.zeros(m0, dtype=torch.float64, device=A.device)
        self.res = torch.zeros(m0, dtype=torch.float64, device=A.device)
        self.X = torch.zeros((m0, n), dtype=A.dtype, device=A.device).t()
        p = Problem()
        p.kind = 1 if A.is_complex() else 0
        p.uplo = uplo.encode()
        p.n = n
        p.dA = A.data_ptr()
        p.lda = lda
        p.dB = B.data_ptr() if B is not None else None
        p.ldb = ldb
        p.emin, p.emax = float(emin), float(emax)
        p.m0 = int(m0)
        for i in range(64):
            p.fpm[i] = int(fpm[i])
        p.dE, p.dX, p.dres = self.E.data_ptr(), self.X.data_ptr(), self.res.data_ptr()
        p.Zne = p.Wne = None
        self.p = p

    def bytes(self):
        return lib().gbf_problem_bytes(C.byref(self.p))


def batch_solve(problems, nworkers=4, stream=None):
    """gbf_batch_solve over DeviceProblem objects; returns (rc, [Result])."""
    import torch

    arr = (Problem * len(problems))(*[q.p for q in problems])
    outs = (Result * len(problems))()
    if stream is None:
        stream = torch.cuda.current_stream()
    rc = lib().gbf_batch_solve(None, C.c_void_p(stream.cuda_stream), len(problems), arr, outs, int(nworkers))
    return rc, [outs[i] for i in range(len(problems))]


class Server:
    """gbf_server_*: admission by HBM budget, concurrent workers."""

    def __init__(self, hbm_budget_bytes, nworkers=4):
        h = C.c_void_p()
        rc = lib().gbf_server_create(C.c_size_t(int(hbm_budget_bytes)), int(nworkers), C.byref(h))
        if rc:
            raise RuntimeError(f"gbf_server_create failed ({rc}): {last_error()}")
        self.h = h
        self._keep = {}

    def submit(self, prob):
        t = C.c_ulonglong()
        rc = lib().gbf_server_submit(self.h, C.byref(prob.p), C.byref(t))
        if rc:
            raise RuntimeError(f"gbf_server_submit failed ({rc})")
        self._keep[t.value] = prob
        return t.value

    def poll(self, ticket):
        r = Result()
        rc = lib().gbf_server_poll(self.h, C.c_ulonglong(ticket), C.byref(r))
        if rc == 0:
            self._keep.pop(ticket, None)
            return r
        return None

    def wait(self, ticket):
        r = Result()
        rc = lib().gbf_server_wait(self.h, C.c_ulonglong(ticket), C.byref(r))
        if rc:
            raise RuntimeError(f"gbf_server_wait failed ({rc})")
        self._keep.pop(ticket, None)
        return r

    def stats(self):
        a, b = C.c_size_t(), C.c_size_t()
        q, r = C.c_int(), C.c_int()
        lib().gbf_server_stats(self.h, C.byref(a), C.byref(b), C.byref(q), C.byref(r))
        return dict(in_use=a.value, peak=b.value, queued=q.value, running=r.value)

    def close(self):
        if self.h:
            lib().gbf_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tc_gemm_bf16(A, B, stream=None):
    """gbf_tc_gemm_bf16: A (batch, M, K), B (batch, N, K) bf16 CUDA tensors
    (contiguous) -> C (batch, N, M) float32, i.e. C[b].t() = A[b] @ B[b]^T."""
    import torch

    bt, M, K = A.shape
    N = B.shape[1]
    C = torch.empty((bt, N, M), dtype=torch.float32, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    if stream is None:
        stream = torch.cuda.current_stream(A.device)
    rc = lib().gbf_tc_gemm_bf16(_stream_ptr(stream), M, N, K, bt,
                                _ptr(A), _ptr(B), _ptr(C), M, M * N, _ptr(err))
    return C, rc


def _stream_ptr(stream):
    return C.c_void_p(stream.cuda_stream)


def zgemm_sliced(opa, opb, A, B, C_, alpha=1.0, beta=0, S=7, stream=None):
    """gbf_zgemm_sliced on column-major complex CUDA tensors of shape
    (batch, rows, cols) stored as (batch, cols, rows) contiguous: A, B, C_ are
    lists of per-batch column-major 2-D tensors packed in 3-D tensors whose
    [b].t() is the matrix.  C_ is updated in place; returns the code."""
    import torch

    bt = A.shape[0]
    am, ak = A.shape[2], A.shape[1]       # stored matrix (rows, cols) = (shape[2], shape[1])
    bk, bn = B.shape[2], B.shape[1]
    m = am if opa == "N" else ak
    k = ak if opa == "N" else am
    n = bn if opb == "N" else bk
    prec = 0 if A.dtype == torch.complex128 else 1
    work = torch.empty(lib().gbf_zgemm_sliced_work(m, n, bt, S), dtype=torch.uint8, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    if stream is None:
        stream = torch.cuda.current_stream(A.device)
    return lib().gbf_zgemm_sliced(_stream_ptr(stream), prec, S, opa.encode(), opb.encode(), m, n, k, float(alpha),
                                  _ptr(A), am, am * ak, _ptr(B), bk, bk * bn, int(beta), _ptr(C_), C_.shape[2],
                                  C_.shape[1] * C_.shape[2], bt, _ptr(work), work.numel(), _ptr(err))


def gemm_sliced(opa, opb, A, B, C_, alpha=1.0, beta=0, stream=None):
    """gbf_gemm_sliced (any k, FP64 real or complex) on column-major CUDA
    tensors packed as for zgemm_sliced: (batch, cols, rows) contiguous, whose
    [b].t() is the matrix.  C_ is updated in place; returns the code."""
    import torch

    bt = A.shape[0]
    am, ak = A.shape[2], A.shape[1]
    bk, bn = B.shape[2], B.shape[1]
    m = am if opa == "N" else ak
    k = ak if opa == "N" else am
    n = bn if opb == "N" else bk
    cplx = 1 if A.dtype == torch.complex128 else 0
    work = torch.empty(lib().gbf_gemm_sliced_work(cplx, m, n, k, bt), dtype=torch.uint8, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    if stream is None:
        stream = torch.cuda.current_stream(A.device)
    return lib().gbf_gemm_sliced(_stream_ptr(stream), cplx, opa.encode(), opb.encode(), m, n, k, float(alpha),
                                 _ptr(A), am, am * ak, _ptr(B), bk, bk * bn, int(beta), _ptr(C_), C_.shape[2],
                                 C_.shape[1] * C_.shape[2], bt, _ptr(work), work.numel(), _ptr(err))


def zgemm_sliced_noalloc(opa, opb, A, B, C_, alpha=1.0, beta=0, S=7, stream=None):
    """gbf_zgemm_sliced_noalloc (no device allocation; fixed library scratch);
    same tensor layout as zgemm_sliced.  Returns the code."""
    import torch

    bt = A.shape[0]
    am, ak = A.shape[2], A.shape[1]
    bk, bn = B.shape[2], B.shape[1]
    m = am if opa == "N" else ak
    k = ak if opa == "N" else am
    n = bn if opb == "N" else bk
    prec = 0 if A.dtype == torch.complex128 else 1
    if stream is None:
        stream = torch.cuda.current_stream(A.device)
    return lib().gbf_zgemm_sliced_noalloc(_stream_ptr(stream), prec, S, opa.encode(), opb.encode(), m, n, k,
                                          float(alpha), _ptr(A), am, am * ak, _ptr(B), bk, bk * bn, int(beta),
                                          _ptr(C_), C_.shape[2], C_.shape[1] * C_.shape[2], bt)


def cgemm_tf32(opa, opb, A, B, C_, alpha=1.0, beta=0, stream=None):
    """gbf_cgemm_tf32 (any k, complex FP32, 3xTF32) on column-major complex64
    CUDA tensors packed as for zgemm_sliced.  C_ is updated in place; returns
    the code."""
    import torch

    bt = A.shape[0]
    am, ak = A.shape[2], A.shape[1]
    bk, bn = B.shape[2], B.shape[1]
    m = am if opa == "N" else ak
    k = ak if opa == "N" else am
    n = bn if opb == "N" else bk
    work = torch.empty(lib().gbf_cgemm_tf32_work(m, n, k, bt), dtype=torch.uint8, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    if stream is None:
        stream = torch.cuda.current_stream(A.device)
    return lib().gbf_cgemm_tf32(_stream_ptr(stream), opa.encode(), opb.encode(), m, n, k, float(alpha), _ptr(A), am,
                                am * ak, _ptr(B), bk, bk * bn, int(beta), _ptr(C_), C_.shape[2],
                                C_.shape[1] * C_.shape[2], bt, _ptr(work), work.numel(), _ptr(err))
