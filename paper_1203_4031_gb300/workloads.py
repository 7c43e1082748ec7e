"""Seeded synthetic workloads for the Hermitian FEAST hot path.

This module only builds INPUTS (matrices, intervals, subspace sizes and fpm
overrides); it holds none of the eigensolver's arithmetic.  Both the CUDA
path's tests/benchmark and the CPU oracle draw their inputs from here.

Randomness is counter-based SplitMix64 (Steele, Lea & Flood 2014):
value(i) = mix(seed + (i+1) * 0x9E3779B97F4A7C15), so every entry is a pure
function of (seed, index) and identical on x86 and Arm hosts.  Normals use
the Box-Muller transform.

Workloads (the guide's example matrices are not available, these synthetic
problems stand in for them):
  * ``laplacian``: dense 1-D Laplacian tridiag(-1, 2, -1), B = I; closed-form
    spectrum 2 - 2 cos(k pi / (n+1)).
  * ``dense_real_generalized``: A = Q diag(lam) Q^T, Q a product of 8 seeded
    Householder reflectors, lam ~ U[-1, 1]; B = Q_B diag(mu) Q_B^T with its
    own reflectors, mu log-uniform in [1, 100]; interval [-delta, delta]
    holding a fixed count of pencil eigenvalues.
  * ``dense_complex_hermitian``: A = U diag(lam) U^H, U a product of 8 seeded
    complex reflectors, lam ~ U[-1, 1], B = I; the spectrum is lam itself.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """Counter-based SplitMix64 over an index array (uint64 wrap-around)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(idx, dtype=np.uint64) + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def derive_seed(seed: int, tag: int) -> int:
    return int(splitmix64(seed, np.array([tag], dtype=np.uint64))[0])


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform [0, 1) doubles from the top 53 bits."""
    idx = np.arange(offset, offset + count, dtype=np.uint64)
    return (splitmix64(seed, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, count: int, lo: float = -1.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, count, offset)


def normal(seed: int, count: int) -> np.ndarray:
    """Box-Muller normals: pairs of uniforms (u1 in (0,1], u2 in [0,1))."""
    u = uniform01(seed, 2 * count)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def reflector_vectors(seed: int, n: int, count: int = 8, complex_: bool = False) -> list:
    out = []
    for r in range(count):
        s = derive_seed(seed, 1000 + r)
        v = normal(s, n)
        if complex_:
            v = v + 1j * normal(derive_seed(s, 7), n)
        out.append(v)
    return out


def conjugate_by_reflectors(d: np.ndarray, vs: list) -> np.ndarray:
    """M = H_1 ... H_k diag(d) H_k ... H_1 with H = I - 2 v v^H / (v^H v).

    Applied as a sequence of two-sided rank-1 updates, innermost reflector
    first, and symmetrised at the end so M is exactly Hermitian."""
    cplx = any(np.iscomplexobj(v) for v in vs)
    M = np.diag(d).astype(np.complex128 if cplx else np.float64)
    for v in reversed(vs):
        beta = 2.0 / np.real(np.vdot(v, v))
        w = v.conj() @ M                      # v^H M
        M -= beta * np.outer(v, w)            # H M
        u = M @ v                             # (H M) v
        M -= beta * np.outer(u, v.conj())     # (H M) H
    M = 0.5 * (M + M.conj().T)
    return np.asfortranarray(M)


@dataclass
class Problem:
    name: str
    hermitian: bool                 # True: complex Hermitian, False: real symmetric
    A: np.ndarray
    B: np.ndarray | None
    emin: float
    emax: float
    m0: int
    fpm: dict = field(default_factory=dict)   # {fortran index i: value} over feastinit
    spectrum: np.ndarray | None = None         # exact eigenvalues when known
    note: str = ""

    @property
    def n(self) -> int:
        return self.A.shape[0]

    def apply_fpm(self, fpm):
        for i, v in self.fpm.items():
            fpm[i - 1] = v
        return fpm


def laplacian(n: int = 500, emin: float = 0.5, emax: float = 1.0, m0: int = 80) -> Problem:
    A = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    k = np.arange(1, n + 1)
    lam = 2.0 - 2.0 * np.cos(k * np.pi / (n + 1))
    return Problem(f"laplacian-n{n}", False, np.asfortranarray(A), None, emin, emax, m0,
                   fpm={2: 8, 3: 12, 4: 20, 6: 0}, spectrum=lam,
                   note="dense 1-D Laplacian, B=I, trace criterion 1e-12, <=20 loops")


def dense_complex_hermitian(n: int = 8192, emin: float = 0.0, emax: float = 0.04, m0: int = 240,
                            ne: int = 16, seed: int = 20260103) -> Problem:
    lam = uniform(derive_seed(seed, 1), n)
    A = conjugate_by_reflectors(lam, reflector_vectors(seed, n, 8, complex_=True))
    return Problem(f"complex-hermitian-n{n}", True, A, None, emin, emax, m0,
                   fpm={2: ne, 3: 10, 6: 1}, spectrum=np.sort(lam),
                   note="U diag(lam) U^H, 8 complex reflectors, lam~U[-1,1], B=I")


# Half-widths delta of [-delta, delta] holding exactly `count` pencil eigenvalues
# of dense_real_generalized(n, seed); each value sits halfway between the
# count-th and (count+1)-th smallest |lambda| of the pencil, from
# scipy.linalg.eigh(A, B) on the generated matrices (see interval_for_count).
_DELTA = {
    (4096, 20260102, 200): 0.0023589538297558448,
}


def dense_real_generalized(n: int = 4096, count: int = 200, m0: int = 300, ne: int = 8,
                           seed: int = 20260102, delta: float | None = None) -> Problem:
    lam = uniform(derive_seed(seed, 1), n)
    mu = 10.0 ** uniform(derive_seed(seed, 2), n, 0.0, 2.0)
    A = conjugate_by_reflectors(lam, reflector_vectors(seed, n, 8))
    B = conjugate_by_reflectors(mu, reflector_vectors(derive_seed(seed, 3), n, 8))
    if delta is None:
        delta = _DELTA.get((n, seed, count))
    if delta is None:
        delta = interval_for_count(A, B, count)
        _DELTA[(n, seed, count)] = delta
    return Problem(f"real-generalized-n{n}", False, A, B, -delta, delta, m0,
                   fpm={2: ne, 3: 10, 6: 1},
                   note=f"QAQ^T / Q_B M Q_B^T, interval [-d,d] holding {count} eigenvalues")


def interval_for_count(A: np.ndarray, B: np.ndarray | None, count: int) -> float:
    """delta such that [-delta, delta] holds exactly `count` pencil eigenvalues
    (midpoint of the gap between the count-th and next smallest |lambda|)."""
    import scipy.linalg as sl

    w = sl.eigh(A, B, eigvals_only=True)
    a = np.sort(np.abs(w))
    return float(0.5 * (a[count - 1] + a[count]))


# --------------------------------------------------- batched / serving --
def _interval_around(w: np.ndarray, count: int, seed: int) -> tuple:
    """[a, b] holding exactly `count` of the sorted values w, at a seeded
    position, with ends halfway between neighbouring values."""
    w = np.sort(w)
    n = len(w)
    lo = 1
    hi = n - count - 1
    s = lo + int(uniform01(seed, 1)[0] * max(1, hi - lo))
    a = 0.5 * (w[s - 1] + w[s])
    b = 0.5 * (w[s + count - 1] + w[s + count])
    return float(a), float(b)


def batched_generalized(count: int = 256, nmin: int = 64, nmax: int = 1024, seed: int = 20260104,
                        kmin: int = 10, kmax: int = 40, ne: int = 8) -> list:
    """Independent real symmetric generalized problems built as
    dense_real_generalized (own reflectors for A and B), n log-uniform in
    [nmin, nmax], each interval holding a count drawn uniformly from
    [kmin, kmax] (located with scipy's generalized eigenvalues), M0 =
    ceil(1.5 count)."""
    import scipy.linalg as sl

    u = uniform01(derive_seed(seed, 1), count)
    ks = uniform01(derive_seed(seed, 2), count)
    out = []
    for i in range(count):
        n = int(round(np.exp(np.log(nmin) + u[i] * (np.log(nmax) - np.log(nmin)))))
        k = kmin + int(ks[i] * (kmax - kmin + 1))
        si = derive_seed(seed, 100 + i)
        lam = uniform(derive_seed(si, 1), n)
        mu = 10.0 ** uniform(derive_seed(si, 2), n, 0.0, 2.0)
        A = conjugate_by_reflectors(lam, reflector_vectors(si, n, 8))
        B = conjugate_by_reflectors(mu, reflector_vectors(derive_seed(si, 3), n, 8))
        w = sl.eigh(A, B, eigvals_only=True)
        a, b = _interval_around(w, k, derive_seed(si, 4))
        out.append(Problem(f"batch-{i}-n{n}", False, A, B, a, b, int(np.ceil(1.5 * k)),
                           fpm={2: ne, 3: 10, 6: 1}, spectrum=np.sort(w),
                           note="config-2 style generalized, interval holding k"))
    return out


def serving_requests(count: int = 2000, nmin: int = 128, nmax: int = 4096, seed: int = 20260105,
                     kmin: int = 8, kmax: int = 64, rate: float = 1.0):
    """Request descriptors of the serving workload: kind (real symmetric
    generalized / complex Hermitian standard, 50/50), n log-uniform in
    [nmin, nmax], a count uniform in [kmin, kmax], M0 = ceil(1.5 count),
    Poisson arrival times at `rate` requests per second.  Matrices are built
    by `serving_matrices` when a request arrives."""
    u = uniform01(derive_seed(seed, 1), count)
    ks = uniform01(derive_seed(seed, 2), count)
    kind = uniform01(derive_seed(seed, 3), count) < 0.5
    gaps = -np.log(1.0 - uniform01(derive_seed(seed, 4), count)) / rate
    t = np.cumsum(gaps)
    reqs = []
    for i in range(count):
        n = int(round(np.exp(np.log(nmin) + u[i] * (np.log(nmax) - np.log(nmin)))))
        k = kmin + int(ks[i] * (kmax - kmin + 1))
        reqs.append(dict(i=i, n=n, count=k, m0=int(np.ceil(1.5 * k)), hermitian=bool(kind[i]),
                         t_arrival=float(t[i]), seed=derive_seed(seed, 1000 + i)))
    return reqs


def serving_matrices(req: dict, device="cuda"):
    """Matrices of one serving request on the GPU (torch), with a known
    spectrum lam ~ U[-1, 1]:
      complex Hermitian standard: A = U diag(lam) U^H, 8 complex reflectors;
      real generalized: B = Q_B diag(mu) Q_B^T, mu log-uniform [1, 100], and
      A = S (Q diag(lam) Q^T) S^T with S = Q_B diag(sqrt(mu)), so that the
      pencil (A, B) has exactly the eigenvalues lam (eigenvectors S^{-T} Q).
    Returns (A, B or None, emin, emax) with the interval holding `count`
    eigenvalues."""
    import torch

    n, s = req["n"], req["seed"]
    lam = uniform(derive_seed(s, 1), n)
    a, b = _interval_around(lam, req["count"], derive_seed(s, 4))

    def reflect(M, vs):
        for v in reversed(vs):
            vt = torch.as_tensor(v, device=device, dtype=M.dtype)
            beta = 2.0 / float(np.real(np.vdot(v, v)))
            M = M - beta * torch.outer(vt, vt.conj() @ M)
            M = M - beta * torch.outer(M @ vt, vt.conj())
        return M

    if req["hermitian"]:
        M = torch.diag(torch.as_tensor(lam, device=device, dtype=torch.complex128))
        A = reflect(M, reflector_vectors(s, n, 8, complex_=True))
        A = 0.5 * (A + A.conj().T)
        return A.t().contiguous().t(), None, a, b
    mu = 10.0 ** uniform(derive_seed(s, 2), n, 0.0, 2.0)
    qb = reflector_vectors(derive_seed(s, 3), n, 8)
    B = reflect(torch.diag(torch.as_tensor(mu, device=device, dtype=torch.float64)), qb)
    C = reflect(torch.diag(torch.as_tensor(lam, device=device, dtype=torch.float64)), reflector_vectors(s, n, 8))
    sq = torch.as_tensor(np.sqrt(mu), device=device, dtype=torch.float64)
    C = sq[:, None] * C * sq[None, :]          # D C D
    A = reflect(C, qb)                          # Q_B (D C D) Q_B^T
    A = 0.5 * (A + A.T)
    B = 0.5 * (B + B.T)
    return A.t().contiguous().t(), B.t().contiguous().t(), a, b


# ------------------------------------------------------- non-Hermitian --
def _reflect_left(M: np.ndarray, v: np.ndarray) -> np.ndarray:
    """(I - 2 v v^H / v^H v) M."""
    beta = 2.0 / np.real(np.vdot(v, v))
    return M - beta * np.outer(v, v.conj() @ M)


def _reflect_right(M: np.ndarray, v: np.ndarray) -> np.ndarray:
    """M (I - 2 v v^H / v^H v)."""
    beta = 2.0 / np.real(np.vdot(v, v))
    return M - beta * np.outer(M @ v, v.conj())


@dataclass
class GeneralProblem:
    """A non-Hermitian pencil (A, B) with a known spectrum and a circular
    contour (centre emid, radius r) holding exactly `count` eigenvalues."""
    name: str
    complex_: bool                  # False: A, B real non-symmetric
    A: np.ndarray
    B: np.ndarray | None
    emid: complex
    r: float
    m0: int
    spectrum: np.ndarray
    count: int
    fpm: dict = field(default_factory=dict)
    note: str = ""

    @property
    def n(self) -> int:
        return self.A.shape[0]

    def apply_fpm(self, fpm):
        for i, v in self.fpm.items():
            fpm[i - 1] = v
        return fpm


def general_spectrum(n: int, seed: int, complex_: bool) -> np.ndarray:
    """Eigenvalues of dense_nonsymmetric: complex: uniform in the box
    [-1, 1] x [-1/2, 1/2]; real: half of them real, uniform in [-1, 1], the
    rest conjugate pairs a +- ib, a ~ U[-1, 1], b ~ U(0, 1/2]."""
    if complex_:
        return uniform(derive_seed(seed, 11), n) + 0.5j * uniform(derive_seed(seed, 12), n)
    npair = n // 4
    nreal = n - 2 * npair
    re = uniform(derive_seed(seed, 11), nreal)
    a = uniform(derive_seed(seed, 12), npair)
    b = 0.5 * (1.0 - uniform01(derive_seed(seed, 13), npair))
    lam = np.concatenate([re.astype(np.complex128), a + 1j * b, a - 1j * b])
    return lam


def dense_nonsymmetric(n: int = 4096, count: int = 40, m0: int = 64, ne: int = 16, complex_: bool = False,
                       generalized: bool = False, emid: complex | None = None, seed: int = 20260106,
                       nref: int = 4) -> GeneralProblem:
    """Non-normal dense pencil with a known spectrum and well-conditioned
    eigenvectors.  M = S D S^{-1} with S = H_1 diag(s) H_2 (H_i products of
    `nref` seeded reflectors, s ~ U[1, 2], so cond(S) <= 2) and D the
    spectrum (real problems: 1x1 blocks and 2x2 blocks [[a, b], [-b, a]]).
    Standard: A = M.  Generalized: B = G_1 diag(mu) G_2 (mu log-uniform in
    [1, 10], its own reflectors, non-symmetric) and A = B M, so that the
    pencil's eigenvalues are D's.  The circle is centred at emid (real for
    real problems, so that the node set is conjugate-symmetric) with the
    radius halfway between the count-th and next distance to emid."""
    lam = general_spectrum(n, seed, complex_)
    dt = np.complex128 if complex_ else np.float64
    D = np.zeros((n, n), dtype=dt)
    if complex_:
        D[np.arange(n), np.arange(n)] = lam
    else:
        npair = n // 4
        nreal = n - 2 * npair
        D[np.arange(nreal), np.arange(nreal)] = lam[:nreal].real
        for k in range(npair):
            i = nreal + 2 * k
            a, b = lam[nreal + k].real, lam[nreal + k].imag
            D[i, i] = D[i + 1, i + 1] = a
            D[i, i + 1] = b
            D[i + 1, i] = -b
    s = 1.0 + uniform01(derive_seed(seed, 21), n)
    h1 = reflector_vectors(derive_seed(seed, 22), n, nref, complex_=complex_)
    h2 = reflector_vectors(derive_seed(seed, 23), n, nref, complex_=complex_)
    # M = H1 diag(s) H2 D H2^H diag(1/s) H1^H (H_i Hermitian unitary products)
    M = D
    for v in h2:
        M = _reflect_right(_reflect_left(M, v), v)
    M = (s[:, None] * M) / s[None, :]
    for v in h1:
        M = _reflect_right(_reflect_left(M, v), v)
    B = None
    if generalized:
        mu = 10.0 ** uniform(derive_seed(seed, 31), n, 0.0, 1.0)
        g1 = reflector_vectors(derive_seed(seed, 32), n, nref, complex_=complex_)
        g2 = reflector_vectors(derive_seed(seed, 33), n, nref, complex_=complex_)
        # B = G1 diag(mu) G2, A = B M = G1 diag(mu) (G2 M)
        Am = M.copy()
        G2 = np.eye(n, dtype=dt)
        for v in reversed(g2):
            G2 = _reflect_left(G2, v)
            Am = _reflect_left(Am, v)
        Bm = mu[:, None] * G2
        Am = mu[:, None] * Am
        for v in reversed(g1):
            Bm = _reflect_left(Bm, v)
            Am = _reflect_left(Am, v)
        A, B = Am, Bm
    else:
        A = M
    if emid is None:
        emid = 0.1 + (0.05j if complex_ else 0.0)
    dist = np.sort(np.abs(lam - emid))
    r = float(0.5 * (dist[count - 1] + dist[count]))
    kind = "complex" if complex_ else "real"
    return GeneralProblem(f"{kind}-nonsymmetric{'-generalized' if generalized else ''}-n{n}", bool(complex_),
                          np.asfortranarray(A), None if B is None else np.asfortranarray(B), complex(emid), r, m0,
                          lam, count, fpm={8: ne, 3: 10, 6: 1},
                          note="S D S^-1, cond(S) <= 2; generalized: A = B M, B = G1 diag(mu) G2")
