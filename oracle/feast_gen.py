"""Plain FP64 CPU oracle of non-Hermitian FEAST -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
leg may import this module.  The CUDA product path never calls it and
shares no code with it.

What it computes (FEAST v3.0 user guide, Polizzi & Kestyn, arXiv:1203.4031):
  - the non-Hermitian variant of section "From v2.1 to v3.0": dual subspaces,
    Q for the right and Q^ for the left eigenvectors, and a full contour that
    encloses the wanted complex eigenvalues;
  - the contour of the gcontour tool (section "List of all FEAST tool
    routines"): fpm(8) nodes on a circle or ellipse of centre Emid and
    horizontal semi-axis r, vertical/horizontal ratio fpm(18)/100, rotated by
    fpm(19) degrees, Gauss (fpm(17)=0) or trapezoidal (fpm(17)=1) in the angle;
  - the RCI cases of Table "tab_ijob" for the general types: solves with
    z_e B - A (case 11) and its adjoint (case 21), products with A, A^H, B, B^H
    (cases 30, 31, 40, 41);
  - the outputs of Table "tab_common" for the general types: complex E, X
    holding the right vectors in columns 1..M0 and the left ones in M0+1..,
    res(1:M0) right and res(M0+1:2M0) left residuals
    ||A x - lambda B x||_1 / ||alpha B x||_1 and
    ||A^H x^ - conj(lambda) B^H x^||_1 / ||alpha B^H x^||_1, alpha = |Emid|+r;
  - the info codes of Table "tab_info" (6: converged, subspace not
    bi-orthonormal).

The guide prints no formula for the full-contour quadrature; it follows from
the residue theorem.  On z(t) = Emid + r e^{i phi} (cos t + i rho sin t),
t in [0, 2 pi), the filter (1 / 2 pi i) int dz / (z - lambda) is 1 inside and
0 outside, and z'(t) / i = r e^{i phi} (rho cos t + i sin t), so a rule in t
with points t_e and weights (2 pi) omega_e / 2 (omega summing to 2) gives
w_e = (omega_e / 2) r e^{i phi} (rho cos t_e + i sin t_e) and
f(lambda) = sum_e w_e / (z_e - lambda).

One iteration (the dual-subspace Rayleigh-Ritz the guide names):
  Q  = sum_e w_e        (z_e B - A)^{-1}   B   Y
  Q^ = sum_e conj(w_e)  (z_e B - A)^{-H}   B^H Y^
  Aq = Q^^H A Q,  Bq = Q^^H B Q,  Aq W = Bq W Lambda,  V^H Aq = Lambda V^H Bq,
  V^H Bq W = I;  X = Q W,  X^ = Q^ V;  next Y = X, Y^ = X^.

Readings where the guide is silent (each listed in the design notes):
  - initial Y = Y^ = the complex SplitMix64 subspace of the Hermitian
    oracle (u(2i) + i u(2i+1), u uniform in [-1, 1)); fpm(5)=1 takes
    right/left guesses from X(:, 1:M0) and X(:, M0+1:2 M0);
  - the reduced pencil is solved by a library routine (scipy's QZ, the
    reduced problem's "dense eigenvalue problem" step); the right vectors
    are unit 2-norm, the left ones scaled so that V^H Bq W = I; the Ritz
    vectors X are rescaled to unit 2-norm with X^ scaled inversely, and the
    next left subspace Y^ is X^ with unit columns;
  - inside: |(lambda - Emid) e^{-i phi} / r| in the ellipse metric <= 1;
    output order: inside pairs by ascending (Re, Im), then the others;
  - convergence: fpm(6)=1 on the largest right or left residual of the
    pairs inside, fpm(6)=0 on |trace - trace_prev| / alpha with the complex
    trace of the pairs inside; epsout = 1 at loop 0;
  - info 6 when, at convergence, max |X^_M^H B X_M - I| exceeds 1e-8;
  - info 3 when every one of the kept mk Ritz values is inside and mk < N;
  - no spurious-pair test (the guide gives no criterion for this variant);
  - Q and Q^ are replaced by orthonormal bases of their numerical ranges
    (Gram eigenvalues above 1e-14 of the largest), both cut to the smaller
    rank mk: the returned "new suitable M0" of Table tab_common.  Without
    it, the columns of eigenvalues far outside (filter values below the
    solves' rounding level) shrink by orders of magnitude against the
    others and the reduced pencil becomes numerically singular when M0
    exceeds the count by a wide margin; the threshold sits at the Gram's
    resolution, so the nearly parallel eigenvectors of a nearly defective
    pair are kept down to angles of about 1e-7.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

SUBSPACE_SEED = 0x3C6EF372FE94F82B
BIORTH_TOL = 1e-8

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _splitmix64(seed, idx):
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), counter-based form."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(idx, dtype=np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def initial_subspace(n, m0, seed=SUBSPACE_SEED):
    """n x m0 complex, column-major entry i = u(2i) + i u(2i+1)."""
    i = np.arange(n * m0, dtype=np.uint64)
    u = lambda k: (_splitmix64(seed, k) >> np.uint64(11)).astype(np.float64) * (2.0 / 9007199254740992.0) - 1.0
    v = u(2 * i) + 1j * u(2 * i + 1)
    return np.asfortranarray(v.reshape(m0, n).T)


def gauss_legendre(ne):
    """Gauss-Legendre points (ascending) and weights on [-1, 1]: numpy's
    routine (a library step; the C oracle's own rule is pinned against it)."""
    return np.polynomial.legendre.leggauss(ne)


def gcontour(emid, r, ne, qtype=1, ratio=100, angle=0):
    """Full-contour nodes and weights (gcontour tool).  Points in the angle
    t in [0, 2 pi): Gauss t_e = pi (1 + x_e), x ascending; trapezoidal
    t_e = 2 pi (e + 1/2) / ne.  Nodes e and ne-1-e are mirror images
    (t -> 2 pi - t), so for real Emid and angle 0 the set is closed under
    conjugation."""
    if ne < 1 or not r > 0 or ratio <= 0:
        raise ValueError("bad contour")
    if qtype == 0:
        x, om = gauss_legendre(ne)
        t = np.pi * (1.0 + x)
    elif qtype == 1:
        t = 2.0 * np.pi * (np.arange(ne) + 0.5) / ne
        om = np.full(ne, 2.0 / ne)
    else:
        raise ValueError("fpm(17) must be 0 or 1")
    rho = ratio / 100.0
    rot = np.exp(1j * np.deg2rad(angle))
    c, s = np.cos(t), np.sin(t)
    z = emid + r * rot * (c + 1j * rho * s)
    w = 0.5 * om * r * rot * (rho * c + 1j * s)
    return z, w


def grationalx(z, w, lam):
    """f(lambda) = sum_e w_e / (z_e - lambda) (complex)."""
    lam = np.asarray(lam, dtype=np.complex128)
    return np.array([np.sum(w / (z - l)) for l in lam.ravel()]).reshape(lam.shape)


def inside(lam, emid, r, ratio=100, angle=0):
    u = (np.asarray(lam) - emid) * np.exp(-1j * np.deg2rad(angle)) / r
    return u.real ** 2 + (u.imag / (ratio / 100.0)) ** 2 <= 1.0


def feastinit_gen():
    """Table tab_fpm defaults used here (fpm[i-1] = fpm(i))."""
    fpm = np.zeros(64, dtype=np.int32)
    fpm[2] = 12    # fpm(3): eps = 1e-12
    fpm[3] = 20    # fpm(4): max loops
    fpm[5] = 1     # fpm(6): residual criterion
    fpm[7] = 16    # fpm(8): full-contour nodes
    fpm[16] = 1    # fpm(17): trapezoidal
    fpm[17] = 100  # fpm(18): circle
    return fpm


def _res(Mx, Nx, lam, alpha):
    """||Mx_j - lam_j Nx_j||_1 / ||alpha Nx_j||_1 per column."""
    num = np.sum(np.abs(Mx - Nx * lam[None, :]), axis=0)
    den = np.sum(np.abs(alpha * Nx), axis=0)
    return num / den


def _range_basis(M):
    """Orthonormal basis of the numerical range of M's columns: the Gram
    matrix M^H M diagonalised (library eigh), directions with eigenvalue at
    most 1e-14 of the largest (the Gram matrix's own rounding level; singular
    values below 1e-7 of the largest) dropped, the rest scaled to unit length
    (M V diag(w)^-1/2).  Returns the basis (largest directions last) and its
    size."""
    w, V = np.linalg.eigh(M.conj().T @ M)
    keep = w > 1e-14 * w[-1]
    return (M @ V[:, keep]) / np.sqrt(w[keep])[None, :], int(keep.sum())


def feast_gen(A, B, emid, r, m0, fpm=None, X0=None, zne=None, wne=None):
    """Non-Hermitian FEAST on the dense pencil (A, B) (B None: identity).
    Returns dict(E (m0 complex), X (n x 2 m0), res (2 m0), M, loop, epsout,
    info, biorth) in the layout of Table tab_common."""
    if fpm is None:
        fpm = feastinit_gen()
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    Bm = np.eye(n, dtype=np.complex128) if B is None else np.asarray(B, dtype=np.complex128)
    ne = int(fpm[7])
    ratio, angle = int(fpm[17]), int(fpm[18])
    if zne is None:
        zne, wne = gcontour(emid, r, ne, int(fpm[16]), ratio, angle)
    eps = 10.0 ** (-int(fpm[2]))
    alpha = abs(emid) + r
    E = np.zeros(m0, dtype=np.complex128)
    X = np.zeros((n, 2 * m0), dtype=np.complex128, order="F")
    res = np.zeros(2 * m0)
    out = dict(E=E, X=X, res=res, M=0, loop=0, epsout=1.0, info=0, biorth=0.0, m0=m0)
    if fpm[4] == 1 and X0 is not None:
        Y = np.array(X0[:, :m0], dtype=np.complex128)
        Yh = np.array(X0[:, m0:2 * m0], dtype=np.complex128)
    else:
        Y = initial_subspace(n, m0)
        Yh = Y.copy()
    m = m0
    trace_prev = 0.0
    for k in range(10 ** 6):
        # spectral projections (RCI cases 40/41, 10/11 and 21)
        BY, BhYh = Bm @ Y, Bm.conj().T @ Yh
        Q = np.zeros((n, m), dtype=np.complex128)
        Qh = np.zeros((n, m), dtype=np.complex128)
        for e in range(ne):
            S = zne[e] * Bm - A
            Q += wne[e] * np.linalg.solve(S, BY)
            Qh += np.conj(wne[e]) * np.linalg.solve(S.conj().T, BhYh)
        if fpm[13] == 1:
            X[:, :m] = Q
            X[:, m0:m0 + m] = Qh
            out.update(loop=k, info=4)
            return out
        # numerical ranges: directions the filter reduced below the solves'
        # rounding level carry noise that makes the reduced pencil singular;
        # both subspaces keep their mk largest directions (the new M0)
        Qo, r1 = _range_basis(Q)
        Qho, r2 = _range_basis(Qh)
        m = min(r1, r2)
        Q, Qh = Qo[:, -m:], Qho[:, -m:]
        # Rayleigh-Ritz on the dual subspaces (cases 30/31, 40/41)
        AQ, BQ = A @ Q, Bm @ Q
        AhQh, BhQh = A.conj().T @ Qh, Bm.conj().T @ Qh
        Aq = Qh.conj().T @ AQ
        Bq = Qh.conj().T @ BQ
        lam, VL, VR = sla.eig(Aq, Bq, left=True, right=True)
        W = VR / np.linalg.norm(VR, axis=0)[None, :]
        d = np.einsum("ij,ij->j", VL.conj(), Bq @ W)
        V = VL / np.conj(d)[None, :]
        Xr, AXr, BXr = Q @ W, AQ @ W, BQ @ W
        Xl, AXl, BXl = Qh @ V, AhQh @ V, BhQh @ V
        # right vectors to unit 2-norm, left ones scaled inversely (X^^H B X
        # stays I); the next Y^ takes unit columns as well, so that the
        # columns' scales do not drift apart over the iterations
        nr = np.linalg.norm(Xr, axis=0)
        Xr, AXr, BXr = Xr / nr, AXr / nr, BXr / nr
        Xl, AXl, BXl = Xl * nr, AXl * nr, BXl * nr
        rr = _res(AXr, BXr, lam, alpha)
        rl = _res(AXl, BXl, lam.conj(), alpha)
        ins = inside(lam, emid, r, ratio, angle)
        idx_in = [j for j in np.lexsort((lam.imag, lam.real)) if ins[j]]
        idx_out = [j for j in np.lexsort((lam.imag, lam.real)) if not ins[j]]
        order = idx_in + idx_out
        nin = len(idx_in)
        trace = np.sum(lam[idx_in]) if nin else 0.0
        maxres = max([max(rr[j], rl[j]) for j in idx_in], default=0.0)
        eout = 1.0 if k == 0 else abs(trace - trace_prev) / alpha
        E[:] = 0
        res[:] = 0
        X[:, :] = 0
        E[:m] = lam[order]
        res[:m] = rr[order]
        res[m0:m0 + m] = rl[order]
        X[:, :m] = Xr[:, order]
        X[:, m0:m0 + m] = Xl[:, order]
        out.update(M=nin, loop=k, epsout=eout, m0=m)
        info = None
        if not (np.all(np.isfinite(lam)) and np.all(np.isfinite(rr)) and np.all(np.isfinite(rl))):
            info = -2
        elif nin == 0:
            info = 1
        elif nin >= m and m < n:
            info = 3
        elif (eout < eps) if fpm[5] == 0 else (maxres < eps):
            info = 0
            G = X[:, m0:m0 + nin].conj().T @ (Bm @ X[:, :nin])
            out["biorth"] = float(np.max(np.abs(G - np.eye(nin))))
            if out["biorth"] > BIORTH_TOL:
                info = 6
        elif k >= fpm[3]:
            info = 2
        if info is not None:
            out["info"] = info
            return out
        Y = Xr[:, order]
        Yh = Xl[:, order] / np.linalg.norm(Xl[:, order], axis=0)
        trace_prev = trace
    raise RuntimeError("unreachable")
